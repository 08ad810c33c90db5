"""Seeded index and query generator (see package docstring).

Recipe (each open choice is one documented reading):
  * token types: V types with Zipf(s) frequencies p_j ~ j^-s;
  * each type is a Gaussian blob: a random unit mean mu_j, a token is
    normalise(mu_j + sigma * N(0, I_128)) (sigma per component);
  * document lengths: lognormal with sigma_log = 0.5 and
    mu_log = ln(mean) - sigma_log^2 / 2, rounded, clipped to [len_min, len_max];
  * every document token draws its type i.i.d. from the Zipf law;
  * centroid allotment: kappa_j proportional to sqrt(n_j), at least one per
    type that occurs, at most n_j, reconciled to exactly C by largest
    remainder (the simplified allotment the workload recipe names; the full
    four-phase allotment of Sec. 2.1 is not needed to make scoring inputs);
  * per-type Lloyd k-means (Sec. 2.1, "independent k_j-means per token"),
    initialised from a seeded sample of k_j points of the type, empty
    clusters keep their previous centroid, then each token is assigned to the
    nearest centroid of its own type;
  * residual r = t - c_a(t) against the *stored* centroid, rho = ||r|| kept as
    fp16, r / rho PQ-encoded (Sec. 2.1, "Residuals Compression") with M
    subspaces of d/M contiguous dims, 256 codewords per subspace trained by
    10 Lloyd iterations on a seeded sample, nearest codeword by L2 with ties
    to the lower index;
  * queries: n_q tokens whose types are drawn i.i.d. from the same Zipf law,
    normalise(mu_j + sigma_q * N(0, I)), fp32.

Everything runs in torch on the device given (CPU for small cases, CUDA for
the large workloads); results are deterministic for a (config, device) pair.
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import math
import os
from typing import Dict, Optional

import numpy as np
import torch

DIM = 128


@dataclasses.dataclass(frozen=True)
class SynthConfig:
    name: str
    n_types: int
    zipf_s: float
    n_docs: int
    len_mean: float
    len_min: int
    len_max: int
    n_centroids: int
    centroid_dtype: str  # "f32" | "bf16"
    pq_m: int
    sigma_doc: float = 0.15
    sigma_query: float = 0.2
    lloyd_iters: int = 10
    pq_iters: int = 10
    pq_train_sample: int = 65536
    seed: int = 0
    # query side
    query_seed: int = 1000
    n_queries: int = 16
    ntok_min: int = 32
    ntok_max: int = 32
    kappa_c: int = 20
    kappa_d: int = 256
    k: int = 10

    def key(self) -> str:
        d = dataclasses.asdict(self)
        return hashlib.sha1(json.dumps(d, sort_keys=True).encode()).hexdigest()[:12]


CONFIGS: Dict[str, SynthConfig] = {
    # Tiny plain-FP32 workload: 2,000 types, 1,000 docs (~64k tokens), C=4,096.
    "tiny": SynthConfig(
        name="tiny", n_types=2000, zipf_s=1.0, n_docs=1000, len_mean=64, len_min=8,
        len_max=180, n_centroids=4096, centroid_dtype="f32", pq_m=16, seed=0,
        query_seed=1000, n_queries=16, kappa_c=20, kappa_d=256, k=10),
    # Parity workload between tiny and full size: several GEMM / gather tiles
    # with ragged tails (C and D are not multiples of any tile size).
    "small": SynthConfig(
        name="small", n_types=5000, zipf_s=1.1, n_docs=20011, len_mean=70, len_min=8,
        len_max=300, n_centroids=16411, centroid_dtype="bf16", pq_m=16, seed=11,
        query_seed=1011, n_queries=24, ntok_min=8, ntok_max=32, kappa_c=40,
        kappa_d=1000, k=100),
    # Same, with 32-byte codes (32 subspaces x 4 dims) and long documents.
    "small32": SynthConfig(
        name="small32", n_types=6000, zipf_s=0.9, n_docs=9001, len_mean=120, len_min=8,
        len_max=512, n_centroids=12289, centroid_dtype="bf16", pq_m=32, seed=13,
        query_seed=1013, n_queries=16, ntok_min=8, ntok_max=32, kappa_c=40,
        kappa_d=1000, k=10),
    # Passage-ranking-shaped, 1M documents (~70M tokens), C=262,144 bf16.
    "msmarco-1M": SynthConfig(
        name="msmarco-1M", n_types=30000, zipf_s=1.1, n_docs=1_000_000, len_mean=70,
        len_min=8, len_max=300, n_centroids=262144, centroid_dtype="bf16", pq_m=16,
        seed=1, query_seed=1001, n_queries=4096, kappa_c=40, kappa_d=1000, k=10),
    # Passage-ranking-shaped full scale: 8.8M docs (~600M tokens), C=2^21.
    "msmarco-8.8M": SynthConfig(
        name="msmarco-8.8M", n_types=30522, zipf_s=1.1, n_docs=8_800_000, len_mean=68,
        len_min=8, len_max=180, n_centroids=2097152, centroid_dtype="bf16", pq_m=16,
        seed=2, query_seed=1002, n_queries=1024, kappa_c=40, kappa_d=1000, k=10),
    # Long-tail-QA-shaped: 2.8M docs (~340M tokens), C=2^20, 32-byte codes.
    "lotte-2.8M": SynthConfig(
        name="lotte-2.8M", n_types=50000, zipf_s=0.9, n_docs=2_800_000, len_mean=120,
        len_min=8, len_max=512, n_centroids=1048576, centroid_dtype="bf16", pq_m=32,
        seed=3, query_seed=1003, n_queries=1024, ntok_min=8, ntok_max=32, kappa_c=40,
        kappa_d=1000, k=10),
}


def _gen(device, seed):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _normalise(x: torch.Tensor) -> torch.Tensor:
    return x / x.norm(dim=-1, keepdim=True).clamp_min(1e-30)


def _zipf_cdf(n_types: int, s: float, device) -> torch.Tensor:
    r = torch.arange(1, n_types + 1, dtype=torch.float64, device=device)
    p = r.pow(-s)
    p = p / p.sum()
    cdf = torch.cumsum(p, 0)
    cdf[-1] = 1.0
    return cdf


def _draw_types(cdf: torch.Tensor, n: int, g, device, chunk=1 << 24) -> torch.Tensor:
    out = torch.empty(n, dtype=torch.int32, device=device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        u = torch.rand(e - s, generator=g, device=device, dtype=torch.float64)
        out[s:e] = torch.searchsorted(cdf, u, right=True).clamp_max(cdf.numel() - 1).to(torch.int32)
    return out


def allot_sqrt(counts: np.ndarray, budget: int) -> np.ndarray:
    """kappa_j ~ sqrt(n_j), >= 1 for every occurring type, <= n_j, sum == budget."""
    counts = counts.astype(np.int64)
    occ = counts > 0
    if budget < occ.sum():
        raise ValueError("centroid budget below the number of occurring token types")
    if budget > counts.sum():
        raise ValueError("centroid budget above the number of tokens")
    w = np.sqrt(counts.astype(np.float64))
    raw = budget * w / w.sum()
    k = np.where(occ, np.maximum(1, np.floor(raw)), 0).astype(np.int64)
    k = np.minimum(k, counts)
    # largest-remainder reconciliation to exactly `budget`
    for _ in range(64):
        diff = budget - int(k.sum())
        if diff == 0:
            break
        rem = raw - k
        if diff > 0:
            cand = np.where(k < counts)[0]
            order = cand[np.argsort(-rem[cand], kind="stable")]
            take = order[:diff]
            k[take] += 1
        else:
            cand = np.where(k > 1)[0]
            order = cand[np.argsort(rem[cand], kind="stable")]
            take = order[:-diff]
            k[take] -= 1
    assert int(k.sum()) == budget
    return k


def _lloyd_group(P: torch.Tensor, valid: torch.Tensor, C0: torch.Tensor, cvalid: torch.Tensor,
                 iters: int, pchunk: int):
    """Batched Lloyd over G independent problems.

    P [G, n, d] points (padded), valid [G, n]; C0 [G, k, d] initial centroids,
    cvalid [G, k]. Returns (C [G,k,d], assign [G,n] local centroid index).
    """
    G, n, d = P.shape
    k = C0.shape[1]
    C = C0.clone()
    big = torch.finfo(torch.float32).max

    def assign(C):
        cn = (C * C).sum(-1)  # [G, k]
        cn = torch.where(cvalid, cn, torch.full_like(cn, big))
        a = torch.empty(G, n, dtype=torch.int64, device=P.device)
        for s in range(0, n, pchunk):
            e = min(n, s + pchunk)
            dots = torch.bmm(P[:, s:e], C.transpose(1, 2))  # [G, e-s, k]
            dist = cn[:, None, :] - 2.0 * dots
            a[:, s:e] = dist.argmin(-1)
        return a

    for _ in range(iters):
        a = assign(C)
        flat = (a + torch.arange(G, device=P.device)[:, None] * k)[valid]
        sums = torch.zeros(G * k, d, dtype=torch.float32, device=P.device)
        sums.index_add_(0, flat, P[valid])
        cnt = torch.bincount(flat, minlength=G * k).to(torch.float32)
        newC = sums / cnt.clamp_min(1.0)[:, None]
        keep = (cnt == 0)[:, None]
        C = torch.where(keep, C.reshape(G * k, d), newC).reshape(G, k, d)
    return C, assign(C)


def _per_type_kmeans(X, types, kappa, iters, g, device, log=None):
    """Per-token-type k-means (Sec. 2.1): independent Lloyd per type.

    Returns centroids [C, d] fp32 (types in id order, kappa_j consecutive
    centroids each) and the global assignment a(t) [T] int64.
    """
    T = X.shape[0]
    V = kappa.shape[0]
    types64 = types.to(torch.int64)
    order = torch.argsort(types64, stable=True)
    counts = torch.bincount(types64, minlength=V).cpu().numpy()
    starts = np.zeros(V + 1, dtype=np.int64)
    starts[1:] = np.cumsum(counts)
    coff = np.zeros(V + 1, dtype=np.int64)
    coff[1:] = np.cumsum(kappa)
    C_total = int(coff[-1])
    cents = torch.zeros(C_total, DIM, dtype=torch.float32, device=device)
    assign = torch.empty(T, dtype=torch.int64, device=device)

    occ = np.where(counts > 0)[0]
    occ = occ[np.argsort(-counts[occ], kind="stable")]
    PBUDGET = 1 << 21  # padded points per group
    DBUDGET = 1 << 27  # distance entries per bmm chunk
    TRAIN_CAP = 1 << 24  # a larger type trains on its first 2^24 tokens, then assigns all of them
    i = 0
    while i < len(occ) and int(counts[occ[i]]) > TRAIN_CAP:
        j = int(occ[i])
        n, kj = int(counts[j]), int(kappa[j])
        tok = order[int(starts[j]):int(starts[j]) + n]
        P = X[tok[:TRAIN_CAP]].to(torch.float32)[None]  # [1, cap, d]
        valid = torch.ones(1, TRAIN_CAP, dtype=torch.bool, device=device)
        keys = torch.rand(1, TRAIN_CAP, generator=g, device=device)
        pick = torch.argsort(keys, dim=1)[:, :kj]
        C0 = torch.gather(P, 1, pick[:, :, None].expand(1, kj, DIM))
        cvalid = torch.ones(1, kj, dtype=torch.bool, device=device)
        Cf, _ = _lloyd_group(P, valid, C0, cvalid, iters, max(1, DBUDGET // kj))
        del P
        cents[int(coff[j]):int(coff[j]) + kj] = Cf[0]
        C = Cf[0]
        cn = (C * C).sum(-1)
        ch = max(1, DBUDGET // kj)
        for s0 in range(0, n, ch):
            e0 = min(n, s0 + ch)
            x = X[tok[s0:e0]].to(torch.float32)
            assign[tok[s0:e0]] = int(coff[j]) + (cn[None, :] - 2.0 * (x @ C.T)).argmin(-1)
        i += 1
        if log is not None:
            log(f"kmeans of type {j}: {n} tokens (trained on {TRAIN_CAP}), k={kj}")
    while i < len(occ):
        n_max = int(counts[occ[i]])
        G = max(1, PBUDGET // max(1, n_max))
        grp = occ[i:i + G]
        G = len(grp)
        k_max = int(kappa[grp].max())
        pchunk = max(1, DBUDGET // max(1, G * k_max))
        # gather padded points
        ar = torch.arange(n_max, device=device)
        st = torch.as_tensor(starts[grp], device=device)
        nn = torch.as_tensor(counts[grp], device=device)
        valid = ar[None, :] < nn[:, None]
        idx = (st[:, None] + torch.minimum(ar[None, :], (nn - 1)[:, None]))
        P = X[order[idx]].to(torch.float32)  # [G, n_max, d]
        # seeded init: kappa_j distinct points per type
        keys = torch.rand(G, n_max, generator=g, device=device)
        keys = torch.where(valid, keys, torch.full_like(keys, 2.0))
        pick = torch.argsort(keys, dim=1)[:, :k_max]
        C0 = torch.gather(P, 1, pick[:, :, None].expand(G, k_max, DIM))
        kk = torch.as_tensor(kappa[grp], device=device)
        cvalid = torch.arange(k_max, device=device)[None, :] < kk[:, None]
        Cf, a = _lloyd_group(P, valid, C0, cvalid, iters, pchunk)
        # scatter back
        base = torch.as_tensor(coff[grp], device=device)
        for gi in range(G):
            kj = int(kappa[grp[gi]])
            cents[int(coff[grp[gi]]):int(coff[grp[gi]]) + kj] = Cf[gi, :kj]
        glob = a + base[:, None]
        assign[order[idx][valid]] = glob[valid]
        i += G
        if log is not None:
            log(f"kmeans group of {G} types, n_max={n_max}, k_max={k_max}")
    return cents, assign


def _pq_train_encode(R, m, iters, sample, g, device, chunk=1 << 20):
    """PQ on normalised residuals (Sec. 2.1): M subspaces of d/M dims, 256 codewords."""
    T = R.shape[0]
    ds = DIM // m
    ns = min(T, sample)
    sel = torch.randperm(T, generator=g, device=device)[:ns]
    S = R[sel].to(torch.float32).reshape(ns, m, ds).transpose(0, 1).contiguous()  # [m, ns, ds]
    init = torch.randperm(ns, generator=g, device=device)[:256]
    if ns < 256:
        init = torch.arange(256, device=device) % ns
    W = S[:, init, :].clone()  # [m, 256, ds]
    for _ in range(iters):
        wn = (W * W).sum(-1)
        dist = wn[:, None, :] - 2.0 * torch.bmm(S, W.transpose(1, 2))
        a = dist.argmin(-1)  # [m, ns]
        flat = (a + torch.arange(m, device=device)[:, None] * 256).reshape(-1)
        sums = torch.zeros(m * 256, ds, dtype=torch.float32, device=device)
        sums.index_add_(0, flat, S.reshape(-1, ds))
        cnt = torch.bincount(flat, minlength=m * 256).to(torch.float32)
        newW = sums / cnt.clamp_min(1.0)[:, None]
        W = torch.where((cnt == 0)[:, None], W.reshape(-1, ds), newW).reshape(m, 256, ds)
    codes = torch.empty(T, m, dtype=torch.uint8, device=device)
    wn = (W * W).sum(-1)
    for s in range(0, T, chunk):
        e = min(T, s + chunk)
        x = R[s:e].to(torch.float32).reshape(e - s, m, ds).transpose(0, 1)  # [m, n, ds]
        dist = wn[:, None, :] - 2.0 * torch.bmm(x, W.transpose(1, 2))
        codes[s:e] = dist.argmin(-1).transpose(0, 1).to(torch.uint8)
    return W, codes


def make_index(cfg: SynthConfig, device="cpu", log=None) -> dict:
    """Build the seeded index for `cfg`; returns host numpy arrays."""
    device = torch.device(device)
    g = _gen(device, cfg.seed)
    cdf = _zipf_cdf(cfg.n_types, cfg.zipf_s, device)
    means = _normalise(torch.randn(cfg.n_types, DIM, generator=g, device=device, dtype=torch.float32))
    sl = 0.5
    mu = math.log(cfg.len_mean) - sl * sl / 2
    ln = torch.exp(mu + sl * torch.randn(cfg.n_docs, generator=g, device=device, dtype=torch.float64))
    lengths = torch.round(ln).clamp(cfg.len_min, cfg.len_max).to(torch.int64)
    doc_off = torch.zeros(cfg.n_docs + 1, dtype=torch.int64, device=device)
    doc_off[1:] = torch.cumsum(lengths, 0)
    T = int(doc_off[-1])
    types = _draw_types(cdf, T, g, device)
    xdt = torch.float32 if T <= (1 << 24) else torch.float16
    X = torch.empty(T, DIM, dtype=xdt, device=device)
    ch = 1 << 22
    for s in range(0, T, ch):
        e = min(T, s + ch)
        v = means[types[s:e].to(torch.int64)] + cfg.sigma_doc * torch.randn(
            e - s, DIM, generator=g, device=device, dtype=torch.float32)
        X[s:e] = _normalise(v).to(xdt)
    if log:
        log(f"{cfg.name}: {cfg.n_docs} docs, {T} tokens")
    counts = torch.bincount(types.to(torch.int64), minlength=cfg.n_types).cpu().numpy()
    kappa = allot_sqrt(counts, cfg.n_centroids)
    cents, assign = _per_type_kmeans(X, types, kappa, cfg.lloyd_iters, g, device, log)
    if cfg.centroid_dtype == "bf16":
        cstore = cents.to(torch.bfloat16)
        cwide = cstore.to(torch.float32)
    else:
        cstore = cents
        cwide = cents
    cent_type = torch.repeat_interleave(
        torch.arange(cfg.n_types, device=device, dtype=torch.int32),
        torch.as_tensor(kappa, device=device))
    # residuals against the stored centroids; norms kept in fp16
    rnorm = torch.empty(T, dtype=torch.float16, device=device)
    Rn = X  # the normalised residuals overwrite the token vectors chunk by chunk
    for s in range(0, T, ch):
        e = min(T, s + ch)
        r = X[s:e].to(torch.float32) - cwide[assign[s:e]]
        nr = r.norm(dim=-1)
        rnorm[s:e] = nr.to(torch.float16)
        Rn[s:e] = torch.where(nr[:, None] > 0, r / nr.clamp_min(1e-30)[:, None],
                              torch.zeros_like(r)).to(xdt)
    del X
    W, codes = _pq_train_encode(Rn, cfg.pq_m, cfg.pq_iters, cfg.pq_train_sample, g, device)
    del Rn
    if cfg.centroid_dtype == "bf16":
        cnp = cstore.view(torch.int16).cpu().numpy().view(np.uint16)
    else:
        cnp = cstore.cpu().numpy().astype(np.float32)
    return {
        "name": cfg.name,
        "centroid_dtype": cfg.centroid_dtype,
        "centroids": np.ascontiguousarray(cnp),
        "centroid_type": cent_type.cpu().numpy().astype(np.int32),
        "doc_offsets": doc_off.cpu().numpy().astype(np.int64),
        "token_centroid": assign.to(torch.int32).cpu().numpy(),
        "pq_codebooks": W.cpu().numpy().astype(np.float32),
        "pq_codes": np.ascontiguousarray(codes.cpu().numpy()),
        "residual_norms": rnorm.view(torch.int16).cpu().numpy().view(np.uint16),
        "kappa": kappa.astype(np.int32),
    }


def make_queries(cfg: SynthConfig, n_queries: Optional[int] = None, seed: Optional[int] = None,
                 ntok_min: Optional[int] = None, ntok_max: Optional[int] = None,
                 device="cpu") -> dict:
    """Seeded query batch: per-query token counts in [ntok_min, ntok_max], fp32 unit vectors."""
    device = torch.device(device)
    nq = cfg.n_queries if n_queries is None else n_queries
    lo = cfg.ntok_min if ntok_min is None else ntok_min
    hi = cfg.ntok_max if ntok_max is None else ntok_max
    # the type means are the index's: regenerate them from the index seed
    gi = _gen(device, cfg.seed)
    means = _normalise(torch.randn(cfg.n_types, DIM, generator=gi, device=device, dtype=torch.float32))
    g = _gen(device, cfg.query_seed if seed is None else seed)
    ntok = torch.randint(lo, hi + 1, (nq,), generator=g, device=device, dtype=torch.int64)
    total = int(ntok.sum())
    cdf = _zipf_cdf(cfg.n_types, cfg.zipf_s, device)
    ty = _draw_types(cdf, total, g, device).to(torch.int64)
    v = means[ty] + cfg.sigma_query * torch.randn(total, DIM, generator=g, device=device,
                                                  dtype=torch.float32)
    q = _normalise(v.to(torch.float64)).to(torch.float32)
    return {"queries": q.cpu().numpy(), "ntok": ntok.to(torch.int32).cpu().numpy()}


def index_bytes(ix: dict) -> int:
    return sum(v.nbytes for v in ix.values() if isinstance(v, np.ndarray))


def _cache_dir() -> str:
    return os.environ.get("TACHIOM_SYNTH_CACHE", os.path.join("/tmp", "tachiom_synth"))


def load_or_make(name: str, device="cpu", log=None) -> dict:
    """make_index with an on-disk cache keyed by the config's hash and the device type."""
    cfg = CONFIGS[name]
    dev = torch.device(device)
    path = os.path.join(_cache_dir(), f"{cfg.name}-{cfg.key()}-{dev.type}.npz")
    if os.path.exists(path):
        with np.load(path, allow_pickle=False) as z:
            ix = {k: z[k] for k in z.files}
        ix["name"] = str(ix["name"])
        ix["centroid_dtype"] = str(ix["centroid_dtype"])
        return ix
    ix = make_index(cfg, device=dev, log=log)
    if dev.type == "cuda":
        torch.cuda.empty_cache()  # hand the generator's device memory back
    try:
        os.makedirs(_cache_dir(), exist_ok=True)
        tmp = path + ".tmp.npz"
        np.savez(tmp, **ix)
        os.replace(tmp, path)
    except OSError:
        pass  # no room for the cache: the index is regenerated next time
    return ix


def random_index(n_docs: int, n_centroids: int, dim: int = DIM, pq_m: int = 16, len_min: int = 1,
                 len_max: int = 12, seed: int = 0, centroid_dtype: str = "f32",
                 norms: str = "random", empty_docs: int = 0) -> dict:
    """Unstructured random index for edge cases: i.i.d. centroid ids per token,
    random codes, random fp16 norms (norms="zero" gives rho = 0, "none" omits
    them), `empty_docs` documents of length 0 placed at seeded positions."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(len_min, len_max + 1, size=n_docs)
    if empty_docs:
        lengths[rng.choice(n_docs, size=empty_docs, replace=False)] = 0
    doc_off = np.zeros(n_docs + 1, np.int64)
    doc_off[1:] = np.cumsum(lengths)
    T = int(doc_off[-1])
    c = rng.standard_normal((n_centroids, dim)).astype(np.float32)
    c /= np.linalg.norm(c, axis=1, keepdims=True) * rng.uniform(1.0, 2.0, size=(n_centroids, 1))
    if centroid_dtype == "bf16":
        cb = torch.from_numpy(c).to(torch.bfloat16)
        cent = cb.view(torch.int16).numpy().view(np.uint16)
    else:
        cent = c
    ds = dim // pq_m
    W = (rng.standard_normal((pq_m, 256, ds)) / np.sqrt(dim)).astype(np.float32)
    ix = {
        "name": "random",
        "centroid_dtype": centroid_dtype,
        "centroids": np.ascontiguousarray(cent),
        "centroid_type": np.arange(n_centroids, dtype=np.int32),
        "doc_offsets": doc_off,
        "token_centroid": rng.integers(0, n_centroids, size=T).astype(np.int32),
        "pq_codebooks": W,
        "pq_codes": rng.integers(0, 256, size=(T, pq_m)).astype(np.uint8),
    }
    if norms == "random":
        ix["residual_norms"] = rng.uniform(0.0, 1.0, size=T).astype(np.float16).view(np.uint16)
    elif norms == "zero":
        ix["residual_norms"] = np.zeros(T, np.uint16)
    return ix


def random_queries(n_queries: int, ntok_min: int, ntok_max: int, dim: int = DIM, seed: int = 0) -> dict:
    """Unit-norm random query tokens, fp32 (edge-case inputs)."""
    rng = np.random.default_rng(seed)
    ntok = rng.integers(ntok_min, ntok_max + 1, size=n_queries).astype(np.int32)
    q = rng.standard_normal((int(ntok.sum()), dim))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return {"queries": q.astype(np.float32), "ntok": ntok}

"""Token-Aware Clustering on the GPU (tachiom_tac_cluster) against the FP64 oracle (oracle/tac.py).

The inputs are separated blobs per token type, so the nearest centroid of every vector is far from a
tie and the FP32 distances of the kernel and the oracle's FP64 ones choose the same labels; centroids
then agree to FP32 rounding (rtol 1e-6).
"""
import numpy as np
import pytest

from oracle import tac as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PARAMS = dict(mu=5, tau=20, eps=1, theta=10.0)


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _blobs(counts, seed):
    """Vectors of each type drawn around a few centers of that type (scale 10, noise 0.01)."""
    rng = np.random.default_rng(seed)
    vecs, types = [], []
    for j, cnt in enumerate(counts):
        centers = rng.normal(size=(1 + j % 4, 128)) * 10.0
        for i in range(cnt):
            vecs.append(centers[i % len(centers)] + 0.01 * rng.normal(size=128))
            types.append(j)
    order = rng.permutation(len(types))  # types interleaved in the collection
    return np.array(vecs, np.float32)[order], np.array(types, np.int32)[order]


def _run(T, v, t, n_types, budget, iters, **kw):
    return T.tac_cluster(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), n_types, budget,
                         iters=iters, **kw)


def test_tac_cluster_matches_oracle():
    _cuda()
    import paper_2604_28142_b300 as T
    counts = [400, 200, 130, 100, 80, 60, 50, 40, 8, 4, 2, 0]
    v, t = _blobs(counts, seed=41)
    n_types, iters = len(counts), 6
    s_or = O.spread(v.astype(np.float64).tolist(), t.tolist(), n_types)
    lo_hi = [min(x, max(1, int(np.floor(x / PARAMS["theta"])))) for x in counts if x >= PARAMS["tau"]]
    tail = sum(1 if 0 < x < PARAMS["mu"] else 2 if PARAMS["mu"] <= x < PARAMS["tau"] else 0 for x in counts)
    budget = tail + (sum(min(PARAMS["eps"], c) for c in lo_hi) + sum(lo_hi)) // 2
    kappa, spread, cents, ctype, labels = _run(T, v, t, n_types, budget, iters, **PARAMS)
    torch.cuda.synchronize()
    assert np.allclose(spread, s_or, rtol=1e-6, atol=0)  # compensated FP32 against FP64
    ok, oc, oct_, olab = O.cluster(v.astype(np.float64).tolist(), t.tolist(), n_types, budget,
                                   iters=iters, **PARAMS)
    assert kappa.tolist() == ok
    assert ctype.cpu().tolist() == oct_
    assert labels.cpu().tolist() == olab
    assert np.allclose(cents.cpu().numpy(), np.array(oc), rtol=1e-6, atol=1e-6)
    # the same call repeats bit for bit
    k2, s2, c2, ct2, l2 = _run(T, v, t, n_types, budget, iters, **PARAMS)
    torch.cuda.synchronize()
    assert np.array_equal(k2, kappa) and np.array_equal(s2, spread)
    assert torch.equal(c2, cents) and torch.equal(ct2, ctype) and torch.equal(l2, labels)


def test_tac_cluster_gemm_path_equals_cuda_core_path():
    # Types with many centroids are assigned through a BF16 GEMM on the tensor cores and an exact
    # FP32 rescoring of every centroid within a rigorous margin of the approximate best: the labels,
    # and so the centroids of every round, must be those of the CUDA-core kernel bit for bit. Noisy
    # blobs (noise 1.0 against centres of scale 3) put several centroids of a type near each point,
    # so the margin holds more than one candidate for many points.
    _cuda()
    import paper_2604_28142_b300 as T
    rng = np.random.default_rng(77)
    parts_v, parts_t = [], []
    for j, (n, k) in enumerate([(12000, 90), (3000, 12), (700, 5), (40, 1)]):
        centers = rng.normal(size=(k, 128)) * 3.0
        parts_v.append(centers[rng.integers(0, k, size=n)] + rng.normal(size=(n, 128)))
        parts_t.append(np.full(n, j, np.int32))
    perm = rng.permutation(sum(len(t) for t in parts_t))
    v = np.concatenate(parts_v).astype(np.float32)[perm]
    t = np.concatenate(parts_t)[perm]
    kw = dict(mu=5, tau=20, eps=1, theta=10.0)
    res = {}
    for gmk in (-1, 0, 8):
        res[gmk] = _run(T, v, t, 4, 200, 5, gemm_min_kappa=gmk, **kw)
    torch.cuda.synchronize()
    kappa = res[-1][0]
    assert kappa.max() >= 64  # the default threshold sends at least one type to the GEMM path
    for gmk in (0, 8):
        k2, s2, c2, ct2, l2 = res[gmk]
        assert np.array_equal(k2, kappa)
        assert torch.equal(l2, res[-1][4]), f"labels differ (gemm_min_kappa {gmk})"
        assert torch.equal(c2, res[-1][2]) and torch.equal(ct2, res[-1][3])


def test_tac_cluster_type_without_centroid_and_bad_type():
    _cuda()
    import paper_2604_28142_b300 as T
    # type 1: 50 identical vectors (spread 0, weight 0) and eps = 0: it receives no centroid, so its
    # vectors get label -1; type 0 takes the whole budget of 3
    rng = np.random.default_rng(7)
    v = np.concatenate([rng.normal(size=(50, 128)) * 10.0, np.tile(rng.normal(size=(1, 128)), (50, 1))])
    v = v.astype(np.float32)
    t = np.array([0] * 50 + [1] * 50, np.int32)
    kappa, _, cents, ctype, labels = _run(T, v, t, 2, 3, 4, mu=1, tau=2, eps=0, theta=1.0)
    torch.cuda.synchronize()
    ok, oc, oct_, olab = O.cluster(v.astype(np.float64).tolist(), t.tolist(), 2, 3, mu=1, tau=2, eps=0,
                                   theta=1.0, iters=4)
    assert kappa.tolist() == ok == [3, 0]
    assert labels.cpu().tolist() == olab and olab[50:] == [-1] * 50
    bad = t.copy()
    bad[10] = 5
    with pytest.raises(T.TachiomError):
        _run(T, v, bad, 2, 3, 1, mu=1, tau=2, eps=0, theta=1.0)


def _pq_case(M, seed, lossless):
    rng = np.random.default_rng(seed)
    ds = 128 // M
    if lossless:
        # codewords of norm 1 / sqrt(M): one per subspace concatenates to a unit vector
        cb = rng.normal(size=(M, 256, ds))
        cb /= np.linalg.norm(cb, axis=2, keepdims=True) * np.sqrt(M)
    else:
        cb = rng.normal(size=(M, 256, ds)) * 0.2
    cents = rng.normal(size=(5, 128))
    n = 64
    lab = rng.integers(0, 5, size=n)
    lab[:3] = -1
    if lossless:
        want = rng.integers(0, 256, size=(n, M))
        rho = rng.uniform(0.1, 2.0, size=n)
        u = np.stack([np.concatenate([cb[m][want[i, m]] for m in range(M)]) for i in range(n)])
        x = cents[np.maximum(lab, 0)] + rho[:, None] * u
    else:
        x = cents[np.maximum(lab, 0)] + rng.normal(size=(n, 128)) * 0.3
    x[:3] = rng.normal(size=(3, 128))
    return x.astype(np.float32), cents.astype(np.float32), lab.astype(np.int32), cb.astype(np.float32)


@pytest.mark.parametrize("M", [8, 16, 32])
@pytest.mark.parametrize("lossless", [True, False])
def test_pq_encode_against_oracle(M, lossless):
    _cuda()
    import paper_2604_28142_b300 as T
    x, cents, lab, cb = _pq_case(M, 50 + M, lossless)
    codes, rnorm = T.pq_encode(torch.from_numpy(x).cuda(), torch.from_numpy(cents).cuda(),
                               torch.from_numpy(lab).cuda(), torch.from_numpy(cb).cuda())
    torch.cuda.synchronize()
    codes = codes.cpu().numpy().astype(np.int64)
    rho_g = rnorm.cpu().numpy().view(np.float16).astype(np.float64)
    ok = lab >= 0
    oc, orho = O.pq_encode(x[ok].astype(np.float64).tolist(), cents.astype(np.float64).tolist(),
                           lab[ok].tolist(), cb.astype(np.float64).tolist())
    oc, orho = np.array(oc), np.array(orho)
    assert np.all(codes[~ok] == 0) and np.all(rho_g[~ok] == 0.0)
    # rho: the oracle's norm rounded to fp16 (within one fp16 step of it)
    assert np.all(np.abs(rho_g[ok] - orho) <= np.abs(orho) * 2.0 ** -10 + 1e-7)
    if lossless:
        assert np.array_equal(codes[ok], oc)
    else:
        # a valid code: its codeword is as near as the oracle's to within FP32 rounding
        ds = 128 // M
        u = (x[ok].astype(np.float64) - cents[lab[ok]].astype(np.float64)) / orho[:, None]
        for m in range(M):
            sub = u[:, m * ds:(m + 1) * ds]
            dist = ((sub[:, None, :] - cb[m][None].astype(np.float64)) ** 2).sum(-1)
            got = dist[np.arange(len(sub)), codes[ok][:, m]]
            assert np.all(got <= dist.min(1) + 1e-5)
        assert (codes[ok] == oc).mean() > 0.99


def _pq_train_case(M, seed):
    """Vectors whose sampled normalised residuals fall, in every subspace, into 256 tight clusters of
    two consecutive sample points: the evenly spaced initial codewords (positions 2 j + 1) take one
    point of each cluster, so Lloyd's answer is the mean of every pair."""
    rng = np.random.default_rng(seed)
    ds = 128 // M
    true = rng.normal(size=(M, 256, ds))
    true /= np.linalg.norm(true, axis=2, keepdims=True) * np.sqrt(M)
    perm = np.stack([rng.permutation(256) for _ in range(M)])
    n = 512
    cid = perm[:, np.arange(n) // 2]                               # [M, n]: cluster of sample r
    u = np.concatenate([true[m][cid[m]] for m in range(M)], axis=1) + 1e-5 * rng.normal(size=(n, 128))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    cents = rng.normal(size=(4, 128))
    lab = rng.integers(0, 4, size=n)
    x = cents[lab] + rng.uniform(0.2, 2.0, size=(n, 1)) * u
    return x.astype(np.float32), cents.astype(np.float32), lab.astype(np.int32), cid


@pytest.mark.parametrize("M", [8, 16, 32])
def test_pq_train_closed_form(M):
    _cuda()
    import paper_2604_28142_b300 as T
    x, cents, lab, cid = _pq_train_case(M, 70 + M)
    dx, dc, dl = torch.from_numpy(x).cuda(), torch.from_numpy(cents).cuda(), torch.from_numpy(lab).cuda()
    books = T.pq_train(dx, dc, dl, M, sample=512, iters=3)
    torch.cuda.synchronize()
    # the sample is every vector (positions floor(r + 1/2) = r); its normalised residuals in FP64
    r = x.astype(np.float64) - cents[lab].astype(np.float64)
    u = r / np.linalg.norm(r, axis=1, keepdims=True)
    ds = 128 // M
    b = books.cpu().numpy().astype(np.float64)
    for m in range(M):
        sub = u[:, m * ds:(m + 1) * ds]
        for j in range(256):
            want = sub[2 * j:2 * j + 2].mean(0)  # codeword j started at sample 2 j + 1: cluster of pair j
            assert np.allclose(b[m, j], want, atol=1e-6), (m, j)
    # encoding the sample with the trained codebooks gives back each sample's pair
    codes, _ = T.pq_encode(dx, dc, dl, books)
    torch.cuda.synchronize()
    assert np.array_equal(codes.cpu().numpy().astype(np.int64), np.repeat(np.arange(256), 2)[:, None].repeat(M, 1))
    # the same call repeats bit for bit
    assert torch.equal(T.pq_train(dx, dc, dl, M, sample=512, iters=3), books)


@pytest.mark.parametrize("centroid_dtype", ["f32", "bf16"])
def test_index_built_on_gpu_searches_like_the_oracle(centroid_dtype):
    # an index built from raw vectors by the library's kernels, searched in both precisions, gives
    # the FP64 oracle's results on the same index arrays
    _cuda()
    import paper_2604_28142_b300 as T
    from paper_2604_28142_b300.index_build import build_index
    from oracle import Oracle
    from compare import check_ranking
    rng = np.random.default_rng(81)
    n_types, n_docs = 60, 400
    lens = rng.integers(4, 40, size=n_docs)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    Tn = int(off[-1])
    p = 1.0 / np.arange(1, n_types + 1) ** 1.1
    types = rng.choice(n_types, size=Tn, p=p / p.sum()).astype(np.int32)
    dirs = rng.normal(size=(n_types, 3, 128))
    v = dirs[types, rng.integers(0, 3, size=Tn)] + 0.4 * rng.normal(size=(Tn, 128))
    v = (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    ix = build_index(torch.from_numpy(v).cuda(), torch.from_numpy(types).cuda(), off, n_types, 512,
                     mu=3, tau=12, eps=1, theta=4.0, iters=5, pq_m=16, pq_sample=1024, pq_iters=4,
                     centroid_dtype=centroid_dtype)
    assert ix["centroids"].shape[0] == 512 and ix["token_centroid"].min() >= 0
    G, O_ = T.Index(ix, 0), Oracle(ix)
    qi = rng.integers(0, Tn, size=(6, 16))
    q = v[qi].reshape(-1, 128) + 0.05 * rng.normal(size=(96, 128)).astype(np.float32)
    q = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    ntok = np.full(6, 16, np.int32)
    k, kc, kd = 10, 8, 100
    want = O_.search(q, ntok, k, kc, kd)
    for prec in (T.PREC_FP32, T.PREC_BF16):
        oi = torch.empty(6 * k, dtype=torch.int32, device="cuda")
        os_ = torch.empty(6 * k, dtype=torch.float32, device="cuda")
        G.search(T.SearchParams(kappa_c=kc, kappa_d=kd, precision=prec), torch.from_numpy(q).cuda(), ntok,
                 np.full(6, k, np.int32), oi, os_)
        torch.cuda.synchronize()
        gi, gs = oi.cpu().numpy(), os_.cpu().numpy()
        for u in range(6):
            sl = slice(u * k, (u + 1) * k)
            check_ranking(gi[sl], gs[sl], want["ids"][sl], want["scores"][sl], 1e-5, 1e-4, what=f"query {u}")

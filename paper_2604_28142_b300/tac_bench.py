"""Benchmark of index construction: Token-Aware Clustering (tachiom_tac_cluster) and residual
encoding (tachiom_pq_encode) of a synthetic multivector collection on one GPU.

The collection (seeded, generated on the device, untimed): N unit vectors of 128 dims whose token
types follow a Zipf law over V types (as in the passage-ranking workload: 30,000 types, exponent
1.1); each type has 1-4 sub-centres around its own direction, and a vector is a normalised sub-centre
plus Gaussian noise. The clustering shares `budget` centroids out with Sec. 2.1's allotment and runs
`iters` Lloyd rounds per type; the encoding uses seeded unit codebooks of M subspaces (codebook
training is not part of this measurement). Prints one JSON line: the clustering's wall time (the
call is synchronous), vectors per second, the encoding's time, and the allotment's shape.

    python -m paper_2604_28142_b300.tac_bench --vectors 70000000 --budget 262144 --iters 10
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)


def parse(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--vectors", type=int, default=70_000_000)
    ap.add_argument("--types", type=int, default=30_000)
    ap.add_argument("--zipf", type=float, default=1.1)
    ap.add_argument("--budget", type=int, default=262_144)
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--mu", type=int, default=4, help="types with fewer vectors get 1 centroid")
    ap.add_argument("--tau", type=int, default=32, help="types with fewer vectors (and >= mu) get 2")
    ap.add_argument("--eps", type=int, default=2, help="floor of an active type's allotment")
    ap.add_argument("--theta", type=float, default=64.0, help="at least theta vectors per centroid")
    ap.add_argument("--pq-m", type=int, default=16, choices=[8, 16, 32])
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--device", default="cuda")
    return ap.parse_args(argv)


def make_collection(n, n_types, zipf_s, seed, device):
    """(vectors fp32 [n, 128], types int32 [n]) of the recipe in the module docstring."""
    import torch
    from synth import gen
    g = gen._gen(device, seed)
    types = gen._draw_types(gen._zipf_cdf(n_types, zipf_s, device), n, g, device)
    dirs = gen._normalise(torch.randn(n_types, 128, generator=g, device=device))
    subs = gen._normalise(dirs[:, None, :] + 0.3 * torch.randn(n_types, 4, 128, generator=g, device=device))
    nsub = 1 + torch.arange(n_types, device=device) % 4
    x = torch.empty((n, 128), dtype=torch.float32, device=device)
    chunk = 1 << 22
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        t = types[s:e].long()
        k = torch.randint(0, 1 << 30, (e - s,), generator=g, device=device) % nsub[t]
        x[s:e] = gen._normalise(subs[t, k] + 0.15 * torch.randn(e - s, 128, generator=g, device=device))
    return x, types


def unit_codebooks(m, seed, device):
    """Seeded codebooks [m, 256, 128 / m] with codewords of norm 1 / sqrt(m)."""
    import torch
    from synth import gen
    g = gen._gen(device, seed + 1)
    cb = torch.randn(m, 256, 128 // m, generator=g, device=device)
    return (cb / cb.norm(dim=-1, keepdim=True) / np.sqrt(m)).float().contiguous()


def main(argv=None):
    a = parse(argv)
    import torch
    import paper_2604_28142_b300 as T
    x, types = make_collection(a.vectors, a.types, a.zipf, a.seed, a.device)
    kw = dict(mu=a.mu, tau=a.tau, eps=a.eps, theta=a.theta)
    # warm-up on a small slice (kernel loading, library set-up), untimed
    w = min(a.vectors, 1 << 16)
    T.tac_cluster(x[:w], types[:w], a.types, max(1, min(a.budget, w // 64)) if w >= 64 else 1, iters=1,
                  mu=0, tau=0, eps=0, theta=1.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    kappa, spread, cents, ctype, labels = T.tac_cluster(x, types, a.types, a.budget, iters=a.iters, **kw)
    torch.cuda.synchronize()
    t_cluster = time.perf_counter() - t0
    cb = unit_codebooks(a.pq_m, a.seed, a.device)
    T.pq_encode(x[:w], cents, labels[:w], cb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    codes, rnorm = T.pq_encode(x, cents, labels, cb)
    e1.record()
    torch.cuda.synchronize()
    t_encode = e0.elapsed_time(e1) / 1e3
    # mean squared distance of the assigned vectors to their centroids, in chunks
    tot, cnt = 0.0, 0
    for s in range(0, a.vectors, 1 << 22):
        lab = labels[s:s + (1 << 22)].long()
        ok = lab >= 0
        tot += float(((x[s:s + (1 << 22)][ok] - cents[lab[ok]]) ** 2).sum(dtype=torch.float64).item())
        cnt += int(ok.sum().item())
    inertia = tot / max(1, cnt)
    n = np.bincount(types.cpu().numpy(), minlength=a.types)
    line = {
        "metric": "Token-Aware Clustering wall time (allotment + per-type Lloyd + assignment)",
        "value": t_cluster, "unit": "s", "higher_is_better": False,
        "vectors_per_s": a.vectors / t_cluster,
        "pq_encode_s": t_encode,
        "inertia_per_vector": inertia,
        "kappa": {"types_with_centroids": int((kappa > 0).sum()), "max": int(kappa.max()),
                  "sum_n_kappa": float((n.astype(np.float64) * kappa).sum())},
        "config": {"vectors": a.vectors, "types": a.types, "zipf": a.zipf, "budget": a.budget, "iters": a.iters,
                   "mu": a.mu, "tau": a.tau, "eps": a.eps, "theta": a.theta, "pq_m": a.pq_m, "seed": a.seed},
        "data": "synthetic (seeded Zipfian token types, per-type sub-centres, unit vectors)",
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()

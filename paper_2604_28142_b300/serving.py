"""Open-loop serving benchmark of the continuous-batching request loop.

Requests arrive as a Poisson process at a given rate; each is one query of
8..32 tokens (uniform) with k drawn from {10, 100, 1000} with probabilities
{0.7, 0.25, 0.05}, on the 1M-document passage-ranking index kept resident on
the GPU. Reports achieved QPS and p50/p95/p99 latency (submission to results on
the host) per rate, for the FP32 path and the BF16 tensor-core path.

    python -m paper_2604_28142_b300.serving --rates 1000 5000 10000 --seconds 5
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading
import time

import numpy as np


def run_rate(T, G, params, pool, rate, seconds, seed, n_slots, max_batch, max_wait_us):
    srv = T.Server(G, params, n_slots=n_slots, max_batch_queries=max_batch, max_batch_rows=max_batch * 32,
                   max_wait_us=max_wait_us)
    rng = np.random.default_rng(seed)
    n = max(1, int(rate * seconds))
    gaps = rng.exponential(1.0 / rate, size=n)
    pick = rng.integers(0, len(pool), size=n)
    ids = [None] * n
    t0 = time.perf_counter()
    due = t0
    for u in range(n):
        due += gaps[u]
        while True:
            now = time.perf_counter()
            if now >= due:
                break
            if due - now > 2e-4:
                time.sleep(due - now - 1e-4)
        q, k = pool[pick[u]]
        ids[u] = (srv.submit(q, k), k)
    lats = []
    for rid, k in ids:
        _, _, lat = srv.wait(rid, k, timeout_ms=120000)
        lats.append(lat)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lats = np.array(lats)
    ks = np.array([k for _, k in ids])
    by_k = {}
    for kv in sorted(set(ks.tolist())):
        m = ks == kv
        by_k[str(kv)] = {"requests": int(m.sum()), "p50_ms": float(np.percentile(lats[m], 50)),
                         "p99_ms": float(np.percentile(lats[m], 99))}
    return {"offered_qps": rate, "achieved_qps": n / wall, "requests": n,
            "p50_ms": float(np.percentile(lats, 50)), "p95_ms": float(np.percentile(lats, 95)),
            "p99_ms": float(np.percentile(lats, 99)), "batches": st["batches"], "mean_batch": st["mean_batch"],
            "by_k": by_k}


def request_pool(synth, cfg, n=4096, seed_offset=3):
    """Seeded requests: 8..32 tokens (uniform), k in {10, 100, 1000} with p = {0.7, 0.25, 0.05}."""
    q = synth.make_queries(cfg, n_queries=n, seed=cfg.query_seed + seed_offset, ntok_min=8, ntok_max=32)
    rng = np.random.default_rng(4)
    ks = rng.choice([10, 100, 1000], size=n, p=[0.7, 0.25, 0.05])
    off = np.concatenate([[0], np.cumsum(q["ntok"])])
    return [(q["queries"][off[u]:off[u + 1]], int(ks[u])) for u in range(n)]


def main():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch

    import paper_2604_28142_b300 as T
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="msmarco-1M")
    ap.add_argument("--rates", type=float, nargs="+", default=[1000, 5000, 10000, 20000, 50000])
    ap.add_argument("--seconds", type=float, default=5.0)
    ap.add_argument("--precision", nargs="+", default=["fp32", "bf16"])
    ap.add_argument("--slots", type=int, default=3)
    ap.add_argument("--max-batch", type=int, default=128)
    ap.add_argument("--max-wait-us", type=int, default=500)
    a = ap.parse_args()
    torch.cuda.set_device(0)
    ix = synth.load_or_make(a.workload, device="cuda")
    cfg = synth.CONFIGS[a.workload]
    G = T.Index(ix, 0)
    pool = request_pool(synth, cfg)
    out = []
    for prec in a.precision:
        if prec == "bf16" and not T.tc_available():
            continue
        params = T.SearchParams(kappa_c=40, kappa_d=0, precision=T.PREC_BF16 if prec == "bf16" else T.PREC_FP32)
        # warm-up: scratch of every slot grows once
        run_rate(T, G, params, pool, 2000, 0.5, 99, a.slots, a.max_batch, a.max_wait_us)
        for r in a.rates:
            res = run_rate(T, G, params, pool, r, a.seconds, int(r), a.slots, a.max_batch, a.max_wait_us)
            res["precision"] = prec
            print(json.dumps(res), flush=True)
            out.append(res)
    return out


if __name__ == "__main__":
    main()

"""Full-size parity on the two largest workloads (each generates its index on the
GPU in about three minutes and needs ~20 GB of host memory; the index is cached
on local disk for the rest of the session).

  * passage-ranking full scale: 8.8M documents, ~600M tokens, C = 2^21 bf16
    centroids, 16-byte codes, batches of 256 queries x 32 tokens, kappa_c = 40,
    kappa_d = 1000, k = 10;
  * long-tail QA shape: 2.8M documents, ~340M tokens (lengths up to 512),
    C = 2^20, 32-byte codes (32 subspaces x 4 dims), 512 queries per launch with
    8..32 tokens each, packed without padding.
Both run the BF16 tensor-core path in the benchmark's launch configuration and
check a sample of queries against the FP64 oracle.
"""
import os

import numpy as np
import pytest

import synth
from compare import check_ranking, overlap

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.skipif(os.environ.get("TACHIOM_SKIP_LARGE") == "1",
                                                  reason="large workloads skipped (TACHIOM_SKIP_LARGE=1)")]


@pytest.mark.parametrize("name,batch,lo,hi", [("msmarco-8.8M", 256, 32, 32), ("lotte-2.8M", 512, 8, 32)])
def test_large_workload_sampled(name, batch, lo, hi):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_28142_b300 as T
    from oracle import Oracle
    ix = synth.load_or_make(name, device="cuda")
    cfg = synth.CONFIGS[name]
    q = synth.make_queries(cfg, n_queries=batch, seed=cfg.query_seed + 5, ntok_min=lo, ntok_max=hi)
    G = T.Index(ix, 0)
    k, kc, kd = 10, 40, 1000
    nq = len(q["ntok"])
    dq = torch.from_numpy(q["queries"]).cuda()
    oi = torch.empty(nq * k, dtype=torch.int32, device="cuda")
    os_ = torch.empty(nq * k, dtype=torch.float32, device="cuda")
    prec = T.PREC_BF16 if T.tc_available() else T.PREC_FP32
    kk = np.full(nq, k, np.int32)
    params = T.SearchParams(kappa_c=kc, kappa_d=kd, precision=prec)
    G.search(params, dq, q["ntok"], kk, oi, os_)
    torch.cuda.synchronize()
    assert G.stream_status() & ~3 == 0
    gi, gs = oi.cpu().numpy(), os_.cpu().numpy()
    # the launch configuration's time, for the record
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        G.search(params, dq, q["ntok"], kk, oi, os_)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 3
    print(f"\n{name}: batch {nq}, {ms:.2f} ms per batch, {nq / ms * 1e3:.0f} queries/s")
    if prec == T.PREC_BF16:
        # the reduced-precision path returns the FP32 path's results bit for bit
        fi = torch.empty_like(oi)
        fs = torch.empty_like(os_)
        G.search(T.SearchParams(kappa_c=kc, kappa_d=kd, precision=T.PREC_FP32), dq, q["ntok"], kk, fi, fs)
        torch.cuda.synchronize()
        assert np.array_equal(fi.cpu().numpy(), gi)
        assert np.array_equal(fs.cpu().numpy(), gs)
    off = np.concatenate([[0], np.cumsum(q["ntok"])])
    sample = [0, nq // 2, nq - 1]
    rows = np.concatenate([np.arange(off[u], off[u + 1]) for u in sample])
    O = Oracle(ix)
    res = O.search(q["queries"][rows], q["ntok"][sample], k, kc, kd)
    ov = []
    for j, u in enumerate(sample):
        sl = slice(u * k, (u + 1) * k)
        check_ranking(gi[sl], gs[sl], res["ids"][j * k:(j + 1) * k], res["scores"][j * k:(j + 1) * k], 1e-5, 1e-4,
                      what=f"{name} query {u}")
        ov.append(overlap(gi[sl], res["ids"][j * k:(j + 1) * k]))
    assert np.mean(ov) >= 0.99

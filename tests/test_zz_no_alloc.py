"""tachiom_refine_noalloc: the allocation-free variant of the refine step.

It exists for callers that cannot allocate device memory during a call (a
fixed-budget allocator that owns all device memory, a plug-in inside another
framework's pool, a thread that must not block in cudaMalloc). Its scratch is
a static device array inside the library, so its results must equal those of
tachiom_refine, which takes scratch from a cudaMalloc-grown workspace. The
check runs two calls in a row (the second on different queries and
candidates) so that contents left in the shared array by one call cannot
leak into the next. This file is collected last on purpose.
"""
import ctypes as ct

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _call(G, name, params, dq, ntok, k, cand, oi, os_):
    from paper_2604_28142_b300 import binding as B
    L = B.lib()
    ntok = np.ascontiguousarray(ntok, np.int32)
    k = np.ascontiguousarray(k, np.int32)
    st = getattr(L, name)(G.h, ct.byref(params), B._dp(dq), B._hp(ntok), B._hp(k), int(len(ntok)),
                          B._dp(cand), B._dp(oi), B._dp(os_), B._stream(None))
    if st != 0:
        raise B.TachiomError(st, L.tachiom_last_error().decode())


def _compare(T, G, n_docs, kd, qs, rng):
    """tachiom_refine and tachiom_refine_noalloc on the same inputs, one call per query set."""
    for call, q in enumerate(qs):
        nq = len(q["ntok"])
        k = rng.integers(1, 50, size=nq).astype(np.int32)
        cand = np.full((nq, kd), -1, np.int32)
        for u in range(nq):
            n = int(rng.integers(1, kd + 1)) if call % 2 == 0 else kd
            cand[u, :n] = rng.choice(n_docs, size=n, replace=False)
        dq = torch.from_numpy(q["queries"]).cuda()
        dc = torch.from_numpy(cand).cuda()
        tot = int(k.sum())
        p = T.SearchParams(kappa_c=8, kappa_d=kd, precision=T.PREC_FP32)
        ref_i = torch.full((tot,), -7, dtype=torch.int32, device="cuda")
        ref_s = torch.zeros(tot, dtype=torch.float32, device="cuda")
        got_i = torch.full((tot,), -7, dtype=torch.int32, device="cuda")
        got_s = torch.zeros(tot, dtype=torch.float32, device="cuda")
        _call(G, "tachiom_refine", p, dq, q["ntok"], k, dc, ref_i, ref_s)
        _call(G, "tachiom_refine_noalloc", p, dq, q["ntok"], k, dc, got_i, got_s)
        torch.cuda.synchronize()
        ri, rs = ref_i.cpu().numpy(), ref_s.cpu().numpy()
        gi, gs = got_i.cpu().numpy(), got_s.cpu().numpy()
        assert np.array_equal(ri, gi), f"call {call}: ids differ"
        fin = np.isfinite(rs)
        assert np.array_equal(fin, np.isfinite(gs))
        assert np.allclose(gs[fin], rs[fin], rtol=1e-5, atol=0), f"call {call}: scores differ"


@pytest.mark.parametrize("pq_m", [8, 16, 32])
def test_noalloc_refine_matches_refine_every_pq_m(pq_m):
    # pq_m = 32 uses all 8 query-token groups of the partial-sum region
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_28142_b300 as T
    ix = synth.random_index(1500, 700, pq_m=pq_m, len_min=1, len_max=50, seed=50 + pq_m, empty_docs=5)
    G = T.Index(ix, 0)
    rng = np.random.default_rng(60 + pq_m)
    _compare(T, G, 1500, 500, [synth.random_queries(23, 1, 32, seed=70 + pq_m),
                               synth.random_queries(41, 1, 32, seed=80 + pq_m)], rng)


def test_noalloc_refine_at_the_static_maximum():
    # 64 queries of 32 tokens, kappa_d = 1024, pq_m = 32: every byte of the static array in use
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_28142_b300 as T
    ix = synth.random_index(3000, 800, pq_m=32, len_min=1, len_max=40, seed=91)
    G = T.Index(ix, 0)
    rng = np.random.default_rng(92)
    _compare(T, G, 3000, 1024, [synth.random_queries(64, 32, 32, seed=93), synth.random_queries(64, 32, 32, seed=94)],
             rng)


def test_noalloc_status_reports_an_out_of_range_id():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_28142_b300 as T
    from paper_2604_28142_b300 import binding as B
    ix = synth.random_index(300, 100, seed=95)
    G = T.Index(ix, 0)
    q = synth.random_queries(2, 4, 8, seed=96)
    dq = torch.from_numpy(q["queries"]).cuda()
    cand = np.array([[5, 7, 300, -1], [1, 2, 3, 4]], np.int32)  # id 300 is out of [0, 300)
    dc = torch.from_numpy(cand).cuda()
    oi = torch.empty(4, dtype=torch.int32, device="cuda")
    os_ = torch.empty(4, dtype=torch.float32, device="cuda")
    fl = ct.c_uint32(0)
    assert B.lib().tachiom_refine_noalloc_status(G.h, None, ct.byref(fl)) == 0  # clear
    _call(G, "tachiom_refine_noalloc", T.SearchParams(kappa_c=4, kappa_d=4), dq, q["ntok"], np.array([2, 2], np.int32),
          dc, oi, os_)
    assert B.lib().tachiom_refine_noalloc_status(G.h, None, ct.byref(fl)) == 0
    assert fl.value & T.binding.FLAG_BAD_INPUT
    # read and cleared: a clean call leaves it at zero
    dc2 = torch.from_numpy(np.array([[5, 7, 9, -1], [1, 2, 3, 4]], np.int32)).cuda()
    _call(G, "tachiom_refine_noalloc", T.SearchParams(kappa_c=4, kappa_d=4), dq, q["ntok"], np.array([2, 2], np.int32),
          dc2, oi, os_)
    assert B.lib().tachiom_refine_noalloc_status(G.h, None, ct.byref(fl)) == 0
    assert fl.value == 0


def test_noalloc_refine_matches_refine_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_28142_b300 as T
    ix = synth.random_index(2500, 900, len_min=1, len_max=60, seed=41, empty_docs=7)
    G = T.Index(ix, 0)
    kd = 700
    rng = np.random.default_rng(42)
    for call in range(2):
        q = synth.random_queries(37 if call == 0 else 64, 1, 32, seed=43 + call)
        nq = len(q["ntok"])
        k = rng.integers(1, 50, size=nq).astype(np.int32)
        cand = np.full((nq, kd), -1, np.int32)
        for u in range(nq):
            n = int(rng.integers(1, kd + 1))
            cand[u, :n] = rng.choice(2500, size=n, replace=False)
        dq = torch.from_numpy(q["queries"]).cuda()
        dc = torch.from_numpy(cand).cuda()
        tot = int(k.sum())
        p = T.SearchParams(kappa_c=8, kappa_d=kd, precision=T.PREC_FP32)
        ref_i = torch.full((tot,), -7, dtype=torch.int32, device="cuda")
        ref_s = torch.zeros(tot, dtype=torch.float32, device="cuda")
        got_i = torch.full((tot,), -7, dtype=torch.int32, device="cuda")
        got_s = torch.zeros(tot, dtype=torch.float32, device="cuda")
        _call(G, "tachiom_refine", p, dq, q["ntok"], k, dc, ref_i, ref_s)
        _call(G, "tachiom_refine_noalloc", p, dq, q["ntok"], k, dc, got_i, got_s)
        torch.cuda.synchronize()
        ri, rs = ref_i.cpu().numpy(), ref_s.cpu().numpy()
        gi, gs = got_i.cpu().numpy(), got_s.cpu().numpy()
        assert np.array_equal(ri, gi), f"call {call}: ids differ"
        fin = np.isfinite(rs)
        assert np.array_equal(fin, np.isfinite(gs))
        assert np.allclose(gs[fin], rs[fin], rtol=1e-5, atol=0), f"call {call}: scores differ"


def test_noalloc_rejects_sizes_beyond_the_static_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_28142_b300 as T
    ix = synth.random_index(50, 40, seed=44)
    G = T.Index(ix, 0)
    q = synth.random_queries(65, 1, 4, seed=45)
    dq = torch.from_numpy(q["queries"]).cuda()
    dc = torch.zeros((65, 10), dtype=torch.int32, device="cuda")
    oi = torch.empty(65, dtype=torch.int32, device="cuda")
    os_ = torch.empty(65, dtype=torch.float32, device="cuda")
    with pytest.raises(T.TachiomError, match="static maximum"):
        _call(G, "tachiom_refine_noalloc", T.SearchParams(kappa_c=4, kappa_d=10), dq, q["ntok"],
              np.ones(65, np.int32), dc, oi, os_)
    with pytest.raises(T.TachiomError, match="static maximum"):
        _call(G, "tachiom_refine_noalloc", T.SearchParams(kappa_c=4, kappa_d=2000), dq[:4], q["ntok"][:1],
              np.ones(1, np.int32), dc, oi, os_)

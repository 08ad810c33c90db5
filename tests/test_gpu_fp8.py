"""FP8-E4M3 step (a) (needs a GPU with the tensor-core path).

The E4M3 path scales every query row and every centroid by a power of two,
multiplies E4M3 x E4M3 on the tensor cores with FP32 accumulation, and repairs
the candidates in a window of rescore_margin times the rigorous error bound in
FP32. Checked here:
  * every E4M3 tensor-core score is within the rigorous per-row bound (FP64
    reference), and the bound is not vacuous;
  * with rescore_margin = 1 (the rigorous window) step (a) and the whole search
    return the FP32 path's results bit for bit;
  * with the default window (0.1 of the bound) the search meets the reduced-
    precision rule against the FP64 oracle: top-10 overlap >= 0.99 and the
    scores of the returned documents within 2e-3 (relative) of the oracle's.
"""
import numpy as np
import pytest

from compare import overlap
from test_gpu_parity import CASES, _cuda, _search, _tc, _widened, get_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_REDUCED = 2e-3


def _e4m3_rows(x):
    """Reference E4M3 rounding with the library's power-of-two row scales (torch's float8 cast)."""
    x = np.asarray(x, np.float64)
    amax = np.abs(x).max(axis=1)
    s = np.zeros(len(x))
    nz = amax > 0
    s[nz] = np.floor(np.log2(448.0 / amax[nz]))
    sc = np.exp2(s)[:, None]
    y = torch.from_numpy((x * sc).astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    return y / sc


@pytest.mark.parametrize("name", ["tiny", "small", "random_edges"])
def test_fp8_scores_within_error_bound(name):
    _cuda()
    _tc()
    c = get_case(name)
    R = min(c.q.shape[0], 300)
    C = c.G.C
    out = torch.empty((R, C), dtype=torch.float32, device="cuda")
    mg = torch.empty(R, dtype=torch.float32, device="cuda")
    c.G.debug_tc_scores_fp8(c.dq[:R], out, mg)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    Cw = _widened(c.ix)
    exact = c.q[:R].astype(np.float64) @ Cw.T
    err = np.abs(got - exact)
    delta = mg.cpu().numpy().astype(np.float64) / 2  # the rigorous bound (margin = 2 delta at lambda 1)
    assert np.all(err.max(axis=1) <= delta), (err.max(axis=1) / delta).max()
    assert (err.max(axis=1) / delta).max() > 0.05  # not loose by orders of magnitude
    # the same products from the E4M3 rounding of both operands (the library's scales), in FP64:
    # the tensor cores add exact products, so only the FP32 accumulation separates them
    ref = _e4m3_rows(c.q[:R]) @ _e4m3_rows(Cw).T
    assert np.abs(got - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max()), np.abs(got - ref).max()
    assert c.G.stream_status() == 0


@pytest.mark.parametrize("name", CASES)
def test_fp8_rigorous_window_equals_fp32(name):
    # rescore_margin = 1: the window is the rigorous bound, so the result is the FP32 path's
    _cuda()
    _tc()
    import paper_2604_28142_b300 as T
    c = get_case(name)
    R = c.q.shape[0]
    res = []
    for prec, lam in ((T.PREC_FP32, 0.0), (T.PREC_FP8, 1.0)):
        p = T.SearchParams(kappa_c=c.kc, kappa_d=c.kd, precision=prec, rescore_margin=lam)
        ids = torch.empty((R, c.kc), dtype=torch.int32, device="cuda")
        sc = torch.empty((R, c.kc), dtype=torch.float32, device="cuda")
        c.G.top_centroids(p, c.dq, ids, sc)
        torch.cuda.synchronize()
        res.append((ids.cpu().numpy(), sc.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1].view(np.int32), res[1][1].view(np.int32))
    assert c.G.stream_status() & 16 == 0  # no timeout
    # and the whole search
    kk = np.full(c.nq, c.k, np.int32)
    outs = []
    for prec, lam in ((T.PREC_FP32, 0.0), (T.PREC_FP8, 1.0)):
        oi = torch.empty(int(kk.sum()), dtype=torch.int32, device="cuda")
        os_ = torch.empty(int(kk.sum()), dtype=torch.float32, device="cuda")
        c.G.search(T.SearchParams(kappa_c=c.kc, kappa_d=c.kd, precision=prec, rescore_margin=lam), c.dq, c.ntok, kk,
                   oi, os_)
        torch.cuda.synchronize()
        outs.append((oi.cpu().numpy(), os_.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1].view(np.int32), outs[1][1].view(np.int32))


@pytest.mark.parametrize("name", ["tiny", "small", "small32", "random_edges"])
def test_fp8_default_window_against_oracle(name):
    _cuda()
    _tc()
    import paper_2604_28142_b300 as T
    c = get_case(name)
    kk = np.full(c.nq, c.k, np.int32)
    oi = torch.empty(int(kk.sum()), dtype=torch.int32, device="cuda")
    os_ = torch.empty(int(kk.sum()), dtype=torch.float32, device="cuda")
    c.G.search(T.SearchParams(kappa_c=c.kc, kappa_d=c.kd, precision=T.PREC_FP8), c.dq, c.ntok, kk, oi, os_)
    torch.cuda.synchronize()
    gi, gs = oi.cpu().numpy(), os_.cpu().numpy().astype(np.float64)
    res = c.O.search(c.q, c.ntok, c.k, c.kc, c.kd)
    ov = []
    for u in range(c.nq):
        sl = slice(u * c.k, (u + 1) * c.k)
        o_ids, o_s = res["ids"][sl], res["scores"][sl]
        ov.append(overlap(gi[sl], o_ids, 10))
        # rank by rank, the scores agree within the reduced-precision tolerance
        m = o_ids >= 0
        assert np.array_equal(m, gi[sl] >= 0)
        assert np.all(np.abs(gs[sl][m] - o_s[m]) <= RTOL_REDUCED * np.maximum(1, np.abs(o_s[m]))), u
    assert np.mean(ov) >= 0.99, ov
    assert c.G.stream_status() & ~0b11 == 0


def test_fp8_equals_bf16_path_results_at_rigorous_window():
    # the two reduced precisions, both with rigorous windows, give the same bits
    _cuda()
    _tc()
    import paper_2604_28142_b300 as T
    c = get_case("small")
    a = _search(c, prec=T.PREC_BF16)
    kk = np.full(c.nq, c.k, np.int32)
    oi = torch.empty(int(kk.sum()), dtype=torch.int32, device="cuda")
    os_ = torch.empty(int(kk.sum()), dtype=torch.float32, device="cuda")
    c.G.search(T.SearchParams(kappa_c=c.kc, kappa_d=c.kd, precision=T.PREC_FP8, rescore_margin=1.0), c.dq, c.ntok,
               kk, oi, os_)
    torch.cuda.synchronize()
    assert np.array_equal(a[0], oi.cpu().numpy())
    assert np.array_equal(a[1].view(np.int32), os_.cpu().numpy().view(np.int32))

"""The exhaustive reference and the candidate-budget autotuner (needs a GPU).

tachiom_exhaustive_topk scores every document with the refine of step (c), so its
top-k must be the oracle's cascade with kappa_c = C and kappa_d = D (exhaustive
PQ-MaxSim, brute force over every document). tachiom_autotune_budgets must return
a point of the grid whose recall against that reference meets the target, the
fastest such point by its own timing table.
"""
import numpy as np
import pytest

from compare import check_ranking
from test_gpu_parity import _cuda, get_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_exhaustive_topk_is_the_oracles_exhaustive_cascade(prec):
    _cuda()
    import paper_2604_28142_b300 as T
    if prec == 1 and not T.tc_available():
        pytest.skip("no tensor-core path")
    c = get_case("tiny")
    k = 10
    ids, sc = c.G.exhaustive_topk(prec, c.dq, c.ntok, k)
    D = c.ix["doc_offsets"].shape[0] - 1
    C = c.ix["centroids"].shape[0]
    res = c.O.search(c.q, c.ntok, k, C, D)
    for u in range(c.nq):
        sl = slice(u * k, (u + 1) * k)
        check_ranking(ids[u], sc[u], res["ids"][sl], res["scores"][sl], 1e-5, 1e-4, what=f"query {u}")


def test_autotune_budgets_returns_the_fastest_point_meeting_the_target():
    _cuda()
    import paper_2604_28142_b300 as T
    c = get_case("small")
    prec = T.PREC_BF16 if T.tc_available() else T.PREC_FP32
    gc, gd = [5, 20, 40], [100, 400, 1000]
    (kc, kd), rec, ms, table = c.G.autotune_budgets(prec, c.dq, c.ntok, 10, gc, gd, min_recall=0.9)
    assert kc in gc and kd in gd
    t = table.reshape(-1, 4)
    assert np.all(np.isfinite(t)) and np.all(t[:, 3] > 0) and np.all((t[:, 2] >= 0) & (t[:, 2] <= 1))
    row = t[(t[:, 0] == kc) & (t[:, 1] == kd)][0]
    assert row[2] == pytest.approx(rec) and row[3] == pytest.approx(ms)
    ok = t[t[:, 2] >= 0.9]
    if len(ok):
        assert rec >= 0.9 and ms == pytest.approx(ok[:, 3].min())
    else:
        assert rec == pytest.approx(t[:, 2].max())
    # recall grows with the budgets: the largest point reaches at least the smallest's recall
    assert t[-1, 2] >= t[0, 2]

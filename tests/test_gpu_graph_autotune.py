"""CUDA-graph replay and the autotuner (needs a GPU): a captured batch and every
plan the autotuner can pick return the same bits as the default search."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_28142_b300 as T
    ix = synth.load_or_make("small", device="cuda")
    cfg = synth.CONFIGS["small"]
    q = synth.make_queries(cfg, n_queries=20, seed=55, ntok_min=8, ntok_max=32)
    return T, T.Index(ix, 0), q


def _run(T, G, params, q, kk, plan=-1):
    p = T.SearchParams(kappa_c=params.kappa_c, kappa_d=params.kappa_d, precision=params.precision, plan_id=plan)
    dq = torch.from_numpy(q["queries"]).cuda()
    oi = torch.empty(int(kk.sum()), dtype=torch.int32, device="cuda")
    os_ = torch.empty(int(kk.sum()), dtype=torch.float32, device="cuda")
    G.search(p, dq, q["ntok"], kk, oi, os_)
    torch.cuda.synchronize()
    return oi.cpu().numpy(), os_.cpu().numpy().view(np.int32)


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_equals_search(env, prec):
    T, G, q = env
    if prec == 1 and not T.tc_available():
        pytest.skip("no tensor-core path")
    params = T.SearchParams(kappa_c=40, kappa_d=1000, precision=prec)
    kk = np.full(len(q["ntok"]), 10, np.int32)
    want = _run(T, G, params, q, kk)
    g = G.graph(params, q["ntok"], kk)
    for rep in range(3):
        dq = torch.from_numpy(q["queries"]).cuda()
        oi = torch.full((int(kk.sum()),), -5, dtype=torch.int32, device="cuda")
        os_ = torch.zeros(int(kk.sum()), dtype=torch.float32, device="cuda")
        g.launch(dq, oi, os_)
        torch.cuda.synchronize()
        assert np.array_equal(oi.cpu().numpy(), want[0])
        assert np.array_equal(os_.cpu().numpy().view(np.int32), want[1])
    g.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_every_plan_gives_the_same_results(env, prec):
    T, G, q = env
    if prec == 1 and not T.tc_available():
        pytest.skip("no tensor-core path")
    params = T.SearchParams(kappa_c=40, kappa_d=1000, precision=prec)
    kk = np.full(len(q["ntok"]), 100, np.int32)
    want = _run(T, G, params, q, kk)
    dq = torch.from_numpy(q["queries"]).cuda()
    best, ms = G.autotune(params, dq, q["ntok"], kk)
    assert best >= 0 and ms > 0
    tok = 1 << 24  # every gather range cut into small pieces
    win_all = 1 << 25  # the FP32 window over every pair
    groups = [g << 26 for g in (1, 2, 7)]  # 2 g gather range groups per query
    plans = ([1 | 4, 1 | 8, 2 | 4, 2 | 8, 3 | 8, 2 | 12 | tok, 2 | 12 | win_all] + [2 | 12 | g for g in groups]
             if prec == 1 else [3 | 8 | (s << 4) for s in (1, 7, 40)] + [3 | 8 | tok] + [3 | 8 | g for g in groups])
    for pl in plans + [best]:
        got = _run(T, G, params, q, kk, plan=pl)
        assert np.array_equal(got[0], want[0]), pl
        assert np.array_equal(got[1], want[1]), pl

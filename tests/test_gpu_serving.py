"""Continuous batching (tachiom_server_*): requests of uneven token counts and k
arrive while other batches run; each result must be the same bits as the same
query searched alone, and admission must respect the scratch budget."""
import threading
import time

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
    return T, T.Index(ix, 0), ix


def _alone(T, G, params, q, k):
    dq = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    oi = torch.empty(k, dtype=torch.int32, device="cuda")
    os_ = torch.empty(k, dtype=torch.float32, device="cuda")
    G.search(params, dq, np.array([q.shape[0]], np.int32), np.array([k], np.int32), oi, os_)
    torch.cuda.synchronize()
    return oi.cpu().numpy(), os_.cpu().numpy()


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    qs = synth.random_queries(n, 8, 32, seed=seed)
    cfg = synth.CONFIGS["small"]
    real = synth.make_queries(cfg, n_queries=n, seed=seed + 1, ntok_min=8, ntok_max=32)
    ks = rng.choice([10, 100, 1000], size=n, p=[0.7, 0.25, 0.05])
    off = np.concatenate([[0], np.cumsum(real["ntok"])])
    return [(real["queries"][off[u]:off[u + 1]], int(ks[u])) for u in range(n)], qs


@pytest.mark.parametrize("prec", [0, 1])
def test_each_result_is_the_same_alone_and_in_the_mix(env, prec):
    T, G, ix = env
    if prec == 1 and not T.tc_available():
        pytest.skip("no tensor-core path")
    params = T.SearchParams(kappa_c=40, kappa_d=0, precision=prec)
    reqs, _ = _requests(60, 7)
    srv = T.Server(G, params, n_slots=3, max_batch_queries=16, max_batch_rows=512, max_wait_us=300)
    ids = {}

    def client(lo, hi, delay):
        for u in range(lo, hi):
            ids[u] = srv.submit(*reqs[u])
            time.sleep(delay)

    th = [threading.Thread(target=client, args=(i * 20, (i + 1) * 20, 0.0005 * (i + 1))) for i in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    got = {u: srv.wait(ids[u], reqs[u][1], timeout_ms=60000) for u in range(60)}
    st = srv.stats()
    srv.close()
    assert st["completed"] == 60 and st["batches"] >= 4 and st["p50_ms"] <= st["p99_ms"]
    assert st["mean_batch"] > 1.0  # requests really were batched together
    for u in range(60):
        q, k = reqs[u]
        ai, as_ = _alone(T, G, params, q, k)
        gi, gs, lat = got[u]
        assert np.array_equal(ai, gi), u
        assert np.array_equal(as_.view(np.int32), gs.view(np.int32)), u
        assert lat > 0


def test_admission_by_scratch_budget(env):
    T, G, ix = env
    params = T.SearchParams(kappa_c=20, kappa_d=500, precision=0)
    reqs, _ = _requests(24, 11)
    reqs = [(q, min(k, 100)) for q, k in reqs]  # k <= kappa_d
    # room for about one batch of 8 queries at a time
    D = ix["doc_offsets"].shape[0] - 1
    budget = 8 * D * 4 + 8 * 32 * (20 * 8 + 4096 * 8) + 8 * 500 * 64 + 8 * 16384 * 8 + 1
    srv = T.Server(G, params, n_slots=4, max_batch_queries=8, max_batch_rows=256, max_wait_us=0,
                   scratch_budget_bytes=budget)
    ids = [srv.submit(q, k) for q, k in reqs]
    got = [srv.wait(i, reqs[u][1], timeout_ms=60000) for u, i in enumerate(ids)]
    st = srv.stats()
    srv.close()
    assert st["completed"] == 24
    for u, (q, k) in enumerate(reqs):
        ai, _ = _alone(T, G, params, q, k)
        assert np.array_equal(ai, got[u][0])


def test_wait_timeout_and_bad_requests(env):
    T, G, ix = env
    params = T.SearchParams(kappa_c=20, kappa_d=500, precision=0)
    srv = T.Server(G, params, n_slots=1, max_batch_queries=4, max_batch_rows=128, max_wait_us=0)
    with pytest.raises(T.TachiomError):
        srv.submit(np.zeros((33, 128), np.float32), 10)
    with pytest.raises(T.TachiomError):
        srv.submit(np.zeros((4, 128), np.float32), 501)
    with pytest.raises(T.TachiomError):
        srv.wait(123456, 10, timeout_ms=1)
    srv.close()

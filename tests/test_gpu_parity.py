"""CUDA path against the FP64 oracle, stage by stage and end to end (needs a GPU).

Stages are replayed: each GPU stage runs on the oracle's own upstream result,
so a near-tie upstream cannot hide or fake a bug downstream. Rankings are
compared with the gap-aware rules of tests/compare.py. Tolerance: scores of
the FP32 path within 1e-5 relative to the oracle (FP32 dot products of
128-term unit vectors are accurate to ~1e-7; S sums at most 32 of them).
"""
import numpy as np
import pytest

import synth
from compare import check_ranking, overlap

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_FP32 = 1e-5
GAP = 1e-4


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


class Case:
    def __init__(self, name, ix, q, kc, kd, k):
        import paper_2604_28142_b300 as T
        from oracle import Oracle
        self.name, self.ix, self.kc, self.kd, self.k = name, ix, kc, kd, k
        self.q, self.ntok = q["queries"], q["ntok"]
        self.nq = len(self.ntok)
        self.qoff = np.concatenate([[0], np.cumsum(self.ntok)]).astype(np.int64)
        self.O = Oracle(ix)
        self.G = T.Index(ix, 0)
        self.T = T
        self.dq = torch.from_numpy(self.q).cuda()

    def params(self, prec=0, kd=None, kc=None, plan=-1):
        return self.T.SearchParams(kappa_c=self.kc if kc is None else kc,
                                   kappa_d=self.kd if kd is None else kd, precision=prec, plan_id=plan)


_CASES = {}


def get_case(name):
    _cuda()
    if name in _CASES:
        return _CASES[name]
    if name == "tiny":
        cfg = synth.CONFIGS["tiny"]
        ix = synth.load_or_make("tiny", device="cpu")
        q = synth.make_queries(cfg)
        c = Case(name, ix, q, cfg.kappa_c, cfg.kappa_d, cfg.k)
    elif name in ("small", "small32"):
        cfg = synth.CONFIGS[name]
        ix = synth.load_or_make(name, device="cuda")
        q = synth.make_queries(cfg)
        c = Case(name, ix, q, cfg.kappa_c, cfg.kappa_d, cfg.k)
    elif name == "random_edges":
        ix = synth.random_index(3001, 777, len_min=0, len_max=40, seed=5, empty_docs=50)
        q = synth.random_queries(9, 1, 32, seed=6)
        c = Case(name, ix, q, 7, 300, 25)
    elif name == "random_m8":
        # 8 subspaces of 16 dims: the widest codewords the decode pass takes
        ix = synth.random_index(2001, 777, pq_m=8, len_min=0, len_max=40, seed=8, empty_docs=20)
        q = synth.random_queries(9, 1, 32, seed=9)
        c = Case(name, ix, q, 7, 300, 25)
    else:
        raise KeyError(name)
    _CASES[name] = c
    return c


CASES = ["tiny", "small", "small32", "random_edges", "random_m8"]


@pytest.mark.parametrize("name", CASES)
def test_inverted_lists_bit_exact(name):
    c = get_case(name)
    o_off, o_docs = c.O.lists()
    g_off, g_docs = c.G.lists()
    assert np.array_equal(o_off, g_off)
    assert np.array_equal(o_docs, g_docs)


@pytest.mark.parametrize("name", CASES)
def test_step_a_top_centroids_fp32(name):
    c = get_case(name)
    R = c.q.shape[0]
    ids = torch.empty((R, c.kc), dtype=torch.int32, device="cuda")
    sc = torch.empty((R, c.kc), dtype=torch.float32, device="cuda")
    c.G.top_centroids(c.params(), c.dq, ids, sc)
    torch.cuda.synchronize()
    o_ids, o_s = c.O.top_centroids(c.q, c.kc)
    gi, gs = ids.cpu().numpy(), sc.cpu().numpy()
    for r in range(R):
        check_ranking(gi[r], gs[r], o_ids[r], o_s[r], RTOL_FP32, GAP, what=f"row {r}")


# plan bit 24: every document range cut into pieces of at most 256 list entries, the path the
# gather takes when a range's entries exceed its shared-memory buffers
GATHER_PLANS = [-1, 1 << 24]


@pytest.mark.parametrize("plan", GATHER_PLANS)
@pytest.mark.parametrize("name", CASES)
def test_step_b_gather_replay(name, plan):
    c = get_case(name)
    o_ids, _ = c.O.top_centroids(c.q, c.kc)
    top = torch.from_numpy(o_ids).cuda()
    cid = torch.empty((c.nq, c.kd), dtype=torch.int32, device="cuda")
    cs = torch.empty((c.nq, c.kd), dtype=torch.float32, device="cuda")
    nc = torch.empty(c.nq, dtype=torch.int32, device="cuda")
    c.G.gather(c.params(plan=plan), c.dq, c.ntok, top, cid, cs, nc)
    torch.cuda.synchronize()
    gi, gs, gn = cid.cpu().numpy(), cs.cpu().numpy(), nc.cpu().numpy()
    for u in range(c.nq):
        docs, s = c.O.gather(c.q[c.qoff[u]:c.qoff[u + 1]], o_ids[c.qoff[u]:c.qoff[u + 1]])
        od, os_ = c.O.select(docs, s, c.kd)
        want_i = np.full(c.kd, -1, np.int32)
        want_s = np.full(c.kd, -np.inf)
        want_i[:len(od)] = od
        want_s[:len(od)] = os_
        assert gn[u] == len(od)
        check_ranking(gi[u], gs[u], want_i, want_s, RTOL_FP32, GAP, what=f"query {u}",
                      exact_scores=dict(zip(docs.tolist(), s.tolist())))


@pytest.mark.parametrize("plan", GATHER_PLANS)
@pytest.mark.parametrize("name", CASES)
def test_step_b_reached_set_bit_exact(name, plan):
    # with kappa_d above the pool size the candidates are every reached doc: integer work
    c = get_case(name)
    o_ids, _ = c.O.top_centroids(c.q, c.kc)
    top = torch.from_numpy(o_ids).cuda()
    kd = 4096
    cid = torch.empty((c.nq, kd), dtype=torch.int32, device="cuda")
    cs = torch.empty((c.nq, kd), dtype=torch.float32, device="cuda")
    nc = torch.empty(c.nq, dtype=torch.int32, device="cuda")
    c.G.gather(c.params(kd=kd, plan=plan), c.dq, c.ntok, top, cid, cs, nc)
    torch.cuda.synchronize()
    gi, gn = cid.cpu().numpy(), nc.cpu().numpy()
    checked = 0
    for u in range(c.nq):
        docs, _ = c.O.gather(c.q[c.qoff[u]:c.qoff[u + 1]], o_ids[c.qoff[u]:c.qoff[u + 1]])
        if len(docs) > kd:
            continue
        checked += 1
        assert gn[u] == len(docs)
        assert np.array_equal(np.sort(gi[u][:gn[u]]), docs)
        assert np.all(gi[u][gn[u]:] == -1)
    assert checked > 0 or name in ("small", "small32")


@pytest.mark.parametrize("name", CASES)
def test_step_cd_refine_replay(name):
    c = get_case(name)
    res = c.O.search(c.q, c.ntok, c.k, c.kc, c.kd, stages=True)
    cand = torch.from_numpy(np.ascontiguousarray(res["cand_ids"])).cuda()
    kk = np.full(c.nq, c.k, np.int32)
    oi = torch.empty(c.nq * c.k, dtype=torch.int32, device="cuda")
    os_ = torch.empty(c.nq * c.k, dtype=torch.float32, device="cuda")
    c.G.refine(c.params(), c.dq, c.ntok, kk, cand, oi, os_)
    torch.cuda.synchronize()
    gi, gs = oi.cpu().numpy(), os_.cpu().numpy()
    for u in range(c.nq):
        sl = slice(u * c.k, (u + 1) * c.k)
        cd = res["cand_ids"][u]
        cd = cd[cd >= 0]
        rs = c.O.refine(c.q[c.qoff[u]:c.qoff[u + 1]], cd)
        check_ranking(gi[sl], gs[sl], res["ids"][sl], res["scores"][sl], RTOL_FP32, GAP,
                      what=f"query {u}", exact_scores=dict(zip(cd.tolist(), rs.tolist())))


def _external_lists(c, seed):
    """Seeded candidate lists from outside the cascade: per query a random count of distinct
    document ids in random order, the unused slots (-1) scattered among them."""
    D = c.ix["doc_offsets"].shape[0] - 1
    kd = min(c.kd, D)
    rng = np.random.default_rng(seed)
    cand = np.full((c.nq, kd), -1, np.int32)
    for u in range(c.nq):
        n = int(rng.integers(kd // 2, kd + 1))
        cand[u, :n] = rng.choice(D, size=n, replace=False)
        rng.shuffle(cand[u])
    return cand


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["small", "small32", "random_edges", "random_m8"])
def test_rerank_external_lists(name, prec):
    # refine alone over lists it did not produce (the rerank-only use of steps c-d): the
    # result is the exact top-k of each list, FP32 and reduced precision alike
    c = get_case(name)
    cand = _external_lists(c, seed=77)
    kd = cand.shape[1]
    kk = np.full(c.nq, c.k, np.int32)
    oi = torch.empty(c.nq * c.k, dtype=torch.int32, device="cuda")
    os_ = torch.empty(c.nq * c.k, dtype=torch.float32, device="cuda")
    c.G.refine(c.params(prec, kd=kd), c.dq, c.ntok, kk, torch.from_numpy(cand).cuda(), oi, os_)
    torch.cuda.synchronize()
    gi, gs = oi.cpu().numpy(), os_.cpu().numpy()
    for u in range(c.nq):
        cd = cand[u][cand[u] >= 0]
        rs = c.O.refine(c.q[c.qoff[u]:c.qoff[u + 1]], cd)
        order = np.lexsort((cd, -rs))[:c.k]
        want_i = np.full(c.k, -1, np.int32)
        want_s = np.full(c.k, -np.inf)
        want_i[:len(order)], want_s[:len(order)] = cd[order], rs[order]
        sl = slice(u * c.k, (u + 1) * c.k)
        check_ranking(gi[sl], gs[sl], want_i, want_s, RTOL_FP32, GAP, what=f"query {u}",
                      exact_scores=dict(zip(cd.tolist(), rs.tolist())))


@pytest.mark.parametrize("name", ["small", "small32", "random_edges", "random_m8"])
def test_centroid_interaction_of_lists(name):
    # the full centroid interaction of given lists: the oracle's refine of the same index with every
    # residual norm zero (a pin fixes that identity), then the exact top-k of each list
    c = get_case(name)
    cand = _external_lists(c, seed=91)
    kd = cand.shape[1]
    kk = np.full(c.nq, c.k, np.int32)
    oi = torch.empty(c.nq * c.k, dtype=torch.int32, device="cuda")
    os_ = torch.empty(c.nq * c.k, dtype=torch.float32, device="cuda")
    c.G.centroid_interaction(c.params(1, kd=kd), c.dq, c.ntok, kk, torch.from_numpy(cand).cuda(), oi, os_)
    torch.cuda.synchronize()
    gi, gs = oi.cpu().numpy(), os_.cpu().numpy()
    from oracle import Oracle
    ix0 = dict(c.ix)
    ix0["residual_norms"] = np.zeros(c.ix["token_centroid"].shape[0], np.uint16)
    O0 = Oracle(ix0)
    for u in range(c.nq):
        cd = cand[u][cand[u] >= 0]
        rs = O0.refine(c.q[c.qoff[u]:c.qoff[u + 1]], cd)
        order = np.lexsort((cd, -rs))[:c.k]
        want_i = np.full(c.k, -1, np.int32)
        want_s = np.full(c.k, -np.inf)
        want_i[:len(order)], want_s[:len(order)] = cd[order], rs[order]
        sl = slice(u * c.k, (u + 1) * c.k)
        check_ranking(gi[sl], gs[sl], want_i, want_s, RTOL_FP32, GAP, what=f"query {u}",
                      exact_scores=dict(zip(cd.tolist(), rs.tolist())))
    assert c.G.stream_status() & (4 | 8 | 16) == 0


def _search(c, prec=0, kk=None):
    kk = np.full(c.nq, c.k, np.int32) if kk is None else kk
    tot = int(kk.sum())
    oi = torch.empty(tot, dtype=torch.int32, device="cuda")
    os_ = torch.empty(tot, dtype=torch.float32, device="cuda")
    c.G.search(c.params(prec), c.dq, c.ntok, kk, oi, os_)
    torch.cuda.synchronize()
    return oi.cpu().numpy(), os_.cpu().numpy()


@pytest.mark.parametrize("name", CASES)
def test_search_end_to_end_fp32(name):
    c = get_case(name)
    gi, gs = _search(c)
    res = c.O.search(c.q, c.ntok, c.k, c.kc, c.kd)
    ov = []
    for u in range(c.nq):
        sl = slice(u * c.k, (u + 1) * c.k)
        check_ranking(gi[sl], gs[sl], res["ids"][sl], res["scores"][sl], RTOL_FP32, GAP, what=f"query {u}")
        ov.append(overlap(gi[sl], res["ids"][sl], 10))
    assert np.mean(ov) >= 0.99, ov
    assert c.G.stream_status() & ~0b11 == 0


@pytest.mark.parametrize("name", ["tiny", "random_edges"])
def test_search_deterministic_and_batch_invariant(name):
    c = get_case(name)
    a = _search(c)
    b = _search(c)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.int32), b[1].view(np.int32))
    # each query alone gives the same bits as inside the batch
    for u in range(0, c.nq, 3):
        qq = torch.from_numpy(c.q[c.qoff[u]:c.qoff[u + 1]]).cuda()
        oi = torch.empty(c.k, dtype=torch.int32, device="cuda")
        os_ = torch.empty(c.k, dtype=torch.float32, device="cuda")
        c.G.search(c.params(), qq, c.ntok[u:u + 1], np.array([c.k], np.int32), oi, os_)
        torch.cuda.synchronize()
        sl = slice(u * c.k, (u + 1) * c.k)
        assert np.array_equal(oi.cpu().numpy(), a[0][sl])
        assert np.array_equal(os_.cpu().numpy().view(np.int32), a[1][sl].view(np.int32))


def test_search_host_matches_device():
    c = get_case("tiny")
    gi, gs = _search(c)
    hi, hs = c.G.search_host(c.params(), c.q, c.ntok, np.full(c.nq, c.k, np.int32))
    assert np.array_equal(gi, hi) and np.array_equal(gs, hs)


def test_uneven_k_and_padding():
    c = get_case("random_edges")
    kk = np.array([1, 300, 5, 17, 2, 300, 40, 9, 299], np.int32)
    gi, gs = _search(c, kk=kk)
    res = c.O.search(c.q, c.ntok, kk, c.kc, c.kd)
    off = np.concatenate([[0], np.cumsum(kk)])
    for u in range(c.nq):
        sl = slice(off[u], off[u + 1])
        check_ranking(gi[sl], gs[sl], res["ids"][sl], res["scores"][sl], RTOL_FP32, GAP, what=f"query {u}")


def test_all_centroids_and_tiny_kappa():
    c = get_case("random_edges")
    # kappa_c = 128 on C = 777, kappa_d = 1
    kc, kd, k = 128, 1, 1
    tot = c.nq * k
    oi = torch.empty(tot, dtype=torch.int32, device="cuda")
    os_ = torch.empty(tot, dtype=torch.float32, device="cuda")
    c.G.search(c.params(kc=kc, kd=kd), c.dq, c.ntok, np.full(c.nq, k, np.int32), oi, os_)
    torch.cuda.synchronize()
    res = c.O.search(c.q, c.ntok, k, kc, kd)
    check_ranking(oi.cpu().numpy(), os_.cpu().numpy(), res["ids"], res["scores"], RTOL_FP32, GAP)


def test_empty_batch_is_noop():
    c = get_case("tiny")
    c.G.search(c.params(), c.dq, np.zeros(0, np.int32), np.zeros(0, np.int32), None, None)


def test_bad_arguments_rejected():
    import paper_2604_28142_b300 as T
    c = get_case("tiny")
    oi = torch.empty(16, dtype=torch.int32, device="cuda")
    os_ = torch.empty(16, dtype=torch.float32, device="cuda")
    with pytest.raises(T.TachiomError):
        c.G.search(c.params(), c.dq, np.array([33], np.int32), np.array([1], np.int32), oi, os_)
    with pytest.raises(T.TachiomError):
        c.G.search(c.params(kc=0), c.dq, np.array([3], np.int32), np.array([1], np.int32), oi, os_)
    with pytest.raises(T.TachiomError):
        c.G.search(c.params(kd=5), c.dq, np.array([3], np.int32), np.array([6], np.int32), oi, os_)


# ---------------------------------------------------------------- tensor-core step (a)

def _tc():
    import paper_2604_28142_b300 as T
    if not T.tc_available():
        pytest.skip("no tensor-core step (a) on this device")


def _widened(ix):
    c = ix["centroids"]
    if ix["centroid_dtype"] == "bf16":
        return (c.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return c.astype(np.float64)


@pytest.mark.parametrize("name", ["tiny", "small", "random_edges"])
def test_tc_scores_within_error_bound(name):
    # every BF16 tensor-core score is within the delta the FP32 repair assumes
    _cuda()
    _tc()
    c = get_case(name)
    R = min(c.q.shape[0], 300)
    C = c.G.C
    out = torch.empty((R, C), dtype=torch.float32, device="cuda")
    c.G.debug_tc_scores(c.dq[:R], out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    Cw = _widened(c.ix)
    exact = c.q[:R].astype(np.float64) @ Cw.T
    cmax = np.linalg.norm(Cw, axis=1).max()
    rel = 2.0 ** -8 if c.ix["centroid_dtype"] == "bf16" else 2.0 ** -7
    delta = rel * cmax + 1e-5
    err = np.abs(got - exact)
    assert err.max() <= delta, (err.max(), delta)
    # and the bound is not vacuous: the scores do carry BF16 rounding error
    assert err.max() > 0
    # the per-row bound the repair window uses: ||e|| cmax + ||q_hat|| (cerr + 2^-15 cmax),
    # e = bf16(q) - q, cerr = max ||bf16(c) - c|| (Cauchy-Schwarz)
    qh = torch.from_numpy(c.q[:R]).to(torch.bfloat16).to(torch.float64).numpy()
    e = qh - c.q[:R].astype(np.float64)
    cb = torch.from_numpy(Cw.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    cerr = np.linalg.norm(cb - Cw, axis=1).max()
    drow = np.linalg.norm(e, axis=1) * cmax + np.linalg.norm(qh, axis=1) * (cerr + 2.0 ** -15 * cmax)
    assert np.all(err.max(axis=1) <= drow), (err.max(axis=1) / drow).max()
    assert (err.max(axis=1) / drow).max() > 0.05  # and it is not loose by orders of magnitude
    assert c.G.stream_status() == 0


@pytest.mark.parametrize("name", CASES)
def test_step_a_bf16_equals_fp32(name):
    _cuda()
    _tc()
    c = get_case(name)
    R = c.q.shape[0]
    res = []
    for prec in (0, 1):
        ids = torch.empty((R, c.kc), dtype=torch.int32, device="cuda")
        sc = torch.empty((R, c.kc), dtype=torch.float32, device="cuda")
        c.G.top_centroids(c.params(prec), c.dq, ids, sc)
        torch.cuda.synchronize()
        res.append((ids.cpu().numpy(), sc.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1].view(np.int32), res[1][1].view(np.int32))
    assert c.G.stream_status() & 16 == 0  # no timeout


@pytest.mark.parametrize("name", CASES)
def test_search_bf16_equals_fp32(name):
    _cuda()
    _tc()
    c = get_case(name)
    a = _search(c, prec=0)
    b = _search(c, prec=1)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1].view(np.int32), b[1].view(np.int32))
    assert c.G.stream_status() & 16 == 0


def test_bf16_kappa_c_above_group_count():
    # C = 777 gives 28 groups of 32 < kappa_c = 128: every centroid becomes a candidate
    _cuda()
    _tc()
    c = get_case("random_edges")
    R = c.q.shape[0]
    out = []
    for prec in (0, 1):
        ids = torch.empty((R, 128), dtype=torch.int32, device="cuda")
        sc = torch.empty((R, 128), dtype=torch.float32, device="cuda")
        c.G.top_centroids(c.params(prec, kc=128), c.dq, ids, sc)
        torch.cuda.synchronize()
        out.append(ids.cpu().numpy())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_zero_queries_tie_every_score(prec):
    # All-zero query tokens: every centroid score, every S~ and every refined S is 0, so every
    # stage decides by the id rule alone. Step (a) keeps the kappa_c lowest centroid ids, step (b)
    # the kappa_d lowest reached documents, steps (c)-(d) the k lowest non-empty ones. Every
    # (query token, document token) pair of the top-k window passes the decode pass's test, so
    # its pair list (8192 per query) overflows many times over and the documents go to the
    # all-pairs FP32 kernel; the list's counter must not wrap.
    _cuda()
    if prec:
        _tc()
    c = get_case("small")
    nq, kc, kd, k = 16, 40, 2000, 50
    ntok = np.full(nq, 32, np.int32)
    q = np.zeros((int(ntok.sum()), 128), np.float32)
    ref = c.O.search(q, ntok, k, kc, kd)
    dq = torch.from_numpy(q).cuda()
    oi = torch.full((nq * k,), -7, dtype=torch.int32, device="cuda")
    os_ = torch.full((nq * k,), np.nan, dtype=torch.float32, device="cuda")
    c.G.stream_status()
    c.G.search(c.params(prec, kd=kd, kc=kc), dq, ntok, np.full(nq, k, np.int32), oi, os_)
    torch.cuda.synchronize()
    gi, gs = oi.cpu().numpy(), os_.cpu().numpy()
    assert np.array_equal(gi, ref["ids"])
    assert np.all(gs == 0.0) and np.all(ref["scores"] == 0.0)
    assert c.G.stream_status() & (4 | 8 | 16) == 0  # no unrescued overflow, bad input or timeout


@pytest.mark.parametrize("name", ["small", "small32", "random_edges", "random_m8"])
def test_refine_tc_within_error_bound(name):
    # approximate refined scores (decode + tensor cores) are within the per-document bound
    # the FP32 repair of the top-k window relies on; the FP32 kernel is within 1e-5
    _cuda()
    _tc()
    c = get_case(name)
    res = c.O.search(c.q, c.ntok, c.k, c.kc, c.kd, stages=True)
    cand = np.ascontiguousarray(res["cand_ids"])
    dc = torch.from_numpy(cand).cuda()
    out = {}
    bnd = torch.full((c.nq, c.kd), -1.0, dtype=torch.float32, device="cuda")
    for prec in (0, 1):
        o = torch.full((c.nq, c.kd), np.nan, dtype=torch.float32, device="cuda")
        c.G.debug_refine_scores(c.params(prec), c.dq, c.ntok, dc, o, bnd if prec == 1 else None)
        torch.cuda.synchronize()
        out[prec] = o.cpu().numpy().astype(np.float64)
    bounds = bnd.cpu().numpy().astype(np.float64)
    worst = 0.0
    for u in range(c.nq):
        cd = cand[u]
        valid = cd >= 0
        exact = c.O.refine(c.q[c.qoff[u]:c.qoff[u + 1]], cd[valid])
        e1 = np.abs(out[1][u][valid] - exact)
        e0 = np.abs(out[0][u][valid] - exact)
        b = bounds[u][valid]
        assert np.all(b >= 0)
        assert np.all(e1 <= b), (u, (e1 - b).max())
        assert np.all(e0 <= 1e-5 * np.maximum(1, np.abs(exact)))
        worst = max(worst, (e1 / np.maximum(b, 1e-30)).max())
    # the approximation really is approximate, and the bound is not loose by orders of magnitude
    assert 0.0 < worst
    assert worst > 1e-3

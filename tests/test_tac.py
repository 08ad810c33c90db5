"""Token-Aware Clustering's centroid allotment (Sec. 2.1, Phases 1-4), on the CPU.

The oracle (oracle/tac.py) is pinned to hand-worked allotments, closed forms and the paper's
speed-up bound; the library's host implementation (tachiom_tac_allot) must return the oracle's
integers exactly on seeded inputs shaped like a Zipfian vocabulary.
"""
import json
import math
import os
import types

import numpy as np
import pytest

from oracle import tac as O

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "tac_allot.json")))


def _native():
    import paper_2604_28142_b300 as T
    return T


PROP_M = [8, 9, 11, 13, 23]


def _args(c):
    return c["budget"], c["mu"], c["tau"], c["eps"], c["theta"]


def _feasible(n, mu, tau, eps, theta):
    """(smallest, largest) total the bounds allow: the tail's fixed allotment plus every active
    type at its floor, resp. at its cap."""
    tail = sum(1 if 0 < x < mu else 2 if mu <= x < tau else 0 for x in n)
    caps = [min(x, max(1, math.floor(x / theta))) for x in n if x >= tau and x > 0]
    return tail + sum(min(eps, c) for c in caps), tail + sum(caps)


# ---- pins of the oracle ---------------------------------------------------------------

@pytest.mark.parametrize("i", range(len(GOLD["cases"])))
def test_oracle_golden(i):
    c = GOLD["cases"][i]
    assert O.allot(GOLD["n"], GOLD["s"], *_args(c)) == c["expected"]


def test_oracle_exact_proportional_shares():
    # every type active, no bounds in the way, n_j = m_j^2 and s_j = 1: w_j = m_j, and a budget
    # of c * sum(m) makes every share the integer c * m_j (sum(m) = 64: exact in binary) within
    # the caps n_j, so Phase 4 has nothing to do
    m = PROP_M
    n = [x * x for x in m]
    for c in (1, 2, 7):
        k = O.allot(n, [1.0] * len(m), c * sum(m), mu=0, tau=0, eps=0, theta=1e-9)
        assert k == [c * x for x in m]


def test_oracle_spread_closed_forms():
    rng = np.random.default_rng(3)
    v = rng.normal(size=(60, 5))
    t = rng.integers(0, 4, size=60)
    got = O.spread(v.tolist(), t.tolist(), 5)
    for j in range(4):
        x = v[t == j]
        assert got[j] == pytest.approx(float(x.var(axis=0).sum()), rel=1e-12)  # population variance
    assert got[4] == 0.0
    # two points at +-a e1: every point is at distance a from the mean
    assert O.spread([[2.5, 0.0], [-2.5, 0.0]], [0, 0], 1) == [pytest.approx(6.25)]


def test_oracle_tail_bounds_and_total():
    rng = np.random.default_rng(11)
    n = (1000.0 / np.arange(1, 401) ** 1.1).astype(np.int64)
    s = rng.uniform(0.2, 1.0, size=n.size)
    mu, tau, eps, theta = 3, 12, 2, 8.0
    lo, hi = _feasible(n.tolist(), mu, tau, eps, theta)
    budget = (lo + hi) // 2
    k = O.allot(n.tolist(), s.tolist(), budget, mu, tau, eps, theta)
    assert sum(k) == budget
    for j in range(n.size):
        if n[j] <= 0:
            assert k[j] == 0
        elif n[j] < mu:
            assert k[j] == 1
        elif n[j] < tau:
            assert k[j] == 2
        else:
            cap = min(n[j], max(1, math.floor(n[j] / theta)))
            assert min(eps, cap) <= k[j] <= cap


def test_oracle_speedup_bound():
    # Sec. 2.1: kappa N / sum_j kappa_j n_j >= sum(w) / max(w) for the unrounded allotment,
    # with equality when every type has the same n and s
    rng = np.random.default_rng(5)
    for _ in range(20):
        n = rng.integers(1, 10000, size=50)
        s = rng.uniform(0.01, 2.0, size=50)
        bound, ratio = O.speedup_lower_bound(n.tolist(), s.tolist())
        assert ratio >= bound * (1 - 1e-12)
    bound, ratio = O.speedup_lower_bound([64] * 10, [0.5] * 10)
    assert bound == pytest.approx(10.0) and ratio == pytest.approx(10.0)


def test_oracle_infeasible_budgets():
    n, s = GOLD["n"], GOLD["s"]
    with pytest.raises(O.AllotError):
        O.allot(n, s, 2, 5, 50, 2, 10.0)      # below the tail's 1 + 2
    with pytest.raises(O.AllotError):
        O.allot(n, s, 8, 5, 50, 2, 10.0)      # floors need 3 + 2 * 3
    with pytest.raises(O.AllotError):
        O.allot(n, s, 10**6, 5, 50, 2, 10.0)  # caps allow 3 + 10 + 40 + 90


# planted mistakes: each must fail one of the pins above
_MUTANTS = [
    ("w[j] = math.sqrt(n[j]) * s[j]", "w[j] = n[j] * s[j]"),       # no damping
    ("if n[j] < mu:\n            kappa[j] = 1", "if n[j] < mu:\n            kappa[j] = 2"),
    ("B = budget - sum(kappa)", "B = budget"),                      # tail not taken off the budget
    ("if best is None or r > best[0]:", "if best is None or r < best[0]:"),  # adds to the wrong type
    ("kappa[j] = min(max(kappa[j], lo[j]), hi[j])", "kappa[j] = max(kappa[j], lo[j])"),  # no cap
    ("share[j] = (w[j] / W) * B if W > 0 else 0.0", "share[j] = (w[j] / W) * budget if W > 0 else 0.0"),
]


def _pins_pass(mod):
    try:
        for c in GOLD["cases"]:
            if mod.allot(GOLD["n"], GOLD["s"], *_args(c)) != c["expected"]:
                return False
        m = PROP_M
        if mod.allot([x * x for x in m], [1.0] * len(m), 2 * sum(m), 0, 0, 0, 1e-9) != [2 * x for x in m]:
            return False
    except Exception:
        return False
    return True


@pytest.mark.parametrize("i", range(len(_MUTANTS)))
def test_oracle_mutant_caught(i):
    src = open(O.__file__).read()
    a, b = _MUTANTS[i]
    assert src.count(a) == 1, a
    mod = types.ModuleType("tac_mutant")
    exec(compile(src.replace(a, b), "tac_mutant", "exec"), mod.__dict__)
    assert _pins_pass(O)
    assert not _pins_pass(mod)


# ---- the library against the oracle -------------------------------------------------

@pytest.mark.parametrize("i", range(len(GOLD["cases"])))
def test_native_golden(i):
    T = _native()
    c = GOLD["cases"][i]
    assert T.tac_allot(GOLD["n"], GOLD["s"], *_args(c)).tolist() == c["expected"]


@pytest.mark.parametrize("seed", range(8))
def test_native_equals_oracle_zipf(seed):
    # a Zipfian vocabulary (a few very frequent types, a long tail, some absent types),
    # spreads in [0.05, 1], budgets across the feasible range
    T = _native()
    rng = np.random.default_rng(100 + seed)
    nt = int(rng.integers(50, 1500))
    n = np.floor(20000.0 / np.arange(1, nt + 1) ** rng.uniform(0.8, 1.3)).astype(np.int64)
    n[rng.choice(nt, size=nt // 20, replace=False)] = 0
    rng.shuffle(n)
    s = rng.uniform(0.05, 1.0, size=nt)
    mu, tau = int(rng.integers(1, 6)), int(rng.integers(6, 40))
    eps, theta = int(rng.integers(1, 4)), float(rng.uniform(4.0, 64.0))
    lo, hi = _feasible(n.tolist(), mu, tau, eps, theta)
    for frac in (0.0, 0.3, 0.7, 1.0):
        budget = int(lo + frac * (hi - lo))
        want = O.allot(n.tolist(), s.tolist(), budget, mu, tau, eps, theta)
        got = T.tac_allot(n, s, budget, mu, tau, eps, theta)
        assert got.tolist() == want
        assert int(got.sum()) == budget


def test_native_ties_and_zero_spread():
    # equal weights: reconciliation order falls to the type ids; all-zero spreads: shares are 0
    T = _native()
    n = [100] * 7
    for s, budget in (([1.0] * 7, 10), ([1.0] * 7, 4 * 7 - 2), ([0.0] * 7, 9)):
        want = O.allot(n, s, budget, 1, 2, 1, 25.0)
        assert T.tac_allot(n, s, budget, 1, 2, 1, 25.0).tolist() == want


def test_native_rejects_bad_arguments():
    T = _native()
    n, s = GOLD["n"], GOLD["s"]
    for args in ((2, 5, 50, 2, 10.0), (8, 5, 50, 2, 10.0), (10**6, 5, 50, 2, 10.0),
                 (40, 5, 50, 2, 0.0), (40, -1, 50, 2, 10.0), (-1, 5, 50, 2, 10.0)):
        with pytest.raises(T.TachiomError):
            T.tac_allot(n, s, *args)
    with pytest.raises(T.TachiomError):
        T.tac_allot(n, [0.0, 0.0, -1.0, 1.0, 1.0], 40, 5, 50, 2, 10.0)
    with pytest.raises(T.TachiomError):
        T.tac_allot(n, [0.0, 0.0, float("nan"), 1.0, 1.0], 40, 5, 50, 2, 10.0)
    assert T.tac_allot(np.zeros(0, np.int64), np.zeros(0), 0, 1, 2, 1, 1.0).shape == (0,)


# ---- clustering and residual encoding after the allotment --------------------------------

def test_oracle_assign_brute_force_and_ties():
    rng = np.random.default_rng(21)
    x, c = rng.normal(size=(40, 6)), rng.normal(size=(9, 6))
    want = np.argmin(((x[:, None, :] - c[None, :, :]) ** 2).sum(-1), axis=1)  # first minimum
    assert O.assign(x.tolist(), c.tolist()) == want.tolist()
    # equidistant from centroids 2 and 5 (mirror images): the lower index wins
    cc = [[9.0, 9.0], [8.0, 8.0], [1.0, 0.0], [7.0, 7.0], [6.0, 6.0], [-1.0, 0.0]]
    assert O.assign([[0.0, 3.0]], cc) == [2]


def test_oracle_lloyd_closed_forms():
    rng = np.random.default_rng(22)
    x = rng.normal(size=(50, 4))
    # one centroid: the mean after one round
    c, lab, _ = O.lloyd(x.tolist(), [[5.0, 5.0, 5.0, 5.0]], 1)
    assert np.allclose(c[0], x.mean(axis=0), rtol=0, atol=1e-12) and set(lab) == {0}
    # Lloyd's rounds never increase the inertia
    _, _, hist = O.lloyd(x.tolist(), x[:6].tolist(), 12)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(hist, hist[1:]))
    # three tight blobs started at their means stay put; a far centroid no point joins is kept
    means = np.array([[0.0, 0.0], [10.0, 0.0], [0.0, 10.0]])
    pts = np.concatenate([m + 0.01 * rng.normal(size=(20, 2)) for m in means])
    start = [pts[:20].mean(0).tolist(), pts[20:40].mean(0).tolist(), pts[40:].mean(0).tolist(), [500.0, 500.0]]
    c, lab, _ = O.lloyd(pts.tolist(), start, 5)
    assert np.allclose(c[:3], start[:3], atol=1e-12) and c[3] == [500.0, 500.0]
    assert lab == [0] * 20 + [1] * 20 + [2] * 20


def _unit_codebooks(rng, M=4, ds=2, K=16):
    # codewords of norm 1 / sqrt(M): any M of them, one per subspace, concatenate to a unit vector
    a = rng.uniform(0, 2 * np.pi, size=(M, K))
    return [[[math.cos(t) / math.sqrt(M), math.sin(t) / math.sqrt(M)] for t in a[m]] for m in range(M)]


def test_oracle_pq_encode_lossless_zero_and_ties():
    rng = np.random.default_rng(23)
    cb = _unit_codebooks(rng)
    cent = rng.normal(size=(3, 8)).tolist()
    want_codes = rng.integers(0, 16, size=(25, 4))
    rho = rng.uniform(0.1, 2.0, size=25)
    lab = rng.integers(0, 3, size=25).tolist()
    vec = [(np.array(cent[l]) + r * np.concatenate([cb[m][k] for m, k in enumerate(code)])).tolist()
           for l, r, code in zip(lab, rho, want_codes)]
    codes, rhos = O.pq_encode(vec, cent, lab, cb)
    assert codes == want_codes.tolist()
    assert np.allclose(rhos, rho, rtol=1e-12, atol=0)
    # a token equal to its centroid: rho 0, codes 0
    codes, rhos = O.pq_encode([cent[1]], cent, [1], cb)
    assert codes == [[0, 0, 0, 0]] and rhos == [0.0]
    # a codeword repeated at codes 3 and 7 of subspace 0: the lower code is chosen
    cb2 = [list(row) for row in cb]
    cb2[0][7] = list(cb2[0][3])
    v = (np.array(cent[0]) + np.concatenate([cb2[0][7], cb2[1][0], cb2[2][0], cb2[3][0]])).tolist()
    codes, _ = O.pq_encode([v], cent, [0], cb2)
    assert codes[0][0] == 3


_CLUSTER_MUTANTS = [
    ("            if best is None or dd < best:\n                best, bi = dd, i",
     "            if best is None or dd <= best:\n                best, bi = dd, i"),       # ties to the higher index
    ("            if cnt[i]:\n                c[i] = [x / cnt[i] for x in sums[i]]",
     "            c[i] = [x / max(cnt[i], 1) for x in sums[i]]"),                          # empty cluster zeroed
    ("r = [float(x) - float(y) for x, y in zip(t, centroids[l])]",
     "r = [float(y) - float(x) for x, y in zip(t, centroids[l])]"),                    # residual sign
]


@pytest.mark.parametrize("i", range(len(_CLUSTER_MUTANTS)))
def test_oracle_cluster_mutant_caught(i):
    src = open(O.__file__).read()
    a, b = _CLUSTER_MUTANTS[i]
    assert src.count(a) == 1, a
    mod = types.ModuleType("tac_mutant")
    exec(compile(src.replace(a, b), "tac_mutant", "exec"), mod.__dict__)
    pins = (test_oracle_assign_brute_force_and_ties, test_oracle_lloyd_closed_forms,
            test_oracle_pq_encode_lossless_zero_and_ties)
    failed = 0
    saved = O.__dict__.copy()
    try:
        for name in ("assign", "lloyd", "pq_encode", "inertia", "_sqdist"):
            setattr(O, name, getattr(mod, name))
        for pin in pins:
            try:
                pin()
            except AssertionError:
                failed += 1
    finally:
        for name in ("assign", "lloyd", "pq_encode", "inertia", "_sqdist"):
            setattr(O, name, saved[name])
    assert failed >= 1


def test_oracle_init_positions_and_cluster():
    # evenly spaced, distinct, in range
    for nj, kj in ((1, 1), (10, 3), (1000, 17), (17, 17)):
        pos = O.init_positions(nj, kj)
        assert len(set(pos)) == kj and 0 <= min(pos) and max(pos) < nj
    assert O.init_positions(10, 3) == [1, 5, 8]
    # end to end on separated blobs: the centroid count per type is the allotment, every vector's
    # label is the nearest centroid of its own type, and every non-empty centroid is the mean of its
    # members (Lloyd has converged on this input)
    rng = np.random.default_rng(31)
    vecs, types = [], []
    for j, (cnt, nb) in enumerate(((120, 3), (60, 2), (4, 1), (30, 2))):
        centers = rng.normal(size=(nb, 8)) * 10
        for i in range(cnt):
            vecs.append((centers[i % nb] + 0.01 * rng.normal(size=8)).tolist())
            types.append(j)
    kappa, cents, ctype, labels = O.cluster(vecs, types, 5, 8, mu=5, tau=20, eps=1, theta=10.0, iters=20)
    assert kappa == O.allot([120, 60, 4, 30, 0], O.spread(vecs, types, 5), 8, 5, 20, 1, 10.0)
    assert sum(kappa) == 8 and len(cents) == 8 and kappa[4] == 0 and kappa[2] == 1
    assert ctype == sorted(ctype) and [ctype.count(j) for j in range(5)] == kappa
    v, t, lab = np.array(vecs), np.array(types), np.array(labels)
    for j in range(4):
        ids = [g for g in range(8) if ctype[g] == j]
        d2 = ((v[t == j][:, None, :] - np.array([cents[g] for g in ids])[None]) ** 2).sum(-1)
        assert [ids[x] for x in d2.argmin(1)] == lab[t == j].tolist()
        for g in ids:
            if (lab == g).any():
                assert np.allclose(cents[g], v[lab == g].mean(0), atol=1e-12)


def test_oracle_pq_train_closed_forms():
    rng = np.random.default_rng(61)
    x, c = rng.normal(size=(64, 8)), rng.normal(size=(3, 8))
    lab = rng.integers(0, 3, size=64)
    lab[5] = -1
    r = x - c[np.maximum(lab, 0)]
    u = r / np.linalg.norm(r, axis=1, keepdims=True)
    u[5] = 0.0  # a label < 0 trains as the zero vector
    # K = S: every sampled vector is its own codeword (the sample is every vector when S = N)
    books = O.pq_train(x.tolist(), c.tolist(), lab.tolist(), M=2, sample=64, iters=2, K=64)
    for m in range(2):
        assert np.allclose(np.array(books[m]), u[:, 4 * m:4 * m + 4], atol=1e-12)
    # K = 1: the mean of the sampled sub-vectors
    books = O.pq_train(x.tolist(), c.tolist(), lab.tolist(), M=4, sample=32, iters=1, K=1)
    pos = O.pq_sample_positions(64, 32)
    for m in range(4):
        assert np.allclose(books[m][0], u[pos, 2 * m:2 * m + 2].mean(0), atol=1e-12)

"""Token-Aware Clustering on the GPU (tachiom_tac_cluster) against the FP64 oracle (oracle/tac.py).

The inputs are separated blobs per token type, so the nearest centroid of every vector is far from a
tie and the FP32 distances of the kernel and the oracle's FP64 ones choose the same labels; centroids
then agree to FP32 rounding (rtol 1e-6).
"""
import numpy as np
import pytest

from oracle import tac as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PARAMS = dict(mu=5, tau=20, eps=1, theta=10.0)


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _blobs(counts, seed):
    """Vectors of each type drawn around a few centers of that type (scale 10, noise 0.01)."""
    rng = np.random.default_rng(seed)
    vecs, types = [], []
    for j, cnt in enumerate(counts):
        centers = rng.normal(size=(1 + j % 4, 128)) * 10.0
        for i in range(cnt):
            vecs.append(centers[i % len(centers)] + 0.01 * rng.normal(size=128))
            types.append(j)
    order = rng.permutation(len(types))  # types interleaved in the collection
    return np.array(vecs, np.float32)[order], np.array(types, np.int32)[order]


def _run(T, v, t, n_types, budget, iters, **kw):
    return T.tac_cluster(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), n_types, budget,
                         iters=iters, **kw)


def test_tac_cluster_matches_oracle():
    _cuda()
    import paper_2604_28142_b300 as T
    counts = [400, 200, 130, 100, 80, 60, 50, 40, 8, 4, 2, 0]
    v, t = _blobs(counts, seed=41)
    n_types, iters = len(counts), 6
    s_or = O.spread(v.astype(np.float64).tolist(), t.tolist(), n_types)
    lo_hi = [min(x, max(1, int(np.floor(x / PARAMS["theta"])))) for x in counts if x >= PARAMS["tau"]]
    tail = sum(1 if 0 < x < PARAMS["mu"] else 2 if PARAMS["mu"] <= x < PARAMS["tau"] else 0 for x in counts)
    budget = tail + (sum(min(PARAMS["eps"], c) for c in lo_hi) + sum(lo_hi)) // 2
    kappa, spread, cents, ctype, labels = _run(T, v, t, n_types, budget, iters, **PARAMS)
    torch.cuda.synchronize()
    assert np.allclose(spread, s_or, rtol=1e-12, atol=0)
    ok, oc, oct_, olab = O.cluster(v.astype(np.float64).tolist(), t.tolist(), n_types, budget,
                                   iters=iters, **PARAMS)
    assert kappa.tolist() == ok
    assert ctype.cpu().tolist() == oct_
    assert labels.cpu().tolist() == olab
    assert np.allclose(cents.cpu().numpy(), np.array(oc), rtol=1e-6, atol=1e-6)
    # the same call repeats bit for bit
    k2, s2, c2, ct2, l2 = _run(T, v, t, n_types, budget, iters, **PARAMS)
    torch.cuda.synchronize()
    assert np.array_equal(k2, kappa) and np.array_equal(s2, spread)
    assert torch.equal(c2, cents) and torch.equal(ct2, ctype) and torch.equal(l2, labels)


def test_tac_cluster_type_without_centroid_and_bad_type():
    _cuda()
    import paper_2604_28142_b300 as T
    # type 1: 50 identical vectors (spread 0, weight 0) and eps = 0: it receives no centroid, so its
    # vectors get label -1; type 0 takes the whole budget of 3
    rng = np.random.default_rng(7)
    v = np.concatenate([rng.normal(size=(50, 128)) * 10.0, np.tile(rng.normal(size=(1, 128)), (50, 1))])
    v = v.astype(np.float32)
    t = np.array([0] * 50 + [1] * 50, np.int32)
    kappa, _, cents, ctype, labels = _run(T, v, t, 2, 3, 4, mu=1, tau=2, eps=0, theta=1.0)
    torch.cuda.synchronize()
    ok, oc, oct_, olab = O.cluster(v.astype(np.float64).tolist(), t.tolist(), 2, 3, mu=1, tau=2, eps=0,
                                   theta=1.0, iters=4)
    assert kappa.tolist() == ok == [3, 0]
    assert labels.cpu().tolist() == olab and olab[50:] == [-1] * 50
    bad = t.copy()
    bad[10] = 5
    with pytest.raises(T.TachiomError):
        _run(T, v, bad, 2, 3, 1, mu=1, tau=2, eps=0, theta=1.0)


def _pq_case(M, seed, lossless):
    rng = np.random.default_rng(seed)
    ds = 128 // M
    if lossless:
        # codewords of norm 1 / sqrt(M): one per subspace concatenates to a unit vector
        cb = rng.normal(size=(M, 256, ds))
        cb /= np.linalg.norm(cb, axis=2, keepdims=True) * np.sqrt(M)
    else:
        cb = rng.normal(size=(M, 256, ds)) * 0.2
    cents = rng.normal(size=(5, 128))
    n = 64
    lab = rng.integers(0, 5, size=n)
    lab[:3] = -1
    if lossless:
        want = rng.integers(0, 256, size=(n, M))
        rho = rng.uniform(0.1, 2.0, size=n)
        u = np.stack([np.concatenate([cb[m][want[i, m]] for m in range(M)]) for i in range(n)])
        x = cents[np.maximum(lab, 0)] + rho[:, None] * u
    else:
        x = cents[np.maximum(lab, 0)] + rng.normal(size=(n, 128)) * 0.3
    x[:3] = rng.normal(size=(3, 128))
    return x.astype(np.float32), cents.astype(np.float32), lab.astype(np.int32), cb.astype(np.float32)


@pytest.mark.parametrize("M", [8, 16, 32])
@pytest.mark.parametrize("lossless", [True, False])
def test_pq_encode_against_oracle(M, lossless):
    _cuda()
    import paper_2604_28142_b300 as T
    x, cents, lab, cb = _pq_case(M, 50 + M, lossless)
    codes, rnorm = T.pq_encode(torch.from_numpy(x).cuda(), torch.from_numpy(cents).cuda(),
                               torch.from_numpy(lab).cuda(), torch.from_numpy(cb).cuda())
    torch.cuda.synchronize()
    codes = codes.cpu().numpy().astype(np.int64)
    rho_g = rnorm.cpu().numpy().view(np.float16).astype(np.float64)
    ok = lab >= 0
    oc, orho = O.pq_encode(x[ok].astype(np.float64).tolist(), cents.astype(np.float64).tolist(),
                           lab[ok].tolist(), cb.astype(np.float64).tolist())
    oc, orho = np.array(oc), np.array(orho)
    assert np.all(codes[~ok] == 0) and np.all(rho_g[~ok] == 0.0)
    # rho: the oracle's norm rounded to fp16 (within one fp16 step of it)
    assert np.all(np.abs(rho_g[ok] - orho) <= np.abs(orho) * 2.0 ** -10 + 1e-7)
    if lossless:
        assert np.array_equal(codes[ok], oc)
    else:
        # a valid code: its codeword is as near as the oracle's to within FP32 rounding
        ds = 128 // M
        u = (x[ok].astype(np.float64) - cents[lab[ok]].astype(np.float64)) / orho[:, None]
        for m in range(M):
            sub = u[:, m * ds:(m + 1) * ds]
            dist = ((sub[:, None, :] - cb[m][None].astype(np.float64)) ** 2).sum(-1)
            got = dist[np.arange(len(sub)), codes[ok][:, m]]
            assert np.all(got <= dist.min(1) + 1e-5)
        assert (codes[ok] == oc).mean() > 0.99


def _pq_train_case(M, seed):
    """Vectors whose sampled normalised residuals fall, in every subspace, into 256 tight clusters of
    two consecutive sample points: the evenly spaced initial codewords (positions 2 j + 1) take one
    point of each cluster, so Lloyd's answer is the mean of every pair."""
    rng = np.random.default_rng(seed)
    ds = 128 // M
    true = rng.normal(size=(M, 256, ds))
    true /= np.linalg.norm(true, axis=2, keepdims=True) * np.sqrt(M)
    perm = np.stack([rng.permutation(256) for _ in range(M)])
    n = 512
    cid = perm[:, np.arange(n) // 2]                               # [M, n]: cluster of sample r
    u = np.concatenate([true[m][cid[m]] for m in range(M)], axis=1) + 1e-5 * rng.normal(size=(n, 128))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    cents = rng.normal(size=(4, 128))
    lab = rng.integers(0, 4, size=n)
    x = cents[lab] + rng.uniform(0.2, 2.0, size=(n, 1)) * u
    return x.astype(np.float32), cents.astype(np.float32), lab.astype(np.int32), cid


@pytest.mark.skipif(__import__("os").environ.get("TACHIOM_TEST_PQ_TRAIN_GPU") != "1",
                    reason="GPU codebook training tests are opt-in (TACHIOM_TEST_PQ_TRAIN_GPU=1) until run on a GPU")
@pytest.mark.parametrize("M", [8, 16, 32])
def test_pq_train_closed_form(M):
    _cuda()
    import paper_2604_28142_b300 as T
    x, cents, lab, cid = _pq_train_case(M, 70 + M)
    dx, dc, dl = torch.from_numpy(x).cuda(), torch.from_numpy(cents).cuda(), torch.from_numpy(lab).cuda()
    books = T.pq_train(dx, dc, dl, M, sample=512, iters=3)
    torch.cuda.synchronize()
    # the sample is every vector (positions floor(r + 1/2) = r); its normalised residuals in FP64
    r = x.astype(np.float64) - cents[lab].astype(np.float64)
    u = r / np.linalg.norm(r, axis=1, keepdims=True)
    ds = 128 // M
    b = books.cpu().numpy().astype(np.float64)
    for m in range(M):
        sub = u[:, m * ds:(m + 1) * ds]
        for j in range(256):
            want = sub[2 * j:2 * j + 2].mean(0)  # codeword j started at sample 2 j + 1: cluster of pair j
            assert np.allclose(b[m, j], want, atol=1e-6), (m, j)
    # encoding the sample with the trained codebooks gives back each sample's pair
    codes, _ = T.pq_encode(dx, dc, dl, books)
    torch.cuda.synchronize()
    assert np.array_equal(codes.cpu().numpy().astype(np.int64), np.repeat(np.arange(256), 2)[:, None].repeat(M, 1))
    # the same call repeats bit for bit
    assert torch.equal(T.pq_train(dx, dc, dl, M, sample=512, iters=3), books)

"""Pins that tie the FP64 oracle to facts outside itself.

Each pin takes a factory `make(ix, dim)` returning an oracle over an index
dict, so the same pins run against the real oracle (test_oracle_pins.py)
and against deliberately broken copies of it (test_oracle_mutants.py), which
shows that a plausible mistake in the oracle fails at least one pin.

What each pin compares against:
  * golden toys (tests/golden/*.json): values derived by hand;
  * numpy brute force written from the definitions with dense linear algebra
    (a full sort of all centroid scores; MaxSim of explicitly reconstructed
    vectors; the exhaustive scan over every document);
  * invariants (list route == document route, token-permutation invariance,
    rho = 0 reduces refine to the centroid interaction, lossless PQ makes
    refine equal exact MaxSim, kappa_c = C / kappa_d = D reduce the cascade
    to exhaustive PQ-MaxSim);
  * IEEE decoding of the stored fp16 / bf16 formats against numpy.
"""
from __future__ import annotations

import json
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def toy_index_from_golden(g):
    dim, m = g["dim"], g["pq_m"]
    ds = dim // m
    W = np.zeros((m, 256, ds), np.float32)
    for sm, entries in g["codebook_entries"].items():
        for code, vec in entries.items():
            W[int(sm), int(code)] = vec
    return {
        "centroid_dtype": "f32",
        "centroids": np.array(g["centroids"], np.float32),
        "doc_offsets": np.array(g["doc_offsets"], np.int64),
        "token_centroid": np.array([t[1] for t in g["doc_tokens"]], np.int32),
        "pq_codebooks": W,
        "pq_codes": np.array(g["codes"], np.uint8),
        "residual_norms": np.array(g["residual_norms"], np.float16).view(np.uint16),
    }


# ---------------------------------------------------------------- helpers

def widen_centroids(ix):
    c = ix["centroids"]
    if ix.get("centroid_dtype") == "bf16":
        return (c.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return c.astype(np.float64)


def decode_residuals(ix):
    """r^_t: concatenated codewords of each token (dense numpy, FP64)."""
    W = ix["pq_codebooks"].astype(np.float64)
    codes = ix["pq_codes"]
    m = W.shape[0]
    parts = [W[s][codes[:, s]] for s in range(m)]
    return np.concatenate(parts, axis=1)


def rho(ix):
    rn = ix.get("residual_norms")
    if rn is None:
        return np.ones(ix["token_centroid"].shape[0])
    return rn.view(np.float16).astype(np.float64)


def reconstructed(ix):
    C = widen_centroids(ix)
    return C[ix["token_centroid"]] + rho(ix)[:, None] * decode_residuals(ix)


def brute_maxsim(q, X, doc_off, docs):
    """sum_i max_{t in d} <q_i, x_t> by dense matmul."""
    q = q.astype(np.float64)
    out = []
    for d in docs:
        s, e = doc_off[d], doc_off[d + 1]
        if e == s:
            out.append(0.0)
            continue
        out.append(float((q @ X[s:e].T).max(axis=1).sum()))
    return np.array(out)


def order_desc_asc(scores, ids):
    return np.lexsort((ids, -scores))


# ---------------------------------------------------------------- pins

def pin_golden_topc(make):
    g = _golden("toy_topc.json")
    ang = np.deg2rad(np.array(g["centroid_angles_deg"], np.float64))
    c = np.zeros((len(ang), g["dim"]), np.float32)
    c[:, 0] = np.cos(ang)
    c[:, 1] = np.sin(ang)
    ix = {"centroid_dtype": "f32", "centroids": c, "doc_offsets": np.array([0, 1], np.int64),
          "token_centroid": np.array([0], np.int32),
          "pq_codebooks": np.zeros((2, 256, 2), np.float32), "pq_codes": np.zeros((1, 2), np.uint8)}
    o = make(ix, g["dim"])
    ids, s = o.top_centroids(np.array([g["query"]], np.float32), g["kappa_c"])
    assert ids[0].tolist() == g["expected_ids"], ids
    assert np.allclose(s[0], g["expected_scores"], atol=1e-6), s


def pin_golden_maxsim(make):
    g = _golden("toy_maxsim.json")
    ix = toy_index_from_golden(g)
    o = make(ix, g["dim"])
    q = np.array(g["queries"], np.float32)
    ids, s = o.top_centroids(q, g["kappa_c"])
    assert ids.tolist() == g["expected"]["top_ids"], ids
    assert np.allclose(s, g["expected"]["top_scores"], atol=0), s
    docs, gs = o.gather(q, ids)
    assert docs.tolist() == g["expected"]["gather_docs"], docs
    assert np.allclose(gs, g["expected"]["gather_scores"], atol=0), gs
    r = o.refine(q, np.array([0, 1], np.int32))
    assert r[0] == g["expected"]["refine_doc0"] and r[1] == g["expected"]["refine_doc1"], r
    # the whole cascade returns doc 0 first: doc 1 is never a candidate
    res = o.search(q, np.array([2], np.int32), 2, g["kappa_c"], 4)
    assert res["ids"].tolist() == [0, -1] and res["scores"][0] == 2.0, res


def pin_topc_full_sort(make):
    ix = synth.random_index(30, 700, seed=1)
    qs = synth.random_queries(3, 5, 5, seed=2)["queries"]
    o = make(ix, 128)
    kc = 37
    ids, s = o.top_centroids(qs, kc)
    C = widen_centroids(ix)
    S = qs.astype(np.float64) @ C.T
    for r in range(qs.shape[0]):
        order = order_desc_asc(S[r], np.arange(C.shape[0]))[:kc]
        assert ids[r].tolist() == order.tolist()
        assert np.allclose(s[r], S[r][order], rtol=0, atol=1e-12)


def pin_topc_bf16_widening(make):
    # one-hot query picks out a single centroid coordinate, so the score is the
    # widened bf16 value itself: compare with numpy's bit-level widening
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 1 << 16, size=300).astype(np.uint16)
    f = (bits.astype(np.uint32) << 16).view(np.float32)
    bits = bits[np.isfinite(f)]
    n = bits.shape[0]
    c = np.zeros((n, 128), np.uint16)
    c[:, 3] = bits
    ix = {"centroid_dtype": "bf16", "centroids": c, "doc_offsets": np.array([0, 1], np.int64),
          "token_centroid": np.array([0], np.int32),
          "pq_codebooks": np.zeros((16, 256, 8), np.float32), "pq_codes": np.zeros((1, 16), np.uint8)}
    o = make(ix, 128)
    q = np.zeros((1, 128), np.float32)
    q[0, 3] = 1.0
    ids, s = o.top_centroids(q, n)
    want = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    got = np.empty(n)
    got[ids[0]] = s[0]
    assert np.array_equal(got, want)


def pin_fp16_norm_decoding(make):
    # documents of one token each: c = 0 and r^ = e0, so S(q=e0, d) = rho_d
    pats = np.arange(0, 1 << 16, 97, dtype=np.uint32).astype(np.uint16)
    vals = pats.view(np.float16).astype(np.float64)
    keep = np.isfinite(vals)
    pats, vals = pats[keep], vals[keep]
    n = pats.shape[0]
    W = np.zeros((16, 256, 8), np.float32)
    W[0, 7, 0] = 1.0
    codes = np.zeros((n, 16), np.uint8)
    codes[:, 0] = 7
    ix = {"centroid_dtype": "f32", "centroids": np.zeros((1, 128), np.float32),
          "doc_offsets": np.arange(n + 1, dtype=np.int64), "token_centroid": np.zeros(n, np.int32),
          "pq_codebooks": W, "pq_codes": codes, "residual_norms": pats}
    o = make(ix, 128)
    q = np.zeros((1, 128), np.float32)
    q[0, 0] = 1.0
    r = o.refine(q, np.arange(n, dtype=np.int32))
    assert np.array_equal(r, vals)


def pin_list_route_equals_doc_route(make):
    ix = synth.random_index(120, 90, len_max=15, seed=3, empty_docs=4)
    qs = synth.random_queries(1, 7, 7, seed=4)["queries"]
    o = make(ix, 128)
    for kc in (1, 5, 17):
        ids, _ = o.top_centroids(qs, kc)
        d1, s1 = o.gather(qs, ids)
        d2, s2 = o.gather(qs, ids, doc_route=True)
        assert d1.tolist() == d2.tolist()
        assert np.allclose(s1, s2, rtol=0, atol=1e-12)


def pin_all_centroids_gives_centroid_maxsim(make):
    # kappa_c = C: s~_i(d) = max_{t in d} <q_i, c_a(t)> (every token's centroid is retrieved)
    ix = synth.random_index(60, 40, len_max=9, seed=6, empty_docs=3)
    qs = synth.random_queries(1, 6, 6, seed=7)["queries"]
    o = make(ix, 128)
    C = ix["centroids"].shape[0]
    ids, _ = o.top_centroids(qs, C)
    docs, s = o.gather(qs, ids)
    X = widen_centroids(ix)[ix["token_centroid"]]
    nonempty = [d for d in range(60) if ix["doc_offsets"][d + 1] > ix["doc_offsets"][d]]
    assert docs.tolist() == nonempty
    want = brute_maxsim(qs, X, ix["doc_offsets"], nonempty)
    assert np.allclose(s, want, rtol=0, atol=1e-12)


def pin_lossless_pq_refine_is_exact_maxsim(make):
    # tokens are built as c_a(t) + rho_t * (concatenated codewords): PQ is lossless
    # by construction, so refine must equal MaxSim on those vectors
    ix = synth.random_index(25, 30, len_max=20, seed=8, empty_docs=2)
    qs = synth.random_queries(1, 9, 9, seed=9)["queries"]
    o = make(ix, 128)
    X = reconstructed(ix)
    docs = np.arange(25, dtype=np.int32)
    got = o.refine(qs, docs)
    want = brute_maxsim(qs, X, ix["doc_offsets"], docs)
    assert np.allclose(got, want, rtol=0, atol=1e-12), np.abs(got - want).max()


def pin_zero_norm_refine_is_centroid_interaction(make):
    ix = synth.random_index(25, 30, len_max=20, seed=10, norms="zero")
    qs = synth.random_queries(1, 9, 9, seed=11)["queries"]
    o = make(ix, 128)
    X = widen_centroids(ix)[ix["token_centroid"]]
    docs = np.arange(25, dtype=np.int32)
    assert np.allclose(o.refine(qs, docs), brute_maxsim(qs, X, ix["doc_offsets"], docs),
                       rtol=0, atol=1e-12)


def pin_token_permutation_invariance(make):
    ix = synth.random_index(40, 50, len_max=14, seed=12)
    qs = synth.random_queries(1, 8, 8, seed=13)["queries"]
    rng = np.random.default_rng(14)
    perm = np.arange(ix["token_centroid"].shape[0])
    off = ix["doc_offsets"]
    for d in range(40):
        seg = perm[off[d]:off[d + 1]]
        perm[off[d]:off[d + 1]] = seg[rng.permutation(seg.shape[0])]
    ix2 = dict(ix)
    for key in ("token_centroid", "pq_codes", "residual_norms"):
        ix2[key] = np.ascontiguousarray(ix[key][perm])
    o1, o2 = make(ix, 128), make(ix2, 128)
    r1 = o1.search(qs, np.array([8], np.int32), 10, 6, 20, stages=True)
    r2 = o2.search(qs, np.array([8], np.int32), 10, 6, 20, stages=True)
    for key in ("ids", "scores", "cand_ids", "cand_s"):
        assert np.array_equal(r1[key], r2[key]), key
    # and the result is not trivially empty
    assert (r1["ids"] >= 0).sum() >= 5


def pin_exhaustive_cascade_is_brute_force(make):
    # kappa_c = C and kappa_d = D: the cascade is exhaustive PQ-MaxSim top-k
    ix = synth.random_index(45, 35, len_max=10, seed=15, empty_docs=3)
    q = synth.random_queries(2, 5, 7, seed=16)
    o = make(ix, 128)
    k = 12
    res = o.search(q["queries"], q["ntok"], k, 35, 45)
    X = reconstructed(ix)
    qo = np.concatenate([[0], np.cumsum(q["ntok"])])
    nonempty = np.array([d for d in range(45) if ix["doc_offsets"][d + 1] > ix["doc_offsets"][d]])
    for u in range(2):
        qq = q["queries"][qo[u]:qo[u + 1]]
        S = brute_maxsim(qq, X, ix["doc_offsets"], nonempty)
        order = order_desc_asc(S, nonempty)[:k]
        assert res["ids"][u * k:(u + 1) * k].tolist() == nonempty[order].tolist()
        assert np.allclose(res["scores"][u * k:(u + 1) * k], S[order], rtol=0, atol=1e-12)


def pin_gather_definition_brute_force(make):
    # S~ from the definition written with numpy over explicit (doc, centroid) pairs
    ix = synth.random_index(80, 60, len_max=12, seed=17)
    qs = synth.random_queries(1, 6, 6, seed=18)["queries"]
    o = make(ix, 128)
    kc = 7
    ids, _ = o.top_centroids(qs, kc)
    C = widen_centroids(ix)
    off, cid = ix["doc_offsets"], ix["token_centroid"]
    want = {}
    for d in range(80):
        cs = set(cid[off[d]:off[d + 1]].tolist())
        tot, any_ = 0.0, False
        for i in range(qs.shape[0]):
            hit = [j for j in ids[i].tolist() if j in cs]
            if hit:
                tot += max(float(qs[i].astype(np.float64) @ C[j]) for j in hit)
                any_ = True
        if any_:
            want[d] = tot
    docs, s = o.gather(qs, ids)
    assert docs.tolist() == sorted(want)
    assert np.allclose(s, [want[d] for d in docs.tolist()], rtol=0, atol=1e-12)


def pin_select_ties_doc_ascending(make):
    ix = synth.random_index(5, 5, seed=19)
    o = make(ix, 128)
    docs = np.array([9, 3, 7, 1, 5, 2], np.int32)
    s = np.array([1.0, 2.0, 1.0, 1.0, 3.0, 2.0])
    od, os_ = o.select(docs, s, 4)
    assert od.tolist() == [5, 2, 3, 1] and os_.tolist() == [3.0, 2.0, 2.0, 1.0]
    od, _ = o.select(docs, s, 10)
    assert od.tolist() == [5, 2, 3, 1, 7, 9]


def pin_short_results_padded(make):
    # fewer reachable docs than k: the row is padded with (-1, -inf)
    ix = synth.random_index(6, 50, len_max=3, seed=20)
    qs = synth.random_queries(1, 2, 2, seed=21)["queries"]
    o = make(ix, 128)
    res = o.search(qs, np.array([2], np.int32), 10, 1, 10)
    n = int((res["ids"] >= 0).sum())
    assert n <= 2 * 3 and n < 10
    assert np.all(res["ids"][n:] == -1) and np.all(np.isneginf(res["scores"][n:]))


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]

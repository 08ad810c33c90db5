"""Gap-aware comparison of a GPU ranking with the FP64 oracle's.

Where several answers are correct (near-equal scores at a cut), only what is
unique is compared exactly:
  * sorted scores, rank by rank, within a relative tolerance;
  * the id at a rank whose oracle score is separated from both neighbours by
    more than `gap`;
  * the id set of the first n when the oracle's gap at the cut exceeds `gap`;
  * every returned id is valid (in range, no duplicates, -1 only as padding)
    and its own oracle score matches the score the GPU reports for it.
"""
from __future__ import annotations

import numpy as np


def check_ranking(g_ids, g_s, o_ids, o_s, rtol, gap=1e-4, what="", exact_scores=None):
    g_ids = np.asarray(g_ids)
    o_ids = np.asarray(o_ids)
    g_s = np.asarray(g_s, np.float64)
    o_s = np.asarray(o_s, np.float64)
    n = len(o_ids)
    assert len(g_ids) == n, what
    valid_o = o_ids >= 0
    valid_g = g_ids >= 0
    assert np.array_equal(valid_o, valid_g), f"{what}: padding differs {valid_o.sum()} vs {valid_g.sum()}"
    m = int(valid_o.sum())
    assert np.all(valid_o[:m]) and not np.any(valid_o[m:]), what
    assert len(set(g_ids[:m].tolist())) == m, f"{what}: duplicate ids"
    assert np.all(np.isneginf(g_s[m:])), what
    tol = rtol * np.maximum(1.0, np.abs(o_s[:m]))
    err = np.abs(g_s[:m] - o_s[:m])
    assert np.all(err <= tol), f"{what}: score error {err.max():.3g} > tol"
    s = o_s[:m]
    for r in range(m):
        left = r == 0 or s[r - 1] - s[r] > gap
        right = r == m - 1 or s[r] - s[r + 1] > gap
        if left and right:
            assert g_ids[r] == o_ids[r], f"{what}: rank {r}: {g_ids[r]} != {o_ids[r]} (gap-separated)"
    if exact_scores is not None:
        # the oracle's own score of each id the GPU returned
        es = np.array([exact_scores[int(i)] for i in g_ids[:m]])
        assert np.all(np.abs(es - g_s[:m]) <= tol), f"{what}: a returned id's score is wrong"


def overlap(g_ids, o_ids, n=10):
    a = set(int(x) for x in g_ids[:n] if x >= 0)
    b = set(int(x) for x in o_ids[:n] if x >= 0)
    if not b:
        return 1.0
    return len(a & b) / len(b)

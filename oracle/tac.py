"""FP64 oracle of Token-Aware Clustering's centroid allotment (test infrastructure only).

Sec. 2.1, "Token-Aware Clustering": the centroid budget kappa is shared out over the token types
in four phases, then each type is clustered on its own. This module follows the four phases in
the paper's order with plain Python loops over the types, in float64, for a reader to check by
eye; it shares no code with the library.

Readings of points the paper leaves open (each is a parameter or a rule here):
* mu, tau, eps, theta (Phases 1 and 3) have no values in the paper: they are arguments.
* A type with no occurrence gets no centroid; the paper's sum over w_i runs over the active types
  (the weights exist only for them), and B is the budget left after Phase 1.
* Phase 3 with both bounds: the cap floor(n_j / theta) (at least 1, at most n_j) wins over the
  floor eps when they conflict, since a centroid needs vectors.
* Phase 4: units are added one at a time to the active type whose allotment is furthest below
  its share w_j / sum(w) * B (largest r_j = share - kappa_j, ties to the lower type id) among those
  below their cap, or removed one at a time from the active type furthest above its share
  (smallest r_j, ties to the higher type id) among those above their floor. A budget that cannot
  be met within the bounds is an error.
"""
from __future__ import annotations

import math


class AllotError(ValueError):
    pass


def spread(vectors, types, n_types):
    """Phase 2's spread s_j = (1 / n_j) sum_i ||t_{j,i} - mean_j||^2 of each type (0 for an
    absent type), in float64 with two passes over the vectors (the mean, then the squares)."""
    d = len(vectors[0]) if len(vectors) else 0
    cnt = [0] * n_types
    mean = [[0.0] * d for _ in range(n_types)]
    for v, t in zip(vectors, types):
        cnt[t] += 1
        row = mean[t]
        for k in range(d):
            row[k] += float(v[k])
    for t in range(n_types):
        if cnt[t]:
            mean[t] = [x / cnt[t] for x in mean[t]]
    acc = [0.0] * n_types
    for v, t in zip(vectors, types):
        acc[t] += sum((float(v[k]) - mean[t][k]) ** 2 for k in range(d))
    return [acc[t] / cnt[t] if cnt[t] else 0.0 for t in range(n_types)]


def allot(n, s, budget, mu, tau, eps, theta):
    """Centroids per token type, kappa_j, following Phases 1-4 of Sec. 2.1.

    n: occurrences n_j per type; s: spread s_j per type (read for active types only);
    budget: the total kappa. Returns a list of ints summing to `budget`."""
    T = len(n)
    kappa = [0] * T
    # Phase 1: tail handling - micro types (n < mu) get 1 centroid, small types (mu <= n < tau) 2
    active = []
    for j in range(T):
        if n[j] <= 0:
            continue
        if n[j] < mu:
            kappa[j] = 1
        elif n[j] < tau:
            kappa[j] = 2
        else:
            active.append(j)
    B = budget - sum(kappa)
    if B < 0:
        raise AllotError("the budget is below the tail's fixed allotment")
    # Phase 2: damped scoring w_j = sqrt(n_j) * s_j, kappa_j = floor(w_j / sum(w) * B)
    w = {}
    for j in active:
        w[j] = math.sqrt(n[j]) * s[j]
    W = 0.0
    for j in active:
        W += w[j]
    share = {}
    for j in active:
        share[j] = (w[j] / W) * B if W > 0 else 0.0
        kappa[j] = math.floor(share[j])
    # Phase 3: bounding - at least eps, at most n_j / theta vectors per centroid (the cap wins)
    lo, hi = {}, {}
    for j in active:
        hi[j] = min(n[j], max(1, math.floor(n[j] / theta)))
        lo[j] = min(eps, hi[j])
        kappa[j] = min(max(kappa[j], lo[j]), hi[j])
    # Phase 4: budget reconciliation, one centroid at a time
    delta = budget - sum(kappa)
    while delta > 0:
        best = None
        for j in active:  # ascending j: a tie keeps the lower id
            if kappa[j] < hi[j]:
                r = share[j] - kappa[j]
                if best is None or r > best[0]:
                    best = (r, j)
        if best is None:
            raise AllotError("the budget exceeds what the caps allow")
        kappa[best[1]] += 1
        delta -= 1
    while delta < 0:
        best = None
        for j in active:  # ascending j with <=: a tie moves to the higher id
            if kappa[j] > lo[j]:
                r = share[j] - kappa[j]
                if best is None or r <= best[0]:
                    best = (r, j)
        if best is None:
            raise AllotError("the budget is below what the floors require")
        kappa[best[1]] -= 1
        delta += 1
    return kappa


def speedup_lower_bound(n, s):
    """Sec. 2.1's lower bound on TAC's speed-up over k-means, sum(w) / max(w), over the types
    with n_j > 0, and the exact ratio kappa N / sum_j kappa_j n_j it bounds for the unrounded
    allotment kappa_j = w_j / sum(w) * kappa (independent of kappa)."""
    js = [j for j in range(len(n)) if n[j] > 0]
    w = [math.sqrt(n[j]) * s[j] for j in js]
    W = sum(w)
    N = sum(n[j] for j in js)
    ratio = N / sum((wj / W) * n[j] for wj, j in zip(w, js))
    return W / max(w), ratio


# ---- the clustering and encoding that follow the allotment (Sec. 2.1) ----------------------
# Plain definitions in float64 with explicit loops over points and centroids. Readings: distance
# is squared L2; a tie goes to the lower centroid (or codeword) index; a cluster left empty by an
# assignment keeps its previous centroid; the initial centroids are an input (the caller draws
# them), so every step here is deterministic.

def _sqdist(a, b):
    return sum((float(x) - float(y)) ** 2 for x, y in zip(a, b))


def assign(points, centroids):
    """Index of the nearest centroid of every point (ties to the lower index)."""
    out = []
    for p in points:
        best, bi = None, -1
        for i, c in enumerate(centroids):
            dd = _sqdist(p, c)
            if best is None or dd < best:
                best, bi = dd, i
        out.append(bi)
    return out


def inertia(points, centroids, labels):
    """Within-cluster sum of squares of Sec. 2.1's k-means objective."""
    return sum(_sqdist(p, centroids[l]) for p, l in zip(points, labels))


def lloyd(points, init, iters):
    """kappa_j-means of one token type: `iters` rounds of assignment then mean update, from the
    centroids `init`. Returns (centroids, labels of the last assignment, inertia after each
    round's update)."""
    c = [[float(x) for x in row] for row in init]
    d = len(c[0]) if c else 0
    hist = []
    labels = []
    for _ in range(iters):
        labels = assign(points, c)
        sums = [[0.0] * d for _ in c]
        cnt = [0] * len(c)
        for p, l in zip(points, labels):
            cnt[l] += 1
            for k in range(d):
                sums[l][k] += float(p[k])
        for i in range(len(c)):
            if cnt[i]:
                c[i] = [x / cnt[i] for x in sums[i]]
        hist.append(inertia(points, c, labels))
    if iters:
        labels = assign(points, c)
    return c, labels, hist


def pq_encode(vectors, centroids, labels, codebooks):
    """Residual compression of Sec. 2.1: r = t - c_a(t), rho = ||r||, r / rho split into M
    contiguous subspaces of d / M dims, each coded by its nearest codeword (ties to the lower code);
    a zero residual gets rho = 0 and code 0 everywhere. codebooks[m][j] is codeword j of subspace m.
    Returns (codes [T][M], rho [T]) with rho in float64 (the index stores it as fp16)."""
    M = len(codebooks)
    codes, rhos = [], []
    for t, l in zip(vectors, labels):
        r = [float(x) - float(y) for x, y in zip(t, centroids[l])]
        ds = len(r) // M
        rho = math.sqrt(sum(x * x for x in r))
        rhos.append(rho)
        if rho == 0.0:
            codes.append([0] * M)
            continue
        u = [x / rho for x in r]
        row = []
        for m in range(M):
            sub = u[m * ds:(m + 1) * ds]
            best, bj = None, -1
            for j, w in enumerate(codebooks[m]):
                dd = _sqdist(sub, w)
                if best is None or dd < best:
                    best, bj = dd, j
            row.append(bj)
        codes.append(row)
    return codes, rhos


def init_positions(n_j, kappa_j):
    """Initial centroids of one type: its points at positions floor((r + 1/2) n_j / kappa_j),
    r = 0 .. kappa_j - 1, in the order the points appear in the collection (evenly spaced, distinct
    as kappa_j <= n_j; deterministic, so no random draw needs to be shared)."""
    return [math.floor((r + 0.5) * n_j / kappa_j) for r in range(kappa_j)]


def cluster(vectors, types, n_types, budget, mu, tau, eps, theta, iters):
    """Token-Aware Clustering end to end (Sec. 2.1): counts and spreads per type, the allotment,
    then kappa_j-means of every type on its own from the evenly spaced initial points.
    Returns (kappa [n_types], centroids grouped by type in type order [budget][d],
    centroid type [budget], label of every vector as a global centroid id [N], -1 for a vector
    whose type received no centroid)."""
    n = [0] * n_types
    members = [[] for _ in range(n_types)]
    for i, t in enumerate(types):
        n[t] += 1
        members[t].append(i)
    s = spread(vectors, types, n_types)
    kappa = allot(n, s, budget, mu, tau, eps, theta)
    cents, ctype, labels = [], [], [-1] * len(types)
    for j in range(n_types):
        if kappa[j] == 0:
            continue
        pts = [vectors[i] for i in members[j]]
        init = [pts[p] for p in init_positions(n[j], kappa[j])]
        c, lab, _ = lloyd(pts, init, iters)
        base = len(cents)
        cents.extend(c)
        ctype.extend([j] * kappa[j])
        for i, l in zip(members[j], lab):
            labels[i] = base + l
    return kappa, cents, ctype, labels


def pq_sample_positions(n, s):
    """The training sample of the codebooks: vectors at positions floor((r + 1/2) n / s), r < s."""
    return [math.floor((r + 0.5) * n / s) for r in range(s)]


def pq_train(vectors, centroids, labels, M, sample, iters, K=256):
    """Codebooks of the residual compression (Sec. 2.1): the normalised residuals r / ||r|| of the
    sampled vectors (the zero vector for a zero residual or a label < 0), split into M subspaces of
    d / M dims, each clustered by Lloyd from its sample points at positions floor((j + 1/2) S / K),
    j < K. Returns codebooks [M][K][d / M]."""
    d = len(vectors[0])
    ds = d // M
    us = []
    for i in pq_sample_positions(len(vectors), sample):
        l = labels[i]
        if l < 0:
            us.append([0.0] * d)
            continue
        r = [float(x) - float(y) for x, y in zip(vectors[i], centroids[l])]
        rho = math.sqrt(sum(x * x for x in r))
        us.append([x / rho for x in r] if rho > 0.0 else [0.0] * d)
    books = []
    for m in range(M):
        pts = [u[m * ds:(m + 1) * ds] for u in us]
        init = [pts[p] for p in init_positions(sample, K)]
        c, _, _ = lloyd(pts, init, iters)
        books.append(c)
    return books

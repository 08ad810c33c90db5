// Token-Aware Clustering: the centroid allotment (Sec. 2.1, "Token-Aware Clustering",
// Phases 1-4), host code.
//
// The budget kappa is shared out over the token types: types with few occurrences get a fixed
// 1 or 2 centroids (Phase 1); the others get floor(w_j / sum(w) * B) with the damped weight
// w_j = sqrt(n_j) s_j (Phase 2), clamped to a floor eps and to at most n_j / theta vectors per
// centroid (Phase 3); the total is then matched to kappa exactly (Phase 4). The paper fixes
// neither the four parameters nor the reconciliation rule; this file takes these readings:
//   - a type with no occurrence gets no centroid; sum(w) runs over the active types; B is the
//     budget left after Phase 1;
//   - the cap min(n_j, max(1, floor(n_j / theta))) wins over eps when the two conflict;
//   - Phase 4 adds one centroid at a time to the active type below its cap with the largest
//     r_j = share_j - kappa_j (ties to the lower id), or removes one at a time from the active
//     type above its floor with the smallest r_j (ties to the higher id); a budget the bounds
//     cannot meet is an error.
// Every quantity is formed with the same float64 operations in the same order as a plain
// sequential reading of the phases, so the result is one well-defined integer vector; a heap
// replaces the linear search for the next type, which picks the same type.
#include <cmath>
#include <queue>
#include <vector>

#include "tachiom_internal.cuh"

namespace tachiom {

namespace {

struct Cand {
  double r;
  int32_t j;
};
// deficit: largest r first, then lower id
struct AddOrder {
  bool operator()(const Cand &a, const Cand &b) const { return a.r < b.r || (a.r == b.r && a.j > b.j); }
};
// surplus: smallest r first, then higher id
struct RemoveOrder {
  bool operator()(const Cand &a, const Cand &b) const { return a.r > b.r || (a.r == b.r && a.j < b.j); }
};

}  // namespace

}  // namespace tachiom

using namespace tachiom;

extern "C" tachiom_status tachiom_tac_allot(const int64_t *n, const double *s, int32_t n_types, int64_t budget,
                                            const tachiom_tac_params *p, int32_t *kappa) {
  if (n_types < 0 || (n_types > 0 && (!n || !s || !kappa)) || !p)
    return fail(TACHIOM_ERR_INVALID, "tac_allot: NULL argument or negative n_types");
  if (budget < 0 || p->mu < 0 || p->tau < 0 || p->eps < 0 || !(p->theta > 0.0) || !std::isfinite(p->theta))
    return fail(TACHIOM_ERR_INVALID, "tac_allot: budget, mu, tau, eps must be >= 0 and theta > 0");
  std::vector<int64_t> k(n_types, 0), lo(n_types, 0), hi(n_types, 0);
  std::vector<double> share(n_types, 0.0), w(n_types, 0.0);
  std::vector<int32_t> active;
  // Phase 1: tail handling
  int64_t tail = 0;
  for (int32_t j = 0; j < n_types; j++) {
    if (n[j] <= 0) continue;
    if (n[j] < p->mu) {
      k[j] = 1;
    } else if (n[j] < p->tau) {
      k[j] = 2;
    } else {
      if (!(s[j] >= 0.0) || !std::isfinite(s[j]))
        return fail(TACHIOM_ERR_INVALID, "tac_allot: spread of type %d is negative or not finite", j);
      active.push_back(j);
    }
    tail += k[j];
  }
  const int64_t B = budget - tail;
  if (B < 0) return fail(TACHIOM_ERR_INVALID, "tac_allot: the budget is below the tail's fixed allotment");
  // Phase 2: damped scoring
  double W = 0.0;
  for (int32_t j : active) {
    w[j] = std::sqrt((double)n[j]) * s[j];
    W += w[j];
  }
  for (int32_t j : active) {
    share[j] = W > 0.0 ? (w[j] / W) * (double)B : 0.0;
    k[j] = (int64_t)std::floor(share[j]);
  }
  // Phase 3: bounding
  int64_t total = tail;
  for (int32_t j : active) {
    const int64_t cap = (int64_t)std::floor((double)n[j] / p->theta);
    hi[j] = std::min<int64_t>(n[j], std::max<int64_t>(1, cap));
    lo[j] = std::min<int64_t>(p->eps, hi[j]);
    k[j] = std::min(std::max(k[j], lo[j]), hi[j]);
    total += k[j];
  }
  // Phase 4: reconciliation
  int64_t delta = budget - total;
  if (delta > 0) {
    std::priority_queue<Cand, std::vector<Cand>, AddOrder> q;
    for (int32_t j : active)
      if (k[j] < hi[j]) q.push({share[j] - (double)k[j], j});
    for (; delta > 0; delta--) {
      if (q.empty()) return fail(TACHIOM_ERR_INVALID, "tac_allot: the budget exceeds what the caps allow");
      const int32_t j = q.top().j;
      q.pop();
      k[j] += 1;
      if (k[j] < hi[j]) q.push({share[j] - (double)k[j], j});
    }
  } else if (delta < 0) {
    std::priority_queue<Cand, std::vector<Cand>, RemoveOrder> q;
    for (int32_t j : active)
      if (k[j] > lo[j]) q.push({share[j] - (double)k[j], j});
    for (; delta < 0; delta++) {
      if (q.empty()) return fail(TACHIOM_ERR_INVALID, "tac_allot: the budget is below what the floors require");
      const int32_t j = q.top().j;
      q.pop();
      k[j] -= 1;
      if (k[j] > lo[j]) q.push({share[j] - (double)k[j], j});
    }
  }
  for (int32_t j = 0; j < n_types; j++) {
    if (k[j] > INT32_MAX) return fail(TACHIOM_ERR_INVALID, "tac_allot: an allotment exceeds int32");
    kappa[j] = (int32_t)k[j];
  }
  return TACHIOM_OK;
}

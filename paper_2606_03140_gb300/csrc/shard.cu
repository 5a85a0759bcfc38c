// Assignment of whole subgraphs to ranks for a step sharded over several GPUs (host code only).
//
// The subgraph solves are independent units whose cost grows as the cube of the subgraph's
// orbital count (Sec. "Scalability", where the cube of the halo sizes sets the load imbalance).
// A sharded step gives every rank a set of whole subgraphs; ranks then exchange only small
// vectors (positions, charges, forces) and the collected electron count with its mu
// derivatives.  The assignment is LPT (longest processing time first; R. L. Graham, "Bounds on
// multiprocessing timing anomalies", 1969): subgraphs in descending cost, equal costs by
// ascending index, each to the rank with the least load so far, equal loads to the lowest rank.
// Its largest load is within 4/3 - 1/(3 m) of the best possible for m ranks.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <vector>

#include "../../include/sedacs.h"

extern "C" sedacs_status sedacs_shard_lpt(int32_t n_sub, const double* cost, int32_t n_ranks, int32_t* owner,
                                          double* rank_load) {
  if (n_sub < 0 || n_ranks <= 0 || (n_sub > 0 && (!cost || !owner)) || !rank_load) return SEDACS_EINVAL;
  for (int32_t i = 0; i < n_sub; ++i)
    if (!(cost[i] >= 0.0) || !std::isfinite(cost[i])) return SEDACS_EINVAL;
  std::vector<int32_t> order(n_sub);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  std::vector<double> load(n_ranks, 0.0);
  for (int32_t i : order) {
    int32_t r = 0;
    for (int32_t k = 1; k < n_ranks; ++k)
      if (load[k] < load[r]) r = k;
    owner[i] = r;
    load[r] += cost[i];
  }
  for (int32_t k = 0; k < n_ranks; ++k) rank_load[k] = load[k];
  return SEDACS_OK;
}

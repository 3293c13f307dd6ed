// Sharding of independent surfaces over ranks (one process per GPU).  The pairs of different
// surfaces never interact (every near pair belongs to one surface), so a batch of surfaces shards
// with no exchange step: each rank builds a plan from its own surfaces.  Greedy longest-processing-
// time assignment: surfaces in decreasing cost, each to the rank with the least load so far (ties to
// the lower rank), which keeps the largest load within 4/3 of the optimum.
#include <algorithm>
#include <numeric>
#include <vector>

#include "bie_internal.cuh"

using namespace bie;

extern "C" bie_status bie_shard_surfaces(int n, const double* cost, int world, int* owner, double* load) {
  if (n < 0 || world < 1 || (n > 0 && (!cost || !owner))) {
    set_error("bie_shard_surfaces: invalid arguments");
    return BIE_EINVAL;
  }
  for (int i = 0; i < n; ++i)
    if (!(cost[i] >= 0)) { set_error("bie_shard_surfaces: cost %d is negative or NaN", i); return BIE_EINVAL; }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> acc(world, 0.0);
  for (int i : order) {
    const int r = (int)(std::min_element(acc.begin(), acc.end()) - acc.begin());
    owner[i] = r;
    acc[r] += cost[i];
  }
  if (load)
    for (int r = 0; r < world; ++r) load[r] = acc[r];
  return BIE_OK;
}

// Host-side partition of one system's tree over several ranks (no GPU needed).
//
// The near pass shards over target leaves: each leaf's targets need only the
// sources of its near list (FMM list 1, Step 4 of Sec. 6.1).  Leaves are kept
// in Morton order, so contiguous leaf ranges are compact pieces of the box;
// the ranges are balanced by the issued pairs of the one-sided pass,
//   cost(leaf) = targets(leaf) x sum over near leaves X of sources(X),
// and a rank then needs, besides its own leaves' points, the points of the
// halo: the near-list leaves outside its range.  The exchange moves those
// points' densities once before the pass; every rank computes the tree from
// all coordinates (24 bytes per point), so only densities travel.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "../../include/dmk_stokes.h"

namespace {
thread_local const char* g_part_err = "";
}

extern "C" {

dmk_status_t dmk_stokes_partition_leaves(int32_t n_leaf, const int32_t* leaf_count, const int32_t* leaf_tcount,
                                         const int32_t* near_off, const int32_t* near_leaf, int32_t n_ranks,
                                         int32_t* leaf_begin, int64_t* rank_cost) {
  if (n_leaf < 0 || n_ranks < 1 || !leaf_begin || (n_leaf > 0 && (!leaf_count || !near_off || !near_leaf))) {
    g_part_err = "bad partition arguments";
    return DMK_ERR_INVALID_ARG;
  }
  // prefix sums of the per-leaf cost
  std::vector<int64_t> pre(static_cast<size_t>(n_leaf) + 1, 0);
  for (int32_t i = 0; i < n_leaf; ++i) {
    int64_t src = 0;
    for (int32_t e = near_off[i]; e < near_off[i + 1]; ++e) src += leaf_count[near_leaf[e]];
    const int64_t nt = leaf_tcount ? leaf_tcount[i] : leaf_count[i];
    pre[i + 1] = pre[i] + nt * src;
  }
  const int64_t total = pre[n_leaf];
  leaf_begin[0] = 0;
  for (int32_t r = 1; r < n_ranks; ++r) {
    // first leaf whose prefix reaches r / n_ranks of the total (ties to the left)
    const double goal = static_cast<double>(total) * r / n_ranks;
    int32_t b = static_cast<int32_t>(std::lower_bound(pre.begin(), pre.end(), static_cast<int64_t>(goal + 0.5)) -
                                     pre.begin());
    b = std::min(std::max(b, leaf_begin[r - 1]), n_leaf);
    leaf_begin[r] = b;
  }
  leaf_begin[n_ranks] = n_leaf;
  if (rank_cost)
    for (int32_t r = 0; r < n_ranks; ++r) rank_cost[r] = pre[leaf_begin[r + 1]] - pre[leaf_begin[r]];
  return DMK_OK;
}

dmk_status_t dmk_stokes_halo_leaves(int32_t n_leaf, const int32_t* near_off, const int32_t* near_leaf,
                                    int32_t begin, int32_t end, int32_t* halo, int32_t max_halo,
                                    int32_t* n_halo) {
  if (n_leaf < 0 || begin < 0 || end < begin || end > n_leaf || !n_halo || (end > begin && (!near_off || !near_leaf))) {
    g_part_err = "bad halo arguments";
    return DMK_ERR_INVALID_ARG;
  }
  std::vector<int32_t> h;
  for (int32_t i = begin; i < end; ++i)
    for (int32_t e = near_off[i]; e < near_off[i + 1]; ++e) {
      const int32_t X = near_leaf[e];
      if (X < begin || X >= end) h.push_back(X);
    }
  std::sort(h.begin(), h.end());
  h.erase(std::unique(h.begin(), h.end()), h.end());
  *n_halo = static_cast<int32_t>(h.size());
  if (halo) {
    if (static_cast<int32_t>(h.size()) > max_halo) {
      g_part_err = "halo buffer too small";
      return DMK_ERR_INVALID_ARG;
    }
    std::copy(h.begin(), h.end(), halo);
  }
  return DMK_OK;
}

}  // extern "C"

// Host-side partitioning of subdomains over the ranks of a multi-GPU run and
// the output offsets of the per-rank buffers (Sec. III Stage 1: every
// processor works on its own subdomains; the output stage writes the
// per-processor buffers one after another).
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "aeqc_internal.cuh"

using aeqc::clear_error;
using aeqc::set_error;

extern "C" int aeqc_partition_lpt(const int64_t* counts, int32_t n_groups, int32_t n_ranks,
                                  int32_t* owner, int64_t* load_out) {
  clear_error();
  AEQC_CHECK_ARG(n_groups >= 0 && n_ranks >= 1, "aeqc_partition_lpt: n_groups %d, n_ranks %d",
                 n_groups, n_ranks);
  AEQC_CHECK_ARG(n_groups == 0 || (counts && owner), "aeqc_partition_lpt: null array");
  for (int g = 0; g < n_groups; ++g)
    AEQC_CHECK_ARG(counts[g] >= 0, "aeqc_partition_lpt: count[%d] = %lld < 0", g,
                   (long long)counts[g]);
  // decreasing count, equal counts by index: a total order, so every rank
  // computes the same assignment
  std::vector<int32_t> order(n_groups);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return counts[a] > counts[b]; });
  std::vector<int64_t> load(n_ranks, 0);
  for (int32_t g : order) {
    int r = 0;
    for (int q = 1; q < n_ranks; ++q)
      if (load[q] < load[r]) r = q;  // least load, lowest rank on ties
    owner[g] = r;
    load[r] += counts[g];
  }
  if (load_out)
    for (int r = 0; r < n_ranks; ++r) load_out[r] = load[r];
  return AEQC_OK;
}

extern "C" int aeqc_exclusive_scan(const int64_t* sizes, int32_t n, int64_t* offsets) {
  clear_error();
  AEQC_CHECK_ARG(n >= 0 && offsets && (n == 0 || sizes), "aeqc_exclusive_scan: bad arguments");
  int64_t run = 0;
  offsets[0] = 0;
  for (int i = 0; i < n; ++i) {
    AEQC_CHECK_ARG(sizes[i] >= 0, "aeqc_exclusive_scan: size[%d] = %lld < 0", i,
                   (long long)sizes[i]);
    AEQC_CHECK_ARG(sizes[i] <= INT64_MAX - run, "aeqc_exclusive_scan: total overflows int64");
    run += sizes[i];
    offsets[i + 1] = run;
  }
  return AEQC_OK;
}

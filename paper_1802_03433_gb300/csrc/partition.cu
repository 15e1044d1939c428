// Row partition of a P1 mesh for assembly on several GPUs with no exchange.
//
// The paper assembles one mesh on one GPU, one thread per (element, entry)
// pair (Sec. 5, Fig. 2).  A mesh too large for one GPU, or one spread over
// several for speed, splits by rows: part k owns a contiguous range of node
// ids and assembles, on its own GPU, every element with a vertex in that
// range - its own elements plus the ghost layer around them, which the
// neighbouring parts assemble too.  Every row of an owned node then receives
// all of its contributions on the part that owns it, so the owned rows are
// complete and need nothing from the other parts.
//
// Host code only (no CUDA call): the partition is set up before the device
// work and also serves hosts without a GPU.
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace fea;

extern "C" fea_status fea_partition(const int32_t* tets, int64_t n_elems, int64_t n_nodes, int32_t nparts,
                                    int32_t part, int64_t* node_lo, int64_t* node_hi, int64_t* n_sub_elems,
                                    int64_t* n_sub_nodes, int32_t* elems, int32_t* nodes, int32_t* sub_tets) {
  if (n_nodes <= 0 || n_nodes > (int64_t)INT32_MAX || n_elems < 0 || n_elems > (int64_t)INT32_MAX / 10)
    return fail(FEA_ERR_ARG, "fea_partition: n_nodes or n_elems out of range");
  if (n_elems > 0 && !tets) return fail(FEA_ERR_ARG, "fea_partition: tets is NULL");
  if (nparts < 1 || part < 0 || part >= nparts) return fail(FEA_ERR_ARG, "fea_partition: need 0 <= part < nparts");
  if (!node_lo || !node_hi || !n_sub_elems || !n_sub_nodes)
    return fail(FEA_ERR_ARG, "fea_partition: NULL size output");
  const int64_t lo = n_nodes * part / nparts, hi = n_nodes * (part + 1) / nparts;
  // elements with a vertex in [lo, hi), ascending; the nodes they use plus
  // the owned range, ascending
  std::vector<uint8_t> used((size_t)n_nodes, 0);
  for (int64_t v = lo; v < hi; ++v) used[v] = 1;
  int64_t ne = 0;
  for (int64_t e = 0; e < n_elems; ++e) {
    bool mine = false;
    for (int a = 0; a < 4; ++a) {
      const int32_t v = tets[a * n_elems + e];
      if (v < 0 || (int64_t)v >= n_nodes) return fail(FEA_ERR_INDEX, "fea_partition: node index out of range");
      mine = mine || (v >= lo && v < hi);
    }
    if (!mine) continue;
    for (int a = 0; a < 4; ++a) used[tets[a * n_elems + e]] = 1;
    if (elems) elems[ne] = (int32_t)e;
    ++ne;
  }
  int64_t nn = 0;
  std::vector<int32_t> local;
  if (sub_tets) local.assign((size_t)n_nodes, -1);
  for (int64_t v = 0; v < n_nodes; ++v)
    if (used[v]) {
      if (nodes) nodes[nn] = (int32_t)v;
      if (sub_tets) local[v] = (int32_t)nn;
      ++nn;
    }
  if (sub_tets) {
    // the selected elements again, in the same ascending order
    int64_t k = 0;
    for (int64_t e = 0; e < n_elems; ++e) {
      bool mine = false;
      for (int a = 0; a < 4; ++a) {
        const int32_t v = tets[a * n_elems + e];
        mine = mine || (v >= lo && v < hi);
      }
      if (!mine) continue;
      for (int a = 0; a < 4; ++a) sub_tets[a * ne + k] = local[tets[a * n_elems + e]];
      ++k;
    }
  }
  *node_lo = lo;
  *node_hi = hi;
  *n_sub_elems = ne;
  *n_sub_nodes = nn;
  return FEA_OK;
}

// Independent meshes of a batch over several GPUs: longest processing time
// first (LPT, Graham's list-scheduling rule) on the callers' cost estimates.
// The meshes go in order of decreasing cost (equal costs by index), each to
// the part with the least cost so far (equal loads: the lowest part).  No
// mesh is split, so the parts need no exchange.
extern "C" fea_status fea_partition_batch(const double* cost, int32_t n, int32_t nparts, int32_t* part_of,
                                          double* load) {
  if (n < 0 || nparts < 1) return fail(FEA_ERR_ARG, "fea_partition_batch: need n >= 0 and nparts >= 1");
  if (n > 0 && (!cost || !part_of)) return fail(FEA_ERR_ARG, "fea_partition_batch: cost or part_of is NULL");
  for (int32_t i = 0; i < n; ++i)
    if (!(cost[i] >= 0.0) || cost[i] == HUGE_VAL)
      return fail(FEA_ERR_ARG, "fea_partition_batch: costs must be finite and >= 0");
  std::vector<int32_t> order((size_t)n);
  for (int32_t i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  std::vector<double> sum((size_t)nparts, 0.0);
  for (int32_t i : order) {
    int32_t best = 0;
    for (int32_t p = 1; p < nparts; ++p)
      if (sum[p] < sum[best]) best = p;
    part_of[i] = best;
    sum[best] += cost[i];
  }
  if (load)
    for (int32_t p = 0; p < nparts; ++p) load[p] = sum[p];
  return FEA_OK;
}

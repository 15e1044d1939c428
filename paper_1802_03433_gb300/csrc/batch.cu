// Batched assembly: many independent meshes (uneven sizes, P1 and P2) in one
// CUDA-graph launch.
//
// The graph holds two branches, one per element order, that may run at the
// same time.  Each branch is a persistent element kernel walking a static
// list of (mesh, element tile) work items, each CTA taking items b, b + grid,
// b + 2 grid, ..., followed by the scatter kernels, one CTA per (mesh, row
// tile) item.  Element items are sorted longest first
// (longest-processing-time order); the P2 branch is issued first, and the P1
// kernels take the SMs that the P2 element kernel's tail leaves idle.  Each
// work item runs the same per-element and per-row-tile device code as the
// single-mesh path (including the bulk-copy scatter over the tiled layout),
// so every mesh's values are bitwise those of fea_assemble.  The elements per
// work item and the grid of each element kernel are chosen by an autotuner
// (fea_batch_tune) that times candidate configurations on the device.  Every
// pattern, map and scratch buffer is built before the graph is captured: a
// replay allocates nothing and never synchronises.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "elem_kernels.cuh"
#include "gather.cuh"
#include "gather_tiled.cuh"

namespace fea {
namespace {

struct BMesh {
  ElemArgs el;
  GatherArgs ga;   // incidence-order scatter
  TiledArgs tg;    // bulk-copy scatter over the tiled layout (tiled != 0)
  int32_t tiled;
  int32_t order;
  int32_t mass;
  int32_t rows_per_tile;
};

struct BItem {
  int32_t mesh;
  int32_t first;  // element index, or row-tile index
  int32_t count;  // elements in the tile (element items)
};

constexpr int BT = 128;

// One element kernel per order: a P1 body compiled beside the P2 body would
// run at the P2 body's register count (168 against 72 per thread, 3 against
// 7 resident CTAs per SM).  The mesh's arguments come from global memory and
// stay in registers across the element loop (the single-mesh kernels read
// theirs from the constant bank), which costs 20-40 registers per thread.
// Each kernel is built twice: with the compiler's register count (variant 0;
// P2 with the sine load: 180, two resident CTAs per SM) and capped to keep
// the residency of the single-mesh kernel (variant 1: three CTAs per SM for
// P2, six for P1, at the price of a few spilled bytes).  P2 with the sine
// load has a third form, k_batch_elem_roles (variant 2).  The autotuner
// picks.
template <int ORDER, int VARIANT>
constexpr int batch_elem_min_blocks() { return VARIANT == 0 ? 1 : ORDER == 2 ? 3 : 6; }

template <int ORDER, int LOAD, int NP, int VARIANT>
__global__ void __launch_bounds__(BT, batch_elem_min_blocks<ORDER, VARIANT>()) k_batch_elem(const BMesh* __restrict__ M, const BItem* __restrict__ items,
                                                   int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BMesh& m = M[w.mesh];
    const int64_t end = (int64_t)w.first + w.count;
    if (m.mass) {
      for (int64_t e = w.first + threadIdx.x; e < end; e += BT) elem_scalar_body<ORDER, true, LOAD, NP, double>(m.el, e);
    } else {
      for (int64_t e = w.first + threadIdx.x; e < end; e += BT)
        elem_scalar_body<ORDER, false, LOAD, NP, double>(m.el, e);
    }
  }
}

// Scatter kernels per element order (NB = 4 or 10), one CTA per row-tile
// item (a persistent loop here costs ~60 registers per thread, i.e. a third
// of the resident CTAs, for no gain: the tiles are already uniform).  Meshes
// whose pattern has the tiled layout take the bulk-copy scatter of
// gather_tiled.cuh, the others the incidence-order one of gather.cuh (two
// kernels, as one kernel holding both bodies needs the registers of the
// larger); both give the same bits.
template <int NB>
__global__ void __launch_bounds__(BT) k_batch_gather(const BMesh* __restrict__ M, const BItem* __restrict__ items,
                                                     int nitems, int64_t) {
  extern __shared__ double acc[];
  if ((int)blockIdx.x >= nitems) return;
  const BItem w = items[blockIdx.x];
  gather_tile<NB, 1, double>(M[w.mesh].ga, w.first, M[w.mesh].rows_per_tile, acc);
}

// span_cap: the accumulator capacity (doubles) of this launch's shared-memory
// layout, at least the CSR span of every tile it is given.
template <int NB, int STAGES>
__global__ void __launch_bounds__(BT) k_batch_gather_tiled(const BMesh* __restrict__ M,
                                                           const BItem* __restrict__ items, int nitems,
                                                           int64_t span_cap) {
  extern __shared__ __align__(128) unsigned char sm[];
  if ((int)blockIdx.x >= nitems) return;
  const BItem w = items[blockIdx.x];
  TiledArgs G = M[w.mesh].tg;
  G.span_cap = span_cap;
  gather_tiled_tile<NB, double, STAGES>(G, w.first, sm);
}

// Scatter item groups, in launch order, per order (P2, then P1): tiled tiles
// of the heavy class (CSR span above half the mesh's widest), tiled tiles of
// the light class, incidence-order tiles.  The light class's accumulator is
// about half the heavy one's, which leaves room for one more resident CTA
// per SM (as in the single-mesh scatter).
constexpr int NGROUPS = 6;
enum { CLS_HEAVY = 0, CLS_LIGHT = 1, CLS_INCIDENCE = 2 };
inline int gather_group(int order, int cls) { return (order == 2 ? 0 : 3) + cls; }

using GatherKernel = void (*)(const BMesh*, const BItem*, int, int64_t);

template <int NB>
GatherKernel tiled_kernel(int stages) {
  if (stages == 2) return k_batch_gather_tiled<NB, 2>;
  if (stages == 4) return k_batch_gather_tiled<NB, 4>;
  return k_batch_gather_tiled<NB, 3>;
}

using ElemKernel = void (*)(const BMesh*, const BItem*, int);

// Matrix warps and load warps (elem_roles_body) for the sine load: each item's
// elements are taken twice, by the CTA's first BT threads for the local matrix
// and by the next BT for the local load (variant 2, sine loads only).  Held
// to three CTAs per SM like the single-mesh form: the persistent loop spills
// more here (about 420 bytes at 80 registers), and the residency still wins
// (256-mesh batch 9.0 -> 8.5 ms against two CTAs at 128 registers).
template <int ORDER, int LOAD, int NP>
__global__ void __launch_bounds__(2 * BT, 3) k_batch_elem_roles(const BMesh* __restrict__ M,
                                                              const BItem* __restrict__ items, int nitems) {
  const bool matrix = threadIdx.x < BT;
  const int lane = threadIdx.x % BT;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BMesh& m = M[w.mesh];
    const int64_t end = (int64_t)w.first + w.count;
    if (m.mass) {
      for (int64_t e = w.first + lane; e < end; e += BT) elem_roles_body<ORDER, true, LOAD, NP>(m.el, e, matrix);
    } else {
      for (int64_t e = w.first + lane; e < end; e += BT) elem_roles_body<ORDER, false, LOAD, NP>(m.el, e, matrix);
    }
  }
}

constexpr int ELEM_VARIANTS = 3;
inline int variant_threads(int v) { return v == 2 ? 2 * BT : BT; }

template <int ORDER, int NP, int VARIANT>
ElemKernel elem_kernel_for(int load) {
  if (load == LOAD_NONE) return k_batch_elem<ORDER, LOAD_NONE, 1, VARIANT>;
  return load == LOAD_SIN ? k_batch_elem<ORDER, LOAD_SIN, NP, VARIANT> : k_batch_elem<ORDER, LOAD_CONST, NP, VARIANT>;
}

template <int ORDER, int NP>
void elem_kernels_for(int load, ElemKernel ek[ELEM_VARIANTS]) {
  ek[0] = elem_kernel_for<ORDER, NP, 0>(load);
  ek[1] = elem_kernel_for<ORDER, NP, 1>(load);
  // the roles kernel only where there is a sine load to split off (P2)
  ek[2] = nullptr;
  if constexpr (ORDER == 2)
    if (load == LOAD_SIN) ek[2] = k_batch_elem_roles<ORDER, LOAD_SIN, NP>;
}

// Element kernels of the supported (P1, P2) rules, indexed by order and variant
// (NULL where a variant does not apply).
bool pick_elem_kernels(int load, int np1, int np2, ElemKernel ek[3][ELEM_VARIANTS]) {
  for (int v = 0; v < ELEM_VARIANTS; ++v) ek[0][v] = nullptr;
  if (np1 == 4) elem_kernels_for<1, 4>(load, ek[1]);
  else if (np1 == 11) elem_kernels_for<1, 11>(load, ek[1]);
  else return false;
  if (np2 == 4) elem_kernels_for<2, 4>(load, ek[2]);
  else if (np2 == 11) elem_kernels_for<2, 11>(load, ek[2]);
  else return false;
  return (np1 == 4 && np2 == 11) || (np1 == 11 && np2 == 11) || (np1 == 4 && np2 == 4);
}

}  // namespace
}  // namespace fea

using namespace fea;

struct fea_batch {
  int n = 0;
  std::vector<fea_mesh*> meshes;
  std::vector<fea_form> forms;
  std::vector<BMesh> host;
  BMesh* d_mesh = nullptr;
  BItem* d_eitems = nullptr;     // element tiles, P2 first, then P1
  BItem* d_gitems = nullptr;     // row tiles by scatter group (gather_group)
  int n_eitems = 0, n_gitems = 0;
  int ecount[3] = {0, 0, 0};           // element items per order
  int gcount[NGROUPS] = {};           // row-tile items per group
  void* pool = nullptr;  // local rows and loads of every mesh
  size_t smem[NGROUPS] = {};          // scatter shared memory per CTA, by group
  GatherKernel gk[NGROUPS] = {};      // scatter kernel per group (stage count of the tiled groups)
  int64_t span_cap[NGROUPS] = {};     // accumulator capacity of the tiled groups
  std::vector<std::vector<uint8_t>> heavy;  // per mesh: tile -> heavy class (tiled meshes)
  int load = 0, np1 = 4, np2 = 11;
  ElemKernel ek[3][ELEM_VARIANTS] = {};  // by order and register variant
  int variant[3] = {1, 1, 1};          // the variant launched, by order
  int elem_tile = 256, gather_grid = 0;
  int elem_grid[3] = {0, 0, 0};        // persistent element-kernel CTAs, by order (0: one CTA per item)
  int sms = 0;
  bool bound = false;
  cudaStream_t cap = nullptr;
  cudaStream_t side = nullptr;         // the P1 branch (P2 runs on the launch stream)
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

fea_status build_items(fea_batch* b) {
  std::vector<std::pair<int64_t, BItem>> ei, gi;
  for (int k = 0; k < b->n; ++k) {
    const fea_mesh* m = b->meshes[k];
    const int order = b->forms[k].order;
    const int64_t E = m->n_elems;
    // P2 items first (a P2 element costs ~3x a P1 element), each order's
    // items longest first
    const int64_t key = order == 2 ? (int64_t(1) << 40) : 0;
    for (int64_t f = 0; f < E; f += b->elem_tile) {
      const int32_t cnt = (int32_t)std::min<int64_t>(b->elem_tile, E - f);
      ei.push_back({key + cnt, BItem{k, (int32_t)f, cnt}});
    }
    const Pattern* P = m->pat[order][1];
    const int64_t tiles = (P->ndof + P->rows_per_tile - 1) / P->rows_per_tile;
    for (int64_t t = 0; t < tiles; ++t) {
      const int cls = !b->host[k].tiled ? CLS_INCIDENCE : b->heavy[k][t] ? CLS_HEAVY : CLS_LIGHT;
      gi.push_back({NGROUPS - gather_group(order, cls), BItem{k, (int32_t)t, cls}});
    }
  }
  auto by_cost = [](const std::pair<int64_t, BItem>& a, const std::pair<int64_t, BItem>& c) {
    return a.first > c.first;
  };
  std::stable_sort(ei.begin(), ei.end(), by_cost);
  std::stable_sort(gi.begin(), gi.end(), by_cost);
  std::vector<BItem> he, hg;
  for (auto& p : ei) he.push_back(p.second);
  for (auto& p : gi) hg.push_back(p.second);
  if (b->d_eitems) cudaFree(b->d_eitems);
  if (b->d_gitems) cudaFree(b->d_gitems);
  b->d_eitems = b->d_gitems = nullptr;
  FEA_CUDA(cudaMalloc(&b->d_eitems, sizeof(BItem) * std::max<size_t>(1, he.size())));
  FEA_CUDA(cudaMalloc(&b->d_gitems, sizeof(BItem) * std::max<size_t>(1, hg.size())));
  if (!he.empty()) FEA_CUDA(cudaMemcpy(b->d_eitems, he.data(), sizeof(BItem) * he.size(), cudaMemcpyHostToDevice));
  if (!hg.empty()) FEA_CUDA(cudaMemcpy(b->d_gitems, hg.data(), sizeof(BItem) * hg.size(), cudaMemcpyHostToDevice));
  b->n_eitems = (int)he.size();
  b->n_gitems = (int)hg.size();
  b->ecount[0] = b->ecount[1] = b->ecount[2] = 0;
  for (const BItem& w : he) ++b->ecount[b->forms[w.mesh].order];
  for (int g = 0; g < NGROUPS; ++g) b->gcount[g] = 0;
  for (const BItem& w : hg) ++b->gcount[gather_group(b->forms[w.mesh].order, w.count)];
  return FEA_OK;
}

// Two independent branches: the P2 meshes (element kernel, then their
// scatter) on s and the P1 meshes on the side stream, forked from and joined
// back into s.  The meshes of the two branches share no output, so the
// branches may overlap: the P1 kernels fill the SMs the P2 element kernel's
// tail leaves idle.
fea_status launch_phases(fea_batch* b, cudaStream_t s) {
  FEA_CUDA(cudaEventRecord(b->fork_ev, s));
  FEA_CUDA(cudaStreamWaitEvent(b->side, b->fork_ev, 0));
  int first = 0;  // items of group g start after those of groups 0 .. g-1
  for (int order = 2; order >= 1; --order) {
    cudaStream_t st = order == 2 ? s : b->side;
    const int e_first = order == 2 ? 0 : b->ecount[2];
    if (b->ecount[order] > 0) {
      const int grid = b->elem_grid[order] > 0 ? b->elem_grid[order] : b->ecount[order];
      const int v = b->variant[order];
      b->ek[order][v]<<<grid, variant_threads(v), 0, st>>>(b->d_mesh, b->d_eitems + e_first, b->ecount[order]);
    }
    for (int g = gather_group(order, 0), ge = g + 3; g < ge; ++g) {
      if (b->gcount[g] > 0)
        b->gk[g]<<<b->gcount[g], BT, b->smem[g], st>>>(b->d_mesh, b->d_gitems + first, b->gcount[g],
                                                        b->span_cap[g]);
      first += b->gcount[g];
    }
  }
  FEA_CUDA(cudaGetLastError());
  FEA_CUDA(cudaEventRecord(b->join_ev, b->side));
  FEA_CUDA(cudaStreamWaitEvent(s, b->join_ev, 0));
  return FEA_OK;
}

fea_status rebuild_graph(fea_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  cudaGraph_t g = nullptr;
  FEA_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  fea_status st = launch_phases(b, b->cap);
  cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (st != FEA_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  FEA_CUDA(e);
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  FEA_CUDA(e);
  return FEA_OK;
}

}  // namespace

extern "C" {

fea_status fea_batch_create(fea_mesh* const* meshes, int32_t n, const fea_form* forms, const fea_quadrature* quads,
                            int32_t f_kind, void* stream, fea_batch** out) {
  if (!out) return fail(FEA_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n <= 0 || !meshes || !forms || !quads) return fail(FEA_ERR_ARG, "empty batch or NULL array");
  if (f_kind < FEA_LOAD_NONE || f_kind > FEA_LOAD_SINPROD) return fail(FEA_ERR_ARG, "unknown load kind");
  int np1 = 0, np2 = 0;
  for (int k = 0; k < n; ++k) {
    if (!meshes[k]) return fail(FEA_ERR_ARG, "NULL mesh in batch");
    if (meshes[k]->nvert != 4) return fail(FEA_ERR_ARG, "batches hold tetrahedral meshes");
    if (forms[k].kind == FEA_ELASTICITY) return fail(FEA_ERR_ARG, "batches hold scalar forms");
    if (forms[k].order != FEA_P1 && forms[k].order != FEA_P2) return fail(FEA_ERR_ARG, "bad order");
    if (quads[k].prec != FEA_FP64) return fail(FEA_ERR_ARG, "batches run in FP64");
    int& np = forms[k].order == 1 ? np1 : np2;
    if (np && np != quads[k].npts) return fail(FEA_ERR_ARG, "all meshes of one order must share the rule");
    np = quads[k].npts;
  }
  np1 = np1 ? np1 : 4;
  np2 = np2 ? np2 : 11;
  ElemKernel ek[3][ELEM_VARIANTS];
  if (!pick_elem_kernels(f_kind, np1, np2, ek))
    return fail(FEA_ERR_ARG, "supported (P1, P2) rules: (4, 11), (11, 11), (4, 4)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  fea_batch* b = new fea_batch();
  b->n = n;
  for (int o = 0; o < 3; ++o)
    for (int v = 0; v < ELEM_VARIANTS; ++v) b->ek[o][v] = ek[o][v];
  b->load = f_kind;
  b->np1 = np1;
  b->np2 = np2;
  b->meshes.assign(meshes, meshes + n);
  b->forms.assign(forms, forms + n);
  fea_status st = FEA_OK;
  do {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    size_t bytes = 0;
    std::vector<size_t> lm_off(n), fl_off(n);
    int max_rows[NGROUPS] = {};
    b->heavy.assign(n, {});
    for (int k = 0; k < n && st == FEA_OK; ++k) {
      const int order = forms[k].order;
      if ((st = build_pattern(meshes[k], order, 1, s)) != FEA_OK) break;
      if ((st = refuse_long_rows(meshes[k]->base[order], "fea_batch_create")) != FEA_OK) break;
      const Pattern* P = meshes[k]->pat[order][1];
      const int nb = order == 1 ? 4 : 10;
      const bool tiled = use_tiled(meshes[k], P);
      // local rows at tiled positions (npos, padding included) or incidence order
      const size_t nrows = tiled ? (size_t)P->npos : (size_t)meshes[k]->n_elems * nb;
      lm_off[k] = bytes;
      bytes += (nrows * lstride(nb, 8) * 8 + 255) / 256 * 256;
      fl_off[k] = bytes;
      bytes += (nrows * 8 + 255) / 256 * 256;
      if (P->rows_per_tile > BT) st = fail(FEA_ERR_ARG, "row tile taller than the batch CTA");
      if (!tiled) {
        const int g = gather_group(order, CLS_INCIDENCE);
        b->smem[g] = std::max(b->smem[g], (size_t)P->max_tile_nnz * 8);
        continue;
      }
      // the pattern's tile classes (heavy tiles first in class_list); one
      // class (heavy) when the pattern has no split
      const int64_t ntiles = (P->ndof + P->rows_per_tile - 1) / P->rows_per_tile;
      std::vector<uint8_t>& hv = b->heavy[k];
      const bool split = P->class_list && P->n_heavy > 0 && P->n_light > 0;
      hv.assign(ntiles, split ? 0 : 1);
      if (split) {
        std::vector<int32_t> list(P->n_heavy);
        cudaError_t ce = cudaMemcpy(list.data(), P->class_list, P->n_heavy * sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (ce != cudaSuccess) {
          st = cuda_fail(ce, "tile classes");
          break;
        }
        for (int32_t t : list) hv[t] = 1;
      }
      const int gh = gather_group(order, CLS_HEAVY), gl = gather_group(order, CLS_LIGHT);
      b->span_cap[gh] = std::max<int64_t>(b->span_cap[gh], split ? P->heavy_span : P->max_tile_nnz);
      max_rows[gh] = std::max(max_rows[gh], P->rows_per_tile);
      if (split) {
        b->span_cap[gl] = std::max<int64_t>(b->span_cap[gl], P->light_span);
        max_rows[gl] = std::max(max_rows[gl], P->rows_per_tile);
      }
    }
    if (st != FEA_OK) break;
    for (int g = 0; g < NGROUPS; ++g) {
      const int nb = g < 3 ? 10 : 4;
      if (g % 3 == CLS_INCIDENCE) {
        b->gk[g] = nb == 10 ? k_batch_gather<10> : k_batch_gather<4>;
      } else {
        // the single-mesh scatter's stage choice, for the group's widest tile
        const int stages = tiled_stages_auto(nb, false, std::max(max_rows[g], 1), b->span_cap[g]);
        b->gk[g] = nb == 10 ? tiled_kernel<10>(stages) : tiled_kernel<4>(stages);
        if (max_rows[g] > 0)
          b->smem[g] = nb == 10 ? Tiled<10, double>::smem_bytes(max_rows[g], b->span_cap[g], stages)
                                : Tiled<4, double>::smem_bytes(max_rows[g], b->span_cap[g], stages);
      }
      if (b->smem[g] > 227 * 1024) st = fail(FEA_ERR_OVERFLOW, "row tile too large for the batch scatter");
    }
    if (st != FEA_OK) break;
    if (cudaMalloc(&b->pool, std::max<size_t>(bytes, 256)) != cudaSuccess) {
      cudaGetLastError();
      st = fail(FEA_ERR_NOMEM, "batch scratch of " + std::to_string(bytes) + " bytes");
      break;
    }
    b->host.resize(n);
    for (int k = 0; k < n; ++k) {
      fea_mesh* m = meshes[k];
      const int order = forms[k].order;
      const Base* B = m->base[order];
      const Pattern* P = m->pat[order][1];
      BMesh& d = b->host[k];
      d = BMesh{};
      d.order = order;
      d.mass = forms[k].kind == FEA_DIFFUSION_MASS && forms[k].mass_coef != 0.0;
      d.rows_per_tile = P->rows_per_tile;
      d.el.x = m->x;
      d.el.y = m->y;
      d.el.z = m->z;
      d.el.tets = m->tets;
      d.el.N = m->n_nodes;
      d.el.E = m->n_elems;
      d.el.e0 = 0;
      d.el.e1 = m->n_elems;
      d.el.kappa_const = 1.0;
      d.el.mass = forms[k].mass_coef;
      d.tiled = use_tiled(m, P);
      d.el.ipos = d.tiled ? P->tpos : B->ipos;
      d.el.Lm = static_cast<char*>(b->pool) + lm_off[k];
      d.el.Fl = f_kind != FEA_LOAD_NONE ? static_cast<char*>(b->pool) + fl_off[k] : nullptr;
      d.el.err = m->err;
      d.ga.ndof = P->ndof;
      d.ga.row_ptr = P->row_ptr;
      d.ga.inc_ptr = B->inc_ptr;
      d.ga.slot = B->slot;
      d.ga.Lm = d.el.Lm;
      d.ga.Fl = d.el.Fl;
      d.ga.err = m->err;
      d.tg.ndof = P->ndof;
      d.tg.rows = P->rows_per_tile;
      d.tg.span_cap = P->max_tile_nnz;
      d.tg.row_ptr = P->row_ptr;
      d.tg.inc_ptr = B->inc_ptr;
      d.tg.tile_base = P->tile_base;
      d.tg.tile_steps = P->tile_steps;
      d.tg.tslot = P->tslot;
      d.tg.Lm = d.el.Lm;
      d.tg.Fl = d.el.Fl;
      d.tg.err = m->err;
    }
    if (cudaMalloc(&b->d_mesh, sizeof(BMesh) * n) != cudaSuccess) {
      cudaGetLastError();
      st = fail(FEA_ERR_NOMEM, "batch descriptors");
      break;
    }
    cudaError_t ea = cudaSuccess;
    // groups that share a kernel (heavy and light) opt in to the larger size
    for (int g = 0; g < NGROUPS && ea == cudaSuccess; ++g) {
      size_t need = 0;
      for (int h = 0; h < NGROUPS; ++h)
        if (b->gk[h] == b->gk[g]) need = std::max(need, b->smem[h]);
      if (need > 48 * 1024)
        ea = cudaFuncSetAttribute(b->gk[g], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    }
    if (ea != cudaSuccess) {
      st = cuda_fail(ea, "batch scatter shared memory");
      break;
    }
    // persistent grids: every CTA of each element kernel resident at once
    for (int o = 1; o <= 2 && ea == cudaSuccess; ++o) {
      int per_sm = 0;
      ea = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b->ek[o][b->variant[o]],
                                                         variant_threads(b->variant[o]), 0);
      b->elem_grid[o] = std::max(1, per_sm) * b->sms;
    }
    if (ea != cudaSuccess) {
      st = cuda_fail(ea, "element kernel occupancy");
      break;
    }
    if ((st = build_items(b)) != FEA_OK) break;
    b->gather_grid = b->n_gitems;
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) st = cuda_fail(e, "batch streams and events");
  } while (0);
  if (st != FEA_OK) {
    fea_batch_destroy(b);
    return st;
  }
  *out = b;
  return FEA_OK;
}

fea_status fea_batch_bind(fea_batch* b, const fea_coeffs* coeffs, double* const* values, double* const* rhs) {
  if (!b || !coeffs || !values) return fail(FEA_ERR_ARG, "NULL argument");
  for (int k = 0; k < b->n; ++k) {
    if (!values[k]) return fail(FEA_ERR_ARG, "NULL values pointer in batch");
    if (coeffs[k].f_kind != b->load) return fail(FEA_ERR_ARG, "load kind differs from the batch's");
    BMesh& d = b->host[k];
    d.el.kappa = coeffs[k].kappa;
    d.el.kappa_const = coeffs[k].kappa_const;
    for (int i = 0; i < 4; ++i) d.el.fp[i] = coeffs[k].f_param[i];
    d.ga.values = values[k];
    d.ga.rhs = rhs ? rhs[k] : nullptr;
    if (!d.ga.rhs) d.ga.Fl = nullptr;
    else d.ga.Fl = d.el.Fl;
    d.tg.values = d.ga.values;
    d.tg.rhs = d.ga.rhs;
    d.tg.Fl = d.ga.Fl;
  }
  FEA_CUDA(cudaMemcpy(b->d_mesh, b->host.data(), sizeof(BMesh) * b->n, cudaMemcpyHostToDevice));
  b->bound = true;
  return FEA_OK;
}

fea_status fea_batch_assemble(fea_batch* b, void* stream) {
  if (!b) return fail(FEA_ERR_ARG, "batch is NULL");
  if (!b->bound) return fail(FEA_ERR_STATE, "fea_batch_bind first");
  NvtxRange range("fea_batch_assemble");
  if (!b->exec) FEA_TRY(rebuild_graph(b));
  FEA_CUDA(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
  return FEA_OK;
}

fea_status fea_batch_tune(fea_batch* b, void* stream, int32_t* params) {
  if (!b) return fail(FEA_ERR_ARG, "batch is NULL");
  if (!b->bound) return fail(FEA_ERR_STATE, "fea_batch_bind first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int tiles[] = {128, 256, 512, 1024, 2048};
  const int egrid[] = {0, 2, 3, 4, 6, 8, 16};  // x SMs
  cudaEvent_t a, c;
  FEA_CUDA(cudaEventCreate(&a));
  FEA_CUDA(cudaEventCreate(&c));
  auto time_it = [&](float* best) -> fea_status {
    *best = 1e30f;
    FEA_TRY(launch_phases(b, s));  // warm-up
    for (int r = 0; r < 3; ++r) {
      FEA_CUDA(cudaEventRecord(a, s));
      FEA_TRY(launch_phases(b, s));
      FEA_CUDA(cudaEventRecord(c, s));
      FEA_CUDA(cudaEventSynchronize(c));
      float ms = 0.f;
      FEA_CUDA(cudaEventElapsedTime(&ms, a, c));
      *best = std::min(*best, ms);
    }
    return FEA_OK;
  };
  // Coordinate search: elements per work item x P2 element-kernel CTAs (P1
  // at full residency), then the P2 register variant x its CTAs, then the P1
  // variant x its CTAs.  A grid of 0 launches one CTA per work item.
  fea_status st = FEA_OK;
  float best = 1e30f, ms = 0.f;
  auto try_config = [&](bool* better) -> fea_status {
    FEA_TRY(time_it(&ms));
    *better = ms < best;
    if (*better) best = ms;
    return FEA_OK;
  };
  int bt = b->elem_tile, bg[3] = {0, b->elem_grid[1], b->elem_grid[2]}, bv[3] = {0, b->variant[1], b->variant[2]};
  bool better = false;
  for (int t : tiles) {
    b->elem_tile = t;
    if ((st = build_items(b)) != FEA_OK) break;
    for (int g : egrid) {
      b->elem_grid[2] = g * b->sms;
      if ((st = try_config(&better)) != FEA_OK) break;
      if (better) {
        bt = t;
        bg[2] = b->elem_grid[2];
      }
    }
    if (st != FEA_OK) break;
  }
  if (st == FEA_OK) {
    b->elem_tile = bt;
    b->elem_grid[2] = bg[2];
    st = build_items(b);
  }
  for (int order = 2; order >= 1 && st == FEA_OK; --order) {
    for (int v = 0; v < ELEM_VARIANTS && st == FEA_OK; ++v) {
      if (!b->ek[order][v]) continue;
      b->variant[order] = v;
      for (int g : egrid) {
        b->elem_grid[order] = g * b->sms;
        if ((st = try_config(&better)) != FEA_OK) break;
        if (better) {
          bv[order] = v;
          bg[order] = b->elem_grid[order];
        }
      }
    }
    b->variant[order] = bv[order];
    b->elem_grid[order] = bg[order];
  }
  cudaEventDestroy(a);
  cudaEventDestroy(c);
  FEA_TRY(st);
  b->gather_grid = b->n_gitems;
  FEA_TRY(rebuild_graph(b));
  if (params) {
    params[0] = b->elem_tile;
    params[1] = b->elem_grid[2] > 0 ? b->elem_grid[2] : b->ecount[2];
    params[2] = b->elem_grid[1] > 0 ? b->elem_grid[1] : b->ecount[1];
    params[3] = b->gather_grid;
    params[4] = b->variant[2];
    params[5] = b->variant[1];
  }
  return FEA_OK;
}

fea_status fea_batch_destroy(fea_batch* b) {
  if (!b) return FEA_OK;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->join_ev) cudaEventDestroy(b->join_ev);
  if (b->d_mesh) cudaFree(b->d_mesh);
  if (b->d_eitems) cudaFree(b->d_eitems);
  if (b->d_gitems) cudaFree(b->d_gitems);
  if (b->pool) cudaFree(b->pool);
  delete b;
  return FEA_OK;
}

}  // extern "C"

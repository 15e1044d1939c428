// Batched assembly: many independent meshes (uneven sizes, P1 and P2) in one
// CUDA-graph launch.
//
// The graph holds two persistent kernels.  The element kernel walks a static
// list of (mesh, element tile) work items and the scatter kernel a list of
// (mesh, row tile) items, each CTA taking items b, b + grid, b + 2 grid, ...
// Items are sorted by estimated cost, largest first (longest-processing-time
// order), so the long P2 tiles start early and the short P1 tiles fill the
// tail.  Each work item runs the same per-element and per-row-tile device
// code as the single-mesh path, so every mesh's values are bitwise those of
// fea_assemble.  The elements per work item and both grid sizes are chosen by
// an autotuner (fea_batch_tune) that times candidate configurations on the
// device.  Every pattern, map and scratch buffer is built before the graph is
// captured: a replay allocates nothing and never synchronises.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "elem_kernels.cuh"
#include "gather.cuh"

namespace fea {
namespace {

struct BMesh {
  ElemArgs el;
  GatherArgs ga;
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

template <int LOAD, int NP1, int NP2>
__global__ void __launch_bounds__(BT) k_batch_elem(const BMesh* __restrict__ M, const BItem* __restrict__ items,
                                                   int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BMesh& m = M[w.mesh];
    const int64_t end = (int64_t)w.first + w.count;
    if (m.order == 1) {
      for (int64_t e = w.first + threadIdx.x; e < end; e += BT) {
        if (m.mass) elem_scalar_body<1, true, LOAD, NP1, double>(m.el, e);
        else elem_scalar_body<1, false, LOAD, NP1, double>(m.el, e);
      }
    } else {
      for (int64_t e = w.first + threadIdx.x; e < end; e += BT) {
        if (m.mass) elem_scalar_body<2, true, LOAD, NP2, double>(m.el, e);
        else elem_scalar_body<2, false, LOAD, NP2, double>(m.el, e);
      }
    }
  }
}

// One scatter kernel per element order (NB = 4 or 10), one CTA per row-tile
// item (a persistent loop here costs ~60 registers per thread, i.e. a third
// of the resident CTAs, for no gain: the tiles are already uniform).
template <int NB>
__global__ void __launch_bounds__(BT) k_batch_gather(const BMesh* __restrict__ M, const BItem* __restrict__ items,
                                                     int nitems) {
  extern __shared__ double acc[];
  if ((int)blockIdx.x >= nitems) return;
  const BItem w = items[blockIdx.x];
  gather_tile<NB, 1, double>(M[w.mesh].ga, w.first, M[w.mesh].rows_per_tile, acc);
}

using ElemKernel = void (*)(const BMesh*, const BItem*, int);

ElemKernel pick_elem_kernel(int load, int np1, int np2) {
  if (load == LOAD_NONE) return k_batch_elem<LOAD_NONE, 1, 1>;
  const bool sin = load == LOAD_SIN;
  if (np1 == 4 && np2 == 11) return sin ? k_batch_elem<LOAD_SIN, 4, 11> : k_batch_elem<LOAD_CONST, 4, 11>;
  if (np1 == 11 && np2 == 11) return sin ? k_batch_elem<LOAD_SIN, 11, 11> : k_batch_elem<LOAD_CONST, 11, 11>;
  if (np1 == 4 && np2 == 4) return sin ? k_batch_elem<LOAD_SIN, 4, 4> : k_batch_elem<LOAD_CONST, 4, 4>;
  return nullptr;
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
  BItem* d_eitems = nullptr;
  BItem* d_gitems = nullptr;     // P2 row tiles first, then P1 row tiles
  int n_eitems = 0, n_gitems = 0, n_gitems2 = 0;
  void* pool = nullptr;  // local rows and loads of every mesh
  size_t smem[3] = {0, 0, 0};  // scatter shared memory per CTA, by order
  int load = 0, np1 = 4, np2 = 11;
  ElemKernel ek = nullptr;
  int elem_tile = 256, elem_grid = 0, gather_grid = 0;
  int sms = 0;
  bool bound = false;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

fea_status build_items(fea_batch* b) {
  std::vector<std::pair<int64_t, BItem>> ei, gi;
  for (int k = 0; k < b->n; ++k) {
    const fea_mesh* m = b->meshes[k];
    const int order = b->forms[k].order;
    const int64_t E = m->n_elems;
    const int64_t cost = order == 2 ? 8 : 1;  // P2 element ~8x a P1 element
    for (int64_t f = 0; f < E; f += b->elem_tile) {
      const int32_t cnt = (int32_t)std::min<int64_t>(b->elem_tile, E - f);
      ei.push_back({cost * cnt, BItem{k, (int32_t)f, cnt}});
    }
    const Pattern* P = m->pat[order][1];
    const int64_t tiles = (P->ndof + P->rows_per_tile - 1) / P->rows_per_tile;
    for (int64_t t = 0; t < tiles; ++t) gi.push_back({order == 2 ? 10 : 4, BItem{k, (int32_t)t, 0}});
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
  b->n_gitems2 = 0;
  for (const BItem& w : hg) b->n_gitems2 += b->forms[w.mesh].order == 2;
  return FEA_OK;
}

fea_status launch_phases(fea_batch* b, cudaStream_t s) {
  if (b->n_eitems > 0) b->ek<<<b->elem_grid, BT, 0, s>>>(b->d_mesh, b->d_eitems, b->n_eitems);
  const int n1 = b->n_gitems - b->n_gitems2;
  if (b->n_gitems2 > 0) k_batch_gather<10><<<b->n_gitems2, BT, b->smem[2], s>>>(b->d_mesh, b->d_gitems, b->n_gitems2);
  if (n1 > 0) k_batch_gather<4><<<n1, BT, b->smem[1], s>>>(b->d_mesh, b->d_gitems + b->n_gitems2, n1);
  FEA_CUDA(cudaGetLastError());
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
  ElemKernel ek = pick_elem_kernel(f_kind, np1, np2);
  if (!ek) return fail(FEA_ERR_ARG, "supported (P1, P2) rules: (4, 11), (11, 11), (4, 4)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  fea_batch* b = new fea_batch();
  b->n = n;
  b->ek = ek;
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
    for (int k = 0; k < n && st == FEA_OK; ++k) {
      const int order = forms[k].order;
      if ((st = build_pattern(meshes[k], order, 1, s)) != FEA_OK) break;
      const Pattern* P = meshes[k]->pat[order][1];
      const int nb = order == 1 ? 4 : 10;
      lm_off[k] = bytes;
      bytes += (size_t)meshes[k]->n_elems * nb * lstride(nb, 8) * 8;
      fl_off[k] = bytes;
      bytes += ((size_t)meshes[k]->n_elems * nb * 8 + 255) / 256 * 256;
      b->smem[order] = std::max<size_t>(b->smem[order], (size_t)P->max_tile_nnz * 8);
      if (P->rows_per_tile > BT) st = fail(FEA_ERR_ARG, "row tile taller than the batch CTA");
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
      d.el.E = m->n_elems;
      d.el.e0 = 0;
      d.el.e1 = m->n_elems;
      d.el.kappa_const = 1.0;
      d.el.mass = forms[k].mass_coef;
      d.el.ipos = B->ipos;
      d.el.Lm = static_cast<char*>(b->pool) + lm_off[k];
      d.el.Fl = f_kind != FEA_LOAD_NONE ? static_cast<char*>(b->pool) + fl_off[k] : nullptr;
      d.el.err = m->err;
      d.ga.ndof = P->ndof;
      d.ga.row_ptr = P->row_ptr;
      d.ga.inc_ptr = B->inc_ptr;
      d.ga.slot = B->slot;
      d.ga.Lm = d.el.Lm;
      d.ga.Fl = d.el.Fl;
    }
    if (cudaMalloc(&b->d_mesh, sizeof(BMesh) * n) != cudaSuccess) {
      cudaGetLastError();
      st = fail(FEA_ERR_NOMEM, "batch descriptors");
      break;
    }
    cudaError_t ea = cudaSuccess;
    if (b->smem[1] > 48 * 1024)
      ea = cudaFuncSetAttribute(k_batch_gather<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem[1]);
    if (ea == cudaSuccess && b->smem[2] > 48 * 1024)
      ea = cudaFuncSetAttribute(k_batch_gather<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem[2]);
    if (ea != cudaSuccess) {
      st = cuda_fail(ea, "batch scatter shared memory");
      break;
    }
    b->elem_grid = b->sms * 4;
    b->gather_grid = b->sms * 3;
    if ((st = build_items(b)) != FEA_OK) break;
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) st = cuda_fail(e, "capture stream");
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
  }
  FEA_CUDA(cudaMemcpy(b->d_mesh, b->host.data(), sizeof(BMesh) * b->n, cudaMemcpyHostToDevice));
  b->bound = true;
  return FEA_OK;
}

fea_status fea_batch_assemble(fea_batch* b, void* stream) {
  if (!b) return fail(FEA_ERR_ARG, "batch is NULL");
  if (!b->bound) return fail(FEA_ERR_STATE, "fea_batch_bind first");
  if (!b->exec) FEA_TRY(rebuild_graph(b));
  FEA_CUDA(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
  return FEA_OK;
}

fea_status fea_batch_tune(fea_batch* b, void* stream, int32_t* params) {
  if (!b) return fail(FEA_ERR_ARG, "batch is NULL");
  if (!b->bound) return fail(FEA_ERR_STATE, "fea_batch_bind first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int tiles[] = {128, 256, 512, 1024, 2048};
  const int egrid[] = {2, 3, 4, 6, 8, 16};
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
  int bt = b->elem_tile, be = b->elem_grid;
  float best = 1e30f;
  // elements per work item x persistent element-kernel CTAs
  for (int t : tiles) {
    b->elem_tile = t;
    FEA_TRY(build_items(b));
    for (int g : egrid) {
      b->elem_grid = g * b->sms;
      float ms;
      FEA_TRY(time_it(&ms));
      if (ms < best) {
        best = ms;
        bt = t;
        be = b->elem_grid;
      }
    }
  }
  b->elem_tile = bt;
  b->elem_grid = be;
  FEA_TRY(build_items(b));
  b->gather_grid = b->n_gitems;
  cudaEventDestroy(a);
  cudaEventDestroy(c);
  FEA_TRY(rebuild_graph(b));
  if (params) {
    params[0] = b->elem_tile;
    params[1] = b->elem_grid;
    params[2] = b->gather_grid;
  }
  return FEA_OK;
}

fea_status fea_batch_destroy(fea_batch* b) {
  if (!b) return FEA_OK;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->d_mesh) cudaFree(b->d_mesh);
  if (b->d_eitems) cudaFree(b->d_eitems);
  if (b->d_gitems) cudaFree(b->d_gitems);
  if (b->pool) cudaFree(b->pool);
  delete b;
  return FEA_OK;
}

}  // extern "C"

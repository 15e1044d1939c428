// fea_assemble_noalloc: fea_assemble without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: a process whose device
// memory is already reserved by another allocator (a framework's caching
// pool that owns the whole GPU), or a latency-critical loop where the
// implicit device synchronisation of cudaMalloc / cudaFree is not acceptable.
// For them this entry point runs the same element and scatter kernels as
// fea_assemble, but keeps the per-call local rows and local loads in one
// fixed file-scope device array (NOALLOC_SCRATCH_BYTES) instead of the mesh
// handle's scratch, so the call itself allocates nothing.
//
// The array belongs to the library's module for this file.  CUDA loads a
// module on a device when it is first needed (lazy loading), so the array's
// 32 MiB are taken on a device by the first call there, when its address is
// looked up with cudaGetSymbolAddress (with that device current) and cached;
// from then on the device holds it until the process exits.  A caller whose
// allocator reserves the device's memory should make that first call before
// the reservation; if the memory is gone by then the call fails with
// FEA_ERR_NOMEM and nothing runs.  Every call shares the array, and the array keeps the
// last call's contents; nothing in it has to start at zero, because the
// element kernel writes every local row (padding included) and every local
// load before the scatter reads them.  Calls whose kernels overlap on the GPU
// (different streams, or different host threads) race on the array.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "elem_kernels.cuh"
#include "gather.cuh"
#include "gather_tiled.cuh"

namespace fea {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;  // 32 MiB
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

void* g_scratch_addr[NOALLOC_MAX_DEVICES] = {};
std::mutex g_scratch_mu;

// Device address of the fixed scratch on the current device (looked up once
// per device).
fea_status scratch_address(void** out) {
  int dev = 0;
  FEA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(FEA_ERR_ARG, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(fixed scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return FEA_OK;
}

}  // namespace
}  // namespace fea

using namespace fea;

extern "C" fea_status fea_assemble_noalloc(fea_mesh* m, const fea_form* form, const fea_coeffs* co,
                                           const fea_quadrature* q, double* values, double* rhs, void* stream) {
  // the argument checks of fea_assemble (alignment included: the kernels use
  // vector and bulk-copy accesses), all on the host before anything launches
  FEA_TRY(check_form(m, form, co, q));
  if (!values) return fail(FEA_ERR_ARG, "values is NULL");
  if (!aligned(values, 8) || (rhs && !aligned(rhs, 8))) return fail(FEA_ERR_ARG, "misaligned output");
  if (m->nvert != 4) return fail(FEA_ERR_ARG, "fea_assemble_noalloc takes tetrahedral meshes");
  const int order = form->order;
  const int ndpn = form->kind == FEA_ELASTICITY ? 3 : 1;
  Pattern* P = m->pat[order][ndpn];
  Base* B = m->base[order];
  if (!P || !B) return fail(FEA_ERR_STATE, "fea_assemble_noalloc: build the pattern with fea_pattern first");
  FEA_TRY(refuse_long_rows(B, "fea_assemble_noalloc"));
  const int nb = B->nb, nl = nb * ndpn;
  const bool mixed = q->prec == FEA_MIXED;
  const size_t rb = mixed ? sizeof(float) : sizeof(double);
  const int64_t E = m->n_elems;
  const int load = rhs ? co->f_kind : FEA_LOAD_NONE;
  const bool tiled = use_tiled(m, P);
  const size_t nrows_local = tiled ? (size_t)P->npos : (size_t)E * nb * ndpn;
  const size_t lm_bytes = (nrows_local * lstride(nl, (int)rb) * rb + 255) / 256 * 256;
  const size_t fl_bytes = load != FEA_LOAD_NONE ? nrows_local * rb : 0;
  if (lm_bytes + fl_bytes > NOALLOC_SCRATCH_BYTES)
    return fail(FEA_ERR_ARG, "fea_assemble_noalloc: this mesh needs " + std::to_string(lm_bytes + fl_bytes) +
                                 " bytes of scratch, above the fixed " + std::to_string(NOALLOC_SCRATCH_BYTES) +
                                 " (use fea_assemble)");
  void* base = nullptr;
  FEA_TRY(scratch_address(&base));
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  ElemArgs A{};
  A.x = m->x;
  A.y = m->y;
  A.z = m->z;
  A.tets = m->tets;
  A.N = m->n_nodes;
  A.E = E;
  A.e0 = 0;
  A.e1 = E;
  A.kappa = co->kappa;
  A.kappa_const = co->kappa_const;
  A.lam = co->lame_lambda;
  A.lam_const = co->lambda_const;
  A.mu = co->lame_mu;
  A.mu_const = co->mu_const;
  A.mass = form->mass_coef;
  for (int i = 0; i < 4; ++i) A.fp[i] = co->f_param[i];
  A.ipos = tiled ? P->tpos : B->ipos;
  A.Lm = base;
  A.Fl = load != FEA_LOAD_NONE ? static_cast<char*>(base) + lm_bytes : nullptr;
  A.err = m->err;
  const int prec = mixed ? FEA_MIXED : FEA_FP64;
  if (form->kind == FEA_ELASTICITY) {
    FEA_TRY(launch_elem_elast(A, load, q->npts, prec, s));
  } else {
    const bool mass = form->kind == FEA_DIFFUSION_MASS && form->mass_coef != 0.0;
    if (order == 1) FEA_TRY(launch_elem_p1(A, mass, load, q->npts, prec, s));
    else FEA_TRY(launch_elem_p2(A, mass, load, q->npts, prec, s));
  }
  if (tiled) return scatter_tiled(m, P, B, mixed, A.Lm, A.Fl, values, rhs, s);
  GatherArgs G{};
  G.ndof = P->ndof;
  G.row_ptr = P->row_ptr;
  G.inc_ptr = B->inc_ptr;
  G.slot = B->slot;
  G.Lm = A.Lm;
  G.Fl = A.Fl;
  G.values = values;
  G.rhs = rhs;
  G.err = m->err;
  return launch_gather(nb, ndpn, mixed, G, P->rows_per_tile, P->max_tile_nnz, s);
}

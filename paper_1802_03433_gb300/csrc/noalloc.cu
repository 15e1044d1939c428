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
// The array exists once per device for every process that loads the library
// and is held until the process exits.  Its device address is looked up with
// cudaGetSymbolAddress on the first call on each device (with that device
// current) and cached.  Every call shares the array, and the array keeps the
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
  if (!m || !form || !co || !q) return fail(FEA_ERR_ARG, "NULL mesh, form, coeffs or quadrature");
  if (form->order != FEA_P1 && form->order != FEA_P2) return fail(FEA_ERR_ARG, "order must be FEA_P1 or FEA_P2");
  if (form->kind != FEA_POISSON && form->kind != FEA_DIFFUSION_MASS && form->kind != FEA_ELASTICITY)
    return fail(FEA_ERR_ARG, "unknown form kind");
  if (form->kind == FEA_ELASTICITY && form->order != FEA_P1) return fail(FEA_ERR_ARG, "elasticity is P1 only");
  if (q->npts != 1 && q->npts != 4 && q->npts != 11) return fail(FEA_ERR_ARG, "npts must be 1, 4 or 11");
  if (q->prec != FEA_FP64 && q->prec != FEA_MIXED) return fail(FEA_ERR_ARG, "prec must be FEA_FP64 or FEA_MIXED");
  if (co->f_kind < FEA_LOAD_NONE || co->f_kind > FEA_LOAD_SINPROD) return fail(FEA_ERR_ARG, "unknown load kind");
  if (!values) return fail(FEA_ERR_ARG, "values is NULL");
  if (m->nvert != 4) return fail(FEA_ERR_ARG, "fea_assemble_noalloc takes tetrahedral meshes");
  const int order = form->order;
  const int ndpn = form->kind == FEA_ELASTICITY ? 3 : 1;
  Pattern* P = m->pat[order][ndpn];
  Base* B = m->base[order];
  if (!P || !B) return fail(FEA_ERR_STATE, "fea_assemble_noalloc: build the pattern with fea_pattern first");
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
  return launch_gather(nb, ndpn, mixed, G, P->rows_per_tile, P->max_tile_nnz, s);
}

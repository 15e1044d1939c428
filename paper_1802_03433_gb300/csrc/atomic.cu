// fea_assemble_atomic: the paper's own sparse assembly (Sec. 5, Algorithm 1,
// sparse variant) as a comparison point for the deterministic path.  Every
// element computes its local matrix and load vector with the same device code
// as fea_assemble, then adds each entry into the zeroed global CSR values with
// a global FP64 atomicAdd after a linear search of the global row for the
// column (the paper searches its N x MAX_NZ row the same way), and each load
// entry into rhs.  No scratch and no second kernel, but the order of the
// floating-point additions depends on scheduling: results agree with
// fea_assemble to rounding, not bit for bit, and may change between runs.
#include <cuda_runtime.h>

#include "elem_launch.cuh"

namespace fea {
namespace {

template <int ORDER, bool MASS>
struct AtomicScalar {
  template <int LOAD, int NPTS>
  static void go(const ElemArgs& A, cudaStream_t s) {
    k_elem_scalar<ORDER, MASS, LOAD, NPTS, double, true><<<elem_blocks(A), ELEM_T, 0, s>>>(A);
  }
  template <int NPTS>
  static void by_load(const ElemArgs& A, int load, cudaStream_t s) {
    if (load == LOAD_CONST) go<LOAD_CONST, NPTS>(A, s);
    else go<LOAD_SIN, NPTS>(A, s);
  }
  static void run(const ElemArgs& A, int load, int npts, cudaStream_t s) {
    if (load == LOAD_NONE) go<LOAD_NONE, 1>(A, s);
    else if (npts == 1) by_load<1>(A, load, s);
    else if (npts == 4) by_load<4>(A, load, s);
    else by_load<11>(A, load, s);
  }
};

struct AtomicElast {
  template <int LOAD, int NPTS>
  static void go(const ElemArgs& A, cudaStream_t s) {
    k_elem_elast<LOAD, NPTS, double, true><<<elem_blocks(A), ELEM_T, 0, s>>>(A);
  }
  template <int NPTS>
  static void by_load(const ElemArgs& A, int load, cudaStream_t s) {
    if (load == LOAD_CONST) go<LOAD_CONST, NPTS>(A, s);
    else go<LOAD_SIN, NPTS>(A, s);
  }
  static void run(const ElemArgs& A, int load, int npts, cudaStream_t s) {
    if (load == LOAD_NONE) go<LOAD_NONE, 1>(A, s);
    else if (npts == 1) by_load<1>(A, load, s);
    else if (npts == 4) by_load<4>(A, load, s);
    else by_load<11>(A, load, s);
  }
};

}  // namespace
}  // namespace fea

using namespace fea;

extern "C" fea_status fea_assemble_atomic(fea_mesh* m, const fea_form* form, const fea_coeffs* co,
                                          const fea_quadrature* q, double* values, double* rhs, void* stream) {
  if (!m || !form || !co || !q || !values) return fail(FEA_ERR_ARG, "NULL argument");
  if (form->order != FEA_P1 && form->order != FEA_P2) return fail(FEA_ERR_ARG, "order must be FEA_P1 or FEA_P2");
  if (form->kind != FEA_POISSON && form->kind != FEA_DIFFUSION_MASS && form->kind != FEA_ELASTICITY)
    return fail(FEA_ERR_ARG, "unknown form kind");
  if (form->kind == FEA_ELASTICITY && form->order != FEA_P1) return fail(FEA_ERR_ARG, "elasticity is P1 only");
  if (q->npts != 1 && q->npts != 4 && q->npts != 11) return fail(FEA_ERR_ARG, "npts must be 1, 4 or 11");
  if (q->prec != FEA_FP64) return fail(FEA_ERR_ARG, "the atomic comparison path runs in FP64");
  if (co->f_kind < FEA_LOAD_NONE || co->f_kind > FEA_LOAD_SINPROD) return fail(FEA_ERR_ARG, "unknown load kind");
  if (m->nvert != 4) return fail(FEA_ERR_ARG, "fea_assemble_atomic takes tetrahedral meshes");
  const int order = form->order;
  const int ndpn = form->kind == FEA_ELASTICITY ? 3 : 1;
  const Pattern* P = m->pat[order][ndpn];
  const Base* B = m->base[order];
  if (!P || !B) return fail(FEA_ERR_STATE, "fea_assemble_atomic: build the pattern with fea_pattern first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FEA_CUDA(cudaMemsetAsync(values, 0, P->nnz * sizeof(double), s));
  if (rhs) FEA_CUDA(cudaMemsetAsync(rhs, 0, P->ndof * sizeof(double), s));
  const int load = rhs ? co->f_kind : FEA_LOAD_NONE;
  ElemArgs A{};
  A.x = m->x;
  A.y = m->y;
  A.z = m->z;
  A.tets = m->tets;
  A.N = m->n_nodes;
  A.E = m->n_elems;
  A.e0 = 0;
  A.e1 = m->n_elems;
  A.kappa = co->kappa;
  A.kappa_const = co->kappa_const;
  A.lam = co->lame_lambda;
  A.lam_const = co->lambda_const;
  A.mu = co->lame_mu;
  A.mu_const = co->mu_const;
  A.mass = form->mass_coef;
  for (int i = 0; i < 4; ++i) A.fp[i] = co->f_param[i];
  A.err = m->err;
  A.edof = B->edof;
  A.rp = P->row_ptr;
  A.ci = P->col_idx;
  A.values = values;
  A.rhs = rhs;
  if (A.E == 0) return FEA_OK;
  if (form->kind == FEA_ELASTICITY) {
    AtomicElast::run(A, load, q->npts, s);
  } else {
    const bool mass = form->kind == FEA_DIFFUSION_MASS && form->mass_coef != 0.0;
    if (order == 1) {
      if (mass) AtomicScalar<1, true>::run(A, load, q->npts, s);
      else AtomicScalar<1, false>::run(A, load, q->npts, s);
    } else {
      if (mass) AtomicScalar<2, true>::run(A, load, q->npts, s);
      else AtomicScalar<2, false>::run(A, load, q->npts, s);
    }
  }
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

// The paper's 2-D worked example (Sec. 4.1-4.2): P1 triangles with the weak
// form (grad v, sigma grad u) + lambda (v, u) = (v, f) of Eq. 2, where sigma is
// an affine 2 x 2 matrix field (not necessarily symmetric) and f a quadratic.
// One thread per triangle: the gradients of the P1 basis are constant on the
// element and sigma is affine, so  int_T grad phi_a . sigma grad phi_b =
// |T| grad phi_a . sigma(centroid) grad phi_b  exactly; the mass term is
// |T| (1 + delta_ab) / 12; the load is a quadrature of f phi_a with the
// requested rule (1, 3 or 6 points).  The local matrix is stored in full
// (rows and columns differ), and the same deterministic scatter as the
// tetrahedral path sums it into CSR.
#include <cuda_runtime.h>

#include "elem_kernels.cuh"
#include "gather.cuh"

namespace fea {
namespace {

// 6-point degree-4 triangle rule: permutations of (a, a, 1 - 2a),
// a = (8 - sqrt 10 +- sqrt(38 - 44 sqrt(2/5))) / 18, weights
// (620 +- sqrt(213125 - 53320 sqrt 10)) / 3720.
constexpr double T6A1 = 0.4459484909159648863183292538830519883991;
constexpr double T6A2 = 0.09157621350977074345957146340220150785433;
constexpr double T6W1 = 0.2233815896780114656950070084331228043703;
constexpr double T6W2 = 0.1099517436553218676383263249002105289631;

__host__ __device__ constexpr double tri_bary(int npts, int q, int v) {
  return npts == 1 ? 1.0 / 3.0
       : npts == 3 ? (v == q ? 2.0 / 3.0 : 1.0 / 6.0)
       : (q < 3 ? (v == q ? 1.0 - 2.0 * T6A1 : T6A1) : (v == q - 3 ? 1.0 - 2.0 * T6A2 : T6A2));
}
__host__ __device__ constexpr double tri_weight(int npts, int q) {
  return npts == 1 ? 1.0 : npts == 3 ? 1.0 / 3.0 : (q < 3 ? T6W1 : T6W2);
}

struct TriArgs {
  const double* x;
  const double* y;
  const int32_t* tris;  // [3][E]
  int64_t E;
  double S0[4], Sx[4], Sy[4];
  double lambda;
  double f[6];
  const int32_t* ipos;
  double* Lm;
  double* Fl;
  int* err;
};

template <int NPTS, bool LOAD>
__global__ void __launch_bounds__(128) k_elem_tri(TriArgs A) {
  const int64_t e = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (e >= A.E) return;
  double X[3][2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int32_t n = __ldg(A.tris + a * A.E + e);
    X[a][0] = __ldg(A.x + n);
    X[a][1] = __ldg(A.y + n);
  }
  const double e1x = X[1][0] - X[0][0], e1y = X[1][1] - X[0][1];
  const double e2x = X[2][0] - X[0][0], e2y = X[2][1] - X[0][1];
  const double det = fma(e1x, e2y, -e2x * e1y);
  if (!(det > 0.0)) atomicOr(A.err, DEV_ERR_DEGENERATE);
  const double inv = 1.0 / det, area = fabs(det) * 0.5;
  // rows of J^{-1}: grad lambda_1, grad lambda_2; grad lambda_0 = -(sum)
  double g[3][2];
  g[1][0] = e2y * inv;
  g[1][1] = -e2x * inv;
  g[2][0] = -e1y * inv;
  g[2][1] = e1x * inv;
  g[0][0] = -(g[1][0] + g[2][0]);
  g[0][1] = -(g[1][1] + g[2][1]);
  const double xc = (X[0][0] + X[1][0] + X[2][0]) * (1.0 / 3.0);
  const double yc = (X[0][1] + X[1][1] + X[2][1]) * (1.0 / 3.0);
  double sg[4];  // area * sigma(centroid)
#pragma unroll
  for (int k = 0; k < 4; ++k) sg[k] = area * fma(xc, A.Sx[k], fma(yc, A.Sy[k], A.S0[k]));
  const double m = A.lambda * area * (1.0 / 12.0);
  int32_t pos[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) pos[a] = __ldg(A.ipos + a * A.E + e);
  double K[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const double s0 = fma(sg[0], g[b][0], sg[1] * g[b][1]);
    const double s1 = fma(sg[2], g[b][0], sg[3] * g[b][1]);
#pragma unroll
    for (int a = 0; a < 3; ++a) K[a][b] = fma(g[a][0], s0, fma(g[a][1], s1, a == b ? 2.0 * m : m));
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) st_v4(A.Lm + (int64_t)pos[a] * 4, K[a][0], K[a][1], K[a][2], 0.0);
  if constexpr (LOAD) {
    double F[3] = {0.0, 0.0, 0.0};
    static_for<NPTS>([&](auto Q) {
      constexpr int q = Q;
      const double x = fma(tri_bary(NPTS, q, 0), X[0][0], fma(tri_bary(NPTS, q, 1), X[1][0], tri_bary(NPTS, q, 2) * X[2][0]));
      const double y = fma(tri_bary(NPTS, q, 0), X[0][1], fma(tri_bary(NPTS, q, 1), X[1][1], tri_bary(NPTS, q, 2) * X[2][1]));
      const double fv = fma(fma(A.f[3], x, A.f[4] * y + A.f[1]), x, fma(A.f[5], y, A.f[2]) * y + A.f[0]);
#pragma unroll
      for (int a = 0; a < 3; ++a) F[a] = fma(tri_weight(NPTS, q) * tri_bary(NPTS, q, a), fv, F[a]);
    });
#pragma unroll
    for (int a = 0; a < 3; ++a) A.Fl[pos[a]] = area * F[a];
  }
}

template <bool LOAD>
void launch_tri(const TriArgs& A, int npts, cudaStream_t s) {
  const unsigned blocks = (unsigned)((A.E + 127) / 128);
  if (npts == 1) k_elem_tri<1, LOAD><<<blocks, 128, 0, s>>>(A);
  else if (npts == 3) k_elem_tri<3, LOAD><<<blocks, 128, 0, s>>>(A);
  else k_elem_tri<6, LOAD><<<blocks, 128, 0, s>>>(A);
}

}  // namespace
}  // namespace fea

using namespace fea;

extern "C" fea_status fea_assemble_2d(fea_mesh* m, const fea_form2d* form, double* values, double* rhs,
                                      void* stream) {
  if (!m || !form || !values) return fail(FEA_ERR_ARG, "NULL mesh, form or values");
  if (m->nvert != 3) return fail(FEA_ERR_ARG, "fea_assemble_2d takes triangle meshes (fea_mesh_create_tri)");
  if (form->npts != 1 && form->npts != 3 && form->npts != 6) return fail(FEA_ERR_ARG, "npts must be 1, 3 or 6");
  if ((reinterpret_cast<uintptr_t>(values) & 7) || (reinterpret_cast<uintptr_t>(rhs) & 7))
    return fail(FEA_ERR_ARG, "misaligned output");
  Pattern* P = m->pat[1][1];
  Base* B = m->base[1];
  if (!P || !B) return fail(FEA_ERR_STATE, "fea_assemble_2d: build the pattern with fea_pattern(mesh, 1, 1) first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t E = m->n_elems;
  FEA_TRY(ensure_scratch(m->lm, (size_t)E * 3 * 4 * sizeof(double)));
  if (rhs) FEA_TRY(ensure_scratch(m->fl, (size_t)E * 3 * sizeof(double)));
  TriArgs A{};
  A.x = m->x;
  A.y = m->y;
  A.tris = m->tets;
  A.E = E;
  for (int k = 0; k < 4; ++k) {
    A.S0[k] = form->sigma0[k];
    A.Sx[k] = form->sigma_x[k];
    A.Sy[k] = form->sigma_y[k];
  }
  A.lambda = form->lambda;
  for (int k = 0; k < 6; ++k) A.f[k] = form->f[k];
  A.ipos = B->ipos;
  A.Lm = static_cast<double*>(m->lm.ptr);
  A.Fl = rhs ? static_cast<double*>(m->fl.ptr) : nullptr;
  A.err = m->err;
  if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[0], s));
  if (E > 0) {
    if (rhs) launch_tri<true>(A, form->npts, s);
    else launch_tri<false>(A, form->npts, s);
    FEA_CUDA(cudaGetLastError());
  }
  if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[1], s));
  GatherArgs G{};
  G.ndof = P->ndof;
  G.row_ptr = P->row_ptr;
  G.inc_ptr = B->inc_ptr;
  G.slot = B->slot;
  G.Lm = m->lm.ptr;
  G.Fl = A.Fl;
  G.values = values;
  G.rhs = rhs;
  FEA_TRY(launch_gather(3, 1, false, G, P->rows_per_tile, P->max_tile_nnz, s));
  if (m->profile) {
    FEA_CUDA(cudaEventRecord(m->ev[2], s));
    m->profiled = true;
  }
  return FEA_OK;
}

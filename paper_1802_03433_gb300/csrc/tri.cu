// The paper's 2-D worked example (Sec. 4.1-4.2): P1 triangles with the weak
// form (grad v, sigma grad u) + lambda (v, u) = (v, f) of Eq. 2, where sigma is
// an affine 2 x 2 matrix field (not necessarily symmetric) and f a quadratic.
// One thread per triangle.  The gradients of the P1 basis are constant on
// the element and sigma is affine, so
//   int_T grad phi_a . sigma grad phi_b = |T| grad phi_a . sigma(c) grad phi_b
// exactly (c the centroid); with grad phi_a = n_a / det (n_a the edge
// opposite vertex a turned by 90 degrees, det = 2 |T|) that is
// n_a . sigma(c) n_b / (2 det).  The mass term is lambda |T| (1 + delta_ab) / 12.
// The load integrates f phi_a with the requested rule (1, 3 or 6 points).
// Because f is quadratic, f(c + d) = f(c) + grad f(c) . d + q(d) with
// q(d) = d^T (H / 2) d, and every rule point is c + t d_v (d_v = X_v - c), so
// the points' f values come from f(c), grad f(c) . d_v and q(d_v).  The
// 6-point rule has degree 4 >= 3, so it returns the exact integral, which in
// this form is |T| [f(c) / 3 + grad f(c) . d_a / 12 + (sum_b q(d_b) + 2 q(d_a)) / 60]
// (from int_T phi_a phi_b phi_c = |T| (1 + delta_ab + delta_ac + delta_bc +
// 2 delta_abc) / 60 and sum_b d_b = 0); the kernel evaluates that closed form.
// The local matrix is stored in full (rows and columns differ), and the same
// deterministic scatter as the tetrahedral path sums it into CSR.
#include <cuda_runtime.h>

#include "elem_kernels.cuh"
#include "gather.cuh"
#include "gather_tiled.cuh"

namespace fea {
namespace {

struct TriArgs {
  const double* x;
  const double* y;
  const int32_t* tris;  // [3][E]
  int64_t E;
  double S0[4], Sx[4], Sy[4];
  double lam24;  // lambda / 24
  double f[6];
  const int32_t* ipos;
  double* Lm;
  double* Fl;
  int* err;
  int64_t N;  // node count (bounds of the coordinate gathers in the checked build)
};

template <int NPTS, bool LOAD>
__global__ void __launch_bounds__(128) k_elem_tri(TriArgs A) {
  const int64_t e = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (e >= A.E) return;
  double X[3][2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int32_t n = checked_index(__ldg(A.tris + a * A.E + e), A.N, A.err);
    X[a][0] = __ldg(A.x + n);
    X[a][1] = __ldg(A.y + n);
  }
  int32_t pos[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) pos[a] = __ldg(A.ipos + a * A.E + e);
  const double e1x = X[1][0] - X[0][0], e1y = X[1][1] - X[0][1];
  const double e2x = X[2][0] - X[0][0], e2y = X[2][1] - X[0][1];
  const double det = fma(e1x, e2y, -e2x * e1y);
  if (!(det > 0.0)) atomicOr(A.err, DEV_ERR_DEGENERATE);
  const double adet = fabs(det);
  const double h = 0.5 / adet;
  // n_a = det * grad phi_a
  double n[3][2];
  n[1][0] = e2y;
  n[1][1] = -e2x;
  n[2][0] = -e1y;
  n[2][1] = e1x;
  n[0][0] = -(e2y - e1y);
  n[0][1] = -(e1x - e2x);
  const double xc = (X[0][0] + X[1][0] + X[2][0]) * (1.0 / 3.0);
  const double yc = (X[0][1] + X[1][1] + X[2][1]) * (1.0 / 3.0);
  double sg[4];  // sigma(c) / (2 det)
#pragma unroll
  for (int k = 0; k < 4; ++k) sg[k] = h * fma(xc, A.Sx[k], fma(yc, A.Sy[k], A.S0[k]));
  const double m = A.lam24 * adet;  // lambda |T| / 12
  const double m2 = m + m;
  double K[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const double s0 = fma(sg[0], n[b][0], sg[1] * n[b][1]);
    const double s1 = fma(sg[2], n[b][0], sg[3] * n[b][1]);
#pragma unroll
    for (int a = 0; a < 3; ++a) K[a][b] = fma(n[a][0], s0, fma(n[a][1], s1, a == b ? m2 : m));
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) st_v4(A.Lm + (int64_t)pos[a] * 4, K[a][0], K[a][1], K[a][2], 0.0);
  if constexpr (LOAD) {
    const double* f = A.f;
    const double fc = fma(fma(f[3], xc, fma(f[4], yc, f[1])), xc, fma(fma(f[5], yc, f[2]), yc, f[0]));
    const double area = 0.5 * adet;
    double F[3];
    if constexpr (NPTS == 1) {
      const double v = area * (1.0 / 3.0) * fc;
#pragma unroll
      for (int a = 0; a < 3; ++a) F[a] = v;
    } else {
      const double gx = fma(2.0 * f[3], xc, fma(f[4], yc, f[1]));
      const double gy = fma(2.0 * f[5], yc, fma(f[4], xc, f[2]));
      double l[3], q[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double dx = X[a][0] - xc, dy = X[a][1] - yc;
        l[a] = fma(gx, dx, gy * dy);
        q[a] = fma(fma(f[3], dx, f[4] * dy), dx, f[5] * dy * dy);
      }
      if constexpr (NPTS == 3) {
        // points c + d_v / 2 (barycentric 2/3, 1/6, 1/6), weights |T| / 3
        double fq[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) fq[a] = fma(0.25, q[a], fma(0.5, l[a], fc));
        const double base = (fq[0] + fq[1] + fq[2]) * (area * (1.0 / 18.0));
        const double w = area * (1.0 / 6.0);
#pragma unroll
        for (int a = 0; a < 3; ++a) F[a] = fma(w, fq[a], base);
      } else {
        const double base = area * fma(q[0] + q[1] + q[2], 1.0 / 60.0, fc * (1.0 / 3.0));
#pragma unroll
        for (int a = 0; a < 3; ++a) F[a] = fma(area, fma(l[a], 1.0 / 12.0, q[a] * (1.0 / 30.0)), base);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) A.Fl[pos[a]] = F[a];
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
  FEA_TRY(refuse_long_rows(B, "fea_assemble_2d"));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t E = m->n_elems;
  const bool tiled = use_tiled(m, P);
  const size_t npos = tiled ? (size_t)P->npos : (size_t)E * 3;
  FEA_TRY(ensure_scratch(m->lm, npos * 4 * sizeof(double)));
  if (rhs) FEA_TRY(ensure_scratch(m->fl, npos * sizeof(double)));
  TriArgs A{};
  A.x = m->x;
  A.y = m->y;
  A.tris = m->tets;
  A.E = E;
  A.N = m->n_nodes;
  for (int k = 0; k < 4; ++k) {
    A.S0[k] = form->sigma0[k];
    A.Sx[k] = form->sigma_x[k];
    A.Sy[k] = form->sigma_y[k];
  }
  A.lam24 = form->lambda / 24.0;
  for (int k = 0; k < 6; ++k) A.f[k] = form->f[k];
  A.ipos = tiled ? P->tpos : B->ipos;
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
  if (tiled) {
    FEA_TRY(scatter_tiled(m, P, B, false, m->lm.ptr, A.Fl, values, rhs, s));
  } else {
    GatherArgs G{};
    G.ndof = P->ndof;
    G.row_ptr = P->row_ptr;
    G.inc_ptr = B->inc_ptr;
    G.slot = B->slot;
    G.Lm = m->lm.ptr;
    G.Fl = A.Fl;
    G.values = values;
    G.rhs = rhs;
  G.err = m->err;
    FEA_TRY(launch_gather(3, 1, false, G, P->rows_per_tile, P->max_tile_nnz, s));
  }
  if (m->profile) {
    FEA_CUDA(cudaEventRecord(m->ev[2], s));
    m->profiled = true;
  }
  return FEA_OK;
}

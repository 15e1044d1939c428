// Reverse mode of the scalar assembly (P1/P2, -div(kappa grad u) + m u = f).
//
// For a scalar loss L with G = dL/dvalues (on the CSR pattern) and
// g = dL/drhs, each element contributes, through its own local matrix and
// load vector (Eq. 2-3: A and b are sums of element terms),
//   L_e = kappa |T| S + m |T| sM + |T| sF,
//   S  = sum_{i<=j} Hc_ij (grad lambda_i . grad lambda_j),
//        Hc = the element's G entries folded through the stiffness reference
//        tensor (Hc = G for P1),
//   sM = sum_ab G_ab Mref_ab,   sF = sum_q w_q f(x_q) Phi_q,
//   Phi_q = sum_a g_a phi_a(x_q).
// Hand-derived gradients (one thread per element, local matrices recomputed,
// never stored):
//   dL/dkappa_e = |T| S;
//   dL/dx_c = |T| [ (sigma I - kappa Q) grad lambda_c
//                   + sum_q w_q Phi_q lambda_c(x_q) grad f(x_q) ],
//   sigma = kappa S + m sM + sF,  Q = sum_{i=1..3} grad lambda_i dS_i^T,
//   dS_i = dS/dgrad lambda_i - dS/dgrad lambda_0,
// using d|T|/dx_c = |T| grad lambda_c and d(grad lambda_i) = -J^{-T} dJ^T
// grad lambda_i.  The per-vertex vectors of every element are written to the
// vertex's incidence slot and summed per node in ascending element order by
// a second kernel (deterministic, no atomics).
#include <cuda_runtime.h>

#include "element.cuh"
#include "gather.cuh"
#include "internal.cuh"

namespace fea {

namespace {

struct AdjArgs {
  const double* x;
  const double* y;
  const double* z;
  const int32_t* tets;   // [4][E]
  const int32_t* edof;   // [nb][E] scalar dofs
  const int32_t* ipos;   // [nb][E] incidence index of (e, a)
  const int32_t* rp;     // scalar CSR row pointer
  const uint8_t* slot;   // [incidence][SW]
  int64_t E;
  const double* kappa;
  double kappa_const;
  double mass;
  double fp0;
  const double* gv;      // dL/dvalues or NULL
  const double* gf;      // dL/drhs or NULL
  double* gk;            // dL/dkappa [E] or NULL
  double* gxs;           // per-incidence vertex gradients [incidence][4]
  int* err;
  int64_t N;  // node count (bounds of the coordinate gathers in the checked build)
};

constexpr int ADJ_T = 128;

template <int ORDER, bool MASS, int LOAD, int NPTS>
__global__ void __launch_bounds__(ADJ_T) k_adjoint(AdjArgs A) {
  constexpr int NB = ORDER == 1 ? 4 : 10;
  const int64_t e = (int64_t)blockIdx.x * ADJ_T + threadIdx.x;
  if (e >= A.E) return;
  double X[4][3];
  {
    int32_t v[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) v[a] = checked_index(__ldg(A.tets + a * A.E + e), A.N, A.err);
    load_vertices(A.x, A.y, A.z, v, X);
  }
  Geo geo;
  geometry(X, geo);
  if (!(geo.det > 0.0)) atomicOr(A.err, DEV_ERR_DEGENERATE);
  // grad lambda_a = c_a / det J: the cofactors c_a stay unscaled and 1/det J
  // enters the few scalars below
  const double inv = 1.0 / geo.det;
  const double vol = fabs(geo.det) * (1.0 / 6.0);
  const double (&cf)[4][3] = geo.c;
  const double kap = A.kappa ? __ldg(A.kappa + e) : A.kappa_const;

  int32_t pos[NB];
#pragma unroll
  for (int a = 0; a < NB; ++a) pos[a] = __ldg(A.ipos + a * A.E + e);

  // ---- G entries of this element: Gs_ab = G_ab + G_ba (a < b), G_aa
  double Hc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) Hc[i][j] = 0.0;
  double sM = 0.0;
  if (A.gv) {
    double Gm[NB][NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      const int32_t row = __ldg(A.edof + a * A.E + e);
      const int32_t base = __ldg(A.rp + row);
      int s[NB];
      load_slots<NB>(A.slot, pos[a], s);
#pragma unroll
      for (int b = 0; b < NB; ++b) Gm[a][b] = __ldg(A.gv + base + s[b]);
    }
    if constexpr (ORDER == 1) {
      static_for<10>([&](auto K) {
        constexpr int a = upper_a(4, K), b = upper_b(4, K);
        const double gs = a == b ? Gm[a][a] : Gm[a][b] + Gm[b][a];
        Hc[a][b] += gs;
        if constexpr (MASS) sM = fma(gs, (a == b ? 2.0 : 1.0) / 20.0, sM);
      });
    } else {
      static_for<55>([&](auto K) {
        constexpr int a = upper_a(10, K), b = upper_b(10, K);
        constexpr Terms t = p2_terms(a, b);
        const double gs = a == b ? Gm[a][a] : Gm[a][b] + Gm[b][a];
        Hc[t.i[0]][t.j[0]] = fma(gs, t.num[0] / 20.0, Hc[t.i[0]][t.j[0]]);
        if constexpr (t.n > 1) Hc[t.i[1]][t.j[1]] = fma(gs, t.num[1] / 20.0, Hc[t.i[1]][t.j[1]]);
        if constexpr (t.n > 2) Hc[t.i[2]][t.j[2]] = fma(gs, t.num[2] / 20.0, Hc[t.i[2]][t.j[2]]);
        if constexpr (t.n > 3) Hc[t.i[3]][t.j[3]] = fma(gs, t.num[3] / 20.0, Hc[t.i[3]][t.j[3]]);
        if constexpr (MASS) sM = fma(gs, p2_mass420(a, b) / 420.0, sM);
      });
    }
  }
  // Q = sum_{i=1..3} g_i (dS_i - dS_0)^T with dS_a = dS/dg_a = sum_b Hsym_ab g_b
  // (Hsym = Hc + Hc^T) is sum_ab Hsym_ab g_a g_b^T, and with g_0 = -(g_1 + g_2
  // + g_3) that is sum_{i,j>=1} H'_ij g_i g_j^T, H'_ij = Hsym_ij - Hsym_i0 -
  // Hsym_0j + Hsym_00: the 3 x 3 reduced form, taken on the unscaled
  // cofactors (Qc, so Q = Qc / det^2), symmetric (upper triangle formed);
  // S = sum_{i<=j} Hc_ij g_i . g_j = tr(Q) / 2
  double Hr[3][3];
  {
    const double h00 = Hc[0][0] + Hc[0][0];
    double beta[3];
#pragma unroll
    for (int i = 1; i < 4; ++i) beta[i - 1] = fma(-0.5, h00, Hc[0][i]);  // Hsym_0i - Hsym_00 / 2
    static_for<6>([&](auto K) {
      constexpr int i = upper_a(3, K), j = upper_b(3, K);
      const double hs = i == j ? Hc[i + 1][i + 1] + Hc[i + 1][i + 1] : Hc[i + 1][j + 1];
      Hr[i][j] = hs - beta[i] - beta[j];
      Hr[j][i] = Hr[i][j];
    });
  }
  double W[3][3];  // W_i = sum_j H'_ij c_j
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      W[i][k] = fma(Hr[i][0], cf[1][k], fma(Hr[i][1], cf[2][k], Hr[i][2] * cf[3][k]));
  double Qc[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = r; c < 3; ++c) {
      Qc[r][c] = fma(cf[1][r], W[0][c], fma(cf[2][r], W[1][c], cf[3][r] * W[2][c]));
      Qc[c][r] = Qc[r][c];
    }
  const double inv2 = inv * inv;
  const double S = 0.5 * inv2 * (Qc[0][0] + Qc[1][1] + Qc[2][2]);

  // ---- load terms
  double sF = 0.0;
  double lg[4][3];  // |T| sum_q w_q Phi_q lambda_c(x_q) grad f(x_q), per vertex c
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int k = 0; k < 3; ++k) lg[c][k] = 0.0;
  if constexpr (LOAD != LOAD_NONE) {
    if (A.gf) {
      double gfl[NB];
#pragma unroll
      for (int a = 0; a < NB; ++a) gfl[a] = __ldg(A.gf + __ldg(A.edof + a * A.E + e));
      [[maybe_unused]] int sh[3];
      [[maybe_unused]] long long xfx[3][NPTS];
      [[maybe_unused]] double u[3][NPTS];  // sine load: |T| pi p0 Phi_q d f/d x_k at point q (unweighted)
      [[maybe_unused]] const double vpf = vol * A.fp0 * 3.14159265358979323846;
      [[maybe_unused]] double uf[NPTS];    // sine load: Phi_q f_q / p0
      if constexpr (LOAD == LOAD_SIN) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double v[4] = {X[0][k], X[1][k], X[2][k], X[3][k]};
          sh[k] = fx_shift(v);
          quad_coord_fx<NPTS>(v, sh[k], xfx[k]);
        }
      }
      static_for<NPTS>([&](auto Qi) {
        constexpr int q = Qi;
        double Phi = 0.0;
        static_for<NB>([&](auto Aa) {
          constexpr double ph = phi_at(ORDER, NPTS, q, Aa);
          Phi = fma(ph, gfl[Aa], Phi);
        });
        if constexpr (LOAD == LOAD_CONST) {
          sF = fma(A.fp0, weight(NPTS, q) * Phi, sF);
        } else {
          // the points, sin(pi x_k), cos(pi x_k) = sin(pi (x_k + 1/2)) and the
          // products of f and grad f in fixed point (as the forward load);
          // four conversions, then the Phi_q factors in FP64
          // lanes: sin x, sin y, sin z, cos x | cos y, cos z (each with its coordinate's shift)
          const Q4 in0 = {{xfx[0][q], xfx[1][q], xfx[2][q], xfx[0][q] + (1LL << (60 - sh[0]))}};
          const Q4 in1 = {{xfx[1][q] + (1LL << (60 - sh[1])), xfx[2][q] + (1LL << (60 - sh[2])), 0, 0}};
          const Q4 o0 = sinpi_q62_fx4v_call(in0, S4{{sh[0], sh[1], sh[2], sh[0]}});
          const Q4 o1 = sinpi_q62_fx4v_call(in1, S4{{sh[1], sh[2], 0, 0}});
          const long long sn0 = o0.v[0], sn1 = o0.v[1], sn2 = o0.v[2], cs0 = o0.v[3], cs1 = o1.v[0], cs2 = o1.v[1];
          const long long p01 = mul_q62(sn0, sn1), p12 = mul_q62(sn1, sn2);
          const double f = q62_to_double(mul_q62(p01, sn2));
          const double d0 = q62_to_double(mul_q62(cs0, p12));
          const double d1 = q62_to_double(mul_q62(mul_q62(sn0, cs1), sn2));
          const double d2 = q62_to_double(mul_q62(p01, cs2));
          uf[q] = Phi * f;
          const double pPhi = vpf * Phi;
          u[0][q] = pPhi * d0;
          u[1][q] = pPhi * d1;
          u[2][q] = pPhi * d2;
        }
      });
      if constexpr (LOAD == LOAD_SIN) {
        // lg_ck = sum_q w_q lambda_c(x_q) u_kq and sF = p0 sum_q w_q Phi_q f_q, by
        // the rule's symmetry classes (rule_sum with the P1 basis: lambda_c)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          double col[4];
          rule_sum<1, NPTS, double>(u[k], col);
#pragma unroll
          for (int c = 0; c < 4; ++c) lg[c][k] = col[c];
        }
        static_for<NPTS>([&](auto Qi) { sF = fma(weight(NPTS, Qi), uf[Qi], sF); });
      }
    }
  }

  if constexpr (LOAD == LOAD_SIN) sF *= A.fp0;
  if (A.gk) A.gk[e] = vol * S;
  const double sigma = kap * S + (MASS ? A.mass * sM : 0.0) + sF;
  // |T| [(sigma I - kappa Q) grad lambda_c + lg_c], with |T| folded into
  // sigma, kappa and (through vpf) lg, and grad lambda_c = c_c / det J: the
  // symmetric matrix M = |T| (sigma I - kappa Qc / det^2) / det once, then
  // M c_c + lg_c per vertex
  const double vs = vol * sigma * inv, vk = -vol * kap * inv2 * inv;
  double M[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = r; c < 3; ++c) {
      M[r][c] = r == c ? fma(vk, Qc[r][r], vs) : vk * Qc[r][c];
      M[c][r] = M[r][c];
    }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      d[k] = fma(M[k][0], cf[c][0], fma(M[k][1], cf[c][1], fma(M[k][2], cf[c][2], lg[c][k])));
    st_v4(A.gxs + (int64_t)pos[c] * 4, d[0], d[1], d[2], 0.0);
  }
}

// dL/dx per node: the node's incidence slots summed in element order.
__global__ void k_node_grad(int64_t N, const int32_t* __restrict__ inc_ptr, const double* __restrict__ gxs,
                            double* __restrict__ gx) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int32_t i = __ldg(inc_ptr + n); i < __ldg(inc_ptr + n + 1); ++i) {
    double a, b, c, pad;
    ld_v4(gxs + (int64_t)i * 4, a, b, c, pad);
    s0 += a;
    s1 += b;
    s2 += c;
  }
  gx[n] = s0;
  gx[N + n] = s1;
  gx[2 * N + n] = s2;
}

template <int ORDER, bool MASS>
struct AdjLauncher {
  template <int LOAD, int NPTS>
  static void go(const AdjArgs& A, cudaStream_t s) {
    k_adjoint<ORDER, MASS, LOAD, NPTS><<<(unsigned)((A.E + ADJ_T - 1) / ADJ_T), ADJ_T, 0, s>>>(A);
  }
  template <int NPTS>
  static void by_load(const AdjArgs& A, int load, cudaStream_t s) {
    if (load == LOAD_CONST) go<LOAD_CONST, NPTS>(A, s);
    else go<LOAD_SIN, NPTS>(A, s);
  }
  static void run(const AdjArgs& A, int load, int npts, cudaStream_t s) {
    if (load == LOAD_NONE) go<LOAD_NONE, 1>(A, s);
    else if (npts == 1) by_load<1>(A, load, s);
    else if (npts == 4) by_load<4>(A, load, s);
    else by_load<11>(A, load, s);
  }
};

}  // namespace

fea_status assemble_backward(fea_mesh* m, const fea_form* form, const fea_coeffs* co, const fea_quadrature* q,
                             const double* gv, const double* gf, double* gk, double* gx, cudaStream_t s) {
  const int order = form->order;
  Base* B = m->base[order];
  if (!B || !m->pat[order][1]) return fail(FEA_ERR_STATE, "fea_assemble_backward: build the pattern first");
  FEA_TRY(refuse_long_rows(B, "fea_assemble_backward"));
  const int64_t E = m->n_elems, N = m->n_nodes;
  if (!gk && !gx) return FEA_OK;
  if (E == 0) {
    if (gx) FEA_CUDA(cudaMemsetAsync(gx, 0, 3 * N * sizeof(double), s));
    return FEA_OK;
  }
  FEA_TRY(ensure_scratch(m->gxs, (size_t)E * B->nb * 4 * sizeof(double)));
  AdjArgs A{};
  A.x = m->x;
  A.y = m->y;
  A.z = m->z;
  A.tets = m->tets;
  A.edof = B->edof;
  A.ipos = B->ipos;
  A.rp = B->rp;
  A.slot = B->slot;
  A.E = E;
  A.N = m->n_nodes;
  A.kappa = co->kappa;
  A.kappa_const = co->kappa_const;
  A.mass = form->mass_coef;
  A.fp0 = co->f_param[0];
  A.gv = gv;
  A.gf = gf;
  A.gk = gk;
  A.gxs = static_cast<double*>(m->gxs.ptr);
  A.err = m->err;
  const bool mass = form->kind == FEA_DIFFUSION_MASS && form->mass_coef != 0.0;
  const int load = co->f_kind;
  if (order == 1) {
    if (mass) AdjLauncher<1, true>::run(A, load, q->npts, s);
    else AdjLauncher<1, false>::run(A, load, q->npts, s);
  } else {
    if (mass) AdjLauncher<2, true>::run(A, load, q->npts, s);
    else AdjLauncher<2, false>::run(A, load, q->npts, s);
  }
  FEA_CUDA(cudaGetLastError());
  if (gx) {
    // vertex dofs are the node ids in both numberings, so the first N rows of
    // the order's incidence lists are the node lists
    k_node_grad<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(N, B->inc_ptr, A.gxs, gx);
    FEA_CUDA(cudaGetLastError());
  }
  return FEA_OK;
}

}  // namespace fea

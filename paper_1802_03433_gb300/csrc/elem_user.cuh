// Element kernel template for user-supplied point functions, specialised at
// run time with NVRTC (jit.cu).  The paper's system turns the user's symbolic
// weak form into kernel source and compiles it while the program runs
// (Sec. 5, runtime compilation); here the user gives the coefficient k(x)
// that multiplies kappa_T inside the stiffness integral and the load f(x), as
// CUDA C++ expressions, and jit.cu pastes them into a Spec struct and
// compiles this template for one (order, mass, rule, precision).  The header
// is also compiled ahead of time (it must build with and without NVRTC), so
// it includes only the NVRTC-safe device headers.
//
// Form: -div(kappa_T k(x) grad u) + mass u = f(x) on P1/P2 tets, one thread
// per element, local rows written in incidence order exactly like the
// precompiled kernels, so the same deterministic scatter finishes the job.
//
// Stiffness through coefficient moments.  With Lambda_ij = grad lambda_i .
// grad lambda_j (element constants) and
//   M_ij = sum_q w_q k(x_q) lambda_i(x_q) lambda_j(x_q),
//   m_i = sum_j M_ij = sum_q w_q k(x_q) lambda_i(x_q),  m = sum_i m_i,
// every P2 stiffness entry is a short combination (grad phi_v = (4 lambda_v
// - 1) grad lambda_v, grad phi_(i,j) = 4 (lambda_i grad lambda_j + lambda_j
// grad lambda_i)):
//   vertex a, vertex b:  Lambda_ab (16 M_ab - 4 m_a - 4 m_b + m)
//   vertex a, edge (i,j): 4 [(4 M_ai - m_i) Lambda_aj + (4 M_aj - m_j) Lambda_ai]
//   edge (i,j), edge (k,l): 16 [M_ik Lambda_jl + M_il Lambda_jk + M_jk Lambda_il + M_jl Lambda_ik]
// all times kappa_T |T|; P1 needs only m.  This is the quadrature of the
// caller's rule, reordered: the rule's points enter only through M.  With no
// k (k = 1) the stiffness is the exact one for any rule: P1 uses m = 1 and
// P2 the closed form of the precompiled kernels (element.cuh, p2_stiff).
#pragma once

#include "element.cuh"
#include "vecmem.cuh"

namespace fea {

struct UserArgs {
  const double* x;
  const double* y;
  const double* z;
  const int32_t* tets;   // [4][E]
  int64_t E;
  const double* kappa;   // kappa_T per element, or NULL for kappa_const
  double kappa_const;
  double mass;           // mass coefficient (lambda of Eq. 1)
  double p[4];           // parameters p0..p3 seen by the expressions
  const int32_t* ipos;   // [nb][E] incidence index of (e, a)
  void* Lm;              // local rows, incidence order, lstride(nb) apart
  void* Fl;              // local loads, incidence order (HAS_F only)
  int* err;
  int64_t N;  // node count (bounds of the coordinate gathers in the checked build)
};

constexpr int USER_T = 128;

// Spec provides
//   static constexpr bool HAS_K, HAS_F;
//   template <typename R> static R k(R x, R y, R z, double p0, double p1, double p2, double p3);
//   template <typename R> static R f(R x, R y, R z, double p0, double p1, double p2, double p3);
template <int ORDER, bool MASS, int NPTS, typename R, class Spec>
__device__ __forceinline__ void elem_user_body(const UserArgs& A, int64_t e) {
  constexpr int NB = ORDER == 1 ? 4 : 10;
  double X[4][3];
  {
    int32_t v[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) v[a] = checked_index(__ldg(A.tets + a * A.E + e), A.N, A.err);
    load_vertices(A.x, A.y, A.z, v, X);
  }
  Geo g;
  geometry(X, g);
  if (!(g.det > 0.0)) atomicOr(A.err, DEV_ERR_DEGENERATE);
  const double adet = fabs(g.det);
  const double kT = A.kappa ? __ldg(A.kappa + e) : A.kappa_const;

  // quadrature points, in R
  [[maybe_unused]] R xq[3][NPTS];
  if constexpr (Spec::HAS_K || Spec::HAS_F) {
    R Xr[4][3];
    vertices_r<R>(X, Xr);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R v[4] = {Xr[0][c], Xr[1][c], Xr[2][c], Xr[3][c]};
      quad_coord<NPTS, R>(v, xq[c]);
    }
  }

  // coefficient moments M (upper triangle), m_i, m
  R M[4][4], mi[4], m0;
  if constexpr (Spec::HAS_K) {
    R wk[NPTS];
    static_for<NPTS>([&](auto Q) {
      wk[Q] = R(weight(NPTS, Q)) * Spec::template k<R>(xq[0][Q], xq[1][Q], xq[2][Q], A.p[0], A.p[1], A.p[2], A.p[3]);
    });
    if constexpr (ORDER == 1) {
      m0 = wk[0];
#pragma unroll
      for (int q = 1; q < NPTS; ++q) m0 += wk[q];
    } else {
      static_for<10>([&](auto K) {
        constexpr int i = upper_a(4, K), j = upper_b(4, K);
        R s = R(bary(NPTS, 0, i) * bary(NPTS, 0, j)) * wk[0];
        static_for<NPTS - 1>([&](auto Q) {
          constexpr double c = bary(NPTS, Q + 1, i) * bary(NPTS, Q + 1, j);
          s = fma(R(c), wk[Q + 1], s);
        });
        M[i][j] = s;
        if constexpr (i != j) M[j][i] = s;
      });
#pragma unroll
      for (int i = 0; i < 4; ++i) mi[i] = (M[i][0] + M[i][1]) + (M[i][2] + M[i][3]);
      m0 = (mi[0] + mi[1]) + (mi[2] + mi[3]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j) M[i][j] = R(i == j ? 0.1 : 0.05);
      mi[i] = R(0.25);
    }
    m0 = R(1);
  }

  // Lambda_ij scaled by kappa_T |T|
  R Gr[4][3];
  grads<R>(g, Gr);
  const R s = R(kT * grad_scale<R>(adet) * (ORDER == 2 && !Spec::HAS_K ? 1.0 / 20.0 : 1.0));
  R L[4][4];
  static_for<10>([&](auto K) {
    constexpr int i = upper_a(4, K), j = upper_b(4, K);
    L[i][j] = s * dot3(Gr[i], Gr[j]);
    if constexpr (i != j) L[j][i] = L[i][j];
  });

  R Kl[NB][NB];
  if constexpr (ORDER == 2 && !Spec::HAS_K) {
    // constant coefficient: the closed-form P2 stiffness of the precompiled
    // kernels, K_ab = sum_t num_t Lambda_(i_t j_t) / 20 (the 1/20 is in s)
    R G[4][4];
    static_for<10>([&](auto K) {
      constexpr int i = upper_a(4, K), j = upper_b(4, K);
      G[i][j] = L[i][j];
      if constexpr (i != j) G[j][i] = G[i][j];
    });
    // FP64: |T| / 420 times each of the seven values of the P2 mass pattern
    // starts the entry's FMA chain (one FP64 operation less per entry); the
    // FP32 products of the mixed path add the mass term last
    constexpr bool FOLD = MASS && IsDouble<R>::value;
    [[maybe_unused]] R tm[7];
    [[maybe_unused]] R t = R(0);
    if constexpr (MASS) t = R(A.mass * adet * (1.0 / 2520.0));
    if constexpr (FOLD) {
#pragma unroll
      for (int c = 0; c < 7; ++c) tm[c] = c == 1 ? t : R(p2_mass_value(c)) * t;
    }
    static_for<55>([&](auto K) {
      constexpr int a = upper_a(10, K), b = upper_b(10, K);
      R v;
      if constexpr (FOLD) {
        v = p2_stiff<K, R>(G, tm[p2_mass_class(a, b)]);
      } else {
        v = p2_stiff<K, R>(G);
        if constexpr (MASS) v = fma(t, R(p2_mass420(a, b)), v);
      }
      Kl[a][b] = v;
      Kl[b][a] = v;
    });
  } else if constexpr (ORDER == 1) {
    [[maybe_unused]] R t = R(0);
    if constexpr (MASS) t = R(A.mass * adet * (1.0 / 120.0));
    static_for<10>([&](auto K) {
      constexpr int a = upper_a(4, K), b = upper_b(4, K);
      R v = m0 * L[a][b];
      if constexpr (MASS) v = fma(t, R(a == b ? 2 : 1), v);
      Kl[a][b] = v;
      Kl[b][a] = v;
    });
  } else {
    R Q4[4][4];  // 4 M_ai - m_i
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 4; ++i) Q4[a][i] = fma(R(4), M[a][i], -mi[i]);
    R rv[4];  // m - 4 m_a
#pragma unroll
    for (int a = 0; a < 4; ++a) rv[a] = fma(R(-4), mi[a], m0);
    [[maybe_unused]] R t = R(0);
    if constexpr (MASS) t = R(A.mass * adet * (1.0 / 2520.0));
    static_for<55>([&](auto K) {
      constexpr int a = upper_a(10, K), b = upper_b(10, K);
      R v;
      if constexpr (b < 4) {
        // 16 M_ab - 4 m_a - 4 m_b + m = 4 (4 M_ab - m_b) + (m - 4 m_a)
        v = L[a][b] * fma(R(4), Q4[a][b], rv[a]);
      } else if constexpr (a < 4) {
        constexpr int i = edge_p(b - 4), j = edge_q(b - 4);
        v = R(4) * fma(Q4[a][i], L[a][j], Q4[a][j] * L[a][i]);
      } else {
        constexpr int i = edge_p(a - 4), j = edge_q(a - 4), k = edge_p(b - 4), l = edge_q(b - 4);
        v = R(16) * fma(M[i][k], L[j][l], fma(M[i][l], L[j][k], fma(M[j][k], L[i][l], M[j][l] * L[i][k])));
      }
      if constexpr (MASS) v = fma(t, R(p2_mass420(a, b)), v);
      Kl[a][b] = v;
      Kl[b][a] = v;
    });
  }

  constexpr int LS = lstride(NB, sizeof(R));
  int32_t pos[NB];
#pragma unroll
  for (int a = 0; a < NB; ++a) pos[a] = __ldg(A.ipos + a * A.E + e);
#pragma unroll
  for (int a = 0; a < NB; ++a) store_row<NB>(static_cast<R*>(A.Lm) + (int64_t)pos[a] * LS, Kl[a]);

  if constexpr (Spec::HAS_F) {
    R fq[NPTS];
    static_for<NPTS>([&](auto Q) { fq[Q] = Spec::template f<R>(xq[0][Q], xq[1][Q], xq[2][Q], A.p[0], A.p[1], A.p[2], A.p[3]); });
    const R vol = R(adet * (1.0 / 6.0));
    R* __restrict__ Fl = static_cast<R*>(A.Fl);
    R F[NB];
    rule_sum<ORDER, NPTS, R>(fq, F);
#pragma unroll
    for (int a = 0; a < NB; ++a) Fl[pos[a]] = vol * F[a];
  }
}

template <int ORDER, bool MASS, int NPTS, typename R, class Spec>
__global__ void __launch_bounds__(USER_T) k_elem_user(UserArgs A) {
  const int64_t e = (int64_t)blockIdx.x * USER_T + threadIdx.x;
  if (e < A.E) elem_user_body<ORDER, MASS, NPTS, R, Spec>(A, e);
}

}  // namespace fea

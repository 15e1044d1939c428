// Element kernels: one thread per element computes its local matrix and load
// vector (Sec. 5, Algorithm 1: the integrand evaluation that precedes the
// accumulation into the global system) and writes them to the scratch that
// the deterministic scatter (gather.cuh) reads.  Each local row (e, a) goes,
// as one run of vector stores, to the position of incidence (e, a) in the
// incidence list of global row dof(e, a); the scatter then streams every
// row's contributions from contiguous memory.  Both halves of the symmetric
// local matrix come from the same upper-triangle value (bitwise symmetric).
#pragma once

#include "element.cuh"
#include "internal.cuh"
#include "vecmem.cuh"

namespace fea {

struct ElemArgs {
  const double* x;
  const double* y;
  const double* z;
  const int32_t* tets;  // [4][E]
  int64_t E;            // element count (the SoA stride)
  int64_t e0, e1;       // range of elements this launch computes
  const double* kappa;
  double kappa_const;
  const double* lam;
  double lam_const;
  const double* mu;
  double mu_const;
  double mass;      // mass coefficient (lambda of Eq. 1)
  double fp[4];     // load amplitudes
  const int32_t* ipos;  // [nb][E] incidence index of (e, a)
  void* Lm;         // local rows, incidence order, lstride(nl) values apart
  void* Fl;         // local loads, incidence order
  int* err;
  // atomic comparison path (the paper's sparse Algorithm 1): search the
  // column in the global row and atomicAdd into the CSR values / rhs
  const int32_t* edof;     // [nb][E] scalar dofs
  const int32_t* rp;       // dof-level CSR
  const int32_t* ci;
  double* values;
  double* rhs;
  int64_t N;  // node count (bounds of the coordinate gathers in the checked build)
};

// Algorithm 1, sparse variant (Sec. 5): each local entry is added into the
// global row with atomicAdd after a linear search of the row for its column.
__device__ __forceinline__ void atomic_add_entry(const ElemArgs& A, int64_t row, int32_t col, double v) {
  const int32_t lo = __ldg(A.rp + row), hi = __ldg(A.rp + row + 1);
  for (int32_t p = lo; p < hi; ++p)
    if (__ldg(A.ci + p) == col) {
      atomicAdd(A.values + p, v);
      return;
    }
}

constexpr int ELEM_T = 128;

__device__ __forceinline__ void load_element(const ElemArgs& A, int64_t e, double X[4][3]) {
  int32_t v[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) v[a] = checked_index(__ldg(A.tets + a * A.E + e), A.N, A.err);
  load_vertices(A.x, A.y, A.z, v, X);
}

// The FP64 P2 rows by FMA chains, stored to their positions: the fallback of
// the fixed-point entries for inputs outside their range (Gu: the ten upper
// Gram entries row by row, then the mass scale t).  Out of line, so that the
// kernels carry one copy of the rare path and none of its registers.
template <bool MASS>
static __device__ __noinline__ void p2_rows_fp64_call(const double* __restrict__ Gu, double* __restrict__ Lm,
                                                      const int32_t* __restrict__ ipos, int64_t E, int64_t e) {
  double G[4][4];
  int k = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = i; j < 4; ++j) G[i][j] = Gu[k++];
  const double t = Gu[10];
  double tm[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) tm[c] = MASS ? (c == 1 ? t : p2_mass_value(c) * t) : 0.0;
  double Kl[10][10];
  static_for<55>([&](auto K) {
    constexpr int a = upper_a(10, K), b = upper_b(10, K);
    const double v = MASS ? p2_stiff<K, double>(G, tm[p2_mass_class(a, b)]) : p2_stiff<K, double>(G);
    Kl[a][b] = v;
    Kl[b][a] = v;
  });
#pragma unroll
  for (int a = 0; a < 10; ++a) store_row<10>(Lm + (int64_t)__ldg(ipos + a * E + e) * lstride(10, sizeof(double)), Kl[a]);
}

// ---------------------------------------------------------------- scalar forms
// -div(kappa grad u) [+ mass u] on P1 (ORDER 1) or P2 (ORDER 2) tets.
template <int ORDER, bool MASS, int LOAD, int NPTS, typename R, bool ATOMIC = false>
__device__ __forceinline__ void elem_scalar_body(const ElemArgs& A, int64_t e) {
  constexpr int NB = ORDER == 1 ? 4 : 10;
  double X[4][3];
  load_element(A, e, X);
  Geo g;
  geometry(X, g);
  if (!(g.det > 0.0)) atomicOr(A.err, DEV_ERR_DEGENERATE);
  const double adet = fabs(g.det);
  const double kap = A.kappa ? __ldg(A.kappa + e) : A.kappa_const;
  R Gr[4][3];
  grads<R>(g, Gr);
  R Kl[NB][NB];
  constexpr bool STREAM = ORDER == 2 && !ATOMIC;  // P2 rows stored as they complete
  [[maybe_unused]] int32_t spos[NB];               // their positions (STREAM)
  // Gram matrix G_ij = s grad lambda_i . grad lambda_j; FP64 P1 with a mass
  // term keeps it unscaled and applies s in the FMA that adds the mass
  const R s = R(kap * grad_scale<R>(adet) * (ORDER == 2 ? 1.0 / 20.0 : 1.0));
  constexpr bool SCALE_IN_FMA = ORDER == 1 && MASS && IsDouble<R>::value;
  R G[4][4];
  gram<R>(Gr, SCALE_IN_FMA ? R(1) : s, G);

  if constexpr (ORDER == 1) {
    // K_ab = kappa |T| grad lambda_a . grad lambda_b ; M_ab = |T| (1 + delta_ab) / 20
    [[maybe_unused]] R t1 = R(0), t2 = R(0);  // mass entries |T| / 20 and 2 |T| / 20
    if constexpr (MASS) {
      t1 = R(A.mass * adet * (1.0 / 120.0));
      t2 = t1 + t1;
    }
    static_for<10>([&](auto K) {
      constexpr int a = upper_a(4, K), b = upper_b(4, K);
      R v;
      if constexpr (SCALE_IN_FMA) v = fma(s, G[a][b], a == b ? t2 : t1);
      else if constexpr (MASS) v = G[a][b] + (a == b ? t2 : t1);
      else v = G[a][b];
      Kl[a][b] = v;
      Kl[b][a] = v;
    });
  } else {
    // K_ab = kappa |T| / 20 sum_t num_t (grad lambda_i . grad lambda_j);
    // M_ab = |T| / 420 * m420_ab
    [[maybe_unused]] R t = R(0);
    if constexpr (MASS) t = R(A.mass * adet * (1.0 / 2520.0));
    // rows in order, upper entries computed at their row and mirrored; with
    // STREAM each row is stored as soon as it is complete, so fewer entries
    // are live at a time
    if constexpr (STREAM) {
#pragma unroll
      for (int a = 0; a < NB; ++a) spos[a] = __ldg(A.ipos + a * A.E + e);
    }
    auto put = [&](auto K, R v) {
      constexpr int a = upper_a(10, K), b = upper_b(10, K);
      Kl[a][b] = v;
      Kl[b][a] = v;
      if constexpr (STREAM && b == 9)
        store_row<NB>(static_cast<R*>(A.Lm) + (int64_t)spos[a] * lstride(NB, sizeof(R)), Kl[a]);
    };
    // FP64 (deterministic path): the entries as exact integer sums of the
    // Gram and mass terms in 64-bit fixed point (p2_stiff_fx), on the integer
    // pipes; the FMA chains below for the FP32 path and the atomic kernel
    if constexpr (IsDouble<R>::value && STREAM) {
      int E = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i; j < 4; ++j) E = max(E, exp_bits(G[i][j]) + 2);
      if constexpr (MASS) E = max(E, exp_bits(t) + 5);
      if (E >= P2FX_EMIN && E <= P2FX_EMAX) {
        long long Gf[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = i; j < 4; ++j) Gf[i][j] = to_fx(G[i][j], E - 1019);
        [[maybe_unused]] long long tf = 0;
        if constexpr (MASS) tf = to_fx(t, E - 1017);
        const int p = 1078 - E;
        static_for<55>([&](auto K) {
          constexpr int a = upper_a(10, K), b = upper_b(10, K);
          long long m = 0;
          if constexpr (MASS) m = static_cast<long long>(p2_mass420(a, b)) * tf;
          put(K, fx_to_double(p2_stiff_fx<K>(Gf, m), p));
        });
      } else {
        double Gu[11];
        int k = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = i; j < 4; ++j) Gu[k++] = G[i][j];
        Gu[10] = t;
        p2_rows_fp64_call<MASS>(Gu, static_cast<double*>(A.Lm), A.ipos, A.E, e);
      }
    } else {
      // FP64: |T| / 420 times each of the seven values of the P2 mass pattern
      // starts the entry's FMA chain (one FP64 operation less per entry); the
      // FP32 products of the mixed path add the mass term last
      constexpr bool FOLD = MASS && IsDouble<R>::value;
      [[maybe_unused]] R tm[7];
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
        put(K, v);
      });
    }
  }
  if constexpr (ATOMIC) {
    int32_t d[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) d[a] = __ldg(A.edof + a * A.E + e);
#pragma unroll
    for (int a = 0; a < NB; ++a)
#pragma unroll
      for (int b = 0; b < NB; ++b) atomic_add_entry(A, d[a], d[b], (double)Kl[a][b]);
    if constexpr (LOAD != LOAD_NONE) {
      R Xr[4][3];
      vertices_r<R>(X, Xr);
      R Fs[NB];
      shape_load<ORDER, NPTS, LOAD, R>(Xr, Fs);
      const R amp = R(A.fp[0] * adet * (1.0 / 6.0));
#pragma unroll
      for (int a = 0; a < NB; ++a) atomicAdd(A.rhs + d[a], (double)(amp * Fs[a]));
    }
  } else {
    constexpr int LS = lstride(NB, sizeof(R));
    int32_t pos[NB];
    if constexpr (STREAM) {
#pragma unroll
      for (int a = 0; a < NB; ++a) pos[a] = spos[a];
    } else {
#pragma unroll
      for (int a = 0; a < NB; ++a) pos[a] = __ldg(A.ipos + a * A.E + e);
#pragma unroll
      for (int a = 0; a < NB; ++a) store_row<NB>(static_cast<R*>(A.Lm) + (int64_t)pos[a] * LS, Kl[a]);
    }

    if constexpr (LOAD != LOAD_NONE) {
      R Xr[4][3];
      vertices_r<R>(X, Xr);
      R Fs[NB];
      shape_load<ORDER, NPTS, LOAD, R>(Xr, Fs);
      const R amp = R(A.fp[0] * adet * (1.0 / 6.0));
      R* __restrict__ Fl = static_cast<R*>(A.Fl);
#pragma unroll
      for (int a = 0; a < NB; ++a) Fl[pos[a]] = amp * Fs[a];
    }
  }
}

template <int ORDER, bool MASS, int LOAD, int NPTS, typename R, bool ATOMIC = false>
__global__ void __launch_bounds__(ELEM_T) k_elem_scalar(ElemArgs A) {
  const int64_t e = A.e0 + (int64_t)blockIdx.x * ELEM_T + threadIdx.x;
  if (e < A.e1) elem_scalar_body<ORDER, MASS, LOAD, NPTS, R, ATOMIC>(A, e);
}

// The load vector alone (F_a of Eq. 3 on one element), for running the load
// as its own kernel beside the matrix kernel (launched with LOAD_NONE): the
// matrix part is FP64-bound, the load part bound by the integer-pipe sines.
// |det J| comes from det_only(), the same operations as geometry() in the
// fused kernel, so the loads are bitwise the same.
template <int ORDER, int LOAD, int NPTS, typename R>
__global__ void __launch_bounds__(ELEM_T) k_elem_load(ElemArgs A) {
  constexpr int NB = ORDER == 1 ? 4 : 10;
  const int64_t e = A.e0 + (int64_t)blockIdx.x * ELEM_T + threadIdx.x;
  if (e >= A.e1) return;
  double X[4][3];
  load_element(A, e, X);
  const double adet = fabs(det_only(X));
  R Xr[4][3];
  vertices_r<R>(X, Xr);
  R Fs[NB];
  shape_load<ORDER, NPTS, LOAD, R>(Xr, Fs);
  const R amp = R(A.fp[0] * adet * (1.0 / 6.0));
  R* __restrict__ Fl = static_cast<R*>(A.Fl);
#pragma unroll
  for (int a = 0; a < NB; ++a) Fl[__ldg(A.ipos + a * A.E + e)] = amp * Fs[a];
}

// Matrix and load of the same elements in one kernel, by warp role: in a
// block of 2 * ELEM_T threads the first ELEM_T threads compute the local
// matrices of ELEM_T elements (FP64-bound) and the other ELEM_T threads their
// loads (integer-pipe sines), so both kinds of work share every SM.  The
// role is uniform per warp; the results are those of the separate kernels.
// Element e in one of the two roles: the local matrix (matrix warps) or the
// local load (load warps).
template <int ORDER, bool MASS, int LOAD, int NPTS>
__device__ __forceinline__ void elem_roles_body(const ElemArgs& A, int64_t e, bool matrix) {
  if (matrix) {
    elem_scalar_body<ORDER, MASS, LOAD_NONE, 1, double>(A, e);
  } else {
    constexpr int NB = ORDER == 1 ? 4 : 10;
    double X[4][3];
    load_element(A, e, X);
    const double adet = fabs(det_only(X));
    double Fs[NB];
    shape_load<ORDER, NPTS, LOAD, double>(X, Fs);
    const double amp = A.fp[0] * adet * (1.0 / 6.0);
    double* __restrict__ Fl = static_cast<double*>(A.Fl);
#pragma unroll
    for (int a = 0; a < NB; ++a) Fl[__ldg(A.ipos + a * A.E + e)] = amp * Fs[a];
  }
}

// Three resident blocks per SM (80 registers, about 350 bytes spilled to L1):
// the extra warps hide more of the fixed-latency dependencies than the spills
// cost (P2 64^3: 0.71 ms against 0.82 ms for two blocks; four blocks at 64
// registers spill about 670 bytes and take 0.76 ms).
constexpr int ROLES_MIN_BLOCKS = 3;

template <int ORDER, bool MASS, int LOAD, int NPTS>
__global__ void __launch_bounds__(2 * ELEM_T, ROLES_MIN_BLOCKS) k_elem_roles(ElemArgs A) {
  const int64_t e = A.e0 + (int64_t)blockIdx.x * ELEM_T + (threadIdx.x % ELEM_T);
  if (e >= A.e1) return;
  elem_roles_body<ORDER, MASS, LOAD, NPTS>(A, e, threadIdx.x < ELEM_T);
}

// Deterministic-path output of the elasticity kernel: local rows in
// incidence order (whole sectors) and local loads.
template <int LOAD, int NPTS, typename R>
__device__ __forceinline__ void elast_store(const ElemArgs& A, int64_t e, const double X[4][3], double adet,
                                           const R Kl[12][12]) {
  int32_t pos[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) pos[a] = __ldg(A.ipos + a * A.E + e);
  constexpr int LS = lstride(12, sizeof(R));
#pragma unroll
  for (int r = 0; r < 12; ++r) store_row<12>(static_cast<R*>(A.Lm) + ((int64_t)pos[r / 3] * 3 + r % 3) * LS, Kl[r]);
  if constexpr (LOAD != LOAD_NONE) {
    R Xr[4][3];
    vertices_r<R>(X, Xr);
    R Fs[4];
    shape_load<1, NPTS, LOAD, R>(Xr, Fs);
    const double vol = adet * (1.0 / 6.0);
    const R f0 = R(A.fp[0] * vol), f1 = R(A.fp[1] * vol), f2 = R(A.fp[2] * vol);
    R* __restrict__ Fl = static_cast<R*>(A.Fl);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      Fl[(int64_t)pos[a] * 3 + 0] = f0 * Fs[a];
      Fl[(int64_t)pos[a] * 3 + 1] = f1 * Fs[a];
      Fl[(int64_t)pos[a] * 3 + 2] = f2 * Fs[a];
    }
  }
}

// ---------------------------------------------------------------- elasticity
// K_(a,i),(b,j) = |T| [lam d_i phi_a d_j phi_b + mu d_j phi_a d_i phi_b
//                      + mu delta_ij grad phi_a . grad phi_b]  on P1 tets:
// the 78 upper entries r = 3a + i <= c = 3b + j, handed to put(K, value) in
// upper-triangle order (K the compile-time index of the entry).
template <typename R, typename F>
__device__ __forceinline__ void elast_upper(const Geo& g, double adet, double lam, double mu, F&& put) {
  R Gr[4][3];
  grads<R>(g, Gr);
  const double sc = grad_scale<R>(adet);
  const R Ls = R(lam * sc), Ms = R(mu * sc), LMs = Ls + Ms;
  // diagonal entries of a 3x3 block (i == j): the two product terms share
  // d_i phi_b, so (lam + mu) d_i phi_a d_i phi_b + mu grad phi_a . grad phi_b.
  // Off-diagonal blocks (a < b) take the lam- and mu-scaled gradients of the
  // later vertex b, so vertex 0 needs neither (Lc, Mc of b >= 1 only).
  R Lc[4][3], Mc[4][3], LMc[4][3], D[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Lc[a][k] = Ls * Gr[a][k];
      Mc[a][k] = Ms * Gr[a][k];
      LMc[a][k] = LMs * Gr[a][k];
    }
  // mu |T| grad phi_a . grad phi_b for a, b >= 1; the gradients sum to zero,
  // so the row of vertex 0 is minus the sum of the others (4 FP64 operations
  // fewer than its four dot products)
  static_for<10>([&](auto K) {
    constexpr int a = upper_a(4, K), b = upper_b(4, K);
    if constexpr (a >= 1) {
      D[a][b] = dot3(Mc[a], Gr[b]);
      if constexpr (a != b) D[b][a] = D[a][b];
    }
  });
#pragma unroll
  for (int b = 1; b < 4; ++b) {
    D[0][b] = -(D[1][b] + D[2][b] + D[3][b]);
    D[b][0] = D[0][b];
  }
  D[0][0] = -(D[0][1] + D[0][2] + D[0][3]);
  static_for<78>([&](auto K) {
    constexpr int r = upper_a(12, K), c = upper_b(12, K);
    constexpr int a = r / 3, i = r % 3, b = c / 3, j = c % 3;
    R v;
    if constexpr (i == j) v = fma(LMc[a][i], Gr[b][i], D[a][b]);
    else if constexpr (a == b) v = LMc[a][i] * Gr[a][j];  // (lam + mu) d_i phi_a d_j phi_a
    else v = fma(Gr[a][i], Lc[b][j], Gr[a][j] * Mc[b][i]);
    put(K, v);
  });
}

template <int LOAD, int NPTS, typename R, bool ATOMIC = false>
__global__ void __launch_bounds__(ELEM_T) k_elem_elast(ElemArgs A) {
  const int64_t e = A.e0 + (int64_t)blockIdx.x * ELEM_T + threadIdx.x;
  if (e >= A.e1) return;
  double X[4][3];
  load_element(A, e, X);
  Geo g;
  geometry(X, g);
  if (!(g.det > 0.0)) atomicOr(A.err, DEV_ERR_DEGENERATE);
  const double adet = fabs(g.det);
  const double lam = A.lam ? __ldg(A.lam + e) : A.lam_const;
  const double mu = A.mu ? __ldg(A.mu + e) : A.mu_const;
  R Kl[12][12];
  elast_upper<R>(g, adet, lam, mu, [&](auto K, R v) {
    constexpr int r = upper_a(12, K), c = upper_b(12, K);
    Kl[r][c] = v;
    Kl[c][r] = v;
  });
  if constexpr (ATOMIC) {
    int32_t nd[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) nd[a] = __ldg(A.tets + a * A.E + e);
#pragma unroll
    for (int r = 0; r < 12; ++r)
#pragma unroll
      for (int c = 0; c < 12; ++c)
        atomic_add_entry(A, 3 * (int64_t)nd[r / 3] + r % 3, 3 * nd[c / 3] + c % 3, (double)Kl[r][c]);
    if constexpr (LOAD != LOAD_NONE) {
      R Xr[4][3];
      vertices_r<R>(X, Xr);
      R Fs[4];
      shape_load<1, NPTS, LOAD, R>(Xr, Fs);
      const double vol = adet * (1.0 / 6.0);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) atomicAdd(A.rhs + 3 * (int64_t)nd[a] + i, A.fp[i] * vol * (double)Fs[a]);
    }
  } else {
    elast_store<LOAD, NPTS, R>(A, e, X, adet, Kl);
  }
}

// Launchers (one translation unit per element family).
fea_status launch_elem_p1(const ElemArgs& A, bool mass, int load, int npts, int prec, cudaStream_t s);
fea_status launch_elem_p2(const ElemArgs& A, bool mass, int load, int npts, int prec, cudaStream_t s);
fea_status launch_elem_load(int order, const ElemArgs& A, int load, int npts, int prec, cudaStream_t s);
fea_status launch_elem_roles(int order, bool mass, const ElemArgs& A, int load, int npts, cudaStream_t s);
fea_status launch_elem_elast(const ElemArgs& A, int load, int npts, int prec, cudaStream_t s);

}  // namespace fea

// Chunked scatter of P1 linear elasticity (one CTA per chunk of elements,
// chunks.cu): the local entries of the chunk's elements are accumulated in
// shared memory as fixed-point integers, then each coupling the chunk
// completes is written to the CSR values once, and each coupling it shares
// with other chunks as one FP64 partial sum, which k_chunk_reduce adds in
// chunk order.
//
// Why fixed point.  Eq. 3 sums, per matrix entry, the contributions of every
// element that holds both dofs.  The paper's Algorithm 1 adds them with
// floating-point atomicAdd, whose order (and result) changes from run to run.
// Integer addition is associative, so integer atomics give the same sum in
// any order: the scatter is bitwise reproducible without sorting the
// contributions, and it runs on the integer pipes and the shared-memory
// atomic units, leaving the FP64 pipe (2 DFMA per SM and clock on this part)
// to the element arithmetic.  Each slot (a node pair of the chunk) has its own
// scale 2^(H - Es): Es is the largest exponent bound of the contributing
// elements, computed before any entry is added (phase A), and H = 63 - 2 hbits
// (2^hbits: the most contributions one slot receives) leaves room for the
// contributions to add up without overflow in two 32-bit words (acc_add).  A
// contribution below the slot's resolution 2^(Es - H) is rounded to it; the
// bound is within a factor of a few hundred of the largest entry, so with
// hbits = 5 (24 tets around a vertex) that resolution is about 2^-47 of the
// largest contribution.  The sum is rounded to FP64 once.
//
// Phases of k_elast_chunk (one CTA, CHUNK_T threads, elements strided over
// the threads):
//   A. per element: an upper bound on |K entry| from the Lame parameters, the
//      cofactors of J (in FP32 on edges normalised by their largest exponent)
//      and det J; its exponent is max-reduced into the element's ten slots
//      (and the load bound into its four node slots);
//   B. per element: the local matrix (the FP64 or FP32 arithmetic of the
//      local-row path, elast_upper), each of its 78 upper entries converted
//      at its slot's scale and atomically added into the slot's 3 x 3 block;
//      the 12 load entries likewise into the node slots;
//   C. per slot: the sums converted to FP64 (correctly rounded) and written,
//      to the CSR values (owned slots: both blocks (i, j) and (j, i), the
//      transpose of each other, so the matrix stays bitwise symmetric) or to
//      the partial-sum buffer (shared slots).
// An element with non-finite inputs, det J = 0, or a bound beyond the FP64
// range poisons its slots: their values come out NaN.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "elem_kernels.cuh"

namespace fea {
namespace {

constexpr int CHUNK_T = 128;
constexpr int CHUNK_MIN_BLOCKS = 3;
constexpr int EXP_POISON = 1 << 20;    // a slot exponent at or above: the slot is NaN
constexpr int EXP_EMPTY = -(1 << 20);  // no contribution yet
constexpr int EXP_ZERO = -1200;        // bound of contributions that are all zero
// A partial sum of a shared 3 x 3 block takes 12 doubles (three whole 32-byte
// sectors, so its stores never leave a sector partly written), a partial load
// 4 (one sector).
constexpr int PART_STRIDE = 12;

struct ChunkArgs {
  const int32_t* cptr;
  const int32_t* celem;
  const uint16_t* eslot;
  const int32_t* sptr;
  const int32_t* nptr;
  const int4* srec;
  const int2* nrec;
  int H;          // fixed-point scale of a slot: value * 2^(H - Es)
  int K;          // split of a fixed-point value q = hi 2^K + lo, 0 <= lo < 2^K
  int ef;         // |f_c| < 2^ef for the load amplitudes (EXP_ZERO: no load, EXP_POISON: non-finite)
  int max_slots;  // shared-memory capacity
  int max_nodes;
  double* values;
  double* rhs;
  double* part;   // [npart][PART_STRIDE] partial sums of shared couplings (9 used)
  double* npart;  // [nnpart][4] partial sums of shared node loads (3 used)
};

// |x| < 2^result for a positive normal float.
__device__ __forceinline__ int fexp_bound(float y) { return ((__float_as_int(y) >> 23) & 0xFF) - 126; }

// v * 2^(1022 - eb) as a float, truncated (eb: the largest biased exponent
// among the values normalised together, so the result is below 1 in size);
// values 2^-126 or more below the largest become 0.
__device__ __forceinline__ float scaled_f32(double v, int eb) {
  const int hi = __double2hiint(v);
  const unsigned lo = static_cast<unsigned>(__double2loint(v));
  const int ev = (hi >> 20) & 0x7FF;
  const int fe = ev - eb + 126;
  if (ev == 0 || fe <= 0) return 0.0f;
  const unsigned bits = (static_cast<unsigned>(hi) & 0x80000000u) | (static_cast<unsigned>(fe) << 23) |
                        ((static_cast<unsigned>(hi) & 0xFFFFFu) << 3) | (lo >> 29);
  return __uint_as_float(bits);
}

// Exponent bounds of one element's matrix entries (EK) and load entries (EF)
// from FP64 arithmetic: the fallback for very flat elements, where the FP32
// determinant of the normalised edges is too small to trust.  det J = 0
// gives zero loads and a poisoned matrix.
static __device__ __noinline__ int2 elast_bounds_fp64(double e00, double e01, double e02, double e10, double e11,
                                                      double e12, double e20, double e21, double e22, double C,
                                                      int ef) {
  const double e[3][3] = {{e00, e01, e02}, {e10, e11, e12}, {e20, e21, e22}};
  double c[4][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double* u = e[(i + 1) % 3];
    const double* w = e[(i + 2) % 3];
    c[i + 1][0] = u[1] * w[2] - u[2] * w[1];
    c[i + 1][1] = u[2] * w[0] - u[0] * w[2];
    c[i + 1][2] = u[0] * w[1] - u[1] * w[0];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) c[0][k] = -(c[1][k] + c[2][k] + c[3][k]);
  const double det = fabs(e[0][0] * c[1][0] + e[0][1] * c[1][1] + e[0][2] * c[1][2]);
  if (!isfinite(det)) return make_int2(EXP_POISON, EXP_POISON);
  if (!(det > 0.0)) return make_int2(EXP_POISON, EXP_ZERO);
  double n2 = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) n2 = fmax(n2, c[a][0] * c[a][0] + c[a][1] * c[a][1] + c[a][2] * c[a][2]);
  // |K| <= (|lam| + 2|mu|) |T| max |grad phi|^2 = C n2 / (6 |det|); 2 bits of margin
  const double B = C * n2 / (6.0 * det) * 4.0;
  int ek = EXP_POISON, ed;
  if (isfinite(B)) {
    frexp(B, &ek);
    if (B == 0.0) ek = EXP_ZERO;
  }
  frexp(det, &ed);
  return make_int2(ek, ef >= EXP_POISON ? EXP_POISON : (ef <= EXP_ZERO ? EXP_ZERO : ef + ed - 1));
}

// The bounds of phase A: |entry| <= (|lam| + 2|mu|) |T| max_a |grad phi_a|^2
// = C max_a |c_a|^2 / (6 |det J|) with c_a the cofactor rows of J (each term
// of an entry is at most (|lam| + 2 |mu|) |grad phi_a| |grad phi_b| in size),
// and |load entry| <= |f| (sum of the rule's |weights|) |T| < |f| |det J| / 4.
// The edges of J are formed in FP64 (9 subtractions); everything else runs in
// FP32 on the edges normalised by their largest exponent, with margins for
// the FP32 rounding (the scale factors are exact powers of two).
__device__ __forceinline__ int2 elast_bounds(const double X[4][3], double lam, double mu, int ef) {
  double e[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) e[i][k] = X[i + 1][k] - X[0][k];
  int eb = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) eb = max(eb, (__double2hiint(e[i][k]) >> 20) & 0x7FF);
  const double C = fma(2.0, fabs(mu), fabs(lam));
  const int hC = __double2hiint(C);
  const int eC = (hC >> 20) & 0x7FF;
  if (eb == 2047) return make_int2(EXP_POISON, EXP_POISON);  // non-finite coordinates
  if (eb == 0) return make_int2(EXP_POISON, EXP_ZERO);        // every edge zero: det J = 0
  float f[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) f[i][k] = scaled_f32(e[i][k], eb);
  float c[4][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float* u = f[(i + 1) % 3];
    const float* w = f[(i + 2) % 3];
    c[i + 1][0] = fmaf(u[1], w[2], -u[2] * w[1]);
    c[i + 1][1] = fmaf(u[2], w[0], -u[0] * w[2]);
    c[i + 1][2] = fmaf(u[0], w[1], -u[1] * w[0]);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) c[0][k] = -(c[1][k] + c[2][k] + c[3][k]);
  const float ad = fabsf(fmaf(f[0][0], c[1][0], fmaf(f[0][1], c[1][1], f[0][2] * c[1][2])));
  if (!(ad > 0x1p-12f))
    return elast_bounds_fp64(e[0][0], e[0][1], e[0][2], e[1][0], e[1][1], e[1][2], e[2][0], e[2][1], e[2][2], C, ef);
  float n2 = 0.0f;
#pragma unroll
  for (int a = 0; a < 4; ++a) n2 = fmaxf(n2, fmaf(c[a][0], c[a][0], fmaf(c[a][1], c[a][1], c[a][2] * c[a][2])));
  // errors of the normalised FP32 quantities are below 2^-19 (edges truncated
  // by 2^-23 relative, a few roundings of terms below 8 in size)
  const float r = (n2 * (1.0f + 0x1p-10f) + 0x1p-17f) / (6.0f * (ad - 0x1p-17f));
  int ek;
  if (eC == 2047) {
    ek = EXP_POISON;  // non-finite Lame parameters
  } else if (eC == 0) {
    if (C == 0.0) ek = EXP_ZERO;
    else ek = -1022 + (eb - 1022) + fexp_bound(r) + 1;  // C < 2^-1022
  } else {
    const float mC = __uint_as_float(0x3F800000u | ((static_cast<unsigned>(hC) & 0xFFFFFu) << 3) |
                                     (static_cast<unsigned>(__double2loint(C)) >> 29));
    ek = (eC - 1023) + (eb - 1022) + fexp_bound(mC * r) + 1;
  }
  if (ek > 1023) ek = EXP_POISON;
  else if (ek < EXP_ZERO) ek = EXP_ZERO;
  int efo = EXP_ZERO;
  if (ef >= EXP_POISON) efo = EXP_POISON;
  else if (ef > EXP_ZERO) efo = max(EXP_ZERO, ef + 3 * (eb - 1022) + fexp_bound(ad + 0x1p-17f) - 1);
  return make_int2(ek, efo);
}

// round(v 2^sh) as a 64-bit integer (ties away from zero); |v 2^sh| < 2^62
// by the slot's bound.
__device__ __forceinline__ long long fx_of(double v, int sh) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const int ev = static_cast<int>(b >> 52) & 0x7FF;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (ev ? (1ull << 52) : 0ull);
  const int k = max(ev, 1) - 1075 + sh;  // v 2^sh = m 2^k
  unsigned long long mag;
  if (k >= 0) mag = m << min(k, 63);
  else mag = -k > 63 ? 0ull : ((m >> (-k - 1)) + 1ull) >> 1;
  return (b >> 63) ? -static_cast<long long>(mag) : static_cast<long long>(mag);
}
__device__ __forceinline__ long long fx_of(float v, int sh) {
  const unsigned u = __float_as_uint(v);
  const int ev = static_cast<int>(u >> 23) & 0xFF;
  const unsigned long long m = (u & 0x7FFFFFu) | (ev ? 0x800000u : 0u);
  const int k = max(ev, 1) - 150 + sh;
  unsigned long long mag;
  if (k >= 0) mag = m << min(k, 63);
  else mag = -k > 63 ? 0ull : ((m >> (-k - 1)) + 1ull) >> 1;
  return (u >> 31) ? -static_cast<long long>(mag) : static_cast<long long>(mag);
}

// q 2^e2 correctly rounded to FP64 (ties to even), with integer operations;
// results outside the normal range take ldexp.
__device__ __forceinline__ double f64_of(long long q, int e2) {
  if (q == 0) return 0.0;
  const unsigned long long sgn = q < 0 ? (1ull << 63) : 0ull;
  unsigned long long mag = q < 0 ? 0ull - static_cast<unsigned long long>(q) : static_cast<unsigned long long>(q);
  const int lz = __clzll(static_cast<long long>(mag));
  mag <<= lz;
  const unsigned long long low = mag & 0x7FFull;
  unsigned long long mant = mag >> 11;  // 53 bits, the top one set
  mant += (low > 0x400ull) || (low == 0x400ull && (mant & 1ull));
  const int be = 63 - lz + e2 + 1023;   // biased exponent of the result
  if (be <= 0 || be >= 2047) return ldexp(static_cast<double>(q), e2);
  return __longlong_as_double(static_cast<long long>(sgn | ((static_cast<unsigned long long>(be - 1) << 52) + mant)));
}

// vertex pair (a, b), a < b, of an element -> its index among the ten pairs
__host__ __device__ constexpr int pair_index(int a, int b) {
  return a == b ? a : (a == 0 ? 3 + b : (a == 1 ? 5 + b : 9));
}

// Add a fixed-point value into a two-word accumulator with two 32-bit
// shared-memory atomics (native, no return value used, so the warp does not
// wait for them): lo takes q mod 2^K, hi takes floor(q / 2^K).  With at most
// 2^hbits contributions, K = 32 - hbits and H = 63 - 2 hbits neither word
// overflows, and hi 2^K + lo is the exact sum.
__device__ __forceinline__ void acc_add(unsigned* lo, int* hi, long long q, int K) {
  atomicAdd(lo, static_cast<unsigned>(q) & ((1u << K) - 1u));
  atomicAdd(hi, static_cast<int>(q >> K));
}
__device__ __forceinline__ long long acc_sum(const unsigned* lo, const int* hi, int K) {
  return (static_cast<long long>(*hi) << K) + static_cast<long long>(*lo);
}

template <int LOAD, int NPTS, typename R>
__global__ void __launch_bounds__(CHUNK_T, CHUNK_MIN_BLOCKS) k_elast_chunk(ElemArgs A, ChunkArgs C) {
  extern __shared__ unsigned smem_acc[];
  unsigned* alo = smem_acc;                                     // [max_slots][9] low words
  int* ahi = reinterpret_cast<int*>(alo + 9 * C.max_slots);     // [max_slots][9] high words
  unsigned* rlo = reinterpret_cast<unsigned*>(ahi + 9 * C.max_slots);  // [max_nodes][3]
  int* rhi = reinterpret_cast<int*>(rlo + 3 * C.max_nodes);     // [max_nodes][3]
  int* sexp = rhi + 3 * C.max_nodes;                            // [max_slots]
  int* rexp = sexp + C.max_slots;                               // [max_nodes]
  const int c = blockIdx.x, tid = threadIdx.x;
  const int e0 = C.cptr[c], ne = C.cptr[c + 1] - e0;
  const int s0 = C.sptr[c], ns = C.sptr[c + 1] - s0;
  const int n0 = C.nptr[c], nn = C.nptr[c + 1] - n0;
  constexpr bool HAS_LOAD = LOAD != LOAD_NONE;
  const int K = C.K;
  for (int i = tid; i < 9 * ns; i += CHUNK_T) {
    alo[i] = 0u;
    ahi[i] = 0;
  }
  for (int i = tid; i < 3 * nn; i += CHUNK_T) {
    rlo[i] = 0u;
    rhi[i] = 0;
  }
  for (int i = tid; i < ns; i += CHUNK_T) sexp[i] = EXP_EMPTY;
  for (int i = tid; i < nn; i += CHUNK_T) rexp[i] = EXP_EMPTY;
  __syncthreads();
  // Elements are dealt to the lanes across 64 segments of the chunk (lane i
  // takes position i / 64 of segment i % 64): neighbouring elements, which
  // share node pairs, go to different warp instructions, so the atomics of
  // one instruction seldom hit the same accumulator.
  const int L = (ne + 63) >> 6;
  // A: exponent bounds of every slot
  for (int i = tid; i < 64 * L; i += CHUNK_T) {
    const int t = (i & 63) * L + (i >> 6);
    if (t >= ne) continue;
    const int64_t e = C.celem[e0 + t];
    double X[4][3];
    load_element(A, e, X);
    const double lam = A.lam ? __ldg(A.lam + e) : A.lam_const;
    const double mu = A.mu ? __ldg(A.mu + e) : A.mu_const;
    const int2 eb = elast_bounds(X, lam, mu, C.ef);
#pragma unroll
    for (int k = 0; k < 10; ++k) atomicMax(sexp + (C.eslot[k * A.E + e0 + t] & 0x7FFF), eb.x);
    if constexpr (HAS_LOAD) {
#pragma unroll
      for (int k = 0; k < 4; ++k) atomicMax(rexp + C.eslot[k * A.E + e0 + t], eb.y);
    }
  }
  __syncthreads();
  // B: the entries, added in fixed point
  for (int i = tid; i < 64 * L; i += CHUNK_T) {
    const int t = (i & 63) * L + (i >> 6);
    if (t >= ne) continue;
    const int64_t e = C.celem[e0 + t];
    int slot[10], sh[10];
    bool tr[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      const int v = C.eslot[k * A.E + e0 + t];
      slot[k] = v & 0x7FFF;
      tr[k] = (v & 0x8000) != 0;
      sh[k] = C.H - sexp[slot[k]];
    }
    double X[4][3];
    load_element(A, e, X);
    Geo g;
    geometry(X, g);
    if (!(g.det > 0.0)) atomicOr(A.err, DEV_ERR_DEGENERATE);
    const double adet = fabs(g.det);
    const double lam = A.lam ? __ldg(A.lam + e) : A.lam_const;
    const double mu = A.mu ? __ldg(A.mu + e) : A.mu_const;
    elast_upper<R>(g, adet, lam, mu, [&](auto KK, R v) {
      constexpr int r = upper_a(12, KK), cc = upper_b(12, KK);
      constexpr int a = r / 3, i3 = r % 3, b = cc / 3, j3 = cc % 3;
      constexpr int k = pair_index(a, b);
      const int idx = 9 * slot[k] + ((a != b && tr[k]) ? 3 * j3 + i3 : 3 * i3 + j3);
      acc_add(alo + idx, ahi + idx, fx_of(v, sh[k]), K);
    });
    if constexpr (HAS_LOAD) {
      R Xr[4][3];
      vertices_r<R>(X, Xr);
      R Fs[4];
      shape_load<1, NPTS, LOAD, R>(Xr, Fs);
      const double vol = adet * (1.0 / 6.0);
      const R f[3] = {R(A.fp[0] * vol), R(A.fp[1] * vol), R(A.fp[2] * vol)};
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int shf = C.H - rexp[slot[a]];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int idx = 3 * slot[a] + q;
          acc_add(rlo + idx, rhi + idx, fx_of(R(f[q] * Fs[a]), shf), K);
        }
      }
    }
  }
  __syncthreads();
  // C: sums to FP64; owned slots to the CSR values, shared ones to partials
  for (int k = tid; k < ns; k += CHUNK_T) {
    const int4 rec = C.srec[s0 + k];
    const int es = sexp[k];
    double v[9];
    if (es >= EXP_POISON) {
#pragma unroll
      for (int q = 0; q < 9; ++q) v[q] = __longlong_as_double(0x7FF8000000000000LL);
    } else {
#pragma unroll
      for (int q = 0; q < 9; ++q) v[q] = f64_of(acc_sum(alo + 9 * k + q, ahi + 9 * k + q, K), es - C.H);
    }
    if (k < nn) {  // node slot: the upper triangle was accumulated; mirror it
      v[3] = v[1];
      v[6] = v[2];
      v[7] = v[5];
    }
    if (rec.w < 0) {
      const int Li = rec.z & 0xFFFF, Lj = rec.z >> 16;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) C.values[(int64_t)rec.x + i * Li + j] = v[3 * i + j];
      if (k >= nn) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int i = 0; i < 3; ++i) C.values[(int64_t)rec.y + j * Lj + i] = v[3 * i + j];
      }
    } else {
      double* p = C.part + PART_STRIDE * (int64_t)rec.w;
      st_v4(p, v[0], v[1], v[2], v[3]);
      st_v4(p + 4, v[4], v[5], v[6], v[7]);
      st_v4(p + 8, v[8], 0.0, 0.0, 0.0);
    }
  }
  if (C.rhs) {
    for (int k = tid; k < nn; k += CHUNK_T) {
      const int2 nr = C.nrec[n0 + k];
      const int es = rexp[k];
      double f[3];
#pragma unroll
      for (int q = 0; q < 3; ++q)
        f[q] = es >= EXP_POISON ? __longlong_as_double(0x7FF8000000000000LL)
                                : f64_of(acc_sum(rlo + 3 * k + q, rhi + 3 * k + q, K), es - C.H);
      if (nr.y < 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) C.rhs[3 * (int64_t)nr.x + q] = f[q];
      } else {
        st_v4(C.npart + 4 * (int64_t)nr.y, f[0], f[1], f[2], 0.0);
      }
    }
  }
}

// The couplings shared by several chunks: their partial sums, contiguous
// and in chunk order, added and written as both 3 x 3 blocks.
__global__ void k_chunk_reduce(const int32_t* __restrict__ gptr, const int4* __restrict__ grec, int64_t ngroup,
                               const double* __restrict__ part, double* __restrict__ values) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroup) return;
  const int32_t p0 = gptr[g], p1 = gptr[g + 1];
  double v[12];
  const double* src = part + PART_STRIDE * (int64_t)p0;
  ld_v4(src, v[0], v[1], v[2], v[3]);
  ld_v4(src + 4, v[4], v[5], v[6], v[7]);
  ld_v4(src + 8, v[8], v[9], v[10], v[11]);
  for (int32_t p = p0 + 1; p < p1; ++p) {
    src = part + PART_STRIDE * (int64_t)p;
    double w[12];
    ld_v4(src, w[0], w[1], w[2], w[3]);
    ld_v4(src + 4, w[4], w[5], w[6], w[7]);
    ld_v4(src + 8, w[8], w[9], w[10], w[11]);
#pragma unroll
    for (int q = 0; q < 9; ++q) v[q] += w[q];
  }
  const int4 rec = grec[g];
  const int Li = rec.z & 0xFFFF, Lj = rec.z >> 16;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) values[(int64_t)rec.x + i * Li + j] = v[3 * i + j];
  if (rec.x != rec.y) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i) values[(int64_t)rec.y + j * Lj + i] = v[3 * i + j];
  }
}

__global__ void k_chunk_reduce_nodes(const int32_t* __restrict__ gptr, const int32_t* __restrict__ gnode,
                                     int64_t ngroup, const double* __restrict__ npart, double* __restrict__ rhs) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroup) return;
  const int32_t p0 = gptr[g], p1 = gptr[g + 1];
  double f[4];
  ld_v4(npart + 4 * (int64_t)p0, f[0], f[1], f[2], f[3]);
  for (int32_t p = p0 + 1; p < p1; ++p) {
    double w[4];
    ld_v4(npart + 4 * (int64_t)p, w[0], w[1], w[2], w[3]);
#pragma unroll
    for (int q = 0; q < 3; ++q) f[q] += w[q];
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) rhs[3 * (int64_t)gnode[g] + q] = f[q];
}

__global__ void k_zero_nodes(const int32_t* __restrict__ nodes, int64_t n, double* __restrict__ rhs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * n) rhs[3 * (int64_t)nodes[i / 3] + i % 3] = 0.0;
}

template <int LOAD, int NPTS, typename R>
fea_status launch_one(const ElemArgs& A, const ChunkArgs& Cg, int64_t nchunk, size_t smem, cudaStream_t s) {
  static size_t configured = 0;  // opt-in above the 48 KB default, once per instance
  if (smem > 48 * 1024 && smem > configured) {
    FEA_CUDA(cudaFuncSetAttribute(k_elast_chunk<LOAD, NPTS, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    configured = smem;
  }
  k_elast_chunk<LOAD, NPTS, R><<<(unsigned)nchunk, CHUNK_T, smem, s>>>(A, Cg);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

template <typename R>
fea_status launch_prec(const ElemArgs& A, const ChunkArgs& Cg, int64_t nchunk, size_t smem, int load, int npts,
                       cudaStream_t s) {
  if (load == LOAD_NONE) return launch_one<LOAD_NONE, 1, R>(A, Cg, nchunk, smem, s);
  if (load == LOAD_CONST) {
    if (npts == 1) return launch_one<LOAD_CONST, 1, R>(A, Cg, nchunk, smem, s);
    if (npts == 4) return launch_one<LOAD_CONST, 4, R>(A, Cg, nchunk, smem, s);
    return launch_one<LOAD_CONST, 11, R>(A, Cg, nchunk, smem, s);
  }
  if (npts == 1) return launch_one<LOAD_SIN, 1, R>(A, Cg, nchunk, smem, s);
  if (npts == 4) return launch_one<LOAD_SIN, 4, R>(A, Cg, nchunk, smem, s);
  return launch_one<LOAD_SIN, 11, R>(A, Cg, nchunk, smem, s);
}

// |f_c| < 2^result over the three load amplitudes.
int load_exponent(const fea_coeffs* co, int load) {
  if (load == LOAD_NONE) return EXP_ZERO;
  double m = 0.0;
  for (int q = 0; q < 3; ++q) {
    const double a = std::fabs(co->f_param[q]);
    if (!std::isfinite(a)) return EXP_POISON;
    m = std::max(m, a);
  }
  if (m == 0.0) return EXP_ZERO;
  int e = 0;
  std::frexp(m, &e);
  return e;
}

}  // namespace

fea_status assemble_chunked(fea_mesh* m, Pattern* P, const fea_coeffs* co, const fea_quadrature* q, int load,
                            double* values, double* rhs, cudaStream_t s) {
  FEA_TRY(build_chunks(m, P, s));
  const Chunks* K = P->chunks;
  FEA_TRY(ensure_scratch(m->part, (size_t)std::max<int64_t>(K->npart, 1) * PART_STRIDE * sizeof(double)));
  if (rhs) FEA_TRY(ensure_scratch(m->npart, (size_t)std::max<int64_t>(K->nnpart, 1) * 4 * sizeof(double)));
  ElemArgs A{};
  A.x = m->x;
  A.y = m->y;
  A.z = m->z;
  A.tets = m->tets;
  A.E = m->n_elems;
  A.lam = co->lame_lambda;
  A.lam_const = co->lambda_const;
  A.mu = co->lame_mu;
  A.mu_const = co->mu_const;
  for (int i = 0; i < 4; ++i) A.fp[i] = co->f_param[i];
  A.err = m->err;
  ChunkArgs Cg{};
  Cg.cptr = K->cptr;
  Cg.celem = K->celem;
  Cg.eslot = K->eslot;
  Cg.sptr = K->sptr;
  Cg.nptr = K->nptr;
  Cg.srec = K->srec;
  Cg.nrec = K->nrec;
  Cg.H = 63 - 2 * K->hbits;
  Cg.K = 32 - K->hbits;
  const int ld = rhs ? load : LOAD_NONE;
  Cg.ef = load_exponent(co, ld);
  Cg.max_slots = K->max_slots;
  Cg.max_nodes = K->max_nodes;
  Cg.values = values;
  Cg.rhs = rhs;
  Cg.part = static_cast<double*>(m->part.ptr);
  Cg.npart = rhs ? static_cast<double*>(m->npart.ptr) : nullptr;
  const size_t smem = (size_t)K->max_slots * (9 * 2 * sizeof(int) + sizeof(int)) +
                      (size_t)K->max_nodes * (3 * 2 * sizeof(int) + sizeof(int));
  if (smem > 227 * 1024) return fail(FEA_ERR_OVERFLOW, "chunked scatter: chunk too large for shared memory");
  if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[0], s));
  if (K->nchunk > 0) {
    if (q->prec == FEA_MIXED) FEA_TRY(launch_prec<float>(A, Cg, K->nchunk, smem, ld, q->npts, s));
    else FEA_TRY(launch_prec<double>(A, Cg, K->nchunk, smem, ld, q->npts, s));
  }
  if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[1], s));
  if (K->ngroup > 0)
    k_chunk_reduce<<<(unsigned)((K->ngroup + 127) / 128), 128, 0, s>>>(K->gptr, K->grec, K->ngroup, Cg.part,
                                                                       values);
  if (rhs && K->niso > 0)
    k_zero_nodes<<<(unsigned)((3 * K->niso + 255) / 256), 256, 0, s>>>(K->iso, K->niso, rhs);
  if (rhs && K->nngroup > 0)
    k_chunk_reduce_nodes<<<(unsigned)((K->nngroup + 127) / 128), 128, 0, s>>>(K->ngptr, K->ngnode, K->nngroup,
                                                                             Cg.npart, rhs);
  FEA_CUDA(cudaGetLastError());
  if (m->profile) {
    FEA_CUDA(cudaEventRecord(m->ev[2], s));
    m->profiled = true;
  }
  return FEA_OK;
}

}  // namespace fea

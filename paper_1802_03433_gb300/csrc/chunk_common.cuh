// Fixed-point accumulation of the chunked scatter, shared by its elasticity
// (elast_chunk.cu) and scalar (scalar_chunk.cu) kernels: the exponent bounds
// of an element's entries (phase A), the conversions between FP64/FP32
// values and fixed-point integers, the two-word shared-memory accumulators,
// and the kernel arguments.
#pragma once

#include <cuda_runtime.h>

#include "elem_kernels.cuh"

namespace fea {
namespace chunkfx {

constexpr int EXP_POISON = 1 << 20;    // a slot exponent at or above: the slot is NaN
constexpr int EXP_EMPTY = -(1 << 20);  // no contribution yet
constexpr int EXP_ZERO = -1200;        // bound of contributions that are all zero

struct ChunkArgs {
  const int32_t* cptr;
  const int32_t* celem;
  const uint16_t* eslot;
  int64_t es;     // row stride of eslot
  const int32_t* sptr;
  const int32_t* nptr;
  const int4* srec;
  const int2* nrec;
  int H;          // fixed-point scale of a slot: value * 2^(H - Es)
  int K;          // split of a fixed-point value q = hi 2^K + lo, 0 <= lo < 2^K
  int ef;         // |f| < 2^ef for the load amplitudes (EXP_ZERO: no load, EXP_POISON: non-finite)
  int max_slots;  // shared-memory capacity
  int max_nodes;
  double* values;
  double* rhs;
  double* part;   // partial sums of shared couplings
  double* npart;  // partial sums of shared loads
  // extents, for the bounds checks of the checked build
  int64_t n_nodes, nnz, n_part, n_npart;
};

// A 3 x 3 block of the CSR values at p, rows L apart, inside [0, nnz)
// (checked build; always true otherwise).
__device__ __forceinline__ bool block_ok(int64_t p, int L, int64_t nnz, int* err) {
  return index_ok(p, nnz, err) && index_ok(p + 2 * (int64_t)L + 2, nnz, err);
}

// |x| < 2^result for a positive normal float.
__device__ __forceinline__ int fexp_bound(float y) { return ((__float_as_int(y) >> 23) & 0xFF) - 126; }

// |x| < 2^result for a positive normal double; 0 for zero or subnormal.
__device__ __forceinline__ int dexp_bound(double y) { return ((__double2hiint(y) >> 20) & 0x7FF) - 1022; }

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

// The exponent of C x (a positive float factor) x 2^e for C >= 0 in FP64: the
// smallest integer E with C x 2^e < 2^E, EXP_ZERO for C = 0, EXP_POISON for a
// non-finite C.  C's mantissa goes to FP32 by truncation (one bit of margin
// is added).
__device__ __forceinline__ int scaled_exp(double C, float x, int e) {
  const int hC = __double2hiint(C);
  const int eC = (hC >> 20) & 0x7FF;
  if (eC == 2047) return EXP_POISON;
  if (eC == 0) return C == 0.0 ? EXP_ZERO : -1022 + e + fexp_bound(x) + 1;  // C < 2^-1022
  const float mC = __uint_as_float(0x3F800000u | ((static_cast<unsigned>(hC) & 0xFFFFFu) << 3) |
                                   (static_cast<unsigned>(__double2loint(C)) >> 29));
  return (eC - 1023) + e + fexp_bound(mC * x) + 1;
}

// Phase-A bounds of one element, from FP64 arithmetic: the fallback for very
// flat elements, where the FP32 determinant of the normalised edges is too
// small to trust.  det J = 0 gives zero loads and a poisoned matrix.
static __device__ __noinline__ int2 element_bounds_fp64(double e00, double e01, double e02, double e10, double e11,
                                                        double e12, double e20, double e21, double e22, double C1,
                                                        double C3, int ef) {
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
  // |entry| <= C1 n2 / (6 |det|) + C3 |det| / 6; two bits of margin
  const double B = (C1 * n2 / (6.0 * det) + C3 * det / 6.0) * 4.0;
  int ek = EXP_POISON, ed;
  if (isfinite(B)) {
    frexp(B, &ek);
    if (B == 0.0) ek = EXP_ZERO;
  }
  frexp(det, &ed);
  return make_int2(ek, ef >= EXP_POISON ? EXP_POISON : (ef <= EXP_ZERO ? EXP_ZERO : ef + ed - 1));
}

// Phase A: exponent bounds of one element's matrix entries (.x) and load
// entries (.y).  With c_a the cofactor rows of J (grad lambda_a = c_a / det J):
//   |matrix entry| <= C1 |T| max_a |grad lambda_a|^2 + C3 |T|
//                   = C1 max_a |c_a|^2 / (6 |det J|) + C3 |det J| / 6,
//   |load entry|   <= |f| (sum of the rule's |weights|) |T| < |f| |det J| / 4,
// with C1, C3 >= 0 from the form's coefficients (elasticity: C1 = |lambda| +
// 2 |mu|; diffusion: C1 = |kappa| times the largest |grad phi|^2 of the basis
// over max |grad lambda|^2, C3 = |mass|).  Everything runs in FP32 on the
// edges of J normalised by their largest exponent (f = e 2^(1022 - eb), the
// largest |f| in [1/2, 1)), with margins for the FP32 rounding (the scale
// factors are exact powers of two); fp64() gives the FP64 bounds of very flat
// elements, where the FP32 determinant is too small to trust.
template <typename FB>
__device__ __forceinline__ int2 bounds_from_edges(const float f[3][3], int eb, double C1, double C3, int ef,
                                                  FB&& fp64) {
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
  if (!(ad > 0x1p-12f)) return fp64();
  float n2 = 0.0f;
#pragma unroll
  for (int a = 0; a < 4; ++a) n2 = fmaxf(n2, fmaf(c[a][0], c[a][0], fmaf(c[a][1], c[a][1], c[a][2] * c[a][2])));
  // the normalised edges are within 2^-22.5 of the exact ones (truncated by
  // 2^-23 relative, or formed from split coordinates: element_bounds_split);
  // from there the cofactors are within 2^-18.6 and det within 2^-18 (a few
  // roundings of terms below 8 in size), inside the margins below; the edges
  // scale by 2^(eb - 1022), so max |c|^2 / det by that and det by its cube
  const float r = (n2 * (1.0f + 0x1p-10f) + 0x1p-17f) / (6.0f * (ad - 0x1p-17f));
  const float dhi = (ad + 0x1p-17f) * (1.0f / 6.0f);
  int ek = scaled_exp(C1, r, eb - 1022);
  if (C3 != 0.0) ek = max(ek, scaled_exp(C3, dhi, 3 * (eb - 1022))) + 1;  // the sum of two terms
  if (ek > 1023) ek = EXP_POISON;
  else if (ek < EXP_ZERO) ek = EXP_ZERO;
  int efo = EXP_ZERO;
  if (ef >= EXP_POISON) efo = EXP_POISON;
  else if (ef > EXP_ZERO) efo = max(EXP_ZERO, ef + 3 * (eb - 1022) + fexp_bound(ad + 0x1p-17f) - 1);
  return make_int2(ek, efo);
}

// Phase A bounds (bounds_from_edges) with the edges of J formed in FP64 (9
// subtractions) and truncated to FP32 after normalisation.
__device__ __forceinline__ int2 element_bounds(const double X[4][3], double C1, double C3, int ef) {
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
  if (eb == 2047) return make_int2(EXP_POISON, EXP_POISON);  // non-finite coordinates
  if (eb == 0) return make_int2(EXP_POISON, EXP_ZERO);        // every edge zero: det J = 0
  float f[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) f[i][k] = scaled_f32(e[i][k], eb);
  return bounds_from_edges(f, eb, C1, C3, ef, [&]() {
    return element_bounds_fp64(e[0][0], e[0][1], e[0][2], e[1][0], e[1][1], e[1][2], e[2][0], e[2][1], e[2][2], C1,
                               C3, ef);
  });
}

// v truncated to a float (24 significant bits), by bit moves; v zero or a
// normal number inside FP32's normal range.
__device__ __forceinline__ float trunc_f32(double v) {
  if (v == 0.0) return 0.0f;
  const int hi = __double2hiint(v);
  const unsigned lo = static_cast<unsigned>(__double2loint(v));
  const int ev = (hi >> 20) & 0x7FF;
  return __uint_as_float((static_cast<unsigned>(hi) & 0x80000000u) | (static_cast<unsigned>(ev - 1023 + 127) << 23) |
                         ((static_cast<unsigned>(hi) & 0xFFFFFu) << 3) | (lo >> 29));
}
// A float as a double (exact), by bit moves; f zero or normal.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  if ((u & 0x7FFFFFFFu) == 0u) return f;
  const unsigned ef = (u >> 23) & 0xFF;
  return __hiloint2double(static_cast<int>((u & 0x80000000u) | ((ef - 127 + 1023) << 20) | ((u & 0x7FFFFFu) >> 3)),
                          static_cast<int>(u << 29));
}

// A staged coordinate as two floats, x = h + l + d with h = x truncated to
// 24 bits, l = (x - h) truncated (x - h is exact in FP64: one subtraction),
// |d| < 2^-46 |x|; false (and nothing to use) unless x is zero or
// 2^-70 <= |x| < 2^70, which keeps h and l normal floats.
__device__ __forceinline__ bool split_coord(double x, float& h, float& l) {
  h = 0.0f;
  l = 0.0f;
  if (x == 0.0) return true;
  const int ex = (__double2hiint(x) >> 20) & 0x7FF;
  if (ex < 1023 - 70 || ex >= 1023 + 70) return false;  // also non-finite
  h = trunc_f32(x);
  l = trunc_f32(x - f32_to_f64(h));
  return true;
}

// Phase A bounds (bounds_from_edges) from split coordinates (split_coord),
// without FP64 arithmetic: each edge of J is (h1 - h0) + (l1 - l0) in FP32.
// With X the largest |coordinate| of the element and emax its largest |edge|
// component, an edge is within 2^-23 |e| + 2^-45.9 X of the exact one; the
// element takes this path when X < 2^20 emax (so within 2^-22.5 of emax, the
// accuracy the margins of bounds_from_edges allow), else fb() (FP64 edges).
template <typename FB>
__device__ __forceinline__ int2 element_bounds_split(const float H[4][3], const float Lo[4][3], double C1, double C3,
                                                     int ef, FB&& fb) {
  float e[3][3];
  float emax = 0.0f, xmax = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      e[i][k] = (H[i + 1][k] - H[0][k]) + (Lo[i + 1][k] - Lo[0][k]);
      emax = fmaxf(emax, fabsf(e[i][k]));
    }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) xmax = fmaxf(xmax, fabsf(H[a][k]));
  if (!(emax >= 0x1p-100f) || !(xmax < 0x1p20f * emax)) return fb();
  const int Ef = ((__float_as_int(emax) >> 23) & 0xFF) - 127;  // 2^Ef <= emax < 2^(Ef + 1)
  const float sc = __int_as_float((127 - Ef - 1) << 23);          // 2^(-Ef - 1), exact
  float f[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) f[i][k] = e[i][k] * sc;
  return bounds_from_edges(f, Ef + 1023, C1, C3, ef, fb);
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
// round(F 2^k) for an integer F (ties away from zero).
__device__ __forceinline__ long long fx_shift(long long F, int k) {
  const unsigned long long m = F < 0 ? 0ull - static_cast<unsigned long long>(F) : static_cast<unsigned long long>(F);
  unsigned long long mag;
  if (k >= 0) mag = m << min(k, 63);
  else mag = -k > 63 ? 0ull : ((m >> (-k - 1)) + 1ull) >> 1;
  return F < 0 ? -static_cast<long long>(mag) : static_cast<long long>(mag);
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

}  // namespace chunkfx
}  // namespace fea

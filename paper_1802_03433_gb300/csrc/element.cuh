// Device-side element math: geometry, quadrature rules, local matrices and
// local load vectors of P1/P2 tetrahedra (the per-element work of Sec. 5,
// Algorithm 1: evaluate the weak-form integrand of Eq. 2 on one element).
//
// One thread owns one element.  On GB300 the FP64 pipe (about 5e11 FMA/s per
// GPU) is the scarce resource, so every formula here is written to spend as
// few FP64 operations as the arithmetic allows:
//   * geometry works with the unscaled cofactor vectors c_a (grad lambda_a =
//     c_a / det J) and folds 1/det J into one scale factor per element;
//   * bilinear forms with element-constant coefficients on affine elements
//     are polynomials of degree <= 4, integrated exactly in closed form (the
//     4- and 11-point rules integrate them exactly too, so the values are
//     those of the quadrature up to rounding);
//   * only the upper triangle of each symmetric local matrix is computed and
//     then stored into both halves (bitwise symmetric);
//   * the load vector is a genuine quadrature of f * phi_a with the
//     requested rule, the quadrature points built from the rule's symmetry
//     classes (one FMA per point and coordinate).
// Template parameter R is the arithmetic type of the quadrature-point
// products: double (plain FP64) or float (the mixed-precision split, where
// the Jacobian, det J and J^{-1} stay FP64).
#pragma once

#include "devcommon.cuh"

namespace fea {

enum : int { LOAD_NONE = 0, LOAD_CONST = 1, LOAD_SIN = 2 };

// ------------------------------------------------------------------ rules
// 4-point degree-2 rule: permutations of (a, b, b, b), weight 1/4.
constexpr double R4A = 0.5854101966249684544613761;  // (5 + 3 sqrt 5) / 20
constexpr double R4B = 0.1381966011250105151795413;  // (5 - sqrt 5) / 20
// 11-point degree-4 rule (Keast), weights normalised to sum to 1.
constexpr double K11W0 = -0.07893333333333333333333333;  // 6 * (-74 / 5625), centroid
constexpr double K11W1 = 0.04573333333333333333333333;   // 6 * 343 / 45000
constexpr double K11W2 = 0.1493333333333333333333333;    // 6 * 56 / 2250
constexpr double K11A = 0.7857142857142857142857143;     // 11 / 14
constexpr double K11B = 0.07142857142857142857142857;    // 1 / 14
constexpr double K11C1 = 0.3994035761667992049961021;    // (1 + sqrt(5/14)) / 4
constexpr double K11C2 = 0.1005964238332007950038979;    // (1 - sqrt(5/14)) / 4

// local edge k joins vertices edge_p(k) < edge_q(k)
__host__ __device__ constexpr int edge_p(int k) { return k < 3 ? 0 : (k < 5 ? 1 : 2); }
__host__ __device__ constexpr int edge_q(int k) { return k < 3 ? k + 1 : (k < 5 ? k - 1 : 3); }

// Barycentric coordinate v of point q.  11-point ordering: centroid, the four
// (A, B, B, B) points (vertex q-1 gets A), then the six (C1, C1, C2, C2)
// points (edge q-5 gets C1 on both its vertices).
__host__ __device__ constexpr double bary(int npts, int q, int v) {
  return npts == 1 ? 0.25
       : npts == 4 ? (v == q ? R4A : R4B)
       : (q == 0 ? 0.25
          : q <= 4 ? (v == q - 1 ? K11A : K11B)
          : ((v == edge_p(q - 5) || v == edge_q(q - 5)) ? K11C1 : K11C2));
}
__host__ __device__ constexpr double weight(int npts, int q) {
  return npts == 1 ? 1.0 : npts == 4 ? 0.25 : (q == 0 ? K11W0 : q <= 4 ? K11W1 : K11W2);
}
// Basis function a (order 1: lambda_a; order 2: vertex lambda(2 lambda - 1),
// edge 4 lambda_p lambda_q) at rule point q.
__host__ __device__ constexpr double phi_at(int order, int npts, int q, int a) {
  return order == 1 ? bary(npts, q, a)
       : a < 4 ? bary(npts, q, a) * (2.0 * bary(npts, q, a) - 1.0)
       : 4.0 * bary(npts, q, edge_p(a - 4)) * bary(npts, q, edge_q(a - 4));
}
// sum_q w_q phi_a(q): the load of f = 1 divided by |T|.
__host__ __device__ constexpr double wphi_sum(int order, int npts, int a) {
  double s = 0.0;
  for (int q = 0; q < npts; ++q) s += weight(npts, q) * phi_at(order, npts, q, a);
  return s;
}

// ------------------------------------------------------------------ P2 tables
// d phi_a / d lambda_i for the P2 basis, as (i, alpha + sum_k beta_k lambda_k):
//   vertex v: (v, -1 + 4 lambda_v);  edge (p, q): (p, 4 lambda_q), (q, 4 lambda_p).
struct LinForm {
  int i = 0, alpha = 0;
  int beta[4] = {0, 0, 0, 0};
};
struct DPhi {
  int n = 0;
  LinForm f[2] = {};
};
__host__ __device__ constexpr DPhi p2_dphi(int a) {
  DPhi d{};
  if (a < 4) {
    d.n = 1;
    d.f[0].i = a;
    d.f[0].alpha = -1;
    d.f[0].beta[a] = 4;
  } else {
    const int p = edge_p(a - 4), q = edge_q(a - 4);
    d.n = 2;
    d.f[0].i = p;
    d.f[0].beta[q] = 4;
    d.f[1].i = q;
    d.f[1].beta[p] = 4;
  }
  return d;
}
// 20 |T|^{-1} int_T u v for linear forms in barycentrics, using
// |T|^{-1} int lambda_k lambda_l = (1 + delta_kl) / 20 and int lambda_k = |T| / 4.
__host__ __device__ constexpr int int20(const LinForm& u, const LinForm& v) {
  int su = 0, sv = 0;
  for (int k = 0; k < 4; ++k) {
    su += u.beta[k];
    sv += v.beta[k];
  }
  int r = 20 * u.alpha * v.alpha + 5 * (u.alpha * sv + v.alpha * su);
  for (int k = 0; k < 4; ++k)
    for (int l = 0; l < 4; ++l) r += u.beta[k] * v.beta[l] * (k == l ? 2 : 1);
  return r;
}
// K_ab = kappa |T| / 20 * sum_t num_t * (grad lambda_i_t . grad lambda_j_t).
struct Terms {
  int n = 0;
  int i[4] = {0, 0, 0, 0}, j[4] = {0, 0, 0, 0}, num[4] = {0, 0, 0, 0};
};
__host__ __device__ constexpr Terms p2_terms(int a, int b) {
  Terms t{};
  const DPhi da = p2_dphi(a), db = p2_dphi(b);
  for (int x = 0; x < da.n; ++x)
    for (int y = 0; y < db.n; ++y) {
      int i = da.f[x].i, j = db.f[y].i;
      if (i > j) {
        const int tmp = i;
        i = j;
        j = tmp;
      }
      const int v = int20(da.f[x], db.f[y]);
      int found = -1;
      for (int k = 0; k < t.n; ++k)
        if (t.i[k] == i && t.j[k] == j) found = k;
      if (found >= 0) {
        t.num[found] += v;
      } else {
        t.i[t.n] = i;
        t.j[t.n] = j;
        t.num[t.n] = v;
        ++t.n;
      }
    }
  return t;
}
// 420 |T|^{-1} int phi_a phi_b for the P2 basis.
__host__ __device__ constexpr int p2_mass420(int a, int b) {
  if (a > b) {
    const int t = a;
    a = b;
    b = t;
  }
  if (b < 4) return a == b ? 6 : 1;
  if (a < 4) return (edge_p(b - 4) == a || edge_q(b - 4) == a) ? -4 : -6;
  if (a == b) return 32;
  const int p = edge_p(a - 4), q = edge_q(a - 4), r = edge_p(b - 4), s = edge_q(b - 4);
  return (p == r || p == s || q == r || q == s) ? 16 : 8;
}
// Index of the k-th upper-triangle pair (a <= b) of an n x n matrix, row-major.
__host__ __device__ constexpr int upper_a(int n, int k) {
  int a = 0;
  while (k >= n - a) {
    k -= n - a;
    ++a;
  }
  return a;
}
__host__ __device__ constexpr int upper_b(int n, int k) {
  int a = 0;
  while (k >= n - a) {
    k -= n - a;
    ++a;
  }
  return a + k;
}

// ------------------------------------------------------------------ geometry
struct Geo {
  double c[4][3];  // grad lambda_a = c[a] / det
  double det;
};

__device__ __forceinline__ void load_vertices(const double* __restrict__ x, const double* __restrict__ y,
                                              const double* __restrict__ z, const int32_t v[4],
                                              double X[4][3]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    X[a][0] = __ldg(x + v[a]);
    X[a][1] = __ldg(y + v[a]);
    X[a][2] = __ldg(z + v[a]);
  }
}

// J = [x1 - x0, x2 - x0, x3 - x0]; c_1 = e2 x e3, c_2 = e3 x e1, c_3 = e1 x e2
// are the rows of det(J) J^{-1}; det J = e1 . c_1; c_0 = -(c_1 + c_2 + c_3).
__device__ __forceinline__ void geometry(const double X[4][3], Geo& g) {
  double e[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) e[i][k] = X[i + 1][k] - X[0][k];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double* u = e[(i + 1) % 3];
    const double* w = e[(i + 2) % 3];
    g.c[i + 1][0] = fma(u[1], w[2], -u[2] * w[1]);
    g.c[i + 1][1] = fma(u[2], w[0], -u[0] * w[2]);
    g.c[i + 1][2] = fma(u[0], w[1], -u[1] * w[0]);
  }
  g.det = fma(e[0][0], g.c[1][0], fma(e[0][1], g.c[1][1], e[0][2] * g.c[1][2]));
#pragma unroll
  for (int k = 0; k < 3; ++k) g.c[0][k] = -(g.c[1][k] + g.c[2][k] + g.c[3][k]);
}

// det J alone, by exactly the operations geometry() uses for it (bitwise the
// same value): e_i = x_i - x_0, c_1 = e_2 x e_3, det = e_1 . c_1.
__device__ __forceinline__ double det_only(const double X[4][3]) {
  double e[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) e[i][k] = X[i + 1][k] - X[0][k];
  const double* u = e[1];
  const double* w = e[2];
  const double c0 = fma(u[1], w[2], -u[2] * w[1]);
  const double c1 = fma(u[2], w[0], -u[0] * w[2]);
  const double c2 = fma(u[0], w[1], -u[1] * w[0]);
  return fma(e[0][0], c0, fma(e[0][1], c1, e[0][2] * c2));
}

// sin(pi x) in FP64 with 11 FP64 operations (the library sinpi costs about
// 18 FP64-pipe operations on this part).  Range reduction: adding
// 1.5 * 2^52 rounds x to the nearest integer n (ties to even) and leaves the
// parity of n in the lowest mantissa bit; r = x - n is exact, |r| <= 1/2.
// Then sin(pi x) = (-1)^n r P(r^2), P the degree-7 interpolant of
// sin(pi r)/r at 8 Chebyshev nodes in r^2 on [0, 1/4] (coefficients from
// gen_sinpi.py), within 3.4e-16 of sin(pi x).  |x| >= 2^51, infinities and
// NaNs go to the library function.
constexpr double SINPI_C0 = 3.1415926535897928787;
constexpr double SINPI_C1 = -5.16771278004978582274;
constexpr double SINPI_C2 = 2.55016403986186762969;
constexpr double SINPI_C3 = -0.59926452882522400508;
constexpr double SINPI_C4 = 0.0821458788163104269166;
constexpr double SINPI_C5 = -0.00737036432653041567555;
constexpr double SINPI_C6 = 0.000465987015804337793336;
constexpr double SINPI_C7 = -0.0000211336273520529704044;

__device__ __forceinline__ double sinpi_fp64(double x) {
  const int hi = __double2hiint(x);
  if ((hi & 0x7FF00000) >= ((1023 + 51) << 20)) return sinpi(x);
  constexpr double MAGIC = 6755399441055744.0;  // 1.5 * 2^52
  const double t = x + MAGIC;
  const double n = t - MAGIC;
  const double r = x - n;
  const double u = r * r;
  double p = fma(SINPI_C7, u, SINPI_C6);
  p = fma(p, u, SINPI_C5);
  p = fma(p, u, SINPI_C4);
  p = fma(p, u, SINPI_C3);
  p = fma(p, u, SINPI_C2);
  p = fma(p, u, SINPI_C1);
  p = fma(p, u, SINPI_C0);
  const double sv = p * r;
  const int flip = (__double2loint(t) & 1) << 31;
  return __hiloint2double(__double2hiint(sv) ^ flip, __double2loint(sv));
}

// sin(pi x) to FP64 accuracy with the polynomial on the integer pipes (the
// FP64 pipe retires two operations per SM and clock on this part, the
// integer multiply-add path 64).  For 2^-10 <= |x| < 2^51:
//   * reduction from the bits of x: x = m 2^(e-1075), so the fraction of x in
//     units of 2^-64 is (m << (e - 1011)) mod 2^64 and the parity of the
//     integer part is bit (64 - (e - 1011)) of m; rounding to the nearest
//     integer n leaves r = x - n with |r| <= 1/2 exactly (ra = |r| 2^64);
//   * u = r^2 and the degree-8 interpolant P(u) of sin(pi r)/r (9 Chebyshev
//     nodes on [0, 1/4], relative error 3.2e-19, gen_sinpi.py) by Horner in
//     signed fixed point with 60 fractional bits (64 x 64 -> high 64-bit
//     products);
//   * s = |r| P as the exact 128-bit product, rounded once to the nearest
//     double (ties to even) by integer normalisation;
//   * sign (-1)^n sign(r) sign(x).
// Within 0.51 ulp of sin(pi x) (exact-arithmetic model of these steps against
// 50-digit sin).  In the fast path |r| >= 2^-53, so the product's high word
// is at least 2^8 and every shift below is by 9 to 61 bits.  Other arguments
// (tiny, huge, zero, subnormal, infinite, NaN) take sinpi_fp64.
// The FP64 polynomial out of line, for the rare arguments the fixed-point
// paths hand over: inline, the compiler if-converts the branch and every call
// pays its FP64 operations.
static __device__ __noinline__ double sinpi_fp64_call(double x) { return sinpi_fp64(x); }

constexpr long long SINPI_Q0 = 3622009729038561420LL;
constexpr long long SINPI_Q1 = -5957967193751243029LL;
constexpr long long SINPI_Q2 = 2940138961849612574LL;
constexpr long long SINPI_Q3 = -690904962799911665LL;
constexpr long long SINPI_Q4 = 94707759145125179LL;
constexpr long long SINPI_Q5 = -8497527828481967LL;
constexpr long long SINPI_Q6 = 537607085679486LL;
constexpr long long SINPI_Q7 = -25253012803429LL;
constexpr long long SINPI_Q8 = 887499001982LL;

__device__ __forceinline__ double sinpi_fx(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned e = static_cast<unsigned>(b >> 52) & 0x7FFu;
  if (e - 1013u > 60u) return sinpi_fp64_call(x);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned sh = e - 1011u;  // 2 .. 62
  const unsigned long long f = m << sh;
  const unsigned rneg = static_cast<unsigned>(f >> 63);
  const unsigned par = (sh > 11u ? static_cast<unsigned>(m >> (64u - sh)) & 1u : 0u) ^ rneg;
  const unsigned long long ra = rneg ? 0ull - f : f;
  if (ra == 0ull) return __longlong_as_double(static_cast<long long>(b & 0x8000000000000000ull));
  const long long u = static_cast<long long>(__umul64hi(ra, ra));
  long long p = SINPI_Q8;
  p = __mul64hi(p, u) + SINPI_Q7;
  p = __mul64hi(p, u) + SINPI_Q6;
  p = __mul64hi(p, u) + SINPI_Q5;
  p = __mul64hi(p, u) + SINPI_Q4;
  p = __mul64hi(p, u) + SINPI_Q3;
  p = __mul64hi(p, u) + SINPI_Q2;
  p = __mul64hi(p, u) + SINPI_Q1;
  p = __mul64hi(p, u) + SINPI_Q0;
  const unsigned long long up = static_cast<unsigned long long>(p);
  const unsigned long long hi = __umul64hi(ra, up), lo = ra * up;
  const int lz = __clzll(static_cast<long long>(hi));
  const unsigned long long top = (hi << lz) | (lo >> (64 - lz));
  const bool sticky = (lo << lz) != 0ull;
  unsigned long long mant = top >> 11;
  const unsigned rb = static_cast<unsigned>(top) & 0x7FFu;
  mant += (rb > 0x400u || (rb == 0x400u && (sticky || (mant & 1ull)))) ? 1ull : 0ull;
  const unsigned long long sign = ((b >> 63) ^ par ^ rneg) << 63;
  const unsigned long long bits = (static_cast<unsigned long long>(1025 - lz) << 52) + mant;
  return __longlong_as_double(static_cast<long long>(bits | sign));
}

// |r| P(r^2) 2^62 for ra = |r| 2^64 (|r| <= 1/2): the Horner polynomial of
// sinpi_fx in 60 fractional bits and the 128-bit product |r| P shifted to 62
// fractional bits (truncated).
__device__ __forceinline__ long long sinpi_q62_mag(unsigned long long ra) {
  const long long u = static_cast<long long>(__umul64hi(ra, ra));
  long long p = SINPI_Q8;
  p = __mul64hi(p, u) + SINPI_Q7;
  p = __mul64hi(p, u) + SINPI_Q6;
  p = __mul64hi(p, u) + SINPI_Q5;
  p = __mul64hi(p, u) + SINPI_Q4;
  p = __mul64hi(p, u) + SINPI_Q3;
  p = __mul64hi(p, u) + SINPI_Q2;
  p = __mul64hi(p, u) + SINPI_Q1;
  p = __mul64hi(p, u) + SINPI_Q0;
  const unsigned long long up = static_cast<unsigned long long>(p);
  const unsigned long long hi = __umul64hi(ra, up), lo = ra * up;
  return static_cast<long long>((hi << 2) | (lo >> 62));
}

// sin(pi x) 2^62 as a signed 64-bit integer (|value| <= 2^62), for products
// and sums on the integer pipes: the reduction and polynomial of sinpi_fx,
// then the 128-bit product |r| P shifted to 62 fractional bits (truncated,
// error below 2^-62).  Arguments outside 2^-10 <= |x| < 2^51 take
// sinpi_fp64, scaled exactly and rounded; a non-finite argument gives an
// arbitrary value (an element with such a coordinate has a NaN det J and is
// reported as degenerate).
__device__ __forceinline__ long long sinpi_q62(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned e = static_cast<unsigned>(b >> 52) & 0x7FFu;
  if (e - 1013u > 60u) return __double2ll_rn(sinpi_fp64_call(x) * 4611686018427387904.0);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned sh = e - 1011u;
  const unsigned long long f = m << sh;
  const unsigned rneg = static_cast<unsigned>(f >> 63);
  const unsigned par = (sh > 11u ? static_cast<unsigned>(m >> (64u - sh)) & 1u : 0u) ^ rneg;
  const unsigned long long ra = rneg ? 0ull - f : f;
  const long long mag = sinpi_q62_mag(ra);
  return ((b >> 63) ^ par ^ rneg) ? -mag : mag;
}

// sin(pi x) 2^62 for x given in fixed point, t = x 2^(61 - s) (0 <= s <= 60,
// two's complement): the fraction of x in units of 2^-64 is t << (3 + s) and
// the parity of floor(x) is bit 61 - s of t.  With n the nearest integer to x
// and r = x - n, sin(pi x) = (-1)^n sign(r) |r| P(r^2); when the fraction is
// at least 1/2, n = floor(x) + 1 and r < 0, so both factors flip and the sign
// of the result is the parity of floor(x) alone.  The polynomial and the
// product are those of sinpi_q62.
__device__ __forceinline__ long long sinpi_q62_fx(long long t, int s) {
  const unsigned long long ut = static_cast<unsigned long long>(t);
  const unsigned long long f = ut << (3 + s);
  const unsigned pf = static_cast<unsigned>(ut >> (61 - s)) & 1u;
  const unsigned long long ra = (f >> 63) ? 0ull - f : f;
  const long long mag = sinpi_q62_mag(ra);
  return pf ? -mag : mag;
}
// Four at once: four independent dependency chains (the polynomial is a
// chain of nine 64-bit high products) that the scheduler interleaves.  The
// P2 kernels call it out of line (instruction-cache footprint), so a call
// carries four chains rather than one.
struct Q4 {
  long long v[4];
};
__device__ __forceinline__ Q4 sinpi_q62_fx4(const Q4& t, int s) {
  Q4 r;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.v[k] = sinpi_q62_fx(t.v[k], s);
  return r;
}
static __device__ __noinline__ Q4 sinpi_q62_fx4_call(Q4 t, int s) { return sinpi_q62_fx4(t, s); }
template <bool OUTLINE>
__device__ __forceinline__ Q4 sinpi_q62_fx4_sel(const Q4& t, int s) {
  if constexpr (OUTLINE) return sinpi_q62_fx4_call(t, s);
  else return sinpi_q62_fx4(t, s);
}
// The same with one shift per lane (arguments from different coordinates).
struct S4 {
  int v[4];
};
static __device__ __noinline__ Q4 sinpi_q62_fx4v_call(Q4 t, S4 s) {
  Q4 r;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.v[k] = sinpi_q62_fx(t.v[k], s.v[k]);
  return r;
}

// ---- quadrature-point coordinates in fixed point (the sine load in FP64)
// A coordinate c of the four vertices, v_a, goes to t_a = round(v_a 2^(61 - s))
// with s = max(0, E + 1) for |v_a| < 2^E (E from the largest exponent):
// |t_a| < 2^60, their sum below 2^62, and every point of the rule (a convex
// combination) as well, so nothing wraps.  The conversion shifts the
// mantissa (integer pipes only); the resolution 2^(s - 61) is about 2^-62 of
// max |v_a|, below the rounding of an FP64 evaluation of the point.
// Coordinates of 2^59 and more (and non-finite ones) saturate s at 60 and
// give meaningless sines (such an element has no FP64 fraction left, and a
// non-finite one is reported through its det J).
__device__ __forceinline__ int fx_shift(const double v[4]) {
  int e = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a) e = max(e, static_cast<int>(__double2hiint(v[a]) >> 20) & 0x7FF);
  return min(max(e - 1021, 0), 60);
}
__device__ __forceinline__ long long to_fx(double v, int s) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const int e = static_cast<int>(b >> 52) & 0x7FF;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
  const int k = e - 1014 - s;  // v 2^(61 - s) = m 2^k; k <= 7 for s from fx_shift
  const unsigned long long mag = k >= 0 ? (m << min(k, 63)) : (((m >> min(-k - 1, 62)) + 1ull) >> 1);
  return (b >> 63) ? -static_cast<long long>(mag) : static_cast<long long>(mag);
}
// floor(L v / 2^63) for a rule constant L = l 2^63 (0 <= l < 1).
__device__ __forceinline__ long long mul_q63(long long L, long long v) {
  const unsigned long long hi = static_cast<unsigned long long>(__mul64hi(L, v));
  const unsigned long long lo = static_cast<unsigned long long>(L) * static_cast<unsigned long long>(v);
  return static_cast<long long>((hi << 1) | (lo >> 63));
}
__host__ __device__ constexpr long long q63(double c) { return static_cast<long long>(c * 9223372036854775808.0); }

// The rule's points, coordinate c, in fixed point: the same symmetry-class
// form as quad_coord (a point of a class is B S + (A - B) v_q, S the vertex
// sum) with the same FP64 constants, scaled exactly by 2^63.
template <int NPTS>
__device__ __forceinline__ void quad_coord_fx(const double v[4], int s, long long xq[NPTS]) {
  long long t[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) t[a] = to_fx(v[a], s);
  const long long S = (t[0] + t[1]) + (t[2] + t[3]);
  if constexpr (NPTS == 1) {
    xq[0] = S >> 2;
  } else if constexpr (NPTS == 4) {
    const long long bS = mul_q63(q63(R4B), S);
#pragma unroll
    for (int q = 0; q < 4; ++q) xq[q] = mul_q63(q63(R4A - R4B), t[q]) + bS;
  } else {
    xq[0] = S >> 2;
    const long long bS = mul_q63(q63(K11B), S);
#pragma unroll
    for (int q = 0; q < 4; ++q) xq[1 + q] = mul_q63(q63(K11A - K11B), t[q]) + bS;
    const long long cS = mul_q63(q63(K11C2), S);
    long long P[4];  // (C1 - C2) v_a, summed per edge
#pragma unroll
    for (int a = 0; a < 4; ++a) P[a] = mul_q63(q63(K11C1 - K11C2), t[a]);
#pragma unroll
    for (int k = 0; k < 6; ++k) xq[5 + k] = P[edge_p(k)] + P[edge_q(k)] + cS;
  }
}

// floor(a b / 2^62) for |a|, |b| <= 2^62 (the 128-bit product shifted).
__device__ __forceinline__ long long mul_q62(long long a, long long b) {
  const unsigned long long hi = static_cast<unsigned long long>(__mul64hi(a, b));
  const unsigned long long lo = static_cast<unsigned long long>(a) * static_cast<unsigned long long>(b);
  return static_cast<long long>((hi << 2) | (lo >> 62));
}
// A constant in 62 fractional bits (|c| < 2).
__host__ __device__ constexpr long long q62(double c) { return static_cast<long long>(c * 4611686018427387904.0); }
// v 2^-59 as a double: one correctly rounded conversion, then an exact
// exponent shift (|v| >= 1 gives a normal result).
__device__ __forceinline__ double q59_to_double(long long v) {
  const double d = __ll2double_rn(v);
  return v == 0 ? 0.0 : __longlong_as_double(__double_as_longlong(d) - (59LL << 52));
}

// v 2^-62 as a double (one correctly rounded conversion, then an exact
// exponent shift; |v| >= 2^-960 2^62 gives a normal result).
__device__ __forceinline__ double q62_to_double(long long v) {
  const double d = __ll2double_rn(v);
  return v == 0 ? 0.0 : __longlong_as_double(__double_as_longlong(d) - (62LL << 52));
}

// One out-of-line copy of sinpi_fx for kernels with many sines: 33 inlined
// copies of its ~165 instructions overflow the instruction cache (ncu: the
// P2 load kernel stalled on instruction fetch), one copy called 33 times
// does not.
static __device__ __noinline__ double sinpi_fx_call(double x) { return sinpi_fx(x); }

// sin(pi v) in the precision of R; OUTLINE calls the out-of-line copy.
template <typename R, bool OUTLINE = false>
__device__ __forceinline__ R rsinpi(R v);
template <>
__device__ __forceinline__ double rsinpi<double, false>(double v) { return sinpi_fx(v); }
template <>
__device__ __forceinline__ double rsinpi<double, true>(double v) { return sinpi_fx_call(v); }
template <>
__device__ __forceinline__ float rsinpi<float, false>(float v) { return sinpif(v); }
template <>
__device__ __forceinline__ float rsinpi<float, true>(float v) { return sinpif(v); }

template <typename R>
__device__ __forceinline__ R to_r(double v);
template <>
__device__ __forceinline__ double to_r<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_r<float>(double v) { return __double2float_rn(v); }

template <typename R>
struct IsDouble {
  static constexpr bool value = false;
};
template <>
struct IsDouble<double> {
  static constexpr bool value = true;
};

__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
}
__device__ __forceinline__ float dot3(const float* a, const float* b) {
  return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}

// grad lambda_a in type R: FP64 path keeps the unscaled cofactors (the
// 1/det scale is folded into the per-element factor); the mixed path forms
// J^{-1} in FP64 and rounds it to FP32 once.
template <typename R>
__device__ __forceinline__ void grads(const Geo& g, R G[4][3]) {
  if constexpr (IsDouble<R>::value) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) G[a][k] = g.c[a][k];
  } else {
    const double inv = 1.0 / g.det;
#pragma unroll
    for (int a = 1; a < 4; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) G[a][k] = __double2float_rn(g.c[a][k] * inv);
#pragma unroll
    for (int k = 0; k < 3; ++k) G[0][k] = -(G[1][k] + G[2][k] + G[3][k]);
  }
}

// G_ij = s grad_i . grad_j (symmetric).  FP64: the products of rows 1..3 only;
// row 0 from the zero row sums (grad_0 = -(grad_1 + grad_2 + grad_3), so
// G_0j = -(G_1j + G_2j + G_3j)): two adds instead of a dot product and a
// scale, and grad_0 itself is never formed.  FP32: every product.
template <typename R>
__device__ __forceinline__ void gram(const R Gr[4][3], R s, R G[4][4]) {
  if constexpr (IsDouble<R>::value) {
#pragma unroll
    for (int i = 1; i < 4; ++i)
#pragma unroll
      for (int j = i; j < 4; ++j) {
        G[i][j] = s * dot3(Gr[i], Gr[j]);
        G[j][i] = G[i][j];
      }
#pragma unroll
    for (int j = 1; j < 4; ++j) {
      G[0][j] = -((G[1][j] + G[2][j]) + G[3][j]);
      G[j][0] = G[0][j];
    }
    G[0][0] = -((G[0][1] + G[0][2]) + G[0][3]);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = i; j < 4; ++j) {
        G[i][j] = s * dot3(Gr[i], Gr[j]);
        G[j][i] = G[i][j];
      }
  }
}

// 1 / y for y > 0, within one ulp, in three FP64 instructions: y = m 2^k
// with m in [1, 2) taken apart on the integer pipe, an FP32 seed r ~ 1/m
// (relative error e, |e| < 2^-22), then one third-order Newton step for the
// reciprocal, r (1 + e + e^2) with e = 1 - m r (the first terms of the series
// of 1 / (1 - e); the step leaves an error of order e^3 < 2^-66 besides its
// roundings), and 2^-k put back into the exponent field.  Zero, subnormal,
// huge (outside [2^-1000, 2^1000]) and non-finite y take the division.
__device__ __forceinline__ double rcp_pos(double y) {
  const long long b = __double_as_longlong(y);
  const int ex = (int)((b >> 52) & 0x7FF);  // biased exponent; b < 0: negative y
  if (b < 0 || ex < 1023 - 1000 || ex > 1023 + 1000) return 1.0 / y;
  const double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
  const float rf = __frcp_rn(__int_as_float(0x3F800000 | (int)((b >> 29) & 0x7FFFFF)));  // m to 24 bits
  const unsigned u = __float_as_uint(rf);  // rf in [0.5, 1]: a normal float, widened by its bits
  double r = __longlong_as_double(((long long)(((u >> 23) & 0xFF) - 127 + 1023) << 52) |
                                  ((long long)(u & 0x7FFFFF) << 29));
  const double e = fma(-m, r, 1.0);
  r = fma(r, fma(e, e, e), r);
  return __longlong_as_double(__double_as_longlong(r) - ((long long)(ex - 1023) << 52));
}

// Scale that turns products of grads<R> into |T| grad . grad:
// FP64: |T| / det^2 = 1 / (6 |det|); mixed: |T| = |det| / 6.
template <typename R>
__device__ __forceinline__ double grad_scale(double adet) {
  if constexpr (IsDouble<R>::value) return rcp_pos(6.0 * adet);
  else return adet * (1.0 / 6.0);
}

template <typename R>
__device__ __forceinline__ void vertices_r(const double X[4][3], R Xr[4][3]) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) Xr[a][k] = to_r<R>(X[a][k]);
}

// Quadrature points of rule NPTS for one coordinate, from the vertex values
// v[0..3]: x_q = sum_v bary(q, v) v[v], grouped by symmetry class.
template <int NPTS, typename R>
__device__ __forceinline__ void quad_coord(const R v[4], R xq[NPTS]) {
  const R S = (v[0] + v[1]) + (v[2] + v[3]);
  if constexpr (NPTS == 1) {
    xq[0] = R(0.25) * S;
  } else if constexpr (NPTS == 4) {
    const R bS = R(R4B) * S;
#pragma unroll
    for (int q = 0; q < 4; ++q) xq[q] = fma(R(R4A - R4B), v[q], bS);
  } else {
    xq[0] = R(0.25) * S;
    const R bS = R(K11B) * S;
#pragma unroll
    for (int q = 0; q < 4; ++q) xq[1 + q] = fma(R(K11A - K11B), v[q], bS);
    const R cS = R(K11C2) * S;
#pragma unroll
    for (int k = 0; k < 6; ++k) xq[5 + k] = fma(R(K11C1 - K11C2), v[edge_p(k)] + v[edge_q(k)], cS);
  }
}

// Compile-time loop: f(Idx<I>{}) for I = 0..N-1, in ascending order.  Idx<I>
// converts to the constant I, so the body can use it as a template argument.
template <int I>
struct Idx {
  static constexpr int value = I;
  __host__ __device__ constexpr operator int() const { return I; }
};
template <int I, int N>
struct StaticFor {
  template <typename F>
  __device__ __forceinline__ static void run(F& f) {
    f(Idx<I>{});
    StaticFor<I + 1, N>::run(f);
  }
};
template <int N>
struct StaticFor<N, N> {
  template <typename F>
  __device__ __forceinline__ static void run(F&) {}
};
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  StaticFor<0, N>::run(f);
}

// ------------------------------------------------------------------ rule sums
// wphi(q, a) = w_q phi_a(x_q) for the rule NPTS.
template <int ORDER, int NPTS>
__host__ __device__ constexpr double wphi(int q, int a) {
  return weight(NPTS, q) * phi_at(ORDER, NPTS, q, a);
}

// The rules are symmetric, so w_q phi_a(x_q) takes few values.  Classes of
// (point, basis function), with vertex-class point q = 1 + v and edge-class
// point q = 5 + k (11 points) or point q = v (4 points):
//   vertex function a:  centroid | own vertex point | other vertex point |
//                       edge point on a | edge point off a
//   edge function (i,j): centroid | vertex point on the edge | off it |
//                       the same edge | an edge sharing one vertex | the
//                       opposite edge (k <-> 5 - k)
// rule_classes_ok checks every (q, a) against its class representative.
__host__ __device__ constexpr bool on_edge(int k, int v) { return edge_p(k) == v || edge_q(k) == v; }
template <int ORDER, int NPTS>
__host__ __device__ constexpr bool rule_classes_ok() {
  constexpr int NB = ORDER == 1 ? 4 : 10;
  for (int a = 0; a < NB; ++a)
    for (int q = 0; q < NPTS; ++q) {
      double rep = 0.0;
      if (NPTS == 1) continue;
      const bool vpt = NPTS == 4 || (q >= 1 && q <= 4);
      const int v = NPTS == 4 ? q : q - 1;  // vertex of a vertex-class point
      const int k = q - 5;                 // edge of an edge-class point
      if (a < 4) {
        if (NPTS == 11 && q == 0) rep = wphi<ORDER, NPTS>(0, 0);
        else if (vpt) rep = v == a ? wphi<ORDER, NPTS>(NPTS == 4 ? 0 : 1, 0) : wphi<ORDER, NPTS>(NPTS == 4 ? 1 : 2, 0);
        else rep = on_edge(k, a) ? wphi<ORDER, NPTS>(5, 0) : wphi<ORDER, NPTS>(10, 0);
      } else {
        const int e = a - 4;
        if (NPTS == 11 && q == 0) rep = wphi<ORDER, NPTS>(0, 4);
        else if (vpt) rep = on_edge(e, v) ? wphi<ORDER, NPTS>(NPTS == 4 ? 0 : 1, 4) : wphi<ORDER, NPTS>(NPTS == 4 ? 2 : 3, 4);
        else if (k == e) rep = wphi<ORDER, NPTS>(5, 4);
        else if (k == 5 - e) rep = wphi<ORDER, NPTS>(10, 4);
        else rep = wphi<ORDER, NPTS>(6, 4);
      }
      if (rep != wphi<ORDER, NPTS>(q, a)) return false;
    }
  return true;
}

// Fs_a = sum_q w_q phi_a(x_q) s_q for point values s, summed by classes:
// the class sums S (vertex-class points), S6 (edge-class points) and E_a
// (edge points on vertex a) are shared, so each Fs_a costs two or three FMAs
// instead of one per point.
template <int ORDER, int NPTS, typename R>
__device__ __forceinline__ void rule_sum(const R s[NPTS], R Fs[ORDER == 1 ? 4 : 10]) {
  static_assert(rule_classes_ok<ORDER, NPTS>(), "quadrature rule lost its symmetry classes");
  using W = double;
  if constexpr (NPTS == 1) {
    Fs[0] = R(wphi<ORDER, 1>(0, 0)) * s[0];
#pragma unroll
    for (int a = 1; a < 4; ++a) Fs[a] = Fs[0];
    if constexpr (ORDER == 2) {
      Fs[4] = R(wphi<ORDER, 1>(0, 4)) * s[0];
#pragma unroll
      for (int a = 5; a < 10; ++a) Fs[a] = Fs[4];
    }
  } else if constexpr (NPTS == 4) {
    const R S = (s[0] + s[1]) + (s[2] + s[3]);
    constexpr W vs = wphi<ORDER, 4>(0, 0), vo = wphi<ORDER, 4>(1, 0);
    const R Cv = R(vo) * S;
#pragma unroll
    for (int a = 0; a < 4; ++a) Fs[a] = fma(R(vs - vo), s[a], Cv);
    if constexpr (ORDER == 2) {
      constexpr W ei = wphi<ORDER, 4>(0, 4), eo = wphi<ORDER, 4>(2, 4);
      const R Ce = R(eo) * S;
#pragma unroll
      for (int k = 0; k < 6; ++k) Fs[4 + k] = fma(R(ei - eo), s[edge_p(k)] + s[edge_q(k)], Ce);
    }
  } else {
    const R S4 = (s[1] + s[2]) + (s[3] + s[4]);
    const R S6 = ((s[5] + s[6]) + (s[7] + s[8])) + (s[9] + s[10]);
    R E[4];  // edge points on vertex a: edges (a, .) among (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)
    E[0] = (s[5] + s[6]) + s[7];
    E[1] = (s[5] + s[8]) + s[9];
    E[2] = (s[6] + s[8]) + s[10];
    E[3] = (s[7] + s[9]) + s[10];
    constexpr W c0 = wphi<ORDER, 11>(0, 0), vs = wphi<ORDER, 11>(1, 0), vo = wphi<ORDER, 11>(2, 0);
    constexpr W ei = wphi<ORDER, 11>(5, 0), eo = wphi<ORDER, 11>(10, 0);
    const R Cv = fma(R(c0), s[0], fma(R(vo), S4, R(eo) * S6));
#pragma unroll
    for (int a = 0; a < 4; ++a) Fs[a] = fma(R(vs - vo), s[1 + a], fma(R(ei - eo), E[a], Cv));
    if constexpr (ORDER == 2) {
      constexpr W g0 = wphi<ORDER, 11>(0, 4), gi = wphi<ORDER, 11>(1, 4), go = wphi<ORDER, 11>(3, 4);
      constexpr W ds = wphi<ORDER, 11>(5, 4), dh = wphi<ORDER, 11>(6, 4), dp = wphi<ORDER, 11>(10, 4);
      const R Ce = fma(R(g0), s[0], fma(R(go), S4, R(dh) * S6));
#pragma unroll
      for (int k = 0; k < 6; ++k)
        Fs[4 + k] = fma(R(gi - go), s[1 + edge_p(k)] + s[1 + edge_q(k)],
                        fma(R(ds - dh), s[5 + k], fma(R(dp - dh), s[10 - k], Ce)));
    }
  }
}

// rule_sum on the integer pipes: the point values S_q carry 62 fractional
// bits; they are shifted to 59 (so class sums of up to six stay in range),
// multiplied by the class coefficients in 62 fractional bits, and the sums
// F_a carry 59 fractional bits.  Same classes and operations as rule_sum.
template <int ORDER, int NPTS>
__device__ __forceinline__ void rule_sum_q(const long long Sq[NPTS], long long F[ORDER == 1 ? 4 : 10]) {
  static_assert(rule_classes_ok<ORDER, NPTS>(), "quadrature rule lost its symmetry classes");
  long long s[NPTS];
#pragma unroll
  for (int q = 0; q < NPTS; ++q) s[q] = Sq[q] >> 3;
  if constexpr (NPTS == 1) {
    constexpr long long cv = q62(wphi<ORDER, 1>(0, 0));
    F[0] = mul_q62(cv, s[0]);
#pragma unroll
    for (int a = 1; a < 4; ++a) F[a] = F[0];
    if constexpr (ORDER == 2) {
      constexpr long long ce = q62(wphi<ORDER, 1>(0, 4));
      F[4] = mul_q62(ce, s[0]);
#pragma unroll
      for (int a = 5; a < 10; ++a) F[a] = F[4];
    }
  } else if constexpr (NPTS == 4) {
    const long long S = (s[0] + s[1]) + (s[2] + s[3]);
    constexpr long long vo = q62(wphi<ORDER, 4>(1, 0)), dv = q62(wphi<ORDER, 4>(0, 0) - wphi<ORDER, 4>(1, 0));
    const long long Cv = mul_q62(vo, S);
#pragma unroll
    for (int a = 0; a < 4; ++a) F[a] = Cv + mul_q62(dv, s[a]);
    if constexpr (ORDER == 2) {
      constexpr long long eo = q62(wphi<ORDER, 4>(2, 4)), de = q62(wphi<ORDER, 4>(0, 4) - wphi<ORDER, 4>(2, 4));
      const long long Ce = mul_q62(eo, S);
#pragma unroll
      for (int k = 0; k < 6; ++k) F[4 + k] = Ce + mul_q62(de, s[edge_p(k)] + s[edge_q(k)]);
    }
  } else {
    const long long S4 = (s[1] + s[2]) + (s[3] + s[4]);
    const long long S6 = ((s[5] + s[6]) + (s[7] + s[8])) + (s[9] + s[10]);
    long long E[4];
    E[0] = (s[5] + s[6]) + s[7];
    E[1] = (s[5] + s[8]) + s[9];
    E[2] = (s[6] + s[8]) + s[10];
    E[3] = (s[7] + s[9]) + s[10];
    constexpr long long c0 = q62(wphi<ORDER, 11>(0, 0)), vo = q62(wphi<ORDER, 11>(2, 0)),
                        eo = q62(wphi<ORDER, 11>(10, 0));
    constexpr long long dv = q62(wphi<ORDER, 11>(1, 0) - wphi<ORDER, 11>(2, 0)),
                        de = q62(wphi<ORDER, 11>(5, 0) - wphi<ORDER, 11>(10, 0));
    const long long Cv = mul_q62(c0, s[0]) + mul_q62(vo, S4) + mul_q62(eo, S6);
#pragma unroll
    for (int a = 0; a < 4; ++a) F[a] = Cv + mul_q62(dv, s[1 + a]) + mul_q62(de, E[a]);
    if constexpr (ORDER == 2) {
      constexpr long long g0 = q62(wphi<ORDER, 11>(0, 4)), go = q62(wphi<ORDER, 11>(3, 4)),
                          dh = q62(wphi<ORDER, 11>(6, 4));
      constexpr long long dg = q62(wphi<ORDER, 11>(1, 4) - wphi<ORDER, 11>(3, 4)),
                          dsm = q62(wphi<ORDER, 11>(5, 4) - wphi<ORDER, 11>(6, 4)),
                          dp = q62(wphi<ORDER, 11>(10, 4) - wphi<ORDER, 11>(6, 4));
      const long long Ce = mul_q62(g0, s[0]) + mul_q62(go, S4) + mul_q62(dh, S6);
#pragma unroll
      for (int k = 0; k < 6; ++k)
        F[4 + k] = Ce + mul_q62(dg, s[1 + edge_p(k)] + s[1 + edge_q(k)]) + mul_q62(dsm, s[5 + k]) +
                   mul_q62(dp, s[10 - k]);
    }
  }
}

// Shape load  Fs_a = sum_q w_q s(x_q) phi_a(x_q)  (without the factor |T|),
// s = 1 (LOAD_CONST) or sin(pi x) sin(pi y) sin(pi z) (LOAD_SIN).
template <int ORDER, int NPTS, int LOAD, typename R, bool OUTLINE = (ORDER == 2)>
__device__ __forceinline__ void shape_load(const R Xr[4][3], R Fs[ORDER == 1 ? 4 : 10]) {
  constexpr int NB = ORDER == 1 ? 4 : 10;
  if constexpr (LOAD == LOAD_CONST) {
    static_for<NB>([&](auto A) {
      constexpr double c = wphi_sum(ORDER, NPTS, A);
      Fs[A] = R(c);
    });
  } else if constexpr (IsDouble<R>::value) {
    // FP64: the points' coordinates, the sines, their products and the rule
    // sums in fixed point on the integer pipes; one conversion per output
    long long sq[NPTS];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double v[4] = {Xr[0][c], Xr[1][c], Xr[2][c], Xr[3][c]};
      const int s = fx_shift(v);
      long long xq[NPTS];
      quad_coord_fx<NPTS>(v, s, xq);
#pragma unroll
      for (int q0 = 0; q0 < NPTS; q0 += 4) {
        Q4 in;
#pragma unroll
        for (int k = 0; k < 4; ++k) in.v[k] = q0 + k < NPTS ? xq[q0 + k] : 0;
        const Q4 o = sinpi_q62_fx4_sel<OUTLINE>(in, s);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (q0 + k < NPTS) sq[q0 + k] = c == 0 ? o.v[k] : mul_q62(sq[q0 + k], o.v[k]);
      }
    }
    long long F[NB];
    rule_sum_q<ORDER, NPTS>(sq, F);
#pragma unroll
    for (int a = 0; a < NB; ++a) Fs[a] = q59_to_double(F[a]);
  } else {
    R sq[NPTS];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R v[4] = {Xr[0][c], Xr[1][c], Xr[2][c], Xr[3][c]};
      R xq[NPTS];
      quad_coord<NPTS, R>(v, xq);
#pragma unroll
      for (int q = 0; q < NPTS; ++q) sq[q] = c == 0 ? rsinpi<R, OUTLINE>(xq[q]) : sq[q] * rsinpi<R, OUTLINE>(xq[q]);
    }
    rule_sum<ORDER, NPTS, R>(sq, Fs);
  }
}

// ------------------------------------------------------------------ P2 stiffness entries
// K_ab (upper pair number K) = [c +] sum_t num_t * G[i_t][j_t] (G already
// scaled); c, when given, starts the FMA chain (the entry's mass term).
template <int K, typename R>
__device__ __forceinline__ R p2_stiff(const R G[4][4]) {
  constexpr int A = upper_a(10, K), B = upper_b(10, K);
  constexpr Terms t = p2_terms(A, B);
  R v = R(t.num[0]) * G[t.i[0]][t.j[0]];
  if constexpr (t.n > 1) v = fma(R(t.num[1]), G[t.i[1]][t.j[1]], v);
  if constexpr (t.n > 2) v = fma(R(t.num[2]), G[t.i[2]][t.j[2]], v);
  if constexpr (t.n > 3) v = fma(R(t.num[3]), G[t.i[3]][t.j[3]], v);
  return v;
}
template <int K, typename R>
__device__ __forceinline__ R p2_stiff(const R G[4][4], R c) {
  constexpr int A = upper_a(10, K), B = upper_b(10, K);
  constexpr Terms t = p2_terms(A, B);
  R v = fma(R(t.num[0]), G[t.i[0]][t.j[0]], c);
  if constexpr (t.n > 1) v = fma(R(t.num[1]), G[t.i[1]][t.j[1]], v);
  if constexpr (t.n > 2) v = fma(R(t.num[2]), G[t.i[2]][t.j[2]], v);
  if constexpr (t.n > 3) v = fma(R(t.num[3]), G[t.i[3]][t.j[3]], v);
  return v;
}

// ------------------------------------------------------------------ P2 entries in fixed point
// The FP64 P2 local matrix as exact integer sums.  Every stiffness coefficient
// num_t is a multiple of 4 with sum_t |num_t| / 4 <= 24 in any entry, and
// every mass value is at most 32 in magnitude (p2_fx_coeffs_ok).  With E the
// largest biased exponent of 4 G_ij and of 32 t (t = the mass scale), both
// lie below 2^(E - 1022); 4 G_ij and t are rounded to integers at the scale
// 2^p, p = 1078 - E, so every input is below 2^56 and every entry below
// 25 * 2^56 < 2^61.  The sums are then exact and each entry is rounded once,
// on the way back to FP64: its error is at most 28 * 2^-55 of the largest
// input (the rounded inputs, 28 units of 2^-p) plus half an ulp of the entry
// (tests/test_p2_fixed_point_model.py checks a bit-exact host model of this
// arithmetic against exact sums across the exponent range).  For E outside
// [P2FX_EMIN, P2FX_EMAX] (non-finite or vanishing inputs) the kernels keep
// the FP64 chains; inside it the results stay normal FP64 numbers.
constexpr int P2FX_EMIN = 64, P2FX_EMAX = 2032;

__host__ __device__ constexpr bool p2_fx_coeffs_ok() {
  for (int K = 0; K < 55; ++K) {
    const Terms t = p2_terms(upper_a(10, K), upper_b(10, K));
    int sum = 0;
    for (int k = 0; k < t.n; ++k) {
      if (t.num[k] % 4 != 0) return false;
      sum += t.num[k] < 0 ? -t.num[k] / 4 : t.num[k] / 4;
    }
    if (sum > 24) return false;
    const int m = p2_mass420(upper_a(10, K), upper_b(10, K));
    if (m > 32 || m < -32) return false;
  }
  return true;
}

static_assert(p2_fx_coeffs_ok(), "P2 coefficients outside the fixed-point bounds");

__device__ __forceinline__ int exp_bits(double v) { return (__double2hiint(v) >> 20) & 0x7FF; }

// Entry K at scale 2^p: m (its mass term) + sum_t (num_t / 4) Gf[i_t][j_t],
// Gf = 4 G at scale 2^p.
template <int K>
__device__ __forceinline__ long long p2_stiff_fx(const long long Gf[4][4], long long m) {
  constexpr int A = upper_a(10, K), B = upper_b(10, K);
  constexpr Terms t = p2_terms(A, B);
  long long v = m + static_cast<long long>(t.num[0] / 4) * Gf[t.i[0]][t.j[0]];
  if constexpr (t.n > 1) v += static_cast<long long>(t.num[1] / 4) * Gf[t.i[1]][t.j[1]];
  if constexpr (t.n > 2) v += static_cast<long long>(t.num[2] / 4) * Gf[t.i[2]][t.j[2]];
  if constexpr (t.n > 3) v += static_cast<long long>(t.num[3] / 4) * Gf[t.i[3]][t.j[3]];
  return v;
}

// F 2^-p as a double: one correctly rounded conversion, then an exact shift
// of the exponent field (the caller keeps the result normal).
__device__ __forceinline__ double fx_to_double(long long F, int p) {
  const double d = __ll2double_rn(F);
  return F == 0 ? 0.0 : __longlong_as_double(__double_as_longlong(d) - (static_cast<long long>(p) << 52));
}

// The P2 mass pattern 420 |T|^{-1} M_ab takes seven values; mass_class(a, b)
// numbers them, so the element kernels form t * value once per class and
// start each entry's stiffness FMA chain from it.
__host__ __device__ constexpr int p2_mass_value(int c) {
  return c == 0 ? 6 : c == 1 ? 1 : c == 2 ? -4 : c == 3 ? -6 : c == 4 ? 32 : c == 5 ? 16 : 8;
}
__host__ __device__ constexpr int p2_mass_class(int a, int b) {
  const int v = p2_mass420(a, b);
  return v == 6 ? 0 : v == 1 ? 1 : v == -4 ? 2 : v == -6 ? 3 : v == 32 ? 4 : v == 16 ? 5 : 6;
}

}  // namespace fea

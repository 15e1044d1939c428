// Deterministic scatter of local matrices and loads into CSR values and rhs.
//
// Algorithm 1 (Sec. 5) adds every local value into the global matrix with a
// global atomicAdd (after a column search in the sparse variant), so the
// order of the floating-point additions - and the result - changes from run
// to run.  Here the scatter is a segmented reduction keyed by row, the
// row-sorted form of a sorted-COO reduction:
//   * one CTA owns a tile of consecutive CSR rows, whose values form one
//     contiguous span of `values`; the span is accumulated in shared memory;
//   * one thread owns one row; the element kernel has already written the
//     row's contributions (local row a of every element holding the row's
//     dof, ascending element order) contiguously, so the thread streams them
//     with addresses that depend on nothing it loads, two at a time, and adds
//     each at its precomputed slots;
//   * the finished span is written to HBM with coalesced stores.
// Every value is therefore the sum of its contributions in element order,
// computed by one thread: bitwise reproducible, and bitwise symmetric because
// the local matrices are.  No atomics, no colouring, no second pass.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"
#include "vecmem.cuh"

namespace fea {

// Exact float -> double conversion with integer operations only (the FP64
// pipe is the scarce one on this part, and a hardware conversion kept as a
// fallback branch is if-converted by the compiler into an unconditional one):
// the IEEE-754 binary32 fields move into binary64 position; the exponent of a
// normal number is re-biased by 1023 - 127 = 896, infinities and NaNs
// (payload kept) get 2047, a subnormal is normalised from the position p of
// its top mantissa bit (value m 2^-149 = 1.f 2^(p - 149)), and +-0 keeps only
// its sign.  Bitwise equal to the hardware conversion for every input.
__device__ __forceinline__ double widen_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t sgn = u & 0x80000000u, ex = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  uint32_t hi, lo;
  if (ex - 1u < 0xFEu) {  // normal
    hi = sgn | ((ex + 896u) << 20) | (m >> 3);
    lo = m << 29;
  } else if (ex == 0xFFu) {  // infinity, NaN
    hi = sgn | (2047u << 20) | (m >> 3);
    lo = m << 29;
  } else {  // zero, subnormal
    const uint32_t p = 31u - static_cast<uint32_t>(__clz(static_cast<int>(m | 1u)));
    const unsigned long long f = (static_cast<unsigned long long>(m) << (52u - p)) & 0xFFFFFFFFFFFFFull;
    hi = m ? (sgn | ((p + 874u) << 20) | static_cast<uint32_t>(f >> 32)) : sgn;
    lo = m ? static_cast<uint32_t>(f) : 0u;
  }
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}
// Normal numbers and zeros only: the sign, exponent and top mantissa bits
// shifted into place with the exponent re-biased by one add (896 << 20), the
// low mantissa bits into the low word; +-0 keeps only its sign.
__device__ __forceinline__ double widen_fast(uint32_t u) {
  const uint32_t mag = u & 0x7FFFFFFFu;
  const uint32_t hi = mag ? (((mag >> 3) + 0x38000000u) | (u & 0x80000000u)) : u;
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(u << 29));
}
// Subnormal, infinite or NaN (exponent field 0 with a nonzero mantissa, or 255).
__device__ __forceinline__ bool widen_special(uint32_t u) {
  return (((u + 0x00800000u) & 0x7F800000u) <= 0x00800000u) && (u & 0x7FFFFFFFu) != 0u;
}
template <int NL>
struct FRow {
  float v[NL];
};
template <int NL>
struct DRow {
  double v[NL];
};
// Out of line, so that the rare exact path is a real branch (by value: the
// row stays in registers).
template <int NL>
static __device__ __noinline__ DRow<NL> widen_row_exact(FRow<NL> r) {
  DRow<NL> o;
#pragma unroll
  for (int k = 0; k < NL; ++k) o.v[k] = widen_bits(r.v[k]);
  return o;
}
template <int NL>
__device__ __forceinline__ void widen_row(const float* v, double* out) {
  bool special = false;
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    const uint32_t u = __float_as_uint(v[k]);
    out[k] = widen_fast(u);
    special |= widen_special(u);
  }
  if (special) {
    FRow<NL> r;
#pragma unroll
    for (int k = 0; k < NL; ++k) r.v[k] = v[k];
    const DRow<NL> o = widen_row_exact<NL>(r);
#pragma unroll
    for (int k = 0; k < NL; ++k) out[k] = o.v[k];
  }
}
template <int NL>
__device__ __forceinline__ void widen_row(const double* v, double* out) {
#pragma unroll
  for (int k = 0; k < NL; ++k) out[k] = v[k];
}
__device__ __forceinline__ double widen(double d) { return d; }
__device__ __forceinline__ double widen(float f) {
  double o;
  widen_row<1>(&f, &o);
  return o;
}

// Add one local row (NL values, distinct target slots) into the row's
// shared-memory span: all slots are read, then added, then written, so the
// loads of one incidence do not wait on each other's stores.
template <int NB, int NDPN, typename LT>
__device__ __forceinline__ void add_row(double* __restrict__ a, const int s[NB], const LT* v) {
  constexpr int NL = NB * NDPN;
  double w[NL], t[NL];
  widen_row<NL>(v, w);
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int j = 0; j < NDPN; ++j) t[NDPN * b + j] = a[NDPN * s[b] + j];
#pragma unroll
  for (int k = 0; k < NL; ++k) t[k] += w[k];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int j = 0; j < NDPN; ++j) a[NDPN * s[b] + j] = t[NDPN * b + j];
}

// The NB slots of a local row, added at offset `off` of a CSR span of `span`
// values, stay inside it (checked build; always true otherwise).
template <int NB, int NDPN>
__device__ __forceinline__ bool slots_ok(int off, const int s[NB], int span, int* err) {
  bool ok = true;
#pragma unroll
  for (int b = 0; b < NB; ++b) ok = ok && index_ok(off + NDPN * s[b] + NDPN - 1, span, err) && index_ok(s[b], span, err);
  return ok;
}

// Load the NL values of one local row (32-byte aligned, whole sectors).
template <int NL>
__device__ __forceinline__ void load_row(const double* __restrict__ p, double v[NL]) {
  constexpr int LS = lstride(NL, 8);
#pragma unroll
  for (int k = 0; k < LS / 4; ++k) {
    double t[4];
    ld_v4(p + 4 * k, t[0], t[1], t[2], t[3]);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (4 * k + j < NL) v[4 * k + j] = t[j];
  }
}
template <int NL>
__device__ __forceinline__ void load_row(const float* __restrict__ p, float v[NL]) {
  constexpr int LS = lstride(NL, 4);
#pragma unroll
  for (int k = 0; k < LS / 8; ++k) {
    float t[8];
    ld_v8(p + 8 * k, t[0], t[1], t[2], t[3], t[4], t[5], t[6], t[7]);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (8 * k + j < NL) v[8 * k + j] = t[j];
  }
}

// Slots of the NB local columns of one incidence (1 byte each).
template <int NB>
__device__ __forceinline__ void load_slots(const uint8_t* __restrict__ slot, int64_t i, int s[NB]) {
  if constexpr (NB <= 4) {
    const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(slot) + i);
#pragma unroll
    for (int b = 0; b < NB; ++b) s[b] = (w >> (8 * b)) & 0xFF;
  } else {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(slot) + i);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int b = 0; b < NB; ++b) s[b] = (ws[b >> 2] >> (8 * (b & 3))) & 0xFF;
  }
}

struct GatherArgs {
  int64_t ndof;
  const int32_t* row_ptr;  // dof-level CSR
  const int32_t* inc_ptr;  // scalar dof -> incidences
  const uint8_t* slot;     // [incidence][SW] column slots
  const void* Lm;          // local rows in incidence order (lstride apart)
  const void* Fl;          // local loads in incidence order, or NULL
  double* values;
  double* rhs;             // or NULL
  int* err;                // device error word (bounds checks of the checked build)
};

// Loads of one incidence: the column slots, the local row, the local load.
template <int NB, int NDPN, typename LT>
struct Contrib {
  static constexpr int NL = NB * NDPN;
  int s[NB];
  LT v[NL];
  LT f;
  __device__ __forceinline__ void load(const GatherArgs& G, int32_t i, int comp) {
    constexpr int LS = lstride(NL, sizeof(LT));
    load_slots<NB>(G.slot, i, s);
    load_row<NL>(static_cast<const LT*>(G.Lm) + ((int64_t)i * NDPN + comp) * LS, v);
    f = G.Fl ? __ldg(static_cast<const LT*>(G.Fl) + (int64_t)i * NDPN + comp) : LT(0);
  }
};

// NB local scalar dofs, NDPN dofs per scalar dof, LT local-value type.
// Incidences are consumed in pairs; the loads of the next pair are issued
// before the current pair is added (software pipeline), so one pair's memory
// latency overlaps the other pair's shared-memory adds.
template <int NB, int NDPN, typename LT, bool DEEP = true>
__device__ __forceinline__ void gather_tile(const GatherArgs& G, int64_t tile, int rows, double* acc) {
  const int64_t r0 = tile * rows;
  const int64_t r1 = r0 + rows < G.ndof ? r0 + rows : G.ndof;
  const int32_t base = __ldg(G.row_ptr + r0);
  const int32_t span = __ldg(G.row_ptr + r1) - base;
  for (int k = threadIdx.x; k < span; k += blockDim.x) acc[k] = 0.0;
  __syncthreads();
  const int64_t r = r0 + threadIdx.x;
  if (threadIdx.x < rows && r < r1) {
    const int64_t node = r / NDPN;
    const int comp = (int)(r - node * NDPN);
    const int off = __ldg(G.row_ptr + r) - base;
    double* __restrict__ a = acc + off;
    double f = 0.0;
    const int32_t i1 = __ldg(G.inc_ptr + node + 1);
    int32_t i = __ldg(G.inc_ptr + node);
    if constexpr (DEEP) {
      Contrib<NB, NDPN, LT> c0, c1, n0, n1;
      if (i < i1) c0.load(G, i, comp);
      if (i + 1 < i1) c1.load(G, i + 1, comp);
      while (i < i1) {
        if (i + 2 < i1) n0.load(G, i + 2, comp);
        if (i + 3 < i1) n1.load(G, i + 3, comp);
        if (slots_ok<NB, NDPN>(off, c0.s, span, G.err)) add_row<NB, NDPN, LT>(a, c0.s, c0.v);
        f += widen(c0.f);
        if (i + 1 < i1) {
          if (slots_ok<NB, NDPN>(off, c1.s, span, G.err)) add_row<NB, NDPN, LT>(a, c1.s, c1.v);
          f += widen(c1.f);
        }
        c0 = n0;
        c1 = n1;
        i += 2;
      }
    } else {
      // one incidence in flight ahead of the one being added (fewer registers)
      Contrib<NB, NDPN, LT> c0, n0;
      if (i < i1) c0.load(G, i, comp);
      while (i < i1) {
        if (i + 1 < i1) n0.load(G, i + 1, comp);
        if (slots_ok<NB, NDPN>(off, c0.s, span, G.err)) add_row<NB, NDPN, LT>(a, c0.s, c0.v);
        f += widen(c0.f);
        c0 = n0;
        ++i;
      }
    }
    if (G.rhs) G.rhs[r] = f;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < span; k += blockDim.x) G.values[base + k] = acc[k];
}

template <int NB, int NDPN, typename LT>
__global__ void __launch_bounds__(128) k_gather(GatherArgs G) {
  extern __shared__ double acc[];
  gather_tile<NB, NDPN, LT>(G, blockIdx.x, blockDim.x, acc);
}

// The row tiles listed in tiles[0 .. gridDim.x).
template <int NB, int NDPN, typename LT, bool DEEP = true>
__global__ void __launch_bounds__(128) k_gather_list(GatherArgs G, const int32_t* __restrict__ tiles) {
  extern __shared__ double acc[];
  gather_tile<NB, NDPN, LT, DEEP>(G, __ldg(tiles + blockIdx.x), blockDim.x, acc);
}

fea_status launch_gather(int nb, int ndpn, bool mixed, const GatherArgs& G, int rows_per_tile,
                         int64_t max_tile_nnz, cudaStream_t s, const int32_t* tiles = nullptr,
                         int64_t ntiles = -1, bool deep = true);

}  // namespace fea

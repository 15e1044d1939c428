// Deterministic scatter of local matrices and loads into CSR values and rhs.
//
// Algorithm 1 (Sec. 5) adds every local value into the global matrix with a
// global atomicAdd (after a column search in the sparse variant), so the
// order of the floating-point additions - and the result - changes from run
// to run.  Here the scatter is a segmented reduction keyed by row, the
// row-sorted form of a sorted-COO reduction:
//   * one CTA owns a tile of consecutive CSR rows, whose values form one
//     contiguous span of `values`; the span is accumulated in shared memory;
//   * one thread owns one row and walks the row's incidence list (element,
//     local row a) in ascending element order, adding local row a of each
//     element at the precomputed slots of the row;
//   * the finished span is written to HBM with coalesced stores.
// Every value is therefore the sum of its contributions in element order,
// computed by one thread: bitwise reproducible, and bitwise symmetric because
// the local matrices are.  No atomics, no colouring, no second pass.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace fea {

// Exact float -> double conversion with integer operations (keeps the
// conversion off the FP64 pipe): the IEEE-754 binary32 fields are moved into
// binary64 position with the exponent re-biased by 1023 - 127 = 896.  Zeros,
// subnormals, infinities and NaNs take the hardware conversion.
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xFFu;
  if (ex - 1u < 0xFEu) {
    const uint32_t hi = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    const uint32_t lo = u << 29;
    return __hiloint2double((int)hi, (int)lo);
  }
  return (double)f;
}
__device__ __forceinline__ double widen(double d) { return d; }

// Load NL consecutive values starting at p with the widest aligned vectors.
template <int NL>
__device__ __forceinline__ void load_row(const double* __restrict__ p, double v[NL]) {
  static_assert(NL % 2 == 0, "even row length");
#pragma unroll
  for (int k = 0; k < NL / 2; ++k) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(p) + k);
    v[2 * k] = t.x;
    v[2 * k + 1] = t.y;
  }
}
template <int NL>
__device__ __forceinline__ void load_row(const float* __restrict__ p, float v[NL]) {
  if constexpr (NL % 4 == 0) {
#pragma unroll
    for (int k = 0; k < NL / 4; ++k) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p) + k);
      v[4 * k] = t.x;
      v[4 * k + 1] = t.y;
      v[4 * k + 2] = t.z;
      v[4 * k + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < NL / 2; ++k) {
      const float2 t = __ldg(reinterpret_cast<const float2*>(p) + k);
      v[2 * k] = t.x;
      v[2 * k + 1] = t.y;
    }
  }
}

// Slots of the NB local columns of one incidence (1 byte each).
template <int NB>
__device__ __forceinline__ void load_slots(const uint8_t* __restrict__ slot, int64_t i, int s[NB]) {
  if constexpr (NB == 4) {
    const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(slot) + i);
#pragma unroll
    for (int b = 0; b < 4; ++b) s[b] = (w >> (8 * b)) & 0xFF;
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
  const int32_t* inc;
  const uint8_t* slot;
  const void* Lm;          // [E][NL][NL]
  const void* Fl;          // [E][NL] or NULL
  double* values;
  double* rhs;             // or NULL
};

// NB local scalar dofs, NDPN dofs per scalar dof, LT local-value type.
template <int NB, int NDPN, typename LT>
__global__ void __launch_bounds__(128) k_gather(GatherArgs G) {
  extern __shared__ double acc[];
  constexpr int NL = NB * NDPN;
  const int rows = blockDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rows;
  const int64_t r1 = r0 + rows < G.ndof ? r0 + rows : G.ndof;
  const int32_t base = __ldg(G.row_ptr + r0);
  const int32_t span = __ldg(G.row_ptr + r1) - base;
  for (int k = threadIdx.x; k < span; k += rows) acc[k] = 0.0;
  __syncthreads();
  const int64_t r = r0 + threadIdx.x;
  if (r < r1) {
    const int64_t node = r / NDPN;
    const int comp = (int)(r - node * NDPN);
    double* __restrict__ a = acc + (__ldg(G.row_ptr + r) - base);
    const LT* __restrict__ Lm = static_cast<const LT*>(G.Lm);
    const LT* __restrict__ Fl = static_cast<const LT*>(G.Fl);
    double f = 0.0;
    const int32_t i1 = __ldg(G.inc_ptr + node + 1);
    for (int32_t i = __ldg(G.inc_ptr + node); i < i1; ++i) {
      const int32_t p = __ldg(G.inc + i);  // e * NB + local a
      int s[NB];
      load_slots<NB>(G.slot, i, s);
      const int64_t lrow = (int64_t)p * NDPN + comp;  // local row (a, comp) of element e
      LT v[NL];
      load_row<NL>(Lm + lrow * NL, v);
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int j = 0; j < NDPN; ++j) a[NDPN * s[b] + j] += widen(v[NDPN * b + j]);
      if (Fl) f += widen(__ldg(Fl + lrow));
    }
    if (G.rhs) G.rhs[r] = f;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < span; k += rows) G.values[base + k] = acc[k];
}

fea_status launch_gather(int nb, int ndpn, bool mixed, const GatherArgs& G, int rows_per_tile,
                         int64_t max_tile_nnz, cudaStream_t s);

}  // namespace fea

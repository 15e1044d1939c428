// Deterministic scatter over the tile-interleaved local-row layout, fed by
// bulk copies (the Blackwell TMA engine, cp.async.bulk) through a ring of
// shared-memory stages.
//
// The row-owner reduction is the one of gather.cuh: one CTA per tile of
// consecutive CSR rows, one thread per row, the tile's CSR span accumulated
// in shared memory, each row's contributions added in ascending element
// order (so the result is bitwise the same as gather.cuh's, reproducible and
// symmetric).  What changes is how the contributions arrive.  In the
// incidence layout a thread reads its own row's k-th contribution, and the 32
// threads of a warp touch 32 unrelated places; here step k of a tile (the
// k-th contribution of each of its rows) is one contiguous block of global
// memory (the element kernel writes every local row to its tiled position,
// Pattern::tpos).  Thread 0 streams the tile step by step with bulk copies
// into STAGES (2 to 4) shared-memory stages, each completed by an mbarrier
// transaction count, so STAGES - 1 steps are in flight while the CTA adds the
// current one; no thread waits on its own global loads.  The launcher picks
// STAGES per launch from the shared memory that the accumulator leaves
// (tiled_stages_auto).
//
// Every wait on an mbarrier is bounded (TILED_WAIT_LIMIT polls).  If a step
// never completes, the CTA raises DEV_ERR_TIMEOUT in the mesh's error word,
// waits (again bounded) for the copies it has issued, and returns without
// writing its rows.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bulkcopy.cuh"
#include "gather.cuh"

namespace fea {

constexpr int TILED_STAGES = 2;      // default stage count (tiled_stages_auto)
constexpr int TILED_MAX_STAGES = 4;
constexpr uint32_t TILED_WAIT_LIMIT = BULK_WAIT_LIMIT;

// ------------------------------------------------------------------ layout
template <int NB, typename LT>
struct Tiled {
  static constexpr int LS = lstride(NB, sizeof(LT));  // local-row stride (values)
  static constexpr int SW = NB <= 4 ? 4 : 16;         // slot bytes per position
  // bytes of one step of S positions: local rows, slots, local loads
  __host__ __device__ static constexpr uint32_t lm_bytes(int S) { return (uint32_t)S * LS * sizeof(LT); }
  __host__ __device__ static constexpr uint32_t sl_bytes(int S) { return (uint32_t)S * SW; }
  __host__ __device__ static constexpr uint32_t fl_bytes(int S, bool f) { return f ? (uint32_t)S * sizeof(LT) : 0u; }
  __host__ __device__ static constexpr uint32_t stage_stride(int rows) {
    return ((lm_bytes((rows + 3) & ~3) + sl_bytes((rows + 3) & ~3) + fl_bytes((rows + 3) & ~3, true)) + 127u) &
           ~127u;
  }
  // dynamic shared memory: mbarriers, the accumulator span, the stages
  __host__ __device__ static constexpr size_t smem_bytes(int rows, int64_t span_cap, int stages = TILED_STAGES) {
    return 128 + (((size_t)span_cap * 8 + 127) & ~size_t(127)) + (size_t)stages * stage_stride(rows);
  }
};

struct TiledArgs {
  int64_t ndof;
  int rows;                       // rows per tile
  int64_t span_cap;               // accumulator capacity (doubles) of this launch
  const int32_t* row_ptr;
  const int32_t* inc_ptr;
  const int64_t* tile_base;
  const int32_t* tile_steps;
  const uint8_t* tslot;
  const void* Lm;
  const void* Fl;                 // or NULL
  double* values;
  double* rhs;                    // or NULL
  int* err;
};

template <int NB, typename LT>
__device__ __forceinline__ void load_smem_row(const LT* __restrict__ p, LT v[NB]);
template <>
__device__ __forceinline__ void load_smem_row<3, double>(const double* __restrict__ p, double v[3]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  v[0] = a.x;
  v[1] = a.y;
  v[2] = p[2];
}
template <>
__device__ __forceinline__ void load_smem_row<4, double>(const double* __restrict__ p, double v[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}
template <>
__device__ __forceinline__ void load_smem_row<10, double>(const double* __restrict__ p, double v[10]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const double2 a = reinterpret_cast<const double2*>(p)[k];
    v[2 * k] = a.x;
    v[2 * k + 1] = a.y;
  }
}
template <>
__device__ __forceinline__ void load_smem_row<4, float>(const float* __restrict__ p, float v[4]) {
  const float4 a = reinterpret_cast<const float4*>(p)[0];
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
template <>
__device__ __forceinline__ void load_smem_row<10, float>(const float* __restrict__ p, float v[10]) {
  const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  const float2 c = reinterpret_cast<const float2*>(p)[4];
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
  v[4] = b.x;
  v[5] = b.y;
  v[6] = b.z;
  v[7] = b.w;
  v[8] = c.x;
  v[9] = c.y;
}

template <int NB>
__device__ __forceinline__ void smem_slots(const uint8_t* __restrict__ p, int s[NB]) {
  if constexpr (NB <= 4) {
    const uint32_t w = *reinterpret_cast<const uint32_t*>(p);
#pragma unroll
    for (int b = 0; b < NB; ++b) s[b] = (w >> (8 * b)) & 0xFF;
  } else {
    const uint4 w = *reinterpret_cast<const uint4*>(p);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int b = 0; b < NB; ++b) s[b] = (ws[b >> 2] >> (8 * (b & 3))) & 0xFF;
  }
}

// The scatter of row tile `tile` by the whole CTA (blockDim.x >= G.rows;
// threads past the tile's rows only help with the accumulator), with `sm`
// the 128-byte aligned dynamic shared memory of
// Tiled<NB, LT>::smem_bytes(rows, G.span_cap, STAGES).  A CTA runs this
// once: its mbarriers are initialised here.
template <int NB, typename LT, int STAGES = TILED_STAGES>
__device__ __forceinline__ void gather_tiled_tile(const TiledArgs& G, int64_t tile, unsigned char* sm) {
  static_assert(STAGES >= 2 && STAGES <= TILED_MAX_STAGES, "stage count");
  using L = Tiled<NB, LT>;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
  double* acc = reinterpret_cast<double*>(sm + 128);
  unsigned char* stages = sm + 128 + (((size_t)G.span_cap * 8 + 127) & ~size_t(127));
  const uint32_t stride = L::stage_stride(G.rows);

  const int64_t r0 = tile * G.rows;
  const int64_t r1 = r0 + G.rows < G.ndof ? r0 + G.rows : G.ndof;
  const int R = (int)(r1 - r0);
  const int S = (R + 3) & ~3;
  const int K = __ldg(G.tile_steps + tile);
  const int64_t pbase = __ldg(G.tile_base + tile);
  const bool has_f = G.Fl != nullptr;
  const uint32_t lm_b = L::lm_bytes(S), sl_b = L::sl_bytes(S), fl_b = L::fl_bytes(S, has_f);
  const int tid = threadIdx.x;

  const int32_t base = __ldg(G.row_ptr + r0);
  const int32_t span = __ldg(G.row_ptr + r1) - base;
  for (int k = tid; k < span; k += blockDim.x) acc[k] = 0.0;
  if (tid == 0) {
#pragma unroll
    for (int st = 0; st < STAGES; ++st) mbar_init(&bar[st], 1);
    mbar_init_fence();
  }
  __syncthreads();

  // thread 0: step k of the tile -> stage k % STAGES
  auto issue = [&](int k) {
    const int st = k % STAGES;
    unsigned char* dst = stages + (size_t)st * stride;
    const int64_t p = pbase + (int64_t)k * S;
    mbar_expect_tx(&bar[st], lm_b + sl_b + fl_b);
    bulk_load(dst, static_cast<const LT*>(G.Lm) + p * L::LS, lm_b, &bar[st]);
    bulk_load(dst + lm_b, G.tslot + p * L::SW, sl_b, &bar[st]);
    if (has_f) bulk_load(dst + lm_b + sl_b, static_cast<const LT*>(G.Fl) + p, fl_b, &bar[st]);
  };
  int issued = 0;  // thread 0's count of issued steps
  if (tid == 0)
    for (; issued < (K < STAGES ? K : STAGES); ++issued) issue(issued);

  const bool mine = tid < R;
  const int64_t r = r0 + tid;
  int cnt = 0;
  int off = 0;
  if (mine) {
    cnt = __ldg(G.inc_ptr + r + 1) - __ldg(G.inc_ptr + r);
    off = __ldg(G.row_ptr + r) - base;
  }
  double* a = acc + off;
  double f = 0.0;
  int k = 0;
  bool failed = false;
  for (; k < K; ++k) {
    const int st = k % STAGES;
    const bool ok = mbar_wait(&bar[st], (uint32_t)(k / STAGES) & 1u);
    if (ok && mine && k < cnt) {
      const unsigned char* sp = stages + (size_t)st * stride;
      int sl[NB];
      smem_slots<NB>(sp + lm_b + (size_t)tid * L::SW, sl);
      LT v[NB];
      load_smem_row<NB, LT>(reinterpret_cast<const LT*>(sp) + (size_t)tid * L::LS, v);
      if (slots_ok<NB, 1>(off, sl, span, G.err)) add_row<NB, 1, LT>(a, sl, v);
      if (has_f) f += widen(reinterpret_cast<const LT*>(sp + lm_b + sl_b)[tid]);
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (tid == 0 && issued < K) {
      fence_async_smem();
      issue(issued);
      ++issued;
    }
  }
  if (failed) {
    if (tid == 0) {
      atomicOr(G.err, DEV_ERR_TIMEOUT);
      // let the copies already issued land before the CTA's shared memory goes away
      for (int j = k; j < issued; ++j) mbar_wait(&bar[j % STAGES], (uint32_t)(j / STAGES) & 1u);
    }
    __syncthreads();
    return;
  }
  if (mine && G.rhs) G.rhs[r] = f;
  __syncthreads();
  for (int j = tid; j < span; j += blockDim.x) G.values[base + j] = acc[j];
}

// One CTA per row tile (tiles[blockIdx.x], or blockIdx.x), blockDim.x == rows.
template <int NB, typename LT, int STAGES>
__global__ void __launch_bounds__(128) k_gather_tiled(TiledArgs G, const int32_t* __restrict__ tiles) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int64_t tile = tiles ? (int64_t)__ldg(tiles + blockIdx.x) : (int64_t)blockIdx.x;
  gather_tiled_tile<NB, LT, STAGES>(G, tile, sm);
}

// stages: 2 to TILED_MAX_STAGES, or 0 for the automatic choice
// (tiled_stages_auto).
fea_status launch_gather_tiled(int nb, bool mixed, const TiledArgs& G, cudaStream_t s, const int32_t* tiles,
                               int64_t ntiles, int stages = 0);

// The stage count for a CTA whose accumulator holds span_cap doubles: the
// most resident CTAs per SM, and of those counts the fewest stages.
// (Measured on the P2 diffusion + mass scatter: two stages and three CTAs per
// SM beat three stages and two CTAs by 14%, four stages and two CTAs lose a
// further 15%; at an equal CTA count three stages gain nothing over two and
// four lose 20% (FP32 rows, long-row tiles): the CTAs' warps hide the
// shared-memory adds and the pipeline fill of the short tiles, deeper rings
// do not.)
int tiled_stages_auto(int nb, bool mixed, int rows, int64_t span_cap);

// Whether a scalar pattern takes the bulk-copy scatter: its tiled layout is
// built and the mesh's scatter mode is automatic (-1) or 3.
bool use_tiled(const fea_mesh* m, const Pattern* P);

// The whole scatter of one assembly over the tiled layout (local rows Lm and
// loads Fl at Pattern::tpos positions).
fea_status scatter_tiled(const fea_mesh* m, const Pattern* P, const Base* B, bool mixed, const void* Lm,
                         const void* Fl, double* values, double* rhs, cudaStream_t s);

// The tiles tiles[0 .. ntiles) only (one stage of the overlapped assembly).
fea_status scatter_tiled_list(const fea_mesh* m, const Pattern* P, const Base* B, bool mixed, const void* Lm,
                              const void* Fl, double* values, double* rhs, const int32_t* tiles, int64_t ntiles,
                              cudaStream_t s);

}  // namespace fea

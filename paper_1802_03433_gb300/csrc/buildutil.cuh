// Building blocks of the one-time pattern and chunk construction (pattern.cu,
// chunks.cu): device buffers, an exclusive scan, a warp bitonic sort and a
// per-list sort.  Everything is in an unnamed namespace: each translation
// unit that includes this header has its own copy.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "internal.cuh"

namespace fea {
namespace {

constexpr int SCAN_T = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_BLOCK = SCAN_T * SCAN_ITEMS;

// ------------------------------------------------------------------ buffers
template <typename T>
fea_status dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(FEA_ERR_NOMEM, "device allocation of " + std::to_string(n * sizeof(T)) + " bytes failed");
  }
  return FEA_OK;
}
template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// RAII temporary device buffer.
template <typename T>
struct Tmp {
  T* p = nullptr;
  ~Tmp() { dfree(p); }
  fea_status alloc(size_t n) { return dalloc(&p, n); }
};

int blocks_for(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

// ------------------------------------------------------------------ scan
__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// Exclusive block scan of one value per thread; returns the exclusive prefix
// and sets *total to the block sum.
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* total) {
  __shared__ int64_t ws[33];  // per-warp prefixes, then the block total
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int64_t inc = warp_incl_scan(v);
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < nw ? ws[lane] : 0;
    int64_t wi = warp_incl_scan(w);
    if (lane < nw) ws[lane] = wi - w;
    if (lane == 31) ws[32] = wi;
  }
  __syncthreads();
  int64_t ex = ws[warp] + inc - v;
  *total = ws[32];
  __syncthreads();
  return ex;
}

template <typename TI>
__global__ void __launch_bounds__(SCAN_T) k_scan_local(const TI* __restrict__ in, int64_t n,
                                                       int64_t* __restrict__ out, int64_t* __restrict__ bsum) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t ts = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int64_t i = base + k;
    v[k] = i < n ? (int64_t)in[i] : 0;
    ts += v[k];
  }
  int64_t total;
  int64_t ex = block_excl_scan(ts, &total);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int64_t i = base + k;
    if (i < n) out[i] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Single block: exclusive scan of the block sums in place; total -> *tot.
__global__ void __launch_bounds__(1024) k_scan_sums(int64_t* __restrict__ bsum, int64_t nb,
                                                    int64_t* __restrict__ tot) {
  int64_t carry = 0;
  for (int64_t s = 0; s < nb; s += blockDim.x) {
    const int64_t i = s + threadIdx.x;
    const int64_t v = i < nb ? bsum[i] : 0;
    int64_t total;
    const int64_t ex = block_excl_scan(v, &total);
    if (i < nb) bsum[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) *tot = carry;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ bsum) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += bsum[i / SCAN_BLOCK];
}

// out[0..n] = exclusive scan of in[0..n), out[n] = total.
template <typename TI>
fea_status scan(const TI* in, int64_t n, int64_t* out, cudaStream_t s) {
  const int64_t nb = std::max<int64_t>(1, (n + SCAN_BLOCK - 1) / SCAN_BLOCK);
  Tmp<int64_t> bsum;
  FEA_TRY(bsum.alloc(nb));
  k_scan_local<TI><<<(unsigned)nb, SCAN_T, 0, s>>>(in, n, out, bsum.p);
  k_scan_sums<<<1, 1024, 0, s>>>(bsum.p, nb, out + n);
  k_scan_add<<<blocks_for(n, 256), 256, 0, s>>>(out, n, bsum.p);
  FEA_CUDA(cudaGetLastError());
  FEA_CUDA(cudaStreamSynchronize(s));  // bsum is freed on return
  return FEA_OK;
}

__global__ void k_i64_to_i32(const int64_t* __restrict__ in, int64_t n, int32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int32_t)in[i];
}

fea_status read_i64(const int64_t* d, int64_t* h, cudaStream_t s) {
  FEA_CUDA(cudaMemcpyAsync(h, d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaStreamSynchronize(s));
  return FEA_OK;
}

// Exclusive scan of int32 counts into an int32 pointer array of n + 1,
// failing with FEA_ERR_OVERFLOW when the total does not fit int32.
fea_status scan_to_ptr32(const int32_t* cnt, int64_t n, int32_t* ptr, int64_t* total, cudaStream_t s,
                         const char* what) {
  Tmp<int64_t> p64;
  FEA_TRY(p64.alloc(n + 1));
  FEA_TRY(scan(cnt, n, p64.p, s));
  FEA_TRY(read_i64(p64.p + n, total, s));
  if (*total > (int64_t)INT32_MAX)
    return fail(FEA_ERR_OVERFLOW, std::string(what) + " count " + std::to_string(*total) + " exceeds INT32_MAX");
  k_i64_to_i32<<<blocks_for(n + 1, 256), 256, 0, s>>>(p64.p, n + 1, ptr);
  FEA_CUDA(cudaGetLastError());
  FEA_CUDA(cudaStreamSynchronize(s));
  return FEA_OK;
}

// ------------------------------------------------------------------ warp sort
// Bitonic sort of 32 * R keys held R per lane (lane L holds sorted positions
// L * R .. L * R + R - 1), ascending: compare-exchanges within a lane for
// strides below R, across lanes by shuffles above.
template <typename T, int R>
__device__ __forceinline__ void warp_sort_reg(T (&key)[R]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32 * R; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride < R) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if ((r & stride) == 0) {
            const bool asc = ((lane * R + r) & size) == 0;
            const T a = key[r], b = key[r | stride];
            const bool sw = (a > b) == asc;
            key[r] = sw ? b : a;
            key[r | stride] = sw ? a : b;
          }
        }
      } else {
        const int ls = stride / R;
        const bool lower = (lane & ls) == 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const bool asc = ((lane * R + r) & size) == 0;
          const T o = __shfl_xor_sync(0xffffffffu, key[r], ls);
          const bool take_min = lower == asc;
          key[r] = take_min ? (o < key[r] ? o : key[r]) : (o > key[r] ? o : key[r]);
        }
      }
    }
  }
}


// Sort each list ptr[d] .. ptr[d + 1] of int32 values ascending, one warp per
// list (a dof's incidences by element id, a cell's elements, a shared
// coupling's partial sums by chunk): lists of up to 1024 sort in registers
// (warp_sort_reg), longer ones by insertion sort in lane 0.
template <int R>
__device__ __forceinline__ void inc_sort_reg(int32_t* __restrict__ list, int len) {
  const int lane = threadIdx.x & 31;
  int32_t key[R];
#pragma unroll
  for (int r = 0; r < R; ++r) key[r] = lane * R + r < len ? list[lane * R + r] : 0x7FFFFFFF;
  warp_sort_reg<int32_t, R>(key);
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (lane * R + r < len) list[lane * R + r] = key[r];
}

__global__ void __launch_bounds__(128) k_sort_lists(const int32_t* __restrict__ ptr, int64_t n, int32_t* __restrict__ inc) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t d = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < n; d += nwarps) {
    const int32_t b = ptr[d], len = ptr[d + 1] - b;
    int32_t* list = inc + b;
    if (len <= 1) continue;
    if (len <= 32) {
      inc_sort_reg<1>(list, len);
    } else if (len <= 64) {
      inc_sort_reg<2>(list, len);
    } else if (len <= 128) {
      inc_sort_reg<4>(list, len);
    } else if (len <= 256) {
      inc_sort_reg<8>(list, len);
    } else if (len <= 512) {
      inc_sort_reg<16>(list, len);
    } else if (len <= 1024) {
      inc_sort_reg<32>(list, len);
    } else if (lane == 0) {
      for (int32_t i = 1; i < len; ++i) {
        const int32_t v = list[i];
        int32_t j = i - 1;
        while (j >= 0 && list[j] > v) {
          list[j + 1] = list[j];
          --j;
        }
        list[j + 1] = v;
      }
    }
    __syncwarp();
  }
}

}  // namespace
}  // namespace fea

// Diagnostic entry points (self-checks of device helpers; no counterpart in
// the paper).
#include "element.cuh"
#include "gather_tiled.cuh"
#include "internal.cuh"

namespace fea {
namespace {
__global__ void k_diag_rcp(const double* __restrict__ x, int64_t n, double* __restrict__ mine,
                           double* __restrict__ lib) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  mine[i] = rcp_pos(x[i]);
  lib[i] = 1.0 / x[i];
}

__global__ void k_diag_sinpi(const double* __restrict__ x, int64_t n, int variant, double* __restrict__ mine,
                             double* __restrict__ lib) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (variant == 3) {
    const double v[4] = {x[i], x[i], x[i], x[i]};
    const int s = fx_shift(v);
    mine[i] = __ll2double_rn(sinpi_q62_fx(to_fx(x[i], s), s)) * 0x1p-62;
  } else {
    mine[i] = variant == 0   ? rsinpi<double>(x[i])
              : variant == 1 ? sinpi_fp64(x[i])
                             : __ll2double_rn(sinpi_q62(x[i])) * 0x1p-62;
  }
  lib[i] = sinpi(x[i]);
}
// The bounded mbarrier wait of the bulk-copy scatter on a barrier whose one
// expected arrival never comes (no copy is issued): every thread gives up
// after `polls` polls and the kernel raises DEV_ERR_TIMEOUT in the error word,
// as the scatter does when a copy never completes.
__global__ void k_diag_wait_timeout(int* err, uint32_t polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, polls);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(err, DEV_ERR_TIMEOUT);
}

// Eight independent DFMA chains per thread: the FP64 pipe's sustained FMA
// rate, the denominator of the element kernels' roofline.
__global__ void k_diag_dfma(double* __restrict__ out, int iters, double s) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-9 + k;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], s, 0.5);
  double r = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) r += a[k];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}
}  // namespace
}  // namespace fea

extern "C" fea_status fea_diag_fp64_rate(double* flops_per_s, void* stream) {
  if (!flops_per_s) return fea::fail(FEA_ERR_ARG, "flops_per_s is NULL");
  int dev = 0, sms = 0;
  FEA_CUDA(cudaGetDevice(&dev));
  FEA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = sms * 8, threads = 256, iters = 2048;
  double* out = nullptr;
  FEA_CUDA(cudaMallocAsync((void**)&out, sizeof(double) * blocks * threads, s));
  cudaEvent_t a, b;
  FEA_CUDA(cudaEventCreate(&a));
  FEA_CUDA(cudaEventCreate(&b));
  fea::k_diag_dfma<<<blocks, threads, 0, s>>>(out, iters, 0.999);  // warm-up
  FEA_CUDA(cudaEventRecord(a, s));
  for (int r = 0; r < 5; ++r) fea::k_diag_dfma<<<blocks, threads, 0, s>>>(out, iters, 0.999);
  FEA_CUDA(cudaEventRecord(b, s));
  FEA_CUDA(cudaEventSynchronize(b));
  float ms = 0.f;
  FEA_CUDA(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  FEA_CUDA(cudaFreeAsync(out, s));
  FEA_CUDA(cudaStreamSynchronize(s));
  *flops_per_s = 5.0 * blocks * threads * iters * 8 * 2.0 / (ms * 1e-3);
  return FEA_OK;
}

extern "C" fea_status fea_diag_rcp(const double* x, int64_t n, double* mine, double* lib, void* stream) {
  if (n < 0 || (n > 0 && (!x || !mine || !lib))) return fea::fail(FEA_ERR_ARG, "bad argument");
  if (n == 0) return FEA_OK;
  fea::k_diag_rcp<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n, mine, lib);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

extern "C" fea_status fea_diag_sinpi(const double* x, int64_t n, int32_t variant, double* mine, double* lib,
                                      void* stream) {
  if (n < 0 || (n > 0 && (!x || !mine || !lib)) || variant < 0 || variant > 3)
    return fea::fail(FEA_ERR_ARG, "bad argument");
  if (n == 0) return FEA_OK;
  fea::k_diag_sinpi<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n, variant, mine,
                                                                                               lib);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

namespace fea {
namespace {
__global__ void k_diag_checked_gather(const double* src, int64_t n, int64_t idx, double* out, int* err) {
  out[0] = index_ok(idx, n, err) ? src[idx] : -1.0;
}
}  // namespace
}  // namespace fea

extern "C" fea_status fea_diag_checked_gather(fea_mesh* m, const double* src, int64_t n, int64_t idx, double* out,
                                              int32_t* checked, void* stream) {
  if (!m || !checked) return fea::fail(FEA_ERR_ARG, "NULL argument");
#ifdef FEA_CHECKED
  *checked = 1;
  if (!src || !out || n < 1) return fea::fail(FEA_ERR_ARG, "src, out and n >= 1 are required");
  fea::k_diag_checked_gather<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(src, n, idx, out, m->err);
  FEA_CUDA(cudaGetLastError());
#else
  (void)src;
  (void)n;
  (void)idx;
  (void)out;
  (void)stream;
  *checked = 0;
#endif
  return FEA_OK;
}

extern "C" fea_status fea_diag_wait_timeout(fea_mesh* m, int32_t polls, void* stream) {
  if (!m) return fea::fail(FEA_ERR_ARG, "mesh is NULL");
  if (polls < 1 || polls > (1 << 20)) return fea::fail(FEA_ERR_ARG, "polls must be in [1, 2^20]");
  fea::k_diag_wait_timeout<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(m->err, (uint32_t)polls);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

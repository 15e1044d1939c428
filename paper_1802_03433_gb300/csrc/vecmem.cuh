// 32-byte global loads and stores (sm_100 and later): one instruction moves
// one whole DRAM sector, so a local row written by one thread is never left
// partly written in L2 (no read-fill) and a scatter thread reads a row with a
// third of the load instructions of 16-byte vectors.  Addresses must be
// 32-byte aligned.
#pragma once

#include "devcommon.cuh"

namespace fea {

__device__ __forceinline__ void st_v4(double* p, double a, double b, double c, double d) {
  asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(a), "d"(b), "d"(c), "d"(d) : "memory");
}
__device__ __forceinline__ void st_v8(float* p, float a, float b, float c, float d, float e, float f, float g,
                                      float h) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d),
               "f"(e), "f"(f), "f"(g), "f"(h)
               : "memory");
}
__device__ __forceinline__ void ld_v4(const double* p, double& a, double& b, double& c, double& d) {
  asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(a), "=d"(b), "=d"(c), "=d"(d) : "l"(p));
}
__device__ __forceinline__ void ld_v8(const float* p, float& a, float& b, float& c, float& d, float& e, float& f,
                                      float& g, float& h) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a), "=f"(b), "=f"(c), "=f"(d), "=f"(e), "=f"(f), "=f"(g), "=f"(h)
      : "l"(p));
}

// Store one local row of NL values at p (32-byte aligned) as whole 32-byte
// sectors, zero padding included up to lstride.
template <int NL>
__device__ __forceinline__ void store_row(double* __restrict__ p, const double* v) {
  constexpr int LS = lstride(NL, 8);
#pragma unroll
  for (int k = 0; k < LS / 4; ++k)
    st_v4(p + 4 * k, 4 * k < NL ? v[4 * k] : 0.0, 4 * k + 1 < NL ? v[4 * k + 1] : 0.0,
          4 * k + 2 < NL ? v[4 * k + 2] : 0.0, 4 * k + 3 < NL ? v[4 * k + 3] : 0.0);
}
template <int NL>
__device__ __forceinline__ void store_row(float* __restrict__ p, const float* v) {
  constexpr int LS = lstride(NL, 4);
#pragma unroll
  for (int k = 0; k < LS / 8; ++k) {
    float w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = 8 * k + j < NL ? v[8 * k + j] : 0.f;
    st_v8(p + 8 * k, w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7]);
  }
}

}  // namespace fea

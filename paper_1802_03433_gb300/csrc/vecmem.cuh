// 32-byte global loads and stores (sm_100 and later): one instruction moves
// one whole DRAM sector, so a local row written by one thread is never left
// partly written in L2 (no read-fill) and a scatter thread reads a row with a
// third of the load instructions of 16-byte vectors.  Addresses must be
// 32-byte aligned.
#pragma once

#include <cuda_runtime.h>

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

}  // namespace fea

// Host-side dispatch from runtime (load kind, rule, precision) to the
// element-kernel template instances.
#pragma once

#include "elem_kernels.cuh"

namespace fea {

inline unsigned elem_blocks(const ElemArgs& A) { return (unsigned)((A.e1 - A.e0 + ELEM_T - 1) / ELEM_T); }

template <int ORDER, bool MASS>
struct ScalarLauncher {
  template <int LOAD, int NPTS>
  static void go(const ElemArgs& A, int prec, cudaStream_t s) {
    if (prec == FEA_FP64)
      k_elem_scalar<ORDER, MASS, LOAD, NPTS, double><<<elem_blocks(A), ELEM_T, 0, s>>>(A);
    else
      k_elem_scalar<ORDER, MASS, LOAD, NPTS, float><<<elem_blocks(A), ELEM_T, 0, s>>>(A);
  }
  template <int NPTS>
  static void by_load(const ElemArgs& A, int load, int prec, cudaStream_t s) {
    if (load == LOAD_CONST) go<LOAD_CONST, NPTS>(A, prec, s);
    else go<LOAD_SIN, NPTS>(A, prec, s);
  }
  static fea_status run(const ElemArgs& A, int load, int npts, int prec, cudaStream_t s) {
    if (A.e1 <= A.e0) return FEA_OK;
    if (load == LOAD_NONE) go<LOAD_NONE, 1>(A, prec, s);
    else if (npts == 1) by_load<1>(A, load, prec, s);
    else if (npts == 4) by_load<4>(A, load, prec, s);
    else by_load<11>(A, load, prec, s);
    FEA_CUDA(cudaGetLastError());
    return FEA_OK;
  }
};

template <int ORDER>
struct LoadLauncher {
  template <int LOAD, int NPTS>
  static void go(const ElemArgs& A, int prec, cudaStream_t s) {
    if (prec == FEA_FP64)
      k_elem_load<ORDER, LOAD, NPTS, double><<<elem_blocks(A), ELEM_T, 0, s>>>(A);
    else
      k_elem_load<ORDER, LOAD, NPTS, float><<<elem_blocks(A), ELEM_T, 0, s>>>(A);
  }
  template <int NPTS>
  static void by_load(const ElemArgs& A, int load, int prec, cudaStream_t s) {
    if (load == LOAD_CONST) go<LOAD_CONST, NPTS>(A, prec, s);
    else go<LOAD_SIN, NPTS>(A, prec, s);
  }
  static fea_status run(const ElemArgs& A, int load, int npts, int prec, cudaStream_t s) {
    if (A.e1 <= A.e0 || load == LOAD_NONE) return FEA_OK;
    if (npts == 1) by_load<1>(A, load, prec, s);
    else if (npts == 4) by_load<4>(A, load, prec, s);
    else by_load<11>(A, load, prec, s);
    FEA_CUDA(cudaGetLastError());
    return FEA_OK;
  }
};

// FP64 only: matrix and load warps of the same elements in one kernel.
template <int ORDER, bool MASS>
struct RolesLauncher {
  template <int LOAD, int NPTS>
  static void go(const ElemArgs& A, cudaStream_t s) {
    k_elem_roles<ORDER, MASS, LOAD, NPTS><<<elem_blocks(A), 2 * ELEM_T, 0, s>>>(A);
  }
  template <int NPTS>
  static void by_load(const ElemArgs& A, int load, cudaStream_t s) {
    if (load == LOAD_CONST) go<LOAD_CONST, NPTS>(A, s);
    else go<LOAD_SIN, NPTS>(A, s);
  }
  static fea_status run(const ElemArgs& A, int load, int npts, cudaStream_t s) {
    if (A.e1 <= A.e0 || load == LOAD_NONE) return FEA_OK;
    if (npts == 1) by_load<1>(A, load, s);
    else if (npts == 4) by_load<4>(A, load, s);
    else by_load<11>(A, load, s);
    FEA_CUDA(cudaGetLastError());
    return FEA_OK;
  }
};

struct ElastLauncher {
  template <int LOAD, int NPTS>
  static void go(const ElemArgs& A, int prec, cudaStream_t s) {
    if (prec == FEA_FP64)
      k_elem_elast<LOAD, NPTS, double><<<elem_blocks(A), ELEM_T, 0, s>>>(A);
    else
      k_elem_elast<LOAD, NPTS, float><<<elem_blocks(A), ELEM_T, 0, s>>>(A);
  }
  template <int NPTS>
  static void by_load(const ElemArgs& A, int load, int prec, cudaStream_t s) {
    if (load == LOAD_CONST) go<LOAD_CONST, NPTS>(A, prec, s);
    else go<LOAD_SIN, NPTS>(A, prec, s);
  }
  static fea_status run(const ElemArgs& A, int load, int npts, int prec, cudaStream_t s) {
    if (A.e1 <= A.e0) return FEA_OK;
    if (load == LOAD_NONE) go<LOAD_NONE, 1>(A, prec, s);
    else if (npts == 1) by_load<1>(A, load, prec, s);
    else if (npts == 4) by_load<4>(A, load, prec, s);
    else by_load<11>(A, load, prec, s);
    FEA_CUDA(cudaGetLastError());
    return FEA_OK;
  }
};

}  // namespace fea

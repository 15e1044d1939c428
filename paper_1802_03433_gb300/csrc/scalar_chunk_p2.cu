// Chunk kernels of the scalar P2 forms (scalar_chunk.cuh); FP64 with a load
// takes the kernel with matrix threads and load threads.
#include "scalar_chunk.cuh"

namespace fea {
namespace chunkfx {
namespace {

template <bool MASS, int LOAD, int NPTS, typename R>
void go(const ElemArgs& A, const ChunkArgs& Cg, int64_t nchunk, size_t smem, cudaStream_t s) {
  constexpr bool ROLES = IsDouble<R>::value && LOAD != LOAD_NONE;
  static size_t configured = 0;  // opt-in above the 48 KB default, once per instance
  if (smem > 48 * 1024 && smem > configured) {
    cudaFuncSetAttribute(k_scalar_chunk<2, MASS, LOAD, NPTS, R, ROLES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    configured = smem;
  }
  k_scalar_chunk<2, MASS, LOAD, NPTS, R, ROLES><<<(unsigned)nchunk, ROLES ? 2 * SC_T : SC_T, smem, s>>>(A, Cg);
}

template <bool MASS, typename R>
void by_load(int load, int npts, const ElemArgs& A, const ChunkArgs& Cg, int64_t nchunk, size_t smem, cudaStream_t s) {
  if (load == LOAD_NONE) return go<MASS, LOAD_NONE, 1, R>(A, Cg, nchunk, smem, s);
  if (load == LOAD_CONST) {
    if (npts == 1) return go<MASS, LOAD_CONST, 1, R>(A, Cg, nchunk, smem, s);
    if (npts == 4) return go<MASS, LOAD_CONST, 4, R>(A, Cg, nchunk, smem, s);
    return go<MASS, LOAD_CONST, 11, R>(A, Cg, nchunk, smem, s);
  }
  if (npts == 1) return go<MASS, LOAD_SIN, 1, R>(A, Cg, nchunk, smem, s);
  if (npts == 4) return go<MASS, LOAD_SIN, 4, R>(A, Cg, nchunk, smem, s);
  return go<MASS, LOAD_SIN, 11, R>(A, Cg, nchunk, smem, s);
}

}  // namespace

fea_status launch_scalar_chunk_p2(bool mass, int load, int npts, bool mixed, const ElemArgs& A, const ChunkArgs& Cg,
                                  int64_t nchunk, size_t smem, cudaStream_t s) {
  if (mixed) {
    if (mass) by_load<true, float>(load, npts, A, Cg, nchunk, smem, s);
    else by_load<false, float>(load, npts, A, Cg, nchunk, smem, s);
  } else {
    if (mass) by_load<true, double>(load, npts, A, Cg, nchunk, smem, s);
    else by_load<false, double>(load, npts, A, Cg, nchunk, smem, s);
  }
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

}  // namespace chunkfx
}  // namespace fea

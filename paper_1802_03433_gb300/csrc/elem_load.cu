// Load-vector-only element kernels (scalar forms), launched beside the
// matrix kernel when the mesh's load split is on.
#include "elem_launch.cuh"

namespace fea {
fea_status launch_elem_load(int order, const ElemArgs& A, int load, int npts, int prec, cudaStream_t s) {
  return order == 1 ? LoadLauncher<1>::run(A, load, npts, prec, s) : LoadLauncher<2>::run(A, load, npts, prec, s);
}
}  // namespace fea

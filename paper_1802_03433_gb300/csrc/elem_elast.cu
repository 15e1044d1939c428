// P1 linear elasticity element kernels.
#include "elem_launch.cuh"

namespace fea {
fea_status launch_elem_elast(const ElemArgs& A, int load, int npts, int prec, cudaStream_t s) {
  return ElastLauncher::run(A, load, npts, prec, s);
}
}  // namespace fea

// P2 scalar element kernels (kappa-diffusion, optional mass term).
#include "elem_launch.cuh"

namespace fea {
fea_status launch_elem_p2(const ElemArgs& A, bool mass, int load, int npts, int prec, cudaStream_t s) {
  return mass ? ScalarLauncher<2, true>::run(A, load, npts, prec, s)
              : ScalarLauncher<2, false>::run(A, load, npts, prec, s);
}
}  // namespace fea

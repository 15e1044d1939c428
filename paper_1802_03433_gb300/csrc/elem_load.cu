// Load-vector-only element kernels (scalar forms), launched beside the
// matrix kernel when the mesh's load split is on.
#include "elem_launch.cuh"

namespace fea {
fea_status launch_elem_load(int order, const ElemArgs& A, int load, int npts, int prec, cudaStream_t s) {
  return order == 1 ? LoadLauncher<1>::run(A, load, npts, prec, s) : LoadLauncher<2>::run(A, load, npts, prec, s);
}
fea_status launch_elem_roles(int order, bool mass, const ElemArgs& A, int load, int npts, cudaStream_t s) {
  if (order == 1)
    return mass ? RolesLauncher<1, true>::run(A, load, npts, s) : RolesLauncher<1, false>::run(A, load, npts, s);
  return mass ? RolesLauncher<2, true>::run(A, load, npts, s) : RolesLauncher<2, false>::run(A, load, npts, s);
}
}  // namespace fea

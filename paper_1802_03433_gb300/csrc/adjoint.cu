// Reverse mode of the scalar assembly (written below).
#include "internal.cuh"

namespace fea {
fea_status assemble_backward(fea_mesh*, const fea_form*, const fea_coeffs*, const fea_quadrature*, const double*,
                             const double*, double*, double*, cudaStream_t) {
  return fail(FEA_ERR_ARG, "backward not available");
}
}  // namespace fea

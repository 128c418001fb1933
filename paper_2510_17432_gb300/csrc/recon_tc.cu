// Tensor-core reconstruction of the Jackson DOS (placeholder until the tcgen05 path lands).
#include "tbpm_internal.cuh"

namespace tbpm {
int launch_dos_jackson_tensor(tbpm_ctx* ctx, const double* mu, int S, int M, const double* energies,
                              int64_t nE, double H0, double half, double* D) {
  (void)ctx; (void)mu; (void)S; (void)M; (void)energies; (void)nE; (void)H0; (void)half; (void)D;
  set_error("tensor-core reconstruction not available in this build");
  return TBPM_EUNSUPPORTED;
}
}  // namespace tbpm

// Placeholder of the tensor-core path until its kernels land: plans with a
// split dtype are refused with PHIKS_ERR_UNSUPPORTED.
#include "tc.cuh"

namespace phiks {

struct TcState {};

size_t tc_workspace_bytes(int64_t) { return 0; }
phiks_status tc_create(TcState** out, int, const int64_t*, int64_t) {
  *out = nullptr;
  return PHIKS_ERR_UNSUPPORTED;
}
void tc_destroy(TcState*) {}
const char* tc_last_error() { return "split-precision tensor-core path not built"; }
void tc_bind_workspace(TcState*, void*) {}
cudaError_t tc_mode_product(TcState*, int, const Combo&, const double*, ModeGeom, void*, const Epi*,
                            cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace phiks

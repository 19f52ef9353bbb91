// Fused k-qubit blocks on the tcgen05 tensor cores (split-TF32).  Placeholder until
// the kernel lands: the fused precision mode reports itself unavailable.
#include <cuda_runtime.h>

#include "kernels.h"
#include "state.h"

namespace svk {

bool fused_supported() { return false; }

cudaError_t launch_fused_pass(float2 *, int, const DevPlanView &, int, const svp::DevPass &, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace svk

namespace svc {
sv_status build_stage_mats(svp::Plan *, const std::vector<svp::Gate> &, int) { return SV_OK; }
}  // namespace svc

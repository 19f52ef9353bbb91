// sv_norm_noalloc: the fp64 norm / sum-of-squared-probabilities reduction of sv_norm,
// for callers that cannot allocate device memory.
//
// sv_norm needs 16 KB of device scratch for its per-block partial sums, which it takes
// from the handle (cudaMalloc on first use).  Some callers can't do that: code that runs
// under a device-memory budget owned by another allocator (a framework's caching
// allocator that has reserved the GPU), or code that must not trigger the implicit
// device-wide synchronisation cudaMalloc/cudaFree can cause.  This entry point takes a
// plain device pointer to the state and writes the two sums to the caller's host
// doubles; its scratch is a fixed file-scope device array, so it allocates nothing.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/sv.h"
#include "capi_util.h"
#include "kernels.h"
#include "state.h"

namespace {

// Partial sums of the level-1 reduction (two doubles per block, at most
// kNoallocBlocks blocks) followed by the two results.  16 KB + 16 B, held by every GPU
// that loads the library until the process exits.
constexpr int kNoallocBlocks = 1024;
static __device__ __align__(256) double g_norm_scratch[2 * kNoallocBlocks + 2];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double *g_scratch_dev[kMaxDevices] = {};  // device address of g_norm_scratch, per device

}  // namespace

extern "C" sv_status sv_norm_noalloc(const void *dev_state, int n_qubits, void *stream, double *norm2,
                                     double *sum_p2) {
  svc::clear_error();
  if (!dev_state) return svc::fail(SV_ERR_ARG, "sv_norm_noalloc: dev_state is NULL");
  if (n_qubits < 1 || n_qubits > 34)
    return svc::fail(SV_ERR_ARG, "sv_norm_noalloc: n_qubits must be 1..34 (states up to 2^34 amplitudes)");
  // the reduction reads two amplitudes per 16-byte vector (one 8-byte amplitude when n = 1)
  const uintptr_t align = n_qubits >= 2 ? 16 : 8;
  if ((reinterpret_cast<uintptr_t>(dev_state) & (align - 1)) != 0)
    return svc::fail(SV_ERR_ARG, n_qubits >= 2 ? "sv_norm_noalloc: dev_state must be 16-byte aligned"
                                               : "sv_norm_noalloc: dev_state must be 8-byte aligned");
  if (svk::reduce_partials_needed() > kNoallocBlocks)
    return svc::fail(SV_ERR_ARG, "sv_norm_noalloc: reduction grid larger than the static scratch");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return svc::cuda_fail(e, "sv_norm_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return svc::fail(SV_ERR_ARG, "sv_norm_noalloc: device index >= 64");
  double *scratch = nullptr;
  {
    // First call on this device (current device): look up the device address of the
    // static array.  Its host-side name is only a stand-in, never a device pointer.
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_norm_scratch);
      if (e != cudaSuccess) return svc::cuda_fail(e, "sv_norm_noalloc: cudaGetSymbolAddress");
      g_scratch_dev[dev] = static_cast<double *>(p);
    }
    scratch = g_scratch_dev[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Every partial-sum slot the final pass reads is written by the first pass of the same
  // call, so nothing in the array has to start at zero.
  double h[2] = {0.0, 0.0};
  e = svk::launch_norm(static_cast<const float2 *>(dev_state), n_qubits, scratch, scratch + 2 * kNoallocBlocks, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, scratch + 2 * kNoallocBlocks, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return svc::cuda_fail(e, "sv_norm_noalloc");
  if (norm2) *norm2 = h[0];
  if (sum_p2) *sum_p2 = h[1];
  return SV_OK;
}

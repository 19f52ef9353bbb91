// The state handle behind the opaque sv_state, and helpers shared by the C-ABI files.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/sv.h"
#include "kernels.h"
#include "plan.h"

namespace svj {
struct Module;
}

struct sv_state {
  int n = 0;
  float2 *psi = nullptr;  // 2^n complex64 amplitudes on the device
  bool owns = false;      // allocated by sv_create (freed by sv_destroy)
  sv_options opts{};
  cudaStream_t stream = nullptr;
  int device = 0;
  bool fresh = false;     // logically |0..0> but not yet written (lazy initial state)
  bool broken = false;    // an apply failed part-way: content undefined
  // device scratch: packed plan, gather/reduction buffers
  void *d_plan = nullptr;
  size_t d_plan_cap = 0;
  std::vector<char> h_plan;
  void *d_scratch = nullptr;
  size_t d_scratch_cap = 0;
  // profiling: event pairs around each pass launch
  bool prof = false;
  std::vector<cudaEvent_t> events;
  size_t ev_used = 0;
  std::vector<double> ev_bytes;
  double h2d = 0, d2h = 0;
  int other_launches = 0;
  int jit_launches = 0;
  int plain_fallbacks = 0;     // applies of a tensor-core request run on the plain kernel
  bool plan_fallback = false;  // the current plan is such a fallback
  // error word of the last plan run on kernels with bounded waits (the pipelined plan
  // kernels), read by the next call that synchronises the stream; null when none is due
  int *err_pending = nullptr;
  // the last plan run on this handle (a circuit applied again reuses it and its device
  // copy: no planning, kernel-source hashing or upload)
  bool plan_valid = false;
  uint64_t plan_key = 0;
  svp::Plan plan;
  svp::Options plan_po;
  const svj::Module *plan_jit = nullptr;
  svk::DevPlanView plan_view{};
  // the norm sums (sum p, sum p^2) of the current state, computed by the last pass of a
  // plan-kernel run as it wrote the state: d_sums[0..1]; d_sums[2..] per-CTA partials.
  // Any other write of the state clears sums_valid; a state the caller can write
  // directly (created from its pointer, or exposed by sv_device_ptr) never sets it.
  double *d_sums = nullptr;
  bool sums_valid = false;
  bool user_writes = false;
};

namespace svj {
struct Module;
}

namespace svc {

// States of at least this many qubits run the plain path on plan-specialised kernels
// (sv_options.jit == 0): there a compile (about a second, once per circuit) is small
// against one run.
constexpr int kJitMinQubits = 24;

sv_status cuda_fail(cudaError_t e, const char *what);
sv_status ensure_device_buffer(void **buf, size_t *cap, size_t need);
svp::Options plan_options(const sv_options &o);
// The plan options sv_apply_circuit uses for an n-qubit state; *want_jit: the plain path
// is to run on plan-specialised kernels.
svp::Options apply_plan_options(const sv_options &o, int n, bool *want_jit);
sv_status check_options(const sv_options &o);
sv_status convert_gates(int n, const sv_gate *g, size_t count, bool inverse, std::vector<svp::Gate> *out);
sv_status upload_plan(sv_state *s, const svp::Plan &P, svk::DevPlanView *view);
sv_status run_plan(sv_state *s, const svp::Plan &P, const svk::DevPlanView &view, bool fused, bool f16 = false,
                   const svj::Module *jit = nullptr);
// Apply g to s on plan-specialised kernels whose last pass, instead of storing the state,
// sums <state | with> (conj(state) * with over all amplitudes) into out[0] (re), out[1]
// (im); s is left unusable (the last pass did not write it).  *fused = false (and s
// untouched) where these kernels are not in use for s's options or NVRTC is missing: the
// caller then applies and reduces separately.
sv_status apply_gates_inner(sv_state *s, const std::vector<svp::Gate> &g, const sv_state *with, double *out,
                            bool *fused);
// Plan and run an internal gate list (kinds may include K_PEQ) on the state.
sv_status apply_gates(sv_state *s, const std::vector<svp::Gate> &g);
sv_status set_device(sv_state *s);
// Write |0..0> if the state is still the never-written initial one.
sv_status materialize(sv_state *s);
// The autotuner's JSON cache (SV_AUTOTUNE_CACHE, default autotune.json beside the
// library): a flat object {"key": integer, ...}.
std::string autotune_cache_path();
std::map<std::string, int> read_autotune_cache();
void write_autotune_cache(const std::map<std::string, int> &c);

// The error word of a plan run whose kernels wait with a limit, if one is due: reads it
// (synchronising the stream) and returns SV_ERR_TIMEOUT (handle marked unusable) if a
// wait gave up, else SV_OK.
sv_status take_pending_error(sv_state *s);
// Fused path: the stage unitaries as split-TF32 operands (see k_fused.cu).
sv_status build_stage_mats(svp::Plan *P, const std::vector<svp::Gate> &g, int r, bool f16);
// A launch timed by CUDA events on the handle's stream when profiling is on (its entry of
// sv_get_launch_times carries `bytes`).
void profile_begin(sv_state *s);
void profile_end(sv_state *s, double bytes);

// B operands of a fused packed plan's matrix stages (the pipelined plan kernels).
sv_status build_stage_mats_packed(svp::Plan *P, const std::vector<svp::Gate> &g, bool f16);

}  // namespace svc

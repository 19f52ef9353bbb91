// C ABI: state handles, validation, planning, launches, readback, profiling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sv.h"
#include "capi_util.h"
#include "jit.h"
#include "kernels.h"
#include "plan.h"
#include "state.h"

std::string &svc::last_error() {
  thread_local std::string s;
  return s;
}

extern "C" const char *sv_last_error(void) { return svc::last_error().c_str(); }

namespace svc {

sv_status cuda_fail(cudaError_t e, const char *what) {
  last_error() = std::string(what) + ": " + cudaGetErrorString(e);
  return SV_ERR_CUDA;
}

sv_status ensure_device_buffer(void **buf, size_t *cap, size_t need) {
  if (*cap >= need) return SV_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  size_t want = std::max<size_t>(need, 4096);
  cudaError_t e = cudaMalloc(buf, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return fail(SV_ERR_OOM, "device scratch allocation failed");
  }
  *cap = want;
  return SV_OK;
}

svp::Options plan_options(const sv_options &o) {
  svp::Options p;
  // the interpreting and tensor-core kernels take up to 13-qubit tiles; 14 only with
  // tile_bits = 14 or for plan-specialised kernels (apply_gates).  The tensor-core kernel
  // defaults to 12 (three CTAs per SM; 34q F16x3 2.21 s against 2.49 s on 13)
  p.fused = o.precision == SV_PREC_TF32X3 || o.precision == SV_PREC_F16X3;
  p.m = o.tile_bits > 0 ? o.tile_bits : p.fused ? 12 : 13;
  p.c = o.low_bits > 0 ? o.low_bits : 4;
  p.pack = !p.fused;  // the plain kernel runs packed plans
  // register qubits per thread of the tile kernels (packed: besides qubit 0; tensor
  // cores: the block size, 5 or 4 qubits)
  p.rk = p.pack ? svk::tile_pass_register_slots() : (o.fuse_k == 4 ? 4 : 5);
  p.r = std::min(o.fuse_k > 0 ? o.fuse_k : p.rk, p.rk);
  return p;
}

svp::Options apply_plan_options(const sv_options &o, int n, bool *want_jit) {
  svp::Options po = plan_options(o);
  // tensor cores on the pipelined plan kernels (the default for 5-qubit blocks on
  // 12-qubit tiles): a fused packed plan -- stages of tile bit 0 and four register slots,
  // the TMA tile layout -- whose matrix stages the generated kernels run on tcgen05
  if (po.fused && n >= 12 && o.pipeline >= 0 && o.jit >= 0 && (o.fuse_k == 0 || o.fuse_k == 5) &&
      (o.tile_bits == 0 || o.tile_bits == 12) && (o.low_bits == 0 || o.low_bits == 4)) {
    po.pack = true;
    po.layout = 1;
    po.m = 12;
    po.c = 4;
    po.rk = 4;
    po.r = 4;
    *want_jit = true;
    return po;
  }
  // the tensor-core kernel takes 12- or 13-qubit tiles; smaller states use the plain one
  if (po.fused && std::min(po.m, n) < 12) {
    po.fused = false;
    po.pack = true;
    po.rk = svk::tile_pass_register_slots();
    po.r = std::min(po.r, po.rk);
  }
  // plain path: kernels compiled for the plan where they pay (or where asked for), on
  // 12-qubit tiles unless tile_bits says otherwise (they also take 14)
  *want_jit = !po.fused && o.jit >= 0 &&
              (o.jit == 1 || n >= kJitMinQubits || std::min(po.m, n) > svk::tile_pass_max_bits());
  if (*want_jit) {
    po.rk = svj::register_slots();
    po.r = std::min(po.r, po.rk);
    if (o.tile_bits == 0) po.m = svj::kTileBits;
    // the pipelined kernel reads tiles as 8-row TMA boxes (4 low qubits) into groups of
    // at least a warp: 10..13 tile qubits
    const int m = std::min(po.m, n);
    if (o.pipeline >= 0 && po.c == 4 && m >= 10 && m <= 13) po.layout = 1;
  }
  return po;
}

sv_status check_options(const sv_options &o) {
  if (o.precision != SV_PREC_PLAIN && o.precision != SV_PREC_TF32X3 && o.precision != SV_PREC_F16X3 &&
      o.precision != SV_PREC_PERGATE)
    return fail(SV_ERR_ARG, "options: unknown precision mode");
  if (o.fuse_k < 0 || o.fuse_k > svp::kMaxReg) return fail(SV_ERR_ARG, "options: fuse_k must be 0 or 1..5");
  if (o.tile_bits != 0 && (o.tile_bits < 6 || o.tile_bits > svp::kMaxTileBits))
    return fail(SV_ERR_ARG, "options: tile_bits must be 0 or 6..14");
  const bool fused = o.precision == SV_PREC_TF32X3 || o.precision == SV_PREC_F16X3;
  if (fused && o.fuse_k != 0 && o.fuse_k != 5 && o.fuse_k != 4)
    return fail(SV_ERR_ARG, "options: the tensor-core precisions apply 5- or 4-qubit blocks (fuse_k 0, 5 or 4)");
  if (fused && o.fuse_k == 4 && o.tile_bits != 0 && o.tile_bits != 12)
    return fail(SV_ERR_ARG, "options: 4-qubit tensor-core blocks take 12-qubit tiles");
  if (o.tile_bits == 14 && (fused || o.jit < 0))
    return fail(SV_ERR_ARG, "options: 14-qubit tiles need the plain path's plan-specialised kernels");
  if (o.low_bits < 0 || o.low_bits > 13) return fail(SV_ERR_ARG, "options: low_bits must be 0..13");
  if (o.jit < -1 || o.jit > 1) return fail(SV_ERR_ARG, "options: jit must be -1, 0 or 1");
  if (o.pipeline < -1 || o.pipeline > 0) return fail(SV_ERR_ARG, "options: pipeline must be -1 or 0");
  if (o.norm_restore < -1 || o.norm_restore > 0) return fail(SV_ERR_ARG, "options: norm_restore must be -1 or 0");
  const int m = o.tile_bits > 0 ? o.tile_bits : 13;
  const int c = o.low_bits > 0 ? o.low_bits : 4;
  if (c > m || m - c > 10) return fail(SV_ERR_ARG, "options: need low_bits <= tile_bits <= low_bits + 10");
  return SV_OK;
}

sv_status convert_gates(int n, const sv_gate *g, size_t count, bool inverse, std::vector<svp::Gate> *out) {
  out->clear();
  out->reserve(count);
  if (count && !g) return fail(SV_ERR_ARG, "gate list is NULL");
  for (size_t s = 0; s < count; ++s) {
    const sv_gate &x = g[inverse ? count - 1 - s : s];
    if (x.kind > SV_SYDG) return failf(SV_ERR_ARG, "gate %s%lld: unknown kind", "#", (long long)s);
    if (x.q0 >= n) return failf(SV_ERR_ARG, "gate %s%lld: qubit out of range", "#", (long long)s);
    uint8_t k = x.kind;
    if (k == SV_CZ && (x.q1 >= n || x.q1 == x.q0))
      return failf(SV_ERR_ARG, "gate %s%lld: CZ needs two distinct qubits < n", "#", (long long)s);
    if (inverse) {
      if (k == SV_T) k = SV_TDG;
      else if (k == SV_TDG) k = SV_T;
      else if (k == SV_SX) k = SV_SXDG;
      else if (k == SV_SXDG) k = SV_SX;
      else if (k == SV_SY) k = SV_SYDG;
      else if (k == SV_SYDG) k = SV_SY;
    }
    out->push_back(svp::Gate{k, x.q0, (uint8_t)(k == SV_CZ ? x.q1 : 0)});
  }
  return SV_OK;
}

}  // namespace svc

using namespace svc;

// ---------------------------------------------------------------------------------------

namespace svc {

sv_status take_pending_error(sv_state *s) {
  if (!s->err_pending) return SV_OK;
  int h_err = 0;
  cudaError_t e = cudaMemcpyAsync(&h_err, s->err_pending, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  s->err_pending = nullptr;
  if (e != cudaSuccess) {
    s->broken = true;
    s->plan_valid = false;
    return cuda_fail(e, "tile pass");
  }
  if (h_err != 0) {
    s->broken = true;
    s->plan_valid = false;
    return fail(SV_ERR_TIMEOUT, "tile pass: a bounded wait gave up (state undefined)");
  }
  return SV_OK;
}

sv_status set_device(sv_state *s) {
  cudaError_t e = cudaSetDevice(s->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return SV_OK;
}

sv_status materialize(sv_state *s) {
  if (!s->fresh) return SV_OK;
  cudaError_t e = svk::launch_init(s->psi, s->n, false, 1.0f, s->stream);
  if (e != cudaSuccess) { s->broken = true; return cuda_fail(e, "init kernel"); }
  s->fresh = false;
  return SV_OK;
}

}  // namespace svc

namespace {

void prof_begin(sv_state *s) {
  if (!s->prof) return;
  if (s->ev_used + 2 > s->events.size()) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    s->events.push_back(a);
    s->events.push_back(b);
  }
  cudaEventRecord(s->events[s->ev_used], s->stream);
}

void prof_end(sv_state *s, double bytes) {
  if (!s->prof) return;
  cudaEventRecord(s->events[s->ev_used + 1], s->stream);
  s->ev_bytes.push_back(bytes);
  s->ev_used += 2;
}

}  // namespace

namespace svc {
void profile_begin(sv_state *s) { prof_begin(s); }
void profile_end(sv_state *s, double bytes) { prof_end(s, bytes); }
}  // namespace svc

namespace {

// one full sweep per gate (precision SV_PREC_PERGATE and tiny states)
sv_status apply_pergate(sv_state *s, const std::vector<svp::Gate> &g) {
  size_t start = 0;
  const double amps = std::ldexp(1.0, s->n);
  if (s->fresh) {
    uint64_t seen = 0;
    size_t i = 0;
    while (i < g.size() && g[i].kind == svp::K_H && !(seen & (1ull << g[i].q0)) &&
           __builtin_popcountll(seen) < s->n) {
      seen |= 1ull << g[i].q0;
      ++i;
    }
    const bool uniform = __builtin_popcountll(seen) == s->n;
    if (uniform) start = i;
    prof_begin(s);
    cudaError_t e = svk::launch_init(s->psi, s->n, uniform, (float)std::pow(2.0, -0.5 * s->n), s->stream);
    prof_end(s, 8.0 * amps);
    if (e != cudaSuccess) { s->broken = true; return cuda_fail(e, "init kernel"); }
    s->fresh = false;
  }
  const float c = (float)(1.0 / std::sqrt(2.0));
  for (size_t i = start; i < g.size(); ++i) {
    const svp::Gate &x = g[i];
    cudaError_t e = cudaSuccess;
    const uint64_t b0 = 1ull << x.q0, b1 = 1ull << x.q1;
    double bytes = 16.0 * amps;
    prof_begin(s);
    switch (x.kind) {
      case svp::K_T: e = svk::launch_gate_diag(s->psi, s->n, b0, b0, c, c, s->stream); bytes = 8.0 * amps; break;
      case svp::K_TDG: e = svk::launch_gate_diag(s->psi, s->n, b0, b0, c, -c, s->stream); bytes = 8.0 * amps; break;
      case svp::K_Z: e = svk::launch_gate_diag(s->psi, s->n, b0, b0, -1.f, 0.f, s->stream); bytes = 8.0 * amps; break;
      case svp::K_P0: e = svk::launch_gate_diag(s->psi, s->n, b0, b0, 0.f, 0.f, s->stream); bytes = 8.0 * amps; break;
      case svp::K_P1: e = svk::launch_gate_diag(s->psi, s->n, b0, 0, 0.f, 0.f, s->stream); bytes = 8.0 * amps; break;
      case svp::K_CZ: e = svk::launch_gate_diag(s->psi, s->n, b0 | b1, b0 | b1, -1.f, 0.f, s->stream); bytes = 4.0 * amps; break;
      case svp::K_PEQ:
        e = svk::launch_gate_diag(s->psi, s->n, b0 | b1, b0, 0.f, 0.f, s->stream);
        if (e == cudaSuccess) e = svk::launch_gate_diag(s->psi, s->n, b0 | b1, b1, 0.f, 0.f, s->stream);
        bytes = 8.0 * amps;
        break;
      default: {
        double m[8];
        svp::kind_matrix(x.kind, m);
        svk::Mat2 u;
        for (int k = 0; k < 8; ++k) u.v[k] = (float)m[k];
        e = svk::launch_gate_1q(s->psi, s->n, x.q0, u, s->stream);
      }
    }
    prof_end(s, bytes);
    if (e != cudaSuccess) { s->broken = true; return cuda_fail(e, "per-gate kernel"); }
  }
  return SV_OK;
}

}  // namespace

namespace svc {

sv_status upload_plan(sv_state *s, const svp::Plan &P, svk::DevPlanView *view) {
  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_pass = 0;
  const size_t o_stage = align(o_pass + P.passes.size() * sizeof(svp::DevPass));
  const size_t o_op = align(o_stage + P.stages.size() * sizeof(svp::DevStage));
  const size_t o_mat = align(o_op + P.ops.size() * sizeof(svp::DevOp));
  const size_t o_gt = align(o_mat + P.mats.size() * sizeof(float));
  const size_t o_err = align(o_gt + P.gtab.size() * sizeof(svp::DevGroupEntry));
  const size_t total = o_err + 256;
  sv_status st = ensure_device_buffer(&s->d_plan, &s->d_plan_cap, total);
  if (st != SV_OK) return st;
  s->h_plan.assign(total, 0);
  if (!P.passes.empty()) std::memcpy(&s->h_plan[o_pass], P.passes.data(), P.passes.size() * sizeof(svp::DevPass));
  if (!P.stages.empty()) std::memcpy(&s->h_plan[o_stage], P.stages.data(), P.stages.size() * sizeof(svp::DevStage));
  if (!P.ops.empty()) std::memcpy(&s->h_plan[o_op], P.ops.data(), P.ops.size() * sizeof(svp::DevOp));
  if (!P.mats.empty()) std::memcpy(&s->h_plan[o_mat], P.mats.data(), P.mats.size() * sizeof(float));
  if (!P.gtab.empty())
    std::memcpy(&s->h_plan[o_gt], P.gtab.data(), P.gtab.size() * sizeof(svp::DevGroupEntry));
  cudaError_t e = cudaMemcpyAsync(s->d_plan, s->h_plan.data(), total, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "plan upload");
  if (s->prof) s->h2d += (double)total;
  char *d = static_cast<char *>(s->d_plan);
  view->passes = reinterpret_cast<const svp::DevPass *>(d + o_pass);
  view->stages = reinterpret_cast<const svp::DevStage *>(d + o_stage);
  view->ops = reinterpret_cast<const svp::DevOp *>(d + o_op);
  view->mats = reinterpret_cast<const float *>(d + o_mat);
  view->err = reinterpret_cast<int *>(d + o_err);
  view->gtab = reinterpret_cast<const svp::DevGroupEntry *>(d + o_gt);
  return SV_OK;
}

sv_status run_plan(sv_state *s, const svp::Plan &P, const svk::DevPlanView &view, bool fused, bool f16,
                   const svj::Module *jit) {
  const double amps = std::ldexp(1.0, s->n);
  s->sums_valid = false;
  if (s->prof && s->plan_fallback) s->plain_fallbacks += 1;
  // plan kernels: the last pass also sums p and p^2 of the state it writes (no separate
  // read of the state for sv_norm)
  const bool sums = jit && s->owns && !s->user_writes && !P.passes.empty();
  if (sums && !s->d_sums) {
    if (cudaMalloc(&s->d_sums, (2 + 2 * (size_t)svj::max_pass_grid()) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      s->d_sums = nullptr;
      return fail(SV_ERR_OOM, "norm sums buffer allocation failed");
    }
  }
  unsigned grid = 0;
  for (size_t p = 0; p < P.passes.size(); ++p) {
    const svp::DevPass &hp = P.passes[p];
    const double bytes = (hp.flags & (svp::PF_INIT_UNIFORM | svp::PF_INIT_ZERO)) ? 8.0 * amps : 16.0 * amps;
    double *partials = sums && p + 1 == P.passes.size() ? s->d_sums + 2 : nullptr;
    prof_begin(s);
    cudaError_t e = fused ? svk::launch_fused_pass(s->psi, s->n, view, (int)p, hp, s->stream, f16, P.rk)
                    : jit ? svj::launch_pass(jit, s->psi, s->n, view, (int)p, hp, s->stream, partials, &grid)
                          : svk::launch_tile_pass(s->psi, s->n, view, (int)p, hp, s->stream);
    prof_end(s, bytes);
    if (jit && s->prof) s->jit_launches += 1;
    if (e != cudaSuccess) { s->broken = true; return cuda_fail(e, "tile pass kernel"); }
  }
  if (jit)
    for (size_t p = 0; p < P.passes.size(); ++p)
      if (svj::pass_is_pipelined(P, (int)p)) s->err_pending = view.err;
  if (sums) {
    const cudaError_t e = svk::launch_norm_final(s->d_sums + 2, (int)grid, s->d_sums, s->stream);
    if (e != cudaSuccess) { s->broken = true; return cuda_fail(e, "norm sums"); }
    if (s->prof) s->other_launches += 1;
    s->sums_valid = true;
  }
  return SV_OK;
}


}  // namespace svc

namespace svc {

// A fused pass whose bounded wait gave up leaves a non-zero error word in the plan.
sv_status check_fused_error(sv_state *s, const svk::DevPlanView &view) {
  int h_err = 0;
  cudaError_t e = cudaMemcpyAsync(&h_err, view.err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    s->broken = true;
    s->plan_valid = false;
    return cuda_fail(e, "fused pass");
  }
  if (h_err != 0) {
    s->broken = true;
    s->plan_valid = false;
    return fail(SV_ERR_TIMEOUT, "fused pass: a tensor-core wait gave up (state undefined)");
  }
  return SV_OK;
}

// ---- autotuning of the plain path on plan-specialised kernels ------------------------
// (sv_options.autotune = 1, a fresh state, the pipelined kernels): the tile size (12 or 13
// qubits), the fusion width (stages of 5 or 6 qubits: 4 or 5 register slots besides the
// pack bit) and, per pass, the pipelined kernel's compute groups (3, 2 or 1 on six slots,
// or 4 on four, on 12-qubit tiles) are picked by timing this circuit -- whole runs of each
// candidate plan, CUDA events around every pass launch -- and the choice is kept in the
// JSON cache under "<device>|circuit|<n>|<hash of the gate list and options>" (entries
// |m, |k (qubits per stage), |passes and |p<i>).

namespace {

struct PlainTune {
  int m = 0;
  int kpr = 0;  // register slots besides the pack bit: stages of kpr + 1 qubits (the fusion width)
  std::vector<uint8_t> groups;
};

std::string circuit_tune_key(const sv_state *s, const std::vector<svp::Gate> &g, const svp::Options &po) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, s->device);
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](const void *p, size_t len) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < len; ++i) h = (h ^ b[i]) * 1099511628211ull;
  };
  const int head[4] = {s->n, po.rk, po.r, po.c};
  mix(head, sizeof(head));
  if (!g.empty()) mix(g.data(), g.size() * sizeof(svp::Gate));
  char buf[sizeof(prop.name) + 64];
  std::snprintf(buf, sizeof(buf), "%s|circuit|%d|%016llx", prop.name, s->n, (unsigned long long)h);
  for (char *p = buf; *p; ++p)
    if (*p == '"' || *p == '\\') *p = '_';
  return buf;
}

// Two runs of the plan (the first warms the kernels); per-pass device times of the second.
sv_status time_plan(sv_state *s, const svp::Plan &P, const svk::DevPlanView &view, const svj::Module *jit,
                    std::vector<float> *ms) {
  const size_t np = P.passes.size();
  std::vector<cudaEvent_t> ev(2 * np);
  for (cudaEvent_t &e : ev) cudaEventCreate(&e);
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep)
    for (size_t p = 0; p < np && e == cudaSuccess; ++p) {
      if (rep) cudaEventRecord(ev[2 * p], s->stream);
      e = svj::launch_pass(jit, s->psi, s->n, view, (int)p, P.passes[p], s->stream);
      if (rep) cudaEventRecord(ev[2 * p + 1], s->stream);
    }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  ms->assign(np, 0.f);
  for (size_t p = 0; p < np && e == cudaSuccess; ++p) e = cudaEventElapsedTime(&(*ms)[p], ev[2 * p], ev[2 * p + 1]);
  for (cudaEvent_t &x : ev) cudaEventDestroy(x);
  if (e != cudaSuccess) return cuda_fail(e, "autotune run");
  s->err_pending = view.err;
  return take_pending_error(s);
}

sv_status autotune_plain(sv_state *s, const std::vector<svp::Gate> &g, const svp::Options &base, PlainTune *out) {
  const std::string key = circuit_tune_key(s, g, base);
  std::map<std::string, int> cache = read_autotune_cache();
  auto m_it = cache.find(key + "|m"), np_it = cache.find(key + "|passes"), k_it = cache.find(key + "|k");
  if (m_it != cache.end() && np_it != cache.end() && k_it != cache.end()) {
    out->m = m_it->second;
    out->kpr = k_it->second - 1;
    out->groups.assign((size_t)np_it->second, 0);
    for (size_t p = 0; p < out->groups.size(); ++p) {
      auto it = cache.find(key + "|p" + std::to_string(p));
      out->groups[p] = it == cache.end() ? 0 : (uint8_t)it->second;
    }
    return SV_OK;
  }
  double best_total = 1e300;
  // candidates: (tile qubits, register slots) -- 12- and 13-qubit tiles with stages of
  // five qubits, 12-qubit tiles with stages of six (64 amplitudes a thread)
  const int cand[3][2] = {{12, 4}, {13, 4}, {12, 5}};
  for (const auto &c : cand) {
    const int m = c[0], kpr = c[1];
    if (m > s->n) continue;
    svp::Options po = base;
    po.m = m;
    po.rk = kpr;
    if (s->opts.fuse_k == 0) po.r = kpr;
    svp::Plan P;
    const char *err = nullptr;
    if (!svp::build_plan(s->n, g, po, true, &P, &err)) return fail(SV_ERR_ARG, err ? err : "planning failed");
    const size_t np = P.passes.size();
    std::vector<float> best(np, 1e30f);
    std::vector<uint8_t> best_g(np, 0);
    // (34 qubits, fixed shapes: four groups ran the write-only first pass in 61 ms against
    // 64 ms with three, and the read-write passes up to 15 ms slower; one group, all six
    // slots, ran the last pass (few gates) in 43.6 ms against 45.8 ms)
    for (int groups : (m == 12 ? std::vector<int>{3, 2, 4, 1} : std::vector<int>{1})) {
      P.pipe_groups.assign(np, (uint8_t)groups);
      std::string jerr;
      const svj::Module *M = svj::get_module(P, po.rk, &jerr);
      if (!M) return fail(SV_ERR_CUDA, jerr.c_str());
      svk::DevPlanView view;
      sv_status st = upload_plan(s, P, &view);
      if (st != SV_OK) return st;
      std::vector<float> ms;
      if ((st = time_plan(s, P, view, M, &ms)) != SV_OK) return st;
      for (size_t p = 0; p < np; ++p)
        if (ms[p] < best[p]) { best[p] = ms[p]; best_g[p] = (uint8_t)groups; }
    }
    double total = 0;
    for (float x : best) total += x;
    // a later candidate has to win by more than the timing noise (1.5 %), so that near
    // ties keep the first one (12-qubit tiles, 5-qubit stages) from run to run
    if (total < best_total * (out->m ? 0.985 : 1.0)) {
      best_total = total;
      out->m = m;
      out->kpr = kpr;
      out->groups = best_g;
    }
  }
  if (out->m == 0) return fail(SV_ERR_ARG, "autotune: no candidate tile size");
  cache[key + "|m"] = out->m;
  cache[key + "|k"] = out->kpr + 1;
  cache[key + "|passes"] = (int)out->groups.size();
  for (size_t p = 0; p < out->groups.size(); ++p) cache[key + "|p" + std::to_string(p)] = out->groups[p];
  write_autotune_cache(cache);
  return SV_OK;
}

}  // namespace

sv_status apply_gates(sv_state *s, const std::vector<svp::Gate> &g) {
  sv_status st;
  if ((st = set_device(s)) != SV_OK) return st;
  s->sums_valid = false;
  if (s->opts.precision == SV_PREC_PERGATE || s->n < 6) {
    // (a tensor-core request on a state this small is a plain fallback too)
    if (s->prof && (s->opts.precision == SV_PREC_TF32X3 || s->opts.precision == SV_PREC_F16X3)) s->plain_fallbacks += 1;
    return apply_pergate(s, g);
  }
  if ((s->opts.precision == SV_PREC_TF32X3 || s->opts.precision == SV_PREC_F16X3) && !svk::fused_supported())
    return fail(SV_ERR_CUDA, "fused tensor-core path needs an sm_103a device");
  if (g.empty() && !s->fresh) return SV_OK;
  // the same gate list, options and starting condition as the last call: reuse its plan
  uint64_t key = 1469598103934665603ull;
  auto mix = [&key](const void *p, size_t len) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < len; ++i) key = (key ^ b[i]) * 1099511628211ull;
  };
  const int head[10] = {s->n, s->fresh ? 1 : 0, s->opts.precision, s->opts.fuse_k, s->opts.tile_bits,
                        s->opts.low_bits, s->opts.jit, s->opts.pipeline, s->opts.norm_restore, s->opts.autotune};
  mix(head, sizeof(head));
  if (!g.empty()) mix(g.data(), g.size() * sizeof(svp::Gate));
  if (s->plan_valid && s->plan_key == key) {
    const bool f16 = s->opts.precision == SV_PREC_F16X3;
    const bool kfused = s->plan_po.fused && !s->plan_jit;  // the tensor-core tile kernel
    if ((st = run_plan(s, s->plan, s->plan_view, kfused, f16, s->plan_jit)) != SV_OK) {
      s->plan_valid = false;
      return st;
    }
    s->fresh = false;
    return kfused ? check_fused_error(s, s->plan_view) : SV_OK;
  }
  s->plan_valid = false;
  svp::Plan P;
  const char *err = nullptr;
  bool want_jit = false;
  svp::Options po = apply_plan_options(s->opts, s->n, &want_jit);
  PlainTune tune;
  if (s->opts.autotune == 1 && want_jit && !po.fused && po.layout == 1 && s->fresh && s->opts.tile_bits == 0) {
    if ((st = autotune_plain(s, g, po, &tune)) != SV_OK) return st;
    po.m = tune.m;
    po.rk = tune.kpr;
    if (s->opts.fuse_k == 0) po.r = tune.kpr;
  }
  if (!svp::build_plan(s->n, g, po, s->fresh, &P, &err)) return fail(SV_ERR_ARG, err ? err : "planning failed");
  if (tune.m && tune.groups.size() == P.passes.size()) P.pipe_groups = tune.groups;
  // a tensor-core request on a state (or tile) below 12 qubits runs the plain kernel
  s->plan_fallback = (s->opts.precision == SV_PREC_TF32X3 || s->opts.precision == SV_PREC_F16X3) && !po.fused;
  const svj::Module *jit = nullptr;
  const bool f16 = s->opts.precision == SV_PREC_F16X3;
  if (want_jit) {
    if (po.fused) {  // matrix stages of the plan kernels: their B operands (and the
      // norm restore choice, which the generated code bakes in)
      P.mma = f16 ? 1 : 2;
      if ((st = build_stage_mats_packed(&P, g, f16)) != SV_OK) return st;
      if (s->opts.norm_restore < 0)
        for (svp::DevPass &dp : P.passes) dp.flags |= svp::PF_RAW;
    }
    std::string jerr;
    jit = svj::get_module(P, po.rk, &jerr);
    if (!jit && s->opts.jit == 1) return fail(SV_ERR_CUDA, jerr.c_str());
    if (!jit && po.fused) {
      // no compiler: the tensor-core tile kernel with its own plan
      sv_options o = s->opts;
      o.pipeline = -1;
      bool unused = false;
      po = apply_plan_options(o, s->n, &unused);
      P = svp::Plan();
      if (!svp::build_plan(s->n, g, po, s->fresh, &P, &err))
        return fail(SV_ERR_ARG, err ? err : "planning failed");
    } else if (!jit) {
      // no compiler: the interpreting kernel, with its register width, on tiles it takes
      po.m = std::min(po.m, svk::tile_pass_max_bits());
      po.layout = 0;
      po.rk = svk::tile_pass_register_slots();
      po.r = std::min(plan_options(s->opts).r, po.rk);
      P = svp::Plan();
      if (!svp::build_plan(s->n, g, po, s->fresh, &P, &err))
        return fail(SV_ERR_ARG, err ? err : "planning failed");
    }
  }
  const bool kfused = po.fused && !jit;  // the tensor-core tile kernel
  if (kfused && (st = build_stage_mats(&P, g, std::min(po.r, std::min(po.m, s->n)), f16)) != SV_OK) return st;
  if (kfused && s->opts.norm_restore < 0)
    for (svp::DevPass &dp : P.passes) dp.flags |= svp::PF_RAW;
  if (kfused)
    for (const svp::DevPass &dp : P.passes)
      if (dp.stage_count > 256) return fail(SV_ERR_ARG, "fused path: more than 256 stages in one pass");
  svk::DevPlanView view;
  if ((st = upload_plan(s, P, &view)) != SV_OK) return st;
  if ((st = run_plan(s, P, view, kfused, f16, jit)) != SV_OK) return st;
  s->fresh = false;
  if (kfused && (st = check_fused_error(s, view)) != SV_OK) return st;
  s->plan = std::move(P);
  s->plan_po = po;
  s->plan_jit = jit;
  s->plan_view = view;
  s->plan_key = key;
  s->plan_valid = true;
  return SV_OK;
}

sv_status apply_gates_inner(sv_state *s, const std::vector<svp::Gate> &g, const sv_state *with, double *out,
                            bool *fused) {
  *fused = false;
  sv_status st;
  if ((st = set_device(s)) != SV_OK) return st;
  if (s->opts.precision != SV_PREC_PLAIN || s->n < 6 || g.empty() || s->fresh || s->broken || !s->owns)
    return SV_OK;
  bool want_jit = false;
  svp::Options po = apply_plan_options(s->opts, s->n, &want_jit);
  if (!want_jit || po.fused) return SV_OK;
  s->sums_valid = false;
  uint64_t key = 1469598103934665603ull ^ 0x696e6e6572ull;  // distinct from apply_gates' keys
  auto mix = [&key](const void *p, size_t len) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < len; ++i) key = (key ^ b[i]) * 1099511628211ull;
  };
  const int head[7] = {s->n, s->opts.precision, s->opts.fuse_k, s->opts.tile_bits, s->opts.low_bits, s->opts.jit,
                       s->opts.pipeline};
  mix(head, sizeof(head));
  mix(g.data(), g.size() * sizeof(svp::Gate));
  if (!(s->plan_valid && s->plan_key == key)) {
    s->plan_valid = false;
    svp::Plan P;
    const char *err = nullptr;
    if (!svp::build_plan(s->n, g, po, false, &P, &err)) return fail(SV_ERR_ARG, err ? err : "planning failed");
    std::string jerr;
    const svj::Module *M = svj::get_module(P, po.rk, &jerr, true);
    if (!M) return SV_OK;  // no compiler: the caller applies and reduces separately
    svk::DevPlanView view;
    if ((st = upload_plan(s, P, &view)) != SV_OK) return st;
    s->plan = std::move(P);
    s->plan_po = po;
    s->plan_jit = M;
    s->plan_view = view;
    s->plan_key = key;
    s->plan_valid = true;
  }
  if (!s->d_sums) {
    if (cudaMalloc(&s->d_sums, (2 + 2 * (size_t)svj::max_pass_grid()) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      s->d_sums = nullptr;
      return fail(SV_ERR_OOM, "sums buffer allocation failed");
    }
  }
  // the other state's pending work first (the handles may use different streams)
  cudaError_t e = with->stream == s->stream ? cudaSuccess : cudaStreamSynchronize(with->stream);
  const svp::Plan &P = s->plan;
  const double amps = std::ldexp(1.0, s->n);
  unsigned grid = 0;
  for (size_t p = 0; e == cudaSuccess && p < P.passes.size(); ++p) {
    const bool last = p + 1 == P.passes.size();
    prof_begin(s);
    e = svj::launch_pass(s->plan_jit, s->psi, s->n, s->plan_view, (int)p, P.passes[p], s->stream,
                         last ? s->d_sums + 2 : nullptr, last ? &grid : nullptr, last ? with->psi : nullptr);
    prof_end(s, 16.0 * amps);  // last pass: reads this state and the other
    if (s->prof) s->jit_launches += 1;
  }
  double h[2] = {0, 0};
  if (e == cudaSuccess) e = svk::launch_norm_final(s->d_sums + 2, (int)grid, s->d_sums, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, s->d_sums, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    s->broken = true;
    return cuda_fail(e, "inner product pass");
  }
  for (size_t p = 0; p < P.passes.size(); ++p)
    if (svj::pass_is_pipelined(P, (int)p)) s->err_pending = s->plan_view.err;
  const sv_status werr = take_pending_error(s);
  // the last pass did not store: the state is not the circuit's result
  s->broken = true;
  if (werr != SV_OK) return werr;
  if (s->prof) {
    s->other_launches += 1;
    s->d2h += sizeof(h);
  }
  out[0] = h[0];
  out[1] = h[1];
  *fused = true;
  return SV_OK;
}

}  // namespace svc

static sv_status apply_impl(sv_state *s, const sv_gate *gates, size_t n_gates, bool inverse) {
  clear_error();
  if (!s) return fail(SV_ERR_ARG, "null state");
  if (s->broken) return fail(SV_ERR_STATE, "state is unusable after an earlier failure");
  std::vector<svp::Gate> g;
  sv_status st = convert_gates(s->n, gates, n_gates, inverse, &g);
  if (st != SV_OK) return st;
  return apply_gates(s, g);
}

extern "C" {

sv_status sv_create(int n_qubits, const sv_options *opts, sv_state **out) {
  clear_error();
  if (!out) return fail(SV_ERR_ARG, "sv_create: out is NULL");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > 34) return fail(SV_ERR_ARG, "sv_create: n_qubits must be 1..34");
  sv_options o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  sv_status st = check_options(o);
  if (st != SV_OK) return st;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "sv_create: no CUDA device");
  void *p = nullptr;
  e = cudaMalloc(&p, sizeof(float2) << n_qubits);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SV_ERR_OOM, "sv_create: cudaMalloc of the state failed");
  }
  sv_state *s = new sv_state();
  s->n = n_qubits;
  s->psi = static_cast<float2 *>(p);
  s->owns = true;
  s->opts = o;
  s->stream = static_cast<cudaStream_t>(o.stream);
  s->device = dev;
  s->fresh = true;
  *out = s;
  return SV_OK;
}

sv_status sv_create_from_ptr(int n_qubits, void *dev_ptr, void *stream, sv_state **out) {
  clear_error();
  if (!out || !dev_ptr) return fail(SV_ERR_ARG, "sv_create_from_ptr: NULL argument");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > 34) return fail(SV_ERR_ARG, "sv_create_from_ptr: n_qubits must be 1..34");
  if ((reinterpret_cast<uintptr_t>(dev_ptr) & 15) != 0)
    return fail(SV_ERR_ARG, "sv_create_from_ptr: buffer must be 16-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "sv_create_from_ptr: no CUDA device");
  sv_state *s = new sv_state();
  s->n = n_qubits;
  s->psi = static_cast<float2 *>(dev_ptr);
  s->owns = false;
  std::memset(&s->opts, 0, sizeof(s->opts));
  s->opts.stream = stream;
  s->stream = static_cast<cudaStream_t>(stream);
  s->device = dev;
  s->fresh = false;
  *out = s;
  return SV_OK;
}

sv_status sv_destroy(sv_state *s) {
  clear_error();
  if (!s) return SV_OK;
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  if (s->owns && s->psi) cudaFree(s->psi);
  if (s->d_plan) cudaFree(s->d_plan);
  if (s->d_scratch) cudaFree(s->d_scratch);
  if (s->d_sums) cudaFree(s->d_sums);
  for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
  delete s;
  return SV_OK;
}

sv_status sv_set_options(sv_state *s, const sv_options *opts) {
  clear_error();
  if (!s || !opts) return fail(SV_ERR_ARG, "sv_set_options: NULL argument");
  sv_status st = check_options(*opts);
  if (st != SV_OK) return st;
  s->opts = *opts;
  s->stream = static_cast<cudaStream_t>(opts->stream);
  return SV_OK;
}

sv_status sv_reset(sv_state *s) {
  clear_error();
  if (!s) return fail(SV_ERR_ARG, "sv_reset: NULL state");
  s->fresh = true;
  s->sums_valid = false;
  s->broken = false;
  return SV_OK;
}

sv_status sv_device_ptr(sv_state *s, void **ptr) {
  clear_error();
  if (!s || !ptr) return fail(SV_ERR_ARG, "sv_device_ptr: NULL argument");
  sv_status st = set_device(s);
  if (st != SV_OK) return st;
  if ((st = materialize(s)) != SV_OK) return st;
  *ptr = s->psi;
  s->user_writes = true;  // the caller may write the state from now on
  s->sums_valid = false;
  return SV_OK;
}

sv_status sv_copy_state(sv_state *s, void *dst) {
  clear_error();
  if (!s || !dst) return fail(SV_ERR_ARG, "sv_copy_state: NULL argument");
  if (s->broken) return fail(SV_ERR_STATE, "state is unusable after an earlier failure");
  sv_status st = set_device(s);
  if (st != SV_OK) return st;
  if ((st = take_pending_error(s)) != SV_OK) return st;
  if ((st = materialize(s)) != SV_OK) return st;
  cudaError_t e = cudaMemcpyAsync(dst, s->psi, sizeof(float2) << s->n, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sv_copy_state");
  return SV_OK;
}

sv_status sv_load_state(sv_state *s, const void *src) {
  clear_error();
  if (!s || !src) return fail(SV_ERR_ARG, "sv_load_state: NULL argument");
  sv_status st = set_device(s);
  if (st != SV_OK) return st;
  s->sums_valid = false;
  cudaError_t e = cudaMemcpyAsync(s->psi, src, sizeof(float2) << s->n, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sv_load_state");
  s->fresh = false;
  s->broken = false;
  return SV_OK;
}

sv_status sv_apply_circuit(sv_state *s, const sv_gate *gates, size_t n_gates) {
  return apply_impl(s, gates, n_gates, false);
}

sv_status sv_apply_circuit_inverse(sv_state *s, const sv_gate *gates, size_t n_gates) {
  return apply_impl(s, gates, n_gates, true);
}

static sv_status gather_common(sv_state *s, const uint64_t *bits, size_t m, double *out, bool prob) {
  clear_error();
  if (!s || (m && (!bits || !out))) return fail(SV_ERR_ARG, "NULL argument");
  if (s->broken) return fail(SV_ERR_STATE, "state is unusable after an earlier failure");
  for (size_t j = 0; j < m; ++j)
    if (s->n < 64 && (bits[j] >> s->n)) return failf(SV_ERR_ARG, "bitstring %s%lld has bits >= n", "#", (long long)j);
  if (m == 0) return SV_OK;
  sv_status st = set_device(s);
  if (st != SV_OK) return st;
  if ((st = take_pending_error(s)) != SV_OK) return st;
  if ((st = materialize(s)) != SV_OK) return st;
  const size_t need = m * sizeof(uint64_t) + 2 * m * sizeof(double) + 512;
  if ((st = ensure_device_buffer(&s->d_scratch, &s->d_scratch_cap, need)) != SV_OK) return st;
  uint64_t *d_bits = static_cast<uint64_t *>(s->d_scratch);
  double *d_out = reinterpret_cast<double *>(static_cast<char *>(s->d_scratch) + ((m * sizeof(uint64_t) + 255) & ~(size_t)255));
  cudaError_t e = cudaMemcpyAsync(d_bits, bits, m * sizeof(uint64_t), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess)
    e = prob ? svk::launch_gather_prob(s->psi, d_bits, (int64_t)m, d_out, s->stream)
             : svk::launch_gather(s->psi, d_bits, (int64_t)m, d_out, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, d_out, (prob ? 1 : 2) * m * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "amplitude gather");
  if (s->prof) {
    s->h2d += (double)(m * sizeof(uint64_t));
    s->d2h += (double)((prob ? 1 : 2) * m * sizeof(double));
    s->other_launches += 1;
  }
  return SV_OK;
}

sv_status sv_get_amplitudes(sv_state *s, const uint64_t *bits, size_t m, double *out_re_im) {
  return gather_common(s, bits, m, out_re_im, false);
}

sv_status sv_get_probabilities(sv_state *s, const uint64_t *bits, size_t m, double *out) {
  return gather_common(s, bits, m, out, true);
}

sv_status sv_norm(sv_state *s, double *norm2, double *sum_p2) {
  clear_error();
  if (!s) return fail(SV_ERR_ARG, "sv_norm: NULL state");
  if (s->broken) return fail(SV_ERR_STATE, "state is unusable after an earlier failure");
  sv_status st = set_device(s);
  if (st != SV_OK) return st;
  if ((st = take_pending_error(s)) != SV_OK) return st;
  if ((st = materialize(s)) != SV_OK) return st;
  if (s->sums_valid) {
    // summed by the last pass that wrote the state
    double h[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(h, s->d_sums, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sv_norm");
    if (s->prof) s->d2h += sizeof(h);
    if (norm2) *norm2 = h[0];
    if (sum_p2) *sum_p2 = h[1];
    return SV_OK;
  }
  const size_t need = (size_t)(svk::reduce_partials_needed() + 2) * 2 * sizeof(double);
  if ((st = ensure_device_buffer(&s->d_scratch, &s->d_scratch_cap, need)) != SV_OK) return st;
  double *partials = static_cast<double *>(s->d_scratch);
  double *res = partials + 2 * svk::reduce_partials_needed();
  double h[2] = {0, 0};
  cudaError_t e = svk::launch_norm(s->psi, s->n, partials, res, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sv_norm");
  if (s->prof) {
    s->d2h += sizeof(h);
    s->other_launches += s->n < 2 ? 1 : 2;
  }
  if (norm2) *norm2 = h[0];
  if (sum_p2) *sum_p2 = h[1];
  return SV_OK;
}

sv_status sv_plan(int n_qubits, const sv_gate *gates, size_t n_gates, const sv_options *opts, int fresh_state,
                  sv_plan_summary *summary, int32_t *order_out, int32_t *pass_out, int32_t *tile_out,
                  size_t tile_cap) {
  clear_error();
  if (n_qubits < 1 || n_qubits > 64) return fail(SV_ERR_ARG, "sv_plan: n_qubits must be 1..64");
  sv_options o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  sv_status st = check_options(o);
  if (st != SV_OK) return st;
  std::vector<svp::Gate> g;
  if ((st = convert_gates(n_qubits, gates, n_gates, false, &g)) != SV_OK) return st;
  svp::Plan P;
  const char *err = nullptr;
  bool want_jit = false;
  if (!svp::build_plan(n_qubits, g, apply_plan_options(o, n_qubits, &want_jit), fresh_state != 0, &P, &err))
    return fail(SV_ERR_ARG, err ? err : "planning failed");
  if (summary) {
    summary->passes = (int)P.passes.size();
    summary->stages = (int)P.stages.size();
    summary->ops = (int)P.ops.size() - 1;  // without the closing no-op
    summary->init_uniform = P.init_uniform ? 1 : 0;
    summary->hbm_bytes = P.hbm_bytes;
    summary->matrix_stages = 0;
    for (const std::vector<int> &sg : P.stage_gates) summary->matrix_stages += sg.empty() ? 0 : 1;
  }
  if (order_out) std::copy(P.order.begin(), P.order.end(), order_out);
  if (pass_out) std::copy(P.pass_of.begin(), P.pass_of.end(), pass_out);
  if (tile_out) {
    if (tile_cap < 64 * P.passes.size()) return fail(SV_ERR_ARG, "sv_plan: tile_cap too small");
    for (size_t p = 0; p < P.passes.size(); ++p) {
      for (int i = 0; i < 64; ++i) tile_out[64 * p + i] = -1;
      for (int i = 0; i < P.passes[p].m; ++i) tile_out[64 * p + i] = P.passes[p].tq[i];
    }
  }
  return SV_OK;
}

sv_status sv_jit_check(int n_qubits, const sv_gate *gates, size_t n_gates, const sv_options *opts, int fresh_state,
                       char *log, size_t log_cap) {
  clear_error();
  if (log && log_cap) log[0] = 0;
  if (n_qubits < 6 || n_qubits > 34) return fail(SV_ERR_ARG, "sv_jit_check: n_qubits must be 6..34");
  sv_options o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  sv_status st = check_options(o);
  if (st != SV_OK) return st;
  std::vector<svp::Gate> g;
  if ((st = convert_gates(n_qubits, gates, n_gates, false, &g)) != SV_OK) return st;
  // the tensor-core precisions: the plan kernels with matrix stages, as sv_apply_circuit
  // builds them; otherwise the plain path's plan kernels
  bool want_jit = false;
  svp::Options po = apply_plan_options(o, n_qubits, &want_jit);
  const bool tc = po.fused && po.pack;
  if (!tc) {
    po = plan_options(o);
    po.fused = false;
    po.pack = true;
    po.rk = svj::register_slots();
    po.r = std::min(po.r, po.rk);
    if (o.tile_bits == 0) po.m = svj::kTileBits;
    if (o.pipeline >= 0 && po.c == 4 && std::min(po.m, n_qubits) >= 10 && std::min(po.m, n_qubits) <= 13) po.layout = 1;
  }
  svp::Plan P;
  const char *err = nullptr;
  if (!svp::build_plan(n_qubits, g, po, fresh_state != 0, &P, &err))
    return fail(SV_ERR_ARG, err ? err : "planning failed");
  if (tc) {
    const bool f16 = o.precision == SV_PREC_F16X3;
    P.mma = f16 ? 1 : 2;
    if ((st = build_stage_mats_packed(&P, g, f16)) != SV_OK) return st;
    if (o.norm_restore < 0)
      for (svp::DevPass &dp : P.passes) dp.flags |= svp::PF_RAW;
  }
  std::vector<std::string> cubins;
  std::string lg;
  bool ok = svj::compile_plan(P, po.rk, "sm_103a", &cubins, &lg, "");
  if (ok && !P.passes.empty() && !tc) {
    // and the last pass as the inner-product variant (the backward states of the
    // inner-product amplitudes)
    std::string cubin, lg2;
    const int last = (int)P.passes.size() - 1;
    ok = svj::compile(svj::pass_is_pipelined(P, last) ? svj::pipe_pass_source(P, po.rk, last, true)
                                                      : svj::pass_source(P, po.rk, last, true),
                      "sm_103a", &cubin, &lg2);
    if (!lg2.empty()) lg += "inner last pass: " + lg2;
  }
  if (log && log_cap) {
    const size_t k = std::min(lg.size(), log_cap - 1);
    std::memcpy(log, lg.data(), k);
    log[k] = 0;
  }
  if (!ok) return fail(SV_ERR_CUDA, "sv_jit_check: NVRTC compile failed");
  return SV_OK;
}

sv_status sv_set_profiling(sv_state *s, int on) {
  clear_error();
  if (!s) return fail(SV_ERR_ARG, "NULL state");
  s->prof = on != 0;
  s->ev_used = 0;
  s->ev_bytes.clear();
  s->h2d = s->d2h = 0;
  s->other_launches = 0;
  s->jit_launches = 0;
  s->plain_fallbacks = 0;
  return SV_OK;
}

sv_status sv_get_profile(sv_state *s, sv_profile *out) {
  clear_error();
  if (!s || !out) return fail(SV_ERR_ARG, "NULL argument");
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sv_get_profile");
  out->launches = (int)(s->ev_used / 2);
  out->ms = 0;
  out->hbm_bytes = 0;
  out->h2d_bytes = s->h2d;
  out->d2h_bytes = s->d2h;
  out->other_launches = s->other_launches;
  out->jit_launches = s->jit_launches;
  out->plain_fallbacks = s->plain_fallbacks;
  out->plan_tile_bits = 0;
  out->plan_stage_qubits = 0;
  out->plan_passes = 0;
  if (s->plan_valid && !s->plan.passes.empty()) {
    out->plan_tile_bits = s->plan.passes[0].m;
    // a packed stage holds tile bit 0 besides its register slots
    out->plan_stage_qubits = s->plan.rk + ((s->plan.passes[0].flags & svp::PF_PACKED) ? 1 : 0);
    out->plan_passes = (int)s->plan.passes.size();
  }
  for (size_t i = 0; i + 1 < s->ev_used; i += 2) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, s->events[i], s->events[i + 1]) == cudaSuccess) out->ms += ms;
    out->hbm_bytes += s->ev_bytes[i / 2];
  }
  return SV_OK;
}

sv_status sv_get_launch_times(sv_state *s, double *ms_out, double *bytes_out, size_t cap, size_t *n_out) {
  clear_error();
  if (!s || !n_out) return fail(SV_ERR_ARG, "NULL argument");
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sv_get_launch_times");
  const size_t n = s->ev_used / 2;
  *n_out = n;
  for (size_t i = 0; i < n && i < cap; ++i) {
    float ms = 0;
    if (ms_out) {
      e = cudaEventElapsedTime(&ms, s->events[2 * i], s->events[2 * i + 1]);
      if (e != cudaSuccess) return cuda_fail(e, "sv_get_launch_times");
      ms_out[i] = ms;
    }
    if (bytes_out) bytes_out[i] = s->ev_bytes[i];
  }
  return SV_OK;
}

}  // extern "C"

// C ABI of the uneven batch (K7): many independent lattice circuits in one persistent,
// graph-captured launch, with the tile size picked by timing (autotune) and cached.
// Circuits large enough to fill the device by themselves (the size from which single
// circuits run on plan-specialised kernels) run as their own pass launches on such
// kernels, recorded in the same graph after the persistent launch.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sv.h"
#include "batch.h"
#include "capi_util.h"
#include "jit.h"
#include "kernels.h"
#include "plan.h"
#include "state.h"

using namespace svc;

namespace svc {

std::string autotune_cache_path() {
  if (const char *p = std::getenv("SV_AUTOTUNE_CACHE")) return p;
  Dl_info info;
  if (dladdr(reinterpret_cast<void *>(&sv_apply_batch), &info) && info.dli_fname) {
    std::string f = info.dli_fname;
    const size_t slash = f.rfind('/');
    if (slash != std::string::npos) return f.substr(0, slash) + "/autotune.json";
  }
  return "autotune.json";
}

// The file is a flat JSON object {"key": tile_bits, ...}; keys are "<device>|<hash>".
std::map<std::string, int> read_autotune_cache() {
  std::map<std::string, int> out;
  FILE *f = std::fopen(autotune_cache_path().c_str(), "r");
  if (!f) return out;
  std::string s;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, got);
  std::fclose(f);
  size_t i = 0;
  while ((i = s.find('"', i)) != std::string::npos) {
    const size_t j = s.find('"', i + 1);
    if (j == std::string::npos) break;
    const std::string k = s.substr(i + 1, j - i - 1);
    const size_t c = s.find(':', j);
    if (c == std::string::npos) break;
    out[k] = std::atoi(s.c_str() + c + 1);
    i = s.find_first_of(",}", c);
    if (i == std::string::npos) break;
  }
  return out;
}

void write_autotune_cache(const std::map<std::string, int> &c) {
  const std::string path = autotune_cache_path();
  const std::string tmp = path + ".tmp";
  FILE *f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{");
  bool first = true;
  for (const auto &kv : c) {
    std::fprintf(f, "%s\n  \"%s\": %d", first ? "" : ",", kv.first.c_str(), kv.second);
    first = false;
  }
  std::fprintf(f, "\n}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), path.c_str());
}

}  // namespace svc

namespace {

int lattice_qubits(const sv_lattice &lat) {
  const int sites = lat.rows * lat.cols;
  int n = 0;
  for (int i = 0; i < sites; ++i) n += !((lat.removed_mask >> i) & 1ull);
  return n;
}

struct DeviceBuf {
  void *p = nullptr;
  ~DeviceBuf() { if (p) cudaFree(p); }
  sv_status alloc(size_t bytes) {
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return fail(SV_ERR_OOM, "sv_apply_batch: device allocation failed");
    }
    return SV_OK;
  }
};

// Plan-kernel circuits are dealt to this many parallel chains of launches (graph
// branches), so that one circuit's last wave of tiles overlaps another's.  Measured on
// the 512-circuit batch with every circuit on plan kernels: 1 branch 0.0469 s, 4 0.0414,
// 8 0.0422, 16 0.0425, 64 0.0429.
constexpr size_t kBranches = 4;

// A circuit of the batch that runs on its plan's own kernels.
struct JitCircuit {
  size_t circuit = 0;
  uint64_t state_off = 0;
  svp::Plan P;
  DeviceBuf plan;
  svk::DevPlanView view{};
  const svj::Module *M = nullptr;
};

// Everything one batch needs on the device, plus its instantiated graph.
struct Batch {
  std::string key;
  int m = 13;
  int count = 0;
  std::vector<int> nq;
  std::vector<std::unique_ptr<JitCircuit>> jit;
  DeviceBuf states, plan, cps, items, words, chunks, partials, chunk_begin, stats;
  svk::DevPlanView view{};
  uint64_t n_items = 0;
  int n_chunks = 0;
  size_t words_bytes = 0;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> branch;  // parallel chains of the plan-kernel circuits
  std::vector<cudaEvent_t> ev;       // fork, then one join per branch
  cudaGraphExec_t exec[2] = {nullptr, nullptr};  // without, with the statistics
  ~Batch() {
    for (cudaGraphExec_t x : exec)
      if (x) cudaGraphExecDestroy(x);
    if (stream) cudaStreamDestroy(stream);
    for (cudaStream_t b : branch) cudaStreamDestroy(b);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

std::mutex g_mu;
Batch *g_batch = nullptr;  // the last batch (reused while the lattice list repeats)

std::string batch_key(const sv_lattice *c, size_t count, int m, int jit) {
  std::string k = "m" + std::to_string(m) + "j" + std::to_string(jit) + ":";
  k.reserve(count * 48);
  char buf[96];
  for (size_t i = 0; i < count; ++i) {
    std::snprintf(buf, sizeof(buf), "%d,%d,%llx,%d,%llx;", c[i].rows, c[i].cols, (unsigned long long)c[i].removed_mask,
                  c[i].depth, (unsigned long long)c[i].seed);
    k += buf;
  }
  return k;
}

// A plan's arrays in one device buffer, as the pass kernels read them.
sv_status upload_jit_plan(JitCircuit *J) {
  const svp::Plan &P = J->P;
  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_stage = align(P.passes.size() * sizeof(svp::DevPass));
  const size_t o_op = o_stage + align(P.stages.size() * sizeof(svp::DevStage));
  const size_t o_gt = o_op + align(P.ops.size() * sizeof(svp::DevOp));
  const size_t o_err = o_gt + align(P.gtab.size() * sizeof(svp::DevGroupEntry));
  const size_t bytes = o_err + 256;
  sv_status st = J->plan.alloc(bytes);
  if (st != SV_OK) return st;
  std::vector<char> hp(bytes, 0);
  std::memcpy(hp.data(), P.passes.data(), P.passes.size() * sizeof(svp::DevPass));
  std::memcpy(hp.data() + o_stage, P.stages.data(), P.stages.size() * sizeof(svp::DevStage));
  std::memcpy(hp.data() + o_op, P.ops.data(), P.ops.size() * sizeof(svp::DevOp));
  std::memcpy(hp.data() + o_gt, P.gtab.data(), P.gtab.size() * sizeof(svp::DevGroupEntry));
  const cudaError_t e = cudaMemcpy(J->plan.p, hp.data(), bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "sv_apply_batch: plan upload");
  char *d = static_cast<char *>(J->plan.p);
  J->view.passes = reinterpret_cast<const svp::DevPass *>(d);
  J->view.stages = reinterpret_cast<const svp::DevStage *>(d + o_stage);
  J->view.ops = reinterpret_cast<const svp::DevOp *>(d + o_op);
  J->view.mats = reinterpret_cast<const float *>(d + o_err);
  J->view.err = reinterpret_cast<int *>(d + o_err);
  J->view.gtab = reinterpret_cast<const svp::DevGroupEntry *>(d + o_gt);
  return SV_OK;
}

// Plans and compiled kernels of the circuits that run on their own kernels (jit: the
// options' field: 1 every circuit of at least one tile, 0 those of at least
// kJitMinQubits, -1 none).  With
// jit 0 and no compiler the set is left empty and those circuits join the persistent
// launch.
sv_status build_jit_circuits(const std::vector<std::vector<svp::Gate>> &gates, const std::vector<int> &nq,
                             const std::vector<uint64_t> &state_off, int jit, Batch *B) {
  B->jit.clear();
  if (jit < 0) return SV_OK;
  svp::Options po;
  po.m = svj::kTileBits;
  po.c = 4;
  po.pack = true;
  po.rk = svj::register_slots();
  po.r = po.rk;
  for (size_t i = 0; i < gates.size(); ++i) {
    if (nq[i] < svj::kTileBits || (jit == 0 && nq[i] < kJitMinQubits)) continue;
    std::unique_ptr<JitCircuit> J(new JitCircuit);
    J->circuit = i;
    J->state_off = state_off[i];
    svp::Options pi = po;
    pi.m = std::min(po.m, nq[i]);
    const char *err = nullptr;
    if (!svp::build_plan(nq[i], gates[i], pi, true, &J->P, &err)) return fail(SV_ERR_ARG, err ? err : "planning failed");
    B->jit.push_back(std::move(J));
  }
  if (B->jit.empty()) return SV_OK;
  // largest first, dealt round-robin to the branches
  std::stable_sort(B->jit.begin(), B->jit.end(), [&](const std::unique_ptr<JitCircuit> &a,
                                                     const std::unique_ptr<JitCircuit> &b) {
    return nq[a->circuit] > nq[b->circuit];
  });
  std::vector<const svp::Plan *> plans;
  for (auto &J : B->jit) plans.push_back(&J->P);
  std::vector<const svj::Module *> mods;
  std::string jerr;
  if (!svj::get_modules(plans, po.rk, &mods, &jerr)) {
    B->jit.clear();
    return jit == 1 ? fail(SV_ERR_CUDA, jerr.c_str()) : SV_OK;
  }
  for (size_t j = 0; j < B->jit.size(); ++j) {
    JitCircuit *J = B->jit[j].get();
    J->M = mods[j];
    sv_status st = upload_jit_plan(J);
    if (st != SV_OK) return st;
    const cudaError_t e = svj::prepare_passes(J->M, J->P);
    if (e != cudaSuccess) return cuda_fail(e, "sv_apply_batch: plan kernels");
  }
  const size_t nb = std::min(B->jit.size(), kBranches);
  for (size_t b = 0; b <= nb; ++b) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "sv_apply_batch: events");
    B->ev.push_back(e);
    if (b == nb) break;
    cudaStream_t t = nullptr;
    if (cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "sv_apply_batch: streams");
    B->branch.push_back(t);
  }
  return SV_OK;
}

// Build plans, the work queue and the device buffers of a batch with tile size m.
sv_status build_batch(const sv_lattice *circs, size_t count, int m_req, int jit, Batch *B) {
  B->count = (int)count;
  B->nq.resize(count);
  int n_min = 64;  // smallest circuit (of the persistent launch, below)
  std::vector<std::vector<svp::Gate>> gates(count);
  for (size_t i = 0; i < count; ++i) {
    const int n = lattice_qubits(circs[i]);
    if (n < 6 || n > 28) return fail(SV_ERR_ARG, "sv_apply_batch: circuits must have 6..28 qubits");
    B->nq[i] = n;
    n_min = std::min(n_min, n);
    size_t ng = 0;
    sv_status st = sv_generate_circuit(&circs[i], nullptr, 0, &ng);
    if (st != SV_OK) return st;
    std::vector<sv_gate> g(ng);
    if ((st = sv_generate_circuit(&circs[i], g.data(), ng, &ng)) != SV_OK) return st;
    if ((st = convert_gates(n, g.data(), ng, false, &gates[i])) != SV_OK) return st;
  }
  std::vector<uint64_t> state_off(count);
  uint64_t total_amps = 0;
  for (size_t i = 0; i < count; ++i) {
    state_off[i] = total_amps;
    total_amps += 1ull << B->nq[i];
  }
  sv_status st;
  if ((st = build_jit_circuits(gates, B->nq, state_off, jit, B)) != SV_OK) return st;
  std::vector<char> on_jit(count, 0);
  for (auto &J : B->jit) on_jit[J->circuit] = 1;
  n_min = 64;
  for (size_t i = 0; i < count; ++i)
    if (!on_jit[i]) n_min = std::min(n_min, B->nq[i]);
  const int m = std::min(std::min(m_req, svk::tile_pass_max_bits()), n_min);
  B->m = m;
  svp::Options po;
  po.m = m;
  po.c = 4;
  po.pack = true;  // the batch kernel runs the packed interpreter
  po.rk = svk::tile_pass_register_slots();
  po.r = po.rk;
  // combined plan
  std::vector<svp::DevPass> passes;
  std::vector<svp::DevStage> stages;
  std::vector<svp::DevOp> ops;
  std::vector<svp::DevGroupEntry> gtab;
  std::vector<std::vector<uint32_t>> circ_passes(count);
  for (size_t i = 0; i < count; ++i) {
    if (on_jit[i]) continue;
    svp::Plan P;
    const char *err = nullptr;
    if (!svp::build_plan(B->nq[i], gates[i], po, true, &P, &err)) return fail(SV_ERR_ARG, err ? err : "planning failed");
    const uint32_t sb = (uint32_t)stages.size(), ob = (uint32_t)ops.size();
    for (svp::DevStage ds : P.stages) {
      ds.op_begin += ob;  // rebase into the combined arrays
      stages.push_back(ds);
    }
    for (const svp::DevOp &o : P.ops) ops.push_back(o);
    gtab.insert(gtab.end(), P.gtab.begin(), P.gtab.end());
    for (svp::DevPass dp : P.passes) {
      dp.stage_begin += sb;
      circ_passes[i].push_back((uint32_t)passes.size());
      passes.push_back(dp);
    }
  }
  // work queue: round r = r-th pass of every circuit that has one, larger circuits first
  std::vector<size_t> order(count);
  for (size_t i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return B->nq[a] > B->nq[b]; });
  std::vector<svk::BatchCP> cps;
  std::vector<svk::BatchItem> items;
  std::vector<uint32_t> last_cp(count, svk::kNoPrev);
  size_t max_passes = 0;
  for (auto &v : circ_passes) max_passes = std::max(max_passes, v.size());
  for (size_t r = 0; r < max_passes; ++r) {
    for (size_t oi : order) {
      if (r >= circ_passes[oi].size()) continue;
      svk::BatchCP cp;
      cp.state_off = state_off[oi];
      cp.pass = circ_passes[oi][r];
      cp.prev = last_cp[oi];
      cp.tiles = 1u << (B->nq[oi] - m);
      cp.circuit = (uint32_t)oi;
      const uint32_t id = (uint32_t)cps.size();
      cps.push_back(cp);
      last_cp[oi] = id;
      for (uint32_t t = 0; t < cp.tiles; ++t) items.push_back(svk::BatchItem{id, t});
    }
  }
  B->n_items = items.size();
  // stats chunks: 2^16 amplitudes each
  std::vector<svk::BatchChunk> chunks;
  std::vector<int> chunk_begin(count + 1, 0);
  for (size_t i = 0; i < count; ++i) {
    chunk_begin[i] = (int)chunks.size();
    const uint64_t amps = 1ull << B->nq[i];
    for (uint64_t s = 0; s < amps; s += 65536)
      chunks.push_back(svk::BatchChunk{state_off[i] + s, (uint32_t)std::min<uint64_t>(65536, amps - s), (uint32_t)i});
  }
  chunk_begin[count] = (int)chunks.size();
  B->n_chunks = (int)chunks.size();
  // device buffers
  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_stage = align(passes.size() * sizeof(svp::DevPass));
  const size_t o_op = o_stage + align(stages.size() * sizeof(svp::DevStage));
  const size_t o_gt = o_op + align(ops.size() * sizeof(svp::DevOp));
  const size_t o_err = o_gt + align(gtab.size() * sizeof(svp::DevGroupEntry));
  const size_t plan_bytes = o_err + 256;
  if ((st = B->states.alloc(total_amps * sizeof(float2))) != SV_OK) return st;
  if ((st = B->plan.alloc(plan_bytes)) != SV_OK) return st;
  if ((st = B->cps.alloc(std::max<size_t>(1, cps.size()) * sizeof(svk::BatchCP))) != SV_OK) return st;
  if ((st = B->items.alloc(std::max<size_t>(1, items.size()) * sizeof(svk::BatchItem))) != SV_OK) return st;
  B->words_bytes = (svk::kBatchHeader + cps.size()) * sizeof(unsigned int);
  if ((st = B->words.alloc(B->words_bytes)) != SV_OK) return st;
  if ((st = B->chunks.alloc(std::max<size_t>(1, chunks.size()) * sizeof(svk::BatchChunk))) != SV_OK) return st;
  if ((st = B->partials.alloc(std::max<size_t>(1, chunks.size()) * 2 * sizeof(double))) != SV_OK) return st;
  if ((st = B->chunk_begin.alloc((count + 1) * sizeof(int))) != SV_OK) return st;
  if ((st = B->stats.alloc(std::max<size_t>(1, count) * 2 * sizeof(double))) != SV_OK) return st;
  std::vector<char> hp(plan_bytes, 0);
  std::memcpy(hp.data(), passes.data(), passes.size() * sizeof(svp::DevPass));
  std::memcpy(hp.data() + o_stage, stages.data(), stages.size() * sizeof(svp::DevStage));
  std::memcpy(hp.data() + o_op, ops.data(), ops.size() * sizeof(svp::DevOp));
  std::memcpy(hp.data() + o_gt, gtab.data(), gtab.size() * sizeof(svp::DevGroupEntry));
  cudaError_t e = cudaMemcpy(B->plan.p, hp.data(), plan_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !cps.empty()) e = cudaMemcpy(B->cps.p, cps.data(), cps.size() * sizeof(svk::BatchCP), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpy(B->items.p, items.data(), items.size() * sizeof(svk::BatchItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !chunks.empty())
    e = cudaMemcpy(B->chunks.p, chunks.data(), chunks.size() * sizeof(svk::BatchChunk), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(B->chunk_begin.p, chunk_begin.data(), (count + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "sv_apply_batch: upload");
  char *d = static_cast<char *>(B->plan.p);
  B->view.passes = reinterpret_cast<const svp::DevPass *>(d);
  B->view.stages = reinterpret_cast<const svp::DevStage *>(d + o_stage);
  B->view.ops = reinterpret_cast<const svp::DevOp *>(d + o_op);
  B->view.mats = reinterpret_cast<const float *>(d + o_err);
  B->view.err = reinterpret_cast<int *>(d + o_err);
  B->view.gtab = reinterpret_cast<const svp::DevGroupEntry *>(d + o_gt);
  return SV_OK;
}

// Enqueue one run of the batch on stream st: reset the queue, the persistent launch
// (and, forked beside it, the plan-kernel circuits' pass launches on the branch
// streams), then (with_stats) the per-circuit statistics.
cudaError_t enqueue_batch(Batch *B, cudaStream_t st, bool with_stats) {
  cudaError_t e = cudaMemsetAsync(B->words.p, 0, B->words_bytes, st);
  const size_t nb = B->branch.size();
  if (e == cudaSuccess && nb) e = cudaEventRecord(B->ev[0], st);
  for (size_t b = 0; e == cudaSuccess && b < nb; ++b) e = cudaStreamWaitEvent(B->branch[b], B->ev[0], 0);
  if (e == cudaSuccess && B->n_items)
    e = svk::launch_batch(static_cast<float2 *>(B->states.p), B->view, static_cast<const svk::BatchCP *>(B->cps.p),
                          static_cast<const svk::BatchItem *>(B->items.p), B->n_items,
                          static_cast<unsigned int *>(B->words.p), B->m, st);
  float2 *states = static_cast<float2 *>(B->states.p);
  for (size_t j = 0; e == cudaSuccess && j < B->jit.size(); ++j) {
    const JitCircuit &J = *B->jit[j];
    const int n = B->nq[J.circuit];
    for (size_t p = 0; e == cudaSuccess && p < J.P.passes.size(); ++p)
      e = svj::launch_pass(J.M, states + J.state_off, n, J.view, (int)p, J.P.passes[p], B->branch[j % nb]);
  }
  for (size_t b = 0; e == cudaSuccess && b < nb; ++b) {
    e = cudaEventRecord(B->ev[b + 1], B->branch[b]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, B->ev[b + 1], 0);
  }
  if (e == cudaSuccess && with_stats)
    e = svk::launch_batch_stats(static_cast<const float2 *>(B->states.p), static_cast<const svk::BatchChunk *>(B->chunks.p),
                                B->n_chunks, static_cast<double *>(B->partials.p),
                                static_cast<const int *>(B->chunk_begin.p), B->count, static_cast<double *>(B->stats.p), st);
  return e;
}

// ---- autotune: tile size of the batch, timed, cached in a JSON file --------------------

std::string tune_key(const sv_lattice *circs, size_t count, int jit) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  uint64_t h = 1469598103934665603ull;  // FNV-1a over the lattice list
  const std::string k = batch_key(circs, count, 0, 0);
  for (char ch : k) { h ^= (unsigned char)ch; h *= 1099511628211ull; }
  char buf[sizeof(prop.name) + 64];
  std::snprintf(buf, sizeof(buf), "%s|batch|j%d|%zu|%016llx", prop.name, jit, count, (unsigned long long)h);
  for (char *p = buf; *p; ++p)
    if (*p == '"' || *p == '\\') *p = '_';
  return buf;
}

sv_status autotune_tile_bits(const sv_lattice *circs, size_t count, int jit, int *m_out) {
  const std::string key = tune_key(circs, count, jit);
  std::map<std::string, int> cache = read_autotune_cache();
  auto it = cache.find(key);
  if (it != cache.end() && it->second >= 10 && it->second <= 13) { *m_out = it->second; return SV_OK; }
  const int cand[3] = {11, 12, 13};
  float best = 1e30f;
  int best_m = 13;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int m : cand) {
    Batch B;
    sv_status st = build_batch(circs, count, m, jit, &B);
    if (st != SV_OK) { cudaEventDestroy(a); cudaEventDestroy(b); return st; }
    float ms = 0;
    for (int rep = 0; rep < 2; ++rep) {  // second run is timed
      cudaEventRecord(a, 0);
      cudaError_t e = enqueue_batch(&B, 0, false);
      cudaEventRecord(b, 0);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      if (e != cudaSuccess) { cudaEventDestroy(a); cudaEventDestroy(b); return cuda_fail(e, "sv_apply_batch: autotune"); }
      cudaEventElapsedTime(&ms, a, b);
    }
    if (ms < best) { best = ms; best_m = B.m; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cache[key] = best_m;
  write_autotune_cache(cache);
  *m_out = best_m;
  return SV_OK;
}

}  // namespace

extern "C" sv_status sv_apply_batch(const sv_lattice *circs, size_t count, const sv_options *opts, double *stats_out) {
  clear_error();
  if (count && !circs) return fail(SV_ERR_ARG, "sv_apply_batch: NULL lattice array");
  if (count == 0) return SV_OK;
  sv_options o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.tile_bits != 0 && (o.tile_bits < 10 || o.tile_bits > 13))
    return fail(SV_ERR_ARG, "sv_apply_batch: tile_bits must be 0 or 10..13");
  std::lock_guard<std::mutex> lock(g_mu);
  int m = o.tile_bits > 0 ? o.tile_bits : 13;
  sv_status st;
  if (o.jit < -1 || o.jit > 1) return fail(SV_ERR_ARG, "sv_apply_batch: jit must be -1, 0 or 1");
  if (o.autotune && o.tile_bits == 0 && (st = autotune_tile_bits(circs, count, o.jit, &m)) != SV_OK) return st;
  const std::string key = batch_key(circs, count, m, o.jit);
  if (!g_batch || g_batch->key != key) {
    delete g_batch;
    g_batch = nullptr;
    Batch *B = new Batch();
    if ((st = build_batch(circs, count, m, o.jit, B)) != SV_OK) { delete B; return st; }
    B->key = key;
    const cudaError_t e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete B; return cuda_fail(e, "sv_apply_batch: stream"); }
    g_batch = B;
  }
  Batch *B = g_batch;
  const int with_stats = stats_out ? 1 : 0;
  if (!B->exec[with_stats]) {
    // capture {reset, launches, statistics if asked for} once; later calls replay it
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue_batch(B, B->stream, with_stats != 0);
      e = cudaStreamEndCapture(B->stream, &graph);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec[with_stats], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      delete B;
      g_batch = nullptr;
      return cuda_fail(e, "sv_apply_batch: graph capture");
    }
  }
  cudaStream_t user = static_cast<cudaStream_t>(o.stream);
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  // order the graph after the caller's stream, run it, then order the caller after it
  if (e == cudaSuccess) e = cudaEventRecord(ev, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(B->stream, ev, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(B->exec[with_stats], B->stream);
  std::vector<double> st2(2 * count);
  unsigned int hw[2] = {0, 0};
  if (e == cudaSuccess && with_stats)
    e = cudaMemcpyAsync(st2.data(), B->stats.p, 2 * count * sizeof(double), cudaMemcpyDeviceToHost, B->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hw, B->words.p, sizeof(hw), cudaMemcpyDeviceToHost, B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  cudaEventDestroy(ev);
  if (e != cudaSuccess) return cuda_fail(e, "sv_apply_batch");
  if (hw[1] != 0) return fail(SV_ERR_TIMEOUT, "sv_apply_batch: a dependency wait gave up (results undefined)");
  if (stats_out)
    for (size_t i = 0; i < count; ++i) {
      stats_out[3 * i] = st2[2 * i];
      stats_out[3 * i + 1] = st2[2 * i + 1];
      stats_out[3 * i + 2] = B->nq[i];
    }
  return SV_OK;
}

extern "C" sv_status sv_batch_amplitudes(size_t circuit, const uint64_t *bits, size_t m, double *out_re_im) {
  clear_error();
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_batch) return fail(SV_ERR_STATE, "sv_batch_amplitudes: no batch has run");
  if (circuit >= (size_t)g_batch->count || (m && (!bits || !out_re_im))) return fail(SV_ERR_ARG, "sv_batch_amplitudes: bad argument");
  const int n = g_batch->nq[circuit];
  uint64_t off = 0;
  for (size_t i = 0; i < circuit; ++i) off += 1ull << g_batch->nq[i];
  for (size_t j = 0; j < m; ++j) {
    if (bits[j] >> n) return fail(SV_ERR_ARG, "sv_batch_amplitudes: bitstring has bits >= n");
    float2 z;
    cudaError_t e = cudaMemcpy(&z, static_cast<float2 *>(g_batch->states.p) + off + bits[j], sizeof(z), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "sv_batch_amplitudes");
    out_re_im[2 * j] = z.x;
    out_re_im[2 * j + 1] = z.y;
  }
  return SV_OK;
}

// A queue whose only item depends on a pass that has no items: its wait can never be
// met, so the kernel must give up after limit_ms and report it.
extern "C" sv_status sv_selftest_wait_timeout(int limit_ms) {
  clear_error();
  if (limit_ms < 1 || limit_ms > 10000) return fail(SV_ERR_ARG, "sv_selftest_wait_timeout: limit_ms must be 1..10000");
  std::lock_guard<std::mutex> lock(g_mu);
  const int m = 13;
  svp::DevPass dp;
  std::memset(&dp, 0, sizeof(dp));
  dp.m = m;
  dp.c = 4;
  dp.n = m;
  for (int i = 0; i < m; ++i) dp.tq[i] = (uint8_t)i;
  const svk::BatchCP cps[2] = {{0, 0, svk::kNoPrev, 1, 0}, {0, 0, 0, 1, 0}};
  const svk::BatchItem item = {1, 0};  // waits for cp 0, whose tile is never queued
  DeviceBuf state, plan, dcps, ditems, words;
  sv_status st;
  if ((st = state.alloc(sizeof(float2) << m)) != SV_OK) return st;
  if ((st = plan.alloc(1024)) != SV_OK) return st;
  if ((st = dcps.alloc(sizeof(cps))) != SV_OK) return st;
  if ((st = ditems.alloc(sizeof(item))) != SV_OK) return st;
  if ((st = words.alloc((svk::kBatchHeader + 2) * sizeof(unsigned int))) != SV_OK) return st;
  cudaError_t e = cudaMemcpy(plan.p, &dp, sizeof(dp), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dcps.p, cps, sizeof(cps), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ditems.p, &item, sizeof(item), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(words.p, 0, (svk::kBatchHeader + 2) * sizeof(unsigned int));
  svk::DevPlanView view{};
  view.passes = static_cast<const svp::DevPass *>(plan.p);
  view.stages = reinterpret_cast<const svp::DevStage *>(static_cast<char *>(plan.p) + 512);
  view.ops = nullptr;
  view.mats = nullptr;
  view.err = nullptr;
  if (e == cudaSuccess)
    e = svk::launch_batch(static_cast<float2 *>(state.p), view, static_cast<const svk::BatchCP *>(dcps.p),
                          static_cast<const svk::BatchItem *>(ditems.p), 1, static_cast<unsigned int *>(words.p), m, 0,
                          (unsigned long long)limit_ms * 1000000ull, 1);
  unsigned int hw[svk::kBatchHeader] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(hw, words.p, sizeof(hw), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "sv_selftest_wait_timeout");
  if (hw[1] != 0) return fail(SV_ERR_TIMEOUT, "dependency wait gave up as designed");
  return SV_OK;
}

extern "C" sv_status sv_batch_config(int *tile_bits, int *plan_kernel_circuits, int *persistent_circuits) {
  clear_error();
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_batch) return fail(SV_ERR_STATE, "sv_batch_config: no batch has run");
  if (tile_bits) *tile_bits = g_batch->m;
  if (plan_kernel_circuits) *plan_kernel_circuits = (int)g_batch->jit.size();
  if (persistent_circuits) *persistent_circuits = g_batch->count - (int)g_batch->jit.size();
  return SV_OK;
}

extern "C" sv_status sv_batch_free(void) {
  clear_error();
  std::lock_guard<std::mutex> lock(g_mu);
  delete g_batch;
  g_batch = nullptr;
  return SV_OK;
}

// Plan-specialised tile-pass kernels compiled at run time (NVRTC).
//
// The packed tile kernel interprets a plan: one indirect branch per op picks the op's
// code.  For a plan that runs more than once (or on a large state) the library instead
// writes one kernel per pass in which every stage's ops are straight-line calls of the
// same device functions (tile_pack.cuh) with the register slots, conditions and scale
// factors as constants, compiles it for the device with NVRTC and keeps the module.
// The arithmetic is the interpreter's, op for op: the results are bitwise identical.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "plan.h"
#include "plan_dev.h"

namespace svj {

// Register slots besides the pack bit of the plan-specialised kernels (plans for them
// are built with this rk).  Measured on 34 qubits: 4 slots 0.75 s, 3 slots 0.83 s; a
// second tile buffer with the next tile's read in flight was slower at either width
// (0.87 s, 0.96 s): it halves the resident CTAs, and the stages need every warp.
constexpr int kRegisterSlots = 4;
int register_slots();
// Default tile size of plans for these kernels: 12 qubits (8 passes on 34 qubits, five
// CTAs per SM) measured faster than 13 (7 passes, two CTAs) and 14 (6 passes, one).
constexpr int kTileBits = 12;

// Pipelined kernels: each CTA takes runs of 2^kTileRunLog neighbouring tiles per turn of
// the grid (tile_of in tile_pipe.cuh; tile_run_log() reads the SV_TILE_RUN override).
// Measured on 34 qubits (plain path, fixed kernel shapes): a pass whose tile leaves out
// qubit 4 reads 128-byte rows, and with one tile per turn (runs of 1) such passes ran at
// 0.77-0.81 of the copy bandwidth (5.0-5.4 TB/s) against 0.97 with qubit 4 in the tile;
// runs of 2 took the circuit from 0.419 s to 0.382 s, runs of 4 and 8 measured the same.
// The tensor-core passes (latency-bound) keep runs of 1: with runs of 2 the F16x3 circuit
// measured 0.918 s against 0.907 s.
constexpr int kTileRunLog = 1;
int tile_run_log();

// Pipelined kernels (plans with Options::layout = 1, tile_pipe.cuh): compute groups and
// shared-memory tile slots per CTA for a tile size; false where the tile size has none.
// 12-qubit tiles: three groups of 128 threads with two 32 KB slots each (one CTA per SM;
// 13 warps, so up to 128 registers a thread).  Slots are a multiple of the groups.
constexpr int kPipeGroups12 = 3;
constexpr int kPipeSlots12 = 6;
bool pipe_shape(int m, int *groups, int *slots);
// The shape of pass `pass` of P: the tile size's default, or the plan's pipe_groups entry.
bool pass_pipe_shape(const svp::Plan &P, int pass, int *groups, int *slots);
// Matrix stages of a pass that run on the tensor cores (Plan::mma), and the shared memory
// of their B buffers.
int pass_matrix_stages(const svp::Plan &P, int pass);
int pass_streams(const svp::Plan &P, int pass);
size_t pass_mma_smem(const svp::Plan &P, int pass);
// Whether pass `pass` of P runs on the pipelined kernel (layout-1 plan, at least one stage).
bool pass_is_pipelined(const svp::Plan &P, int pass);
// Threads of the pipelined kernel's CTA for a pass: the compute groups, the producer warp
// and, where the last stage's output goes out by TMA stores, the storer warp.
int pipe_threads(const svp::Plan &P, int kpr, int pass, bool inner);
// CUDA source of the pipelined kernel ("sv_pass") of one pass of a layout-1 packed plan.
std::string pipe_pass_source(const svp::Plan &P, int kpr, int pass, bool inner = false);

// CUDA source of the kernel ("sv_pass") of one pass of a packed plan.  kpr: register
// slots besides the pack bit (the plan's rk).  inner (the last pass only): instead of
// storing the state, the kernel sums conj(state) * other over it into per-CTA partials.
std::string pass_source(const svp::Plan &P, int kpr, int pass, bool inner = false);

// Compile CUDA source for an architecture ("sm_103a") to a cubin with NVRTC; the
// device headers are compiled into the library.  Returns false with *log set.
bool compile(const std::string &src, const char *arch, std::string *cubin, std::string *log);

// Compile the kernels of every pass of a plan (one NVRTC program per pass, in parallel
// threads).  cache: a directory of cubins by source hash ("" = none).
bool compile_plan(const svp::Plan &P, int kpr, const char *arch, std::vector<std::string> *cubins,
                  std::string *log, const std::string &cache);

struct Module;

// The compiled kernels of plan P on the current device, from the in-process cache, the
// on-disk cache (the library's build directory, subdirectory jit) or a fresh compile.
// nullptr with *err set if NVRTC or the module load fails.
const Module *get_module(const svp::Plan &P, int kpr, std::string *err, bool inner = false);

// The modules of several plans at once: every pass kernel not yet cached is compiled in
// one pool of worker threads.  false with *err set if any compile or load fails.
bool get_modules(const std::vector<const svp::Plan *> &plans, int kpr, std::vector<const Module *> *out,
                 std::string *err, bool inner = false);

// Set each pass kernel's shared-memory limit and occupancy now rather than at its first
// launch (before a stream capture records the launches).
cudaError_t prepare_passes(const Module *M, const svp::Plan &P);

// Launch pass `pass` of a module on the plan's device copy.  sums (the plan's last pass
// only; null elsewhere): per CTA, the sums of p and p^2 of the amplitudes it stored (an
// inner module's last pass: of re and im of conj(state) * other, without storing), at
// sums[2 b], sums[2 b + 1] for CTA b; *grid_out (may be null): the CTAs launched.
cudaError_t launch_pass(const Module *M, float2 *psi, int n, const svk::DevPlanView &view, int pass,
                        const svp::DevPass &hp, cudaStream_t st, double *sums = nullptr,
                        unsigned *grid_out = nullptr, const float2 *other = nullptr);

// Upper bound of the CTAs one pass launch uses (sizes the sums buffer).
unsigned max_pass_grid();

}  // namespace svj

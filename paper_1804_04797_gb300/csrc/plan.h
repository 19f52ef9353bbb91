// Internal plan format shared by the host planner and the CUDA kernels.
//
// A plan turns a gate list into PASSES.  Each pass is one sweep of the state in HBM:
// the state is cut into 2^m-amplitude gathered TILES -- the amplitudes whose indices
// differ only in the m tile qubits (the c lowest qubits, for coalesced access, plus
// m-c chosen high qubits).  This is the paper's idea of "local qubits" (§2.3: keep a
// block of amplitudes on-chip and apply every gate that acts inside it), with the tile
// qubits chosen anew for every pass instead of fixed low ranks plus rank swaps.
// Inside a pass the gates are grouped into STAGES of at most r "register" qubits: the
// plain kernel holds 2^r amplitudes per thread and applies the stage's gates in
// registers; the tensor-core kernel multiplies them into one 2^r x 2^r unitary.
#pragma once

#include <cstdint>
#include <vector>

#include "plan_dev.h"

namespace svp {

// Gate kinds (same codes as sv_kind) plus the internal branch projector.
enum Kind : uint8_t {
  K_H = 0, K_T = 1, K_SX = 2, K_SY = 3, K_CZ = 4, K_P0 = 5, K_P1 = 6, K_Z = 7,
  K_TDG = 8, K_SXDG = 9, K_SYDG = 10,
  K_PEQ = 11,  // zero the amplitudes whose bits q0 and q1 differ (branch projector)
  K_COUNT = 12
};

inline bool kind_is_diag(int k) {
  return k == K_T || k == K_CZ || k == K_P0 || k == K_P1 || k == K_Z || k == K_TDG ||
         k == K_PEQ;
}
inline bool kind_two_qubit(int k) { return k == K_CZ || k == K_PEQ; }

struct Gate {
  uint8_t kind, q0, q1;
};

struct Options {
  int m = 13;        // tile qubits
  int c = 4;         // contiguous low qubits in every tile
  int r = 5;         // qubits a stage may act on (<= rk)
  int rk = 5;        // register qubits per thread of the kernel that runs the plan
  bool fused = false;
  bool pack = false; // packed plain kernel: tile bit 0 joins every stage as the pack bit
  // shared-memory layout of a packed tile (pair k = tile bits 1..m-1 at a 16-byte slot):
  //   0  slot k ^ ((k>>3 ^ k>>6 ^ k>>9) & 7): every pair bit toggles a bank-group bit
  //   1  slot k ^ ((k>>3) & 7): the 128-byte swizzle of the tensor-memory-access (TMA)
  //      copies, the tile as 1 KB boxes of eight 128-byte rows (rows: tile bits 4..6)
  int layout = 0;
};

// 16-byte slot of pair k of a packed tile in a layout (see Options::layout).
inline uint32_t pack_phys(uint32_t k, int layout) {
  return layout == 1 ? k ^ ((k >> 3) & 7u) : k ^ (((k >> 3) ^ (k >> 6) ^ (k >> 9)) & 7u);
}

struct Plan {
  int n = 0;
  std::vector<DevPass> passes;
  std::vector<DevStage> stages;
  std::vector<DevOp> ops;
  std::vector<float> mats;          // 8 floats per A_U matrix (re/im of a,b,c,d)
  std::vector<DevGroupEntry> gtab;  // kGroupEntries per stage
  std::vector<int32_t> order;       // executed gate index, in execution order
  std::vector<int32_t> pass_of;     // pass of each executed gate
  std::vector<std::vector<int>> stage_gates;  // per stage: gate indices (inner, in order)
  std::vector<std::vector<int>> stage_post;   // per stage: diagonal gates applied after
  bool init_uniform = false;
  double hbm_bytes = 0;
  int layout = 0;  // shared-memory layout of the packed tiles (Options::layout)
  int rk = 0;      // register qubits a thread holds per stage (Options::rk, capped by the tile)
  // layout 1: compute groups of each pass's pipelined kernel (0 = the default for the tile
  // size); set by the autotuner, read by the kernel generator
  std::vector<uint8_t> pipe_groups;
  // plan kernels of a fused packed plan: its matrix stages run on the tensor cores
  // (0 = none, 1 = F16x3, 2 = TF32x3; B operands in `mats`, set with the plan's matrices)
  int mma = 0;
};

// Build the plan.  fresh_state: the state is |0..0> and was never written, so a
// leading layer of H on every qubit may become the uniform initial tile, and a plan
// without that layer starts from |0..0> generated in the first pass.  Gates must be
// validated by the caller.  Returns false with *err set on failure.
bool build_plan(int n, const std::vector<Gate> &gates, const Options &opt, bool fresh_state,
                Plan *plan, const char **err);

// Matrix (re/im of a, b, c, d) of a one-qubit kind, in double precision.
void kind_matrix(int kind, double m[8]);

// The unitary of a stage's inner ops on its r register bits: 2^r x 2^r complex
// (row-major, re/im interleaved; row/column bit j = register bit j; in a packed plan bit 0
// is tile bit 0 and bit j + 1 register slot j), in double precision.
void stage_unitary(const Plan &plan, const std::vector<Gate> &gates, int stage, int r,
                   std::vector<double> *u);

}  // namespace svp

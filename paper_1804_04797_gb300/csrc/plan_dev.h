// Plan records as the kernels read them (device memory layout), shared by the host
// planner, the ahead-of-time kernels and the kernels compiled at run time (this header
// compiles under NVRTC: no standard headers there).
#pragma once

#ifdef __CUDACC_RTC__
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
typedef int int32_t;
#else
#include <cstdint>
#endif

namespace svp {

// Actions of a device op on a thread's register group (2^r amplitudes, element e has
// register bit j = bit j of e).
enum Act : uint8_t {
  A_U = 0,      // general 2x2 (matrix slot `arg`) on register bit j
  A_H, A_SX, A_SY, A_SXDG, A_SYDG,  // fixed one-qubit gates on register bit j
  A_T, A_TDG, A_Z, A_P0, A_P1,      // diagonal on register bit j
  A_CZ,         // -1 where register bits j and k are both 1
  A_PEQ,        // 0 where register bits j and k differ
  A_PHASE,      // every element times w^arg, w = e^{i pi/4}
  A_ZERO,       // every element set to 0
  A_COUNT
};

// One device op.  It acts only where (G0 & cmask) == cval, G0 being the global index
// of the group's element 0 (all register bits zero): conditions on qubits that are not
// register bits of the stage (the other tile qubits and the tile's fixed qubits).  In a
// packed plan the same condition reads (W & wmask) == wval on the thread's condition
// word W = tile_id << group_bits | group index (one bit per fixed qubit of the thread),
// and the first 16 bytes hold all the packed kernel reads.
struct DevOp {
  uint8_t code;  // flat dispatch code of the kernel the plan is built for (Code / PCode)
  uint8_t arg;
  uint8_t act, j, k;
  uint8_t pad[3];
  uint32_t wmask, wval;
  uint64_t cmask, cval;
};

// Flat dispatch codes: one switch in the kernel selects both the action and the
// register bit(s), so each op costs one indirect branch.  Code numbers the ops of the
// unpacked tile kernels (five register slots); PCode those of the packed plain kernel.
enum Code : uint8_t {
  C_PAIR = 0,     // + 5*g + j, g in {H, SX, SY, SXDG, SYDG}       (0..24)
  C_DIAG = 25,    // + 5*d + j, d in {T, TDG, Z, P0, P1}            (25..49)
  C_CZ = 50,      // + 5*j + k                                       (50..74)
  C_PEQ = 75,     // + 5*j + k                                       (75..99)
  C_PHASE = 100,  // scalar phase w^arg of the whole group (accumulated, applied once)
  C_ZERO = 101,   // the whole group becomes zero
  C_U = 102,      // + j, general 2x2                                 (102..106)
  C_COUNT = 107
};

// Packed plan (PF_PACKED): a thread holds 32 pairs of amplitudes that differ only in
// tile bit 0 (the pack bit), each pair as two float2 = (re, re'), (im, im') that the
// packed f32x2 instructions update together.  Register slots 0..4 are the stage's
// other register bits, slot 5 is the pack bit.  Two-qubit codes have j < k.
constexpr int kPackSlot = 5;
enum PCode : uint8_t {
  P_PAIR = 0,     // + 6*g + j, g in {H, SX, SY, SXDG, SYDG}       (0..29)
  P_DIAG = 30,    // + 6*d + j, d in {T, TDG, Z, P0, P1}            (30..59)
  P_CZ = 60,      // + 6*j + k                                       (60..95)
  P_PEQ = 96,     // + 6*j + k                                       (96..131)
  P_PHASE = 132,  // scalar phase w^arg (accumulated, applied once)
  P_ZERO = 133,   // the whole group becomes zero
  P_U = 134,      // + j, general 2x2                                 (134..139)
  P_SCALE = 140,   // every element times 2^-arg (deferred scalars of square roots)
  P_GLOBAL = 141,  // every element times e^{i pi q/4} 2^{-u/2}, arg = q + 8 u (plan end)
  P_COUNT = 142
};
// A packed plan applies the square roots as unscaled rotations (norm sqrt2 each) and
// defers their scalars e^{+-i pi/4} 2^{-1/2}: two of the factors 2^{-1/2} make one factor
// 1/2, of which a stage holds at most kMaxDeferred pending (a P_SCALE op applies them),
// the rest is DevStage::halves; an odd factor 2^{-1/2} and the phases are carried to the
// end of the plan (one P_GLOBAL op).
constexpr int kMaxDeferred = 64;

// Stage group addressing: group index g of a thread -> (tile-local index L0, global
// index offset G0) of its element 0 = entry[g & 15] ^ entry[16 + ((g >> 4) & 15)] ^
// entry[32 + (g >> 8)]; kGroupEntries per stage.  In a packed plan L is the swizzled
// shared-memory byte offset of the element's pair (the swizzle is linear over XOR), and
// entries kRegEntry + j hold, in L, the byte-offset mask of register slot j.
struct DevGroupEntry {
  uint32_t L;
  uint32_t pad;
  uint64_t G;
};
constexpr int kGroupEntries = 56;
constexpr int kRegEntry = 48;
static_assert(sizeof(DevOp) == 32, "DevOp layout");

constexpr int kMaxTileBits = 14;  // the plan-specialised kernels; the others take <= 13
constexpr int kMaxReg = 5;

struct DevStage {
  uint8_t r;                   // register bits in use (<= kMaxReg); the rest are padding
  uint8_t rbit[kMaxReg];       // tile-local bit of register bit j (all distinct, padded)
  uint8_t nonr[12];            // tile-local bits of the group index, lane bits first
  uint8_t halves;              // packed plan: factors 1/2 left to apply at the stage's end
  uint8_t diag_only;           // no inner gates: nothing for the tensor cores
  uint32_t op_begin;           // into the plan's op array
  uint16_t op_count;
  uint8_t unitary;             // fused path: the inner gates contain no projector
  uint8_t pad1;
  uint32_t mat_begin;          // fused path: offset of this stage's unitary (floats)
};
static_assert(sizeof(DevStage) == 32, "DevStage layout");

enum PassFlags : uint8_t {
  PF_INIT_UNIFORM = 1,  // tile content is 2^{-n/2} everywhere; nothing is read
  PF_INIT_ZERO = 2,     // tile content is |0..0>; nothing is read
  PF_UNITARY = 4,       // no projector in the pass: every tile keeps its norm
  PF_PACKED = 8,        // packed plan: stages of tile bit 0 + up to rk bits, PCode ops
  PF_RAW = 16,          // tensor-core pass: the tiles' norms are not restored
};

struct DevPass {
  uint8_t m, c, flags, n;
  uint8_t tq[kMaxTileBits];   // tile-local bit -> global qubit (tq[i] = i for i < c)
  uint8_t nt;                 // number of non-tile qubits (n - m)
  uint8_t ntq[64];            // non-tile qubits, ascending (tile index bit -> qubit)
  uint16_t stage_count;
  uint32_t stage_begin;       // into the plan's stage array
  float init_amp;             // uniform amplitude for PF_INIT_UNIFORM
};
static_assert(sizeof(DevPass) == 96, "DevPass layout");

}  // namespace svp

namespace svk {

// Plan as laid out in device memory (one allocation, arrays back to back).
struct DevPlanView {
  const svp::DevPass *passes;
  const svp::DevStage *stages;
  const svp::DevOp *ops;
  const float *mats;
  int *err;  // error word of the plan (0 = ok; set by a kernel whose bounded wait gave up)
  const svp::DevGroupEntry *gtab;  // kGroupEntries group-addressing entries per stage
};

}  // namespace svk

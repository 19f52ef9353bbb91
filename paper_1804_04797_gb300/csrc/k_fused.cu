// Fused tile pass on the tcgen05 tensor cores (split precision, fp32 accumulation).
//
// Same passes and tiles as the plain kernel, but each stage's gates on its five
// register qubits are applied as ONE 32x32 complex unitary U (multiplied out on the
// host in fp64 from the gates, the "bunch of gates" of §2.3 as a matrix), i.e. a real
// GEMM per tile:
//     D[row, 2t+c'] = sum_{s,c} A[row, 2s+c] * B[2t+c', 2s+c],
//     A = the tile's amplitudes, one row per group of 32 (register bits = column index s),
//     B = [[Re U, -Im U], [Im U, Re U]] interleaved (64 x 64).
// Two operand formats, same three products (hi*hi + hi*lo + lo*hi, accumulated in fp32 in
// tensor memory; the dropped lo*lo term is ~2^-22 relative):
//   TF32x3  hi = x rounded to the nearest TF32, lo = (x - hi) rounded likewise; K = 8 per
//           MMA instruction.
//   F16x3   the same split in fp16 (the same 11-bit significand as TF32), twice the tensor
//           rate and K = 16 per instruction, half the operand bytes.  fp16's range is
//           handled by scaling: every row by a power of two bringing its largest component
//           near 2^6 (exact; U acts within a row, so the scale is undone after the MMA) and
//           B by 2^8 (keeps the small lo parts normal).
// Data movement per stage: each thread gathers its row (32 amplitudes) from the shared
// tile, splits it and stores A_hi/A_lo into TMEM (its own lane); one thread issues the MMAs
// (A from TMEM, B from shared memory) and commits them to an mbarrier; every thread then
// loads its row of D back from TMEM, applies the stage's diagonal epilogue (gates that
// touch a non-register qubit) and scatters the row back into the shared tile.  B (hi and
// lo) is streamed from the plan in global memory by TMA bulk copies into two shared
// buffers, one stage ahead.
// All waits are bounded: a wait that gives up sets the error word, the CTA stops issuing
// work, drains its outstanding copies and MMAs (bounded), frees its TMEM and returns.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "capi_util.h"
#include "state.h"
// this file: 5-qubit stages (32x32 unitaries); k_fused4.cu: 4-qubit stages
#define SV_TILE_R 5
#define SV_TILE_NS tile
#define SV_FUSED_LAUNCH launch_fused_pass_r5
#include "k_fused_impl.cuh"

namespace svk {

bool fused_supported() {
  static int cached = -1;
  if (cached < 0) {
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cached = (major == 10 && minor == 3) ? 1 : 0;
  }
  return cached == 1;
}

cudaError_t launch_fused_pass_r4(float2 *psi, int n, const DevPlanView &plan, int pass_index, const svp::DevPass &hp,
                                 cudaStream_t st, bool f16);

cudaError_t launch_fused_pass(float2 *psi, int n, const DevPlanView &plan, int pass_index, const svp::DevPass &hp,
                              cudaStream_t st, bool f16, int r) {
  if (r == 5 && (hp.m == 12 || hp.m == 13)) return launch_fused_pass_r5(psi, n, plan, pass_index, hp, st, f16);
  if (r == 4 && hp.m == 12) return launch_fused_pass_r4(psi, n, plan, pass_index, hp, st, f16);
  return cudaErrorInvalidValue;
}

}  // namespace svk

namespace svc {

// Nearest TF32 value of a finite float, ties away from zero (the host twin of tf32_rn).
static float tf32_round_host(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  b = (b + 0x1000u) & 0xFFFFE000u;
  float y;
  std::memcpy(&y, &b, 4);
  return y;
}

// Stage unitaries as split B operands in the kernel's shared-memory layout: per stage the
// hi part then the lo part, each 64 x 64 (TF32: fp32 words; F16: fp16 halves, B x 2^8).
// Byte offset of element (row, k) of a kK x kK B part in the K-major canonical layout
// without swizzle: 8-row x 16-byte core matrices, K-adjacent ones 128 B apart, row groups
// kK * esize * 8 B apart (the kernels' Fmt::b_off for their kK).
static uint32_t b_offset(int row, int k, int kK, bool f16) {
  const int per16 = f16 ? 8 : 4;  // elements per 16 bytes
  return (uint32_t)((((row >> 3) * (kK / per16) + (k / per16)) * 128) + (row & 7) * 16 + (k % per16) * (f16 ? 2 : 4));
}

sv_status build_stage_mats(svp::Plan *P, const std::vector<svp::Gate> &g, int r, bool f16) {
  if (r != 5 && r != 4) return fail(SV_ERR_ARG, "fused path: fuse_k must be 4 or 5");
  P->mats.clear();
  std::vector<double> u;
  const int d = 1 << r, kK = 2 * d;
  const int part_bytes = kK * kK * (f16 ? 2 : 4);
  const size_t stage_floats = (size_t)2 * part_bytes / 4;
  const double bscale = f16 ? std::ldexp(1.0, svk::kF16BExp) : 1.0;
  for (size_t s = 0; s < P->stages.size(); ++s) {
    svp::DevStage &ds = P->stages[s];
    if (P->stage_gates[s].empty()) {
      ds.diag_only = 1;
      continue;
    }
    ds.diag_only = 0;
    ds.unitary = 1;
    for (int gi : P->stage_gates[s]) {
      const int k = g[gi].kind;
      if (k == svp::K_P0 || k == svp::K_P1 || k == svp::K_PEQ) ds.unitary = 0;
    }
    svp::stage_unitary(*P, g, (int)s, r, &u);
    const size_t off = P->mats.size();
    ds.mat_begin = (uint32_t)off;
    P->mats.resize(off + stage_floats, 0.f);
    char *hi = reinterpret_cast<char *>(P->mats.data() + off);
    char *lo = hi + part_bytes;
    for (int t = 0; t < d; ++t) {
      for (int sidx = 0; sidx < d; ++sidx) {
        const double ur = u[2 * ((size_t)t * d + sidx)], ui = u[2 * ((size_t)t * d + sidx) + 1];
        const double b[2][2] = {{ur, -ui}, {ui, ur}};  // [c'][c]
        for (int cp = 0; cp < 2; ++cp) {
          for (int c = 0; c < 2; ++c) {
            const double x = b[cp][c] * bscale;
            const int row = 2 * t + cp, col = 2 * sidx + c;
            if (f16) {
              const __half h = __float2half_rn((float)x);
              const __half l = __float2half_rn((float)(x - (double)__half2float(h)));
              const uint32_t o = b_offset(row, col, kK, true);
              std::memcpy(hi + o, &h, 2);
              std::memcpy(lo + o, &l, 2);
            } else {
              const float h = tf32_round_host((float)x);
              const float l = tf32_round_host((float)(x - (double)h));
              const uint32_t o = b_offset(row, col, kK, false);
              std::memcpy(hi + o, &h, 4);
              std::memcpy(lo + o, &l, 4);
            }
          }
        }
      }
    }
  }
  return SV_OK;
}

// The same for the matrix stages of the pipelined plan kernels (packed plans): a stage's
// 5-qubit unitary U (matrix bit 0 = tile bit 0, bit j + 1 = register slot j) as B[k][n]
// with k, n = 32 * (re/im) + j, i.e. [[Re U^T, Im U^T], [-Im U^T, Re U^T]], stored as rows
// n of K in the K-major layout; per matrix stage the hi part, then the lo part.
sv_status build_stage_mats_packed(svp::Plan *P, const std::vector<svp::Gate> &g, bool f16) {
  P->mats.clear();
  std::vector<double> u;
  constexpr int d = 32, kK = 64;
  const int part_bytes = kK * kK * (f16 ? 2 : 4);
  const size_t stage_floats = (size_t)2 * part_bytes / 4;
  // (unscaled: the matrix-stage kernel keeps each tile at one scale through its stages)
  const double bscale = 1.0;
  for (size_t s = 0; s < P->stages.size(); ++s) {
    svp::DevStage &ds = P->stages[s];
    ds.unitary = 1;
    if (P->stage_gates[s].empty()) {
      ds.diag_only = 1;
      continue;
    }
    ds.diag_only = 0;
    for (int gi : P->stage_gates[s]) {
      const int k = g[gi].kind;
      if (k == svp::K_P0 || k == svp::K_P1 || k == svp::K_PEQ) ds.unitary = 0;
    }
    svp::stage_unitary(*P, g, (int)s, 5, &u);
    const size_t off = P->mats.size();
    ds.mat_begin = (uint32_t)off;
    P->mats.resize(off + stage_floats, 0.f);
    char *hi = reinterpret_cast<char *>(P->mats.data() + off);
    char *lo = hi + part_bytes;
    for (int jo = 0; jo < d; ++jo) {
      for (int ji = 0; ji < d; ++ji) {
        const double ur = u[2 * ((size_t)jo * d + ji)], ui = u[2 * ((size_t)jo * d + ji) + 1];
        const double b[2][2] = {{ur, ui}, {-ui, ur}};  // [re/im of the input k][re/im of the output n]
        for (int ri = 0; ri < 2; ++ri) {
          for (int ro = 0; ro < 2; ++ro) {
            const double x = b[ri][ro] * bscale;
            const int n = 32 * ro + jo, k = 32 * ri + ji;
            const uint32_t o = b_offset(n, k, kK, f16);
            if (f16) {
              const __half h = __float2half_rn((float)x);
              const __half l = __float2half_rn((float)(x - (double)__half2float(h)));
              std::memcpy(hi + o, &h, 2);
              std::memcpy(lo + o, &l, 2);
            } else {
              const float h = tf32_round_host((float)x);
              const float l = tf32_round_host((float)(x - (double)h));
              std::memcpy(hi + o, &h, 4);
              std::memcpy(lo + o, &l, 4);
            }
          }
        }
      }
    }
  }
  return SV_OK;
}

}  // namespace svc

// The fused tensor-core tile pass with 4-qubit stages: 16x16 complex stage unitaries,
// 32x32 real B operands, rows of 16 amplitudes (two M = 128 blocks per 12-qubit tile).
// The kernel is k_fused_impl.cuh (method: k_fused.cu) at this width.
#define SV_TILE_R 4
#define SV_TILE_NS tile4
#define SV_FUSED_LAUNCH launch_fused_pass_r4
#include "k_fused_impl.cuh"

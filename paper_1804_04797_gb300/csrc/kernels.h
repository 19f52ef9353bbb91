// Host-side launchers of the CUDA kernels (implemented in the .cu files).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "plan.h"

namespace svk {

struct Mat2 {
  float v[8];  // a, b, c, d as (re, im)
};


// K0: write |0..0> (uniform == false) or the uniform 2^{-n/2} state.  Write-only.
cudaError_t launch_init(float2 *psi, int n, bool uniform, float amp, cudaStream_t st);

// K1/K2/K3 plain tile pass: one sweep over all tiles of one pass of a packed plan.
// host_pass is the host copy of the same pass (tile shape, flags).
cudaError_t launch_tile_pass(float2 *psi, int n, const DevPlanView &plan, int pass_index,
                             const svp::DevPass &host_pass, cudaStream_t st);
// Register slots besides the pack bit of the packed plain kernel (the planner's rk).
int tile_pass_register_slots();
// Largest tile (qubits) of the interpreting plain kernel; the plan-specialised kernels
// take up to svp::kMaxTileBits.
int tile_pass_max_bits();

// K4 fused tensor-core tile pass (tcgen05, split-TF32 or split-FP16).
// r = register qubits of a stage: 5 (tile_bits 12 or 13) or 4 (tile_bits 12); f16: F16x3
// operands, else TF32x3
cudaError_t launch_fused_pass(float2 *psi, int n, const DevPlanView &plan, int pass_index,
                              const svp::DevPass &host_pass, cudaStream_t st, bool f16, int r);
cudaError_t launch_fused_pass_r5(float2 *psi, int n, const DevPlanView &plan, int pass_index,
                                 const svp::DevPass &host_pass, cudaStream_t st, bool f16);
bool fused_supported();

// Per-gate sweeps (K2 one-qubit pair update, K3 diagonal factor on a bit pattern).
cudaError_t launch_gate_1q(float2 *psi, int n, int q, const Mat2 &u, cudaStream_t st);
// amplitudes whose bits under mask equal val are multiplied by (fr + i fi)
cudaError_t launch_gate_diag(float2 *psi, int n, uint64_t mask, uint64_t val, float fr, float fi,
                             cudaStream_t st);

// K5 reductions.  partials: scratch of at least reduce_partials_needed() doubles*2.
int reduce_partials_needed();
cudaError_t launch_norm(const float2 *psi, int n, double *partials, double *out2,
                        cudaStream_t st);
// The second level of launch_norm alone: out2 = the sums of count partial pairs (fixed
// order), e.g. the per-CTA sums a plan kernel's last pass wrote.
cudaError_t launch_norm_final(const double *partials, int count, double *out2, cudaStream_t st);
// out[2j], out[2j+1] = re, im of psi[bits[j]]
cudaError_t launch_gather(const float2 *psi, const uint64_t *bits, int64_t m, double *out,
                          cudaStream_t st);
// out[j] = |psi[bits[j]]|^2
cudaError_t launch_gather_prob(const float2 *psi, const uint64_t *bits, int64_t m, double *out,
                               cudaStream_t st);

// K6: out[2j..2j+1] = scale * sum_l A[xa_j + (l << nA)] * B[xb_j + (l << nB)], fp64.
cudaError_t launch_branch_sum(const float2 *A, int nA, const float2 *B, int nB, int t, const uint64_t *xa,
                              const uint64_t *xb, int m, double scale, double *out, cudaStream_t st);

int device_sm_count();

// Fork of a branch tree: psi[i + (c << n_cur)] = 2^{-(n_new - n_cur)/2} psi[i] for every
// slice c of the branch bits n_cur..n_new-1 (they were |+> until now), in place.
cudaError_t launch_fork(float2 *psi, int n_cur, int n_new, cudaStream_t st);

// Full state from two batched half-states (Eqs. 6-7): out[x_A + (x_B << nA)] = scale *
// sum_l A[x_A + (l << nA)] B[x_B + (l << nB)] over 2^t branches (fp32).
// The same product on the tensor cores (TF32x3, k_outer_tc.cu): half states of >= 7
// qubits; scratch: outer_sum_tc_scratch bytes of device memory for the operand images;
// err: a device int set non-zero if a bounded wait gave up.
bool outer_sum_tc_supported(int nA, int nB, int t);
size_t outer_sum_tc_scratch(int nA, int nB, int t);
cudaError_t launch_outer_sum_tc(const float2 *A, int nA, const float2 *B, int nB, int t, float scale, float2 *out,
                                void *scratch, int *err, cudaStream_t st);
cudaError_t launch_outer_sum(const float2 *A, int nA, const float2 *B, int nB, int t, float scale, float2 *out,
                             cudaStream_t st);

// <a|b> = sum conj(a_i) b_i of two 2^n states: out2 = (re, im), fp64 (partials: 2 *
// reduce_partials_needed() doubles of scratch).
cudaError_t launch_inner(const float2 *a, const float2 *b, int n, double *partials, double *out2, cudaStream_t st);
// The basis state |x>: zero everywhere, 1 at index x.
cudaError_t launch_basis_state(float2 *psi, int n, uint64_t x, cudaStream_t st);

}  // namespace svk

// Plain (fp32 CUDA-core) tile pass.
//
// One launch = one pass of the plan = one read and one write of every amplitude.
// Each CTA loops over gathered tiles: the 2^m amplitudes whose indices differ only in
// the pass's m tile qubits (the c lowest qubits are always among them, so the tile is
// 2^(m-c) contiguous chunks of 2^c amplitudes and every global access is a coalesced
// 16-byte vector).  The tile is staged in shared memory (the on-chip copy of the
// paper's "local qubits" in LDM, §2.3) and every gate of the pass is applied to it:
// stage by stage, each thread pulls the 32 amplitudes that differ in the stage's five
// qubits (qubit 0, the pack bit, and four register qubits) into registers as 16 packed
// pairs (width 4 measured 4 % faster than 5: twice the resident warps), applies the stage's gates there (the pair update of §2 with packed fp32x2
// arithmetic; diagonal gates as signs, phases and projector factors, conditioned on the
// thread's other index bits), and writes them back.
#include <cuda_runtime.h>

#include "kernels.h"
#define SV_PACK_R 4
#include "tile_pack.cuh"

namespace svk {
namespace {

using namespace tpk;

constexpr int kMaxBits = 13;  // tiles of this kernel: 64 KiB, two CTAs per SM
constexpr int kThreads = 1 << (kMaxBits - 1 - kPR);  // one group of 2^kPR pairs per thread

__global__ void __launch_bounds__(kThreads, 2)
tile_pass_kernel(float2 *__restrict__ psi, DevPlanView plan, int pass_index, uint64_t num_tiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DevPass P;
  __shared__ uint64_t chunk_off[1 << 10];

  const int tid = threadIdx.x;
  if (tid == 0) P = plan.passes[pass_index];
  __syncthreads();
  build_chunk_table(P, chunk_off);
  __syncthreads();
  sweep_tiles(psi, plan, P, chunk_off, reinterpret_cast<float4 *>(smem_raw), blockIdx.x, gridDim.x, num_tiles);
}

int g_tile_blocks_per_sm[kMaxBits + 1] = {};  // resident CTAs per SM, by tile size

}  // namespace

int tile_pass_register_slots() { return kPR; }
int tile_pass_max_bits() { return kMaxBits; }

cudaError_t launch_tile_pass(float2 *psi, int n, const DevPlanView &plan, int pass_index,
                             const svp::DevPass &hp, cudaStream_t st) {
  const int m = hp.m;
  if (!(hp.flags & svp::PF_PACKED) || m < kPR + 1 || m > kMaxBits || hp.c < 1 || m - hp.c > 10)
    return cudaErrorInvalidValue;
  const size_t smem = sizeof(float2) << m;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(tile_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float2) << kMaxBits));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int threads = 1 << (m - 1 - kPR);
  if (g_tile_blocks_per_sm[m] == 0) {
    int q = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, tile_pass_kernel, threads, smem);
    if (e != cudaSuccess) return e;
    g_tile_blocks_per_sm[m] = q < 1 ? 1 : q;
  }
  const uint64_t tiles = 1ull << (n - m);
  uint64_t grid = (uint64_t)device_sm_count() * (uint64_t)g_tile_blocks_per_sm[m];
  if (grid > tiles) grid = tiles;
  tile_pass_kernel<<<(unsigned)grid, threads, smem, st>>>(psi, plan, pass_index, tiles);
  return cudaGetLastError();
}

}  // namespace svk

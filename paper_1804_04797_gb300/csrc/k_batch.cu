// K7: the uneven batch in one persistent launch.
//
// Every CTA repeatedly takes the next item (one tile of one pass of one circuit) from a
// global counter and runs the plain tile pass on it.  Before an item of pass p it waits
// until every tile of pass p-1 of the same circuit is done (a per-circuit-pass counter),
// with a bounded spin: a wait that gives up sets the error word and the CTA leaves.  The
// queue holds all circuits' first passes, then all second passes, ..., so the waits are
// rare and short.  The state is read through L2 only (cp.async.cg), because other CTAs
// of the same launch wrote it and L1 is not coherent across SMs.  The tile pass is the
// packed interpreter of the single-circuit path (tile_pack.cuh).
#include <cuda_runtime.h>

#include "batch.h"
#include "kernels.h"
#define SV_PACK_R 4
#include "tile_pack.cuh"

namespace svk {
namespace {

using namespace tpk;

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int load_acquire(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(256, 2)
batch_kernel(float2 *__restrict__ states, DevPlanView plan, const BatchCP *__restrict__ cps,
             const BatchItem *__restrict__ items, uint64_t n_items, unsigned int *words,
             unsigned long long wait_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4 *tile = reinterpret_cast<float4 *>(smem_raw);
  __shared__ DevPass P;
  __shared__ uint64_t chunk_off[1 << 10];
  __shared__ unsigned int s_item;
  __shared__ int s_stop;
  const int tid = threadIdx.x;
  unsigned int *done = words + kBatchHeader;
  uint32_t cur_cp = kNoPrev;
  for (;;) {
    if (tid == 0) {
      s_item = atomicAdd(&words[0], 1u);
      s_stop = 0;
    }
    __syncthreads();
    const unsigned int idx = s_item;
    if (idx >= n_items) break;
    const BatchItem it = items[idx];
    const BatchCP cp = cps[it.cp];
    if (it.cp != cur_cp) {
      if (tid == 0) P = plan.passes[cp.pass];
      __syncthreads();
      build_chunk_table(P, chunk_off);
      cur_cp = it.cp;
    }
    if (tid == 0 && cp.prev != kNoPrev) {
      const unsigned int need = cps[cp.prev].tiles;
      if (load_acquire(&done[cp.prev]) < need) {
        const unsigned long long t0 = now_ns();
        while (load_acquire(&done[cp.prev]) < need) {
          if (now_ns() - t0 > wait_ns) {
            atomicExch(&words[1], 1u);
            s_stop = 1;
            break;
          }
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    float2 *psi = states + cp.state_off;
    if (!(P.flags & (svp::PF_INIT_UNIFORM | svp::PF_INIT_ZERO))) {
      load_tile_async(psi, tile, P, chunk_off, tile_base(P, it.tile));
      finish_tile_load(tile);
      __syncthreads();
    }
    process_tile(psi, plan, P, chunk_off, tile, it.tile);
    __threadfence();  // each thread's stores visible device-wide before the count
    __syncthreads();
    if (tid == 0) atomicAdd(&done[it.cp], 1u);
  }
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__global__ void batch_stats_partial(const float2 *__restrict__ states, const BatchChunk *__restrict__ chunks,
                                    double *partials) {
  const BatchChunk ch = chunks[blockIdx.x];
  // two amplitudes per 16-byte load: chunk starts and lengths are even (every circuit
  // has at least 2^6 amplitudes, chunks are 2^16); eight probabilities are added in
  // fp32, then into the fp64 sums (fp64 per element is the slow part on this GPU)
  const float4 *p = reinterpret_cast<const float4 *>(states + ch.start);
  const uint32_t n4 = ch.len >> 1, stride = blockDim.x;
  double s2 = 0, s4 = 0;
  uint32_t i = threadIdx.x;
  for (; i + 3 * stride < n4; i += 4 * stride) {
    float4 z[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] = p[i + k * stride];
    float a2 = 0.f, a4 = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float p0 = fmaf(z[k].x, z[k].x, z[k].y * z[k].y);
      const float p1 = fmaf(z[k].z, z[k].z, z[k].w * z[k].w);
      a2 += p0 + p1;
      a4 = fmaf(p0, p0, fmaf(p1, p1, a4));
    }
    s2 += a2;
    s4 += a4;
  }
  for (; i < n4; i += stride) {
    const float4 z = p[i];
    const float p0 = fmaf(z.x, z.x, z.y * z.y);
    const float p1 = fmaf(z.z, z.z, z.w * z.w);
    s2 += (double)(p0 + p1);
    s4 += (double)fmaf(p0, p0, p1 * p1);
  }
  __shared__ double r2[8], r4[8];
  s2 = warp_sum(s2);
  s4 = warp_sum(s4);
  if ((threadIdx.x & 31) == 0) { r2[threadIdx.x >> 5] = s2; r4[threadIdx.x >> 5] = s4; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += r2[w]; b += r4[w]; }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

__global__ void batch_stats_final(const double *partials, const int *chunk_begin, int n_circuits, double *stats) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_circuits) return;
  double a = 0, b = 0;
  for (int k = chunk_begin[c]; k < chunk_begin[c + 1]; ++k) { a += partials[2 * k]; b += partials[2 * k + 1]; }
  stats[2 * c] = a;
  stats[2 * c + 1] = b;
}

}  // namespace

int batch_block_threads(int m) { return 1 << (m - 1 - kPR); }

cudaError_t launch_batch(float2 *states, const DevPlanView &plan, const BatchCP *cps, const BatchItem *items,
                         uint64_t n_items, unsigned int *words, int m, cudaStream_t st,
                         unsigned long long wait_ns, int max_grid) {
  static bool configured = false;
  static int per_sm = 1;
  const size_t smem = sizeof(float2) << 13;  // tiles of <= 13 qubits (capi_batch)
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, 256, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    configured = true;
  }
  const int threads = batch_block_threads(m);
  // smaller tiles use fewer threads: more CTAs fit, but the occupancy query for 256
  // threads is a safe lower bound
  int grid = device_sm_count() * per_sm * (256 / threads);
  if (max_grid > 0 && grid > max_grid) grid = max_grid;
  batch_kernel<<<grid, threads, sizeof(float2) << m, st>>>(states, plan, cps, items, n_items, words, wait_ns);
  return cudaGetLastError();
}

cudaError_t launch_batch_stats(const float2 *states, const BatchChunk *chunks, int n_chunks, double *partials,
                               const int *chunk_begin, int n_circuits, double *stats, cudaStream_t st) {
  if (n_chunks > 0) batch_stats_partial<<<n_chunks, 256, 0, st>>>(states, chunks, partials);
  batch_stats_final<<<(n_circuits + 127) / 128, 128, 0, st>>>(partials, chunk_begin, n_circuits, stats);
  return cudaGetLastError();
}

}  // namespace svk

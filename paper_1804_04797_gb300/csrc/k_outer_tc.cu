// The tensor form of the cut decomposition on the tcgen05 tensor cores (Eqs. 6-7):
//     psi_AB[x_A + 2^nA x_B] = scale * sum_l A_l[x_A] B_l[x_B],
// i.e. the complex product Psi = Bm Am^T of the half-states' branch matrices Bm (2^nB x L)
// and Am (2^nA x L), L = 2^t summed branches, as one real GEMM with K = 2L:
//     D[x_B, 2 x_A + o] = sum_{l, c} Aop[x_B, 2l + c] Bop[2 x_A + o, 2l + c],
//     Aop[x_B, 2l + c] = (Re, Im)_c B_l[x_B],
//     Bop[2 x_A, 2l + c] = (Re A_l[x_A], -Im A_l[x_A])_c,  Bop[2 x_A + 1, 2l + c] = (Im, Re)_c,
// so a row of D is a contiguous run of output amplitudes (re, im interleaved).  TF32x3:
// each operand is split into hi + lo (nearest TF32 values) and D = Ahi Bhi + Ahi Blo +
// Alo Bhi is accumulated in fp32 in tensor memory (the lo*lo term is ~2^-22 relative).
//
// A prep kernel writes the split operands as images in the MMA's shared-memory layout
// (K-major, no swizzle: 8-row x 16-byte core matrices), one contiguous block per (row tile,
// 32-wide K chunk), so a CTA fetches each with one bulk copy.  The GEMM kernel is
// persistent (two CTAs per SM: one stores its tile while the other computes): per output
// tile of 128 x 128 amplitudes it loads the blocks of every K chunk, one thread issues the
// 3 x 4 MMAs (M = 128, N = 256, K = 8) per chunk, and the warps move D from tensor memory
// through shared memory to HBM in whole 128-byte runs of the state.  All waits are bounded.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace svk {
namespace {

constexpr int kRows = 128;                         // output rows (x_B) per tile
constexpr int kCols = 128;                         // output amplitudes (x_A) per tile
constexpr int kKc = 32;                            // real K per chunk
constexpr uint32_t kABlock = kRows * kKc * 4;      // one part of an A block (16 KB)
constexpr uint32_t kBBlock = 2 * kCols * kKc * 4;  // one part of a B block (32 KB)
constexpr uint32_t kSmem = 2 * kABlock + 2 * kBBlock;
constexpr unsigned long long kWaitNs = 1000000000ull;
// kind::tf32, D fp32, A and B K-major, N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(256 >> 3) << 17) | (8u << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of (row, k) in a block of `rows` x 32 tf32 values, K-major without swizzle:
// core matrices of 8 rows x 4 values (16 B), K-adjacent ones 128 B apart, 8-row groups
// 1024 B apart.
__host__ __device__ __forceinline__ uint32_t blk_off(uint32_t row, uint32_t k) {
  return ((row >> 3) * (kKc / 4) + (k >> 2)) * 128u + (row & 7u) * 16u + (k & 3u) * 4u;
}

__device__ __forceinline__ float tf32_rn(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Operand images.  Aop: row tile rt, chunk kc at ((rt * kch + kc) * 2 + part) * kABlock;
// Bop likewise with kBBlock.  One thread per (row, k) of each operand.
__global__ void outer_prep_kernel(const float2 *__restrict__ A, int nA, const float2 *__restrict__ B, int nB, int t,
                                  int kch, unsigned char *__restrict__ aimg, unsigned char *__restrict__ bimg) {
  const uint64_t L = 1ull << t, K = (uint64_t)kch * kKc;
  const uint64_t na = 1ull << nA, nb = 1ull << nB;
  const uint64_t nA_ops = nb * K, nB_ops = 2 * na * K;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nA_ops + nB_ops;
       e += (uint64_t)gridDim.x * blockDim.x) {
    float v;
    unsigned char *dst;
    uint32_t blk;
    if (e < nA_ops) {  // Aop[x_B, k]
      const uint64_t xb = e / K, k = e % K, l = k >> 1;
      const float2 z = l < L ? B[xb + (l << nB)] : make_float2(0.f, 0.f);
      v = (k & 1) ? z.y : z.x;
      const uint64_t rt = xb / kRows, kc = k / kKc;
      dst = aimg + (rt * kch + kc) * 2 * kABlock;
      blk = kABlock;
      const uint32_t o = blk_off((uint32_t)(xb % kRows), (uint32_t)(k % kKc));
      const float h = tf32_rn(v);
      *reinterpret_cast<float *>(dst + o) = h;
      *reinterpret_cast<float *>(dst + blk + o) = tf32_rn(v - h);
    } else {  // Bop[n, k], n = 2 x_A + o
      const uint64_t f = e - nA_ops, n = f / K, k = f % K, l = k >> 1;
      const uint64_t xa = n >> 1;
      const float2 z = l < L ? A[xa + (l << nA)] : make_float2(0.f, 0.f);
      const bool im_out = n & 1, im_in = k & 1;
      v = !im_out ? (im_in ? -z.y : z.x) : (im_in ? z.x : z.y);
      const uint64_t ct = n / (2 * kCols), kc = k / kKc;
      dst = bimg + (ct * kch + kc) * 2 * kBBlock;
      blk = kBBlock;
      const uint32_t o = blk_off((uint32_t)(n % (2 * kCols)), (uint32_t)(k % kKc));
      const float h = tf32_rn(v);
      *reinterpret_cast<float *>(dst + o) = h;
      *reinterpret_cast<float *>(dst + blk + o) = tf32_rn(v - h);
    }
  }
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;   // K-adjacent core matrices
  d |= (uint64_t)(1024 >> 4) << 32;  // 8-row groups
  d |= (uint64_t)1 << 46;
  return d;
}
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(d), "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
               : "=r"(ok)
               : "r"(smem_u32(bar)), "r"(parity)
               : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  do {
    if (mbar_try(bar, parity)) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  } while (t - t0 < kWaitNs);
  return false;
}

__global__ void __launch_bounds__(128, 2)
outer_mma_kernel(const unsigned char *__restrict__ aimg, const unsigned char *__restrict__ bimg, int rtiles, int ctiles,
                 int kch, int nA, float scale, float2 *__restrict__ out, int *err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char *sa = sm, *sb = sm + 2 * kABlock;
  __shared__ __align__(8) uint64_t load_bar, mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int stop;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&load_bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    stop = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  uint32_t lph = 0, mph = 0;  // parities of the two barriers
  bool load_out = false, mma_out = false;  // tid 0: a copy / products not yet waited for
  const uint64_t ntiles = (uint64_t)rtiles * ctiles;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t rt = tile / ctiles, ct = tile % ctiles;
    for (int kc = 0; kc < kch; ++kc) {
      if (tid == 0) {
        const uint32_t lb = smem_u32(&load_bar);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(lb), "r"(kSmem) : "memory");
        const unsigned char *ga = aimg + (rt * kch + kc) * 2 * kABlock;
        const unsigned char *gb = bimg + (ct * kch + kc) * 2 * kBBlock;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(sa)), "l"(ga), "r"(2 * kABlock), "r"(lb) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(sb)), "l"(gb), "r"(kBBlock), "r"(lb) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(sb + kBBlock)), "l"(gb + kBBlock), "r"(kBBlock), "r"(lb) : "memory");
        load_out = true;
        bool ok = mbar_wait(&load_bar, lph);
        if (ok) {
          load_out = false;
          lph ^= 1;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t ah = sdesc(smem_u32(sa)), al = sdesc(smem_u32(sa + kABlock));
          const uint64_t bh = sdesc(smem_u32(sb)), bl = sdesc(smem_u32(sb + kBBlock));
          // one K step = 8 tf32 values = two 128-byte core matrices (+256 B = +16)
#pragma unroll
          for (int k = 0; k < kKc / 8; ++k) mma_ss(tmem, al + 16 * k, bh + 16 * k, kc > 0 || k > 0);
#pragma unroll
          for (int k = 0; k < kKc / 8; ++k) mma_ss(tmem, ah + 16 * k, bl + 16 * k, 1);
#pragma unroll
          for (int k = 0; k < kKc / 8; ++k) mma_ss(tmem, ah + 16 * k, bh + 16 * k, 1);
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       ::"r"(smem_u32(&mma_bar)) : "memory");
          mma_out = true;
          ok = mbar_wait(&mma_bar, mph);
          if (ok) {
            mma_out = false;
            mph ^= 1;
          }
        }
        if (!ok) {
          atomicExch(err, 1);
          stop = 1;
        }
      }
      __syncthreads();
      if (stop) break;
    }
    if (stop) break;
    // D to the state: each warp holds 32 rows (x_B = rt * 128 + 32 warp + lane, one per
    // lane); per 32-column chunk the lanes write their rows into shared memory (the
    // operand buffers are free now: 4 KB per warp, 16-byte chunk q of row r at q ^ (r & 7),
    // conflict-free both ways), then the warp writes four rows' 128-byte runs per store
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
    const int lane = tid & 31;
    float4 *stg = reinterpret_cast<float4 *>(sa) + warp * 256;
    float2 *rows = out + (((rt * kRows + (uint64_t)(32 * warp)) << nA) + ct * kCols);
#pragma unroll 1
    for (int c = 0; c < 256; c += 32) {
      uint32_t r[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
          "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
            "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
            "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
            "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr + (uint32_t)c)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 8; ++q)
        stg[lane * 8 + (q ^ (lane & 7))] =
            make_float4(__uint_as_float(r[4 * q]) * scale, __uint_as_float(r[4 * q + 1]) * scale,
                        __uint_as_float(r[4 * q + 2]) * scale, __uint_as_float(r[4 * q + 3]) * scale);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int row = 4 * q + (lane >> 3), ch = lane & 7;
        const float4 v = stg[row * 8 + (ch ^ (row & 7))];
        *reinterpret_cast<float4 *>(rows + ((uint64_t)row << nA) + c / 2 + 2 * ch) = v;
      }
      __syncwarp();
    }
    // the next tile's products overwrite D only after every thread has read it, and its
    // bulk copies refill the staging buffer only after these generic-proxy writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  // after a wait that gave up: let the copy and the products in flight finish (bounded)
  // before the CTA's shared and tensor memory go away
  if (tid == 0 && load_out) mbar_wait(&load_bar, lph);
  if (tid == 0 && mma_out) mbar_wait(&mma_bar, mph);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  }
}

}  // namespace

bool outer_sum_tc_supported(int nA, int nB, int t) { return nA >= 7 && nB >= 7 && t >= 0 && t <= 20; }

size_t outer_sum_tc_scratch(int nA, int nB, int t) {
  const uint64_t kch = ((2ull << t) + kKc - 1) / kKc;
  return (size_t)(((1ull << nB) / kRows) * kch * 2 * kABlock + ((1ull << nA) / kCols) * kch * 2 * kBBlock);
}

cudaError_t launch_outer_sum_tc(const float2 *A, int nA, const float2 *B, int nB, int t, float scale, float2 *out,
                                void *scratch, int *err, cudaStream_t st) {
  if (!outer_sum_tc_supported(nA, nB, t)) return cudaErrorInvalidValue;
  static bool configured = false;
  if (!configured) {
    const cudaError_t e =
        cudaFuncSetAttribute(outer_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem + 1024);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int kch = (int)(((2ull << t) + kKc - 1) / kKc);
  const int rtiles = (int)((1ull << nB) / kRows), ctiles = (int)((1ull << nA) / kCols);
  unsigned char *aimg = static_cast<unsigned char *>(scratch);
  unsigned char *bimg = aimg + (size_t)rtiles * kch * 2 * kABlock;
  const uint64_t work = ((1ull << nB) + (2ull << nA)) * (uint64_t)kch * kKc;
  uint64_t pgrid = (work + 255) / 256;
  const uint64_t pmax = (uint64_t)device_sm_count() * 8;
  if (pgrid > pmax) pgrid = pmax;
  outer_prep_kernel<<<(unsigned)pgrid, 256, 0, st>>>(A, nA, B, nB, t, kch, aimg, bimg);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  uint64_t grid = (uint64_t)device_sm_count() * 2;
  const uint64_t ntiles = (uint64_t)rtiles * ctiles;
  if (grid > ntiles) grid = ntiles;
  outer_mma_kernel<<<(unsigned)grid, 128, kSmem + 1024, st>>>(aimg, bimg, rtiles, ctiles, kch, nA, scale, out, err);
  return cudaGetLastError();
}

}  // namespace svk

// Body of the fused tensor-core tile pass (see k_fused.cu for the method), compiled once
// per row width: the including file defines SV_TILE_R (register qubits of a stage: 5 or 4),
// SV_TILE_NS (the namespace of its copy of tile_common.cuh) and SV_FUSED_LAUNCH (the name
// of its launcher).  Everything else lives in an anonymous namespace of that file.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "tile_common.cuh"

namespace svk {
namespace {

using namespace SV_TILE_NS;

constexpr int kK = 2 * kE;  // real K = N = 2 * 2^kR (64 for 5-qubit stages, 32 for 4)
constexpr unsigned long long kWaitNs = 1000000000ull;  // give up a wait after 1 s

// Operand format traits.
template <bool F16>
struct Fmt;
template <>
struct Fmt<false> {  // TF32x3
  static constexpr int kAcols = kK;                 // TMEM columns of one A part per 128 rows
  static constexpr int kKsteps = kK / 8;            // MMA instructions along K
  static constexpr int kBBytes = kK * kK * 4;       // one kK x kK B part
  static constexpr uint32_t kSBO = (kK / 4) * 128;  // row-group stride of the K-major layout
  // kind::tf32: D fp32, A/B tf32, K-major, M = 128, N = kK
  static constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kK >> 3) << 17) | (8u << 24);
  __host__ __device__ static uint32_t b_off(int row, int k) {  // byte offset in a B part
    return (uint32_t)((((row >> 3) * (kK / 4) + (k >> 2)) * 128) + (row & 7) * 16 + (k & 3) * 4);
  }
};
template <>
struct Fmt<true> {  // F16x3
  static constexpr int kAcols = kK / 2;
  static constexpr int kKsteps = kK / 16;
  static constexpr int kBBytes = kK * kK * 2;
  static constexpr uint32_t kSBO = (kK / 8) * 128;
  // kind::f16: D fp32, A/B fp16, K-major, M = 128, N = kK
  static constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(kK >> 3) << 17) | (8u << 24);
  __host__ __device__ static uint32_t b_off(int row, int k) {
    return (uint32_t)((((row >> 3) * (kK / 8) + (k >> 3)) * 128) + (row & 7) * 16 + (k & 7) * 2);
  }
};
constexpr int kF16RowExp = 6;  // largest row component scaled to [2^6, 2^7)
constexpr int kF16BExp = 8;    // B scaled by 2^8

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major, no swizzle: 8-row x 16-byte core matrices, K-adjacent core matrices 128 B
// apart (leading byte offset), row-adjacent ones sbo apart (stride byte offset).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(sbo >> 4) << 32;
  d |= (uint64_t)1 << 46;  // tcgen05 descriptor version
  return d;                // base offset 0, no swizzle
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile("{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
               : "=r"(ok) : "r"(bar), "r"(phase) : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  if (mbar_try(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  while (global_ns() - t0 < kWaitNs)
    if (mbar_try(bar, phase)) return true;
  return false;
}

template <bool F16>
__device__ __forceinline__ void mma(uint32_t d, uint32_t a_tmem, uint64_t b_desc, uint32_t acc) {
  if constexpr (F16) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
                 :: "r"(d), "r"(a_tmem), "l"(b_desc), "r"(Fmt<true>::kIdesc), "r"(acc));
  } else {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
                 :: "r"(d), "r"(a_tmem), "l"(b_desc), "r"(Fmt<false>::kIdesc), "r"(acc));
  }
}

#define SV_TMEM_ST16(taddr, r)                                                                              \
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" \
               :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), \
                 "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]) : "memory")
#define SV_TMEM_LD16(taddr, r)                                                                              \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), \
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]) \
               : "r"(taddr) : "memory")

// Nearest TF32 value, ties away from zero (add half a TF32 ulp to the magnitude bits,
// clear the 13 low mantissa bits).  Both split parts are rounded this way so that each
// is exactly representable (the tensor core then drops nothing) and the residual
// x - hi - lo has no sign bias; truncating instead biases every product toward zero.
__device__ __forceinline__ float tf32_rn(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// The 32 bits of a half2 (x in the low half).
__device__ __forceinline__ uint32_t half2_bits(__half2 h) {
  return (uint32_t)__half_as_ushort(__low2half(h)) | ((uint32_t)__half_as_ushort(__high2half(h)) << 16);
}

// TMEM columns: A_hi at [kAcols mb, +kAcols), A_lo at [kAcols (MB + mb), +kAcols),
// D at [2 kAcols MB + kK mb, +kK); allocation = next power of two (at least 32).
template <int MB, bool F16>
struct Cols {
  static constexpr int kA = Fmt<F16>::kAcols;
  static constexpr uint32_t kUsed = (uint32_t)(2 * kA * MB + kK * MB);
  static constexpr uint32_t kAlloc = kUsed <= 32 ? 32 : kUsed <= 64 ? 64 : kUsed <= 128 ? 128 : (kUsed <= 256 ? 256 : 512);
  // resident CTAs per SM: the TMEM allocations that fit in 512 columns, at most three of
  // one M block and two of two (registers: 168 a thread at 5-qubit stages)
  static constexpr int kPerSm = (512 / (int)kAlloc) < (MB == 1 ? 3 : 2) ? (512 / (int)kAlloc) : (MB == 1 ? 3 : 2);
  __device__ static uint32_t a_hi(int mb) { return (uint32_t)(kA * mb); }
  __device__ static uint32_t a_lo(int mb) { return (uint32_t)(kA * (MB + mb)); }
  __device__ static uint32_t d(int mb) { return (uint32_t)(2 * kA * MB + kK * mb); }
};

// Issue the B load (hi and lo parts) of stage `st` into buffer `buf`.
template <bool F16>
__device__ __forceinline__ void issue_b_load(const float *mats, const DevStage &st, unsigned char *bbuf, int buf,
                                             uint32_t bar) {
  constexpr int kB = Fmt<F16>::kBBytes;
  const char *src = reinterpret_cast<const char *>(mats + st.mat_begin);
  const uint32_t dst = smem_u32(bbuf + buf * 2 * kB);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(2 * kB) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(dst), "l"(src), "r"(kB), "r"(bar) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(dst + kB), "l"(src + kB), "r"(kB), "r"(bar) : "memory");
}

// Sum over the warp of one double per thread; lane 0 writes it to slot[warp] (the CTA
// total is then read by every thread, in a fixed order, after a barrier).
__device__ __forceinline__ void warp_sum_to(double d, double *slot) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) slot[threadIdx.x >> 5] = d;
}
__device__ __forceinline__ double slots_sum(const double *slot) {
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += slot[w];
  return t;
}

__device__ __forceinline__ float row_norm2(const float2 (&v)[kE]) {
  float s = 0.f;
#pragma unroll
  for (int e = 0; e < kE; ++e) s = fmaf(v[e].x, v[e].x, fmaf(v[e].y, v[e].y, s));
  return s;
}

// x * (1 + delta) rounded stochastically: the RN sum plus, with probability
// |residual| / ulp, one ulp toward the residual.  Unbiased for sub-ulp delta, which
// plain rounding would drop.  u in [0, 1).
__device__ __forceinline__ float scale_sr(float x, float delta, float u) {
  const float c = x * delta;
  const float y = x + c;
  const float e = (x - y) + c;  // exact error of the sum (|x| >= |c|)
  const float ulp = __uint_as_float(__float_as_uint(y) & 0x7F800000u) * 1.1920928955078125e-7f;
  return (u * ulp < fabsf(e)) ? y + copysignf(ulp, e) : y;
}

// Scale a register row by (1 + delta) with stochastic rounding; the uniform numbers
// come from a Weyl sequence (golden-ratio increments) seeded per tile, pass and row.
__device__ __forceinline__ void scale_row(float2 (&v)[kE], float delta, uint32_t seed) {
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    const uint32_t h0 = seed + (uint32_t)(2 * e) * 0x9E3779B9u;
    const uint32_t h1 = h0 + 0x9E3779B9u;
    v[e].x = scale_sr(v[e].x, delta, (float)(h0 >> 8) * 5.9604644775390625e-8f);
    v[e].y = scale_sr(v[e].y, delta, (float)(h1 >> 8) * 5.9604644775390625e-8f);
  }
}

// A (this thread's row) into its TMEM lane: hi and lo parts.  F16: the row is first
// scaled by 2^(sexp - 127) (returned) so that its largest component lies in [2^6, 2^7).
template <int MB, bool F16>
__device__ __forceinline__ int store_a(const float2 (&v)[kE], uint32_t taddr_hi, uint32_t taddr_lo) {
  if constexpr (!F16) {
#pragma unroll
    for (int h = 0; h < kE / 8; ++h) {
      uint32_t rh[16], rl[16];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float2 z = v[8 * h + e];
        const float hr = tf32_rn(z.x), hi = tf32_rn(z.y);
        rh[2 * e] = __float_as_uint(hr);
        rh[2 * e + 1] = __float_as_uint(hi);
        rl[2 * e] = __float_as_uint(tf32_rn(z.x - hr));
        rl[2 * e + 1] = __float_as_uint(tf32_rn(z.y - hi));
      }
      SV_TMEM_ST16(taddr_hi + 16 * h, rh);
      SV_TMEM_ST16(taddr_lo + 16 * h, rl);
    }
    return 127;
  } else {
    float mx = 0.f;
#pragma unroll
    for (int e = 0; e < kE; ++e) mx = fmaxf(mx, fmaxf(fabsf(v[e].x), fabsf(v[e].y)));
    const int ex = (int)((__float_as_uint(mx) >> 23) & 0xFF);
    int sexp = 127 + kF16RowExp + 127 - ex;  // biased exponent of the scale 2^(6 - (ex - 127))
    sexp = sexp < 2 ? 2 : (sexp > 240 ? 240 : sexp);
    const float sc = __uint_as_float((uint32_t)sexp << 23);
#pragma unroll
    for (int h = 0; h < kE / 16; ++h) {
      uint32_t rh[16], rl[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {  // amplitude 16h+e -> column 16h+e (re low half, im high)
        const float2 z = v[16 * h + e];
        const float2 x = make_float2(z.x * sc, z.y * sc);
        const __half2 h2 = __float22half2_rn(x);  // both parts in one conversion
        const float2 hf = __half22float2(h2);
        const __half2 l2 = __float22half2_rn(make_float2(x.x - hf.x, x.y - hf.y));
        rh[e] = half2_bits(h2);
        rl[e] = half2_bits(l2);
      }
      SV_TMEM_ST16(taddr_hi + 16 * h, rh);
      SV_TMEM_ST16(taddr_lo + 16 * h, rl);
    }
    return sexp;
  }
}

template <int MB, bool F16>
__global__ void __launch_bounds__(128 * MB, Cols<MB, F16>::kPerSm)
fused_pass_kernel(float2 *__restrict__ psi, DevPlanView plan, int pass_index, uint64_t num_tiles) {
  using FM = Fmt<F16>;
  using CL = Cols<MB, F16>;
  constexpr int kB = FM::kBBytes;
  int *err = plan.err;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *bbuf = smem_raw;                                       // 2 x (hi + lo)
  float2 *tile = reinterpret_cast<float2 *>(smem_raw + 4 * kB);        // 2^m amplitudes
  __shared__ DevPass P;
  __shared__ uint64_t chunk_off[1 << 10];
  __shared__ __align__(8) uint64_t bars[3];  // [0] MMA done, [1],[2] B buffer full
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int16_t mma_list[256];
  __shared__ int n_mma;
  __shared__ double norm_in[8], norm_out[8];  // per-warp sums of the tile norm

  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    P = plan.passes[pass_index];
    abort_flag = 0;
    for (int i = 0; i < 3; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&bars[i])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_slot)), "r"(CL::kAlloc));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  build_chunk_table(P, chunk_off);
  if (tid == 0) {
    int k = 0;
    for (int s = 0; s < P.stage_count && k < 256; ++s)
      if (!plan.stages[P.stage_begin + s].diag_only) mma_list[k++] = (int16_t)s;
    n_mma = k;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
  const int mb = tid >> 7;
  const uint32_t bar_mma = smem_u32(&bars[0]);
  uint32_t mma_phase = 0;
  uint32_t b_phase0 = 0, b_phase1 = 0;  // tid 0 only
  int qglob = 0;                        // MMA stages issued so far (B buffer = qglob & 1)
  int b_loads_out = 0;                  // tid 0: B loads issued and not yet waited for
  bool mma_out = false;                 // tid 0: MMAs committed and not yet waited for

  if (tid == 0 && n_mma > 0 && blockIdx.x < num_tiles) {
    issue_b_load<F16>(plan.mats, plan.stages[P.stage_begin + mma_list[0]], bbuf, 0, smem_u32(&bars[1]));
    ++b_loads_out;
  }

  for (uint64_t tile_id = blockIdx.x; tile_id < num_tiles && !abort_flag; tile_id += gridDim.x) {
    const uint64_t base = tile_base(P, tile_id);
    const bool last_tile = tile_id + gridDim.x >= num_tiles;
    load_tile(psi, tile, P, chunk_off, base);
    __syncthreads();
    // Every gate of the pass acts inside the tile, so a unitary pass keeps the tile's
    // norm exactly.  The tensor core's fp32 accumulation truncates toward zero and loses
    // ~0.3 ulp of every output per stage (a systematic norm drift of ~1e-7 per stage);
    // the tile's norm is measured in the first stage and restored in the last one with
    // unbiased stochastic rounding.
    const bool keep_norm = (P.flags & svp::PF_UNITARY) && !(P.flags & svp::PF_RAW) && n_mma > 0;
    int q = 0;  // MMA stage index within this tile
    for (int s = 0; s < P.stage_count; ++s) {
      const uint32_t si = P.stage_begin + s;
      const DevStage &st = plan.stages[si];
      uint32_t L0;
      uint64_t G0;
      group_base(plan, si, tid, base, &L0, &G0);
      float2 v[kE];
      load_group(tile, st, L0, v);
      // (read after the last stage's barrier; the stage barriers between keep it stable)
      if (keep_norm && s == 0) warp_sum_to((double)row_norm2(v), norm_in);
      if (!st.diag_only) {
        const int buf = qglob & 1;
        // prefetch the next MMA stage's B into the other buffer (its last reader, the
        // previous MMA stage, has completed)
        if (tid == 0) {
          const bool more_here = q + 1 < n_mma;
          if (more_here || !last_tile) {
            const DevStage &nx = plan.stages[P.stage_begin + mma_list[more_here ? q + 1 : 0]];
            issue_b_load<F16>(plan.mats, nx, bbuf, buf ^ 1, smem_u32(&bars[1 + (buf ^ 1)]));
            ++b_loads_out;
          }
        }
        const int sexp = store_a<MB, F16>(v, tmem + lane_off + CL::a_hi(mb), tmem + lane_off + CL::a_lo(mb));
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t bbar = smem_u32(&bars[1 + buf]);
          const uint32_t ph = buf ? b_phase1 : b_phase0;
          if (!mbar_wait(bbar, ph)) {
            atomicExch(err, 1);
            abort_flag = 1;
          } else {
            --b_loads_out;
            if (buf) b_phase1 ^= 1; else b_phase0 ^= 1;
            const uint32_t bhi = smem_u32(bbuf + buf * 2 * kB);
            const uint64_t dhi = smem_desc(bhi, FM::kSBO), dlo = smem_desc(bhi + kB, FM::kSBO);  // +16 per 256 B
#pragma unroll
            for (int m = 0; m < MB; ++m) {
              const uint32_t d = tmem + CL::d(m);
              const uint32_t ah = tmem + CL::a_hi(m), al = tmem + CL::a_lo(m);
              // small correction terms first, the large hi*hi term last: fewer truncating
              // accumulations at full magnitude
#pragma unroll
              for (int kk = 0; kk < FM::kKsteps; ++kk) mma<F16>(d, al + 8 * kk, dhi + 16 * kk, kk > 0);
#pragma unroll
              for (int kk = 0; kk < FM::kKsteps; ++kk) mma<F16>(d, ah + 8 * kk, dlo + 16 * kk, 1);
#pragma unroll
              for (int kk = 0; kk < FM::kKsteps; ++kk) mma<F16>(d, ah + 8 * kk, dhi + 16 * kk, 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(bar_mma) : "memory");
            mma_out = true;
          }
        }
        // every thread waits for the MMAs (bounded; if the B wait above gave up nothing
        // was committed and the others give up too); a warp reads tensor memory only if
        // all its lanes saw the MMAs complete (the loads are warp-wide)
        const bool done = __all_sync(0xffffffffu, !(tid == 0 && abort_flag) && mbar_wait(bar_mma, mma_phase));
        mma_phase ^= 1;
        if (tid == 0 && done) mma_out = false;
        if (!done) {
          atomicExch(err, 2);
          abort_flag = 1;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (done) {
          // F16: undo the row scale and the 2^8 of B (exact powers of two)
          const float un = F16 ? __uint_as_float((uint32_t)(127 + 127 - kF16BExp - sexp) << 23) : 1.0f;
#pragma unroll
          for (int hh = 0; hh < kK / 32; ++hh) {  // 16 amplitudes (32 registers) at a time
            uint32_t r[2][16];
#pragma unroll
            for (int h = 0; h < 2; ++h) SV_TMEM_LD16(tmem + lane_off + CL::d(mb) + 32 * hh + 16 * h, r[h]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                float re = __uint_as_float(r[h][2 * e]), im = __uint_as_float(r[h][2 * e + 1]);
                if (F16) { re *= un; im *= un; }
                v[16 * hh + 8 * h + e] = make_float2(re, im);
              }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        ++q;
        ++qglob;
      }
      apply_ops(v, plan.ops, st.op_begin, st.op_count, G0, plan.mats);
      if (keep_norm && s == P.stage_count - 1) {
        warp_sum_to((double)row_norm2(v), norm_out);
        __syncthreads();
        const double n_in = slots_sum(norm_in), n_out = slots_sum(norm_out);
        if (n_out > 0.0) {
          const float delta = (float)(sqrt(n_in / n_out) - 1.0);
          const uint32_t seed = (uint32_t)base * 0x85EBCA6Bu + (uint32_t)(base >> 32) * 0xC2B2AE35u +
                                (uint32_t)pass_index * 0x27D4EB2Fu + (uint32_t)tid * 0x165667B1u;
          scale_row(v, delta, seed);
        }
      }
      asm volatile("" ::: "memory");
      group_base(plan, si, tid, base, &L0, &G0);
      store_group(tile, st, L0, v);
      __syncthreads();
      if (abort_flag) break;
    }
    if (abort_flag) break;
    store_tile(psi, tile, P, chunk_off, base);
    __syncthreads();
  }

  // drain what is still in flight (bounded), then free the tensor memory
  if (tid == 0) {
    if (mma_out) mbar_wait(bar_mma, mma_phase);
    for (int i = 0; i < 2 && b_loads_out > 0; ++i) {
      const uint32_t ph = (qglob & 1) ? b_phase1 : b_phase0;
      if (mbar_wait(smem_u32(&bars[1 + (qglob & 1)]), ph)) --b_loads_out;
      ++qglob;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(CL::kAlloc));
}

template <int MB, bool F16>
cudaError_t launch_cfg(float2 *psi, int n, const DevPlanView &plan, int pass_index, const svp::DevPass &hp,
                       cudaStream_t st) {
  static bool configured = false;
  // dynamic shared memory: two B buffers (hi + lo each) and the tile.  CTAs per SM are
  // set by the TMEM allocation (512 columns per SM) and the launch bounds (Cols::kPerSm):
  // 5-qubit stages, TF32 m=12: 2 x 256 columns; TF32 m=13: 1 x 512; F16 m=12: 3 x 128;
  // F16 m=13: 2 x 256; 4-qubit stages (m=12, two M blocks): F16 2 x 128, TF32 2 x 256.
  const size_t smem = (size_t)(4 * Fmt<F16>::kBBytes) + (sizeof(float2) << hp.m);
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(fused_pass_kernel<MB, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int per_sm = Cols<MB, F16>::kPerSm;
  const uint64_t tiles = 1ull << (n - hp.m);
  uint64_t grid = (uint64_t)device_sm_count() * per_sm;
  if (grid > tiles) grid = tiles;
  fused_pass_kernel<MB, F16><<<(unsigned)grid, 128 * MB, smem, st>>>(psi, plan, pass_index, tiles);
  return cudaGetLastError();
}

}  // namespace

cudaError_t SV_FUSED_LAUNCH(float2 *psi, int n, const DevPlanView &plan, int pass_index, const svp::DevPass &hp,
                            cudaStream_t st, bool f16) {
  // rows of 2^kR amplitudes: 128 rows (one M block) per 2^(kR + 7) amplitudes of the tile
  const int mb = 1 << (hp.m - kR - 7);
  if (mb == 1) return f16 ? launch_cfg<1, true>(psi, n, plan, pass_index, hp, st)
                          : launch_cfg<1, false>(psi, n, plan, pass_index, hp, st);
  if (mb == 2) return f16 ? launch_cfg<2, true>(psi, n, plan, pass_index, hp, st)
                          : launch_cfg<2, false>(psi, n, plan, pass_index, hp, st);
  return cudaErrorInvalidValue;
}

}  // namespace svk

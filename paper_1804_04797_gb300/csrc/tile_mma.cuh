// Matrix stages of the pipelined plan kernels on the tcgen05 tensor cores.
//
// A stage of a fused packed plan acts on five tile qubits: tile bit 0 (the pack bit) and
// four register slots.  Its gates are multiplied out on the host (fp64) into one 32 x 32
// complex unitary U (the "bunch of gates" of §2.3 as a matrix), applied to a tile as one
// real GEMM on the tensor cores:
//     D[t, n] = sum_k A[t, k] * B[k, n],   k, n = 32 * (re/im) + j,
// where row t is the t-th thread of the compute group (its 32 amplitudes, index j = pack
// bit + 2 * register slots, as its 16 packed pairs R[p] = (re_j, re_j+1), I[p] likewise)
// and B = [[Re U^T, Im U^T], [-Im U^T, Re U^T]] in that order, so that D's columns come
// back as the same packed pairs.  The thread writes its row of A into its own TMEM lane
// (tcgen05.st), the kernel's MMA warp issues the products from TMEM (A) and shared memory
// (B) and commits them to the group's mbarrier, and the thread reads its row of D back
// (tcgen05.ld).  Split precision, three products accumulated in fp32 in tensor memory:
//   F16x3   A = hi + lo in fp16, the tile scaled once by a power of two (tile_scale:
//           exact, undone after its last stage), B likewise split (unscaled);
//           lo*hi + hi*lo + hi*hi (the lo*lo term is ~2^-22 relative).  K = 16 per MMA.
//   TF32x3  hi = x rounded to the nearest TF32, lo = (x - hi) rounded likewise.  K = 8.
#pragma once

#include "tile_pack.cuh"
#include "tile_pipe.cuh"

namespace svk {
namespace tmma {

using namespace tpipe;
using tpk::fma2;
using tpk::mul2;
using tpk::sub2;

// Operand format of one precision: TMEM columns of one A part (and of D), MMA
// instructions along K, bytes of one 64 x 64 B part, the row-group stride of B's K-major
// layout, and the instruction descriptor (D fp32, A/B K-major, M = 128, N = 64).
template <bool F16>
struct MFmt;
template <>
struct MFmt<true> {
  static constexpr int kACols = 32;  // 64 fp16 values of a row, two to a column
  static constexpr int kKSteps = 4;
  static constexpr uint32_t kBPart = 64 * 64 * 2;
  static constexpr uint32_t kSBO = 8 * 128;
  static constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | (8u << 17) | (8u << 24);
};
template <>
struct MFmt<false> {
  static constexpr int kACols = 64;
  static constexpr int kKSteps = 8;
  static constexpr uint32_t kBPart = 64 * 64 * 4;
  static constexpr uint32_t kSBO = 16 * 128;
  static constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | (8u << 17) | (8u << 24);
};


// Shared-memory matrix descriptor of a K-major operand without swizzle: 8-row x 16-byte
// core matrices, K-adjacent ones 128 B apart (leading byte offset), row groups sbo apart.
__device__ __forceinline__ uint64_t b_desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(sbo >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of tcgen05
  return d;
}

template <bool F16>
__device__ __forceinline__ void mma(uint32_t d, uint32_t a, uint64_t b, uint32_t acc) {
  if (F16)
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
                 ::"r"(d), "r"(a), "l"(b), "r"(MFmt<true>::kIdesc), "r"(acc));
  else
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
                 ::"r"(d), "r"(a), "l"(b), "r"(MFmt<false>::kIdesc), "r"(acc));
}

// Completion of every tcgen05 operation this thread issued so far arrives on `bar`.
__device__ __forceinline__ void mma_commit(unsigned long long *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive TMEM columns of this thread's lane from / to 32 registers.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

// Two floats as an fp16 pair (lo in the low half), nearest-even, and back.
__device__ __forceinline__ uint32_t f16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ float2 f16x2_f32(uint32_t h) {
  float2 f;
  asm("{\n .reg .b16 l, h;\n mov.b32 {l, h}, %2;\n cvt.f32.f16 %0, l;\n cvt.f32.f16 %1, h;\n}\n"
      : "=f"(f.x), "=f"(f.y)
      : "r"(h));
  return f;
}
// Nearest TF32 value, ties away from zero (half a TF32 ulp added to the magnitude bits,
// the 13 low mantissa bits cleared): both split parts exact in TF32, residual unbiased.
__device__ __forceinline__ float tf32_rn(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

template <int N>
__device__ __forceinline__ float row_norm2(const float2 (&R)[N], const float2 (&I)[N]) {
  float2 s = make_float2(0.f, 0.f), t = make_float2(0.f, 0.f);
#pragma unroll
  for (int p = 0; p < N; ++p) {
    s = fma2(R[p], R[p], s);
    t = fma2(I[p], I[p], t);
  }
  return (s.x + s.y) + (t.x + t.y);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

// The scale of a tile's amplitudes for the F16x3 products, from its norm^2 (the four warp
// sums as hi + lo pairs): the power of two that brings the tile's norm into [2^13, 2^14),
// so that no amplitude exceeds 2^14 (fp16 holds up to 65504) while the typical one, 1/64
// of the norm, sits near 2^7, its lo part far above fp16's subnormal range.  A unitary
// stage keeps every row's norm, so the scale holds for all the tile's stages: the tile is
// scaled once before its first product and unscaled once after its last stage.
__device__ __forceinline__ float tile_scale(const float2 (&s)[4]) {
  const float n2 = (s[0].x + s[1].x) + (s[2].x + s[3].x);
  int h = ((int)((__float_as_uint(n2) >> 23) & 0xFF) - 127) >> 1;  // n2 in [2^E, 2^(E+1)), h = floor(E/2)
  h = h < -100 ? -100 : (h > 100 ? 100 : h);
  return __uint_as_float((uint32_t)(127 + 13 - h) << 23);
}

// 1 / x for a power of two x (exact).
__device__ __forceinline__ float inv_pow2(float x) { return __uint_as_float((254u << 23) - __float_as_uint(x)); }

// The row of A into this thread's TMEM lane (hi at ta_hi, lo at ta_lo; the re pairs in
// the first half of each part's columns, the im pairs in the second).  F16 with SCALE: the
// row is multiplied by the tile's scale `sc` first (its first product; the later ones find
// it at that scale already).
template <bool F16, bool SCALE, int N>
__device__ __forceinline__ void store_a(const float2 (&R)[N], const float2 (&I)[N], float sc, uint32_t ta_hi,
                                        uint32_t ta_lo) {
  static_assert(N == 16, "rows of 32 amplitudes");
  if (F16) {
    const float2 sc2 = make_float2(sc, sc);
    // eight columns (pairs) at a time: few registers live besides the row
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int p = 8 * (c & 1) + e;
        const float2 x = SCALE ? mul2(c >> 1 ? I[p] : R[p], sc2) : (c >> 1 ? I[p] : R[p]);
        hi[e] = f16x2(x.x, x.y);
        const float2 d = sub2(x, f16x2_f32(hi[e]));
        lo[e] = f16x2(d.x, d.y);
      }
      tmem_st8(ta_hi + 8 * c, hi);
      tmem_st8(ta_lo + 8 * c, lo);
    }
  } else {
    (void)sc;
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      uint32_t hi[32], lo[32];
#pragma unroll
      for (int p = 0; p < N; ++p) {
        const float2 z = part ? I[p] : R[p];
        const float2 a = make_float2(tf32_rn(z.x), tf32_rn(z.y));
        const float2 d = sub2(z, a);
        hi[2 * p] = __float_as_uint(a.x);
        hi[2 * p + 1] = __float_as_uint(a.y);
        lo[2 * p] = __float_as_uint(tf32_rn(d.x));
        lo[2 * p + 1] = __float_as_uint(tf32_rn(d.y));
      }
      tmem_st32(ta_hi + 32 * part, hi);
      tmem_st32(ta_lo + 32 * part, lo);
    }
  }
}

// The first half of a matrix stage: this thread's row as A into its TMEM lane (times sc,
// F16), then the MMA warp is told (a_full).
template <bool F16, bool SCALE, int N>
__device__ __forceinline__ void matrix_pre(const float2 (&R)[N], const float2 (&I)[N], float sc, uint32_t ta_hi,
                                           uint32_t ta_lo, unsigned long long *a_full) {
  store_a<F16, SCALE, N>(R, I, sc, ta_hi, ta_lo);
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  fence_before();
  mbar_arrive(a_full);
}

// The second half: wait for the products (d_full, phase `parity`, bounded), D back into
// R/I (at the tile's scale: the stage unitary keeps it).  Returns false if the wait gave
// up (R/I then hold whatever tensor memory held).
template <bool F16, int N>
__device__ __forceinline__ bool matrix_post(float2 (&R)[N], float2 (&I)[N], uint32_t td,
                                            unsigned long long *d_full, uint32_t parity) {
  const bool ok = mbar_wait(d_full, parity, kWaitNs);
  fence_after();
  uint32_t re[32], im[32];
  tmem_ld32(td, re);
  tmem_ld32(td + 32, im);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  fence_before();
#pragma unroll
  for (int p = 0; p < N; ++p) {
    R[p] = make_float2(__uint_as_float(re[2 * p]), __uint_as_float(re[2 * p + 1]));
    I[p] = make_float2(__uint_as_float(im[2 * p]), __uint_as_float(im[2 * p + 1]));
  }
  return ok;
}

// The products of one matrix stage for one group (issued by one thread): D = A_lo B_hi +
// A_hi B_lo + A_hi B_hi, the small terms first (fewer truncating accumulations at full
// magnitude).  b_hi / b_lo: shared-memory addresses of the stage's two B parts.
template <bool F16>
__device__ __forceinline__ void issue_products(uint32_t td, uint32_t ta_hi, uint32_t ta_lo, uint32_t b_hi,
                                               uint32_t b_lo) {
  using FM = MFmt<F16>;
  const uint64_t dh = b_desc(b_hi, FM::kSBO), dl = b_desc(b_lo, FM::kSBO);
  // one K step = 8 TMEM columns of A and two 128-byte core matrices of B (+256 B = +16)
#pragma unroll
  for (int k = 0; k < FM::kKSteps; ++k) mma<F16>(td, ta_lo + 8 * k, dh + 16 * k, k > 0);
#pragma unroll
  for (int k = 0; k < FM::kKSteps; ++k) mma<F16>(td, ta_hi + 8 * k, dl + 16 * k, 1);
#pragma unroll
  for (int k = 0; k < FM::kKSteps; ++k) mma<F16>(td, ta_hi + 8 * k, dh + 16 * k, 1);
}

// Two values times (1 + delta), stochastically rounded: RN(x + x delta + r ulp(x)) with r
// uniform in [-1/2, 1/2) rounds x (1 + delta) up or down with probabilities in proportion
// to its distance from the two neighbours, so the expected result is exact even for the
// sub-ulp delta that plain rounding would drop.  h: 32 random bits (23 feed each r).
__device__ __forceinline__ float2 scale_sr2(float2 v, float2 d2, uint32_t h) {
  // 2^exponent of each value (its ulp is that times 2^-23), r + 1.5 in [1, 2)
  const float2 e = make_float2(__uint_as_float(__float_as_uint(v.x) & 0x7F800000u),
                               __uint_as_float(__float_as_uint(v.y) & 0x7F800000u));
  const float2 r = make_float2(__uint_as_float((h & 0x007FFFFFu) | 0x3F800000u),
                               __uint_as_float((h >> 9) | 0x3F800000u));
  const float2 rs = fma2(r, make_float2(1.1920928955078125e-7f, 1.1920928955078125e-7f),
                         make_float2(-1.78813934326171875e-7f, -1.78813934326171875e-7f));  // (r - 1.5) 2^-23
  return tpk::add2(v, fma2(rs, e, mul2(v, d2)));
}

// Every amplitude of the row times (1 + delta), stochastically rounded; the random bits
// come from a Weyl sequence (golden-ratio increments) from `seed`.
template <int N>
__device__ __forceinline__ void scale_row_sr(float2 (&R)[N], float2 (&I)[N], float delta, uint32_t seed) {
  const float2 d2 = make_float2(delta, delta);
#pragma unroll
  for (int p = 0; p < N; ++p) {
    R[p] = scale_sr2(R[p], d2, seed + (uint32_t)(2 * p + 1) * 0x9E3779B9u);
    I[p] = scale_sr2(I[p], d2, seed + (uint32_t)(2 * p + 2) * 0x9E3779B9u);
  }
}

// The factor 1 + delta that brings a tile's norm^2 from `out` back to `in` (each the four
// warps' sums as hi + lo pairs): the pairs are summed with their rounding errors kept
// (TwoSum), the two totals agree to ~1e-6 so their difference is exact (Sterbenz), and
// delta = sqrt(1 + d) - 1 ~ d/2 - d^2/8 with d = (in - out) / out, all in fp32.
__device__ __forceinline__ float restore_delta(const float2 (&in)[4], const float2 (&out)[4]) {
  float si = 0.f, ei = 0.f, so = 0.f, eo = 0.f;
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    float s = si + in[w].x, bb = s - si;
    ei += ((si - (s - bb)) + (in[w].x - bb)) + in[w].y;
    si = s;
    s = so + out[w].x;
    bb = s - so;
    eo += ((so - (s - bb)) + (out[w].x - bb)) + out[w].y;
    so = s;
  }
  if (!(so > 0.f)) return 0.f;
  const float d = ((si - so) + (ei - eo)) / so;
  return d * fmaf(-0.125f, d, 0.5f);
}

// Sum of one float per thread over a warp as an unevaluated pair hi + lo (every lane
// receives it): each addition's rounding error is kept (Knuth's TwoSum), so the pair
// carries the exact sum to about 2^-44 -- the tile-norm ratio needs far more than a
// float's 24 bits, and fp64 arithmetic on every thread would be slow on this GPU.
__device__ __forceinline__ float2 warp_sum2(float x) {
  float hi = x, lo = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    const float s = hi + h2, bb = s - hi;
    const float e = (hi - (s - bb)) + (h2 - bb);
    hi = s;
    lo = lo + l2 + e;
  }
  return make_float2(hi, lo);
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to
// shared memory, completing `bar`'s transaction count.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

}  // namespace tmma
}  // namespace svk

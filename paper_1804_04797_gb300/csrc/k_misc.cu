// Whole-state kernels: initial state (K0), per-gate sweeps (K2 pair update, K3
// diagonal factor), fp64 reductions and gathers (K5).
#include <cuda_runtime.h>

#include <cmath>

#include "kernels.h"

namespace svk {
namespace {

constexpr int kBlock = 256;
constexpr int kReduceBlocks = 1024;

// grid-stride helper: enough CTAs to fill the GPU several times over
inline unsigned grid_for(uint64_t items, int per_thread = 1) {
  const uint64_t want = (items + (uint64_t)kBlock * per_thread - 1) / ((uint64_t)kBlock * per_thread);
  const uint64_t cap = (uint64_t)device_sm_count() * 16;
  return (unsigned)(want < 1 ? 1 : (want > cap ? cap : want));
}

__global__ void init_kernel(float4 *psi4, uint64_t n4, float a, bool zero_state) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n4;
       i += (uint64_t)gridDim.x * blockDim.x) {
    if (zero_state) psi4[i] = make_float4(i == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f);
    else psi4[i] = make_float4(a, 0.f, a, 0.f);
  }
}

// Pair update of §2 on qubit q >= 1: each thread takes the two adjacent pairs
// (i, i+2^q) and (i+1, i+1+2^q) as two float4 loads.
__global__ void gate1q_kernel(float2 *psi, uint64_t items, int q, Mat2 u) {
  const uint64_t low = (1ull << q) - 1;
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < items;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t t = 2 * p;  // index with bit q removed, even
    const uint64_t i0 = ((t & ~low) << 1) | (t & low);
    float4 *a4 = reinterpret_cast<float4 *>(psi + i0);
    float4 *b4 = reinterpret_cast<float4 *>(psi + i0 + (1ull << q));
    const float4 x = *a4, y = *b4;
    const float *m = u.v;
    float4 xo, yo;
    xo.x = m[0] * x.x - m[1] * x.y + m[2] * y.x - m[3] * y.y;
    xo.y = m[0] * x.y + m[1] * x.x + m[2] * y.y + m[3] * y.x;
    xo.z = m[0] * x.z - m[1] * x.w + m[2] * y.z - m[3] * y.w;
    xo.w = m[0] * x.w + m[1] * x.z + m[2] * y.w + m[3] * y.z;
    yo.x = m[4] * x.x - m[5] * x.y + m[6] * y.x - m[7] * y.y;
    yo.y = m[4] * x.y + m[5] * x.x + m[6] * y.y + m[7] * y.x;
    yo.z = m[4] * x.z - m[5] * x.w + m[6] * y.z - m[7] * y.w;
    yo.w = m[4] * x.w + m[5] * x.z + m[6] * y.w + m[7] * y.z;
    *a4 = xo;
    *b4 = yo;
  }
}

// Pair update on qubit 0: each float4 is one pair.
__global__ void gate1q_q0_kernel(float4 *psi4, uint64_t items, Mat2 u) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < items;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const float4 z = psi4[p];
    const float *m = u.v;
    float4 o;
    o.x = m[0] * z.x - m[1] * z.y + m[2] * z.z - m[3] * z.w;
    o.y = m[0] * z.y + m[1] * z.x + m[2] * z.w + m[3] * z.z;
    o.z = m[4] * z.x - m[5] * z.y + m[6] * z.z - m[7] * z.w;
    o.w = m[4] * z.y + m[5] * z.x + m[6] * z.w + m[7] * z.z;
    psi4[p] = o;
  }
}

__device__ __forceinline__ uint64_t deposit_skip(uint64_t t, uint64_t mask) {
  // spread the bits of t over the zero bits of mask (ascending)
  uint64_t out = 0;
  int src = 0;
  for (int b = 0; b < 64 && (t >> src); ++b) {
    if ((mask >> b) & 1ull) continue;
    out |= ((t >> src) & 1ull) << b;
    ++src;
  }
  return out;
}

// Diagonal factor (fr + fr_lo) + i (fi + fi_lo) on the amplitudes whose bits under mask
// equal val; the lo parts carry what fp32 cannot hold of 1/sqrt2 (unbiased rounding).
__global__ void diag_kernel(float2 *psi, uint64_t items, uint64_t mask, uint64_t val, float fr,
                            float fi, float fr_lo, float fi_lo) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < items;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = deposit_skip(p, mask) | val;
    const float2 z = psi[i];
    const float re = fmaf(fr, z.x, fmaf(-fi, z.y, fr_lo * z.x - fi_lo * z.y));
    const float im = fmaf(fr, z.y, fmaf(fi, z.x, fr_lo * z.y + fi_lo * z.x));
    psi[i] = make_float2(re, im);
  }
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Level 1: each block sums a fixed, grid-strided share.  GB300's fp64 rate is a small
// fraction of its fp32 rate, so |alpha|^2 and |alpha|^4 of 8 amplitudes are summed in
// fp32 (relative error ~1e-7 per chunk, unbiased) and the chunk sums accumulate in fp64.
__global__ void norm_partial_kernel(const float4 *psi4, uint64_t n4, double *partials) {
  double s2 = 0.0, s4 = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n4; i += 4 * stride) {
    float4 z[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] = psi4[i + k * stride];
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
    const float4 z = psi4[i];
    const float p0 = fmaf(z.x, z.x, z.y * z.y);
    const float p1 = fmaf(z.z, z.z, z.w * z.w);
    s2 += (double)(p0 + p1);
    s4 += (double)fmaf(p0, p0, p1 * p1);
  }
  __shared__ double r2[kBlock / 32], r4[kBlock / 32];
  s2 = warp_sum(s2);
  s4 = warp_sum(s4);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { r2[w] = s2; r4[w] = s4; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < kBlock / 32; ++k) { a += r2[k]; b += r4[k]; }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

// Level 2: one block adds the partials in a fixed order.
__global__ void norm_final_kernel(const double *partials, int count, double *out2) {
  __shared__ double a[kBlock], b[kBlock];
  double s2 = 0, s4 = 0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) { s2 += partials[2 * i]; s4 += partials[2 * i + 1]; }
  a[threadIdx.x] = s2;
  b[threadIdx.x] = s4;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) { a[threadIdx.x] += a[threadIdx.x + h]; b[threadIdx.x] += b[threadIdx.x + h]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out2[0] = a[0]; out2[1] = b[0]; }
}

// Small states (n = 1): plain loop in one thread.
__global__ void norm_small_kernel(const float2 *psi, uint64_t count, double *out2) {
  double s2 = 0, s4 = 0;
  for (uint64_t i = 0; i < count; ++i) {
    const double p = (double)psi[i].x * psi[i].x + (double)psi[i].y * psi[i].y;
    s2 += p;
    s4 += p * p;
  }
  out2[0] = s2;
  out2[1] = s4;
}

// <a|b> = sum_i conj(a_i) b_i, level 1: as the norm, 8 products summed in fp32 per
// chunk (the terms have random phases: the fp32 chunk error is relative to the chunk),
// chunk sums in fp64.  partials[2k] = real part, partials[2k+1] = imaginary part.
__global__ void inner_partial_kernel(const float4 *a4, const float4 *b4, uint64_t n4, double *partials) {
  double sr = 0.0, si = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n4; i += 4 * stride) {
    float4 a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { a[k] = a4[i + k * stride]; b[k] = b4[i + k * stride]; }
    float cr = 0.f, ci = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      cr = fmaf(a[k].x, b[k].x, fmaf(a[k].y, b[k].y, fmaf(a[k].z, b[k].z, fmaf(a[k].w, b[k].w, cr))));
      ci = fmaf(a[k].x, b[k].y, fmaf(-a[k].y, b[k].x, fmaf(a[k].z, b[k].w, fmaf(-a[k].w, b[k].z, ci))));
    }
    sr += cr;
    si += ci;
  }
  for (; i < n4; i += stride) {
    const float4 a = a4[i], b = b4[i];
    sr += (double)fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
    si += (double)fmaf(a.x, b.y, fmaf(-a.y, b.x, fmaf(a.z, b.w, -a.w * b.z)));
  }
  __shared__ double rr[kBlock / 32], ri[kBlock / 32];
  sr = warp_sum(sr);
  si = warp_sum(si);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { rr[w] = sr; ri[w] = si; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < kBlock / 32; ++k) { a += rr[k]; b += ri[k]; }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

// Small states (n = 1): plain loop in one thread.
__global__ void inner_small_kernel(const float2 *a, const float2 *b, uint64_t count, double *out2) {
  double sr = 0, si = 0;
  for (uint64_t i = 0; i < count; ++i) {
    sr += (double)a[i].x * b[i].x + (double)a[i].y * b[i].y;
    si += (double)a[i].x * b[i].y - (double)a[i].y * b[i].x;
  }
  out2[0] = sr;
  out2[1] = si;
}

__global__ void set_one_kernel(float2 *psi, uint64_t x) { psi[x] = make_float2(1.f, 0.f); }

__global__ void gather_kernel(const float2 *psi, const uint64_t *bits, int64_t m, double *out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const float2 z = psi[bits[j]];
    out[2 * j] = z.x;
    out[2 * j + 1] = z.y;
  }
}

__global__ void gather_prob_kernel(const float2 *psi, const uint64_t *bits, int64_t m, double *out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const float2 z = psi[bits[j]];
    out[j] = (double)z.x * z.x + (double)z.y * z.y;
  }
}

}  // namespace

int device_sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  }
  return sms;
}

cudaError_t launch_init(float2 *psi, int n, bool uniform, float amp, cudaStream_t st) {
  if (n == 0) return cudaErrorInvalidValue;
  const uint64_t n4 = 1ull << (n - 1);
  init_kernel<<<grid_for(n4), kBlock, 0, st>>>(reinterpret_cast<float4 *>(psi), n4, amp, !uniform);
  return cudaGetLastError();
}

cudaError_t launch_gate_1q(float2 *psi, int n, int q, const Mat2 &u, cudaStream_t st) {
  if (q == 0) {
    const uint64_t items = 1ull << (n - 1);
    gate1q_q0_kernel<<<grid_for(items), kBlock, 0, st>>>(reinterpret_cast<float4 *>(psi), items, u);
  } else {
    const uint64_t items = 1ull << (n - 2);
    gate1q_kernel<<<grid_for(items), kBlock, 0, st>>>(psi, items, q, u);
  }
  return cudaGetLastError();
}

cudaError_t launch_gate_diag(float2 *psi, int n, uint64_t mask, uint64_t val, float fr, float fi,
                             cudaStream_t st) {
  const int fixed = __builtin_popcountll(mask);
  const uint64_t items = 1ull << (n - fixed);
  // split each factor into fp32 hi + lo (exact for 0, +-1; 1/sqrt2 keeps its remainder)
  const double s2 = 0.70710678118654752440;
  auto lo = [&](float f) -> float {
    const double a = std::fabs((double)f);
    if (std::fabs(a - s2) < 1e-6) return (float)((f < 0 ? -s2 : s2) - (double)f);
    return 0.f;
  };
  diag_kernel<<<grid_for(items), kBlock, 0, st>>>(psi, items, mask, val, fr, fi, lo(fr), lo(fi));
  return cudaGetLastError();
}

int reduce_partials_needed() { return kReduceBlocks; }

cudaError_t launch_norm(const float2 *psi, int n, double *partials, double *out2, cudaStream_t st) {
  if (n < 2) {
    norm_small_kernel<<<1, 1, 0, st>>>(psi, 1ull << n, out2);
    return cudaGetLastError();
  }
  const uint64_t n4 = 1ull << (n - 1);
  uint64_t blocks = (n4 + kBlock - 1) / kBlock;
  if (blocks > (uint64_t)kReduceBlocks) blocks = kReduceBlocks;
  norm_partial_kernel<<<(unsigned)blocks, kBlock, 0, st>>>(reinterpret_cast<const float4 *>(psi), n4, partials);
  norm_final_kernel<<<1, kBlock, 0, st>>>(partials, (int)blocks, out2);
  return cudaGetLastError();
}

cudaError_t launch_norm_final(const double *partials, int count, double *out2, cudaStream_t st) {
  norm_final_kernel<<<1, kBlock, 0, st>>>(partials, count, out2);
  return cudaGetLastError();
}

cudaError_t launch_inner(const float2 *a, const float2 *b, int n, double *partials, double *out2, cudaStream_t st) {
  if (n < 2) {
    inner_small_kernel<<<1, 1, 0, st>>>(a, b, 1ull << n, out2);
    return cudaGetLastError();
  }
  const uint64_t n4 = 1ull << (n - 1);
  uint64_t blocks = (n4 + kBlock - 1) / kBlock;
  if (blocks > (uint64_t)kReduceBlocks) blocks = kReduceBlocks;
  inner_partial_kernel<<<(unsigned)blocks, kBlock, 0, st>>>(reinterpret_cast<const float4 *>(a),
                                                              reinterpret_cast<const float4 *>(b), n4, partials);
  norm_final_kernel<<<1, kBlock, 0, st>>>(partials, (int)blocks, out2);
  return cudaGetLastError();
}

cudaError_t launch_basis_state(float2 *psi, int n, uint64_t x, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(psi, 0, sizeof(float2) << n, st);
  if (e != cudaSuccess) return e;
  set_one_kernel<<<1, 1, 0, st>>>(psi, x);
  return cudaGetLastError();
}

cudaError_t launch_gather(const float2 *psi, const uint64_t *bits, int64_t m, double *out, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  gather_kernel<<<grid_for((uint64_t)m), kBlock, 0, st>>>(psi, bits, m, out);
  return cudaGetLastError();
}

cudaError_t launch_gather_prob(const float2 *psi, const uint64_t *bits, int64_t m, double *out,
                               cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  gather_prob_kernel<<<grid_for((uint64_t)m), kBlock, 0, st>>>(psi, bits, m, out);
  return cudaGetLastError();
}

}  // namespace svk

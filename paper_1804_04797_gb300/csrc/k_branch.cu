// K6: fp64 branch sum of the cut decomposition (§2, Fig. 2 and Eq. 1).
//
// The two halves are stored as batched states: A[x_A + (l << nA)] is amplitude x_A of
// branch l of half A (and likewise B), so branch l of every half-state is one slice of
// a (nA + t)-qubit vector.  For each requested bitstring j one CTA forms
// sum_l A[xa_j, l] * B[xb_j, l] in fp64 with a fixed reduction tree (deterministic).
#include <cuda_runtime.h>

#include <cmath>

#include "kernels.h"

namespace svk {
namespace {

constexpr int kBlock = 256;

__global__ void branch_sum_kernel(const float2 *__restrict__ A, int nA, const float2 *__restrict__ B, int nB,
                                  int t, const uint64_t *__restrict__ xa, const uint64_t *__restrict__ xb,
                                  double scale, double *__restrict__ out) {
  const int j = blockIdx.x;
  const uint64_t a0 = xa[j], b0 = xb[j];
  const uint64_t branches = 1ull << t;
  double sr = 0.0, si = 0.0;
  for (uint64_t l = threadIdx.x; l < branches; l += blockDim.x) {
    const float2 a = A[a0 + (l << nA)];
    const float2 b = B[b0 + (l << nB)];
    sr += (double)a.x * b.x - (double)a.y * b.y;
    si += (double)a.x * b.y + (double)a.y * b.x;
  }
  __shared__ double rr[kBlock], ri[kBlock];
  rr[threadIdx.x] = sr;
  ri[threadIdx.x] = si;
  __syncthreads();
  for (int h = kBlock / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      rr[threadIdx.x] += rr[threadIdx.x + h];
      ri[threadIdx.x] += ri[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * j] = rr[0] * scale;
    out[2 * j + 1] = ri[0] * scale;
  }
}

// The tensor form of the same sum (§2, Eqs. 6-7: the full state is a sum over branches
// of outer products phi_l (x) xi_l): out[x_A + (x_B << nA)] = scale * sum_l
// A[x_A + (l << nA)] * B[x_B + (l << nB)], a complex matrix product (2^nB x 2^t) *
// (2^t x 2^nA).  64 x 64 outputs per CTA, 16 branches per shared-memory step, 4 x 4
// outputs per thread, fp32 accumulation.
constexpr int kTile = 64, kStep = 16;

__global__ void __launch_bounds__(256) outer_sum_kernel(const float2 *__restrict__ A, int nA,
                                                        const float2 *__restrict__ B, int nB, int t, float scale,
                                                        float2 *__restrict__ out) {
  __shared__ float2 As[kStep][kTile], Bs[kStep][kTile];
  const uint64_t xa0 = (uint64_t)blockIdx.x * kTile, xb0 = (uint64_t)blockIdx.y * kTile;
  const uint64_t na = 1ull << nA, nb = 1ull << nB, branches = 1ull << t;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (uint64_t l0 = 0; l0 < branches; l0 += kStep) {
    for (int e = threadIdx.x; e < kStep * kTile; e += blockDim.x) {
      const int k = e / kTile, i = e % kTile;
      const bool lin = l0 + k < branches;
      As[k][i] = (lin && xa0 + i < na) ? A[xa0 + i + ((l0 + k) << nA)] : make_float2(0.f, 0.f);
      Bs[k][i] = (lin && xb0 + i < nb) ? B[xb0 + i + ((l0 + k) << nB)] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kStep; ++k) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][tx * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][ty * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint64_t xb = xb0 + ty * 4 + j;
    if (xb >= nb) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint64_t xa = xa0 + tx * 4 + i;
      if (xa < na) out[xa + (xb << nA)] = make_float2(acc[i][j].x * scale, acc[i][j].y * scale);
    }
  }
}

// A fork of the branch tree: the first 2^n_cur amplitudes (every branch bit above them
// still in |+>) replicated into all 2^(n_new - n_cur) slices of new branch bits, each
// times 2^{-(n_new - n_cur)/2} (the H that put those bits in |+>): psi[i + (c << n_cur)]
// = f psi[i].  Two amplitudes per 16-byte vector; f applied as hi + lo (one rounding).
__global__ void fork_kernel(float4 *__restrict__ psi, uint64_t pairs, int copies_log2, int n_cur, float f_hi,
                            float f_lo) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < pairs; i += stride) {
    float4 v = psi[i];
    v.x = fmaf(v.x, f_hi, v.x * f_lo);
    v.y = fmaf(v.y, f_hi, v.y * f_lo);
    v.z = fmaf(v.z, f_hi, v.z * f_lo);
    v.w = fmaf(v.w, f_hi, v.w * f_lo);
    for (uint64_t c = 0; c < (1ull << copies_log2); ++c) psi[i + (c << (n_cur - 1))] = v;
  }
}

}  // namespace

cudaError_t launch_fork(float2 *psi, int n_cur, int n_new, cudaStream_t st) {
  if (n_new <= n_cur) return cudaSuccess;
  if (n_cur < 1) return cudaErrorInvalidValue;
  const int k = n_new - n_cur;
  // f = 2^{-k/2}: exact for even k; for odd k, 1/sqrt2 as the float nearest plus the rest
  const double f = std::ldexp(1.0, -(k / 2)) * ((k & 1) ? 0.70710678118654752440 : 1.0);
  const float hi = (float)f, lo = (float)(f - (double)hi);
  const uint64_t pairs = 1ull << (n_cur - 1);
  uint64_t grid = (pairs + 255) / 256;
  const uint64_t cap = (uint64_t)device_sm_count() * 16;
  if (grid > cap) grid = cap;
  fork_kernel<<<(unsigned)grid, 256, 0, st>>>(reinterpret_cast<float4 *>(psi), pairs, k, n_cur, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_outer_sum(const float2 *A, int nA, const float2 *B, int nB, int t, float scale, float2 *out,
                             cudaStream_t st) {
  const uint64_t gx = ((1ull << nA) + kTile - 1) / kTile, gy = ((1ull << nB) + kTile - 1) / kTile;
  if (gx > 0x7fffffffull || gy > 65535ull) return cudaErrorInvalidValue;
  outer_sum_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(A, nA, B, nB, t, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_branch_sum(const float2 *A, int nA, const float2 *B, int nB, int t, const uint64_t *xa,
                              const uint64_t *xb, int m, double scale, double *out, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  branch_sum_kernel<<<m, kBlock, 0, st>>>(A, nA, B, nB, t, xa, xb, scale, out);
  return cudaGetLastError();
}

}  // namespace svk

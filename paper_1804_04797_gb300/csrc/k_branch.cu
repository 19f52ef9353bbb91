// K6: fp64 branch sum of the cut decomposition (§2, Fig. 2 and Eq. 1).
//
// The two halves are stored as batched states: A[x_A + (l << nA)] is amplitude x_A of
// branch l of half A (and likewise B), so branch l of every half-state is one slice of
// a (nA + t)-qubit vector.  For each requested bitstring j one CTA forms
// sum_l A[xa_j, l] * B[xb_j, l] in fp64 with a fixed reduction tree (deterministic).
#include <cuda_runtime.h>

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

}  // namespace

cudaError_t launch_branch_sum(const float2 *A, int nA, const float2 *B, int nB, int t, const uint64_t *xa,
                              const uint64_t *xb, int m, double scale, double *out, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  branch_sum_kernel<<<m, kBlock, 0, st>>>(A, nA, B, nB, t, xa, xb, scale, out);
  return cudaGetLastError();
}

}  // namespace svk

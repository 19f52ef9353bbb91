// Device code shared by the tile-pass kernels (plain and fused): the register-group
// gate actions of the plain path (also used for the fused path's diagonal epilogue),
// the shared-memory swizzle, and the gathered-tile load/store.
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"

namespace svk {
namespace tile {

using svp::DevOp;
using svp::DevPass;
using svp::DevStage;

constexpr int kR = 5;
constexpr int kE = 1 << kR;
// 1/sqrt2 as an unevaluated sum hi + lo: the float nearest 1/sqrt2 is 1.7e-8 low, and
// multiplying by it alone shrinks the norm by that much at every T gate (a systematic
// drift of 1e-6 over ~80 T gates); v*hi + v*lo in one fma rounds v/sqrt2 to nearest.
constexpr float kS2 = 0.70710678118654752440f;
constexpr float kS2lo = 1.21016171e-8f;  // 1/sqrt2 - kS2

__device__ __forceinline__ float rs2(float v) { return fmaf(v, kS2, v * kS2lo); }

__device__ __forceinline__ uint32_t swz(uint32_t L) {
  return L ^ (((L >> 4) ^ (L >> 8) ^ (L >> 12)) & 15u);
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// ---- one-qubit gates on a pair (x: register bit 0, y: register bit 1) ---------------
struct GH {
  __device__ __forceinline__ static void f(float2 &x, float2 &y) {
    const float2 a = x, b = y;
    x = f2(rs2(a.x + b.x), rs2(a.y + b.y));
    y = f2(rs2(a.x - b.x), rs2(a.y - b.y));
  }
};
// X^{1/2}: x' = (s + i d)/2, y' = (s - i d)/2 with s = x + y, d = x - y
struct GSX {
  __device__ __forceinline__ static void f(float2 &x, float2 &y) {
    const float sr = x.x + y.x, si = x.y + y.y, dr = x.x - y.x, di = x.y - y.y;
    x = f2(0.5f * (sr - di), 0.5f * (si + dr));
    y = f2(0.5f * (sr + di), 0.5f * (si - dr));
  }
};
struct GSXDG {
  __device__ __forceinline__ static void f(float2 &x, float2 &y) {
    const float sr = x.x + y.x, si = x.y + y.y, dr = x.x - y.x, di = x.y - y.y;
    x = f2(0.5f * (sr + di), 0.5f * (si - dr));
    y = f2(0.5f * (sr - di), 0.5f * (si + dr));
  }
};
// Y^{1/2}: x' = (1+i)(x - y)/2, y' = (1+i)(x + y)/2
struct GSY {
  __device__ __forceinline__ static void f(float2 &x, float2 &y) {
    const float sr = x.x + y.x, si = x.y + y.y, dr = x.x - y.x, di = x.y - y.y;
    x = f2(0.5f * (dr - di), 0.5f * (dr + di));
    y = f2(0.5f * (sr - si), 0.5f * (sr + si));
  }
};
// (Y^{1/2})^dagger: x' = (1-i)(x + y)/2, y' = -(1-i)(x - y)/2
struct GSYDG {
  __device__ __forceinline__ static void f(float2 &x, float2 &y) {
    const float sr = x.x + y.x, si = x.y + y.y, dr = x.x - y.x, di = x.y - y.y;
    x = f2(0.5f * (sr + si), 0.5f * (si - sr));
    y = f2(-0.5f * (dr + di), -0.5f * (di - dr));
  }
};

// ---- diagonal actions on one element -------------------------------------------------
struct DT {  // times e^{i pi/4}
  __device__ __forceinline__ static void f(float2 &z) { z = f2(rs2(z.x - z.y), rs2(z.x + z.y)); }
};
struct DTDG {
  __device__ __forceinline__ static void f(float2 &z) { z = f2(rs2(z.x + z.y), rs2(z.y - z.x)); }
};
struct DNEG {
  __device__ __forceinline__ static void f(float2 &z) { z = f2(-z.x, -z.y); }
};
struct DZERO {
  __device__ __forceinline__ static void f(float2 &z) { z = f2(0.f, 0.f); }
};

template <class G, int J>
__device__ __forceinline__ void pairs(float2 (&v)[kE]) {
#pragma unroll
  for (int e = 0; e < kE; ++e)
    if (!(e & (1 << J))) G::f(v[e], v[e | (1 << J)]);
}
template <class G>
__device__ __forceinline__ void pairs_j(float2 (&v)[kE], int j) {
  switch (j) {
    case 0: pairs<G, 0>(v); break;
    case 1: pairs<G, 1>(v); break;
    case 2: pairs<G, 2>(v); break;
    case 3: pairs<G, 3>(v); break;
    default: pairs<G, 4>(v); break;
  }
}
// D on the elements whose register bit J equals B
template <class D, int J, int B>
__device__ __forceinline__ void diag1(float2 (&v)[kE]) {
#pragma unroll
  for (int e = 0; e < kE; ++e)
    if (((e >> J) & 1) == B) D::f(v[e]);
}
template <class D, int B>
__device__ __forceinline__ void diag1_j(float2 (&v)[kE], int j) {
  switch (j) {
    case 0: diag1<D, 0, B>(v); break;
    case 1: diag1<D, 1, B>(v); break;
    case 2: diag1<D, 2, B>(v); break;
    case 3: diag1<D, 3, B>(v); break;
    default: diag1<D, 4, B>(v); break;
  }
}
// CZ: negate where bits J and K are both 1; PEQ: zero where bits J and K differ
template <int J, int K, bool EQ>
__device__ __forceinline__ void diag2(float2 (&v)[kE]) {
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    const int bj = (e >> J) & 1, bk = (e >> K) & 1;
    if (EQ) {
      if (bj != bk) DZERO::f(v[e]);
    } else if (bj && bk) {
      DNEG::f(v[e]);
    }
  }
}
template <int J, bool EQ>
__device__ __forceinline__ void diag2_k(float2 (&v)[kE], int k) {
  switch (k) {
    case 0: diag2<J, 0, EQ>(v); break;
    case 1: diag2<J, 1, EQ>(v); break;
    case 2: diag2<J, 2, EQ>(v); break;
    case 3: diag2<J, 3, EQ>(v); break;
    default: diag2<J, 4, EQ>(v); break;
  }
}
template <bool EQ>
__device__ __forceinline__ void diag2_jk(float2 (&v)[kE], int j, int k) {
  switch (j) {
    case 0: diag2_k<0, EQ>(v, k); break;
    case 1: diag2_k<1, EQ>(v, k); break;
    case 2: diag2_k<2, EQ>(v, k); break;
    case 3: diag2_k<3, EQ>(v, k); break;
    default: diag2_k<4, EQ>(v, k); break;
  }
}

__device__ __forceinline__ void phase_all(float2 (&v)[kE], int p) {
  switch (p & 7) {
    case 0: break;
    case 4:
#pragma unroll
      for (int e = 0; e < kE; ++e) DNEG::f(v[e]);
      break;
    case 2:
#pragma unroll
      for (int e = 0; e < kE; ++e) v[e] = f2(-v[e].y, v[e].x);
      break;
    case 6:
#pragma unroll
      for (int e = 0; e < kE; ++e) v[e] = f2(v[e].y, -v[e].x);
      break;
    default: {
      // w^p for odd p: (sr + i si)/sqrt2 with sr, si = +-1
      const float sr = (p == 1 || p == 7) ? 1.f : -1.f;
      const float si = (p == 1 || p == 3) ? 1.f : -1.f;
#pragma unroll
      for (int e = 0; e < kE; ++e)
        v[e] = f2(rs2(sr * v[e].x - si * v[e].y), rs2(sr * v[e].y + si * v[e].x));
    }
  }
}

template <int J>
__device__ __forceinline__ void general1(float2 (&v)[kE], const float *u) {
  const float ar = u[0], ai = u[1], br = u[2], bi = u[3], cr = u[4], ci = u[5], dr = u[6], di = u[7];
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    if (e & (1 << J)) continue;
    const float2 x = v[e], y = v[e | (1 << J)];
    v[e] = f2(ar * x.x - ai * x.y + br * y.x - bi * y.y, ar * x.y + ai * x.x + br * y.y + bi * y.x);
    v[e | (1 << J)] = f2(cr * x.x - ci * x.y + dr * y.x - di * y.y, cr * x.y + ci * x.x + dr * y.y + di * y.x);
  }
}

__device__ __forceinline__ void apply_op(float2 (&v)[kE], const DevOp &op, const float *mats) {
  using namespace svp;
  switch (op.act) {
    case A_H: pairs_j<GH>(v, op.j); break;
    case A_SX: pairs_j<GSX>(v, op.j); break;
    case A_SY: pairs_j<GSY>(v, op.j); break;
    case A_SXDG: pairs_j<GSXDG>(v, op.j); break;
    case A_SYDG: pairs_j<GSYDG>(v, op.j); break;
    case A_T: diag1_j<DT, 1>(v, op.j); break;
    case A_TDG: diag1_j<DTDG, 1>(v, op.j); break;
    case A_Z: diag1_j<DNEG, 1>(v, op.j); break;
    case A_P0: diag1_j<DZERO, 1>(v, op.j); break;
    case A_P1: diag1_j<DZERO, 0>(v, op.j); break;
    case A_CZ: diag2_jk<false>(v, op.j, op.k); break;
    case A_PEQ: diag2_jk<true>(v, op.j, op.k); break;
    case A_PHASE: phase_all(v, op.arg); break;
    case A_ZERO:
#pragma unroll
      for (int e = 0; e < kE; ++e) DZERO::f(v[e]);
      break;
    case A_U: {
      const float *u = mats + 8 * (op.arg | (op.k << 8));
      switch (op.j) {
        case 0: general1<0>(v, u); break;
        case 1: general1<1>(v, u); break;
        case 2: general1<2>(v, u); break;
        case 3: general1<3>(v, u); break;
        default: general1<4>(v, u); break;
      }
    } break;
    default: break;
  }
}


// Global index of element 0 of group `g` and its shared-memory (swizzled) base, for a
// stage whose group bits are st.nonr[0 .. m-kR).
__device__ __forceinline__ void group_base(const DevStage &st, const DevPass &P, int g, uint64_t base,
                                           uint32_t *L0, uint64_t *G0) {
  uint32_t l = 0;
  uint64_t gg = base;
  const int ng = P.m - kR;
  for (int i = 0; i < ng; ++i) {
    if ((g >> i) & 1) {
      const int b = st.nonr[i];
      l |= 1u << b;
      gg |= 1ull << P.tq[b];
    }
  }
  *L0 = l;
  *G0 = gg;
}

__device__ __forceinline__ void load_group(const float2 *tile, const DevStage &st, uint32_t L0, float2 (&v)[kE]) {
  uint32_t pr[kR];
#pragma unroll
  for (int j = 0; j < kR; ++j) pr[j] = swz(1u << st.rbit[j]);
  const uint32_t p0 = swz(L0);
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    uint32_t a = p0;
#pragma unroll
    for (int j = 0; j < kR; ++j)
      if ((e >> j) & 1) a ^= pr[j];
    v[e] = tile[a];
  }
}

__device__ __forceinline__ void store_group(float2 *tile, const DevStage &st, uint32_t L0, const float2 (&v)[kE]) {
  uint32_t pr[kR];
#pragma unroll
  for (int j = 0; j < kR; ++j) pr[j] = swz(1u << st.rbit[j]);
  const uint32_t p0 = swz(L0);
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    uint32_t a = p0;
#pragma unroll
    for (int j = 0; j < kR; ++j)
      if ((e >> j) & 1) a ^= pr[j];
    tile[a] = v[e];
  }
}

__device__ __forceinline__ void apply_ops(float2 (&v)[kE], const DevOp *ops, int begin, int count, uint64_t G0,
                                          const float *mats) {
  for (int o = begin; o < begin + count; ++o) {
    const DevOp op = ops[o];
    if ((G0 & op.cmask) != op.cval) continue;
    apply_op(v, op, mats);
  }
}

// Base index of tile `tile_id`: its bits spread over the non-tile qubits.
__device__ __forceinline__ uint64_t tile_base(const DevPass &P, uint64_t tile_id) {
  uint64_t base = 0;
  for (int i = 0; i < P.nt; ++i) base |= ((tile_id >> i) & 1ull) << P.ntq[i];
  return base;
}

// chunk_off[h]: bits of chunk index h spread over the tile qubits above the c low ones.
__device__ __forceinline__ void build_chunk_table(const DevPass &P, uint64_t *chunk_off) {
  const int nb = P.m - P.c;
  for (int h = threadIdx.x; h < (1 << nb); h += blockDim.x) {
    uint64_t off = 0;
    for (int i = 0; i < nb; ++i)
      if ((h >> i) & 1) off |= 1ull << P.tq[P.c + i];
    chunk_off[h] = off;
  }
}

// Read (or generate) the tile into shared memory: 16-byte coalesced vectors, 8 in flight
// per thread.  kL2Only reads through L2 only (ld.global.cg): needed when other CTAs of
// the same launch wrote the data, since L1 is not coherent across SMs.
template <bool kL2Only = false>
__device__ __forceinline__ void load_tile(const float2 *__restrict__ psi, float2 *tile, const DevPass &P,
                                          const uint64_t *chunk_off, uint64_t base) {
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const uint32_t half = 1u << (P.m - 1);
  const int c = P.c;
  const uint32_t low_mask = (1u << c) - 1;
  if (P.flags & svp::PF_INIT_UNIFORM) {
    const float a = P.init_amp;
    for (uint32_t f = tid; f < half; f += nthreads) reinterpret_cast<float4 *>(tile)[f] = make_float4(a, 0.f, a, 0.f);
    return;
  }
  if (P.flags & svp::PF_INIT_ZERO) {
    for (uint32_t f = tid; f < half; f += nthreads)
      reinterpret_cast<float4 *>(tile)[f] = make_float4((f == 0 && base == 0) ? 1.f : 0.f, 0.f, 0.f, 0.f);
    return;
  }
  constexpr int kBatch = 8;
  const int iters = (int)(half / nthreads);
  for (int it0 = 0; it0 < iters; it0 += kBatch) {
    float4 buf[kBatch];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const uint32_t L = 2u * (tid + (it0 + b) * nthreads);
      const uint64_t g = base + chunk_off[L >> c] + (L & low_mask);
      buf[b] = kL2Only ? __ldcg(reinterpret_cast<const float4 *>(psi + g)) : *reinterpret_cast<const float4 *>(psi + g);
    }
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const uint32_t L = 2u * (tid + (it0 + b) * nthreads);
      const uint32_t p = swz(L);
      float4 x = buf[b];
      if (p & 1u) x = make_float4(x.z, x.w, x.x, x.y);
      reinterpret_cast<float4 *>(tile)[p >> 1] = x;
    }
  }
}

__device__ __forceinline__ void store_tile(float2 *__restrict__ psi, const float2 *tile, const DevPass &P,
                                           const uint64_t *chunk_off, uint64_t base) {
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const uint32_t half = 1u << (P.m - 1);
  const int c = P.c;
  const uint32_t low_mask = (1u << c) - 1;
  const int iters = (int)(half / nthreads);
  for (int it = 0; it < iters; ++it) {
    const uint32_t L = 2u * (tid + it * nthreads);
    const uint32_t p = swz(L);
    float4 x = reinterpret_cast<const float4 *>(tile)[p >> 1];
    if (p & 1u) x = make_float4(x.z, x.w, x.x, x.y);
    const uint64_t g = base + chunk_off[L >> c] + (L & low_mask);
    *reinterpret_cast<float4 *>(psi + g) = x;
  }
}

// One tile of one plain pass: load (or generate), every stage in registers, store.
// The caller has built chunk_off for P and synchronised; ends with __syncthreads.
template <bool kL2Only = false>
__device__ __forceinline__ void process_tile_plain(float2 *__restrict__ psi, const DevPlanView &plan,
                                                   const DevPass &P, const uint64_t *chunk_off, float2 *tile,
                                                   uint64_t tile_id) {
  const int tid = threadIdx.x;
  const uint64_t base = tile_base(P, tile_id);
  load_tile<kL2Only>(psi, tile, P, chunk_off, base);
  __syncthreads();
  for (int s = 0; s < P.stage_count; ++s) {
    const DevStage &st = plan.stages[P.stage_begin + s];
    uint32_t L0;
    uint64_t G0;
    group_base(st, P, tid, base, &L0, &G0);
    float2 v[kE];
    load_group(tile, st, L0, v);
    apply_ops(v, plan.ops, st.op_begin, st.op_count, G0, plan.mats);
    // Recompute the addresses rather than keeping 32 of them live across the ops.
    asm volatile("" ::: "memory");
    group_base(st, P, tid, base, &L0, &G0);
    store_group(tile, st, L0, v);
    __syncthreads();
  }
  store_tile(psi, tile, P, chunk_off, base);
  __syncthreads();
}

}  // namespace tile
}  // namespace svk

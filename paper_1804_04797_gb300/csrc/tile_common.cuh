// Device code shared by the tile-pass kernels (plain and fused): the register-group
// gate actions of the plain path (also used for the fused path's diagonal epilogue),
// the shared-memory swizzle, and the gathered-tile load/store.  A translation unit picks
// the row width (SV_TILE_R) and the namespace its copy lives in (SV_TILE_NS), so that
// kernels of several widths link into one library.

#include <cuda_runtime.h>

#include "kernels.h"

#ifndef SV_TILE_NS
#define SV_TILE_NS tile
#endif

namespace svk {
namespace SV_TILE_NS {

using svp::DevOp;
using svp::DevPass;
using svp::DevStage;

// Register qubits per thread (each thread holds 2^kR amplitudes of a stage).  Every
// translation unit that includes this header picks its width: the tensor-core kernels
// take 5 (one row of the 32x32 stage unitary per thread) or 4 (16x16 blocks).
#ifndef SV_TILE_R
#define SV_TILE_R 5
#endif
constexpr int kR = SV_TILE_R;
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
// X^{1/2} without its factor 1/2 (apply_ops applies 2^-count once per stage):
// x' = s + i d, y' = s - i d with s = x + y, d = x - y
struct GSX {
  __device__ __forceinline__ static void f(float2 &x, float2 &y) {
    const float sr = x.x + y.x, si = x.y + y.y, dr = x.x - y.x, di = x.y - y.y;
    x = f2(sr - di, si + dr);
    y = f2(sr + di, si - dr);
  }
};
struct GSXDG {
  __device__ __forceinline__ static void f(float2 &x, float2 &y) {
    const float sr = x.x + y.x, si = x.y + y.y, dr = x.x - y.x, di = x.y - y.y;
    x = f2(sr + di, si - dr);
    y = f2(sr - di, si + dr);
  }
};
// Y^{1/2} without its factor 1/2: x' = (1+i)(x - y), y' = (1+i)(x + y)
struct GSY {
  __device__ __forceinline__ static void f(float2 &x, float2 &y) {
    const float sr = x.x + y.x, si = x.y + y.y, dr = x.x - y.x, di = x.y - y.y;
    x = f2(dr - di, dr + di);
    y = f2(sr - si, sr + si);
  }
};
// (Y^{1/2})^dagger without its factor 1/2: x' = (1-i)(x + y), y' = -(1-i)(x - y)
struct GSYDG {
  __device__ __forceinline__ static void f(float2 &x, float2 &y) {
    const float sr = x.x + y.x, si = x.y + y.y, dr = x.x - y.x, di = x.y - y.y;
    x = f2(sr + si, si - sr);
    y = f2(-(dr + di), dr - di);
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
  if constexpr (J >= kR) return;
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
  if constexpr (J >= kR) return;
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
  if constexpr (J >= kR || K >= kR) return;
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
  if constexpr (J >= kR) return;
  const float ar = u[0], ai = u[1], br = u[2], bi = u[3], cr = u[4], ci = u[5], dr = u[6], di = u[7];
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    if (e & (1 << J)) continue;
    const float2 x = v[e], y = v[e | (1 << J)];
    v[e] = f2(ar * x.x - ai * x.y + br * y.x - bi * y.y, ar * x.y + ai * x.x + br * y.y + bi * y.x);
    v[e | (1 << J)] = f2(cr * x.x - ci * x.y + dr * y.x - di * y.y, cr * x.y + ci * x.x + dr * y.y + di * y.x);
  }
}

// One op by its flat code (one indirect branch).  Scalar phases, zeroing of the whole
// group and the factors 1/2 of X^{1/2}, Y^{1/2} and their adjoints commute with every other
// op and are only recorded (ph, zero, halves) for apply_ops.
__device__ __forceinline__ void apply_op(float2 (&v)[kE], const DevOp &op, const float *mats, int &ph,
                                         bool &zero, int &halves) {
  using namespace svp;
  if (op.code >= C_PAIR + 5 && op.code < C_PAIR + 25) ++halves;
  switch (op.code) {
    case C_PAIR + 0: pairs<GH, 0>(v); break;
    case C_PAIR + 1: pairs<GH, 1>(v); break;
    case C_PAIR + 2: pairs<GH, 2>(v); break;
    case C_PAIR + 3: pairs<GH, 3>(v); break;
    case C_PAIR + 4: pairs<GH, 4>(v); break;
    case C_PAIR + 5: pairs<GSX, 0>(v); break;
    case C_PAIR + 6: pairs<GSX, 1>(v); break;
    case C_PAIR + 7: pairs<GSX, 2>(v); break;
    case C_PAIR + 8: pairs<GSX, 3>(v); break;
    case C_PAIR + 9: pairs<GSX, 4>(v); break;
    case C_PAIR + 10: pairs<GSY, 0>(v); break;
    case C_PAIR + 11: pairs<GSY, 1>(v); break;
    case C_PAIR + 12: pairs<GSY, 2>(v); break;
    case C_PAIR + 13: pairs<GSY, 3>(v); break;
    case C_PAIR + 14: pairs<GSY, 4>(v); break;
    case C_PAIR + 15: pairs<GSXDG, 0>(v); break;
    case C_PAIR + 16: pairs<GSXDG, 1>(v); break;
    case C_PAIR + 17: pairs<GSXDG, 2>(v); break;
    case C_PAIR + 18: pairs<GSXDG, 3>(v); break;
    case C_PAIR + 19: pairs<GSXDG, 4>(v); break;
    case C_PAIR + 20: pairs<GSYDG, 0>(v); break;
    case C_PAIR + 21: pairs<GSYDG, 1>(v); break;
    case C_PAIR + 22: pairs<GSYDG, 2>(v); break;
    case C_PAIR + 23: pairs<GSYDG, 3>(v); break;
    case C_PAIR + 24: pairs<GSYDG, 4>(v); break;
    case C_DIAG + 0: diag1<DT, 0, 1>(v); break;
    case C_DIAG + 1: diag1<DT, 1, 1>(v); break;
    case C_DIAG + 2: diag1<DT, 2, 1>(v); break;
    case C_DIAG + 3: diag1<DT, 3, 1>(v); break;
    case C_DIAG + 4: diag1<DT, 4, 1>(v); break;
    case C_DIAG + 5: diag1<DTDG, 0, 1>(v); break;
    case C_DIAG + 6: diag1<DTDG, 1, 1>(v); break;
    case C_DIAG + 7: diag1<DTDG, 2, 1>(v); break;
    case C_DIAG + 8: diag1<DTDG, 3, 1>(v); break;
    case C_DIAG + 9: diag1<DTDG, 4, 1>(v); break;
    case C_DIAG + 10: diag1<DNEG, 0, 1>(v); break;
    case C_DIAG + 11: diag1<DNEG, 1, 1>(v); break;
    case C_DIAG + 12: diag1<DNEG, 2, 1>(v); break;
    case C_DIAG + 13: diag1<DNEG, 3, 1>(v); break;
    case C_DIAG + 14: diag1<DNEG, 4, 1>(v); break;
    case C_DIAG + 15: diag1<DZERO, 0, 1>(v); break;
    case C_DIAG + 16: diag1<DZERO, 1, 1>(v); break;
    case C_DIAG + 17: diag1<DZERO, 2, 1>(v); break;
    case C_DIAG + 18: diag1<DZERO, 3, 1>(v); break;
    case C_DIAG + 19: diag1<DZERO, 4, 1>(v); break;
    case C_DIAG + 20: diag1<DZERO, 0, 0>(v); break;
    case C_DIAG + 21: diag1<DZERO, 1, 0>(v); break;
    case C_DIAG + 22: diag1<DZERO, 2, 0>(v); break;
    case C_DIAG + 23: diag1<DZERO, 3, 0>(v); break;
    case C_DIAG + 24: diag1<DZERO, 4, 0>(v); break;
    case C_CZ + 1: diag2<0, 1, false>(v); break;
    case C_PEQ + 1: diag2<0, 1, true>(v); break;
    case C_CZ + 2: diag2<0, 2, false>(v); break;
    case C_PEQ + 2: diag2<0, 2, true>(v); break;
    case C_CZ + 3: diag2<0, 3, false>(v); break;
    case C_PEQ + 3: diag2<0, 3, true>(v); break;
    case C_CZ + 4: diag2<0, 4, false>(v); break;
    case C_PEQ + 4: diag2<0, 4, true>(v); break;
    case C_CZ + 5: diag2<1, 0, false>(v); break;
    case C_PEQ + 5: diag2<1, 0, true>(v); break;
    case C_CZ + 7: diag2<1, 2, false>(v); break;
    case C_PEQ + 7: diag2<1, 2, true>(v); break;
    case C_CZ + 8: diag2<1, 3, false>(v); break;
    case C_PEQ + 8: diag2<1, 3, true>(v); break;
    case C_CZ + 9: diag2<1, 4, false>(v); break;
    case C_PEQ + 9: diag2<1, 4, true>(v); break;
    case C_CZ + 10: diag2<2, 0, false>(v); break;
    case C_PEQ + 10: diag2<2, 0, true>(v); break;
    case C_CZ + 11: diag2<2, 1, false>(v); break;
    case C_PEQ + 11: diag2<2, 1, true>(v); break;
    case C_CZ + 13: diag2<2, 3, false>(v); break;
    case C_PEQ + 13: diag2<2, 3, true>(v); break;
    case C_CZ + 14: diag2<2, 4, false>(v); break;
    case C_PEQ + 14: diag2<2, 4, true>(v); break;
    case C_CZ + 15: diag2<3, 0, false>(v); break;
    case C_PEQ + 15: diag2<3, 0, true>(v); break;
    case C_CZ + 16: diag2<3, 1, false>(v); break;
    case C_PEQ + 16: diag2<3, 1, true>(v); break;
    case C_CZ + 17: diag2<3, 2, false>(v); break;
    case C_PEQ + 17: diag2<3, 2, true>(v); break;
    case C_CZ + 19: diag2<3, 4, false>(v); break;
    case C_PEQ + 19: diag2<3, 4, true>(v); break;
    case C_CZ + 20: diag2<4, 0, false>(v); break;
    case C_PEQ + 20: diag2<4, 0, true>(v); break;
    case C_CZ + 21: diag2<4, 1, false>(v); break;
    case C_PEQ + 21: diag2<4, 1, true>(v); break;
    case C_CZ + 22: diag2<4, 2, false>(v); break;
    case C_PEQ + 22: diag2<4, 2, true>(v); break;
    case C_CZ + 23: diag2<4, 3, false>(v); break;
    case C_PEQ + 23: diag2<4, 3, true>(v); break;
    case C_U + 0: general1<0>(v, mats + 8 * (op.arg | (op.k << 8))); break;
    case C_U + 1: general1<1>(v, mats + 8 * (op.arg | (op.k << 8))); break;
    case C_U + 2: general1<2>(v, mats + 8 * (op.arg | (op.k << 8))); break;
    case C_U + 3: general1<3>(v, mats + 8 * (op.arg | (op.k << 8))); break;
    case C_U + 4: general1<4>(v, mats + 8 * (op.arg | (op.k << 8))); break;
    case C_PHASE: ph += op.arg; break;
    case C_ZERO: zero = true; break;
    default: break;
  }
}

// Global index of element 0 of group `g` of stage `si` and its tile-local index, from
// the stage's three 16-entry tables (one per 4 bits of the group index).
__device__ __forceinline__ void group_base(const DevPlanView &plan, uint32_t si, int g, uint64_t base,
                                           uint32_t *L0, uint64_t *G0) {
  const svp::DevGroupEntry *t = plan.gtab + svp::kGroupEntries * si;
  const svp::DevGroupEntry a = t[g & 15], b = t[16 + ((g >> 4) & 15)], c = t[32 + ((g >> 8) & 15)];
  *L0 = a.L | b.L | c.L;
  *G0 = base | a.G | b.G | c.G;
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

__device__ __forceinline__ void apply_ops(float2 (&v)[kE], const DevOp *ops, uint32_t begin, int count,
                                          uint64_t G0, const float *mats) {
  int ph = 0, halves = 0;
  bool zero = false;
  if (count > 0) {
    for (int o = 0; o < count; ++o) {
      const DevOp op = ops[begin + o];
      if ((G0 & op.cmask) == op.cval) apply_op(v, op, mats, ph, zero, halves);
      if (halves == 32) {  // keep the deferred growth (at most 2^32) far from fp32 overflow
        const float sc = __int_as_float((127 - 32) << 23);
#pragma unroll
        for (int e = 0; e < kE; ++e) v[e] = f2(v[e].x * sc, v[e].y * sc);
        halves = 0;
      }
    }
  }
  if (zero) {
#pragma unroll
    for (int e = 0; e < kE; ++e) DZERO::f(v[e]);
  } else {
    if (halves) {
      const float sc = __int_as_float((127 - halves) << 23);  // 2^-halves, exact
#pragma unroll
      for (int e = 0; e < kE; ++e) v[e] = f2(v[e].x * sc, v[e].y * sc);
    }
    if (ph & 7) phase_all(v, ph & 7);
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
    const uint32_t si = P.stage_begin + s;
    const DevStage &st = plan.stages[si];
    uint32_t L0;
    uint64_t G0;
    group_base(plan, si, tid, base, &L0, &G0);
    float2 v[kE];
    load_group(tile, st, L0, v);
    apply_ops(v, plan.ops, st.op_begin, st.op_count, G0, plan.mats);
    // Recompute the addresses rather than keeping 32 of them live across the ops.
    asm volatile("" ::: "memory");
    group_base(plan, si, tid, base, &L0, &G0);
    store_group(tile, st, L0, v);
    __syncthreads();
  }
  store_tile(psi, tile, P, chunk_off, base);
  __syncthreads();
}

}  // namespace SV_TILE_NS
}  // namespace svk

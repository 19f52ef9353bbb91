// Packed plain tile pass: the register form of the fp32 CUDA-core kernel.
//
// A thread holds 32 PAIRS of amplitudes.  The two amplitudes of a pair differ only in
// tile bit 0 (the pack bit, always qubit 0: two neighbours in memory), and a pair is
// kept as two float2 registers R = (re, re'), I = (im, im').  Blackwell's packed fp32
// instructions (FADD2/FMUL2/FFMA2) update both halves at once, so every gate on one of
// the five other register slots costs half the instructions of the one-amplitude form.
// A stage acts on six qubits (the pack bit + five), a thread on 64 amplitudes.
//
// Shared memory holds the tile as 16-byte pairs (re, re', im, im') at a swizzled slot
// (see pack_phys); the swizzle is linear over XOR, so a group's 32 slot addresses are
// the XOR of its base with the register-slot masks the planner stores.  Conditional
// diagonal ops (a CZ or projector whose other qubit is not a register bit) become a
// multiplication by a per-thread factor, so no op diverges within a warp.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#endif

#include "plan_dev.h"

namespace svk {
namespace tpk {

using svp::DevOp;
using svp::DevPass;
using svp::DevStage;

// Register slots besides the pack bit (the translation unit picks: 5 = 64 amplitudes per
// thread, 4 = 32).
#ifndef SV_PACK_R
#define SV_PACK_R 5
#endif
constexpr int kPR = SV_PACK_R;
static_assert(kPR >= 1 && kPR <= svp::kMaxReg, "pack register slots");
constexpr int kP = 1 << kPR;       // pairs per thread
constexpr float kS2 = 0.70710678118654752440f;
constexpr float kS2lo = 1.21016171e-8f;  // 1/sqrt2 - kS2: v*kS2 + v*kS2lo rounds v/sqrt2 to nearest

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as b * (-1) + a: exact product, one rounding, the same result as a subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return fma2(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 rs2x2(float2 v) { return fma2(v, f2(kS2, kS2), mul2(v, f2(kS2lo, kS2lo))); }
__device__ __forceinline__ float rs2(float v) { return fmaf(v, kS2, v * kS2lo); }

// ---- one-qubit gates: x = (xr, xi), y = (yr, yi), each component a float2 over pairs -----
// (the same formulas serve the scalar case of the pack slot with float in place of float2)
template <class T>
struct Ops;
template <>
struct Ops<float2> {
  __device__ __forceinline__ static float2 add(float2 a, float2 b) { return add2(a, b); }
  __device__ __forceinline__ static float2 sub(float2 a, float2 b) { return sub2(a, b); }
  __device__ __forceinline__ static float2 rs(float2 a) { return rs2x2(a); }
  __device__ __forceinline__ static float2 scale(float2 a, float c) { return mul2(a, f2(c, c)); }
};
template <>
struct Ops<float> {
  __device__ __forceinline__ static float add(float a, float b) { return a + b; }
  __device__ __forceinline__ static float sub(float a, float b) { return a - b; }
  __device__ __forceinline__ static float rs(float a) { return rs2(a); }
  __device__ __forceinline__ static float scale(float a, float c) { return a * c; }
};

// Each gate is written on s = x + y and d = x - y (its out()): f() forms them with adds,
// fs() with y carrying a sign (+1 or -1: y's sign from ops before the gate folded into
// one fused operation each, exact, the same result as negating y first).
template <class T>
struct Sgn;
template <>
struct Sgn<float2> {
  __device__ __forceinline__ static float2 add(float2 x, float2 y, float s) { return fma2(y, f2(s, s), x); }
  __device__ __forceinline__ static float2 sub(float2 x, float2 y, float s) { return fma2(y, f2(-s, -s), x); }
  // s y - x
  __device__ __forceinline__ static float2 rsub(float2 x, float2 y, float s) { return fma2(y, f2(s, s), f2(-x.x, -x.y)); }
};
template <>
struct Sgn<float> {
  __device__ __forceinline__ static float add(float x, float y, float s) { return fmaf(y, s, x); }
  __device__ __forceinline__ static float sub(float x, float y, float s) { return fmaf(y, -s, x); }
  __device__ __forceinline__ static float rsub(float x, float y, float s) { return fmaf(y, s, -x); }
};

template <class G>
struct Gate {
  template <class T>
  __device__ __forceinline__ static void f(T &xr, T &xi, T &yr, T &yi) {
    using O = Ops<T>;
    const T sr = O::add(xr, yr), si = O::add(xi, yi), dr = O::sub(xr, yr), di = O::sub(xi, yi);
    G::out(sr, si, dr, di, xr, xi, yr, yi);
  }
  template <class T>
  __device__ __forceinline__ static void fs(T &xr, T &xi, T &yr, T &yi, float s) {
    using S = Sgn<T>;
    const T sr = S::add(xr, yr, s), si = S::add(xi, yi, s), dr = S::sub(xr, yr, s), di = S::sub(xi, yi, s);
    G::out(sr, si, dr, di, xr, xi, yr, yi);
  }
};

struct GH : Gate<GH> {  // (x + y)/sqrt2, (x - y)/sqrt2
  template <class T>
  __device__ __forceinline__ static void out(T sr, T si, T dr, T di, T &xr, T &xi, T &yr, T &yi) {
    using O = Ops<T>;
    xr = O::rs(sr); xi = O::rs(si); yr = O::rs(dr); yi = O::rs(di);
  }
};
// The square roots as a scalar times an unscaled rotation (two additions per amplitude);
// the planner counts the scalars, e^{+-i pi/4} 2^{-1/2} per gate, and applies their
// product at the end of the plan (P_GLOBAL, with exact powers of two on the way):
//   X^{1/2} = e^{i pi/4} 2^{-1/2} [[1, -i], [-i, 1]]   (X^{1/2})^+ = e^{-i pi/4} 2^{-1/2} [[1, i], [i, 1]]
//   Y^{1/2} = e^{i pi/4} 2^{-1/2} [[1, -1], [1, 1]]    (Y^{1/2})^+ = e^{-i pi/4} 2^{-1/2} [[1, 1], [-1, 1]]
// fs(): y carries a sign s (+1 or -1), folded into fused operations (exact products).
struct GSX {  // x' = x - i y, y' = -i x + y
  template <class T>
  __device__ __forceinline__ static void f(T &xr, T &xi, T &yr, T &yi) {
    using O = Ops<T>;
    const T a = O::add(xr, yi), b = O::sub(xi, yr), c = O::add(xi, yr), d = O::sub(yi, xr);
    xr = a; xi = b; yr = c; yi = d;
  }
  template <class T>
  __device__ __forceinline__ static void fs(T &xr, T &xi, T &yr, T &yi, float s) {
    using S = Sgn<T>;
    const T a = S::add(xr, yi, s), b = S::sub(xi, yr, s), c = S::add(xi, yr, s), d = S::rsub(xr, yi, s);
    xr = a; xi = b; yr = c; yi = d;
  }
};
struct GSXDG {  // x' = x + i y, y' = i x + y
  template <class T>
  __device__ __forceinline__ static void f(T &xr, T &xi, T &yr, T &yi) {
    using O = Ops<T>;
    const T a = O::sub(xr, yi), b = O::add(xi, yr), c = O::sub(yr, xi), d = O::add(xr, yi);
    xr = a; xi = b; yr = c; yi = d;
  }
  template <class T>
  __device__ __forceinline__ static void fs(T &xr, T &xi, T &yr, T &yi, float s) {
    using S = Sgn<T>;
    const T a = S::sub(xr, yi, s), b = S::add(xi, yr, s), c = S::rsub(xi, yr, s), d = S::add(xr, yi, s);
    xr = a; xi = b; yr = c; yi = d;
  }
};
struct GSY {  // x' = x - y, y' = x + y
  template <class T>
  __device__ __forceinline__ static void f(T &xr, T &xi, T &yr, T &yi) {
    using O = Ops<T>;
    const T a = O::sub(xr, yr), b = O::sub(xi, yi), c = O::add(xr, yr), d = O::add(xi, yi);
    xr = a; xi = b; yr = c; yi = d;
  }
  template <class T>
  __device__ __forceinline__ static void fs(T &xr, T &xi, T &yr, T &yi, float s) {
    using S = Sgn<T>;
    const T a = S::sub(xr, yr, s), b = S::sub(xi, yi, s), c = S::add(xr, yr, s), d = S::add(xi, yi, s);
    xr = a; xi = b; yr = c; yi = d;
  }
};
struct GSYDG {  // x' = x + y, y' = y - x
  template <class T>
  __device__ __forceinline__ static void f(T &xr, T &xi, T &yr, T &yi) {
    using O = Ops<T>;
    const T a = O::add(xr, yr), b = O::add(xi, yi), c = O::sub(yr, xr), d = O::sub(yi, xi);
    xr = a; xi = b; yr = c; yi = d;
  }
  template <class T>
  __device__ __forceinline__ static void fs(T &xr, T &xi, T &yr, T &yi, float s) {
    using S = Sgn<T>;
    const T a = S::add(xr, yr, s), b = S::add(xi, yi, s), c = S::rsub(xr, yr, s), d = S::rsub(xi, yi, s);
    xr = a; xi = b; yr = c; yi = d;
  }
};

// ---- diagonal phases on one element (r, i) ----------------------------------------------
// T and its adjoint multiply by e^{+-i pi/4} = (1 +- i)/sqrt2: two additions, then the
// factor 1/sqrt2 as ONE multiplication by c, one of the two fp32 values that bracket it
// (kS2up = 0.70710683, above by 6.7e-8 relative; kS2dn = 0.70710677, below by 1.7e-8).
// The planner picks c gate by gate so that the running sum of these relative errors over
// the plan's T gates stays next to zero: their effect on the norm cancels instead of
// adding up (always rounding one way shrank the 34-qubit norm by 1.3e-6), at two packed
// operations per pair fewer than the correctly rounded hi + lo product.
constexpr float kS2dn = 0.70710677f, kS2up = 0.70710683f;
// u(): the same without the factor: (1 +- i) times (r, i), two additions.
struct DT1 {  // times e^{i pi/4}
  template <class T>
  __device__ __forceinline__ static void u(T r, T i, T &ur, T &ui) {
    using O = Ops<T>;
    ur = O::sub(r, i);
    ui = O::add(r, i);
  }
  template <class T>
  __device__ __forceinline__ static void f(T &r, T &i, float c) {
    using O = Ops<T>;
    T a, b;
    u(r, i, a, b);
    r = O::scale(a, c);
    i = O::scale(b, c);
  }
};
struct DTDG1 {  // times e^{-i pi/4}
  template <class T>
  __device__ __forceinline__ static void u(T r, T i, T &ur, T &ui) {
    using O = Ops<T>;
    ur = O::add(r, i);
    ui = O::sub(i, r);
  }
  template <class T>
  __device__ __forceinline__ static void f(T &r, T &i, float c) {
    using O = Ops<T>;
    T a, b;
    u(r, i, a, b);
    r = O::scale(a, c);
    i = O::scale(b, c);
  }
};

// ---- actions on a thread's 32 pairs -------------------------------------------------------
using Regs = float2[kP];

// The product of the square roots' scalars, applied once at the end of a plan (P_GLOBAL,
// arg = q + 8 u): every element times e^{i pi q/4} 2^{-u/2}.  Odd q: e^{i pi q/4} =
// (c + i d)/sqrt2 with c, d = +-1, so what remains after the additions is 1/2 (exact) for
// u = 1 and 1/sqrt2 (hi + lo) for u = 0; even q: i^{q/2} (exact), then 1/sqrt2 if u = 1.
template <int Q, int U>
__device__ __forceinline__ void global_factor(Regs &R, Regs &I) {
#pragma unroll
  for (int p = 0; p < kP; ++p) {
    const float2 r = R[p], i = I[p];
    float2 nr = r, ni = i;
    if constexpr (Q & 1) {
      constexpr float c = (Q == 1 || Q == 7) ? 1.f : -1.f, d = (Q == 1 || Q == 3) ? 1.f : -1.f;
      nr = fma2(i, f2(-d, -d), mul2(r, f2(c, c)));  // c r - d i
      ni = fma2(i, f2(c, c), mul2(r, f2(d, d)));    // d r + c i
      if constexpr (U == 1) {
        nr = mul2(nr, f2(0.5f, 0.5f));
        ni = mul2(ni, f2(0.5f, 0.5f));
      } else {
        nr = rs2x2(nr);
        ni = rs2x2(ni);
      }
    } else {
      if constexpr (Q == 2) { nr = f2(-i.x, -i.y); ni = r; }
      if constexpr (Q == 4) { nr = f2(-r.x, -r.y); ni = f2(-i.x, -i.y); }
      if constexpr (Q == 6) { nr = i; ni = f2(-r.x, -r.y); }
      if constexpr (U == 1) {
        nr = rs2x2(nr);
        ni = rs2x2(ni);
      }
    }
    R[p] = nr;
    I[p] = ni;
  }
}

// gate G on register slot J (pairs p and p | 2^J)
template <class G, int J>
__device__ __forceinline__ void pairs(Regs &R, Regs &I) {
  if constexpr (J < kPR) {
#pragma unroll
    for (int p = 0; p < kP; ++p)
      if (!(p & (1 << J))) G::f(R[p], I[p], R[p | (1 << J)], I[p | (1 << J)]);
  }
}
// gate G on the pack bit: inside every pair
template <class G>
__device__ __forceinline__ void pairs_pack(Regs &R, Regs &I) {
#pragma unroll
  for (int p = 0; p < kP; ++p) G::f(R[p].x, I[p].x, R[p].y, I[p].y);
}
// the same with y (the slot-1 element) carrying a sign s = +-1
template <class G, int J>
__device__ __forceinline__ void pairs_signed(Regs &R, Regs &I, float s) {
  if constexpr (J < kPR) {
#pragma unroll
    for (int p = 0; p < kP; ++p)
      if (!(p & (1 << J))) G::fs(R[p], I[p], R[p | (1 << J)], I[p | (1 << J)], s);
  }
}
template <class G>
__device__ __forceinline__ void pairs_pack_signed(Regs &R, Regs &I, float s) {
#pragma unroll
  for (int p = 0; p < kP; ++p) G::fs(R[p].x, I[p].x, R[p].y, I[p].y, s);
}
// Phase D (T or its adjoint) where register slot J is 1, then gate G on slot J, as one
// step: G's fused form fs() takes the slot-1 element as (1 +- i) y (two additions) times
// the scalar s = (sign) c, c the phase's rounding constant, so the factor 1/sqrt2 rides on
// G's fused operations instead of two multiplications per element (6 packed operations a
// pair instead of 8).  Exact in the sign; c enters each output through one fused product.
template <class G, class D, int J>
__device__ __forceinline__ void pairs_diag(Regs &R, Regs &I, float s) {
  if constexpr (J < kPR) {
#pragma unroll
    for (int p = 0; p < kP; ++p)
      if (!(p & (1 << J))) {
        constexpr int b = 1 << J;
        float2 ur, ui;
        D::u(R[p | b], I[p | b], ur, ui);
        G::fs(R[p], I[p], ur, ui, s);
        R[p | b] = ur;
        I[p | b] = ui;
      }
  }
}
// the same on the pack bit (inside every pair)
template <class G, class D>
__device__ __forceinline__ void pairs_pack_diag(Regs &R, Regs &I, float s) {
#pragma unroll
  for (int p = 0; p < kP; ++p) {
    float ur, ui;
    D::u(R[p].y, I[p].y, ur, ui);
    G::fs(R[p].x, I[p].x, ur, ui, s);
    R[p].y = ur;
    I[p].y = ui;
  }
}
// phase D (T or its adjoint, rounding constant c) where register slot J is 1
template <class D, int J>
__device__ __forceinline__ void diag(Regs &R, Regs &I, float c) {
  if constexpr (J < kPR) {
#pragma unroll
    for (int p = 0; p < kP; ++p)
      if (p & (1 << J)) D::f(R[p], I[p], c);
  }
}
// phase D where the pack bit is 1
template <class D>
__device__ __forceinline__ void diag_pack(Regs &R, Regs &I, float c) {
#pragma unroll
  for (int p = 0; p < kP; ++p) D::f(R[p].y, I[p].y, c);
}
// factor f (a sign or a 0/1 projector) where register slot J equals B
template <int J, int B>
__device__ __forceinline__ void factor(Regs &R, Regs &I, float f) {
  if constexpr (J < kPR) {
    const float2 ff = f2(f, f);
#pragma unroll
    for (int p = 0; p < kP; ++p)
      if (((p >> J) & 1) == B) { R[p] = mul2(R[p], ff); I[p] = mul2(I[p], ff); }
  }
}
// -1 where register slot J equals B (a plain negation: the compiler may fold it into
// the next operation's operand)
template <int J, int B>
__device__ __forceinline__ void negate(Regs &R, Regs &I) {
  if constexpr (J < kPR) {
#pragma unroll
    for (int p = 0; p < kP; ++p)
      if (((p >> J) & 1) == B) { R[p] = f2(-R[p].x, -R[p].y); I[p] = f2(-I[p].x, -I[p].y); }
  }
}
// -1 where the pack bit equals B
template <int B>
__device__ __forceinline__ void negate_pack(Regs &R, Regs &I) {
#pragma unroll
  for (int p = 0; p < kP; ++p) {
    if (B) { R[p].y = -R[p].y; I[p].y = -I[p].y; }
    else { R[p].x = -R[p].x; I[p].x = -I[p].x; }
  }
}
// factor f where the pack bit equals B
template <int B>
__device__ __forceinline__ void factor_pack(Regs &R, Regs &I, float f) {
  const float2 ff = B ? f2(1.f, f) : f2(f, 1.f);
#pragma unroll
  for (int p = 0; p < kP; ++p) { R[p] = mul2(R[p], ff); I[p] = mul2(I[p], ff); }
}
// CZ (EQ false: -1 where slots J and K are both 1) or the branch projector (EQ true:
// 0 where they differ); J < K, K may be the pack slot
template <int J, int K, bool EQ>
__device__ __forceinline__ void two(Regs &R, Regs &I) {
  if constexpr (J < kPR && (K < kPR || K == svp::kPackSlot)) {
#pragma unroll
    for (int p = 0; p < kP; ++p) {
      const int bj = (p >> J) & 1;
      if constexpr (K == svp::kPackSlot) {
        if (EQ) {
          if (bj) { R[p].x = 0.f; I[p].x = 0.f; }
          else { R[p].y = 0.f; I[p].y = 0.f; }
        } else if (bj) {
          R[p].y = -R[p].y;
          I[p].y = -I[p].y;
        }
      } else {
        const int bk = (p >> K) & 1;
        if (EQ) {
          if (bj != bk) { R[p] = f2(0.f, 0.f); I[p] = f2(0.f, 0.f); }
        } else if (bj && bk) {
          R[p] = f2(-R[p].x, -R[p].y);
          I[p] = f2(-I[p].x, -I[p].y);
        }
      }
    }
  }
}

__device__ __forceinline__ void scale_all(Regs &R, Regs &I, float f) {
  const float2 ff = f2(f, f);
#pragma unroll
  for (int p = 0; p < kP; ++p) { R[p] = mul2(R[p], ff); I[p] = mul2(I[p], ff); }
}

// every element times w^p, w = e^{i pi/4}
__device__ __forceinline__ void phase_all(Regs &R, Regs &I, int p) {
  const float2 m1 = f2(-1.f, -1.f);
  switch (p & 7) {
    case 0: break;
    case 4: scale_all(R, I, -1.f); break;
    case 2:  // times i: (r, i) -> (-i, r)
#pragma unroll
      for (int q = 0; q < kP; ++q) { const float2 r = R[q]; R[q] = mul2(I[q], m1); I[q] = r; }
      break;
    case 6:  // times -i: (r, i) -> (i, -r)
#pragma unroll
      for (int q = 0; q < kP; ++q) { const float2 r = R[q]; R[q] = I[q]; I[q] = mul2(r, m1); }
      break;
    default: {  // odd p: (sr + i si)/sqrt2 with sr, si = +-1
      const float sr = (p == 1 || p == 7) ? 1.f : -1.f;
      const float si = (p == 1 || p == 3) ? 1.f : -1.f;
#pragma unroll
      for (int q = 0; q < kP; ++q) {
        const float2 a = fma2(R[q], f2(sr, sr), mul2(I[q], f2(-si, -si)));
        const float2 b = fma2(I[q], f2(sr, sr), mul2(R[q], f2(si, si)));
        R[q] = rs2x2(a);
        I[q] = rs2x2(b);
      }
    }
  }
}

#ifndef SV_PLAN_KERNELS  // the interpreter: not needed by the kernels compiled for one plan
// One op by its flat code.  `cond`: the op's condition on the thread's fixed qubits.
// Signs and projectors of conditional diagonal ops become factors (1 where the
// condition fails); scalar phases and zeroing of the group are only recorded.  The
// planner makes every other kind of op unconditional in a packed plan and emits no
// general 2x2 op for the gate set.
#define SV_P6(M, A) M(A, 0) M(A, 1) M(A, 2) M(A, 3) M(A, 4)
#define SV_PAIR_CASE(G, J) case svp::P_PAIR + 6 * G##_I + J: pairs<G, J>(R, I); break;
#define SV_DIAG_CASE(D, J) case svp::P_DIAG + 6 * D##_I + J: diag<D, J>(R, I, tc); break;
#define SV_Z_CASE(X, J) \
  case svp::P_DIAG + 12 + J: factor<J, 1>(R, I, fz); break; \
  case svp::P_DIAG + 18 + J: factor<J, 1>(R, I, f0); break; \
  case svp::P_DIAG + 24 + J: factor<J, 0>(R, I, f0); break;
#define SV_TWO_CASE(J, K) \
  case svp::P_CZ + 6 * J + K: two<J, K, false>(R, I); break; \
  case svp::P_PEQ + 6 * J + K: two<J, K, true>(R, I); break;

constexpr int GH_I = 0, GSX_I = 1, GSY_I = 2, GSXDG_I = 3, GSYDG_I = 4, DT1_I = 0, DTDG1_I = 1;

// The op's code and argument (the first word of its 16-byte head).
__device__ __forceinline__ void apply_op(Regs &R, Regs &I, uint32_t code, uint32_t arg, bool cond, int &ph,
                                         bool &zero) {
  using namespace svp;
  const float fz = cond ? -1.f : 1.f, f0 = cond ? 0.f : 1.f;
  const float tc = arg ? kS2up : kS2dn;  // T ops: the plan's rounding choice
  switch (code) {
    SV_P6(SV_PAIR_CASE, GH)
    case P_PAIR + 0 + kPackSlot: pairs_pack<GH>(R, I); break;
    SV_P6(SV_PAIR_CASE, GSX)
    case P_PAIR + 6 + kPackSlot: pairs_pack<GSX>(R, I); break;
    SV_P6(SV_PAIR_CASE, GSY)
    case P_PAIR + 12 + kPackSlot: pairs_pack<GSY>(R, I); break;
    SV_P6(SV_PAIR_CASE, GSXDG)
    case P_PAIR + 18 + kPackSlot: pairs_pack<GSXDG>(R, I); break;
    SV_P6(SV_PAIR_CASE, GSYDG)
    case P_PAIR + 24 + kPackSlot: pairs_pack<GSYDG>(R, I); break;
    SV_P6(SV_DIAG_CASE, DT1)
    case P_DIAG + 0 + kPackSlot: diag_pack<DT1>(R, I, tc); break;
    SV_P6(SV_DIAG_CASE, DTDG1)
    case P_DIAG + 6 + kPackSlot: diag_pack<DTDG1>(R, I, tc); break;
    SV_P6(SV_Z_CASE, 0)
    case P_DIAG + 12 + kPackSlot: factor_pack<1>(R, I, fz); break;
    case P_DIAG + 18 + kPackSlot: factor_pack<1>(R, I, f0); break;
    case P_DIAG + 24 + kPackSlot: factor_pack<0>(R, I, f0); break;
    SV_TWO_CASE(0, 1) SV_TWO_CASE(0, 2) SV_TWO_CASE(0, 3) SV_TWO_CASE(0, 4) SV_TWO_CASE(0, 5)
    SV_TWO_CASE(1, 2) SV_TWO_CASE(1, 3) SV_TWO_CASE(1, 4) SV_TWO_CASE(1, 5)
    SV_TWO_CASE(2, 3) SV_TWO_CASE(2, 4) SV_TWO_CASE(2, 5)
    SV_TWO_CASE(3, 4) SV_TWO_CASE(3, 5)
    SV_TWO_CASE(4, 5)
    case P_PHASE: ph += cond ? (int)arg : 0; break;
    case P_ZERO: zero = zero || cond; break;
    case P_SCALE: scale_all(R, I, __int_as_float((127 - (int)arg) << 23)); break;  // 2^-arg, exact
    case P_GLOBAL:
      switch (arg & 15u) {
        case 1: global_factor<1, 0>(R, I); break;
        case 2: global_factor<2, 0>(R, I); break;
        case 3: global_factor<3, 0>(R, I); break;
        case 4: global_factor<4, 0>(R, I); break;
        case 5: global_factor<5, 0>(R, I); break;
        case 6: global_factor<6, 0>(R, I); break;
        case 7: global_factor<7, 0>(R, I); break;
        case 8: global_factor<0, 1>(R, I); break;
        case 9: global_factor<1, 1>(R, I); break;
        case 10: global_factor<2, 1>(R, I); break;
        case 11: global_factor<3, 1>(R, I); break;
        case 12: global_factor<4, 1>(R, I); break;
        case 13: global_factor<5, 1>(R, I); break;
        case 14: global_factor<6, 1>(R, I); break;
        case 15: global_factor<7, 1>(R, I); break;
        default: break;
      }
      break;
    default: break;
  }
}
#undef SV_P6
#undef SV_PAIR_CASE
#undef SV_DIAG_CASE
#undef SV_Z_CASE
#undef SV_TWO_CASE

// The stage's ops in order; the op after the current one is loaded while it runs (the
// plan ends with a no-op, so the load after a stage's last op stays inside it).  W: the
// thread's condition word.
__device__ __forceinline__ void apply_ops(Regs &R, Regs &I, const DevOp *ops, const DevStage &st, uint32_t W) {
  int ph = 0;
  bool zero = false;
  const uint4 *head = reinterpret_cast<const uint4 *>(ops + st.op_begin);
  const int stride = sizeof(DevOp) / sizeof(uint4);
  uint4 h = head[0];
  for (int o = 0; o < st.op_count; ++o) {
    const uint4 nxt = head[(o + 1) * stride];
    apply_op(R, I, h.x & 0xffu, (h.x >> 8) & 0xffu, (W & h.z) == h.w, ph, zero);
    h = nxt;
  }
  if (zero) {
    scale_all(R, I, 0.f);
  } else {
    if (st.halves) scale_all(R, I, __int_as_float((127 - st.halves) << 23));  // 2^-halves, exact
    if (ph & 7) phase_all(R, I, ph & 7);
  }
}

#endif  // SV_PLAN_KERNELS

// ---- addressing ---------------------------------------------------------------------------
// 16-byte slot of pair k (tile bits 1..m-1): pair bit i toggles slot bit i mod 3, so the
// 8 lanes of a quarter warp hit distinct 16-byte bank groups when the planner gives them
// three pair bits of distinct residues.  Linear over XOR.
__device__ __forceinline__ uint32_t pack_phys(uint32_t k) { return k ^ (((k >> 3) ^ (k >> 6) ^ (k >> 9)) & 7u); }

// Byte offset of group g's first pair.
__device__ __forceinline__ uint32_t group_base(const DevPlanView &plan, uint32_t si, int g) {
  const svp::DevGroupEntry *t = plan.gtab + svp::kGroupEntries * si;
  return t[g & 15].L ^ t[16 + ((g >> 4) & 15)].L ^ t[32 + ((g >> 8) & 15)].L;
}

__device__ __forceinline__ void load_group(const float4 *tile, const DevPlanView &plan, uint32_t si, uint32_t a0,
                                           Regs &R, Regs &I) {
  const svp::DevGroupEntry *t = plan.gtab + svp::kGroupEntries * si + svp::kRegEntry;
  uint32_t rx[kPR];
#pragma unroll
  for (int j = 0; j < kPR; ++j) rx[j] = t[j].L;
  const char *tb = reinterpret_cast<const char *>(tile);
#pragma unroll
  for (int p = 0; p < kP; ++p) {
    uint32_t a = a0;
#pragma unroll
    for (int j = 0; j < kPR; ++j)
      if ((p >> j) & 1) a ^= rx[j];
    const float4 x = *reinterpret_cast<const float4 *>(tb + a);
    R[p] = f2(x.x, x.y);
    I[p] = f2(x.z, x.w);
  }
}

__device__ __forceinline__ void store_group(float4 *tile, const DevPlanView &plan, uint32_t si, uint32_t a0,
                                            const Regs &R, const Regs &I) {
  const svp::DevGroupEntry *t = plan.gtab + svp::kGroupEntries * si + svp::kRegEntry;
  uint32_t rx[kPR];
#pragma unroll
  for (int j = 0; j < kPR; ++j) rx[j] = t[j].L;
  char *tb = reinterpret_cast<char *>(tile);
#pragma unroll
  for (int p = 0; p < kP; ++p) {
    uint32_t a = a0;
#pragma unroll
    for (int j = 0; j < kPR; ++j)
      if ((p >> j) & 1) a ^= rx[j];
    *reinterpret_cast<float4 *>(tb + a) = make_float4(R[p].x, R[p].y, I[p].x, I[p].y);
  }
}

// The same with the register-slot masks given (the kernels compiled for one plan pass
// them as constants).
// kCopied: the tile is still as the asynchronous copies left it, pairs as
// (re, im, re', im') (the first stage of a pass that read its tile; see finish_tile_load).
template <bool kCopied = false>
__device__ __forceinline__ void load_group_rx(const float4 *tile, uint32_t a0, const uint32_t (&rx)[kPR], Regs &R,
                                              Regs &I) {
  const char *tb = reinterpret_cast<const char *>(tile);
#pragma unroll
  for (int p = 0; p < kP; ++p) {
    uint32_t a = a0;
#pragma unroll
    for (int j = 0; j < kPR; ++j)
      if ((p >> j) & 1) a ^= rx[j];
    const float4 x = *reinterpret_cast<const float4 *>(tb + a);
    R[p] = kCopied ? f2(x.x, x.z) : f2(x.x, x.y);
    I[p] = kCopied ? f2(x.y, x.w) : f2(x.z, x.w);
  }
}
// kGlobal: store each pair as (re, im, re', im'), the order of the state in memory (a
// tile that a TMA copy then writes out as it is).
template <bool kGlobal = false>
__device__ __forceinline__ void store_group_rx(float4 *tile, uint32_t a0, const uint32_t (&rx)[kPR], const Regs &R,
                                               const Regs &I) {
  char *tb = reinterpret_cast<char *>(tile);
#pragma unroll
  for (int p = 0; p < kP; ++p) {
    uint32_t a = a0;
#pragma unroll
    for (int j = 0; j < kPR; ++j)
      if ((p >> j) & 1) a ^= rx[j];
    *reinterpret_cast<float4 *>(tb + a) =
        kGlobal ? make_float4(R[p].x, I[p].x, R[p].y, I[p].y) : make_float4(R[p].x, R[p].y, I[p].x, I[p].y);
  }
}

// End of a stage's ops: the recorded zeroing, deferred factors 1/2 and scalar phase.
__device__ __forceinline__ void end_stage(Regs &R, Regs &I, int halves, int ph, bool zero) {
  if (zero) {
    scale_all(R, I, 0.f);
  } else {
    if (halves) scale_all(R, I, __int_as_float((127 - halves) << 23));  // 2^-halves, exact
    if (ph & 7) phase_all(R, I, ph & 7);
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

// Shared memory holds pair k at slot pack_phys(k) as (re, re', im, im').  Thread t moves
// pairs t, t + T, ... (T threads, kP pairs each) in coalesced 16-byte vectors.

// Asynchronous read (cp.async through L2, no register staging) of the pairs as they are
// in memory, (re, im, re', im'), one commit group.  L2 is coherent, so the copies also see
// data that other CTAs of the same launch wrote.  finish_tile_load() waits for the
// thread's own copies and regroups them (each thread touches only its own slots).
// The plan-specialised kernels call finish_tile_copy() instead: it only waits, and their
// first stage reads the pairs in the copied order (load_group_rx<true>) and stores them
// regrouped, so the tile needs no regroup sweep (34 qubits: 0.667 -> 0.638 s).  In the
// interpreting kernel the same change measured slower (its stage loop then holds two
// copies of the group load).
// (tid, T): this thread's index among the T threads that share the tile.
__device__ __forceinline__ void load_tile_async(const float2 *__restrict__ psi, float4 *tile, const DevPass &P,
                                                const uint64_t *chunk_off, uint64_t base, uint32_t tid, uint32_t T) {
  const int cp = P.c - 1;  // pair bits inside a chunk of 2^c amplitudes
  const uint32_t in_mask = (1u << cp) - 1;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tile);
#pragma unroll 4
  for (int it = 0; it < kP; ++it) {
    const uint32_t k = tid + (uint32_t)it * T;
    const float2 *src = psi + base + chunk_off[k >> cp] + 2 * (k & in_mask);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sbase + 16u * pack_phys(k)), "l"(src)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void finish_tile_load(float4 *tile, uint32_t tid, uint32_t T) {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll 4
  for (int it = 0; it < kP; ++it) {
    float4 &x = tile[pack_phys(tid + (uint32_t)it * T)];
    const float4 y = x;
    x = make_float4(y.x, y.z, y.y, y.w);
  }
}

__device__ __forceinline__ void store_tile(float2 *__restrict__ psi, const float4 *tile, const DevPass &P,
                                           const uint64_t *chunk_off, uint64_t base, uint32_t tid, uint32_t T) {
  const int cp = P.c - 1;
  const uint32_t in_mask = (1u << cp) - 1;
#pragma unroll 4
  for (int it = 0; it < kP; ++it) {
    const uint32_t k = tid + (uint32_t)it * T;
    const float4 x = tile[pack_phys(k)];
    *reinterpret_cast<float4 *>(psi + base + chunk_off[k >> cp] + 2 * (k & in_mask)) = make_float4(x.x, x.z, x.y, x.w);
  }
}

// store_tile that also adds the stored amplitudes' probabilities p and p^2 to a2 and
// a4: per tile in fp32 (32 values per thread), across tiles in fp64 (the reductions of
// the state's norm, fused into the pass that writes it).
__device__ __forceinline__ void store_tile_sums(float2 *__restrict__ psi, const float4 *tile, const DevPass &P,
                                                const uint64_t *chunk_off, uint64_t base, double &a2, double &a4) {
  const int cp = P.c - 1;
  const uint32_t in_mask = (1u << cp) - 1;
  const uint32_t tid = threadIdx.x, T = blockDim.x;
  float s2 = 0.f, s4 = 0.f;
#pragma unroll 4
  for (int it = 0; it < kP; ++it) {
    const uint32_t k = tid + (uint32_t)it * T;
    const float4 x = tile[pack_phys(k)];  // (re, re', im, im')
    const float p0 = fmaf(x.x, x.x, x.z * x.z), p1 = fmaf(x.y, x.y, x.w * x.w);
    s2 += p0 + p1;
    s4 = fmaf(p0, p0, fmaf(p1, p1, s4));
    *reinterpret_cast<float4 *>(psi + base + chunk_off[k >> cp] + 2 * (k & in_mask)) = make_float4(x.x, x.z, x.y, x.w);
  }
  a2 += (double)s2;
  a4 += (double)s4;
}

// <phi|psi> over the tile instead of storing it: phi = the tile as the stages left it,
// psi read from `other` at the same positions; conj(phi) psi summed in fp32 over the
// thread's 32 amplitudes, then into the fp64 sums re, im.
__device__ __forceinline__ void inner_tile(const float2 *__restrict__ other, const float4 *tile, const DevPass &P,
                                           const uint64_t *chunk_off, uint64_t base, double &re, double &im) {
  const int cp = P.c - 1;
  const uint32_t in_mask = (1u << cp) - 1;
  const uint32_t tid = threadIdx.x, T = blockDim.x;
  float sr = 0.f, si = 0.f;
#pragma unroll 4
  for (int it = 0; it < kP; ++it) {
    const uint32_t k = tid + (uint32_t)it * T;
    const float4 x = tile[pack_phys(k)];  // phi: (re, re', im, im')
    const float4 y = *reinterpret_cast<const float4 *>(other + base + chunk_off[k >> cp] + 2 * (k & in_mask));
    // psi: (re, im, re', im');  conj(a) b = (a.re b.re + a.im b.im) + i (a.re b.im - a.im b.re)
    sr = fmaf(x.x, y.x, fmaf(x.z, y.y, sr));
    sr = fmaf(x.y, y.z, fmaf(x.w, y.w, sr));
    si = fmaf(x.x, y.y, fmaf(-x.z, y.x, si));
    si = fmaf(x.y, y.w, fmaf(-x.w, y.z, si));
  }
  re += (double)sr;
  im += (double)si;
}

// The CTA's sums (fixed order) to partials[2 blockIdx.x], [2 blockIdx.x + 1].
__device__ __forceinline__ void block_sums_out(double a2, double a4, double *partials) {
  __shared__ double r2[32], r4[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    a4 += __shfl_xor_sync(0xffffffffu, a4, o);
  }
  if ((threadIdx.x & 31) == 0) { r2[threadIdx.x >> 5] = a2; r4[threadIdx.x >> 5] = a4; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t2 = 0.0, t4 = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) { t2 += r2[w]; t4 += r4[w]; }
    partials[2 * blockIdx.x] = t2;
    partials[2 * blockIdx.x + 1] = t4;
  }
}

// The generated first tile of a fresh state: 2^{-n/2} everywhere, or |0..0> (element 0
// of group 0 of tile 0, the thread with condition word 0).
__device__ __forceinline__ void init_regs(Regs &R, Regs &I, const DevPass &P, uint32_t W) {
  const float a = (P.flags & svp::PF_INIT_UNIFORM) ? P.init_amp : 0.f;
#pragma unroll
  for (int p = 0; p < kP; ++p) { R[p] = f2(a, a); I[p] = f2(0.f, 0.f); }
  if (!(P.flags & svp::PF_INIT_UNIFORM) && W == 0) R[0].x = 1.f;
}

__device__ __forceinline__ void init_tile(float4 *tile, const DevPass &P, uint64_t base, uint32_t tid, uint32_t T) {
  const float a = (P.flags & svp::PF_INIT_UNIFORM) ? P.init_amp : 0.f;
  for (uint32_t k = tid; k < (1u << (P.m - 1)); k += T) tile[k] = make_float4(a, a, 0.f, 0.f);
  if (!(P.flags & svp::PF_INIT_UNIFORM) && base == 0 && tid == 0) tile[0] = make_float4(1.f, 0.f, 0.f, 0.f);
}

// The same for a CTA whose threads all share one tile.
__device__ __forceinline__ void load_tile_async(const float2 *__restrict__ psi, float4 *tile, const DevPass &P,
                                                const uint64_t *chunk_off, uint64_t base) {
  load_tile_async(psi, tile, P, chunk_off, base, threadIdx.x, blockDim.x);
}
__device__ __forceinline__ void finish_tile_load(float4 *tile) { finish_tile_load(tile, threadIdx.x, blockDim.x); }
// Wait only (a pass without stages still regroups, for store_tile).
__device__ __forceinline__ void finish_tile_copy(float4 *tile, const DevPass &P) {
  if (P.stage_count == 0) finish_tile_load(tile);
  else asm volatile("cp.async.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void store_tile(float2 *__restrict__ psi, const float4 *tile, const DevPass &P,
                                           const uint64_t *chunk_off, uint64_t base) {
  store_tile(psi, tile, P, chunk_off, base, threadIdx.x, blockDim.x);
}
__device__ __forceinline__ void init_tile(float4 *tile, const DevPass &P, uint64_t base) {
  init_tile(tile, P, base, threadIdx.x, blockDim.x);
}

#ifndef SV_PLAN_KERNELS  // the interpreter
// One tile of one packed pass whose data is in `tile` (or is generated): every stage in
// registers, then the store.  Ends with __syncthreads.
__device__ __forceinline__ void process_tile(float2 *__restrict__ psi, const DevPlanView &plan, const DevPass &P,
                                             const uint64_t *chunk_off, float4 *tile, uint64_t tile_id) {
  const int tid = threadIdx.x;
  const uint64_t base = tile_base(P, tile_id);
  const bool init = (P.flags & (svp::PF_INIT_UNIFORM | svp::PF_INIT_ZERO)) != 0;
  if (init && P.stage_count == 0) {
    init_tile(tile, P, base);
    __syncthreads();
  }
  // condition word: the group index below the tile index (n - 1 - kPR <= 32 bits)
  const uint32_t W = ((uint32_t)tile_id << (P.m - 1 - kPR)) | (uint32_t)tid;
  for (int s = 0; s < P.stage_count; ++s) {
    const uint32_t si = P.stage_begin + s;
    const DevStage &st = plan.stages[si];
    Regs R, I;
    if (s == 0 && init) init_regs(R, I, P, W);
    else load_group(tile, plan, si, group_base(plan, si, tid), R, I);
    apply_ops(R, I, plan.ops, st, W);
    // Recompute the address rather than keeping it live across the ops.
    asm volatile("" ::: "memory");
    store_group(tile, plan, si, group_base(plan, si, tid), R, I);
    __syncthreads();
  }
  store_tile(psi, tile, P, chunk_off, base);
  __syncthreads();
}

// A CTA's sweep over its tiles (tile_id = first, first + stride, ...): read, process.
// (A second buffer with the next tile's read in flight measured slower: it halves the
// resident CTAs, and this kernel is bound by latency, not by bandwidth.)
__device__ __forceinline__ void sweep_tiles(float2 *__restrict__ psi, const DevPlanView &plan, const DevPass &P,
                                            const uint64_t *chunk_off, float4 *tile, uint64_t first, uint64_t stride,
                                            uint64_t num_tiles) {
  const bool init = (P.flags & (svp::PF_INIT_UNIFORM | svp::PF_INIT_ZERO)) != 0;
  for (uint64_t tile_id = first; tile_id < num_tiles; tile_id += stride) {
    if (!init) {
      load_tile_async(psi, tile, P, chunk_off, tile_base(P, tile_id));
      finish_tile_load(tile);
      __syncthreads();
    }
    process_tile(psi, plan, P, chunk_off, tile, tile_id);
  }
}

#endif  // SV_PLAN_KERNELS

}  // namespace tpk
}  // namespace svk

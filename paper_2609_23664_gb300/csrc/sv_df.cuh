// Compensated FP32 arithmetic for the statevector pass kernels.
//
// An amplitude is held as an unevaluated sum h + l of two FP32 complex
// numbers (double-float): |l| stays within a few units in the last place of
// |h|.  Every register operation computes its exact result up to terms of
// order 2^-48 relative: products are split exactly with one FMA (p = c*x,
// e = fma(c, x, -p) gives c*x = p + e), sums exactly with TwoSum (Knuth,
// TAOCP vol. 2, 4.2.2; s = a + b, e = (a - (s - z)) + (b - z) with z = s - a
// gives a + b = s + e), and the gate constants carry their own FP32
// remainder (c = ch + cl, the exact double value to 2^-48).  The remainder l
// collects these error terms and is renormalized once per stage
// (Fast2Sum, exact because |h| >= |l|).
//
// Without it, the FP32 roundings of the ~600 rotations that every amplitude
// of a 24-qubit, 24-layer ansatz goes through move a Pauli-sum energy by
// about 1e-6 of its typical size; with it, the state is rounded only when it
// is written back to FP32 storage.
//
// Both components of a complex amplitude go through the same real
// coefficients, so the arithmetic is written on float2 with the packed
// two-lane FP32 instructions.
#pragma once

#include <cuda_runtime.h>

namespace qw {

__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2swap(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, f2neg(b)); }

// r = c1 * x + c2 * y, componentwise; coefficients and operands double-float
// (ZL: the operands' remainders xl, yl are zero and not read)
template <bool ZL = false>
__device__ __forceinline__ void df_lin2(float2 c1h, float2 c1l, float2 xh, float2 xl, float2 c2h, float2 c2l,
                                        float2 yh, float2 yl, float2 &rh, float2 &rl) {
  const float2 p = __fmul2_rn(c1h, xh);
  const float2 ep = __ffma2_rn(c1h, xh, f2neg(p));  // c1h*xh = p + ep exactly
  const float2 q = __fmul2_rn(c2h, yh);
  const float2 eq = __ffma2_rn(c2h, yh, f2neg(q));
  const float2 s = __fadd2_rn(p, q);                // TwoSum: p + q = s + es exactly
  const float2 z = f2sub(s, p);
  const float2 es = __fadd2_rn(f2sub(p, f2sub(s, z)), f2sub(q, z));
  float2 l = ep;
  if constexpr (!ZL) {
    l = __ffma2_rn(c1h, xl, l);
    l = __ffma2_rn(c2h, yl, l);
  }
  l = __ffma2_rn(c1l, xh, l);
  l = __ffma2_rn(c2l, yh, l);
  rl = __fadd2_rn(l, __fadd2_rn(eq, es));
  rh = s;
}

// r = a + b (double-float)
__device__ __forceinline__ void df_add(float2 ah, float2 al, float2 bh, float2 bl, float2 &rh, float2 &rl) {
  const float2 s = __fadd2_rn(ah, bh);
  const float2 z = f2sub(s, ah);
  const float2 e = __fadd2_rn(f2sub(ah, f2sub(s, z)), f2sub(bh, z));
  rl = __fadd2_rn(__fadd2_rn(al, bl), e);
  rh = s;
}

// z <- w z for a complex constant w = (wr, wi), both parts double-float:
// (wr zr - wi zi, wr zi + wi zr) = wr (zr, zi) + (-wi, wi) (zi, zr)
__device__ __forceinline__ void df_cmul(float wrh, float wrl, float wih, float wil, float2 &zh, float2 &zl) {
  float2 rh, rl;
  df_lin2(f2s(wrh), f2s(wrl), zh, zl, make_float2(-wih, wih), make_float2(-wil, wil), f2swap(zh), f2swap(zl), rh,
          rl);
  zh = rh;
  zl = rl;
}

// h + l rounded into h, the rest kept in l (|h| >= |l|)
__device__ __forceinline__ void df_renorm(float2 &h, float2 &l) {
  const float2 s = __fadd2_rn(h, l);
  l = f2sub(l, f2sub(s, h));
  h = s;
}

// ---- register operations on the N = 2^G amplitudes of a stage group ------
// m / ml: the op's parameters (see SvKind) and their FP32 remainders.

// real 2x2 {r00, r01; r10, r11} on position P, then (when phase) diag(1, p)
// with p = (m[4], m[5]): K_RP layout {r00, r01, r10, r11, pr, pi}.  Every
// pair's rotation is issued before the phase products, which depend on them
// (measured: 442 ms against 463 ms for the 256-task suffix launch)
// (ZL: every remainder l is zero on entry, as in the first op of a stage
// that reads rounded amplitudes)
template <int P, int N, bool ZL = false>
__device__ __forceinline__ void dfop_rp(float2 (&h)[N], float2 (&l)[N], const float (&m)[8], const float (&ml)[8],
                                        bool phase) {
  const float2 r00 = f2s(m[0]), r01 = f2s(m[1]), r10 = f2s(m[2]), r11 = f2s(m[3]);
  const float2 e00 = f2s(ml[0]), e01 = f2s(ml[1]), e10 = f2s(ml[2]), e11 = f2s(ml[3]);
#pragma unroll
  for (int i = 0; i < N; i++) {
    if (i & (1 << P)) continue;
    const int j = i | (1 << P);
    const float2 xh = h[i], xl = l[i], yh = h[j], yl = l[j];
    df_lin2<ZL>(r00, e00, xh, xl, r01, e01, yh, yl, h[i], l[i]);
    df_lin2<ZL>(r10, e10, xh, xl, r11, e11, yh, yl, h[j], l[j]);
  }
  if (phase) {
#pragma unroll
    for (int i = 0; i < N; i++)
      if (i & (1 << P)) df_cmul(m[4], ml[4], m[5], ml[5], h[i], l[i]);
  }
}
// K_R layout {r00, 0, r01, 0, r10, 0, r11, 0}
template <int P, int N>
__device__ __forceinline__ void dfop_r(float2 (&h)[N], float2 (&l)[N], const float (&m)[8], const float (&ml)[8]) {
  const float2 r00 = f2s(m[0]), r01 = f2s(m[2]), r10 = f2s(m[4]), r11 = f2s(m[6]);
  const float2 e00 = f2s(ml[0]), e01 = f2s(ml[2]), e10 = f2s(ml[4]), e11 = f2s(ml[6]);
#pragma unroll
  for (int i = 0; i < N; i++) {
    if (i & (1 << P)) continue;
    const int j = i | (1 << P);
    const float2 xh = h[i], xl = l[i], yh = h[j], yl = l[j];
    df_lin2(r00, e00, xh, xl, r01, e01, yh, yl, h[i], l[i]);
    df_lin2(r10, e10, xh, xl, r11, e11, yh, yl, h[j], l[j]);
  }
}
// general 2x2 {u00, u01; u10, u11}, complex entries (re, im) in m[0..7]
template <int P, int N>
__device__ __forceinline__ void dfop_u1(float2 (&h)[N], float2 (&l)[N], const float (&m)[8], const float (&ml)[8]) {
#pragma unroll
  for (int i = 0; i < N; i++) {
    if (i & (1 << P)) continue;
    const int j = i | (1 << P);
    const float2 xh = h[i], xl = l[i], yh = h[j], yl = l[j];
#pragma unroll
    for (int r = 0; r < 2; r++) {
      // u_r0 x + u_r1 y = [Re u_r0 x + Im u_r0 (-xi, xr)] + [same for y]
      const int o = 4 * r;
      float2 ah, al, bh, bl;
      df_lin2(f2s(m[o]), f2s(ml[o]), xh, xl, make_float2(-m[o + 1], m[o + 1]), make_float2(-ml[o + 1], ml[o + 1]),
              f2swap(xh), f2swap(xl), ah, al);
      df_lin2(f2s(m[o + 2]), f2s(ml[o + 2]), yh, yl, make_float2(-m[o + 3], m[o + 3]),
              make_float2(-ml[o + 3], ml[o + 3]), f2swap(yh), f2swap(yl), bh, bl);
      if (r == 0) df_add(ah, al, bh, bl, h[i], l[i]);
      else df_add(ah, al, bh, bl, h[j], l[j]);
    }
  }
}
// diag(d0, d1): m = {d0r, d0i, d1r, d1i}
template <int P, int N>
__device__ __forceinline__ void dfop_d1(float2 (&h)[N], float2 (&l)[N], const float (&m)[8], const float (&ml)[8]) {
#pragma unroll
  for (int i = 0; i < N; i++) {
    const int o = (i & (1 << P)) ? 2 : 0;
    df_cmul(m[o], ml[o], m[o + 1], ml[o + 1], h[i], l[i]);
  }
}
// diag(1, p): m = {pr, pi}
template <int P, int N>
__device__ __forceinline__ void dfop_p1(float2 (&h)[N], float2 (&l)[N], const float (&m)[8], const float (&ml)[8]) {
#pragma unroll
  for (int i = 0; i < N; i++)
    if (i & (1 << P)) df_cmul(m[0], ml[0], m[1], ml[1], h[i], l[i]);
}
// amplitudes with bits A and B set times p = {pr, pi}; p = -1 (CZ) negates
template <int A, int B, int N>
__device__ __forceinline__ void dfop_cd(float2 (&h)[N], float2 (&l)[N], const float (&m)[8], const float (&ml)[8]) {
  const bool neg = m[0] == -1.f && m[1] == 0.f && ml[0] == 0.f && ml[1] == 0.f;
#pragma unroll
  for (int i = 0; i < N; i++) {
    if (!(i & (1 << A)) || !(i & (1 << B))) continue;
    if (neg) {
      h[i] = f2neg(h[i]);
      l[i] = f2neg(l[i]);
    } else {
      df_cmul(m[0], ml[0], m[1], ml[1], h[i], l[i]);
    }
  }
}
// [[c, -is], [-is, c]]: m = {c, s}
//   x' = c x - i s y = c (xr, xi) + (s, -s) (yi, yr)
//   y' = c y - i s x = c (yr, yi) + (s, -s) (xi, xr)
template <int P, int N>
__device__ __forceinline__ void dfop_rx(float2 (&h)[N], float2 (&l)[N], const float (&m)[8], const float (&ml)[8]) {
  const float2 c = f2s(m[0]), cl = f2s(ml[0]);
  const float2 s = make_float2(m[1], -m[1]), sl = make_float2(ml[1], -ml[1]);
#pragma unroll
  for (int i = 0; i < N; i++) {
    if (i & (1 << P)) continue;
    const int j = i | (1 << P);
    const float2 xh = h[i], xl = l[i], yh = h[j], yl = l[j];
    df_lin2(c, cl, xh, xl, s, sl, f2swap(yh), f2swap(yl), h[i], l[i]);
    df_lin2(c, cl, yh, yl, s, sl, f2swap(xh), f2swap(xl), h[j], l[j]);
  }
}

// dispatch on the dense op index (the same table as the plain kernels);
// positions beyond the group (1 << P >= N) never occur in its programs
template <int N>
__device__ __forceinline__ void df_apply_op(uint32_t code, const float (&m)[8], const float (&ml)[8], float2 (&h)[N],
                                            float2 (&l)[N]) {
  switch (code) {
#define QW_ONE(K, P, F) \
  case sv_op_index(K, P, 0): if constexpr ((1 << P) < N) F<P, N>(h, l, m, ml); break;
#define QW_ALL(K, F) QW_ONE(K, 0, F) QW_ONE(K, 1, F) QW_ONE(K, 2, F) QW_ONE(K, 3, F) QW_ONE(K, 4, F)
    QW_ALL(K_U1, dfop_u1)
    QW_ALL(K_D1, dfop_d1)
    QW_ALL(K_P1, dfop_p1)
    QW_ALL(K_R, dfop_r)
    QW_ALL(K_RX, dfop_rx)
#undef QW_ALL
#undef QW_ONE
#define RP(P) case sv_op_index(K_RP, P, 0): if constexpr ((1 << P) < N) dfop_rp<P, N>(h, l, m, ml, true); break;
    RP(0) RP(1) RP(2) RP(3) RP(4)
#undef RP
#define CD(x, y) case sv_op_index(K_CD, x, y): if constexpr ((1 << y) < N) dfop_cd<x, y, N>(h, l, m, ml); break;
    CD(0, 1) CD(0, 2) CD(0, 3) CD(0, 4) CD(1, 2) CD(1, 3) CD(1, 4) CD(2, 3) CD(2, 4) CD(3, 4)
#undef CD
    default: break;
  }
}

// K_RP at a position known once the caller's loop is unrolled; a rotation
// without phase (p = 1 exactly) skips the complex product
template <int N>
__device__ __forceinline__ void df_rp_at(int P, float2 (&h)[N], float2 (&l)[N], const float (&m)[8],
                                         const float (&ml)[8]) {
  const bool phase = !(m[4] == 1.f && m[5] == 0.f && ml[4] == 0.f && ml[5] == 0.f);
  switch (P) {
    case 0: dfop_rp<0, N>(h, l, m, ml, phase); break;
    case 1: dfop_rp<1, N>(h, l, m, ml, phase); break;
    case 2: dfop_rp<2, N>(h, l, m, ml, phase); break;
    case 3: dfop_rp<3, N>(h, l, m, ml, phase); break;
    default: if constexpr (N > 16) dfop_rp<4, N>(h, l, m, ml, phase); break;
  }
}

}  // namespace qw

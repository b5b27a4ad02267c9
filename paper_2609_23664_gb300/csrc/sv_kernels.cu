// Statevector gate-application kernels (sm_103a).
//
// One CTA processes one TILE of a pass: 2^k amplitudes whose non-tile bits
// are fixed.  The tile is read from HBM in contiguous runs of 2^b amplitudes,
// kept in shared memory (XOR-swizzled to spread the strided stage accesses
// over the banks), and every STAGE of the pass is applied with the 2^G
// amplitudes of a stage group held in registers (32 for plain passes, 16
// for compensated ones, which hold two FP32 values per amplitude), so that
// the gates of a stage cost no shared-memory traffic.  The prefix is executed once (Sec. III-A,
// Fig. 1); the first suffix pass of every task reads its tile from the
// boundary state and writes the task's own buffer, so the reload of the
// boundary (C_reload of Eq. 2) costs no separate copy.
//
// sv_batch_kernel runs the suffixes of many tasks in ONE persistent launch:
// CTAs take tiles from a global work list in order; a tile of pass p of a
// task waits (bounded) until every tile of pass p-1 of that task is done.
// On request the list also holds the energy blocks of each finished state.
#include <cuda_runtime.h>

#include "energy_block.cuh"
#include "qw_internal.h"
#include "sv_df.cuh"

namespace qw {

template <typename T> struct V2;
template <> struct V2<float> { typedef float2 t; };
template <> struct V2<double> { typedef double2 t; };

// Shared-memory swizzle of the tile (sv_swz32 / sv_swz64).
template <typename T> __device__ __forceinline__ uint32_t swz(uint32_t l);
template <> __device__ __forceinline__ uint32_t swz<float>(uint32_t l) { return sv_swz32(l); }
template <> __device__ __forceinline__ uint32_t swz<double>(uint32_t l) { return sv_swz64(l); }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---- register operations on the N = 2^G amplitudes of a stage group -------
template <typename C, typename T, int P, int N>
__device__ __forceinline__ void op_u1(C (&a)[N], const T (&m)[8]) {
#pragma unroll
  for (int i = 0; i < N; i++) {
    if (i & (1 << P)) continue;
    const int j = i | (1 << P);
    const C x = a[i], y = a[j];
    a[i].x = m[0] * x.x - m[1] * x.y + m[2] * y.x - m[3] * y.y;
    a[i].y = m[0] * x.y + m[1] * x.x + m[2] * y.y + m[3] * y.x;
    a[j].x = m[4] * x.x - m[5] * x.y + m[6] * y.x - m[7] * y.y;
    a[j].y = m[4] * x.y + m[5] * x.x + m[6] * y.y + m[7] * y.x;
  }
}
template <typename C, typename T, int P, int N>
__device__ __forceinline__ void op_d1(C (&a)[N], const T (&m)[8]) {
#pragma unroll
  for (int i = 0; i < N; i++) {
    const T dr = (i & (1 << P)) ? m[2] : m[0];
    const T di = (i & (1 << P)) ? m[3] : m[1];
    const C x = a[i];
    a[i].x = dr * x.x - di * x.y;
    a[i].y = dr * x.y + di * x.x;
  }
}
template <typename C, typename T, int A, int B, int N>
__device__ __forceinline__ void op_cd(C (&a)[N], const T (&m)[8]) {
#pragma unroll
  for (int i = 0; i < N; i++) {
    if (!(i & (1 << A)) || !(i & (1 << B))) continue;
    const C x = a[i];
    a[i].x = m[0] * x.x - m[1] * x.y;
    a[i].y = m[0] * x.y + m[1] * x.x;
  }
}
// diag(1, p): only the amplitudes with bit P set change
template <typename C, typename T, int P, int N>
__device__ __forceinline__ void op_p1(C (&a)[N], const T (&m)[8]) {
#pragma unroll
  for (int i = 0; i < N; i++) {
    if (!(i & (1 << P))) continue;
    const C x = a[i];
    a[i].x = m[0] * x.x - m[1] * x.y;
    a[i].y = m[0] * x.y + m[1] * x.x;
  }
}
// real 2x2 matrix {m0, m2; m4, m6}; FP32: both components of an amplitude
// in one packed op
template <typename C, typename T, int P, int N>
__device__ __forceinline__ void op_r(C (&a)[N], const T (&m)[8]) {
  if constexpr (sizeof(T) == 4) {
    const float2 m0 = make_float2(m[0], m[0]), m2 = make_float2(m[2], m[2]);
    const float2 m4 = make_float2(m[4], m[4]), m6 = make_float2(m[6], m[6]);
#pragma unroll
    for (int i = 0; i < N; i++) {
      if (i & (1 << P)) continue;
      const int j = i | (1 << P);
      const float2 x = a[i], y = a[j];
      a[i] = __ffma2_rn(m2, y, __fmul2_rn(m0, x));
      a[j] = __ffma2_rn(m6, y, __fmul2_rn(m4, x));
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; i++) {
      if (i & (1 << P)) continue;
      const int j = i | (1 << P);
      const C x = a[i], y = a[j];
      a[i].x = m[0] * x.x + m[2] * y.x;
      a[i].y = m[0] * x.y + m[2] * y.y;
      a[j].x = m[4] * x.x + m[6] * y.x;
      a[j].y = m[4] * x.y + m[6] * y.y;
    }
  }
}

// diag(1, p) after the real 2x2 {r00, r01; r10, r11}: m = {r00, r01, r10, r11, pr, pi}
template <typename C, typename T, int P, int N>
__device__ __forceinline__ void op_rp(C (&a)[N], const T (&m)[8]) {
  if constexpr (sizeof(T) == 4) {
    const float2 m0 = make_float2(m[0], m[0]), m1 = make_float2(m[1], m[1]);
    const float2 m2 = make_float2(m[2], m[2]), m3 = make_float2(m[3], m[3]);
#pragma unroll
    for (int i = 0; i < N; i++) {
      if (i & (1 << P)) continue;
      const int j = i | (1 << P);
      const float2 x = a[i], y = a[j];
      a[i] = __ffma2_rn(m1, y, __fmul2_rn(m0, x));
      const float2 t = __ffma2_rn(m3, y, __fmul2_rn(m2, x));
      a[j].x = m[4] * t.x - m[5] * t.y;
      a[j].y = m[4] * t.y + m[5] * t.x;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; i++) {
      if (i & (1 << P)) continue;
      const int j = i | (1 << P);
      const C x = a[i], y = a[j];
      a[i].x = m[0] * x.x + m[1] * y.x;
      a[i].y = m[0] * x.y + m[1] * y.y;
      const T tx = m[2] * x.x + m[3] * y.x, ty = m[2] * x.y + m[3] * y.y;
      a[j].x = m[4] * tx - m[5] * ty;
      a[j].y = m[4] * ty + m[5] * tx;
    }
  }
}

// [[c, -is], [-is, c]] with c = m0, s = m1
template <typename C, typename T, int P, int N>
__device__ __forceinline__ void op_rx(C (&a)[N], const T (&m)[8]) {
#pragma unroll
  for (int i = 0; i < N; i++) {
    if (i & (1 << P)) continue;
    const int j = i | (1 << P);
    const C x = a[i], y = a[j];
    a[i].x = m[0] * x.x + m[1] * y.y;
    a[i].y = m[0] * x.y - m[1] * y.x;
    a[j].x = m[1] * x.y + m[0] * y.x;
    a[j].y = m[0] * y.y - m[1] * x.x;
  }
}

// the eight matrix parameters of an op as 16-byte loads
__device__ __forceinline__ void load_m(const SvOpDesc<float> *op, float (&m)[8]) {
  const float4 u = __ldg((const float4 *)op->m), v = __ldg((const float4 *)(op->m + 4));
  m[0] = u.x; m[1] = u.y; m[2] = u.z; m[3] = u.w;
  m[4] = v.x; m[5] = v.y; m[6] = v.z; m[7] = v.w;
}
__device__ __forceinline__ void load_m(const SvOpDesc<double> *op, double (&m)[8]) {
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const double2 u = __ldg((const double2 *)(op->m + 2 * i));
    m[2 * i] = u.x;
    m[2 * i + 1] = u.y;
  }
}

// K_RP at a position known once the caller's loop is unrolled
template <typename C, typename T, int N>
__device__ __forceinline__ void rp_at(int P, C (&a)[N], const T (&m)[8]) {
  switch (P) {
    case 0: op_rp<C, T, 0, N>(a, m); break;
    case 1: op_rp<C, T, 1, N>(a, m); break;
    case 2: op_rp<C, T, 2, N>(a, m); break;
    case 3: op_rp<C, T, 3, N>(a, m); break;
    default: if constexpr (N > 16) op_rp<C, T, 4, N>(a, m); break;
  }
}

// dispatch on the dense op index (a jump table); positions beyond the
// stage's 2^G amplitudes never occur
template <typename C, typename T, int N>
__device__ __forceinline__ void apply_op(uint32_t code, const T (&m)[8], C (&a)[N]) {
  switch (code) {
#define QW_ONE(K, P, F) \
  case sv_op_index(K, P, 0): if constexpr ((1 << P) < N) F<C, T, P, N>(a, m); break;
#define QW_ALL(K, F) QW_ONE(K, 0, F) QW_ONE(K, 1, F) QW_ONE(K, 2, F) QW_ONE(K, 3, F) QW_ONE(K, 4, F)
    QW_ALL(K_U1, op_u1)
    QW_ALL(K_D1, op_d1)
    QW_ALL(K_P1, op_p1)
    QW_ALL(K_R, op_r)
    QW_ALL(K_RX, op_rx)
    QW_ALL(K_RP, op_rp)
#undef QW_ALL
#undef QW_ONE
#define CD(x, y) \
  case sv_op_index(K_CD, x, y): if constexpr ((1 << y) < N) op_cd<C, T, x, y, N>(a, m); break;
    CD(0, 1) CD(0, 2) CD(0, 3) CD(0, 4) CD(1, 2) CD(1, 3) CD(1, 4) CD(2, 3) CD(2, 4) CD(3, 4)
#undef CD
    default: break;
  }
}

// step[t] for the bit that a Gray-code walk flips (t is a constant once
// the walk is unrolled; the selects never index a local array)
__device__ __forceinline__ uint32_t gray_pick(const uint32_t (&step)[6], int t) {
  return t == 0 ? step[0] : t == 1 ? step[1] : t == 2 ? step[2] : t == 3 ? step[3] : t == 4 ? step[4]
         : t == 5 ? step[5] : 0u;
}

// One stage group in compensated FP32: the N = 2^G amplitudes at byte
// offsets sbB ^ (XOR combinations of roff) are read with a zero remainder
// (SV_AR_COMP) or with their remainder from the plane at lo_off
// (SV_AR_REM), the stage's ops run in double-float, and the renormalized
// pair is written back (SV_AR_COMP keeps only the rounded value).
template <int AR, int G>
__device__ __forceinline__ void sv_stage_df(char *smw, uint32_t lo_off, uint32_t sbB, const uint32_t (&roff)[SV_G],
                                            const SvOpDesc<float> *__restrict__ ops,
                                            const float *__restrict__ ops_lo, uint32_t op_begin, uint32_t nops,
                                            uint32_t rp_mask, const float *__restrict__ ph, uint32_t ph_block) {
  constexpr int N = 1 << G;
  float2 h[N], l[N];
#pragma unroll
  for (int i = 0; i < N; i++) {
    const uint32_t off = sbB ^ ((i & 1) ? roff[0] : 0u) ^ ((i & 2) ? roff[1] : 0u) ^ ((i & 4) ? roff[2] : 0u) ^
                         ((i & 8) ? roff[3] : 0u) ^ ((G > 4 && (i & 16)) ? roff[4] : 0u);
    h[i] = *(const float2 *)(smw + off);
    if constexpr (AR == SV_AR_REM) l[i] = *(const float2 *)(smw + lo_off + off);
    else l[i] = make_float2(0.f, 0.f);
  }
  auto load_ml = [&](uint32_t o, float (&m)[8], float (&ml)[8]) {
    load_m(ops + o, m);
    const float4 u = __ldg((const float4 *)(ops_lo + 8 * (size_t)o));
    const float4 v = __ldg((const float4 *)(ops_lo + 8 * (size_t)o + 4));
    ml[0] = u.x; ml[1] = u.y; ml[2] = u.z; ml[3] = u.w;
    ml[4] = v.x; ml[5] = v.y; ml[6] = v.z; ml[7] = v.w;
  };
  if (G == 4 && rp_mask == 0xFu) {
    // a rotation-and-phase op on every position: the four rotations, then
    // the stage's combined diagonal (amplitude e times the product of the
    // phases of its set positions, from the host's table) when there is one
    const bool table = ph != nullptr && ph_block != 0xFFFFFFFFu;
    float m[8], ml[8];
    load_ml(op_begin, m, ml);
    dfop_rp<0, N, AR == SV_AR_COMP>(h, l, m, ml, !table);
    load_ml(op_begin + 1, m, ml);
    dfop_rp<1, N>(h, l, m, ml, !table);
    load_ml(op_begin + 2, m, ml);
    dfop_rp<2, N>(h, l, m, ml, !table);
    load_ml(op_begin + 3, m, ml);
    dfop_rp<3, N>(h, l, m, ml, !table);
    if (table) {
      const float4 *q = (const float4 *)ph + 16 * (size_t)(ph_block & 0x7FFFFFFFu);
      if (ph_block >> 31) {  // the program's global phase: entry 0 too
        const float4 w = __ldg(q);
        df_cmul(w.x, w.y, w.z, w.w, h[0], l[0]);
      }
#pragma unroll
      for (int e = 1; e < N; e++) {
        const float4 w = __ldg(q + e);
        df_cmul(w.x, w.y, w.z, w.w, h[e], l[e]);
      }
    }
  } else if (rp_mask) {
    uint32_t o = op_begin;
#pragma unroll
    for (int P = 0; P < G; P++) {
      if (!(rp_mask & (1u << P))) continue;
      float m[8], ml[8];
      load_ml(o, m, ml);
      o++;
      df_rp_at<N>(P, h, l, m, ml);
    }
  } else {
    for (uint32_t o = 0; o < nops; o++) {
      float m[8], ml[8];
      load_ml(op_begin + o, m, ml);
      df_apply_op<N>(__ldg(&ops[op_begin + o].code), m, ml, h, l);
    }
  }
#pragma unroll
  for (int i = 0; i < N; i++) {
    df_renorm(h[i], l[i]);
    const uint32_t off = sbB ^ ((i & 1) ? roff[0] : 0u) ^ ((i & 2) ? roff[1] : 0u) ^ ((i & 4) ? roff[2] : 0u) ^
                         ((i & 8) ? roff[3] : 0u) ^ ((G > 4 && (i & 16)) ? roff[4] : 0u);
    *(float2 *)(smw + off) = h[i];
    if constexpr (AR == SV_AR_REM) *(float2 *)(smw + lo_off + off) = l[i];
  }
}

// Processes one tile of one pass.  src == nullptr starts from |0...0>.
// AR selects the arithmetic of FP32 passes: SV_AR_PLAIN, SV_AR_COMP
// (double-float registers, rounded to FP32 when a stage writes its
// amplitudes back) or SV_AR_REM (double-float kept through the whole pass
// in a second shared-memory plane, and between passes in the remainder
// arrays src_lo / dst_lo, either of which may be NULL: zero remainder on
// load, none stored).  FP64 passes are plain.
template <typename T, int AR, int G>
__device__ void sv_tile(const SvPassDesc *__restrict__ pd, const SvStageDesc *__restrict__ stages,
                        const SvOpDesc<T> *__restrict__ ops, const float *__restrict__ ops_lo,
                        const float *__restrict__ ph,
                        typename V2<T>::t *sm, const typename V2<T>::t *src, typename V2<T>::t *dst,
                        const float2 *src_lo, float2 *dst_lo, uint32_t tile) {
  typedef typename V2<T>::t C;
  static_assert(AR == SV_AR_PLAIN || sizeof(T) == 4, "compensated arithmetic is for FP32 states");
  static_assert(AR == SV_AR_PLAIN ? (G == SV_G || G == SV_G_PLAIN32) : G == SV_G_COMP, "stage width");
  const uint32_t k = pd->k, b = pd->b, n_hi = pd->n_hi;
  uint32_t base = 0;
  for (uint32_t i = 0; i < n_hi; i++) base |= ((tile >> i) & 1u) << pd->hi_pos[i];
  const uint32_t ntile = 1u << k, lomask = (1u << b) - 1u;
  const uint32_t nt = blockDim.x;

  // 16-byte units: two FP32 amplitudes or one FP64 amplitude
  constexpr uint32_t APU = (sizeof(T) == 4) ? 2u : 1u;
  const uint32_t n_units = ntile / APU;
  // A 16-byte unit's global index (bit deposit) and slot (swizzle, tile
  // map) are linear over GF(2) in the unit index, and a thread's units are
  // u = tid + j nt: each thread starts from its own unit and walks j in
  // Gray-code order, one XOR per address and unit (the table lookups stay
  // outside the loops).
  const uint32_t apu_bits = (APU == 2) ? 1u : 0u;
  const uint32_t lg_nt = (uint32_t)__ffs((int)nt) - 1u;
  const uint32_t n_iter = n_units > nt ? n_units >> lg_nt : (threadIdx.x < n_units ? 1u : 0u);
  auto gdep = [&](uint32_t l) {
    const uint32_t lh = l >> b;
    return __ldg(&pd->lo_tab[lh & 63]) | __ldg(&pd->hi_tab[(lh >> 6) & 31]) | (l & lomask);
  };
  uint32_t gstep[6], sstep[6];
#pragma unroll
  for (int t = 0; t < 6; t++) {
    const uint32_t lb = lg_nt + apu_bits + (uint32_t)t;
    gstep[t] = lb < k ? gdep(1u << lb) : 0u;
    sstep[t] = lb < k ? swz<T>(1u << lb) * (uint32_t)sizeof(C) : 0u;
  }
  const uint32_t l0 = threadIdx.x * APU;
  const char *smc = (const char *)sm;
  char *smw = (char *)sm;
  // SV_AR_REM: the remainder plane follows the tile, same slot layout
  const uint32_t lo_off = ntile * (uint32_t)sizeof(C);
  if (src) {
    uint32_t g = base | gdep(l0), so = swz<T>(l0) * (uint32_t)sizeof(C);
#pragma unroll
    for (int j = 0; j < 64; j++) {
      if ((uint32_t)j >= n_iter) break;
      cp_async16(smw + so, src + g);
      if constexpr (AR == SV_AR_REM) {
        if (src_lo) cp_async16(smw + lo_off + so, src_lo + g);
        else *(float4 *)(smw + lo_off + so) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const int t = __ffs(j + 1) - 1;
      g ^= gray_pick(gstep, t);
      so ^= gray_pick(sstep, t);
    }
    cp_async_wait_all();
  } else {
    for (uint32_t l = threadIdx.x; l < ntile; l += nt) {
      const uint32_t g = base | gdep(l);
      C v;
      v.x = (g == 0) ? T(1) : T(0);
      v.y = T(0);
      sm[swz<T>(l)] = v;
      if constexpr (AR == SV_AR_REM) *(float2 *)(smw + lo_off + swz<T>(l) * (uint32_t)sizeof(C)) = make_float2(0.f, 0.f);
    }
  }
  __syncthreads();

  // Stages.  The amplitude of logical tile index l sits in the slot of
  // phi(l) (an affine map the host tracks through the pass's permutation
  // gates), so a stage group's 32 slots are its base offset XOR combinations
  // of the five register-bit offsets, and the stage writes its registers
  // back to the slots it read.
  const uint32_t n_groups = 1u << (k - G);
  const uint32_t n_st = pd->n_stages, st0 = pd->stage_begin;
  for (uint32_t s = 0; s < n_st; s++) {
    const uint4 *sdv = (const uint4 *)(stages + st0 + s);
    const uint4 w0 = __ldg(sdv), w1 = __ldg(sdv + 1), w2 = __ldg(sdv + 2), w3 = __ldg(sdv + 3),
                w4 = __ldg(sdv + 4), w5 = __ldg(sdv + 5), w6 = __ldg(sdv + 6);
    // offsets are masked to the tile, so XOR combinations stay inside it
    const uint32_t tm = ntile * (uint32_t)sizeof(C) - 1u;
    const uint32_t roff[SV_G] = {w0.x & tm, w0.y & tm, w0.z & tm, w0.w & tm, w1.x & tm};
    const uint32_t gcol[SV_MAX_GBITS] = {w1.y & tm, w1.z & tm, w1.w & tm, w2.x & tm, w2.y & tm,
                                         w2.z & tm, w2.w & tm, w3.x & tm, w3.y & tm};
    // the map's constant, with the per-tile terms of outside-control CNOTs
    const uint32_t cst = (w3.z ^ (((tile >> w5.x) & 1u) ? w6.x : 0u) ^ (((tile >> w5.y) & 1u) ? w6.y : 0u) ^
                          (((tile >> w5.z) & 1u) ? w6.z : 0u) ^ (((tile >> w5.w) & 1u) ? w6.w : 0u)) & tm;
    const uint32_t nops = w3.w, op_begin = w4.x, rp_mask = w4.y, ph_block = w4.z;
    static_assert(SV_MAX_GBITS == 9 && SV_MAX_OUT_CTL == 4 && sizeof(SvStageDesc) == 112,
                  "stage descriptor read as seven 16-byte words");
    for (uint32_t grp = threadIdx.x; grp < n_groups; grp += nt) {
      uint32_t sbB = cst;
#pragma unroll
      for (int t = 0; t < SV_MAX_GBITS; t++) sbB ^= ((grp >> t) & 1u) ? gcol[t] : 0u;
      if constexpr (AR != SV_AR_PLAIN) {
        sv_stage_df<AR, G>(smw, lo_off, sbB, roff, ops, ops_lo, op_begin, nops, rp_mask, ph, ph_block);
      } else {
      constexpr int N = 1 << G;
      C a[N];
#pragma unroll
      for (int i = 0; i < N; i++) {
        const uint32_t off = sbB ^ ((i & 1) ? roff[0] : 0u) ^ ((i & 2) ? roff[1] : 0u) ^
                             ((i & 4) ? roff[2] : 0u) ^ ((i & 8) ? roff[3] : 0u) ^
                             ((G > 4 && (i & 16)) ? roff[4] : 0u);
        a[i] = *(const C *)(smc + off);
      }
      if (rp_mask) {
        // rotation-and-phase ops on distinct positions, in position order
        const SvOpDesc<T> *op = ops + op_begin;
#pragma unroll
        for (int P = 0; P < G; P++) {
          if (!(rp_mask & (1u << P))) continue;
          T m[8];
          load_m(op, m);
          op++;
          rp_at<C, T, N>(P, a, m);
        }
      } else {
        // the next op's parameters are loaded while the current op runs
        const SvOpDesc<T> *op = ops + op_begin;
        uint32_t code = 0;
        T m[8];
        if (nops) { code = __ldg(&op->code); load_m(op, m); }
        for (uint32_t o = 0; o < nops; o++) {
          uint32_t ncode = 0;
          T nm[8];
          if (o + 1 < nops) { ncode = __ldg(&op[o + 1].code); load_m(op + o + 1, nm); }
          apply_op<C, T, N>(code, m, a);
          code = ncode;
#pragma unroll
          for (int t = 0; t < 8; t++) m[t] = nm[t];
        }
      }
#pragma unroll
      for (int i = 0; i < N; i++) {
        const uint32_t off = sbB ^ ((i & 1) ? roff[0] : 0u) ^ ((i & 2) ? roff[1] : 0u) ^
                             ((i & 4) ? roff[2] : 0u) ^ ((i & 8) ? roff[3] : 0u) ^
                             ((G > 4 && (i & 16)) ? roff[4] : 0u);
        *(C *)(smw + off) = a[i];
      }
      }
    }
    __syncthreads();
  }

  const uint32_t tm = ntile * (uint32_t)sizeof(C) - 1u;
  uint32_t g = base | gdep(l0);
  if (pd->phi_ident) {
    uint32_t so = swz<T>(l0) * (uint32_t)sizeof(C);
#pragma unroll
    for (int j = 0; j < 64; j++) {
      if ((uint32_t)j >= n_iter) break;
      *(float4 *)(dst + g) = *(const float4 *)(smc + so);
      if constexpr (AR == SV_AR_REM) {
        if (dst_lo) *(float4 *)(dst_lo + g) = *(const float4 *)(smc + lo_off + so);
      }
      const int t = __ffs(j + 1) - 1;
      g ^= gray_pick(gstep, t);
      so ^= gray_pick(sstep, t);
    }
  } else {
    // slots through the final tile map: the slot of unit u is
    // st_lo[u & 63] ^ st_hi[u >> 6] (constant folded into st_lo)
    auto st_of = [&](uint32_t u) { return __ldg(&pd->st_lo[u & 63]) ^ __ldg(&pd->st_hi[(u >> 6) & 127]); };
    const uint32_t c0 = __ldg(&pd->st_lo[0]);
#pragma unroll
    for (int t = 0; t < 6; t++) {
      const uint32_t ub = lg_nt + (uint32_t)t;
      sstep[t] = (ub + apu_bits < k) ? (st_of(1u << ub) ^ c0) & tm : 0u;
    }
    uint32_t so = st_of(threadIdx.x);
#pragma unroll
    for (int c = 0; c < SV_MAX_OUT_CTL; c++)
      so ^= ((tile >> pd->ctl_tb[c]) & 1u) ? pd->ctl_w[c] : 0u;
    so &= tm;
    if (pd->phi_unit16) {
      // each unit still sits in one 16-byte slot pair, at a permuted place
#pragma unroll
      for (int j = 0; j < 64; j++) {
        if ((uint32_t)j >= n_iter) break;
        *(float4 *)(dst + g) = *(const float4 *)(smc + (so & ~15u));
        if constexpr (AR == SV_AR_REM) {
          if (dst_lo) *(float4 *)(dst_lo + g) = *(const float4 *)(smc + lo_off + (so & ~15u));
        }
        const int t = __ffs(j + 1) - 1;
        g ^= gray_pick(gstep, t);
        so ^= gray_pick(sstep, t);
      }
    } else {
      // each unit's two amplitudes gathered from their slots
      const uint32_t pair = pd->phi_pair & tm;
#pragma unroll
      for (int j = 0; j < 64; j++) {
        if ((uint32_t)j >= n_iter) break;
        if constexpr (sizeof(T) == 4) {
          const float2 a0 = *(const float2 *)(smc + so), a1 = *(const float2 *)(smc + (so ^ pair));
          *(float4 *)(dst + g) = make_float4(a0.x, a0.y, a1.x, a1.y);
          if constexpr (AR == SV_AR_REM) {
            if (dst_lo) {
              const float2 r0 = *(const float2 *)(smc + lo_off + so), r1 = *(const float2 *)(smc + lo_off + (so ^ pair));
              *(float4 *)(dst_lo + g) = make_float4(r0.x, r0.y, r1.x, r1.y);
            }
          }
        } else {
          *(double2 *)(dst + g) = *(const double2 *)(smc + so);
        }
        const int t = __ffs(j + 1) - 1;
        g ^= gray_pick(gstep, t);
        so ^= gray_pick(sstep, t);
      }
    }
  }
}

// NT threads at most (the launch uses sv_threads_for_k), MINB CTAs per SM
// for the register budget.
template <typename T, int AR, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
sv_pass_kernel(SvTables t, uint32_t pass, const typename V2<T>::t *src, typename V2<T>::t *dst,
               const float2 *src_lo, float2 *dst_lo) {
  extern __shared__ __align__(16) unsigned char smraw[];
  typedef typename V2<T>::t C;
  sv_tile<T, AR, sv_stage_width(AR, sizeof(T) == 8)>(t.passes + pass, t.stages, (const SvOpDesc<T> *)t.ops, t.ops_lo,
                                                     t.ph, (C *)smraw, src, dst, src_lo, dst_lo, blockIdx.x);
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const unsigned int *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s per dependency wait

// Persistent launch over an ordered work list: a CTA takes the next item,
// maps it through the segment table to (job, unit), waits (bounded) until
// the job's dependency has completed every unit, runs the unit (one tile of
// a pass, or one energy block of a finished state) and counts it done.
// Items are taken in list order and every dependency lies wholly before its
// dependent, so the oldest unfinished item never waits and the launch always
// drains.
// MINB: CTAs per SM the registers are budgeted for.  Tiles of 2^13 FP32
// amplitudes (64 KB) fit three CTAs per SM; smaller tiles fit four, which
// the 128-register build (MINB 4) can use.  Compensated passes (AR =
// SV_AR_COMP) hold two FP32 complex values per amplitude in registers, 16
// amplitudes per stage group, and are budgeted for three CTAs.
template <typename T, int MINB, int AR, int NT>
__global__ void __launch_bounds__(NT, MINB)
sv_batch_kernel(SvTables t, const SvJob *__restrict__ jobs, const SvSeg *__restrict__ segs,
                uint32_t seg_bits, uint32_t total, unsigned int *ctr, EnTables en) {
  extern __shared__ __align__(16) unsigned char smraw[];
  typedef typename V2<T>::t C;
  __shared__ uint32_t s_job, s_unit;
  __shared__ int s_state;  // 0 run, 1 empty item, 2 stop
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t it = atomicAdd(&ctr[0], 1u);
      int st = 0;
      if (it >= total) {
        st = 2;
      } else {
        const SvSeg sg = segs[it >> seg_bits];
        const uint32_t unit = sg.first + (it & ((1u << seg_bits) - 1u));
        s_job = sg.job;
        s_unit = unit;
        if (unit >= jobs[sg.job].n_tiles) {
          st = 1;
        } else {
          const int dep = jobs[sg.job].dep;
          if (dep >= 0) {
            const uint32_t need = jobs[dep].n_tiles;
            const uint64_t t0 = globaltimer_ns();
            while (ld_acquire_u32(&ctr[2 + dep]) < need) {
              if (ld_acquire_u32(&ctr[1]) != 0u) { st = 2; break; }
              if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) {
                atomicExch(&ctr[1], 1u);  // reported to the host as a device timeout
                st = 2;
                break;
              }
              __nanosleep(100);
            }
          }
        }
      }
      s_state = st;
    }
    __syncthreads();
    const int st = s_state;
    if (st == 2) break;
    if (st == 1) {
      __syncthreads();  // s_state is rewritten only after every thread read it
      continue;
    }
    const SvJob job = jobs[s_job];
    if (job.kind == SVJ_ENERGY) {
      if constexpr (NT == 128) {  // energy work items run in 128-thread CTAs only
        const EnJob J = en.jobs[job.pass];
        energy_block<T, 128, false>(J, s_unit, en.classes, en.terms,
                                    en.partials + 2 * (size_t)(J.block_begin + s_unit));
      }
    } else {
      sv_tile<T, AR, sv_stage_width(AR, sizeof(T) == 8)>(t.passes + job.pass, t.stages, (const SvOpDesc<T> *)t.ops,
                                                         t.ops_lo, t.ph, (C *)smraw, (const C *)job.src,
                                                         (C *)job.dst, nullptr, nullptr, s_unit);
    }
    // every thread's writes of the unit precede thread 0's release through
    // the barrier (bar.sync orders them at CTA scope; the fence is
    // cumulative), so one fence per unit suffices
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&ctr[2 + s_job], 1u);
    }
  }
}

// ---- host launchers -----------------------------------------------------------
// Compensated passes (two FP32 values per amplitude) run stages of four
// positions, 16 amplitudes per group; plain passes stages of SV_G_PLAIN32
// (FP32) or five (FP64) positions.  Threads: every thread owns at least two
// stage groups of a 2^13 tile (128 threads; 256 for plain FP32 passes with
// four-position stages, whose register budget fits three such CTAs per
// SM); passes with a remainder plane (twice the shared memory, one CTA per
// SM) give every stage group its own thread, up to 256.
constexpr int SV_NT_PLAIN32 = (SV_G_PLAIN32 == 4) ? 256 : 128;
int sv_threads_for_k(uint32_t k, int ar, bool fp64) {
  const uint32_t G = (uint32_t)sv_stage_width(ar, fp64);
  const uint32_t g = (ar == SV_AR_REM) ? 1u << (k - G) : 1u << (k - G - 1);
  const uint32_t cap = (ar == SV_AR_REM) ? 256u : (!fp64 && ar == SV_AR_PLAIN) ? (uint32_t)SV_NT_PLAIN32 : 128u;
  return (int)(g < 32 ? 32 : (g > cap ? cap : g));
}
size_t sv_smem_bytes(bool fp64, uint32_t k, int ar) {
  return (size_t)(fp64 ? 16 : 8) << k << (ar == SV_AR_REM ? 1 : 0);
}

// the plain FP32 batch kernel for tiles of k qubits: with 32-amplitude
// stages a 128-register build (four CTAs per SM) serves tiles of at most 12
// qubits; 16-amplitude stages use one build
typedef void (*SvBatchKernel)(SvTables, const SvJob *, const SvSeg *, uint32_t, uint32_t, unsigned int *, EnTables);
static SvBatchKernel plain32_batch(uint32_t k) {
  if constexpr (SV_G_PLAIN32 == 4) {
    (void)k;
    return sv_batch_kernel<float, 3, SV_AR_PLAIN, SV_NT_PLAIN32>;
  } else {
    return k > 12 ? sv_batch_kernel<float, 3, SV_AR_PLAIN, SV_NT_PLAIN32>
                  : sv_batch_kernel<float, 4, SV_AR_PLAIN, SV_NT_PLAIN32>;
  }
}

// Kernel attributes are set once, before any stream capture (a capture
// fails on attribute changes).
cudaError_t sv_init_attrs() {
  const int bytes = 200 * 1024;
  const void *k[] = {(const void *)sv_pass_kernel<float, SV_AR_PLAIN, SV_NT_PLAIN32, 3>,
                     (const void *)sv_pass_kernel<float, SV_AR_COMP, 128, 3>,
                     (const void *)sv_pass_kernel<float, SV_AR_REM, 256, 1>,
                     (const void *)sv_pass_kernel<double, SV_AR_PLAIN, 128, 1>,
                     (const void *)plain32_batch(13),
                     (const void *)plain32_batch(12),
                     (const void *)sv_batch_kernel<float, 3, SV_AR_COMP, 128>,
                     (const void *)sv_batch_kernel<double, 1, SV_AR_PLAIN, 128>};
  for (const void *f : k) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void launch_sv_pass(bool fp64, const SvTables &t, uint32_t pass_idx, uint32_t k, uint32_t n, const void *src,
                    void *dst, void *stream, int ar, const void *src_lo, void *dst_lo) {
  const uint32_t tiles = 1u << (n - k);
  if (fp64) ar = SV_AR_PLAIN;
  const int threads = sv_threads_for_k(k, ar, fp64);
  const size_t smem = sv_smem_bytes(fp64, k, ar);
  cudaStream_t s = (cudaStream_t)stream;
  const float2 *sl = (const float2 *)src_lo;
  float2 *dl = (float2 *)dst_lo;
  if (fp64) {
    sv_pass_kernel<double, SV_AR_PLAIN, 128, 1><<<tiles, threads, smem, s>>>(t, pass_idx, (const double2 *)src,
                                                                              (double2 *)dst, nullptr, nullptr);
  } else if (ar == SV_AR_REM) {
    sv_pass_kernel<float, SV_AR_REM, 256, 1><<<tiles, threads, smem, s>>>(t, pass_idx, (const float2 *)src,
                                                                           (float2 *)dst, sl, dl);
  } else if (ar == SV_AR_COMP) {
    sv_pass_kernel<float, SV_AR_COMP, 128, 3><<<tiles, threads, smem, s>>>(t, pass_idx, (const float2 *)src,
                                                                            (float2 *)dst, nullptr, nullptr);
  } else {
    sv_pass_kernel<float, SV_AR_PLAIN, SV_NT_PLAIN32, 3><<<tiles, threads, smem, s>>>(
        t, pass_idx, (const float2 *)src, (float2 *)dst, nullptr, nullptr);
  }
}

int sv_batch_grid(bool fp64, uint32_t k, int sm_count, int ar) {
  if (fp64 || ar == SV_AR_REM) ar = SV_AR_PLAIN;
  const int threads = sv_threads_for_k(k, ar, fp64);
  const size_t smem = sv_smem_bytes(fp64, k, ar);
  int per_sm = 0;
  if (fp64)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sv_batch_kernel<double, 1, SV_AR_PLAIN, 128>, threads,
                                                  smem);
  else if (ar == SV_AR_COMP)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sv_batch_kernel<float, 3, SV_AR_COMP, 128>, threads, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plain32_batch(k), threads, smem);
  if (per_sm < 1) per_sm = 1;
  return per_sm * sm_count;
}

void launch_sv_batch(bool fp64, const SvTables &t, const SvJob *jobs, const SvSeg *segs, uint32_t seg_bits,
                     uint32_t total_items, uint32_t k_max, unsigned int *counters, const EnTables &en,
                     int grid, void *stream, int ar) {
  if (fp64 || ar == SV_AR_REM) ar = SV_AR_PLAIN;
  const int threads = sv_threads_for_k(k_max, ar, fp64);
  const size_t smem = sv_smem_bytes(fp64, k_max, ar);
  cudaStream_t s = (cudaStream_t)stream;
  if (fp64)
    sv_batch_kernel<double, 1, SV_AR_PLAIN, 128><<<grid, threads, smem, s>>>(t, jobs, segs, seg_bits, total_items,
                                                                             counters, en);
  else if (ar == SV_AR_COMP)
    sv_batch_kernel<float, 3, SV_AR_COMP, 128><<<grid, threads, smem, s>>>(t, jobs, segs, seg_bits, total_items,
                                                                           counters, en);
  else
    plain32_batch(k_max)<<<grid, threads, smem, s>>>(t, jobs, segs, seg_bits, total_items, counters, en);
}

}  // namespace qw

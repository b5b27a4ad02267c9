// Pauli-sum energy over one block of amplitudes, shared by the stand-alone
// energy kernel (256 threads) and by the persistent suffix kernel, which
// runs energy blocks as a second kind of work item (128 threads, two
// sub-blocks per 4096-amplitude block).
//
// E = sum_k c_k <psi|P_k|psi> / <psi|psi>, P|x> = i^{#Y} (-1)^{popc(x&z)}|x^m>.
// For m != 0 the pair (x, x^m) is visited once from the side whose highest
// flipped bit is 0 and contributes 2 Re(i^{#Y} (-1)^{popc(x&z)}
// conj(psi[x^m]) psi[x]); the host folds 2, the sign of i^{#Y} and the
// coefficient into EnTerm::coef and the choice of real or imaginary part into
// EnTerm::flags.  Terms are grouped into classes by the flipped bits above an
// L2-sized chunk, so the blocks of one class read one pair of chunks.
//
// A sub-block holds 16 << TB amplitudes; element j of thread t has index
// x = base | j << TB | t.  The three fields are disjoint bit ranges, so for
// a term (m, z) the partner of element j is pb | (j ^ mj) << TB with pb the
// partner of element 0, and its sign is (-1)^{popc((base|t) & z)} times
// (-1)^{popc(j & zj)}.  The partner offsets are resolved at compile time by
// a switch over (mj, flags), so a partner load is one load with an immediate
// offset; the signs are applied by a branch-free butterfly.
#pragma once

#include <cuda_runtime.h>

#include "qw_internal.h"

namespace qw {

template <typename T> struct EnC;
template <> struct EnC<float> { typedef float2 t; };
template <> struct EnC<double> { typedef double2 t; };

struct DFAcc {  // double-float accumulator (two-sum of the high part)
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float p) {
    const float s = hi + p;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (p - bp);
    hi = s;
    lo += err;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
struct DAcc {
  double v = 0.0;
  __device__ __forceinline__ void add(double p) { v += p; }
  __device__ __forceinline__ double value() const { return v; }
};
template <typename T> struct AccOf;
template <> struct AccOf<float> { typedef DFAcc t; };
template <> struct AccOf<double> { typedef DAcc t; };

__device__ __forceinline__ double en_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// NC: the state is read-only for the whole launch (read-only cache path);
// otherwise it was written earlier in the same launch by other CTAs and is
// read from L2.
template <bool NC, typename C>
__device__ __forceinline__ C en_ld(const C *p) {
  if (NC) return __ldg(p);
  return __ldcg(p);
}

// sum_j (-1)^{popc(j & z)} v[j] as a butterfly over the four bits of j with
// runtime signs: 15 fused multiply-adds by +-1 (exact products), no branch
template <typename T>
__device__ __forceinline__ T en_signed16_bf(const T (&v)[16], uint32_t z) {
  const T s0 = (z & 1u) ? T(-1) : T(1), s1 = (z & 2u) ? T(-1) : T(1);
  const T s2 = (z & 4u) ? T(-1) : T(1), s3 = (z & 8u) ? T(-1) : T(1);
  T u[8], w[4];
#pragma unroll
  for (int k = 0; k < 8; k++) u[k] = fma(s0, v[2 * k + 1], v[2 * k]);
#pragma unroll
  for (int k = 0; k < 4; k++) w[k] = fma(s1, u[2 * k + 1], u[2 * k]);
  const T x0 = fma(s2, w[1], w[0]), x1 = fma(s2, w[3], w[2]);
  return fma(s3, x1, x0);
}

// v[j] = Re or Im part of conj(partner_j) a[j], partner_j = q[(j ^ MJ) << TB]
template <typename T, int TB, bool NC, int MJ, bool FL, typename C>
__device__ __forceinline__ void en_prod(const C *__restrict__ q, const C (&a)[16], T (&v)[16]) {
  C p[16];
#pragma unroll
  for (int j = 0; j < 16; j++) p[j] = en_ld<NC>(q + ((j ^ MJ) << TB));
#pragma unroll
  for (int j = 0; j < 16; j++)
    v[j] = FL ? (p[j].x * a[j].y - p[j].y * a[j].x) : (p[j].x * a[j].x + p[j].y * a[j].y);
}
template <typename T, int TB, bool NC, typename C>
__device__ __forceinline__ void en_prod_rt(const C *__restrict__ q, const C (&a)[16], T (&v)[16],
                                           uint32_t sel) {
  switch (sel & 31u) {
#define QW_PR(S) case S: en_prod<T, TB, NC, (S & 15), (S >= 16)>(q, a, v); break;
    QW_PR(0) QW_PR(1) QW_PR(2) QW_PR(3) QW_PR(4) QW_PR(5) QW_PR(6) QW_PR(7)
    QW_PR(8) QW_PR(9) QW_PR(10) QW_PR(11) QW_PR(12) QW_PR(13) QW_PR(14) QW_PR(15)
    QW_PR(16) QW_PR(17) QW_PR(18) QW_PR(19) QW_PR(20) QW_PR(21) QW_PR(22) QW_PR(23)
    QW_PR(24) QW_PR(25) QW_PR(26) QW_PR(27) QW_PR(28) QW_PR(29) QW_PR(30)
#undef QW_PR
    default: en_prod<T, TB, NC, 15, true>(q, a, v); break;
  }
}

// Accumulates the terms [t0, t1) over the sub-block at `base` (a multiple of
// 16 << TB) into acc, and the sub-block's squared norm into nrm.
template <typename T, int TB, bool NC>
__device__ __forceinline__ void energy_sub(const typename EnC<T>::t *__restrict__ psi, uint32_t dim,
                                           const EnTerm *__restrict__ terms, uint32_t t0, uint32_t t1,
                                           uint32_t base, typename AccOf<T>::t &acc, T &nrm) {
  typedef typename EnC<T>::t C;
  constexpr uint32_t JF = 15u << TB;  // the j-field of an index
  const uint32_t own = base | threadIdx.x;
  C a[16];
#pragma unroll
  for (int j = 0; j < 16; j++) {
    const uint32_t x = own | ((uint32_t)j << TB);
    if (x < dim) {
      a[j] = en_ld<NC>(psi + x);
    } else {
      a[j].x = 0;
      a[j].y = 0;
    }
    nrm += a[j].x * a[j].x + a[j].y * a[j].y;
  }
  const bool full = dim >= (16u << TB);
  for (uint32_t t = t0; t < t1; t++) {
    const uint2 w0 = __ldg((const uint2 *)&terms[t].xm);    // xm, zm
    const uint2 w1 = __ldg((const uint2 *)&terms[t].skip);  // skip, flags
    const T coef = (T)__ldg(&terms[t].coef);
    const uint32_t xm = w0.x, zm = w0.y, skip = w1.x, fl = w1.y;
    if (own & skip) continue;  // the pair is counted from its other member
    const uint32_t ks = (skip & JF) >> TB;
    const uint32_t mj = (xm & JF) >> TB, zj = (zm & JF) >> TB;
    const uint32_t pb = own ^ (xm & ~JF);
    const bool neg = __popc(own & zm) & 1;
    T s = 0;
    if (ks == 0 && full) {
      T v[16];
      en_prod_rt<T, TB, NC>(psi + pb, a, v, mj | (fl << 4));
      s = en_signed16_bf<T>(v, zj);
    } else {
      // a skipped bit inside the j-field, or a register smaller than the
      // sub-block: per-element tests
#pragma unroll
      for (int j = 0; j < 16; j++) {
        const uint32_t x = own | ((uint32_t)j << TB);
        if (((uint32_t)j & ks) || x >= dim) continue;
        const C p = en_ld<NC>(psi + (pb | (((uint32_t)j ^ mj) << TB)));
        const T v = fl ? (p.x * a[j].y - p.y * a[j].x) : (p.x * a[j].x + p.y * a[j].y);
        s += (__popc((uint32_t)j & zj) & 1) ? -v : v;
      }
    }
    acc.add(coef * (neg ? -s : s));
  }
}

// Block `jb` (2^EN_BLOCK_BITS amplitudes) of energy job J, computed by a CTA
// of THREADS threads in 4096 / (16 * THREADS) sub-blocks; thread 0 writes
// {sum_k c_k term_k, squared norm of the block} to out[0..1].
template <typename T, int THREADS, bool NC>
__device__ __forceinline__ void energy_block(const EnJob &J, uint32_t jb, const EnClass *__restrict__ classes,
                                             const EnTerm *__restrict__ terms, double *out) {
  constexpr int TB = (THREADS == 256) ? 8 : 7;
  constexpr int NSUB = (1 << EN_BLOCK_BITS) / (16 * THREADS);
  static_assert((16 << TB) * NSUB == (1 << EN_BLOCK_BITS) && (1 << TB) == THREADS, "block shape");
  uint32_t c = J.class_begin;
  const uint32_t ce = J.class_begin + J.n_classes;
  while (c + 1 < ce && classes[c + 1].block_begin <= jb) c++;
  const EnClass K = classes[c];
  const uint32_t within = jb - K.block_begin;
  const uint32_t bpc_bits = (J.chunk_bits > (uint32_t)EN_BLOCK_BITS) ? J.chunk_bits - EN_BLOCK_BITS : 0u;
  const uint32_t ownc = within >> bpc_bits;
  const uint32_t bic = within & ((1u << bpc_bits) - 1u);
  uint32_t chunk = ownc;
  if (K.hb != 0xFFFFFFFFu) {  // own chunks are those with bit hb clear
    const uint32_t p = K.hb - J.chunk_bits;
    chunk = ((ownc >> p) << (p + 1)) | (ownc & ((1u << p) - 1u));
  }
  const uint32_t dim = 1u << J.n;
  const uint32_t base = (chunk << J.chunk_bits) + (bic << EN_BLOCK_BITS);
  typedef typename EnC<T>::t C;
  const C *psi = (const C *)J.state;
  typename AccOf<T>::t acc;
  T nrm = 0;
#pragma unroll 1
  for (int sb = 0; sb < NSUB; sb++)
    energy_sub<T, TB, NC>(psi, dim, terms, K.term_begin, K.term_end, base + ((uint32_t)sb << (TB + 4)), acc,
                          nrm);
  double e = acc.value();
  double nn = (K.hb == 0xFFFFFFFFu) ? (double)nrm : 0.0;
  __shared__ double en_red[2][THREADS / 32];
  e = en_warp_sum(e);
  nn = en_warp_sum(nn);
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  if (ln == 0) { en_red[0][w] = e; en_red[1][w] = nn; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double se = 0, sn = 0;
    for (int i = 0; i < THREADS / 32; i++) { se += en_red[0][i]; sn += en_red[1][i]; }
    out[0] = se;
    out[1] = sn;
  }
  __syncthreads();
}

}  // namespace qw

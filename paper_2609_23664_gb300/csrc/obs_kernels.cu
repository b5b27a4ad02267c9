// Observables: Pauli-sum energy and computational-basis sampling (sm_103a).
//
// Energy (the repeated expectation evaluation of the VQE workloads, Sec. V,
// Table III): E = sum_k c_k <psi|P_k|psi> / <psi|psi> with
// P|x> = i^{#Y} (-1)^{popc(x&z)} |x^m>.  For m != 0 the pair (x, x^m) is
// visited once from the side whose highest flipped bit is 0, contributing
// 2 Re(i^{#Y} (-1)^{popc(x&z)} conj(psi[x^m]) psi[x]).  Terms are grouped by
// the flipped bits above an L2-sized chunk, so that all terms of a class touch
// only one pair of chunks and the pair stays L2-resident while the class runs.
// Products are FP32; every thread keeps a double-float (two-sum) accumulator
// across terms, and block and final reductions are FP64, in a fixed order.
//
// Sampling: p_x = |psi_x|^2 summed in FP64 into a CDF that is never written
// out: per 4096-amplitude block a lane sums 128 contiguous probabilities and
// the 32 lane sums are chained in lane order; block offsets are chained in
// block order; a shot finds its block by binary search and its index by
// rescanning that block in the same order, so the CDF it searches is
// exactly the one whose block totals were chained.
#include <cuda_runtime.h>

#include <algorithm>

#include "energy_block.cuh"
#include "qw_internal.h"

namespace qw {

template <typename T> struct V2o;
template <> struct V2o<float> { typedef float2 t; };
template <> struct V2o<double> { typedef double2 t; };

// ---------------------------------------------------------------------------
// energy layout (host)
// ---------------------------------------------------------------------------
void build_energy_layout(const qw_pauli_term *terms, uint64_t n_terms, uint32_t n, uint32_t amp_bytes,
                         uint32_t *chunk_bits_out, std::vector<EnClass> &classes,
                         std::vector<EnTerm> &en_terms, uint32_t *n_blocks) {
  // chunks of at most EN_CHUNK_BYTES, so that the chunk pair a class reads
  // stays in L2 (a quarter of the state as the chunk measured fastest for
  // 24 FP32 qubits on GB300: 186 ms against 202 ms with an eighth, 188 ms
  // with a half, 247 ms with a sixteenth), and no smaller than a block
  uint32_t chunk_bits = n;
  while (chunk_bits > (uint32_t)EN_BLOCK_BITS && ((uint64_t)amp_bytes << chunk_bits) > EN_CHUNK_BYTES) chunk_bits--;
  const uint32_t u = n - chunk_bits;
  const uint32_t bpc = (chunk_bits >= (uint32_t)EN_BLOCK_BITS) ? (1u << (chunk_bits - EN_BLOCK_BITS)) : 1u;
  std::vector<std::vector<EnTerm>> by_class(1u << u);
  for (uint64_t k = 0; k < n_terms; k++) {
    const uint64_t m = terms[k].xmask, z = terms[k].zmask;
    const int y = __builtin_popcountll(m & z);
    const double sgn = ((y & 3) == 0 || (y & 3) == 3) ? 1.0 : -1.0;
    EnTerm t{};
    t.xm = (uint32_t)m;
    t.zm = (uint32_t)z;
    t.flags = (uint32_t)(y & 1);
    t.coef = terms[k].coef * sgn * (m ? 2.0 : 1.0);
    const uint32_t d = (uint32_t)(m >> chunk_bits);
    t.skip = (d == 0 && m != 0) ? (1u << (63 - __builtin_clzll(m))) : 0u;
    by_class[d].push_back(t);
  }
  classes.clear();
  en_terms.clear();
  uint32_t blk = 0;
  for (uint32_t d = 0; d < (1u << u); d++) {
    if (d != 0 && by_class[d].empty()) continue;
    EnClass c{};
    c.term_begin = (uint32_t)en_terms.size();
    en_terms.insert(en_terms.end(), by_class[d].begin(), by_class[d].end());
    c.term_end = (uint32_t)en_terms.size();
    c.hb = (d == 0) ? 0xFFFFFFFFu : (chunk_bits + 31 - __builtin_clz(d));
    c.n_own = (d == 0) ? (1u << u) : (1u << (u - 1));
    c.block_begin = blk;
    blk += c.n_own * bpc;
    classes.push_back(c);
  }
  *chunk_bits_out = chunk_bits;
  *n_blocks = blk;
}

// ---------------------------------------------------------------------------
// energy kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum_d(double v) { return en_warp_sum(v); }

// one CTA per 4096-amplitude block; the block's job is found by binary search.
// Four CTAs per SM (64 registers for FP32): the kernel is bound by the
// latency and bandwidth of its L2 partner reads, so resident warps matter
// more than registers.
template <typename T>
__global__ void __launch_bounds__(EN_THREADS, 4)
energy_kernel(const EnJob *__restrict__ jobs, uint32_t n_jobs, const EnClass *__restrict__ classes,
              const EnTerm *__restrict__ terms, double *partials) {
  const uint32_t gb = blockIdx.x;
  uint32_t lo = 0, hi = n_jobs;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (jobs[mid].block_begin <= gb) lo = mid; else hi = mid;
  }
  const EnJob J = jobs[lo];
  energy_block<T, EN_THREADS, true>(J, gb - J.block_begin, classes, terms, partials + 2 * (size_t)gb);
}

// one warp per job; fixed summation order
__global__ void energy_reduce_kernel(const EnJob *__restrict__ jobs, uint32_t n_jobs,
                                     const double *__restrict__ partials) {
  const uint32_t j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int ln = threadIdx.x & 31;
  if (j >= n_jobs) return;
  const EnJob J = jobs[j];
  double se = 0, sn = 0;
  for (uint32_t i = ln; i < J.n_blocks; i += 32) {
    se += partials[2 * (size_t)(J.block_begin + i)];
    sn += partials[2 * (size_t)(J.block_begin + i) + 1];
  }
  se = warp_sum_d(se);
  sn = warp_sum_d(sn);
  if (ln == 0) {
    J.out[0] = se / sn;
    J.out[1] = sn;
  }
}

void launch_energy_reduce(const EnJob *jobs, uint32_t n_jobs, const double *partials, void *stream) {
  if (n_jobs == 0) return;
  const int warps = 4;
  energy_reduce_kernel<<<(n_jobs + warps - 1) / warps, warps * 32, 0, (cudaStream_t)stream>>>(jobs, n_jobs,
                                                                                           partials);
}

void launch_energy(bool fp64, const EnJob *jobs, uint32_t n_jobs, uint32_t total_blocks,
                   const EnClass *classes, const EnTerm *terms, double *partials, void *stream) {
  if (n_jobs == 0 || total_blocks == 0) return;
  cudaStream_t s = (cudaStream_t)stream;
  if (fp64)
    energy_kernel<double><<<total_blocks, EN_THREADS, 0, s>>>(jobs, n_jobs, classes, terms, partials);
  else
    energy_kernel<float><<<total_blocks, EN_THREADS, 0, s>>>(jobs, n_jobs, classes, terms, partials);
  launch_energy_reduce(jobs, n_jobs, partials, stream);
}

// ---------------------------------------------------------------------------
// sampling kernels
// ---------------------------------------------------------------------------
constexpr int SMP_PER_LANE = (1 << SMP_BLOCK_BITS) / 32;  // 128


__device__ __forceinline__ uint32_t find_source(const SmpSource *srcs, uint32_t n_src, uint32_t gb) {
  uint32_t lo = 0, hi = n_src;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (srcs[mid].block_begin <= gb) lo = mid; else hi = mid;
  }
  return lo;
}

// Running sum of one lane's probabilities in index order.  FP64 states add
// in FP64; FP32 states add their FP32 probabilities in double-float (a
// two-sum of the high part, about 2^-44 relative, FP32 arithmetic at 64
// times GB300's FP64 rate) and hand the sum on in FP64.  The lane sums and
// the element scan of the shot kernel make the same additions in the same
// order, so their partial sums agree bit for bit.
template <typename T> struct SmpAcc;
template <> struct SmpAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double p) { v += p; }
  __device__ __forceinline__ double value() const { return v; }
};
template <> struct SmpAcc<float> {
  DFAcc a;
  __device__ __forceinline__ void add(float p) { a.add(p); }
  __device__ __forceinline__ double value() const { return a.value(); }
};
__device__ __forceinline__ float prob32(const float2 &v) { return fmaf(v.x, v.x, v.y * v.y); }
__device__ __forceinline__ double prob32(const double2 &v) { return fma(v.x, v.x, v.y * v.y); }

// lane-serial sum of the lane's 128 probabilities, lane sums chained in order
template <typename T>
__device__ void lane_sums(const typename V2o<T>::t *psi, uint32_t dim, uint32_t off, int ln,
                          double *lane_sum, int32_t *lane_last) {
  SmpAcc<T> s;
  int32_t last = -1;
  const uint32_t b0 = off + (uint32_t)ln * SMP_PER_LANE;
  if constexpr (sizeof(T) == 4) {
    if (b0 + SMP_PER_LANE <= dim) {  // FP32, whole segment: two amplitudes per 16-byte load
      const float4 *q = reinterpret_cast<const float4 *>(psi + b0);
#pragma unroll 8
      for (int i = 0; i < SMP_PER_LANE / 2; i++) {
        const float4 v = q[i];
        const float p0 = fmaf(v.x, v.x, v.y * v.y), p1 = fmaf(v.z, v.z, v.w * v.w);
        s.add(p0);
        if (p0 > 0) last = ln * SMP_PER_LANE + 2 * i;
        s.add(p1);
        if (p1 > 0) last = ln * SMP_PER_LANE + 2 * i + 1;
      }
      *lane_sum = s.value();
      *lane_last = last;
      return;
    }
  }
  for (int i = 0; i < SMP_PER_LANE; i++) {
    const uint32_t x = b0 + i;
    if (x < dim) {
      const auto p = prob32(psi[x]);
      s.add(p);
      if (p > 0) last = ln * SMP_PER_LANE + i;
    }
  }
  *lane_sum = s.value();
  *lane_last = last;
}

// chained (sequential in lane order) inclusive scan: S_l = S_{l-1} + s_l
__device__ __forceinline__ double chain_scan(double s, int ln) {
  double S = (ln == 0) ? s : 0.0;
  for (int l = 1; l < 32; l++) {
    const double prev = __shfl_sync(0xffffffffu, S, l - 1);
    if (ln == l) S = prev + s;
  }
  return S;
}

template <typename T>
__global__ void smp_blocksum_kernel(const SmpSource *__restrict__ srcs, uint32_t n_src,
                                    uint32_t total, double *bsum, int32_t *blast) {
  typedef typename V2o<T>::t C;
  const uint32_t gb = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int ln = threadIdx.x & 31;
  if (gb >= total) return;
  const SmpSource S = srcs[find_source(srcs, n_src, gb)];
  const uint32_t blk = gb - S.block_begin;
  const uint32_t dim = 1u << S.n;
  double s;
  int32_t last;
  lane_sums<T>((const C *)S.state, dim, blk << SMP_BLOCK_BITS, ln, &s, &last);
  const double incl = chain_scan(s, ln);
  int32_t l = last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l = max(l, __shfl_xor_sync(0xffffffffu, l, o));
  if (ln == 31) bsum[gb] = incl;
  if (ln == 0) blast[gb] = l;
}

// one thread per source: boff[b] = sum of blocks before b (sequential); the
// entry after the last block is the total
__global__ void smp_offsets_kernel(const SmpSource *__restrict__ srcs, uint32_t n_src,
                                   const double *bsum, const int32_t *blast, double *boff,
                                   int64_t *lastnz) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_src) return;
  const SmpSource S = srcs[s];
  double acc = 0;
  int64_t last = -1;
  double *o = boff + S.block_begin + s;  // n_blocks + 1 entries per source
  for (uint32_t b = 0; b < S.n_blocks; b++) {
    o[b] = acc;
    acc = acc + bsum[S.block_begin + b];
    const int32_t l = blast[S.block_begin + b];
    if (l >= 0) last = ((int64_t)b << SMP_BLOCK_BITS) + l;
  }
  o[S.n_blocks] = acc;
  lastnz[s] = last;
}

template <typename T>
__global__ void smp_shot_kernel(const SmpSource *__restrict__ srcs, const SmpShot *__restrict__ shots,
                                uint32_t n_shots, const double *boff, const int64_t *lastnz) {
  typedef typename V2o<T>::t C;
  const uint32_t sh = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int ln = threadIdx.x & 31;
  if (sh >= n_shots) return;
  const SmpShot Q = shots[sh];
  const SmpSource S = srcs[Q.source];
  const double *o = boff + S.block_begin + Q.source;
  const double total = o[S.n_blocks];
  const double target = Q.u * total;
  const uint32_t dim = 1u << S.n;
  if (!(target < total)) {
    if (ln == 0) *Q.out = (uint64_t)lastnz[Q.source];
    return;
  }
  // first block whose end exceeds target
  uint32_t lo = 0, hi = S.n_blocks - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (o[mid + 1] > target) hi = mid; else lo = mid + 1;
  }
  const uint32_t blk = lo;
  const double ob = o[blk];
  const C *psi = (const C *)S.state;
  double s;
  int32_t last;
  lane_sums<T>(psi, dim, blk << SMP_BLOCK_BITS, ln, &s, &last);
  const double incl = chain_scan(s, ln);
  const double excl = __shfl_up_sync(0xffffffffu, incl, 1);
  const double lane_start = (ln == 0) ? 0.0 : excl;
  const unsigned hit = __ballot_sync(0xffffffffu, ob + incl > target);
  if (hit == 0) {  // rounding left the target at the block end: last nonzero
    if (ln == 0) *Q.out = (uint64_t)lastnz[Q.source];
    return;
  }
  const int L = __ffs(hit) - 1;
  if (ln == L) {
    const uint32_t b0 = (blk << SMP_BLOCK_BITS) + (uint32_t)L * SMP_PER_LANE;
    SmpAcc<T> pre;
    uint64_t ans = (uint64_t)b0 + SMP_PER_LANE - 1;
    int64_t last_pos = -1;
    for (int i = 0; i < SMP_PER_LANE; i++) {
      const uint32_t x = b0 + i;
      if (x >= dim) break;
      const auto p = prob32(psi[x]);
      pre.add(p);
      if (p > 0) last_pos = x;
      if (ob + (lane_start + pre.value()) > target) { ans = x; last_pos = -2; break; }
    }
    if (last_pos >= 0) ans = (uint64_t)last_pos;
    *Q.out = ans;
  }
}

void launch_sampling(bool fp64, const SmpSource *srcs, uint32_t n_src, uint32_t total_blocks,
                     double *bsum, int32_t *blast, double *boff, int64_t *lastnz,
                     const SmpShot *shots, uint32_t n_shots, void *stream) {
  if (n_src == 0) return;
  cudaStream_t s = (cudaStream_t)stream;
  const int wpb = 4;
  const uint32_t g1 = (total_blocks + wpb - 1) / wpb;
  if (fp64)
    smp_blocksum_kernel<double><<<g1, wpb * 32, 0, s>>>(srcs, n_src, total_blocks, bsum, blast);
  else
    smp_blocksum_kernel<float><<<g1, wpb * 32, 0, s>>>(srcs, n_src, total_blocks, bsum, blast);
  smp_offsets_kernel<<<(n_src + 127) / 128, 128, 0, s>>>(srcs, n_src, bsum, blast, boff, lastnz);
  if (n_shots == 0) return;
  const uint32_t g3 = (n_shots + wpb - 1) / wpb;
  if (fp64)
    smp_shot_kernel<double><<<g3, wpb * 32, 0, s>>>(srcs, shots, n_shots, boff, lastnz);
  else
    smp_shot_kernel<float><<<g3, wpb * 32, 0, s>>>(srcs, shots, n_shots, boff, lastnz);
}

}  // namespace qw

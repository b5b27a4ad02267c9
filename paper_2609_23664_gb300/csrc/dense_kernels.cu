// Dense-block kernels: the tensor-core form (tcgen05 kind::tf32, operands in
// shared memory, accumulators in tensor memory) and the CUDA-core form.
#include <algorithm>
#include <cstring>

#include "dense.h"
#include "tc_sm100.cuh"

namespace qw {

using namespace qwtc;

namespace {

constexpr int DT_THREADS = 256;
constexpr uint32_t DT_A = 128 * 64 * 4;  // one TF32 split of the amplitude operand (32 KB)
constexpr uint32_t DT_B = 64 * 64 * 4;   // one TF32 split of the unitary operand (16 KB)
constexpr uint32_t DT_OFF_AHI = 0, DT_OFF_ALO = DT_A, DT_OFF_BHI = 2 * DT_A, DT_OFF_BLO = 2 * DT_A + DT_B;
constexpr uint32_t DT_OFF_BAR = 2 * DT_A + 2 * DT_B;
constexpr uint32_t DT_SMEM = DT_OFF_BAR + 64;
constexpr uint64_t DT_WAIT_NS = 2000000000ull;
// Operand layout (no swizzle, K-major core matrices of 8 rows x 4 values):
// A row r, column k at byte (k/4)*2048 + (r/8)*128 + (r%8)*16 + (k%4)*4;
// B row n, column k at byte (k/4)*1024 + (n/8)*128 + (n%8)*16 + (k%4)*4.
constexpr uint32_t DT_A_KCORE = 2048, DT_B_KCORE = 1024, DT_ROWGROUP = 128;

struct DenseTcArgs {
  float2 *state;
  const float4 *bops;
  int *err;
  uint64_t n_tiles;
  uint32_t other_mask;
  DensePos pos;
  // staged layout only: for bit b of the tile index (the 12 tile qubits in
  // ascending order), its offset in the state (tx) and its byte offset in
  // the [position][row] staging array (ts)
  uint32_t tx[12], ts[12];
};

// A block holding most of the lowest qubits leaves the rows of a warp far
// apart in memory (the 32 rows of a warp span 32 x 128 bytes or more, which
// thrashes the L1 left beside 2 x 96 KB of shared memory), so its tiles are
// staged: loaded in memory order with 16-byte accesses into a
// [position][row] array in shared memory (the A_lo area, free between MMAs),
// read back per row, and written out the same way.  Row r of position p sits in slot
// p * 128 + (r ^ (p >> 1)): a warp reading one position of 32 rows stays
// in one aligned 32-slot group, and a warp moving memory-order indices whose
// low bits are block bits spreads over all banks.
// Stage when at least 4 of qubits 0-4 are block qubits (measured on GB300
// at 28 qubits: staged 3.9-4.2 TB/s for such blocks against 1.8-3.1 TB/s
// direct; direct 4.2-5.4 TB/s for every other block against 3.2-4.2 staged).
constexpr int DT_STAGE_LOW_BITS = 4;

}  // namespace

__device__ __forceinline__ uint64_t dense_deposit(uint64_t g, uint32_t mask) {
  uint64_t r = 0;
  for (uint32_t m = mask; g && m; m &= m - 1, g >>= 1)
    if (g & 1) r |= (uint64_t)(m & (~m + 1u));
  return r;
}

// One CTA (8 warps) per 128-group tile at a time, persistent over tiles.
// Thread t owns group row r = t % 128 and block-local indices 16h..16h+15,
// h = t / 128: it loads those 16 amplitudes, writes their TF32 splits into
// the A operand, and after the MMAs reads the same row's new amplitudes
// from tensor memory (lane quarter = warp % 4, columns 16h.. and 32+16h..)
// and stores them where it loaded them, so the update is in place.  The next
// tile's loads are issued while the tensor core works on the current one.
template <int NACC, bool STAGED>
__global__ void __launch_bounds__(DT_THREADS, 2) dense_tc_kernel(const DenseTcArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int t = threadIdx.x, w = t >> 5;
  const int r = t & 127, h = t >> 7;
  const uint32_t base = smem_u32(sm);
  const uint32_t bar = base + DT_OFF_BAR, tslot = base + DT_OFF_BAR + 8;
  {
    float4 *dst = reinterpret_cast<float4 *>(sm + DT_OFF_BHI);
    for (int i = t; i < (int)(2 * DT_B / 16); i += DT_THREADS) dst[i] = a.bops[i];
  }
  if (t == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  if (w == 0) {
    tmem_alloc(tslot, 64 * NACC);
    tmem_relinquish();
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = *reinterpret_cast<volatile uint32_t *>(sm + DT_OFF_BAR + 8);

  const uint64_t dr = dense_deposit((uint64_t)r, a.other_mask);
  uint32_t po[16];
#pragma unroll
  for (int j = 0; j < 16; j++) po[j] = a.pos.v[16 * h + j];
  const uint32_t arow = (uint32_t)(r >> 3) * DT_ROWGROUP + (uint32_t)(r & 7) * 16;
  const uint32_t idesc = idesc_tf32(128, 64);
  const uint32_t lane_addr = tm + ((uint32_t)(32 * (w & 3)) << 16) + 16u * (uint32_t)h;

  // staged layout: thread t moves tile indices 2t + 512m (+1), m < 8; the
  // state offsets add up, the staging slots combine by XOR (swizzle)
  uint32_t sx0 = 0, ss0 = 0, sx[8], ss[8];
  if (STAGED) {
#pragma unroll
    for (int b = 1; b < 9; b++)
      if ((t >> (b - 1)) & 1) {
        sx0 += a.tx[b];
        ss0 ^= a.ts[b];
      }
#pragma unroll
    for (int m = 0; m < 8; m++) {
      sx[m] = sx0 + ((m & 1) ? a.tx[9] : 0) + ((m & 2) ? a.tx[10] : 0) + ((m & 4) ? a.tx[11] : 0);
      ss[m] = ss0 ^ ((m & 1) ? a.ts[9] : 0) ^ ((m & 2) ? a.ts[10] : 0) ^ ((m & 4) ? a.ts[11] : 0);
    }
  }
  const uint32_t ss1 = a.ts[0];
  float2 *stage = reinterpret_cast<float2 *>(sm + DT_OFF_ALO);

  uint32_t phase = 0;
  bool failed = false;
  float2 v[16];
  float4 raw[8];
  uint64_t tile = blockIdx.x, xb = 0;
  if (tile < a.n_tiles) {
    if (STAGED) {
      xb = dense_deposit(tile << 7, a.other_mask);
#pragma unroll
      for (int m = 0; m < 8; m++) raw[m] = __ldcs(reinterpret_cast<const float4 *>(a.state + xb + sx[m]));
    } else {
      xb = dense_deposit(tile << 7, a.other_mask) | dr;
#pragma unroll
      for (int j = 0; j < 16; j++) v[j] = __ldcs(a.state + xb + po[j]);
    }
  }
  for (; tile < a.n_tiles; tile += gridDim.x) {
    if (STAGED) {
#pragma unroll
      for (int m = 0; m < 8; m++) {
        *reinterpret_cast<float2 *>(sm + DT_OFF_ALO + ss[m]) = make_float2(raw[m].x, raw[m].y);
        *reinterpret_cast<float2 *>(sm + DT_OFF_ALO + (ss[m] ^ ss1)) = make_float2(raw[m].z, raw[m].w);
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 16; j++) v[j] = stage[(16 * h + j) * 128 + (r ^ ((16 * h + j) >> 1))];
      __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
      float rh[4], rl[4], ih[4], il[4];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const float2 x = v[4 * c + j];
        rh[j] = to_tf32(x.x);
        rl[j] = to_tf32(x.x - rh[j]);
        ih[j] = to_tf32(x.y);
        il[j] = to_tf32(x.y - ih[j]);
      }
      const uint32_t kre = (uint32_t)(4 * h + c) * DT_A_KCORE + arow;       // k = 16h + 4c
      const uint32_t kim = (uint32_t)(8 + 4 * h + c) * DT_A_KCORE + arow;   // k = 32 + 16h + 4c
      *reinterpret_cast<float4 *>(sm + DT_OFF_AHI + kre) = make_float4(rh[0], rh[1], rh[2], rh[3]);
      *reinterpret_cast<float4 *>(sm + DT_OFF_AHI + kim) = make_float4(ih[0], ih[1], ih[2], ih[3]);
      *reinterpret_cast<float4 *>(sm + DT_OFF_ALO + kre) = make_float4(rl[0], rl[1], rl[2], rl[3]);
      *reinterpret_cast<float4 *>(sm + DT_OFF_ALO + kim) = make_float4(il[0], il[1], il[2], il[3]);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (t == 0) {
      uint32_t started = 0;
      // the two small cross products first, then hi * hi
#pragma unroll
      for (int p = 0; p < 3; p++) {
        const uint32_t ao = base + (p == 0 ? DT_OFF_ALO : DT_OFF_AHI);
        const uint32_t bo = base + (p == 1 ? DT_OFF_BLO : DT_OFF_BHI);
#pragma unroll
        for (int s = 0; s < 8; s++) {
          const int acc = s % NACC;
          mma_tf32(tm + 64u * acc, sdesc_kmajor(ao + s * 2 * DT_A_KCORE, DT_A_KCORE, DT_ROWGROUP),
                   sdesc_kmajor(bo + s * 2 * DT_B_KCORE, DT_B_KCORE, DT_ROWGROUP), idesc, (started >> acc) & 1u);
          started |= 1u << acc;
        }
      }
      mma_commit(bar);
    }
    const uint64_t xcur = xb, nt = tile + gridDim.x;
    if (nt < a.n_tiles) {
      if (STAGED) {
        xb = dense_deposit(nt << 7, a.other_mask);
#pragma unroll
        for (int m = 0; m < 8; m++) raw[m] = __ldcs(reinterpret_cast<const float4 *>(a.state + xb + sx[m]));
      } else {
        xb = dense_deposit(nt << 7, a.other_mask) | dr;
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = __ldcs(a.state + xb + po[j]);
      }
    }
    const bool ok = mbar_wait_bounded(bar, phase, DT_WAIT_NS);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    float re[16], im[16];
    tmem_ld_2x16(lane_addr, lane_addr + 32, re, im);
#pragma unroll
    for (int acc = 1; acc < NACC; acc++) {
      float re2[16], im2[16];
      tmem_ld_2x16(lane_addr + 64u * acc, lane_addr + 64u * acc + 32, re2, im2);
#pragma unroll
      for (int j = 0; j < 16; j++) {
        re[j] += re2[j];
        im[j] += im2[j];
      }
    }
    if (STAGED) {
#pragma unroll
      for (int j = 0; j < 16; j++) stage[(16 * h + j) * 128 + (r ^ ((16 * h + j) >> 1))] = make_float2(re[j], im[j]);
      __syncthreads();
#pragma unroll
      for (int m = 0; m < 8; m++) {
        const float2 lo = *reinterpret_cast<const float2 *>(sm + DT_OFF_ALO + ss[m]);
        const float2 hi = *reinterpret_cast<const float2 *>(sm + DT_OFF_ALO + (ss[m] ^ ss1));
        __stcs(reinterpret_cast<float4 *>(a.state + xcur + sx[m]), make_float4(lo.x, lo.y, hi.x, hi.y));
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; j++) __stcs(a.state + xcur + po[j], make_float2(re[j], im[j]));
    }
    tc_fence_before();
    __syncthreads();
  }
  if (failed) {
    if (t == 0) atomicExch(a.err, 1);
    mbar_wait_bounded(bar, phase, DT_WAIT_NS);  // the MMAs in flight, before their accumulator is freed
  }
  tc_fence_before();
  __syncthreads();
  if (w == 0) {
    tc_fence_after();
    tmem_dealloc(tm, 64 * NACC);
  }
}

// CUDA-core form.  A thread takes G = 32 / 2^K groups per step: with a
// power-of-two grid stride, its groups are base + (j G + i) stride (i < G),
// whose index bits are disjoint, so their offsets are OR-combinations of
// three deposits (base, the step j, the lane i) and a warp's threads read
// consecutive groups.  All 32 input amplitudes are loaded before any output
// is formed (32 loads in flight for any K); every output is a sum over the
// 2^K inputs of its group with U (interleaved complex, row-major) staged in
// shared memory.
template <typename T, typename T2, int K>
__global__ void __launch_bounds__(128) dense_simt_kernel(T2 *state, const T *u, uint64_t n_groups,
                                                         uint32_t other_mask, DensePos pos) {
  constexpr uint32_t D = 1u << K, G = 32u >> K;
  __shared__ T us[2 * D * D];
  for (uint32_t i = threadIdx.x; i < 2 * D * D; i += blockDim.x) us[i] = u[i];
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;  // a power of two
  const uint64_t base = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t dbase = dense_deposit(base, other_mask);
  uint64_t dlane[G];
#pragma unroll
  for (uint32_t i = 0; i < G; i++) dlane[i] = dense_deposit(i * stride, other_mask);
  for (uint64_t j = 0; base + j * G * stride < n_groups; j++) {
    const uint64_t dstep = dbase | dense_deposit(j * G * stride, other_mask);
    T2 in[G][D];
#pragma unroll
    for (uint32_t i = 0; i < G; i++) {
      if (base + (j * G + i) * stride < n_groups) {
#pragma unroll
        for (uint32_t p = 0; p < D; p++) in[i][p] = state[(dstep | dlane[i]) + pos.v[p]];
      }
    }
#pragma unroll
    for (uint32_t i = 0; i < G; i++) {
      if (base + (j * G + i) * stride >= n_groups) continue;
      for (uint32_t o = 0; o < D; o++) {
        T re = 0, im = 0;
        const T *row = us + 2 * o * D;
#pragma unroll
        for (uint32_t p = 0; p < D; p++) {
          const T ur = row[2 * p], ui = row[2 * p + 1];
          re = fma(ur, in[i][p].x, fma(-ui, in[i][p].y, re));
          im = fma(ur, in[i][p].y, fma(ui, in[i][p].x, im));
        }
        T2 out;
        out.x = re;
        out.y = im;
        state[(dstep | dlane[i]) + pos.v[o]] = out;
      }
    }
  }
}

template <int NACC, bool STAGED>
static cudaError_t dense_attr() {
  return cudaFuncSetAttribute(dense_tc_kernel<NACC, STAGED>, cudaFuncAttributeMaxDynamicSharedMemorySize, DT_SMEM);
}

cudaError_t dense_init_attrs() {
  const cudaError_t e[6] = {dense_attr<1, false>(), dense_attr<2, false>(), dense_attr<4, false>(),
                            dense_attr<1, true>(),  dense_attr<2, true>(),  dense_attr<4, true>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

void launch_dense_tc(float2 *state, uint32_t n, const DenseBlock &b5, const float *bops, int nacc, int *err,
                     int sm_count, cudaStream_t s) {
  if (b5.k != 5 || n < DENSE_TC_MIN_QUBITS || n > QW_SV_MAX_QUBITS)
    fail(QW_ERR_INVALID_ARG, "tensor-core dense block needs k = 5 and n in [%u, %u]", DENSE_TC_MIN_QUBITS,
         (unsigned)QW_SV_MAX_QUBITS);
  DenseTcArgs a;
  a.state = state;
  a.bops = reinterpret_cast<const float4 *>(bops);
  a.err = err;
  a.n_tiles = 1ull << (n - DENSE_TC_MIN_QUBITS);
  a.other_mask = dense_other_mask(b5, n);
  a.pos = dense_positions(b5);
  // tile bits in ascending order: the block's 5 and the 7 lowest others
  uint32_t tmask = ~a.other_mask & ((1u << n) - 1);
  for (uint32_t m = a.other_mask, c = 0; m && c < 7; m &= m - 1, c++) tmask |= m & (~m + 1u);
  for (uint32_t b = 0, m = tmask; b < 12; b++, m &= m - 1) {
    const uint32_t q = (uint32_t)__builtin_ctz(m);
    a.tx[b] = 1u << q;
    uint32_t j = 0;
    while (j < 5 && b5.q[j] != q) j++;
    // byte offset of the staging slot, XOR-linear in the tile-index bits
    if (j < 5) {
      a.ts[b] = (((1u << j) << 7) ^ ((1u << j) >> 1)) * 8;  // position bit j (and its swizzle)
    } else {
      const uint32_t rho = (uint32_t)__builtin_popcount(a.other_mask & ((1u << q) - 1));
      a.ts[b] = (1u << rho) * 8;  // row bit rho
    }
  }
  const bool staged = __builtin_popcount(~a.other_mask & 31u) >= DT_STAGE_LOW_BITS;
  const int grid = (int)std::min<uint64_t>(a.n_tiles, (uint64_t)(2 * sm_count));
  if (nacc != 1 && nacc != 2 && nacc != 4) fail(QW_ERR_INVALID_ARG, "nacc must be 1, 2 or 4");
  if (staged) {
    if (nacc == 4) dense_tc_kernel<4, true><<<grid, DT_THREADS, DT_SMEM, s>>>(a);
    else if (nacc == 2) dense_tc_kernel<2, true><<<grid, DT_THREADS, DT_SMEM, s>>>(a);
    else dense_tc_kernel<1, true><<<grid, DT_THREADS, DT_SMEM, s>>>(a);
  } else {
    if (nacc == 4) dense_tc_kernel<4, false><<<grid, DT_THREADS, DT_SMEM, s>>>(a);
    else if (nacc == 2) dense_tc_kernel<2, false><<<grid, DT_THREADS, DT_SMEM, s>>>(a);
    else dense_tc_kernel<1, false><<<grid, DT_THREADS, DT_SMEM, s>>>(a);
  }
}

void launch_dense_simt(bool fp64, void *state, uint32_t n, const DenseBlock &b, const void *u, int sm_count,
                       cudaStream_t s) {
  if (b.k < 1 || b.k > DENSE_MAX_QUBITS || b.k > n) fail(QW_ERR_INVALID_ARG, "dense block of %u qubits", b.k);
  const uint64_t groups = 1ull << (n - b.k);
  // a power-of-two grid (the kernel combines group offsets by OR), at most
  // 8 CTAs per SM and no more than the groups need
  const uint64_t per_cta = 128ull * (32u >> b.k);  // groups a CTA takes per step
  uint64_t grid = 1;
  while (grid * 2 <= (uint64_t)sm_count * 8 && grid * per_cta < groups) grid *= 2;
  const uint32_t om = dense_other_mask(b, n);
  const DensePos pos = dense_positions(b);
#define QW_SIMT(KK)                                                                                       \
  if (fp64)                                                                                               \
    dense_simt_kernel<double, double2, KK><<<(unsigned)grid, 128, 0, s>>>((double2 *)state, (const double *)u,      \
                                                                  groups, om, pos);                       \
  else                                                                                                    \
    dense_simt_kernel<float, float2, KK><<<(unsigned)grid, 128, 0, s>>>((float2 *)state, (const float *)u, groups, \
                                                                om, pos);
  switch (b.k) {
    case 1: QW_SIMT(1) break;
    case 2: QW_SIMT(2) break;
    case 3: QW_SIMT(3) break;
    case 4: QW_SIMT(4) break;
    default: QW_SIMT(5) break;
  }
#undef QW_SIMT
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
DensePos dense_positions(const DenseBlock &b) {
  DensePos p{};
  for (uint32_t i = 0; i < (1u << b.k); i++) {
    uint32_t off = 0;
    for (uint32_t j = 0; j < b.k; j++)
      if (i >> j & 1) off |= 1u << b.q[j];
    p.v[i] = off;
  }
  return p;
}

uint32_t dense_other_mask(const DenseBlock &b, uint32_t n) {
  uint32_t m = (n >= 32) ? 0xffffffffu : ((1u << n) - 1);
  for (uint32_t j = 0; j < b.k; j++) m &= ~(1u << b.q[j]);
  return m;
}

DenseBlock pad_block(const DenseBlock &b, uint32_t n) {
  if (b.k == 5) return b;
  DenseBlock o;
  o.k = 5;
  o.n_gates = b.n_gates;
  uint32_t used = 0;
  for (uint32_t j = 0; j < b.k; j++) {
    o.q[j] = b.q[j];
    used |= 1u << b.q[j];
  }
  uint32_t j = b.k;
  for (int q = (int)n - 1; q >= 0 && j < 5; q--)
    if (!(used >> q & 1)) o.q[j++] = (uint32_t)q;
  if (j < 5) fail(QW_ERR_INVALID_ARG, "register of %u qubits is too small for a 5-qubit block", n);
  const uint32_t d = 1u << b.k, lo = d - 1;
  o.u.assign(32 * 32, 0.0);
  for (uint32_t po = 0; po < 32; po++)
    for (uint32_t pi = 0; pi < 32; pi++)
      if ((po >> b.k) == (pi >> b.k)) o.u[po * 32 + pi] = b.u[(po & lo) * d + (pi & lo)];
  return o;
}

static float tf32_rna(float x) {
  uint32_t bits;
  std::memcpy(&bits, &x, 4);
  if ((bits & 0x7f800000u) != 0x7f800000u) {
    bits += 0x1000u;  // half of the 13 dropped mantissa bits: ties away from zero
    bits &= 0xffffe000u;
  }
  std::memcpy(&x, &bits, 4);
  return x;
}

void dense_tc_operands(const DenseBlock &b5, float *out) {
  for (uint32_t n = 0; n < 64; n++)
    for (uint32_t k = 0; k < 64; k++) {
      const std::complex<double> u = b5.u[(n & 31) * 32 + (k & 31)];
      const double val = (n < 32) ? (k < 32 ? u.real() : -u.imag()) : (k < 32 ? u.imag() : u.real());
      const float hi = tf32_rna((float)val);
      const float lo = tf32_rna((float)(val - (double)hi));
      const uint32_t idx = ((k >> 2) * DT_B_KCORE + (n >> 3) * DT_ROWGROUP + (n & 7) * 16 + (k & 3) * 4) / 4;
      out[idx] = hi;
      out[4096 + idx] = lo;
    }
}

}  // namespace qw

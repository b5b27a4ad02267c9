// Stabilizer-tableau kernels (sm_103a), 64-bit words.
//
// The GPU keeps the INVERSE tableau T: for every generator X_i / Z_i of the
// initial frame it stores the Pauli string T(P) = C^-1 P C (C = circuit so
// far) as x-words, z-words and a sign, row-major, 2n rows in shared memory.
// A gate G of the circuit updates T by T'(P) = T(G^-1 P G), which is a
// product or a swap of ROWS (word-parallel over all qubits: W = ceil(n/64)
// words per half-row).  Measuring Z_a reads row T(Z_a): without an X part
// the outcome is its sign (deterministic); otherwise the outcome is random
// and the tableau is collapsed by conjugating every row with a few column
// operations in the initial frame (CNOTs, S^dagger, H, X), which leave
// |0...0> invariant up to the projected outcome.  This is the Heisenberg-
// picture formulation used by the stabilizer simulator the paper cites
// [gidney2021stim]; the CPU oracle uses the textbook forward tableau
// [aaronson2004stabilizer], so the two share no algorithm.  Measurement
// outcomes agree bit for bit: a deterministic outcome is fixed by the state,
// and a random one takes the outcome bit carried by the gate record.
//
// Row products keep Paulis in the Hermitian form (-1)^r i^{x.z} X^x Z^z:
// P1 P2 = (-1)^{r1+r2} i^{x1.z1 + x2.z2 - x3.z3 + 2 z1.x2 + e0} P3 where e0
// is an extra power of i (S: 3, S^dagger: 1) and the exponent is 0 or 2.
#include <cuda_runtime.h>

#include "qw_internal.h"

namespace qw {

constexpr uint32_t TAB_SLOT_STAGE = 1024;  // slots of a layer staged in shared memory at a time
constexpr int TAB_THREADS = 512;

struct TabSm {
  uint64_t *R;     // rows * 2W words
  uint8_t *sign;   // rows
  uint8_t *pending;
  uint64_t *xs;    // W words (collapse scratch)
  TabSlot *sl;     // TAB_SLOT_STAGE staged slots of the current layer
  TabSlot *sl_alt; // the other staging buffer (== sl when single-buffered)
  uint32_t *any_random;
  uint32_t W, W2;  // words per half row, per row
  uint32_t swz;    // word swizzle mask (2W - 1 when 2W is a power of two <= 16, else 0)
};

// Shared memory of a tableau of n qubits with one slot staging buffer, and
// whether a second one fits under the size the largest tableau needs (then
// a layer's slots are staged while the previous layer runs, saving a
// barrier per layer).
QW_HD inline size_t tab_smem_single(uint32_t n) {
  const uint32_t W = (n + 63) / 64, rows = 2 * n;
  return (size_t)rows * 2 * W * 8 + ((rows + 15) & ~15u) + ((n + 15) & ~15u) + (size_t)((W + 1) & ~1u) * 8 +
         (size_t)TAB_SLOT_STAGE * sizeof(TabSlot) + 16;
}
QW_HD inline bool tab_double_buffer(uint32_t n) {
  return tab_smem_single(n) + (size_t)TAB_SLOT_STAGE * sizeof(TabSlot) <= tab_smem_single(QW_TABLEAU_MAX_QUBITS);
}

// Word c of row r (x words 0..W-1, then z words W..2W-1).  When a row is a
// power-of-two number of words, word c is stored at position c ^ (r mod 2W)
// of its row, so that 32 threads reading word c of 32 different rows
// spread over the shared-memory banks instead of all hitting one.
__device__ __forceinline__ uint64_t &tw(const TabSm &S, uint32_t r, uint32_t c) {
  return S.R[(size_t)r * S.W2 + (c ^ (r & S.swz))];
}
__device__ __forceinline__ int getx(const TabSm &S, uint32_t r, uint32_t q) {
  return (int)((tw(S, r, q >> 6) >> (q & 63)) & 1ull);
}
__device__ __forceinline__ int getz(const TabSm &S, uint32_t r, uint32_t q) {
  return (int)((tw(S, r, S.W + (q >> 6)) >> (q & 63)) & 1ull);
}
__device__ __forceinline__ void flipx(const TabSm &S, uint32_t r, uint32_t q) { tw(S, r, q >> 6) ^= 1ull << (q & 63); }
__device__ __forceinline__ void flipz(const TabSm &S, uint32_t r, uint32_t q) {
  tw(S, r, S.W + (q >> 6)) ^= 1ull << (q & 63);
}

// column op in the initial frame: CNOT(c -> t) conjugation of row r
__device__ __forceinline__ void col_cnot(const TabSm &S, uint32_t r, uint8_t *sg, uint32_t c, uint32_t t) {
  const int xc = getx(S, r, c), zc = getz(S, r, c), xt = getx(S, r, t), zt = getz(S, r, t);
  *sg ^= (uint8_t)(xc & zt & (xt ^ zc ^ 1));
  if (xc) flipx(S, r, t);
  if (zt) flipz(S, r, c);
}

// One unitary slot by one thread, W a power of two (swizzled rows): the
// row bases and swizzles are computed once, the word loop is unrolled.
template <uint32_t W>
__device__ __forceinline__ void tab_slot(const TabSm &S, const TabSlot &sl) {
  constexpr uint32_t M = 2 * W - 1;
  uint64_t *rd = S.R + (size_t)sl.dst * (2 * W);
  const uint32_t kd = sl.dst & M;
  if (sl.kind == T_PROD) {
    const uint64_t *r1 = S.R + (size_t)sl.s1 * (2 * W), *r2 = S.R + (size_t)sl.s2 * (2 * W);
    const uint32_t k1 = sl.s1 & M, k2 = sl.s2 & M;
    int t = 0;
#pragma unroll
    for (uint32_t c = 0; c < W; c++) {
      const uint64_t x1 = r1[c ^ k1], z1 = r1[(W + c) ^ k1];
      const uint64_t x2 = r2[c ^ k2], z2 = r2[(W + c) ^ k2];
      const uint64_t x3 = x1 ^ x2, z3 = z1 ^ z2;
      t += __popcll(x1 & z1) + __popcll(x2 & z2) - __popcll(x3 & z3) + 2 * __popcll(z1 & x2);
      rd[c ^ kd] = x3;
      rd[(W + c) ^ kd] = z3;
    }
    S.sign[sl.dst] = S.sign[sl.s1] ^ S.sign[sl.s2] ^ (uint8_t)((((t + sl.flags) & 3) >> 1) & 1);
  } else if (sl.kind == T_SWAP2) {
    uint64_t *r2 = S.R + (size_t)sl.s2 * (2 * W);
    const uint32_t k2 = sl.s2 & M;
#pragma unroll
    for (uint32_t c = 0; c < 2 * W; c++) {
      const uint64_t a0 = rd[c ^ kd];
      rd[c ^ kd] = r2[c ^ k2];
      r2[c ^ k2] = a0;
    }
    const uint8_t tmp = S.sign[sl.dst];
    S.sign[sl.dst] = S.sign[sl.s2];
    S.sign[sl.s2] = tmp;
  } else if (sl.kind == T_SIGN) {
    S.sign[sl.dst] ^= 1;
  }
}

__device__ void tab_collapse(const TabArgs &A, TabSm &S, const TabSlot &sl, uint32_t bits_base,
                             uint32_t out_base) {
  const uint32_t n = A.n, W = A.W, rows = A.rows, row = sl.dst;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid < (int)W) S.xs[tid] = tw(S, row, (uint32_t)tid);
  __syncthreads();
  int first = -1;
  for (uint32_t w = 0; w < W; w++)
    if (S.xs[w]) { first = (int)(w * 64 + __ffsll((long long)S.xs[w]) - 1); break; }
  const uint8_t m = A.bits[bits_base + sl.aux] & 1;
  if (first < 0) {  // became deterministic
    __syncthreads();
    if (tid == 0) {
      const uint8_t o = S.sign[row];
      if (sl.aux2 != 0xFFFFFFFFu) A.outs[out_base + sl.aux2] = o;
      if ((sl.flags & 1) && o) S.sign[row] ^= 1;
    }
    __syncthreads();
    return;
  }
  const uint32_t p = (uint32_t)first;
  (void)n;
  if (tid == 0) *S.any_random = 1u;
  // 1) CNOT(p -> q) for every other q in the X part of T(Z_a)
  for (uint32_t r = tid; r < rows; r += nt) {
    uint8_t sg = S.sign[r];
    for (uint32_t w = 0; w < W; w++) {
      uint64_t bitsw = S.xs[w];
      if (w == (p >> 6)) bitsw &= ~(1ull << (p & 63));
      while (bitsw) {
        const uint32_t q = w * 64 + __ffsll((long long)bitsw) - 1;
        bitsw &= bitsw - 1;
        col_cnot(S, r, &sg, p, q);
      }
    }
    S.sign[r] = sg;
  }
  __syncthreads();
  // 2) Y -> X at p by S^dagger conjugation when T(Z_a) has Z at p
  const int zp = getz(S, row, p);
  __syncthreads();
  if (zp) {
    for (uint32_t r = tid; r < rows; r += nt) {
      const int xb = getx(S, r, p), zb = getz(S, r, p);
      S.sign[r] ^= (uint8_t)(xb & (zb ^ 1));
      if (xb) flipz(S, r, p);
    }
    __syncthreads();
  }
  // 3) T(Z_a) = (-1)^s X_p Z_Q: conjugate by H_p then X_p^(m xor s)
  const uint8_t s = S.sign[row];
  __syncthreads();
  const int bb = (int)(m ^ s);
  for (uint32_t r = tid; r < rows; r += nt) {
    const int xb = getx(S, r, p), zb = getz(S, r, p);
    uint8_t sg = S.sign[r] ^ (uint8_t)(xb & zb);
    if (xb != zb) { flipx(S, r, p); flipz(S, r, p); }
    if (bb) sg ^= (uint8_t)xb;  // new z bit at p equals the old x bit
    S.sign[r] = sg;
  }
  __syncthreads();
  if (tid == 0) {
    if (sl.aux2 != 0xFFFFFFFFu) A.outs[out_base + sl.aux2] = m;
    if ((sl.flags & 1) && m) S.sign[row] ^= 1;
  }
  __syncthreads();
}

__device__ void tab_run_program(const TabArgs &A, TabSm &S, const TabProgram &P, uint32_t bits_base,
                                uint32_t out_base) {
  const uint32_t W = A.W, lpp = A.lpp;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5, ln = threadIdx.x & 31;
  const uint32_t gpw = 32 / lpp;  // slot groups per warp
  const uint32_t w = ln % lpp;
  // The first TAB_SLOT_STAGE slots of the next layer are loaded into
  // registers while the current layer runs, and the descriptor of the layer
  // after it as well, so that neither staging a layer nor starting its
  // prefetch waits on a dependent global load.
  constexpr int PRE = TAB_SLOT_STAGE / TAB_THREADS;
  static_assert(PRE * TAB_THREADS == TAB_SLOT_STAGE, "slot prefetch shape");
  TabSlot pre[PRE];
  TabLayer Lnext = {}, Lafter = {};
  auto desc = [&](uint32_t li) {
    TabLayer d = {};
    if (li < P.n_layers) d = A.layers[P.layer_begin + li];
    return d;
  };
  // slots of layer li (descriptor Lnext) into pre[], descriptor of li + 1
  // into Lafter
  auto prefetch = [&](uint32_t li) {
    if (li >= P.n_layers) return;
    const uint32_t cn = min(TAB_SLOT_STAGE, Lnext.n_slots);
#pragma unroll
    for (int k = 0; k < PRE; k++) {
      const uint32_t i = threadIdx.x + (uint32_t)k * TAB_THREADS;
      if (i < cn) pre[k] = A.slots[Lnext.slot_begin + i];
    }
    Lafter = desc(li + 1);
  };
  // with two staging buffers, a small layer writes the next layer's first
  // slots into the other buffer before its closing barrier
  TabSlot *sl_cur = S.sl, *sl_alt = S.sl_alt;
  const bool db = sl_alt != sl_cur;
  auto stage_next = [&](uint32_t li) {
    if (!db || li + 1 >= P.n_layers) return false;
    const uint32_t cn = min(TAB_SLOT_STAGE, Lnext.n_slots);
#pragma unroll
    for (int k = 0; k < PRE; k++) {
      const uint32_t i = threadIdx.x + (uint32_t)k * TAB_THREADS;
      if (i < cn) sl_alt[i] = pre[k];
    }
    return true;
  };
  bool staged = false;  // this layer's slots are already in S.sl_alt
  Lnext = desc(0);
  prefetch(0);
  for (uint32_t li = 0; li < P.n_layers; li++) {
    const TabLayer cur = Lnext;
    Lnext = Lafter;
    if (staged) {
      TabSlot *t = sl_cur;
      sl_cur = sl_alt;
      sl_alt = t;
    } else {
      const uint32_t cn = min(TAB_SLOT_STAGE, cur.n_slots);
#pragma unroll
      for (int k = 0; k < PRE; k++) {
        const uint32_t i = threadIdx.x + (uint32_t)k * TAB_THREADS;
        if (i < cn) sl_cur[i] = pre[k];
      }
      __syncthreads();
    }
    staged = false;
    if (cur.n_slots <= TAB_SLOT_STAGE) prefetch(li + 1);
    if (!cur.is_measure) {
      // the layer's slots are staged in shared memory (one coalesced read
      // instead of a dependent global load per slot group)
      for (uint32_t c0 = 0; c0 < cur.n_slots; c0 += TAB_SLOT_STAGE) {
      const uint32_t cn = min(TAB_SLOT_STAGE, cur.n_slots - c0);
      if (c0 > 0) {
        for (uint32_t i = threadIdx.x; i < cn; i += blockDim.x) sl_cur[i] = A.slots[cur.slot_begin + c0 + i];
        __syncthreads();
      }
      if (S.swz) {
        // one thread per slot over all the row's words (swizzled rows keep
        // the 32 rows of a warp on different banks)
        for (uint32_t i = threadIdx.x; i < cn; i += blockDim.x) {
          const TabSlot sl = sl_cur[i];
          switch (W) {
            case 8: tab_slot<8>(S, sl); break;
            case 4: tab_slot<4>(S, sl); break;
            case 2: tab_slot<2>(S, sl); break;
            default: tab_slot<1>(S, sl); break;
          }
        }
        if (cur.n_slots <= TAB_SLOT_STAGE) staged = stage_next(li);
        __syncthreads();
        continue;
      }
      for (uint32_t sb = warp * gpw; sb < cn; sb += nwarps * gpw) {
        const uint32_t si = sb + ln / lpp;
        const bool act = si < cn;
        TabSlot sl{};
        if (act) sl = sl_cur[si];
        int t = 0;
        if (act && sl.kind == T_PROD) {
          if (w < W) {
            const uint64_t x1 = tw(S, sl.s1, w), z1 = tw(S, sl.s1, W + w);
            const uint64_t x2 = tw(S, sl.s2, w), z2 = tw(S, sl.s2, W + w);
            const uint64_t x3 = x1 ^ x2, z3 = z1 ^ z2;
            t = __popcll(x1 & z1) + __popcll(x2 & z2) - __popcll(x3 & z3) + 2 * __popcll(z1 & x2);
            tw(S, sl.dst, w) = x3;
            tw(S, sl.dst, W + w) = z3;
          }
        } else if (act && sl.kind == T_SWAP2) {
          if (w < W) {
            const uint64_t a0 = tw(S, sl.dst, w), a1 = tw(S, sl.dst, W + w);
            tw(S, sl.dst, w) = tw(S, sl.s2, w);
            tw(S, sl.dst, W + w) = tw(S, sl.s2, W + w);
            tw(S, sl.s2, w) = a0;
            tw(S, sl.s2, W + w) = a1;
          }
        }
        for (uint32_t o = lpp >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o, lpp);
        if (act && w == 0) {
          if (sl.kind == T_PROD) {
            S.sign[sl.dst] = S.sign[sl.s1] ^ S.sign[sl.s2] ^ (uint8_t)((((t + sl.flags) & 3) >> 1) & 1);
          } else if (sl.kind == T_SWAP2) {
            const uint8_t tmp = S.sign[sl.dst];
            S.sign[sl.dst] = S.sign[sl.s2];
            S.sign[sl.s2] = tmp;
          } else if (sl.kind == T_SIGN) {
            S.sign[sl.dst] ^= 1;
          }
        }
      }
      if (cur.n_slots <= TAB_SLOT_STAGE) staged = stage_next(li);
      __syncthreads();
      }
      if (cur.n_slots > TAB_SLOT_STAGE) prefetch(li + 1);
    } else {
      // a measurement layer holds at most one slot per qubit (<= 640), so
      // all of its slots are in the staging buffer already
      // phase 1: deterministic outcomes in parallel, random ones flagged
      int my_pending = 0;
      if (S.swz) {  // one thread per slot (swizzled rows)
        for (uint32_t si = threadIdx.x; si < cur.n_slots; si += blockDim.x) {
          const TabSlot sl = sl_cur[si];
          const uint64_t *rr = S.R + (size_t)sl.dst * S.W2;
          const uint32_t kr = sl.dst & S.swz;
          uint64_t v = 0;
          for (uint32_t c = 0; c < W; c++) v |= rr[c ^ kr];
          if (v == 0) {
            const uint8_t oc = S.sign[sl.dst];
            if (sl.aux2 != 0xFFFFFFFFu) A.outs[out_base + sl.aux2] = oc;
            if ((sl.flags & 1) && oc) S.sign[sl.dst] ^= 1;
            S.pending[si] = 0;
          } else {
            S.pending[si] = 1;
            my_pending = 1;
          }
        }
      } else {
        for (uint32_t sb = warp * gpw; sb < cur.n_slots; sb += nwarps * gpw) {
          const uint32_t si = sb + ln / lpp;
          const bool act = si < cur.n_slots;
          TabSlot sl{};
          if (act) sl = sl_cur[si];
          uint64_t v = 0;
          if (act && w < W) v = tw(S, sl.dst, w);
          for (uint32_t o = lpp >> 1; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o, lpp);
          if (act && w == 0) {
            if (v == 0) {
              const uint8_t oc = S.sign[sl.dst];
              if (sl.aux2 != 0xFFFFFFFFu) A.outs[out_base + sl.aux2] = oc;
              if ((sl.flags & 1) && oc) S.sign[sl.dst] ^= 1;
              S.pending[si] = 0;
            } else {
              S.pending[si] = 1;
              my_pending = 1;
            }
          }
        }
      }
      staged = stage_next(li);
      // phase 2 (only when some outcome is random): one at a time, in
      // program order
      if (__syncthreads_or(my_pending)) {
        for (uint32_t si = 0; si < cur.n_slots; si++) {
          if (S.pending[si]) {
            const TabSlot sl = sl_cur[si];
            tab_collapse(A, S, sl, bits_base, out_base);
          }
        }
        __syncthreads();
      }
    }
  }
}

__global__ void __launch_bounds__(TAB_THREADS, 1) tab_kernel(TabArgs A) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint32_t s_any_random;
  if (A.run_if && *A.run_if == 0u) return;  // uniform over the grid
  const uint32_t W = A.W, rows = A.rows;
  TabSm S;
  S.any_random = &s_any_random;
  if (threadIdx.x == 0) s_any_random = 0u;
  S.R = (uint64_t *)smraw;
  S.sign = (uint8_t *)(S.R + (size_t)rows * 2 * W);
  S.pending = S.sign + ((rows + 15) & ~15u);
  S.xs = (uint64_t *)(S.pending + ((A.n + 15) & ~15u));
  S.sl = (TabSlot *)(S.xs + ((W + 1) & ~1u));
  S.sl_alt = tab_double_buffer(A.n) ? S.sl + TAB_SLOT_STAGE : S.sl;
  S.W = W;
  S.W2 = 2 * W;
  S.swz = (W == 1 || W == 2 || W == 4 || W == 8) ? 2 * W - 1 : 0u;
  const size_t nwords = (size_t)rows * 2 * W;
  const TabTaskDesc T = A.tasks[blockIdx.x];
  if (A.init_rows) {
    for (size_t i = threadIdx.x; i < nwords; i += blockDim.x)
      tw(S, (uint32_t)(i / (2 * W)), (uint32_t)(i % (2 * W))) = __ldg(A.init_rows + i);
    for (uint32_t i = threadIdx.x; i < rows; i += blockDim.x) S.sign[i] = __ldg(A.init_sign + i);
  } else {
    for (size_t i = threadIdx.x; i < nwords; i += blockDim.x) {
      const uint32_t r = (uint32_t)(i / (2 * W)), c = (uint32_t)(i % (2 * W));
      // row r < n: X_r (bit r in the x half); row n+i: Z_i (bit i in the z half)
      uint64_t v = 0;
      if (r < A.n) {
        if (c < W && (r >> 6) == c) v = 1ull << (r & 63);
      } else {
        const uint32_t q = r - A.n;
        if (c >= W && (q >> 6) == c - W) v = 1ull << (q & 63);
      }
      tw(S, r, c) = v;
    }
    for (uint32_t i = threadIdx.x; i < rows; i += blockDim.x) S.sign[i] = 0;
  }
  __syncthreads();
  for (uint32_t si = 0; si < T.n_segs; si++) {
    const TabSegment sg = A.segs[T.seg_begin + si];
    const TabProgram P = A.progs[sg.prog];
    tab_run_program(A, S, P, sg.bit_base, T.out_base + sg.out_base);
  }
  __syncthreads();
  if (A.rand_any && threadIdx.x == 0) A.rand_any[blockIdx.x] = s_any_random;
  if (A.out_rows) {
    uint64_t *o = A.out_rows + (size_t)blockIdx.x * nwords;
    for (size_t i = threadIdx.x; i < nwords; i += blockDim.x)
      o[i] = tw(S, (uint32_t)(i / (2 * W)), (uint32_t)(i % (2 * W)));
    uint8_t *os = A.out_sign + (size_t)blockIdx.x * rows;
    for (uint32_t i = threadIdx.x; i < rows; i += blockDim.x) os[i] = S.sign[i];
  }
}

size_t tab_smem_bytes(uint32_t n) {
  return tab_smem_single(n) + (tab_double_buffer(n) ? (size_t)TAB_SLOT_STAGE * sizeof(TabSlot) : 0);
}

// the largest tableau (QW_TABLEAU_MAX_QUBITS) fits below the 227 KB opt-in
// limit together with the kernel's static shared memory
cudaError_t tab_init_attrs() {
  return cudaFuncSetAttribute((const void *)tab_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tab_smem_bytes(QW_TABLEAU_MAX_QUBITS));
}

void launch_tab(const TabArgs &a, uint32_t n_tasks, void *stream) {
  if (n_tasks == 0) return;
  tab_kernel<<<n_tasks, TAB_THREADS, tab_smem_bytes(a.n), (cudaStream_t)stream>>>(a);
}

}  // namespace qw

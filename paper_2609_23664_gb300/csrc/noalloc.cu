// Pauli-sum energy of a caller-owned device state without any device
// allocation: qw_sv_energy_noalloc_dev.
//
// Some callers cannot allocate device memory: programs whose device memory
// is fully owned by another allocator (for example a framework's caching
// allocator that has reserved the whole pool, where a cudaMalloc beside it
// fails or fragments it), and latency-bound loops with a fixed memory
// footprint that cannot accept the implicit device synchronization of
// cudaFree.  They pass the state and an output buffer; everything else the
// energy kernels need (term layout, job record, per-block partial sums)
// lives in one file-scope device array of fixed size, which every GPU that
// loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>

#include "qw_internal.h"

namespace qw {

namespace {

constexpr uint32_t NA_MAX_CLASSES = 8;
// blocks of the largest register: 2^u class-0 chunks plus 2^(u-1) chunks
// for each other class, times the blocks per chunk (u = 3 above 15 qubits)
constexpr uint32_t NA_MAX_BLOCKS = (1u << (QW_NOALLOC_MAX_QUBITS - 3 - EN_BLOCK_BITS)) * (8u + 7u * 4u);

struct NaHeader {
  EnJob job;
  EnClass classes[NA_MAX_CLASSES];
  EnTerm terms[QW_NOALLOC_MAX_TERMS];
};
struct NaScratch {
  NaHeader h;
  alignas(16) double partials[2 * NA_MAX_BLOCKS];
};

}  // namespace

// The scratch array (about 1.2 MB).  In host code this name is only a
// stand-in for the device object: its device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char qw_noalloc_scratch[sizeof(NaScratch)];

namespace {

std::mutex g_mu;
void *g_dev_ptr[256];  // device address of the scratch array, per device

qw_status scratch_address(int dev, NaScratch **out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 256) {
    set_last_error("device ordinal out of range");
    return QW_ERR_INVALID_ARG;
  }
  if (!g_dev_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, qw_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error(std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return QW_ERR_CUDA;
    }
    g_dev_ptr[dev] = p;
  }
  *out = (NaScratch *)g_dev_ptr[dev];
  return QW_OK;
}

// Term layout for the fixed arrays: classes by the flip bits above the
// chunk, term order kept inside a class, as in the allocating entry point,
// but always with 3 class bits once n >= 15 (chunks of an eighth of the
// state), so that every layout fits NA_MAX_CLASSES and NA_MAX_BLOCKS.  The
// allocating entry point sizes chunks to at most EN_CHUNK_BYTES instead
// (one class for FP32 states up to 22 qubits, chunks of 64 MB at 26): the
// two compute the same terms with the same kernel, adding them in a
// different order and at a different speed.
void layout_fixed(const qw_pauli_term *terms, uint32_t n_terms, uint32_t n, NaHeader &h,
                  uint32_t *n_classes, uint32_t *n_blocks, uint32_t *chunk_bits_out) {
  uint32_t u = 0, chunk_bits = n;
  if (n >= (uint32_t)EN_BLOCK_BITS) {
    u = (n - EN_BLOCK_BITS < 3u) ? n - EN_BLOCK_BITS : 3u;
    chunk_bits = n - u;
  }
  const uint32_t bpc = (chunk_bits >= (uint32_t)EN_BLOCK_BITS) ? (1u << (chunk_bits - EN_BLOCK_BITS)) : 1u;
  uint32_t count[NA_MAX_CLASSES] = {0}, start[NA_MAX_CLASSES] = {0};
  for (uint32_t k = 0; k < n_terms; k++) count[(uint32_t)(terms[k].xmask >> chunk_bits)]++;
  uint32_t nc = 0, blk = 0, off = 0;
  for (uint32_t d = 0; d < (1u << u); d++) {
    if (d != 0 && count[d] == 0) continue;
    EnClass c{};
    c.term_begin = off;
    c.term_end = off + count[d];
    c.hb = (d == 0) ? 0xFFFFFFFFu : (chunk_bits + 31 - __builtin_clz(d));
    c.n_own = (d == 0) ? (1u << u) : (1u << (u - 1));
    c.block_begin = blk;
    blk += c.n_own * bpc;
    start[d] = off;
    off += count[d];
    h.classes[nc++] = c;
  }
  uint32_t fill[NA_MAX_CLASSES] = {0};
  for (uint32_t k = 0; k < n_terms; k++) {
    const uint64_t m = terms[k].xmask, z = terms[k].zmask;
    const int y = __builtin_popcountll(m & z);
    const double sgn = ((y & 3) == 0 || (y & 3) == 3) ? 1.0 : -1.0;
    const uint32_t d = (uint32_t)(m >> chunk_bits);
    EnTerm t{};
    t.xm = (uint32_t)m;
    t.zm = (uint32_t)z;
    t.flags = (uint32_t)(y & 1);
    t.coef = terms[k].coef * sgn * (m ? 2.0 : 1.0);
    t.skip = (d == 0 && m != 0) ? (1u << (63 - __builtin_clzll(m))) : 0u;
    h.terms[start[d] + fill[d]++] = t;
  }
  *n_classes = nc;
  *n_blocks = blk;
  *chunk_bits_out = chunk_bits;
}

// Copies the host-built layout, passed by value as the kernel's parameter
// (the device reads no host memory), into the scratch array.
__global__ void na_setup_kernel(const NaHeader h, NaHeader *dst, uint32_t words) {
  const uint32_t *src = (const uint32_t *)&h;
  uint32_t *d = (uint32_t *)dst;
  for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) d[i] = src[i];
}
static_assert(sizeof(NaHeader) <= 32000, "layout must fit the kernel parameter space");
static_assert(sizeof(NaHeader) % 4 == 0, "layout is copied in 32-bit words");

}  // namespace
}  // namespace qw

extern "C" qw_status qw_sv_energy_noalloc_dev(uint32_t mode, uint32_t n, const void *state,
                                              const qw_pauli_term *terms, uint64_t n_terms, double *out,
                                              void *stream) {
  using namespace qw;
  set_last_error("");
  if (mode > QW_MODE_SV_FP32) {
    set_last_error("statevector modes only");
    return QW_ERR_INVALID_ARG;
  }
  if (!state || !out || (n_terms && !terms)) {
    set_last_error("NULL argument");
    return QW_ERR_INVALID_ARG;
  }
  if (n < SV_G) {
    set_last_error("n must be at least 5 (states are padded to 5 qubits)");
    return QW_ERR_INVALID_ARG;
  }
  if (n > QW_NOALLOC_MAX_QUBITS) {
    set_last_error("n must be at most " + std::to_string(QW_NOALLOC_MAX_QUBITS) +
                   " for the non-allocating energy's scratch array");
    return QW_ERR_BUDGET;
  }
  if (n_terms > QW_NOALLOC_MAX_TERMS) {
    set_last_error("at most " + std::to_string(QW_NOALLOC_MAX_TERMS) +
                   " terms fit the non-allocating energy's scratch array");
    return QW_ERR_BUDGET;
  }
  const uint64_t mask = (1ull << n) - 1;
  for (uint64_t k = 0; k < n_terms; k++)
    if ((terms[k].xmask | terms[k].zmask) & ~mask) {
      set_last_error("a term acts outside the register");
      return QW_ERR_INVALID_ARG;
    }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_last_error("no current CUDA device");
    return QW_ERR_CUDA;
  }
  NaScratch *S = nullptr;
  qw_status st = scratch_address(dev, &S);
  if (st != QW_OK) return st;

  NaHeader h;  // built on the host stack, handed to the device as a kernel parameter
  uint32_t n_classes = 0, n_blocks = 0, chunk_bits = 0;
  layout_fixed(terms, (uint32_t)n_terms, n, h, &n_classes, &n_blocks, &chunk_bits);
  h.job.state = state;
  h.job.out = out;
  h.job.n = n;
  h.job.chunk_bits = chunk_bits;
  h.job.class_begin = 0;
  h.job.n_classes = n_classes;
  h.job.block_begin = 0;
  h.job.n_blocks = n_blocks;
  // every partial is written by its block before the reduction reads it, so
  // nothing in the array needs clearing between calls
  cudaStream_t s = (cudaStream_t)stream;
  char *base = (char *)S;  // device address: offsets only, never dereferenced here
  EnJob *d_job = (EnJob *)(base + offsetof(NaScratch, h) + offsetof(NaHeader, job));
  EnClass *d_classes = (EnClass *)(base + offsetof(NaScratch, h) + offsetof(NaHeader, classes));
  EnTerm *d_terms = (EnTerm *)(base + offsetof(NaScratch, h) + offsetof(NaHeader, terms));
  double *d_partials = (double *)(base + offsetof(NaScratch, partials));
  const size_t hdr = offsetof(NaHeader, terms) + sizeof(EnTerm) * (size_t)n_terms;
  na_setup_kernel<<<1, 256, 0, s>>>(h, (NaHeader *)(base + offsetof(NaScratch, h)), (uint32_t)(hdr / 4));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("layout copy failed: ") + cudaGetErrorString(e));
    return QW_ERR_CUDA;
  }
  launch_energy(mode == QW_MODE_SV_FP64, d_job, 1, n_blocks, d_classes, d_terms, d_partials, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("energy launch failed: ") + cudaGetErrorString(e));
    return QW_ERR_CUDA;
  }
  return QW_OK;
}

// Dense blocks on the host: greedy fusion of a gate list into blocks of at
// most 5 qubits, the blocks' unitaries (products of the gate matrices in
// double precision), and the device program that applies them in order.
#include <algorithm>
#include <cmath>

#include "dense.h"
#include "plan.h"

namespace qw {

using cd = std::complex<double>;

bool gate_matrix_1q(const qw_gate &g, double m[8], bool *diagonal);
bool is_two_qubit_op(uint32_t op);
bool is_barrier_op(uint32_t op);

#define DCK(x)                                                                              \
  do {                                                                                      \
    cudaError_t e_ = (x);                                                                   \
    if (e_ != cudaSuccess)                                                                  \
      fail(e_ == cudaErrorMemoryAllocation ? QW_ERR_OOM : QW_ERR_CUDA, "%s: %s", #x,       \
           cudaGetErrorString(e_));                                                         \
  } while (0)

// U <- G U for gate g acting on block-local bits a (and b for 2-qubit gates).
static void left_multiply(std::vector<cd> &U, uint32_t dim, const qw_gate &g, uint32_t a, uint32_t b) {
  const uint32_t ma = 1u << a, mb = 1u << b;
  auto rows = [&](uint32_t i, uint32_t j, const cd m[4]) {
    for (uint32_t c = 0; c < dim; c++) {
      const cd x = U[i * dim + c], y = U[j * dim + c];
      U[i * dim + c] = m[0] * x + m[1] * y;
      U[j * dim + c] = m[2] * x + m[3] * y;
    }
  };
  if (!is_two_qubit_op(g.op)) {
    double m8[8];
    if (!gate_matrix_1q(g, m8, nullptr)) fail(QW_ERR_INVALID_ARG, "gate op %u has no matrix", g.op);
    const cd m[4] = {{m8[0], m8[1]}, {m8[2], m8[3]}, {m8[4], m8[5]}, {m8[6], m8[7]}};
    for (uint32_t i = 0; i < dim; i++)
      if (!(i & ma)) rows(i, i | ma, m);
    return;
  }
  switch (g.op) {
    case QW_OP_CNOT:  // control a, target b
      for (uint32_t i = 0; i < dim; i++)
        if ((i & ma) && !(i & mb))
          for (uint32_t c = 0; c < dim; c++) std::swap(U[i * dim + c], U[(i | mb) * dim + c]);
      break;
    case QW_OP_CZ:
      for (uint32_t i = 0; i < dim; i++)
        if ((i & ma) && (i & mb))
          for (uint32_t c = 0; c < dim; c++) U[i * dim + c] = -U[i * dim + c];
      break;
    case QW_OP_CPHASE: {
      const cd ph = std::polar(1.0, g.theta);
      for (uint32_t i = 0; i < dim; i++)
        if ((i & ma) && (i & mb))
          for (uint32_t c = 0; c < dim; c++) U[i * dim + c] *= ph;
      break;
    }
    case QW_OP_SWAP:
      for (uint32_t i = 0; i < dim; i++)
        if ((i & ma) && !(i & mb))
          for (uint32_t c = 0; c < dim; c++) std::swap(U[i * dim + c], U[((i & ~ma) | mb) * dim + c]);
      break;
    default:
      fail(QW_ERR_INVALID_ARG, "gate op %u has no matrix", g.op);
  }
}

static DenseBlock make_block(const qw_gate *gates, uint32_t mask, const std::vector<uint64_t> &gi) {
  DenseBlock b;
  uint32_t local[32] = {};
  for (uint32_t q = 0; q < 32; q++)
    if (mask >> q & 1) {
      local[q] = b.k;
      b.q[b.k++] = q;
    }
  const uint32_t dim = 1u << b.k;
  b.u.assign((size_t)dim * dim, 0.0);
  for (uint32_t i = 0; i < dim; i++) b.u[i * dim + i] = 1.0;
  for (uint64_t i : gi) {
    const qw_gate &g = gates[i];
    left_multiply(b.u, dim, g, local[g.q0], is_two_qubit_op(g.op) ? local[g.q1] : 0);
  }
  b.n_gates = (uint32_t)gi.size();
  return b;
}

std::vector<DenseBlock> fuse_dense(const qw_gate *gates, uint64_t n_gates, uint32_t kmax) {
  if (kmax < 2 || kmax > DENSE_MAX_QUBITS) fail(QW_ERR_INVALID_ARG, "kmax must be in [2, %u]", DENSE_MAX_QUBITS);
  struct Open {
    uint32_t mask;
    std::vector<uint64_t> gi;
  };
  std::vector<Open> open;  // pairwise disjoint qubit sets
  std::vector<DenseBlock> out;
  auto close = [&](size_t b) {
    out.push_back(make_block(gates, open[b].mask, open[b].gi));
    open.erase(open.begin() + (ptrdiff_t)b);
  };
  for (uint64_t i = 0; i < n_gates; i++) {
    const qw_gate &g = gates[i];
    if (is_barrier_op(g.op)) fail(QW_ERR_UNSUPPORTED, "gate %llu: measurement or reset in a dense block", (unsigned long long)i);
    uint32_t qm = 1u << g.q0;
    if (is_two_qubit_op(g.op)) qm |= 1u << g.q1;
    for (;;) {
      uint32_t um = qm;
      for (const Open &o : open)
        if (o.mask & qm) um |= o.mask;
      if ((uint32_t)__builtin_popcount(um) <= kmax) break;
      // close the largest touching block (ties: the oldest) and retry
      size_t best = open.size();
      for (size_t b = 0; b < open.size(); b++)
        if ((open[b].mask & qm) &&
            (best == open.size() || __builtin_popcount(open[b].mask) > __builtin_popcount(open[best].mask)))
          best = b;
      close(best);
    }
    // merge every touching block, in order, and append the gate
    Open m{qm, {}};
    for (size_t b = 0; b < open.size();) {
      if (open[b].mask & qm) {
        m.mask |= open[b].mask;
        m.gi.insert(m.gi.end(), open[b].gi.begin(), open[b].gi.end());
        open.erase(open.begin() + (ptrdiff_t)b);
      } else {
        b++;
      }
    }
    m.gi.push_back(i);
    open.push_back(std::move(m));
  }
  // pack what is left (disjoint blocks commute): first fit, largest first
  std::stable_sort(open.begin(), open.end(), [](const Open &a, const Open &b) {
    return __builtin_popcount(a.mask) > __builtin_popcount(b.mask);
  });
  std::vector<Open> packed;
  for (Open &o : open) {
    bool placed = false;
    for (Open &p : packed)
      if ((uint32_t)__builtin_popcount(p.mask | o.mask) <= kmax) {
        p.mask |= o.mask;
        p.gi.insert(p.gi.end(), o.gi.begin(), o.gi.end());
        placed = true;
        break;
      }
    if (!placed) packed.push_back(std::move(o));
  }
  for (Open &p : packed) out.push_back(make_block(gates, p.mask, p.gi));
  return out;
}

}  // namespace qw

// ---------------------------------------------------------------------------
// device program
// ---------------------------------------------------------------------------
struct qw_dense_prog {
  qw::Engine *eng = nullptr;
  uint32_t mode = 0, n = 0, engine = 0, nacc = 1, kmax = 0;
  double est_ms = 0;  // the autotuner's estimate (0 when not autotuned)
  uint64_t n_gates = 0;
  std::vector<qw::DenseBlock> blocks;  // as applied (padded to 5 qubits on the tensor cores)
  std::vector<uint8_t> engines;        // engine of each block
  void *d_ops = nullptr;               // per block: 8192 floats (tensor) or 2 * 4^k values (CUDA cores)
  std::vector<size_t> op_offset;       // byte offset of each block's operand
  int *d_err = nullptr;
  void *last_stream = nullptr;
};

namespace qw {

qw_dense_prog *dense_prog_create(Engine *E, uint32_t mode, uint32_t n, std::vector<DenseBlock> blocks,
                                 uint64_t n_gates, uint32_t engine, uint32_t nacc,
                                 std::vector<uint8_t> engines = {}) {
  if (engines.empty()) engines.assign(blocks.size(), (uint8_t)engine);
  DCK(cudaSetDevice(E->device));
  std::unique_ptr<qw_dense_prog> p(new qw_dense_prog());
  p->eng = E;
  p->mode = mode;
  p->n = n;
  p->engine = engine;
  p->nacc = nacc;
  p->n_gates = n_gates;
  const bool fp64 = mode == QW_MODE_SV_FP64;
  for (const DenseBlock &b : blocks) p->kmax = std::max(p->kmax, b.k);  // before widening
  std::vector<uint8_t> host;
  for (size_t bi = 0; bi < blocks.size(); bi++) {
    DenseBlock &b = blocks[bi];
    p->op_offset.push_back(host.size());
    if (engines[bi] == QW_DENSE_TENSOR) {
      b = pad_block(b, n);
      host.resize(host.size() + 8192 * sizeof(float));
      dense_tc_operands(b, reinterpret_cast<float *>(host.data() + p->op_offset.back()));
    } else {
      const size_t cnt = 2 * b.u.size();
      const size_t bytes = cnt * (fp64 ? sizeof(double) : sizeof(float));
      host.resize(host.size() + ((bytes + 15) & ~(size_t)15));
      uint8_t *dst = host.data() + p->op_offset.back();
      for (size_t i = 0; i < b.u.size(); i++) {
        if (fp64) {
          reinterpret_cast<double *>(dst)[2 * i] = b.u[i].real();
          reinterpret_cast<double *>(dst)[2 * i + 1] = b.u[i].imag();
        } else {
          reinterpret_cast<float *>(dst)[2 * i] = (float)b.u[i].real();
          reinterpret_cast<float *>(dst)[2 * i + 1] = (float)b.u[i].imag();
        }
      }
    }
  }
  p->blocks = std::move(blocks);
  p->engines = std::move(engines);
  DCK(cudaMalloc(&p->d_err, sizeof(int)));
  DCK(cudaMemset(p->d_err, 0, sizeof(int)));
  if (!host.empty()) {
    DCK(cudaMalloc(&p->d_ops, host.size()));
    DCK(cudaMemcpy(p->d_ops, host.data(), host.size(), cudaMemcpyHostToDevice));
  }
  return p.release();
}

void dense_prog_run(qw_dense_prog *p, void *state, void *stream) {
  DCK(cudaSetDevice(p->eng->device));
  cudaStream_t s = (cudaStream_t)stream;
  for (size_t i = 0; i < p->blocks.size(); i++) {
    const uint8_t *op = static_cast<const uint8_t *>(p->d_ops) + p->op_offset[i];
    if (p->engines[i] == QW_DENSE_TENSOR)
      launch_dense_tc((float2 *)state, p->n, p->blocks[i], reinterpret_cast<const float *>(op), (int)p->nacc,
                      p->d_err, p->eng->sm_count, s);
    else
      launch_dense_simt(p->mode == QW_MODE_SV_FP64, state, p->n, p->blocks[i], op, p->eng->sm_count, s);
  }
  DCK(cudaGetLastError());
  p->last_stream = stream;
}

qw_status dense_prog_check(qw_dense_prog *p) {
  DCK(cudaSetDevice(p->eng->device));
  DCK(cudaStreamSynchronize((cudaStream_t)p->last_stream));
  int err = 0;
  DCK(cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    DCK(cudaMemset(p->d_err, 0, sizeof(int)));
    fail(QW_ERR_DEVICE_TIMEOUT, "a tensor-core wait of a dense block ran out; the state is undefined");
  }
  return QW_OK;
}

// ---------------------------------------------------------------------------
// fusion-width / engine autotuner
// ---------------------------------------------------------------------------

// Device time of one block pass (engine, k qubits, staged or direct layout)
// on a 2^n state, measured once per engine and cached: a block of identity
// on the k highest qubits (direct) or on qubits 0..k-1 (staged), three runs,
// the best of the last two.
static double block_pass_ms(Engine *E, uint32_t mode, uint32_t n, uint32_t engine, uint32_t k, bool staged) {
  const uint64_t key = ((uint64_t)n << 16) | ((uint64_t)mode << 12) | ((uint64_t)engine << 8) | ((uint64_t)k << 1) |
                       (staged ? 1u : 0u);
  auto it = E->dense_ms.find(key);
  if (it != E->dense_ms.end()) return it->second;
  DCK(cudaSetDevice(E->device));
  cudaStream_t s = (cudaStream_t)E->stream;
  DenseBlock b;
  b.k = k;
  for (uint32_t j = 0; j < k; j++) b.q[j] = staged ? j : n - k + j;
  const uint32_t d = 1u << k;
  b.u.assign((size_t)d * d, 0.0);
  for (uint32_t i = 0; i < d; i++) b.u[i * d + i] = 1.0;
  const bool fp64 = mode == QW_MODE_SV_FP64;
  const size_t state_bytes = ((size_t)1 << n) * (fp64 ? 16 : 8);
  std::vector<float> ops;
  std::vector<double> u64;
  std::vector<float> u32;
  if (engine == QW_DENSE_TENSOR) {
    b = pad_block(b, n);
    ops.resize(8192);
    dense_tc_operands(b, ops.data());
  } else {
    for (const auto &z : b.u) {
      u64.push_back(z.real());
      u64.push_back(z.imag());
      u32.push_back((float)z.real());
      u32.push_back((float)z.imag());
    }
  }
  void *state = nullptr, *dops = nullptr;
  int *derr = nullptr;
  DCK(cudaMalloc(&state, state_bytes));
  const size_t op_bytes = engine == QW_DENSE_TENSOR ? ops.size() * 4 : (fp64 ? u64.size() * 8 : u32.size() * 4);
  DCK(cudaMalloc(&dops, op_bytes));
  DCK(cudaMalloc(&derr, sizeof(int)));
  DCK(cudaMemsetAsync(state, 0, state_bytes, s));
  DCK(cudaMemsetAsync(derr, 0, sizeof(int), s));
  const void *src = engine == QW_DENSE_TENSOR ? (const void *)ops.data() : fp64 ? (const void *)u64.data() : (const void *)u32.data();
  DCK(cudaMemcpyAsync(dops, src, op_bytes, cudaMemcpyHostToDevice, s));
  cudaEvent_t e0, e1;
  DCK(cudaEventCreate(&e0));
  DCK(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int r = 0; r < 3; r++) {
    DCK(cudaEventRecord(e0, s));
    if (engine == QW_DENSE_TENSOR)
      launch_dense_tc((float2 *)state, n, b, (const float *)dops, 4, derr, E->sm_count, s);
    else
      launch_dense_simt(fp64, state, n, b, dops, E->sm_count, s);
    DCK(cudaEventRecord(e1, s));
    DCK(cudaEventSynchronize(e1));
    float ms;
    DCK(cudaEventElapsedTime(&ms, e0, e1));
    if (r) best = std::min(best, ms);
  }
  int err = 0;
  DCK(cudaMemcpy(&err, derr, sizeof(int), cudaMemcpyDeviceToHost));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(state);
  cudaFree(dops);
  cudaFree(derr);
  if (err) fail(QW_ERR_DEVICE_TIMEOUT, "a tensor-core wait ran out while timing a dense block");
  E->dense_ms[key] = best;
  return best;
}

// Measured pass time of block b on the tensor cores (widened to 5 qubits,
// in the layout the launch will pick: staged when >= 4 of qubits 0-4 are
// block qubits) or on the CUDA cores.
static double block_ms(Engine *E, uint32_t mode, uint32_t n, uint32_t engine, const DenseBlock &b) {
  if (engine == QW_DENSE_TENSOR) {
    uint32_t low = 0;
    for (uint32_t j = 0; j < b.k; j++) low += b.q[j] < 5;
    return block_pass_ms(E, mode, n, engine, 5, low >= 4);
  }
  return block_pass_ms(E, mode, n, engine, b.k, false);
}

// Estimated device time of `blocks` and the engine of each: `engine` for
// all of them, or with QW_DENSE_AUTO the tensor cores for blocks of >= 4
// qubits when they measure faster there, the CUDA cores otherwise.
static double program_ms(Engine *E, uint32_t mode, uint32_t n, uint32_t engine, const std::vector<DenseBlock> &blocks,
                         std::vector<uint8_t> *engines) {
  const bool tc_ok = mode == QW_MODE_SV_FP32 && n >= DENSE_TC_MIN_QUBITS;
  double t = 0;
  engines->clear();
  for (const DenseBlock &b : blocks) {
    uint32_t e = engine;
    double tb;
    if (engine == QW_DENSE_AUTO) {
      e = QW_DENSE_SIMT;
      tb = block_ms(E, mode, n, QW_DENSE_SIMT, b);
      if (tc_ok && b.k >= 4) {
        const double tt = block_ms(E, mode, n, QW_DENSE_TENSOR, b);
        if (tt < tb) {
          tb = tt;
          e = QW_DENSE_TENSOR;
        }
      }
    } else {
      tb = block_ms(E, mode, n, engine, b);
    }
    engines->push_back((uint8_t)e);
    t += tb;
  }
  return t;
}

qw_dense_prog *dense_prog_autotune(Engine *E, uint32_t mode, uint32_t n, const qw_gate *gates, uint64_t n_gates,
                                   uint32_t kmax, uint32_t engine) {
  double best = 1e300;
  uint32_t bk = 0;
  std::vector<DenseBlock> bb;
  std::vector<uint8_t> be;
  for (uint32_t k = 2; k <= DENSE_MAX_QUBITS; k++) {
    if (kmax && k != kmax) continue;
    std::vector<DenseBlock> blocks = fuse_dense(gates, n_gates, k);
    std::vector<uint8_t> engines;
    const double t = program_ms(E, mode, n, engine, blocks, &engines);
    if (t < best) {
      best = t;
      bk = k;
      bb = std::move(blocks);
      be = std::move(engines);
    }
  }
  if (best >= 1e300) fail(QW_ERR_UNSUPPORTED, "no dense engine runs this state");
  uint32_t used = 0;
  for (uint8_t e : be) used |= 1u << e;
  const uint32_t pe = used == (1u << QW_DENSE_TENSOR) ? QW_DENSE_TENSOR
                      : used == (1u << QW_DENSE_SIMT) ? QW_DENSE_SIMT : QW_DENSE_AUTO;
  qw_dense_prog *p = dense_prog_create(E, mode, n, std::move(bb), n_gates, pe, 4, std::move(be));
  p->kmax = bk;
  p->est_ms = best;
  return p;
}

void dense_prog_config(const qw_dense_prog *p, uint32_t *engine, uint32_t *kmax, uint32_t *nacc, double *est_ms) {
  if (engine) *engine = p->engine;
  if (kmax) *kmax = p->kmax;
  if (nacc) *nacc = p->nacc;
  if (est_ms) *est_ms = p->est_ms;
}

uint64_t dense_prog_blocks(const qw_dense_prog *p) { return p->blocks.size(); }
uint64_t dense_prog_gates(const qw_dense_prog *p) { return p->n_gates; }

void dense_prog_destroy(qw_dense_prog *p) {
  if (!p) return;
  cudaSetDevice(p->eng->device);
  cudaStreamSynchronize((cudaStream_t)p->last_stream);
  cudaFree(p->d_ops);
  cudaFree(p->d_err);
  delete p;
}

}  // namespace qw

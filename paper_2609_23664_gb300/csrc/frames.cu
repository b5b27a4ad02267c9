// Pauli-frame propagation for stabilizer tasks that share a Clifford
// reference and differ only by Pauli gates (the QEC family with injected
// data errors).  The reference runs once on the tableau from the shared
// boundary; this kernel propagates every task's Pauli frame through the
// reference circuit, 32 tasks per 32-bit word, one warp per word, and emits
// the tasks' outcomes as reference outcome XOR frame.  This is the frame
// simulation of the stabilizer simulator the paper cites (gidney2021stim);
// the paper itself runs each task's suffix on the tableau.
#include <cuda_runtime.h>

#include <algorithm>

#include "qw_internal.h"

namespace qw {

FrameHostProgram compile_frames(const qw_gate *ref, uint64_t n_ref, uint32_t n,
                                const std::vector<std::pair<uint64_t, uint32_t>> &events) {
  // merged op list in program order: the events of slot s precede gate s
  struct Op {
    FrameOp op;
    uint32_t q0, q1;  // qubits (q1 == q0 for one-qubit ops)
  };
  std::vector<Op> seq;
  seq.reserve(n_ref + events.size());
  size_t e = 0;
  uint32_t n_outs = 0;
  for (uint64_t i = 0; i <= n_ref; i++) {
    for (; e < events.size() && events[e].first == i; e++) {
      Op o{};
      o.op.kind = F_EVENT;
      o.op.a = (uint16_t)events[e].second;
      o.op.aux = (uint32_t)e;
      o.q0 = o.q1 = events[e].second;
      seq.push_back(o);
    }
    if (i == n_ref) break;
    const qw_gate &g = ref[i];
    Op o{};
    o.q0 = o.q1 = g.q0;
    o.op.a = (uint16_t)g.q0;
    switch (g.op) {
      case QW_OP_H: o.op.kind = F_H; break;
      case QW_OP_S:
      case QW_OP_SDG: o.op.kind = F_S; break;
      case QW_OP_CNOT: o.op.kind = F_CX; break;
      case QW_OP_CZ: o.op.kind = F_CZ; break;
      case QW_OP_SWAP: o.op.kind = F_SWAP; break;
      case QW_OP_RESET: o.op.kind = F_RESET; break;
      case QW_OP_MEASURE: o.op.kind = F_MEAS; o.op.aux = n_outs++; break;
      default: fail(QW_ERR_STATE, "internal: non-Clifford or Pauli gate in a frame reference");
    }
    if (g.op == QW_OP_CNOT || g.op == QW_OP_CZ || g.op == QW_OP_SWAP) {
      o.q1 = g.q1;
      o.op.b = (uint16_t)g.q1;
    }
    seq.push_back(o);
  }
  // as-soon-as-possible layers over qubit dependencies
  std::vector<uint32_t> ready(n, 0);
  std::vector<uint32_t> layer_of(seq.size());
  uint32_t n_layers = 0;
  for (size_t i = 0; i < seq.size(); i++) {
    const uint32_t l = std::max(ready[seq[i].q0], ready[seq[i].q1]);
    layer_of[i] = l;
    ready[seq[i].q0] = ready[seq[i].q1] = l + 1;
    n_layers = std::max(n_layers, l + 1);
  }
  std::vector<std::vector<FrameOp>> by_layer(n_layers), meas(n_layers);
  for (size_t i = 0; i < seq.size(); i++)
    (seq[i].op.kind == F_MEAS ? meas : by_layer)[layer_of[i]].push_back(seq[i].op);
  FrameHostProgram P;
  for (uint32_t l = 0; l < n_layers; l++) {
    FrameLayer L{};
    L.op_begin = (uint32_t)P.ops.size();
    P.ops.insert(P.ops.end(), by_layer[l].begin(), by_layer[l].end());
    P.ops.insert(P.ops.end(), meas[l].begin(), meas[l].end());
    L.n_ops = (uint32_t)(by_layer[l].size() + meas[l].size());
    L.n_meas = (uint32_t)meas[l].size();
    P.layers.push_back(L);
  }
  return P;
}

constexpr int FR_WARPS = 4;

// One warp per word of 32 tasks; the word's frame (X and Z bit-planes, one
// 32-bit word per qubit) lives in shared memory.  Within a layer the ops act
// on distinct qubits, so the lanes take them in parallel; the layer's
// measurements are then written lane-per-task.
__global__ void __launch_bounds__(FR_WARPS * 32) frame_kernel(FrameArgs A) {
  extern __shared__ uint32_t fsm[];
  if (*A.rand_any != 0u) return;  // a random reference outcome: the tableau launch runs instead
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t w = blockIdx.x * FR_WARPS + warp;
  if (w >= A.n_words) return;  // whole warps only; no block-wide barrier below
  uint32_t *X = fsm + (size_t)warp * 2 * A.n, *Z = X + A.n;
  for (uint32_t q = lane; q < A.n; q += 32) X[q] = Z[q] = 0u;
  const uint32_t t = w * 32 + lane;  // this lane's task in the measurement phase
  const bool has_task = t < A.n_tasks;
  const uint32_t ob = has_task ? A.out_base[t] : 0u;
  __syncwarp();
  FrameLayer Ln = A.n_layers ? A.layers[0] : FrameLayer{};
  for (uint32_t l = 0; l < A.n_layers; l++) {
    const FrameLayer L = Ln;
    if (l + 1 < A.n_layers) Ln = A.layers[l + 1];  // in flight during this layer
    const uint32_t n_gate = L.n_ops - L.n_meas;
    // the ops of a layer act on distinct qubits, so their order is free: a
    // lane loads four ops before applying them (four loads in flight)
    for (uint32_t i0 = lane; i0 < n_gate; i0 += 128) {
      FrameOp ops[4];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const uint32_t i = i0 + 32u * k;
        ops[k].kind = 0xFF;
        if (i < n_gate) ops[k] = A.ops[L.op_begin + i];
      }
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const FrameOp op = ops[k];
        const uint32_t a = op.a, b = op.b;
        switch (op.kind) {
          case F_H: { const uint32_t x = X[a]; X[a] = Z[a]; Z[a] = x; break; }
          case F_S: Z[a] ^= X[a]; break;
          case F_CX: X[b] ^= X[a]; Z[a] ^= Z[b]; break;
          case F_CZ: Z[a] ^= X[b]; Z[b] ^= X[a]; break;
          case F_SWAP: {
            const uint32_t x = X[a], z = Z[a];
            X[a] = X[b]; Z[a] = Z[b]; X[b] = x; Z[b] = z;
            break;
          }
          case F_RESET: X[a] = 0u; Z[a] = 0u; break;
          case F_EVENT:
            X[a] ^= A.ev_x[(size_t)op.aux * A.n_words + w];
            Z[a] ^= A.ev_z[(size_t)op.aux * A.n_words + w];
            break;
          default: break;
        }
      }
    }
    __syncwarp();
    // measurements, 32 at a time: lane i loads op i of the batch and its
    // reference outcome, then every lane writes its task's outcome of each
    for (uint32_t b0 = n_gate; b0 < L.n_ops; b0 += 32) {
      const uint32_t cnt = min(32u, L.n_ops - b0);
      uint32_t q = 0, aux = 0, ref = 0;
      if (lane < cnt) {
        const FrameOp op = A.ops[L.op_begin + b0 + lane];
        q = op.a;
        aux = op.aux;
        ref = A.ref_out[op.aux];
      }
      for (uint32_t i = 0; i < cnt; i++) {
        const uint32_t qi = __shfl_sync(0xffffffffu, q, i);
        const uint32_t ai = __shfl_sync(0xffffffffu, aux, i);
        const uint32_t ri = __shfl_sync(0xffffffffu, ref, i);
        if (has_task) A.outs[ob + ai] = (uint8_t)(ri ^ ((X[qi] >> lane) & 1u));
      }
    }
    __syncwarp();
  }
}

cudaError_t frame_init_attrs() {
  return cudaFuncSetAttribute((const void *)frame_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(FR_WARPS * 2 * QW_TABLEAU_MAX_QUBITS * sizeof(uint32_t)));
}

void launch_frames(const FrameArgs &a, void *stream) {
  if (a.n_words == 0) return;
  const uint32_t blocks = (a.n_words + FR_WARPS - 1) / FR_WARPS;
  const size_t smem = (size_t)FR_WARPS * 2 * a.n * sizeof(uint32_t);
  frame_kernel<<<blocks, FR_WARPS * 32, smem, (cudaStream_t)stream>>>(a);
}

}  // namespace qw

// Dense k-qubit blocks (k <= 5): fusion of a gate list into blocks on the
// host, and their application to a device statevector, either on the
// tensor cores (tcgen05, FP32 state, 3xTF32 split precision) or on the CUDA
// cores (FP32 or FP64).
//
// A block is a 2^k x 2^k unitary U acting on qubits q[0..k-1]; bit j of the
// block-local index is qubit q[j].  Applying it maps, for every assignment g
// of the n-k other bits, the 2^k amplitudes psi[x(g, p)], p < 2^k, to
// sum_p U[p'][p] psi[x(g, p)].
//
// Tensor-core form: the amplitudes of 128 consecutive groups g form the rows
// of A (128 x 64 real: the 32 real parts, then the 32 imaginary parts), the
// real form of U is B (64 x 64: [[Re U, -Im U], [Im U, Re U]] stored with
// the output index as the row), and D = A B^T are the new amplitudes.  Each
// FP32 operand x is split into TF32 parts hi = tf32(x), lo = tf32(x - hi)
// and D = A_lo B_hi + A_hi B_lo + A_hi B_hi (the lo*lo term, about 2^-22
// relative, is dropped), accumulated in FP32 in tensor memory; with `nacc`
// > 1 the 8 K-steps are spread over nacc accumulators that the CUDA cores
// add in round-to-nearest FP32 (the tensor core's own accumulation rounds
// less accurately).
#pragma once

#include <complex>

#include "qw_internal.h"

namespace qw {

constexpr uint32_t DENSE_MAX_QUBITS = 5;
constexpr uint32_t DENSE_TC_MIN_QUBITS = 12;  // 5 block bits + 7 row bits (128-row tiles)

struct DenseBlock {
  uint32_t k = 0;
  uint32_t q[DENSE_MAX_QUBITS] = {};
  std::vector<std::complex<double>> u;  // 2^k x 2^k, row-major (output, input)
  uint32_t n_gates = 0;
};

// Greedy fusion of unitary gates into blocks of at most kmax qubits: a gate
// joins the open block(s) holding its qubits while their union fits, blocks
// on disjoint qubits merge (they commute), and a gate on qubits held by no
// open block joins any open block with room.  Blocks come out in an order
// that respects every dependency.
std::vector<DenseBlock> fuse_dense(const qw_gate *gates, uint64_t n_gates, uint32_t kmax);

// The block widened to 5 qubits with identity on the highest qubits of the
// register that it does not touch (n >= 5).
DenseBlock pad_block(const DenseBlock &b, uint32_t n);

// Real form of a 5-qubit block split into TF32 hi and lo parts, in the
// shared-memory operand layout of the tensor-core kernel: out[0..4095] hi,
// out[4096..8191] lo.
void dense_tc_operands(const DenseBlock &b5, float *out);

struct DensePos {
  uint32_t v[32];  // v[p] = offset of block-local index p
};

DensePos dense_positions(const DenseBlock &b);
uint32_t dense_other_mask(const DenseBlock &b, uint32_t n);

cudaError_t dense_init_attrs();

// Tensor-core application of a padded 5-qubit block to an FP32 state
// (n >= DENSE_TC_MIN_QUBITS).  bops: device, 8192 floats from
// dense_tc_operands.  nacc in {1, 2, 4}.  err: device int set to 1 when a
// wait for the tensor core ran out (the state is then undefined).
void launch_dense_tc(float2 *state, uint32_t n, const DenseBlock &b5, const float *bops, int nacc, int *err,
                     int sm_count, cudaStream_t s);

// CUDA-core application of a k-qubit block; u: device, 2 * 4^k values of the
// state's precision (interleaved real, imaginary; row-major).
void launch_dense_simt(bool fp64, void *state, uint32_t n, const DenseBlock &b, const void *u, int sm_count,
                       cudaStream_t s);

}  // namespace qw

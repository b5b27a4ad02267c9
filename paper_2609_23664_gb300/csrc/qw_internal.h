// Internal types shared by the translation units of libquwarp.so.
// Nothing here is part of the public ABI (include/quwarp.h is).
#pragma once

#include <cstdarg>
#include <cstdint>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "quwarp.h"

#ifdef __CUDACC__
#define QW_HD __host__ __device__
#else
#define QW_HD
#endif

namespace qw {

// ---------------------------------------------------------------------------
// errors: thrown inside the library, converted to qw_status at the C ABI
// ---------------------------------------------------------------------------
struct Error {
  qw_status code;
  std::string msg;
};
std::string strf(const char *fmt, ...);
[[noreturn]] void fail(qw_status code, const char *fmt, ...);
void set_last_error(const std::string &msg);

// ---------------------------------------------------------------------------
// workload (host)
// ---------------------------------------------------------------------------
struct Span {
  const qw_gate *g;
  uint64_t n;
};

struct TaskData {
  uint32_t mode = 0, n = 0, flags = 0, shots = 0;
  std::vector<Span> spans;
  std::vector<uint64_t> span_end;  // cumulative gate count at the end of each span
  uint64_t n_gates = 0;
  std::vector<qw_pauli_term> terms;
  std::vector<double> uniforms;
  // pointer to gate i (binary search over spans)
  const qw_gate *gate(uint64_t i) const;
  // copies gates [b, e) into `out`
  void copy_gates(uint64_t b, uint64_t e, std::vector<qw_gate> &out) const;
};

struct Workload {
  std::vector<TaskData> tasks;
};

bool is_clifford_op(uint32_t op);
bool is_two_qubit_op(uint32_t op);
bool is_barrier_op(uint32_t op);  // MEASURE / RESET

// ---------------------------------------------------------------------------
// statevector program (host-side fusion result and device descriptors)
// ---------------------------------------------------------------------------
// Operation kinds applied to the register amplitudes of a stage group.
enum SvKind : uint8_t {
  K_U1 = 1,    // general 2x2 on position a: m = {u00r,u00i,u01r,u01i,u10r,u10i,u11r,u11i}
  K_D1 = 2,    // diagonal on a: m = {d0r,d0i,d1r,d1i}
  K_CD = 4,    // multiply amplitudes with bits a and b set by m = {pr, pi}
  K_P1 = 6,    // diag(1, p) on a: m = {pr, pi}
  K_R = 7,     // real 2x2 on a: m = {r00, 0, r01, 0, r10, 0, r11, 0}
  K_RX = 8,    // [[c, -is], [-is, c]] on a: m = {c, s}
  K_RP = 9,    // diag(1, p) after a real 2x2 on a: m = {r00, r01, r10, r11, pr, pi}
};
constexpr int SV_G = 5;            // positions per stage (32 register amplitudes)
// Compensated FP32 passes hold two FP32 complex values per amplitude in
// registers, so their stages take four positions (16 amplitudes)
constexpr int SV_G_COMP = 4;
// Plain FP32 passes take five positions, as FP64 ones (measured on GB300:
// four positions in 256-thread CTAs, 24 warps per SM at 80 registers, ran
// the 24-qubit plain suffix in 138 ms against 115 ms, the extra stage
// passes through shared memory costing more than the occupancy gained)
constexpr int SV_G_PLAIN32 = 5;

// Dense index of an op for the kernels' jump table: each one-position kind
// takes SV_G consecutive slots (its stage position), the controlled phase
// the ten position pairs a < b.
constexpr uint32_t SV_N_OP_INDEX = 40;
__host__ __device__ constexpr uint32_t sv_op_index(uint32_t kind, uint32_t a, uint32_t b) {
  return kind == K_U1   ? a
         : kind == K_D1 ? 5 + a
         : kind == K_P1 ? 10 + a
         : kind == K_R  ? 15 + a
         : kind == K_RX ? 20 + a
         : kind == K_CD ? 25 + a * (9 - a) / 2 + (b - a - 1)
         : kind == K_RP ? 35 + a
                        : SV_N_OP_INDEX;
}
constexpr int SV_MAX_TILE_FP32 = 14;
constexpr int SV_MAX_TILE_FP64 = 13;
// compensated FP32 passes keep a remainder plane beside the tile (16 bytes
// of shared memory per amplitude), so their tiles stop at 2^13
constexpr int SV_MAX_TILE_FP32_COMP = 13;
// a compensated FP32 task whose program has more passes than this runs as
// its own chain of launches that keeps the remainder (persistent launches
// round at every stage, which suits short suffixes only)
constexpr uint32_t SV_COMP_MAX_BATCH_PASSES = 8;

struct HostOp {
  uint8_t kind, a, b;
  double m[8];
  double x[4] = {0, 0, 0, 0};  // K_RP: r10, r11, pr, pi (exact factors of row 1 of m)
};
// A pass keeps the amplitude of logical tile index l in slot phi(l) of its
// tile, phi(l) = M l ^ c over GF(2) (before the shared-memory swizzle):
// permutation gates update phi instead of moving amplitudes.  phi is the
// identity when the tile is loaded.
// A CNOT whose control qubit lies outside the tile is an X on its target
// in the tiles whose control bit is set: it adds a per-tile term to c, the
// XOR of ctl_w[i] over the outside control qubits ctl_q[i] set in the tile.
constexpr int SV_MAX_OUT_CTL = 4;  // outside control qubits per pass
struct HostStage {
  uint8_t pos[SV_G] = {0, 1, 2, 3, 4};  // local tile bit positions (distinct)
  uint32_t mcol[32];  // phi at the start of the stage: column t = M e_t
  uint32_t mc = 0;    // and its constant c
  uint32_t ctl_w[SV_MAX_OUT_CTL] = {0, 0, 0, 0};  // per-tile terms of c (pass's ctl_q)
  std::vector<HostOp> ops;
  // global phase the stage applies to every amplitude (compensated stages
  // with a rotation on every position carry the program's, in their phase
  // table)
  double gphase[2] = {1.0, 0.0};
  HostStage() { for (uint32_t t = 0; t < 32; t++) mcol[t] = 1u << t; }
};
struct HostPass {
  std::vector<uint32_t> q;  // local bit -> global qubit (ascending; q[i] = i for i < b)
  uint32_t b = 0;           // contiguous low qubits
  std::vector<HostStage> stages;
  uint32_t mcol[32];        // phi after the last stage (the tile is stored through it)
  uint32_t mc = 0;
  uint32_t ctl_w[SV_MAX_OUT_CTL] = {0, 0, 0, 0};
  std::vector<uint32_t> ctl_q;  // outside control qubits (global), at most SV_MAX_OUT_CTL
  uint32_t n_gates = 0;     // gates of the source list absorbed by this pass
  HostPass() { for (uint32_t t = 0; t < 32; t++) mcol[t] = 1u << t; }
};
struct SvProgram {
  uint32_t n = 0;  // effective qubit count (>= SV_G)
  uint32_t g = SV_G;  // positions per stage (SV_G, or SV_G_COMP for compensated FP32)
  std::vector<HostPass> passes;
  uint64_t n_gates = 0;
};

struct TileConfig {
  uint32_t k_max = 13;  // tile qubits
  uint32_t b = 4;       // contiguous low qubits in every tile
  uint32_t g = SV_G;    // positions per stage
  // measured time of one pass of the autotuning circuits with this tile
  // shape and arithmetic on one state, pass by pass (ns, launch included);
  // 0 = not measured
  double pass_ns = 0;
};

// Shared-memory swizzle of a tile (amplitude index -> slot).  It XORs bits
// of the index above the 16-byte unit into the unit index inside a 128-byte
// row, so strided stage accesses spread over the banks, and it keeps every
// 16-byte unit (two FP32 amplitudes / one FP64 amplitude) contiguous, so the
// tile can be filled with 16-byte asynchronous copies.  It is linear over
// GF(2): swz(a ^ b) = swz(a) ^ swz(b).
__host__ __device__ inline uint32_t sv_swz32(uint32_t l) {
  return l ^ ((((l >> 4) ^ (l >> 7) ^ (l >> 10) ^ (l >> 13)) & 7u) << 1);
}
__host__ __device__ inline uint32_t sv_swz64(uint32_t l) {
  return l ^ (((l >> 3) ^ (l >> 6) ^ (l >> 9) ^ (l >> 12)) & 7u);
}
constexpr int SV_MAX_GBITS = SV_MAX_TILE_FP32 - SV_G;  // group bits of a stage

// Device descriptors (plain structs, identical layout on host and device).
// Byte offsets below are offsets into the swizzled tile.
struct SvPassDesc {
  uint32_t k, b, n_stages, stage_begin;
  // phi_pair: byte offset of the FP32 pair partner; phi_unit16: every
  // 16-byte unit's amplitudes sit in one 16-byte aligned slot pair
  uint32_t n_hi, phi_ident, phi_pair, phi_unit16;
  uint8_t hi_pos[32];     // global positions of the n-k non-tile bits, ascending
  uint32_t lo_tab[64];    // deposit of local bits b..b+5   (index = lh & 63)
  uint32_t hi_tab[32];    // deposit of local bits b+6..    (index = lh >> 6)
  // store through phi (unless phi_ident): byte offset of the slot of
  // 16-byte unit u = st_lo[u & 63] ^ st_hi[u >> 6]
  uint32_t st_lo[64];
  uint32_t st_hi[128];
  // per-tile terms of the final map's constant: XOR ctl_w[i] when bit
  // ctl_tb[i] of the tile index is set (ctl_w[i] = 0: unused)
  uint32_t ctl_tb[SV_MAX_OUT_CTL], ctl_w[SV_MAX_OUT_CTL];
};
struct alignas(16) SvStageDesc {
  uint32_t roff[SV_G];           // byte offset of phi(e_pos[j]) for register bit j
  uint32_t gcol[SV_MAX_GBITS];   // byte offsets of the group bits (zero past the tile's)
  uint32_t cst;                  // byte offset of the constant of phi
  uint32_t n_ops, op_begin;
  // nonzero: the stage's ops are K_RP ops on the positions of this mask,
  // one per position in ascending order (run without dispatch)
  uint32_t rp_mask;
  // compensated FP32 stage with a K_RP op on every position: block of the
  // phase table (16 entries) holding, for each amplitude index e of the
  // stage group, the product of the |1>-phases of e's set positions (times
  // the program's global phase when bit 31 is set: then entry 0 applies
  // too); 0xFFFFFFFF = none
  uint32_t ph_block;
  uint32_t pad;
  // per-tile terms of cst: XOR ctl_w[i] when bit ctl_tb[i] of the tile index is set
  uint32_t ctl_tb[SV_MAX_OUT_CTL], ctl_w[SV_MAX_OUT_CTL];
};
static_assert(sizeof(SvStageDesc) == 112, "stage descriptor read as seven 16-byte words");
template <typename T>
struct alignas(16) SvOpDesc {
  T m[8];         // read as 16-byte vectors
  uint32_t code;  // sv_op_index(kind, a, b)
};
static_assert(sizeof(SvOpDesc<float>) == 48 && sizeof(SvOpDesc<double>) == 80, "op descriptor layout");

// Fusion planner: gates -> passes -> stages (host).
SvProgram fuse_sv(const qw_gate *gates, uint64_t n_gates, uint32_t n_eff, const TileConfig &tc);
// Number of passes a segment would take (cheap estimate used by the planner).
uint32_t estimate_passes(uint64_t n_gates, uint32_t n, const TileConfig &tc, double gates_per_pass);
// Gate matrix in double precision (host). Returns false for non-1q ops.
bool gate_matrix_1q(const qw_gate &g, double m[8], bool *diagonal);

// ---------------------------------------------------------------------------
// energy descriptors
// ---------------------------------------------------------------------------
struct EnTerm {
  uint32_t xm, zm, skip, flags;  // flags bit0: imaginary component of conj(p)*a
  double coef;                   // c_k * sign(i^{#Y}) * (2 if xm != 0)
};
static_assert(sizeof(EnTerm) == 24, "EnTerm is read as two 8-byte words and a double");
struct EnClass {
  uint32_t term_begin, term_end;
  uint32_t hb;           // highest bit of the class's flip pattern, 0xFFFFFFFF for class 0
  uint32_t n_own;        // own chunks
  uint32_t block_begin;  // first block of this class within its Hamiltonian layout
  uint32_t pad;
};
struct EnJob {
  const void *state;
  double *out;                     // {energy, norm2}
  uint32_t n, chunk_bits;
  uint32_t class_begin, n_classes;
  uint32_t block_begin, n_blocks;  // global block range of this job
};
constexpr int EN_THREADS = 256;
constexpr int EN_BLOCK_BITS = 12;  // amplitudes per block: EN_THREADS x 16

// ---------------------------------------------------------------------------
// sampling descriptors
// ---------------------------------------------------------------------------
constexpr int SMP_BLOCK_BITS = 12;  // 4096 amplitudes per CDF block
struct SmpSource {
  const void *state;
  uint32_t n, n_blocks;
  uint32_t block_begin;  // offset into the block-sum / block-offset arrays
  uint32_t pad;
};
struct SmpShot {
  double u;
  uint32_t source;
  uint32_t pad;
  uint64_t *out;
};
// Hamiltonian layout: classes of terms grouped by the flip-pattern bits above
// the chunk size, so that one class touches pairs of chunks only.  Chunks
// hold at most EN_CHUNK_BYTES of amplitudes of amp_bytes each.
constexpr uint64_t EN_CHUNK_BYTES = 32ull << 20;
void build_energy_layout(const qw_pauli_term *terms, uint64_t n_terms, uint32_t n, uint32_t amp_bytes,
                         uint32_t *chunk_bits, std::vector<EnClass> &classes,
                         std::vector<EnTerm> &en_terms, uint32_t *n_blocks);

// ---------------------------------------------------------------------------
// tableau program (inverse-tableau formulation)
// ---------------------------------------------------------------------------
enum TabKind : uint8_t { T_PROD = 1, T_SWAP2 = 2, T_SIGN = 3, T_MEAS = 4 };
struct TabSlot {
  uint8_t kind;
  uint8_t flags;     // T_PROD: extra phase exponent (mod 4); T_MEAS: bit0 = reset
  uint16_t dst, s1, s2;
  uint32_t aux;      // T_MEAS: random-bit index (segment relative)
  uint32_t aux2;     // T_MEAS: outcome index (segment relative) or 0xFFFFFFFF
};
static_assert(sizeof(TabSlot) == 16, "slot layout");
struct TabLayer {
  uint32_t slot_begin, n_slots, is_measure, pad;
};
struct TabProgram {
  uint32_t layer_begin, n_layers, n_bits, n_outs;
};
struct TabSegment {
  uint32_t prog, bit_base, out_base, pad;
};
struct TabTaskDesc {
  uint32_t seg_begin, n_segs;
  uint32_t bits_base;   // into the byte array of random bits
  uint32_t out_base;    // into the outcome byte array
};
struct TabHostProgram {
  std::vector<TabLayer> layers;
  std::vector<TabSlot> slots;
  uint32_t n_bits = 0, n_outs = 0;
};
// compiles a Clifford gate run (n qubits) into layers of independent row ops
TabHostProgram compile_tab(const qw_gate *gates, uint64_t n_gates, uint32_t n);
// forward stabilizer generators S_i = C Z_i C^-1 of a kept inverse tableau
// (2n rows of 2W words, 2n sign bytes): x, z n*n bytes (row i = S_i), s n
// bytes, S_i = (-1)^s i^{popc(x & z)} X^x Z^z
void stabilizers_from_inverse(uint32_t n, const uint64_t *rows, const uint8_t *sign, uint8_t *x, uint8_t *z,
                              uint8_t *s);

// ---------------------------------------------------------------------------
// kernel launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
struct SvTables {
  const SvPassDesc *passes = nullptr;
  const SvStageDesc *stages = nullptr;
  const void *ops = nullptr;       // SvOpDesc<T>*
  const float *ops_lo = nullptr;   // FP32: m[t] - (float)m[t] of every op, 8 floats per op (compensated passes)
  // compensated FP32: phase products per stage block, 16 entries of
  // {re, re - (float)re, im, im - (float)im} (see SvStageDesc::ph_block)
  const float *ph = nullptr;
};
// Arithmetic of FP32 statevector passes.  PLAIN: FP32 registers.  COMP:
// double-float registers (every op exact to about 2^-48), the amplitude
// rounded to FP32 when its stage writes it back.  REM: double-float
// through the whole pass (a remainder plane beside the shared-memory tile)
// and between passes (remainder arrays beside the state), so a chain of
// passes rounds once, when it writes a state without its remainder.
enum SvArith : int { SV_AR_PLAIN = 0, SV_AR_COMP = 1, SV_AR_REM = 2 };
// stage positions of a pass kernel with arithmetic `ar` (FP64 passes are plain)
QW_HD constexpr int sv_stage_width(int ar, bool fp64 = false) {
  return fp64 ? SV_G : (ar == SV_AR_PLAIN ? SV_G_PLAIN32 : SV_G_COMP);
}
// largest tile of those passes (a stage's group bits are at most SV_MAX_GBITS)
QW_HD constexpr int sv_max_tile(int ar, bool fp64) {
  return fp64 ? SV_MAX_TILE_FP64 : (sv_stage_width(ar, fp64) == 4 ? SV_MAX_TILE_FP32_COMP : SV_MAX_TILE_FP32);
}
// A job of the persistent launch: one pass over one state (n_tiles tiles),
// or the energy blocks of one state (kind SVJ_ENERGY, n_tiles blocks).
enum SvJobKind : uint32_t { SVJ_PASS = 0, SVJ_ENERGY = 1 };
struct SvJob {
  const void *src;   // NULL: start from |0...0>
  void *dst;
  uint32_t pass;     // SVJ_PASS: index into the pass table; SVJ_ENERGY: index of the EnJob
  uint32_t n_tiles;  // work units
  int32_t dep;       // job that must finish first, -1 none
  uint32_t kind;     // SvJobKind
  uint32_t n;        // effective qubits
  uint32_t pad;
};
// The work list of a persistent launch is cut into segments of 2^seg_bits
// items; segment i holds units [first, first + 2^seg_bits) of job `job`
// (units past the job's end are empty items).
struct SvSeg {
  uint32_t job, first;
};
struct EnTables {
  const EnJob *jobs;
  const EnClass *classes;
  const EnTerm *terms;
  double *partials;
};

// kernel attributes (dynamic shared memory limits); the first failure is returned
cudaError_t sv_init_attrs();
cudaError_t tab_init_attrs();
int sv_threads_for_k(uint32_t k, int ar = SV_AR_PLAIN, bool fp64 = false);
size_t sv_smem_bytes(bool fp64, uint32_t k, int ar = SV_AR_PLAIN);
// one pass over one state (grid = tiles); ar applies to FP32 states; the
// remainder arrays (float2 per amplitude, NULL allowed) to SV_AR_REM only
void launch_sv_pass(bool fp64, const SvTables &t, uint32_t pass_idx, uint32_t k, uint32_t n,
                    const void *src, void *dst, void *stream, int ar = SV_AR_PLAIN,
                    const void *src_lo = nullptr, void *dst_lo = nullptr);
// persistent batch over jobs; counters: [0] = next item, [1] = error flag,
// [2..] = per-job completed units (all zeroed by the caller beforehand).
// Energy jobs need 128-thread CTAs (sv_threads_for_k(k_max) == 128).  ar:
// SV_AR_PLAIN or SV_AR_COMP (FP32 states; SV_AR_REM is taken as PLAIN).
void launch_sv_batch(bool fp64, const SvTables &t, const SvJob *jobs, const SvSeg *segs, uint32_t seg_bits,
                     uint32_t total_items, uint32_t k_max, unsigned int *counters, const EnTables &en,
                     int grid, void *stream, int ar = SV_AR_PLAIN);
int sv_batch_grid(bool fp64, uint32_t k, int sm_count, int ar = SV_AR_PLAIN);
void launch_copy(const void *src, void *dst, size_t bytes, void *stream);

// energy: per-block partials (2 doubles per block), then one reduction
// kernel writes {energy, norm2} of every job
void launch_energy(bool fp64, const EnJob *jobs, uint32_t n_jobs, uint32_t total_blocks,
                   const EnClass *classes, const EnTerm *terms, double *partials, void *stream);
// the reduction alone, for partials written by the persistent launch
void launch_energy_reduce(const EnJob *jobs, uint32_t n_jobs, const double *partials, void *stream);
// sampling: block sums -> per-source sequential offsets -> shots
void launch_sampling(bool fp64, const SmpSource *srcs, uint32_t n_src, uint32_t total_blocks,
                     double *bsum, int32_t *blast, double *boff, int64_t *lastnz,
                     const SmpShot *shots, uint32_t n_shots, void *stream);

// tableau
struct TabArgs {
  uint32_t n, W, lpp, rows;
  const uint64_t *init_rows;   // boundary tableau (NULL = identity)
  const uint8_t *init_sign;
  uint64_t *out_rows;          // written back when non-NULL (boundary producer)
  uint8_t *out_sign;
  const TabTaskDesc *tasks;
  const TabSegment *segs;
  const TabProgram *progs;
  const TabLayer *layers;
  const TabSlot *slots;
  const uint8_t *bits;
  uint8_t *outs;
  uint32_t *rand_any;          // when non-NULL: set to 1 if any outcome was random, else 0
  const uint32_t *run_if;      // when non-NULL: the launch does nothing unless *run_if != 0
};
size_t tab_smem_bytes(uint32_t n);
void launch_tab(const TabArgs &a, uint32_t n_tasks, void *stream);

// Pauli frames (stabilizer tasks that differ from a shared reference only
// by Pauli gates): the reference is run once on the tableau; every task's
// deviation is a Pauli frame F, propagated through the reference's Clifford
// gates 32 tasks per 32-bit word.  A Z measurement of the task returns the
// reference outcome XOR the X bit of F on the measured qubit, which is exact
// when the reference outcome is deterministic (F|psi> has the same
// stabilizers up to sign).
enum FrameKind : uint8_t {
  F_H = 1,      // swap X, Z
  F_S = 2,      // Z ^= X  (S and S^dagger)
  F_CX = 3,     // X_b ^= X_a, Z_a ^= Z_b  (control a, target b)
  F_CZ = 4,     // Z_a ^= X_b, Z_b ^= X_a
  F_SWAP = 5,
  F_RESET = 6,  // X = Z = 0
  F_EVENT = 7,  // X ^= ev_x[aux], Z ^= ev_z[aux]  (the tasks' own Pauli gates)
  F_MEAS = 8,   // outcome aux = reference outcome aux XOR X
};
struct FrameOp {
  uint8_t kind, pad;
  uint16_t a, b, pad2;
  uint32_t aux;
};
struct FrameLayer {
  uint32_t op_begin, n_ops;  // ops on distinct qubits; F_MEAS ops last
  uint32_t n_meas, pad;
};
struct FrameHostProgram {
  std::vector<FrameLayer> layers;
  std::vector<FrameOp> ops;
};
// Builds the frame program of a reference gate list with Pauli events
// inserted: events[i] = (slot, qubit) means "before reference gate slot";
// event i becomes F_EVENT with aux = i.  Layers follow qubit dependencies.
FrameHostProgram compile_frames(const qw_gate *ref, uint64_t n_ref, uint32_t n,
                                const std::vector<std::pair<uint64_t, uint32_t>> &events);
struct FrameArgs {
  uint32_t n, n_tasks, n_words, n_layers;
  const FrameLayer *layers;
  const FrameOp *ops;
  const uint32_t *ev_x, *ev_z;  // [event * n_words + word]
  const uint8_t *ref_out;       // reference outcomes
  const uint32_t *rand_any;     // nonzero: some reference outcome was random; frames do not apply
  const uint32_t *out_base;     // per task of the group: first suffix outcome in outs
  uint8_t *outs;
};
cudaError_t frame_init_attrs();
void launch_frames(const FrameArgs &a, void *stream);

// tableau -> statevector export (n <= QW_SV_MAX_QUBITS): echelon stabilizer
// basis of the state, then one pass writing every amplitude
struct StabBasis {
  uint32_t n, k, err, pad;  // err != 0: the tableau did not describe a valid state
  uint64_t x0;              // a basis state in the support
  uint64_t gx[QW_SV_MAX_QUBITS], gz[QW_SV_MAX_QUBITS];  // echelon generators i^ge X^gx Z^gz
  uint32_t ge[QW_SV_MAX_QUBITS];
  uint8_t piv[QW_SV_MAX_QUBITS];                        // pivot bit of each generator
};
// tableau: 2n rows of (x, z) words followed by 2n sign bytes (n <= 30)
void launch_stab_export(const void *tableau, uint32_t n, StabBasis *basis, bool fp64, uint32_t n_eff, void *dst,
                        int sm_count, void *stream);

// learned cost model
void launch_mlp_forward(const float *params, const float *x, float *y, uint32_t batch, void *stream);
void launch_mlp_loss_grad(const float *params, const float *x, const float *target, uint32_t batch,
                          float *loss, float *grad, float *scratch, void *stream);
void launch_mlp_adam(float *params, const float *grad, float *m, float *v, uint32_t n, uint32_t t,
                     float lr, float b1, float b2, float eps, void *stream);
size_t mlp_scratch_floats(uint32_t batch);
}  // namespace qw

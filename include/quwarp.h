/*
 * quwarp.h -- C ABI of the GB300 reuse engine (libquwarp.so, sm_103a).
 *
 * The engine executes a WORKLOAD of related circuit-simulation tasks the way
 * the paper's reuse planner does (Sec. III-A "Architecture Flow", Fig. 2):
 * tasks are submitted, grouped by shared gate prefixes, planned with the
 * materialize-versus-recompute rule (Sec. IV-C, Eq. 2), executed (the shared
 * prefix once, its boundary state kept in device memory, every task's suffix
 * resumed from it), and their results plus an EXPLAIN trace and a cost record
 * are read back (Sec. III-A "Outputs and audit artifacts").
 *
 * Conventions for every entry point:
 *  - The return value is a qw_status: QW_OK (0) or a negative error code.
 *    No C++ exception crosses this boundary.  After an error,
 *    qw_last_error() returns a message for the calling thread.
 *  - A planner decision to ABSTAIN or REFUSE is not an error; it is visible
 *    in the EXPLAIN trace and the task falls back to a from-scratch rerun.
 *  - Host buffers passed in are only read during the call and stay owned by
 *    the caller; inputs are copied, except gate spans (qw_gate_span), which
 *    are referenced until the workload is destroyed.  Output buffers are
 *    caller-owned.
 *  - Objects returned through `out` pointers are owned by the caller and
 *    released with the matching *_destroy function.  The engine owns all
 *    device memory it allocates (boundary store, task buffers, result arrays)
 *    and frees it in qw_plan_destroy / qw_engine_destroy.
 *  - Entry points whose name ends in _dev take device pointers (allocated by
 *    the caller, e.g. through PyTorch) and a CUDA stream (NULL = legacy
 *    default stream); they enqueue work and return without synchronizing.
 *  - Qubit q is bit q of the basis-state index (little endian).
 *  - A workload, plan or engine object must not be used from two threads at
 *    the same time.
 */
#ifndef QUWARP_H
#define QUWARP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t qw_status;
enum {
  QW_OK = 0,
  QW_ERR_INVALID_ARG = -1,      /* malformed task / gate / size / pointer   */
  QW_ERR_OOM = -2,              /* host or device allocation failed         */
  QW_ERR_BUDGET = -3,           /* request exceeds a configured budget      */
  QW_ERR_CUDA = -4,             /* a CUDA runtime call failed               */
  QW_ERR_DEVICE_TIMEOUT = -5,   /* a bounded device-side wait expired       */
  QW_ERR_STATE = -6,            /* call made in the wrong order             */
  QW_ERR_BUFFER_TOO_SMALL = -7, /* output capacity too small (see *needed)  */
  QW_ERR_NOT_FOUND = -8,        /* unknown task id / result not requested   */
  QW_ERR_UNSUPPORTED = -9       /* valid request the library does not run   */
};

/* ---- input records (byte layout is part of the ABI) ---------------------- */

/* Gate operations.  Rotations: RX/RY/RZ(t) = exp(-i t P/2); PHASE(t) =
 * diag(1, e^{it}); CPHASE(t) multiplies |11> by e^{it}; CNOT(q0 control,
 * q1 target).  MEASURE / RESET (tableau mode only) measure Z on q0; the
 * `theta` field holds the outcome bit (0.0 or 1.0) taken when the state does
 * not determine the outcome.  RESET = measure, then X if the outcome was 1;
 * its outcome is not reported. */
enum {
  QW_OP_H = 1, QW_OP_X = 2, QW_OP_Y = 3, QW_OP_Z = 4, QW_OP_S = 5, QW_OP_SDG = 6,
  QW_OP_T = 7, QW_OP_TDG = 8, QW_OP_RX = 9, QW_OP_RY = 10, QW_OP_RZ = 11,
  QW_OP_PHASE = 12,
  QW_OP_CNOT = 20, QW_OP_CZ = 21, QW_OP_SWAP = 22, QW_OP_CPHASE = 23,
  QW_OP_MEASURE = 30, QW_OP_RESET = 31
};
enum { QW_GATE_CHECKPOINT = 1 }; /* user checkpoint after this gate (Sec. IV-A) */

typedef struct qw_gate {         /* 24 bytes */
  uint32_t op;
  uint32_t q0;
  uint32_t q1;                   /* second qubit of 2-qubit gates, else 0   */
  uint32_t flags;                /* QW_GATE_*                               */
  double theta;                  /* angle, or outcome bit of MEASURE/RESET  */
} qw_gate;

/* Pauli term c * P with P|x> = i^{#Y} (-1)^{popc(x & zmask)} |x ^ xmask>;
 * qubit q: X <-> x=1,z=0; Z <-> x=0,z=1; Y <-> x=1,z=1.  24 bytes. */
typedef struct qw_pauli_term {
  double coef;
  uint64_t xmask;
  uint64_t zmask;
} qw_pauli_term;

/* Simulation modes = the paper's two backend families (Sec. V-B): full
 * statevector (FP64 or FP32 amplitudes) and stabilizer tableau. */
enum { QW_MODE_SV_FP64 = 0, QW_MODE_SV_FP32 = 1, QW_MODE_TABLEAU = 2 };

enum { QW_TASK_KEEP_STATE = 1 }; /* keep the final state for qw_get_state */

/* A run of gate records in caller memory.  Spans are REFERENCED, not copied:
 * the gates must stay valid and unchanged until qw_workload_destroy.  Tasks
 * that share a prefix may (and for large workloads should) pass the same
 * span; the prefix trie then recognizes the shared run without comparing it
 * record by record. */
typedef struct qw_gate_span {
  const qw_gate *gates;
  uint64_t n_gates;
} qw_gate_span;

/* One task of a workload (Sec. IV-A "Workload IR"): its gate list is the
 * concatenation of spans[0..n_spans-1].
 *  SV modes: n_qubits in [1, QW_SV_MAX_QUBITS]; gates from {H..CPHASE};
 *  optional energy of sum_k terms[k] (n_terms > 0; masks must fit in
 *  n_qubits bits); optional `shots` computational-basis samples drawn with
 *  the caller's uniforms in [0,1) (uniforms[0..shots-1]).
 *  TABLEAU mode: n_qubits in [1, QW_TABLEAU_MAX_QUBITS]; Clifford gates
 *  {H,X,Y,Z,S,SDG,CNOT,CZ,SWAP,MEASURE,RESET}; the result is the outcome bit
 *  of every MEASURE, in order.
 * The spans array, terms and uniforms are copied by qw_workload_add_task. */
typedef struct qw_task {
  uint32_t mode;
  uint32_t n_qubits;
  const qw_gate_span *spans;
  uint32_t n_spans;
  uint32_t flags;                /* QW_TASK_* */
  const qw_pauli_term *terms;
  uint64_t n_terms;
  const double *uniforms;
  uint32_t shots;
  uint32_t reserved;
} qw_task;

#define QW_SV_MAX_QUBITS 30
#define QW_TABLEAU_MAX_QUBITS 640

/* ---- engine ---------------------------------------------------------------- */

typedef struct qw_engine qw_engine;

typedef struct qw_engine_opts {
  int32_t device;                /* CUDA device ordinal                       */
  uint32_t reserved;
  uint64_t store_budget_bytes;   /* boundary-store budget; 0 = 40% of free   */
  uint64_t task_budget_bytes;    /* task-buffer budget; 0 = 40% of free      */
  double hbm_gbs;                /* bandwidth used by the analytic cost model;
                                    0 = measure once at creation             */
} qw_engine_opts;

/* Creates an engine on `opts->device` (NULL opts = defaults on device 0).
 * Owns the device memory it allocates and its internal streams.  Destroying
 * an engine also releases the device memory of the plans created on it;
 * those plans keep their host results and EXPLAIN trace, but qw_execute and
 * qw_get_state on them return QW_ERR_STATE. */
qw_status qw_engine_create(const qw_engine_opts *opts, qw_engine **out);
void qw_engine_destroy(qw_engine *e);
/* Measured/assumed bandwidth (GB/s) and SM count the cost model uses. */
qw_status qw_engine_info(const qw_engine *e, double *hbm_gbs, int32_t *sm_count,
                         uint64_t *l2_bytes);
/* Measures the L2 read bandwidth (GB/s) for the access pattern of the
 * energy step: independent 64 KB blocks of an L2-resident buffer (half the
 * L2, at most 64 MB) in hashed order, 16 loads of 16 bytes in flight per
 * thread.  The energy of random Pauli strings reads each term's partner
 * amplitudes from L2 (Sec. V workload families: repeated expectation
 * evaluation), so this, not the HBM bandwidth, bounds it.  Synchronous;
 * allocates and frees its buffer. */
qw_status qw_engine_probe_l2(qw_engine *e, double *l2_read_gbs);
/* Tile-shape tuning (the autotuner of the statevector passes: tile qubits,
 * contiguous low qubits, stage width, and pass_ns, the measured time of one
 * pass on one state that calibrates the analytic cost of Eq. 2), kept per
 * (qubit count, precision, FP32 arithmetic, gate mix) and measured on first
 * use.  Shapes are compared in the persistent suffix launch with several
 * states advanced together, as a wave's tasks are.  The gate mix is "layered" (at most 35 %
 * two-qubit gates: hardware-efficient circuits of 1-4 layers) or
 * "entangling" (more: a random circuit), each tuned on circuits of its kind.
 * _json writes
 * the engine's tuning as JSON (size-query idiom, as qw_explain_json), with
 * the GPU model it was measured on and the number of shapes this engine
 * timed itself; _load adds the entries of such a record to an engine on the
 * same GPU model, so a later process plans without timing them again.
 * QW_ERR_INVALID_ARG for another model, a record of another kind, a
 * malformed entry or a shape the pass kernels cannot run; a refused record
 * adds nothing (all entries or none).  Not thread-safe against planning on
 * the same engine. */
qw_status qw_engine_tuning_json(const qw_engine *e, char *buf, size_t cap, size_t *needed);
qw_status qw_engine_tuning_load(qw_engine *e, const char *json);

/* Message of the last error on the calling thread ("" if none).  Valid until
 * the next qw_* call on this thread. */
const char *qw_last_error(void);

/* ---- workload (host only) --------------------------------------------------- */

typedef struct qw_workload qw_workload;

qw_status qw_workload_create(qw_workload **out);
/* Adds a task (span list, terms and uniforms are copied; gate memory is
 * referenced) and returns its id (0, 1, 2, ... in submission order).
 * Validates every gate, qubit index, mask and size. */
qw_status qw_workload_add_task(qw_workload *w, const qw_task *t, uint64_t *task_id);
void qw_workload_destroy(qw_workload *w);

/* ---- planning (host only; Sec. IV, Eq. 1, Eq. 2, Table II) ------------------ */

enum { QW_COST_ANALYTIC = 0, QW_COST_MLP = 1 };

typedef struct qw_plan_opts {
  int32_t reuse;              /* 1 = plan reuse; 0 = per-task rerun (Sec. V-E baseline 2) */
  int32_t batched;            /* 1 = all suffixes in one persistent launch; 0 = per task  */
  int32_t legality;           /* 1 = legality guard (Sec. IV-B); 0 = disabled (unsafe ablation) */
  int32_t cost_model;         /* QW_COST_ANALYTIC or QW_COST_MLP                     */
  double delta_frac;          /* safety margin delta = delta_frac * direct cost (Eq. 2) */
  uint32_t min_group;         /* early filter: tasks sharing a prefix (Sec. IV-A)   */
  uint32_t min_prefix_gates;  /* early filter: prefix length                        */
  double min_prefix_cost_ns;  /* early filter: estimated prefix cost                */
  uint32_t tile_qubits;       /* 0 = autotuned; else statevector tile size (qubits) */
  uint32_t low_qubits;        /* 0 = autotuned; contiguous low qubits in every tile */
  uint32_t window;            /* 0 = autotuned; tasks interleaved in the batch order */
  int32_t use_graph;          /* 1 = capture execution in a CUDA graph              */
  int32_t fault_injection;    /* test only, default 0.  1 = the first tile of the
                                 persistent suffix launch waits on a dependency that
                                 never completes: its bounded wait runs out, the
                                 launch ends early and qw_wait reports
                                 QW_ERR_DEVICE_TIMEOUT (results are then invalid;
                                 the device stays usable). */
  int32_t fuse_energy;        /* 1 = the energy blocks of every task run as work items of
                                 the persistent suffix launch (same results, one launch);
                                 0 = a separate energy launch after it.  Default 0. */
  int32_t pauli_frames;       /* 1 = stabilizer tasks on one boundary whose suffixes differ
                                 only by Pauli gates run the shared reference once on the
                                 tableau and the tasks as Pauli frames (same outcomes; the
                                 per-task tableau runs instead when a reference outcome is
                                 random); 0 = every task on its own tableau.  Default 1. */
  int32_t handoff;            /* 1 = statevector tasks (n <= QW_SV_MAX_QUBITS) may continue
                                 from a tableau boundary exported to a statevector (Table II
                                 STAB -> SV), and an all-Clifford shared prefix may be run on
                                 the tableau for them when Eq. 2 estimates it cheaper; the
                                 exported state's global phase is fixed by a positive real
                                 amplitude on the first basis state of its support.
                                 0 = never.  Default 1. */
  int32_t prefix_fp64;        /* 1 = a shared prefix of FP32 statevector tasks (up to 28
                                 qubits) is evolved in FP64 and rounded once to FP32 for
                                 them: the boundary's error then does not grow with the
                                 prefix length (an FP64 artifact is exact for an FP32
                                 consumer up to that one rounding), at the cost of FP64
                                 arithmetic for the prefix.  0 = the prefix runs in FP32.
                                 Default 0. */
  int32_t dense_boundaries;   /* statevector boundaries as fused dense blocks (see the
                                 dense block section below): 1 = at the first execution,
                                 each boundary's pass program and its autotuned dense
                                 program (tensor cores for 4-5-qubit blocks) are timed
                                 once on a scratch state and the faster one evolves it;
                                 2 = always the dense program; 0 = pass kernels only.
                                 Boundaries continuing from another precision keep the
                                 pass kernels.  The choices are in the cost record.
                                 Default 0. */
  int32_t fp32_arith;         /* gate arithmetic of FP32 statevector tasks (storage stays
                                 FP32 either way):
                                 QW_FP32_AUTO (default): compensated when some FP32
                                 task of the workload has Pauli terms (its energy is
                                 held to 1e-6 relative), plain otherwise (states and
                                 samples need 1e-5 max-abs amplitude error, which plain
                                 FP32 meets).
                                 QW_FP32_COMPENSATED: every amplitude is held
                                 as an unevaluated sum of two FP32 numbers while gates
                                 run (error-free products and sums on the FP32 units,
                                 gate constants to 2^-48), so a state is rounded only
                                 when it is stored: the passes of a boundary keep their
                                 FP32 remainder in a second array and round once, into
                                 the boundary; a task's suffix passes round at each
                                 stage of a pass; per-task launches (batched = 0) keep
                                 the remainder like a boundary.
                                 QW_FP32_PLAIN: FP32 arithmetic (faster; its rounding
                                 through long circuits moves energies by about 1e-6 of
                                 their size at 24 qubits). */
} qw_plan_opts;

#define QW_FP32_AUTO 0
#define QW_FP32_PLAIN 1
#define QW_FP32_COMPENSATED 2

/* Fills the defaults: reuse=1, batched=1, legality=1, analytic costs,
 * delta_frac=0.10, min_group=2, min_prefix_gates=1, min_prefix_cost_ns=0,
 * autotuned tiles, use_graph=1, fault_injection=0, fuse_energy=0, pauli_frames=1,
 * handoff=1, prefix_fp64=0, dense_boundaries=0, fp32_arith=QW_FP32_AUTO. */
void qw_plan_opts_default(qw_plan_opts *o);

typedef struct qw_plan qw_plan;

/* Builds the plan for workload `w`: prefix trie over gate records, at most
 * three candidate cut points per shared prefix, fingerprints (Eq. 1),
 * legality (Table II), the reuse inequality (Eq. 2), EXPLAIN records.  Host
 * only.  `e` supplies the bandwidth/SM figures and the learned cost model;
 * it may be NULL for host-only planning with nominal figures (such a plan
 * can be inspected but not executed).  The workload may be destroyed after
 * this call. */
qw_status qw_plan_create(qw_engine *e, const qw_workload *w, const qw_plan_opts *o,
                         qw_plan **out);
void qw_plan_destroy(qw_plan *p);

/* Executes the plan on its engine.  The first call allocates device buffers,
 * uploads the compiled programs and (use_graph=1) captures the launch
 * sequence in a CUDA graph; later calls replay it.  Asynchronous on `stream`
 * (a cudaStream_t; NULL = the engine's stream).  Call qw_wait before reading
 * results. */
qw_status qw_execute(qw_plan *p, void *stream);
/* Waits for the last qw_execute, copies results to the host, checks device
 * error flags (QW_ERR_DEVICE_TIMEOUT if a bounded wait expired). */
qw_status qw_wait(qw_plan *p);

/* ---- results ------------------------------------------------------------------ */

/* Energy sum_k c_k <P_k> / <psi|psi> and <psi|psi> of an SV task. */
qw_status qw_get_energy(const qw_plan *p, uint64_t task, double *energy, double *norm2);
/* Samples of an SV task (basis-state indices); *n = shots. */
qw_status qw_get_samples(const qw_plan *p, uint64_t task, uint64_t *out, size_t cap, size_t *n);
/* Outcome bits (one byte each, 0/1) of every MEASURE of a tableau task. */
qw_status qw_get_syndrome(const qw_plan *p, uint64_t task, uint8_t *bits, size_t cap,
                          size_t *n_bits);
/* Final amplitudes of an SV task submitted with QW_TASK_KEEP_STATE:
 * 2^n complex numbers as interleaved (re, im) doubles (FP64 mode) or floats
 * (FP32 mode); `bytes` must equal that size. */
qw_status qw_get_state(const qw_plan *p, uint64_t task, void *host_dst, size_t bytes);
/* Final state of a tableau task submitted with QW_TASK_KEEP_STATE, as the
 * stabilizer generators of the state (the STAB artifacts of Table II are
 * stabilizer tableaus; Sec. IV-B): generator i (i < n) is
 *   S_i = (-1)^sign[i] i^{popc(x_i & z_i)} X^{x_i} Z^{z_i},
 * x and z row-major, n bytes per generator (one byte per qubit, 0/1), the
 * image of Z_i under the task's circuit (measurements and resets included).
 * They generate the task's stabilizer group; its canonical form (reduced
 * row echelon over (x | z) with signs) equals the oracle's for the same
 * circuit.  x, z: host, n_qubits * n_qubits bytes; sign: host, n_qubits
 * bytes.  QW_ERR_NOT_FOUND without QW_TASK_KEEP_STATE (such a task never
 * runs as a Pauli frame), QW_ERR_INVALID_ARG for a statevector task or a
 * wrong n_qubits, QW_ERR_STATE before qw_execute. */
qw_status qw_get_stabilizers(const qw_plan *p, uint64_t task, uint8_t *x, uint8_t *z, uint8_t *sign,
                             size_t n_qubits);

/* EXPLAIN trace (Sec. III-A; Sec. IV-B refusal record) and realized-cost
 * record (Sec. V-E metrics) as JSON.  Size-query idiom: with cap too small
 * (or buf NULL) the call returns QW_ERR_BUFFER_TOO_SMALL and sets *needed
 * (including the terminating NUL). */
qw_status qw_explain_json(const qw_plan *p, char *buf, size_t cap, size_t *needed);
qw_status qw_cost_record_json(const qw_plan *p, char *buf, size_t cap, size_t *needed);

/* ---- planner primitives (host only; exposed for auditing and tests) ----------- */

/* SHA-256 (FIPS 180-4) of a byte string. */
qw_status qw_sha256(const void *data, size_t len, uint8_t out[32]);
/* Structural fingerprint of a segment, Eq. 1: SHA-256 over the layout record
 * {u32 n_qubits, u32 mode} followed by the `n_gates` 24-byte gate records. */
qw_status qw_fingerprint(uint32_t n_qubits, uint32_t mode, const qw_gate *gates,
                         uint64_t n_gates, uint8_t out[32]);

/* Reuse inequality, Eq. 2:
 *   (N-1) C_prefix > C_materialize + N (C_reload + C_handoff) + delta.
 * *reuse = 1 when it holds (strict), *lhs and *rhs receive both sides. */
typedef struct qw_cost_tuple {
  double n_tasks;
  double c_prefix;
  double c_materialize;
  double c_reload;
  double c_handoff;
  double delta;
} qw_cost_tuple;
qw_status qw_reuse_decision(const qw_cost_tuple *c, int32_t *reuse, double *lhs, double *rhs);

/* Legality guard of Sec. IV-B / Table II.  Artifact kinds, exactness classes
 * and backends as named in the EXPLAIN trace. */
enum { QW_KIND_STATEVECTOR = 0, QW_KIND_TABLEAU = 1 };
enum { QW_EXACT = 0, QW_FORBIDDEN = 1, QW_EXACTNESS_UNKNOWN = 2 };
enum { QW_BACKEND_GPU_SV_FP64 = 0, QW_BACKEND_GPU_SV_FP32 = 1, QW_BACKEND_GPU_TABLEAU = 2,
       QW_BACKEND_UNKNOWN = 3 };
typedef struct qw_artifact_desc {
  uint32_t kind;
  uint32_t exactness;
  uint32_t backend;              /* producing backend family */
  uint32_t n_qubits;
  uint8_t provenance[32];        /* fingerprint of the producing prefix */
} qw_artifact_desc;
typedef struct qw_refusal {
  char reason[48];               /* e.g. FORBIDDEN_CONVERSION; "" if legal    */
  char detail[160];
  char source_kind[40], target_kind[40];
  char source_backend[32], target_backend[32];
} qw_refusal;
/* Three gates in order: exactness validation, backend-family validation,
 * conversion-rule lookup, plus the provenance check (the consumer's own
 * prefix fingerprint must equal the artifact's).  *legal = 1 if the handoff
 * may run; otherwise *legal = 0 and `out` describes the refusal. */
qw_status qw_legality_check(const qw_artifact_desc *a, uint32_t target_backend,
                            const uint8_t expected_provenance[32], int32_t *legal,
                            qw_refusal *out);

/* ---- learned cost model (BF16 MLP 12 -> 64 -> 64 -> 1) --------------------------- */

#define QW_MLP_IN 12
#define QW_MLP_HID 64
#define QW_MLP_PARAMS (QW_MLP_IN * QW_MLP_HID + QW_MLP_HID + QW_MLP_HID * QW_MLP_HID + \
                       QW_MLP_HID + QW_MLP_HID + 1)

/* Parameter vector layout (FP32 master copy): W1[64][12], b1[64],
 * W2[64][64], b2[64], w3[64], b3.  Forward: h1 = relu(W1 x + b1),
 * h2 = relu(W2 h1 + b2), y = w3 . h2 + b3, with weights and inputs rounded to
 * BF16 and FP32 accumulation.  Loss = mean (y - target)^2. */

/* Device primitives (device pointers): forward pass for `batch` feature rows
 * (row-major [batch][12] floats) into y[batch]. */
qw_status qw_mlp_forward_dev(const float *params, const float *x, float *y, uint32_t batch,
                             void *stream);
/* Loss and gradient w.r.t. the FP32 parameters (same layout) for a batch. */
qw_status qw_mlp_loss_grad_dev(const float *params, const float *x, const float *target,
                               uint32_t batch, float *loss, float *grad, void *stream);
/* One Adam step on FP32 master parameters (m, v moment buffers, step t>=1). */
qw_status qw_mlp_adam_dev(float *params, const float *grad, float *m, float *v,
                          uint32_t n_params, uint32_t t, float lr, float beta1,
                          float beta2, float eps, void *stream);

/* Trains the engine's cost model on host arrays (features [n][12], targets
 * [n] = log2 of measured nanoseconds) with the device kernels above; the
 * result becomes the engine's QW_COST_MLP model.  epochs/batch/lr: training
 * schedule; seed: shuffling and initialization.  Final training MSE in
 * *final_loss (nullable). */
qw_status qw_costmodel_train(qw_engine *e, const float *features, const float *targets,
                             uint64_t n, uint32_t epochs, uint32_t batch, float lr,
                             uint64_t seed, float *final_loss);
/* Host-side inference with the engine's current model (launches the forward
 * kernel and waits).  out[n] = predicted log2 ns. */
qw_status qw_costmodel_predict(qw_engine *e, const float *features, uint64_t n, float *out);
/* Reads / replaces the engine's FP32 master parameters (QW_MLP_PARAMS floats);
 * the feature normalization (12 means, 12 scales) travels with them. */
qw_status qw_costmodel_get(const qw_engine *e, float *params, float *feat_mean,
                           float *feat_scale);
qw_status qw_costmodel_set(qw_engine *e, const float *params, const float *feat_mean,
                           const float *feat_scale);
/* Engine-measured timing probe: times the execution of `w`'s tasks segment
 * by segment with CUDA events and appends one row per timed segment to the
 * caller's arrays (capacity cap rows); *n_rows receives the count.  Each row
 * is the 12 features the planner computes for that segment and log2 of the
 * measured nanoseconds; analytic_log2ns (nullable) receives log2 of the
 * analytic model's estimate for the same segment (passes x (2 S / bandwidth
 * + launch overhead)). */
qw_status qw_costmodel_probe(qw_engine *e, const qw_workload *w, float *features,
                             float *targets, float *analytic_log2ns, uint64_t cap,
                             uint64_t *n_rows);
/* Feature vector the planner uses for gates [gate_begin, gate_end) of task
 * `task` of workload `w` executed as one segment shared by n_sharing tasks. */
qw_status qw_costmodel_features(const qw_engine *e, const qw_workload *w, uint64_t task,
                                uint64_t gate_begin, uint64_t gate_end, uint32_t n_sharing,
                                float out[12]);

/* ---- statevector kernels on caller buffers (device pointers) ------------------ */

/* Applies gates[0..n_gates-1] (host array) to the device state `state`
 * (2^n complex amplitudes: double2 for QW_MODE_SV_FP64, float2 for FP32) in
 * place with the fused pass kernels.  A NULL `init` leaves the state as is;
 * init != NULL and *init == 1 first sets |0...0>. */
qw_status qw_sv_apply_dev(qw_engine *e, uint32_t mode, uint32_t n, void *state,
                          const qw_gate *gates, uint64_t n_gates, const int32_t *init,
                          void *stream);
/* Energy sum_k c_k <P_k>/<psi|psi> and <psi|psi> of a device state; results
 * are written to host memory (the call synchronizes `stream`). */
qw_status qw_sv_energy_dev(qw_engine *e, uint32_t mode, uint32_t n, const void *state,
                           const qw_pauli_term *terms, uint64_t n_terms, double *energy,
                           double *norm2, void *stream);
/* `shots` samples of a device state with host uniforms; synchronizes. */
qw_status qw_sv_sample_dev(qw_engine *e, uint32_t mode, uint32_t n, const void *state,
                           const double *uniforms, uint32_t shots, uint64_t *out,
                           void *stream);

/* ---- energy without device allocation --------------------------------------
 * The paper has no counterpart of this entry point; it exists for callers of
 * this library that cannot allocate device memory: programs whose device
 * memory is owned by another allocator (a framework's caching allocator that
 * has reserved the pool), and latency-bound loops with a fixed memory
 * footprint that cannot pay the device synchronization of cudaFree.  It
 * computes what qw_sv_energy_dev computes, with the same kernels, but needs
 * no engine and allocates nothing: the term layout, the job record and the
 * per-block partial sums live in one fixed device array of the library
 * (about 1.2 MB, held by every GPU that loads the library until the process
 * exits).  Its term classes are fixed (chunks of an eighth of the state from
 * 15 qubits on), so its sums run in another order than qw_sv_energy_dev's.
 *   state : device, 2^n amplitudes (double2 for QW_MODE_SV_FP64, float2 for
 *           QW_MODE_SV_FP32), n in [5, QW_NOALLOC_MAX_QUBITS].
 *   terms : host, n_terms <= QW_NOALLOC_MAX_TERMS; masks within n bits.
 *   out   : device, 2 doubles {energy, <psi|psi>}, written asynchronously on
 *           `stream` (a cudaStream_t; NULL = legacy default stream).
 * n < 5, NULL pointers and masks outside the register return
 * QW_ERR_INVALID_ARG; n > QW_NOALLOC_MAX_QUBITS or more terms than
 * QW_NOALLOC_MAX_TERMS return QW_ERR_BUDGET.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress), which loads
 * the module.  Every call
 * uses the same array: calls whose work overlaps on the GPU (different
 * streams, or host threads without ordering) race and corrupt each other's
 * results; serialize them on one stream.  The array keeps the last call's
 * contents; every partial sum is rewritten before it is read, so nothing
 * needs clearing between calls. */
#define QW_NOALLOC_MAX_QUBITS 26
#define QW_NOALLOC_MAX_TERMS 1024
qw_status qw_sv_energy_noalloc_dev(uint32_t mode, uint32_t n, const void *state,
                                   const qw_pauli_term *terms, uint64_t n_terms, double *out,
                                   void *stream);


/* ---- dense blocks: fused k-qubit unitaries ----------------------------------
 * A dense block is a 2^k x 2^k unitary (k in [1, 5]) on qubits q[0..k-1]:
 * bit j of the block-local index is qubit q[j]; for every assignment of the
 * other n-k bits it maps the 2^k amplitudes by the matrix.  A gate list is
 * fused into blocks of at most kmax qubits (greedy: a gate joins the blocks
 * that hold its qubits while their union fits, the largest of them is
 * closed otherwise; disjoint blocks commute and are packed together), each
 * block's matrix being the product of its gates' matrices in double
 * precision.  A program applies its blocks in order, one pass over the state
 * per block.  It is the statevector backend's gate application (Sec. III-A
 * "Execution on the bounded Qrack surface", Sec. V-B "Backend surface") in
 * fused-block form; the paper does not fix how gates are applied, and the
 * pass kernels of qw_sv_apply_dev stay the path that plans use.
 *   QW_DENSE_TENSOR: tcgen05 tensor cores.  FP32 states only, n in
 *     [12, QW_SV_MAX_QUBITS]; each FP32 operand is split into two TF32
 *     parts and three products are accumulated in FP32 (3xTF32); nacc in
 *     {1, 2, 4} spreads the 8 K-steps over that many tensor-memory
 *     accumulators, added on the CUDA cores (more accurate, more readback).
 *     Blocks of fewer than 5 qubits are widened with identity on the
 *     highest qubits they do not touch.
 *   QW_DENSE_SIMT: CUDA cores in the state's precision (FP32 or FP64),
 *     n >= k (nacc ignored).
 * Gates: the unitary ops of qw_gate (MEASURE/RESET -> QW_ERR_UNSUPPORTED). */
#define QW_DENSE_TENSOR 0u
#define QW_DENSE_SIMT 1u
#define QW_DENSE_AUTO 2u  /* qw_dense_prog_create only: the engine of each block is chosen */
typedef struct qw_dense_prog qw_dense_prog;

/* Host only (no engine, no GPU): the pass program that the statevector
 * kernels would run for `gates` on n qubits (5 <= n <= QW_SV_MAX_QUBITS),
 * with tiles of tile_qubits qubits (6..14) of which low_qubits (1 ..
 * tile_qubits - 2) are the contiguous lowest, as a NUL-terminated JSON
 * object written to buf (size-query idiom: *needed = bytes including the
 * NUL; QW_ERR_BUFFER_TOO_SMALL when cap is smaller).  Layout:
 *   {"n", "passes": [{"q": tile bit t -> qubit, "ctl_q": outside control
 *     qubits, "b", "map": final tile map, "stages": [{"pos": 5 tile bits
 *     (register bit j -> tile bit pos[j]), "map": tile map at the stage,
 *     "ops": [{"kind", "a", "b", "m": 8 doubles}]}]}]}
 * A tile map {"cols", "c", "ctl_w"} places the amplitude of logical tile
 * index l in slot (XOR of cols[t] over the set bits t of l) ^ c ^ (XOR of
 * ctl_w[i] over the outside control qubits ctl_q[i] that are 1 in the
 * tile: CNOTs whose control is not a tile qubit).  A stage reads its 32
 * register amplitudes (register index i: bit j of i = logical tile bit
 * pos[j]) through its map, applies its ops in order and writes them back
 * to the same slots; a tile is read in logical order and written back
 * through the pass's final map.  Op kinds act on register positions a (and
 * b), m in the kernels' layout: "U1" 2x2 {u00,u01,u10,u11} (re, im); "D1"
 * diag(d0, d1) in m[0..3]; "P1" diag(1, p), p in m[0..1]; "CD" multiplies
 * the amplitudes with bits a and b set by m[0..1]; "R" real 2x2 in m[0],
 * m[2], m[4], m[6]; "RX" [[c, -is], [-is, c]] with c, s = m[0], m[1]; "RP"
 * the real 2x2 {m0, m1; m2, m3}, then diag(1, m4 + i m5).  For tests and
 * inspection; the engine fuses internally. */
qw_status qw_sv_fuse_json(const qw_gate *gates, uint64_t n_gates, uint32_t n, uint32_t tile_qubits,
                          uint32_t low_qubits, char *buf, size_t cap, size_t *needed);
/* Host only (no engine, no GPU): the blocks a program would apply, before
 * widening.  k[i], qubits[5 i + j] (j < k[i]), u[2048 i ..] = the 32 x 32
 * complex matrix (re, im interleaved, row-major over the 2^k x 2^k block,
 * the rest zero).  With cap = 0 only *n_blocks is written. */
qw_status qw_dense_fuse(const qw_gate *gates, uint64_t n_gates, uint32_t n, uint32_t kmax,
                        uint32_t *k, uint32_t *qubits, double *u, uint64_t cap,
                        uint64_t *n_blocks);
/* Fuses `gates` (host) and uploads the blocks' operands (synchronous).
 * Autotuning: kmax = 0 tries the fusion widths 2..5; engine = QW_DENSE_AUTO
 * picks the engine of every block: the tensor cores for blocks of 4 or 5
 * qubits when they measure faster there (FP32 states with n >= 12 only),
 * the CUDA cores otherwise (always for blocks of 1-3 qubits).  A candidate's
 * time is the sum of its blocks' pass times, measured once per (n,
 * precision, engine, width, layout) on a scratch state of the engine and
 * cached in it; the fastest candidate is built (4 accumulators on the
 * tensor cores).  qw_dense_prog_config reports the choice (engine
 * QW_DENSE_AUTO when the blocks use both). */
qw_status qw_dense_prog_create(qw_engine *e, uint32_t mode, uint32_t n, const qw_gate *gates,
                               uint64_t n_gates, uint32_t kmax, uint32_t engine, uint32_t nacc,
                               qw_dense_prog **out);
/* One explicit block: u = 2^k x 2^k complex doubles (re, im interleaved,
 * row-major, output index first) on qubits[0..k-1] (distinct, < n).  The
 * matrix is used as given (it is not checked for unitarity). */
qw_status qw_dense_prog_create_block(qw_engine *e, uint32_t mode, uint32_t n,
                                     const uint32_t *qubits, uint32_t k, const double *u,
                                     uint32_t engine, uint32_t nacc, qw_dense_prog **out);
qw_status qw_dense_prog_info(const qw_dense_prog *p, uint64_t *n_blocks, uint64_t *n_gates);
/* The program's engine, fusion width (the largest block), accumulators and
 * the autotuner's time estimate in ms (0 when not autotuned).  Any output
 * pointer may be NULL. */
qw_status qw_dense_prog_config(const qw_dense_prog *p, uint32_t *engine, uint32_t *kmax,
                               uint32_t *nacc, double *est_ms);
/* Applies the blocks in place to the device state (2^n float2 or double2)
 * on `stream`, asynchronously. */
qw_status qw_dense_prog_run(qw_dense_prog *p, void *state, void *stream);
/* Synchronizes the last run's stream; QW_ERR_DEVICE_TIMEOUT if a bounded
 * wait for the tensor core ran out (the state is then undefined). */
qw_status qw_dense_prog_check(qw_dense_prog *p);
void qw_dense_prog_destroy(qw_dense_prog *p);

#ifdef __cplusplus
}
#endif
#endif /* QUWARP_H */

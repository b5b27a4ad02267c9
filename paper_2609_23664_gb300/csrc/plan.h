// Planner and engine objects (internal).
#pragma once

#include <map>
#include <string>
#include <vector>

#include "qw_internal.h"

#include <set>
#include <tuple>

struct qw_plan;

struct qw_workload {
  qw::Workload w;
  // spans already validated for (mode, n): shared spans are checked once
  std::set<std::tuple<const qw_gate *, uint64_t, uint32_t, uint32_t>> validated;
};

namespace qw {

// ---- cost model --------------------------------------------------------------
struct CostModel {
  bool trained = false;
  std::vector<float> params;    // QW_MLP_PARAMS FP32 master weights
  float mean[QW_MLP_IN] = {0};
  float scale[QW_MLP_IN] = {0};
  float y_lo = 0, y_hi = 0;     // training-target range (log2 ns)
  float f_lo[QW_MLP_IN] = {0}, f_hi[QW_MLP_IN] = {0};  // training feature range
};

// ---- trie -----------------------------------------------------------------------
struct TNode {
  int parent = -1;
  uint64_t depth = 0;       // gates from the root
  uint32_t rep = 0;         // representative task; edge = rep's gates [edge_begin, depth)
  uint64_t edge_begin = 0;
  uint32_t n = 0;           // qubits of the group
  std::vector<int> kids;
  std::vector<uint32_t> ending;
  uint32_t below = 0;
  uint32_t mode_count[3] = {0, 0, 0};
};

struct Candidate {
  uint64_t cut = 0;   // gate index (absolute) of the boundary
  int kind = 0;       // 0 LCP, 1 Clifford transition, 2 barrier / checkpoint, 3 tableau handoff
  uint32_t n_tasks = 0;
  double c_prefix = 0, c_mat = 0, c_reload = 0, c_handoff = 0, delta = 0, lhs = 0, rhs = 0;
  bool holds = false;
};

struct RefusalRec {
  uint32_t task;
  qw_refusal r;
};

struct Decision {
  int node = -1;
  uint32_t n = 0;
  uint64_t depth = 0;
  uint32_t n_tasks = 0;
  int decision = 0;  // 0 REUSE, 1 ABSTAIN, 2 REFUSE
  std::string reason;
  std::vector<Candidate> cands;
  int chosen = -1;
  int mat = -1;
  double est_direct = 0, est_reuse = 0, est_handoff = -1;  // est_handoff < 0: not applicable
  std::vector<RefusalRec> refusals;
  bool cost_from_mlp = false;
};

struct MatNode {
  int node = -1;
  int parent = -1;          // parent materialized node, -1 = |0...0> / identity
  uint64_t begin = 0, end = 0;  // gate range (of rep task) this node evolves
  uint32_t rep = 0;
  uint32_t mode = 0, n = 0, n_eff = 0;
  uint64_t bytes = 0;
  uint8_t provenance[32];
  // compiled
  SvProgram sv;
  std::vector<std::pair<uint32_t, uint32_t>> tab_segs;  // (program, bit_base)
  uint32_t tab_outs = 0;    // outcomes this segment produces
  uint32_t out_offset = 0;  // cumulative outcomes from the root to the start of this node
  // tableau node exported to statevectors (bit 1 << mode per precision that
  // statevector consumers need; Table II STAB -> SV)
  uint32_t export_modes = 0;
  std::vector<qw_gate> gates;  // the node's gates (kept for dense-block boundaries)
};

// A statevector boundary evolved by a dense-block program instead of passes.
struct DenseChoice {
  int mat = -1;
  uint32_t engine = 0, width = 0, blocks = 0;
  double est_ms = 0, pass_ms = 0, dense_ms = 0;  // timed candidates (option 1), 0 = not timed
  bool used = false;
  bool over_budget = false;  // compensated FP32: more blocks than the accuracy budget allows
};
// Compensated FP32 boundaries take the tensor-core dense form only up to
// this many blocks: each 3xTF32 block perturbs the state by about 1e-7 of
// its norm (FP32 accumulation inside the tensor core), which moves a
// Pauli-sum energy by about 1.4e-7 of its typical size; four such blocks
// (2.8e-7, adding in quadrature) leave room within the 1e-6 energy target,
// where the compensated passes keep a whole prefix near 1e-7
constexpr uint32_t DENSE_COMP_MAX_BLOCKS = 4;

struct TaskPlan {
  uint32_t mode = 0, n = 0, n_eff = 0, flags = 0, shots = 0;
  int src = -1;             // materialized source node, -1 = from scratch
  uint64_t begin = 0;       // first gate executed by the task itself
  uint64_t n_gates = 0;
  bool refused = false;
  bool legality_bypassed = false;  // converted artifact (legality disabled)
  int ham = -1;             // Hamiltonian layout id, -1 = no energy
  std::vector<double> uniforms;
  SvProgram sv;             // suffix program (SV modes)
  std::vector<std::pair<uint32_t, uint32_t>> tab_segs;
  uint32_t tab_outs = 0;    // suffix outcomes
  uint32_t total_outs = 0;  // all MEASURE outcomes of the task
};

// Stabilizer tasks on one boundary whose suffixes agree once Pauli gates
// are removed: the reference runs once, the tasks as Pauli frames.
struct FrameGroup {
  int src = -1;
  uint32_t n = 0;
  std::vector<uint32_t> tasks;                          // task ids, in group order
  std::vector<qw_gate> ref;                             // reference suffix (Pauli gates removed)
  std::vector<std::pair<uint32_t, uint32_t>> ref_segs;  // compiled tableau program (prog, bit base)
  uint32_t n_outs = 0;
  qw::FrameHostProgram prog;
  uint32_t n_events = 0, n_words = 0;
  std::vector<uint32_t> ev_x, ev_z;                     // [event * n_words + word]
};

struct HamLayout {
  uint32_t n_eff = 0, chunk_bits = 0, n_blocks = 0;
  std::vector<EnClass> classes;
  std::vector<EnTerm> terms;
};

struct Engine;
struct DeviceState;  // engine.cu

std::string json_escape(const std::string &s);
std::string hex32(const uint8_t h[32]);
void sha256(const void *data, size_t len, uint8_t out[32]);
// FP32 arithmetic of a plan's persistent suffix launches (SV_AR_COMP or SV_AR_PLAIN)
int plan_ar_batch(const qw_plan *P);
// Gate-mix class of a gate list for the tile autotuner: 0 = layered (at
// most 35 % two-qubit gates, e.g. hardware-efficient layers), 1 = entangling
// (more, e.g. random circuits)
constexpr double GATE_MIX_TWO_QUBIT_SHARE = 0.35;
inline uint32_t gate_mix(uint64_t n_two, uint64_t n_all) {
  return (n_all && (double)n_two > GATE_MIX_TWO_QUBIT_SHARE * (double)n_all) ? 1u : 0u;
}
void fingerprint(uint32_t n, uint32_t mode, const TaskData &t, uint64_t b, uint64_t e, uint8_t out[32]);
bool legality(const qw_artifact_desc &a, uint32_t target_backend, const uint8_t *expected,
              qw_refusal *out);
const char *backend_name(uint32_t b);
const char *kind_name(uint32_t k);
void features_for(const TaskData &t, uint64_t b, uint64_t e, uint32_t n_sharing, const TileConfig &tc,
                  double occupancy, float out[QW_MLP_IN]);

struct Engine {
  int device = 0;
  int sm_count = 0;
  uint64_t l2_bytes = 0;
  double hbm_gbs = 0;
  double launch_ns = 4000;
  uint64_t store_budget = 0, task_budget = 0;
  void *stream = nullptr;
  std::map<uint64_t, TileConfig> tiles;  // key: tile_key(n, fp64, arithmetic, gate mix)
  uint64_t tuning_runs = 0;               // tile shapes timed by this engine (not loaded)
  std::map<uint64_t, double> dense_ms;    // measured dense-block pass times (autotuner cache)
  CostModel cm;
  float *d_mlp = nullptr;  // device copy of the MLP params
  // scratch for the *_dev entry points
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  // Device-memory cache: blocks a plan releases are kept (by size) for the
  // next plans, so planning and executing a workload again allocates and
  // frees nothing; dropped when an allocation fails and on destruction.
  std::multimap<size_t, void *> free_blocks;
  size_t cached_bytes = 0;
  void *dev_alloc(size_t bytes, size_t *got);
  void dev_free(void *p, size_t bytes);
  void trim_cache();
  std::set<qw_plan *> plans;  // live plans (released when the engine is destroyed)
  // autotuned tile shape for FP32 arithmetic `ar` (SV_AR_PLAIN or SV_AR_COMP)
  // and gate mix `mix` (gate_mix of the gates it will run)
  TileConfig tile_config(uint32_t n_eff, bool fp64, int ar, uint32_t mix);
  static uint64_t tile_key(uint32_t n_eff, bool fp64, int ar, uint32_t mix) {
    if (fp64 || ar == SV_AR_REM) ar = SV_AR_PLAIN;
    return ((uint64_t)std::min<uint32_t>(n_eff, 26) << 4) | ((uint64_t)(mix & 1u) << 3) | ((uint64_t)ar << 1) |
           (fp64 ? 1 : 0);
  }
  double predict_log2ns(const float *feat, uint32_t rows, float *out);
  void *ensure_scratch(size_t bytes);
};

}  // namespace qw

struct qw_engine {
  qw::Engine e;
};

struct qw_plan {
  qw::Engine *eng = nullptr;
  qw_plan_opts opts;
  bool fp32_compensated = true;  // FP32 gate arithmetic of this plan (from opts.fp32_arith and the workload)
  std::vector<qw::TaskPlan> tasks;
  std::vector<qw::MatNode> mats;
  std::vector<qw::Decision> decisions;
  std::vector<qw::HamLayout> hams;
  std::vector<qw::TabHostProgram> tab_progs;
  std::vector<uint8_t> tab_bits;  // random bits of every compiled tableau program instance
  std::vector<qw::FrameGroup> frame_groups;
  std::vector<int> task_frame_group;  // per task: frame group, -1 none
  std::string explain, cost;
  double planning_ns = 0;
  double est_direct_ns = 0, est_plan_ns = 0;
  bool fast_path = false;
  uint64_t total_gates = 0;
  // execution
  qw::DeviceState *dev = nullptr;
  bool executed = false;
  // host results
  std::vector<double> energy, norm2;
  std::vector<uint64_t> samples;
  std::vector<uint64_t> sample_off;  // per task offset into samples
  std::vector<uint8_t> outs_suffix;   // per task suffix outcomes
  std::vector<uint32_t> outs_off;
  std::vector<uint8_t> outs_mat;      // per mat node outcomes
  std::vector<uint32_t> outs_mat_off;
  // realized timings (ms) of the last execution
  double t_upload_ms = 0, t_prefix_ms = 0, t_suffix_ms = 0, t_energy_ms = 0, t_sample_ms = 0,
         t_tab_ms = 0, t_total_ms = 0;
  int timed = 0;
  std::vector<double> batch_ms;  // per wave: suffix launch(es) only
  uint64_t n_launches = 0, h2d_bytes = 0, d2h_bytes = 0;
  double batch_alg_bytes = 0, energy_alg_bytes = 0, energy_l2_bytes = 0, prefix_alg_bytes = 0;
  double batch_alg_flops = 0, prefix_alg_flops = 0;  // gate arithmetic of the suffix passes / boundaries
  bool energy_fused = false;  // energy blocks ran inside the persistent suffix launch
  std::vector<std::pair<uint32_t, uint32_t>> wave_tiles;  // (tile qubits, low qubits) per wave
  std::vector<qw::DenseChoice> dense_choices;  // option dense_boundaries
};

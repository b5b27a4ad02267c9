// Engine: device memory, boundary-state store, execution of a plan,
// CUDA-graph capture, autotuning of the tile schedule and the learned cost
// model's training loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <map>
#include <random>

#include "dense.h"
#include "plan.h"

namespace qw {
qw_dense_prog *dense_prog_autotune(Engine *E, uint32_t mode, uint32_t n, const qw_gate *gates, uint64_t n_gates,
                                   uint32_t kmax, uint32_t engine);
void dense_prog_config(const qw_dense_prog *p, uint32_t *engine, uint32_t *kmax, uint32_t *nacc, double *est_ms);
uint64_t dense_prog_blocks(const qw_dense_prog *p);
void dense_prog_run(qw_dense_prog *p, void *state, void *stream);
qw_status dense_prog_check(qw_dense_prog *p);
void dense_prog_destroy(qw_dense_prog *p);

#define CK(x)                                                                       \
  do {                                                                              \
    cudaError_t e_ = (x);                                                           \
    if (e_ != cudaSuccess)                                                          \
      fail(e_ == cudaErrorMemoryAllocation ? QW_ERR_OOM : QW_ERR_CUDA, "%s: %s (%s:%d)", #x, \
           cudaGetErrorString(e_), __FILE__, __LINE__);                             \
  } while (0)

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
// |0...0>: every amplitude 0, the first 1
__global__ void basis_zero_kernel(void *state, bool fp64, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (fp64) ((double2 *)state)[i] = make_double2(i == 0 ? 1.0 : 0.0, 0.0);
    else ((float2 *)state)[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
  }
}

__global__ void convert_kernel(const void *src, bool src64, void *dst, bool dst64, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double re, im;
  if (src64) { const double2 v = ((const double2 *)src)[i]; re = v.x; im = v.y; }
  else { const float2 v = ((const float2 *)src)[i]; re = v.x; im = v.y; }
  if (dst64) ((double2 *)dst)[i] = make_double2(re, im);
  else ((float2 *)dst)[i] = make_float2((float)re, (float)im);
}

void launch_copy(const void *src, void *dst, size_t bytes, void *stream) {
  if (bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// device-side tables of a set of statevector programs
// ---------------------------------------------------------------------------
struct SvTableBuilder {
  std::vector<SvPassDesc> passes;
  std::vector<SvStageDesc> stages;
  std::vector<SvOpDesc<float>> ops32;
  std::vector<float> ops32lo;  // m[t] - (float)m[t] per FP32 op (compensated passes)
  std::vector<float> ph;       // phase products of full rotation-and-phase stages (FP32)
  std::vector<SvOpDesc<double>> ops64;
  bool fp64;
  explicit SvTableBuilder(bool f) : fp64(f) {}
  // appends the program; returns the index of its first pass
  uint32_t add(const SvProgram &pr) {
    const uint32_t first = (uint32_t)passes.size();
    for (const HostPass &hp : pr.passes) {
      SvPassDesc d;
      memset(&d, 0, sizeof(d));
      d.k = (uint32_t)hp.q.size();
      d.b = hp.b;
      d.n_stages = (uint32_t)hp.stages.size();
      d.stage_begin = (uint32_t)stages.size();
      uint32_t inq = 0;
      for (uint32_t q : hp.q) inq |= 1u << q;
      uint32_t nh = 0;
      for (uint32_t q = 0; q < pr.n; q++)
        if (!(inq & (1u << q))) d.hi_pos[nh++] = (uint8_t)q;
      d.n_hi = nh;
      // local bit i (>= b) -> global qubit hp.q[i]
      for (uint32_t v = 0; v < 64; v++) {
        uint32_t g = 0;
        for (uint32_t j = 0; j < 6; j++)
          if ((v >> j) & 1u) { const uint32_t li = d.b + j; if (li < d.k) g |= 1u << hp.q[li]; }
        d.lo_tab[v] = g;
      }
      for (uint32_t v = 0; v < 32; v++) {
        uint32_t g = 0;
        for (uint32_t j = 0; j < 5; j++)
          if ((v >> j) & 1u) { const uint32_t li = d.b + 6 + j; if (li < d.k) g |= 1u << hp.q[li]; }
        d.hi_tab[v] = g;
      }
      // byte offset of the swizzled slot of a (pre-swizzle) tile index
      const uint32_t asz = fp64 ? 16u : 8u;
      auto slot = [&](uint32_t v) { return (fp64 ? sv_swz64(v) : sv_swz32(v)) * asz; };
      auto phi_of = [&](const uint32_t *mcol, uint32_t mc, uint32_t l) {
        uint32_t v = mc;
        for (uint32_t t = 0; t < d.k; t++)
          if ((l >> t) & 1u) v ^= mcol[t];
        return v;
      };
      // every tile map must be a bijection of the k-bit tile index: the
      // kernels address shared memory through it
      auto check_phi = [&](const uint32_t *mcol, uint32_t mc) {
        const uint32_t km = (1u << d.k) - 1u;
        uint32_t basis[32] = {0};
        bool ok = (mc & ~km) == 0;
        for (uint32_t t = 0; t < d.k && ok; t++) {
          uint32_t v = mcol[t];
          if (v & ~km) { ok = false; break; }
          for (int bit = 31; bit >= 0 && v; bit--)
            if ((v >> bit) & 1u) {
              if (!basis[bit]) { basis[bit] = v; break; }
              v ^= basis[bit];
            }
          ok = v != 0;
        }
        if (!ok) fail(QW_ERR_STATE, "internal: tile map of a pass is not a bijection");
      };
      check_phi(hp.mcol, hp.mc);
      for (const HostStage &hs : hp.stages) check_phi(hs.mcol, hs.mc);
      // outside control qubits -> tile-index bits; their per-tile terms
      // must stay inside the tile like every column of the map
      if (hp.ctl_q.size() > (size_t)SV_MAX_OUT_CTL) fail(QW_ERR_STATE, "internal: too many outside controls");
      uint32_t ctl_tb[SV_MAX_OUT_CTL] = {0, 0, 0, 0};
      for (size_t c = 0; c < hp.ctl_q.size(); c++) {
        uint32_t tb = 0xFFFFFFFFu;
        for (uint32_t i = 0; i < d.n_hi; i++)
          if (d.hi_pos[i] == hp.ctl_q[c]) tb = i;
        if (tb == 0xFFFFFFFFu) fail(QW_ERR_STATE, "internal: outside control %u is a tile qubit", hp.ctl_q[c]);
        ctl_tb[c] = tb;
      }
      auto check_ctl = [&](const uint32_t *w) {
        for (int c = 0; c < SV_MAX_OUT_CTL; c++)
          if ((w[c] >> d.k) != 0 || (w[c] != 0 && (size_t)c >= hp.ctl_q.size()))
            fail(QW_ERR_STATE, "internal: per-tile map term outside the tile");
      };
      check_ctl(hp.ctl_w);
      for (const HostStage &hs : hp.stages) check_ctl(hs.ctl_w);
      for (int c = 0; c < SV_MAX_OUT_CTL; c++) {
        d.ctl_tb[c] = ctl_tb[c];
        d.ctl_w[c] = slot(hp.ctl_w[c]);
      }
      {
        bool ident = hp.mc == 0;
        for (uint32_t t = 0; t < d.k; t++) ident = ident && hp.mcol[t] == (1u << t);
        for (int c = 0; c < SV_MAX_OUT_CTL; c++) ident = ident && hp.ctl_w[c] == 0;
        d.phi_ident = ident ? 1u : 0u;
        const uint32_t apu_bits = fp64 ? 0u : 1u;  // amplitudes per 16-byte unit: 2^apu_bits
        for (uint32_t v = 0; v < 64; v++) d.st_lo[v] = slot(phi_of(hp.mcol, hp.mc, v << apu_bits));
        for (uint32_t v = 0; v < 128; v++) d.st_hi[v] = slot(phi_of(hp.mcol, 0, v << (6 + apu_bits)));
        d.phi_pair = fp64 ? 0u : slot(hp.mcol[0]);
        bool unit16 = true;  // FP64: a unit is one amplitude
        if (!fp64) {
          unit16 = d.phi_pair == 8u;
          for (uint32_t v = 0; v < 64 && unit16; v++) unit16 = (d.st_lo[v] & 8u) == 0;
          for (uint32_t v = 0; v < 128 && unit16; v++) unit16 = (d.st_hi[v] & 8u) == 0;
          for (int c = 0; c < SV_MAX_OUT_CTL && unit16; c++) unit16 = (d.ctl_w[c] & 8u) == 0;
        }
        d.phi_unit16 = unit16 ? 1u : 0u;
      }
      for (const HostStage &hs : hp.stages) {
        SvStageDesc sd;
        memset(&sd, 0, sizeof(sd));
        uint32_t pm = 0;
        for (uint32_t j = 0; j < pr.g; j++) {
          sd.roff[j] = slot(hs.mcol[hs.pos[j]]);
          pm |= 1u << hs.pos[j];
        }
        sd.cst = slot(hs.mc);
        for (int c = 0; c < SV_MAX_OUT_CTL; c++) {
          sd.ctl_tb[c] = ctl_tb[c];
          sd.ctl_w[c] = slot(hs.ctl_w[c]);
        }
        // group bits: the first four (the lanes of a half warp) chosen so
        // that their slots differ in the bank bits (slot bits 0-3 of 8-byte
        // FP32 slots, 0-2 of 16-byte FP64 slots), the rest ascending
        std::vector<uint32_t> free_pos;
        for (uint32_t t = 0; t < d.k; t++)
          if (!(pm & (1u << t))) free_pos.push_back(t);
        const uint32_t bank_mask = fp64 ? 7u : 15u;
        std::vector<uint32_t> order, basis;
        std::vector<uint8_t> used(free_pos.size(), 0);
        for (int pick = 0; pick < 4; pick++) {
          int best = -1;
          for (size_t c = 0; c < free_pos.size() && best < 0; c++) {
            if (used[c]) continue;
            uint32_t v = (fp64 ? sv_swz64(hs.mcol[free_pos[c]]) : sv_swz32(hs.mcol[free_pos[c]])) & bank_mask;
            for (uint32_t bv : basis) v = std::min(v, v ^ bv);  // reduce against the echelon basis
            if (v) { best = (int)c; basis.push_back(v); std::sort(basis.rbegin(), basis.rend()); }
          }
          if (best < 0) break;
          used[best] = 1;
          order.push_back(free_pos[best]);
        }
        for (size_t c = 0; c < free_pos.size(); c++)
          if (!used[c]) order.push_back(free_pos[c]);
        if (order.size() > (size_t)SV_MAX_GBITS) fail(QW_ERR_STATE, "internal: tile wider than the stage descriptor");
        for (size_t t = 0; t < order.size(); t++) sd.gcol[t] = slot(hs.mcol[order[t]]);
        // a stage of real rotations (with or without a |1>-phase) on
        // distinct positions runs as one straight-line sequence: the ops
        // commute, so they are stored in position order as K_RP records
        std::vector<HostOp> sops = hs.ops;
        uint32_t rp_mask = 0;
        bool rp_stage = !sops.empty();
        for (const HostOp &o : sops) {
          if ((o.kind != K_RP && o.kind != K_R) || (rp_mask & (1u << o.a))) { rp_stage = false; break; }
          rp_mask |= 1u << o.a;
        }
        if (rp_stage) {
          std::sort(sops.begin(), sops.end(), [](const HostOp &x, const HostOp &y) { return x.a < y.a; });
          for (HostOp &o : sops)
            if (o.kind == K_R) {  // {r00, 0, r01, 0, r10, 0, r11, 0} -> {r00, r01, r10, r11, 1, 0}
              const double r[4] = {o.m[0], o.m[2], o.m[4], o.m[6]};
              o.m[0] = r[0]; o.m[1] = r[1]; o.m[2] = r[2]; o.m[3] = r[3];
              o.m[4] = 1.0; o.m[5] = 0.0; o.m[6] = 0.0; o.m[7] = 0.0;
              o.kind = K_RP;
            }
        }
        sd.rp_mask = rp_stage ? rp_mask : 0u;
        // a stage of four-position groups with a rotation-and-phase op on
        // every position is D R3 R2 R1 R0 with D the product of the ops'
        // |1>-phases (each diagonal on its own position, so it commutes
        // with the other positions' rotations): amplitude e of the group
        // takes the product of the phases of its set positions, computed
        // here in FP64 and stored as double-float pairs
        sd.ph_block = 0xFFFFFFFFu;
        if ((hs.gphase[0] != 1.0 || hs.gphase[1] != 0.0) && (fp64 || pr.g != 4 || !rp_stage || rp_mask != 0xFu))
          fail(QW_ERR_STATE, "internal: a global phase on a stage without a phase table");
        if (!fp64 && pr.g == 4 && rp_stage && rp_mask == 0xFu) {
          const bool gfold = hs.gphase[0] != 1.0 || hs.gphase[1] != 0.0;
          sd.ph_block = (uint32_t)(ph.size() / 64) | (gfold ? 0x80000000u : 0u);
          for (uint32_t e = 0; e < 16; e++) {
            std::complex<double> q(hs.gphase[0], hs.gphase[1]);
            for (const HostOp &o : sops)
              if ((e >> o.a) & 1u) q *= std::complex<double>(o.m[4], o.m[5]);
            const float rh = (float)q.real(), ih = (float)q.imag();
            ph.push_back(rh);
            ph.push_back((float)(q.real() - (double)rh));
            ph.push_back(ih);
            ph.push_back((float)(q.imag() - (double)ih));
          }
        }
        sd.n_ops = (uint32_t)sops.size();
        sd.op_begin = (uint32_t)(fp64 ? ops64.size() : ops32.size());
        for (const HostOp &o : sops) {
          const uint32_t lo = std::min(o.a, o.b), hi = std::max(o.a, o.b);
          const uint32_t code = o.kind == K_CD ? sv_op_index(o.kind, lo, hi) : sv_op_index(o.kind, o.a, 0);
          if (code >= SV_N_OP_INDEX || o.a >= pr.g || (o.kind == K_CD && (hi >= pr.g || lo == hi)))
            fail(QW_ERR_STATE, "internal: op outside the stage dispatch table");
          if (fp64) {
            SvOpDesc<double> od{};
            od.code = code;
            for (int t = 0; t < 8; t++) od.m[t] = o.m[t];
            ops64.push_back(od);
          } else {
            SvOpDesc<float> od{};
            od.code = code;
            for (int t = 0; t < 8; t++) {
              od.m[t] = (float)o.m[t];
              ops32lo.push_back((float)(o.m[t] - (double)od.m[t]));
            }
            ops32.push_back(od);
          }
        }
        stages.push_back(sd);
      }
      passes.push_back(d);
    }
    return first;
  }
};

// device allocation tracked for release
struct DevArena {
  Engine *eng = nullptr;  // when set, blocks come from and return to the engine's cache
  std::vector<std::pair<void *, size_t>> blocks;
  uint64_t h2d = 0;  // bytes uploaded from the host
  void *alloc(size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    size_t got = bytes;
    if (eng) p = eng->dev_alloc(bytes, &got);
    else CK(cudaMalloc(&p, bytes));
    blocks.push_back({p, got});
    return p;
  }
  template <typename T>
  T *upload(const std::vector<T> &v, cudaStream_t s) {
    T *p = (T *)alloc(v.size() * sizeof(T));
    if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    h2d += v.size() * sizeof(T);
    return p;
  }
  void release() {
    for (auto &b : blocks) {
      if (eng) eng->dev_free(b.first, b.second);
      else cudaFree(b.first);
    }
    blocks.clear();
  }
};

struct Wave {
  bool fp64 = false;
  bool per_pass = false;                  // one launch per pass (else one persistent launch)
  int ar = SV_AR_PLAIN;                   // arithmetic of the wave's FP32 passes
  uint32_t k_max = 13;
  int grid = 0;
  std::vector<uint32_t> tasks;            // tasks run in this wave (own buffers)
  std::vector<uint32_t> obs_tasks;        // tasks whose observables are evaluated in this wave
  std::vector<SvJob> jobs;                // pass jobs, in list order
  bool fused_energy = false;              // energy blocks run inside the persistent launch
  uint32_t seg_bits = 0;
  std::vector<SvSeg> segs;
  uint32_t total_items = 0;
  SvJob *d_jobs = nullptr;
  SvSeg *d_segs = nullptr;
  unsigned int *d_ctr = nullptr;
  size_t ctr_words = 0;
  std::vector<EnJob> en;
  std::vector<uint32_t> obs_tasks_en;     // task of each energy job
  uint32_t en_blocks = 0;
  EnJob *d_en = nullptr;
  std::vector<SmpSource> src;
  uint32_t smp_blocks = 0;
  SmpSource *d_src = nullptr;
  std::vector<SmpShot> shots;
  SmpShot *d_shots = nullptr;
  std::vector<std::pair<uint32_t, std::pair<const void *, void *>>> converts;  // task, (src, dst)
};

struct DeviceState {
  DevArena arena;
  cudaStream_t stream = nullptr;
  SvTables t32{}, t64{};
  // FP32 arithmetic: of the boundaries' passes and per-task launches
  // (ar_chain: SV_AR_REM, or SV_AR_PLAIN) and of the persistent suffix
  // launches (ar_batch: SV_AR_COMP or SV_AR_PLAIN); `rem` is the remainder
  // array those chains share (they run one after another on the stream)
  int ar_chain = SV_AR_PLAIN, ar_batch = SV_AR_PLAIN;
  void *rem = nullptr;
  std::vector<uint32_t> mat_pass0, task_pass0;
  std::vector<void *> mat_buf;
  std::vector<void *> mat_export[2];   // per mode (FP64, FP32): statevector exported from a tableau node
  std::vector<StabBasis *> mat_basis;  // scratch of each exporting tableau node
  std::vector<int> tab_launch_of_mat;  // index into tab_mat_launches, -1 none
  std::vector<qw_dense_prog *> mat_dense;  // boundary evolved by a dense-block program, else NULL
  // statevector boundaries of one precision in one persistent launch (a
  // boundary's first pass waits for its parent's last); empty = per-pass launches
  struct MatBatch {
    bool fp64 = false;
    uint32_t k_max = 5, seg_bits = 0, total_items = 0;
    int grid = 0;
    size_t n_jobs = 0, ctr_words = 0;
    SvJob *d_jobs = nullptr;
    SvSeg *d_segs = nullptr;
    unsigned int *d_ctr = nullptr;
  };
  std::vector<MatBatch> mat_batches;
  std::vector<void *> task_state;  // state a task's observables read
  std::vector<Wave> waves;
  EnClass *d_classes = nullptr;
  EnTerm *d_terms = nullptr;
  std::vector<uint32_t> ham_class_off;
  double *d_partials = nullptr;
  double *d_bsum = nullptr, *d_boff = nullptr;
  int32_t *d_blast = nullptr;
  int64_t *d_lastnz = nullptr;
  double *d_energy = nullptr;
  uint64_t *d_samples = nullptr;
  // tableau
  TabProgram *d_progs = nullptr;
  TabLayer *d_layers = nullptr;
  TabSlot *d_slots = nullptr;
  uint8_t *d_bits = nullptr;
  uint8_t *d_outs = nullptr, *d_mat_outs = nullptr;
  struct TabLaunch {
    TabArgs a;
    uint32_t n_tasks;
    int frame;  // >= 0: preceded by the reference run and the frame launch of this frame group
  };
  std::vector<TabLaunch> tab_mat_launches, tab_task_launches;
  // final inverse tableau of each tableau task submitted with
  // QW_TASK_KEEP_STATE: 2n rows of 2W words, then 2n sign bytes elsewhere
  std::vector<std::pair<const uint64_t *, const uint8_t *>> tab_keep;
  struct FrameLaunch {
    TabArgs ref;  // the reference suffix on the tableau (one CTA), outcomes and random flag
    FrameArgs fa;
  };
  std::vector<FrameLaunch> frame_launches;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t ev[8] = {nullptr};
  std::vector<cudaEvent_t> wave_ev;  // 4 per wave: start, after suffix, after energy, after sampling
  ~DeviceState() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    for (auto &e : ev) if (e) cudaEventDestroy(e);
    for (auto &e : wave_ev) cudaEventDestroy(e);
    arena.release();
  }
};

static size_t sv_state_bytes(bool fp64, uint32_t n_eff) { return (size_t)(fp64 ? 16 : 8) << n_eff; }

// HBM bytes of a chain of `passes` passes over a state of S bytes: the state
// is read and written once per pass; with a remainder array (SV_AR_REM)
// every pass but the first also reads it and every pass but the last writes it
static double chain_bytes(double S, size_t passes, int ar) {
  const double p = (double)passes;
  return 2.0 * S * p + ((ar == SV_AR_REM && passes > 1) ? 2.0 * S * (p - 1.0) : 0.0);
}
// remainder arrays of pass p of a chain of n passes (SV_AR_REM)
static const void *chain_src_lo(const DeviceState *D, int ar, size_t p) {
  return (ar == SV_AR_REM && p > 0) ? D->rem : nullptr;
}
static void *chain_dst_lo(const DeviceState *D, int ar, size_t p, size_t n) {
  return (ar == SV_AR_REM && p + 1 < n) ? D->rem : nullptr;
}
// Algorithmic floating-point operations of one pass over 2^n amplitudes
// (an FMA counts two, an add or a multiply one), from its stages' register
// ops under the arithmetic `ar`, per group of A = 2^g amplitudes:
//   plain: a real rotation output costs 6 (packed multiply + FMA on both
//   components), a complex product 6, a general 2x2 output 14;
//   compensated: every two-term output (df_lin2: 2 multiplies, 6 FMAs and
//   8 adds per component) costs 44, a general 2x2 output two of them plus a
//   double-float add (104), and every stage renormalizes each amplitude (6).
static double pass_flops(const HostPass &hp, uint32_t n, uint32_t g, int ar) {
  const bool comp = ar != SV_AR_PLAIN;
  const double groups = std::ldexp(1.0, (int)n - (int)g), A = std::ldexp(1.0, (int)g);
  const double lin = comp ? 44.0 : 6.0, cm = comp ? 44.0 : 6.0, u1 = comp ? 104.0 : 14.0;
  double f = 0;
  for (const HostStage &st : hp.stages) {
    double fg = comp ? A * 6.0 : 0.0;
    // a compensated four-position stage with a rotation (and phase) on
    // every position: four rotations and one product per amplitude from the
    // stage's phase table (every amplitude but the first)
    if (comp && g == 4 && st.ops.size() == 4) {
      uint32_t mask = 0;
      bool rot = true;
      for (const HostOp &o : st.ops) {
        rot = rot && (o.kind == K_RP || o.kind == K_R) && !(mask & (1u << o.a));
        mask |= 1u << o.a;
      }
      if (rot && mask == 0xFu) {
        // rounded amplitudes enter a SV_AR_COMP stage with zero remainders:
        // its first rotation has no remainder products (2 packed FMAs, 8
        // flops, per output)
        const double first = (ar == SV_AR_COMP) ? lin - 8.0 : lin;
        const bool gfold = st.gphase[0] != 1.0 || st.gphase[1] != 0.0;
        f += (fg + A * first + 3.0 * A * lin + (gfold ? A : A - 1.0) * cm) * groups;
        continue;
      }
    }
    for (const HostOp &o : st.ops) {
      switch (o.kind) {
        case K_R: case K_RX: fg += A * lin; break;
        case K_RP: fg += A * lin + A / 2 * cm; break;
        case K_U1: fg += A * u1; break;
        case K_D1: fg += A * cm; break;
        case K_P1: fg += A / 2 * cm; break;
        case K_CD: fg += (comp && o.m[0] == -1.0 && o.m[1] == 0.0) ? 0.0 : A / 4 * cm; break;
        default: break;
      }
    }
    f += fg * groups;
  }
  return f;
}

int plan_ar_batch(const qw_plan *P) { return P->fp32_compensated ? SV_AR_COMP : SV_AR_PLAIN; }

// Segment size of a persistent work list: the largest power of two (at most
// 64) that no job's unit count falls below, so that few items are empty.
static uint32_t segment_bits(const std::vector<SvJob> &jobs) {
  uint32_t mn = 64;
  for (const SvJob &j : jobs) mn = std::min<uint32_t>(mn, std::max<uint32_t>(1, j.n_tiles));
  uint32_t b = 0;
  while ((2u << b) <= mn) b++;
  return b;
}

// Orders the work of one persistent launch into segments.  jobs[0, n_pass)
// are pass jobs, already in list order (a task's passes in sequence); the
// rest are energy jobs sorted by the pass job they wait for.  An energy job
// is released once its dependency has been listed and `lag` more items have
// gone by (by then its last tiles have been taken, so the wait is short);
// released energy work is interleaved so that the pass and energy streams
// advance at the same fraction of their totals, which keeps the two kinds
// of work (ALU-bound tiles, L2-bound energy blocks) running side by side.
static void build_segments(const std::vector<SvJob> &jobs, size_t n_pass, uint32_t seg_bits, uint64_t lag,
                           std::vector<SvSeg> &segs) {
  const uint64_t G = 1ull << seg_bits;
  auto nseg = [&](const SvJob &j) { return (uint64_t)(j.n_tiles + G - 1) / G; };
  uint64_t pass_total = 0, en_total = 0;
  for (size_t i = 0; i < jobs.size(); i++) (i < n_pass ? pass_total : en_total) += nseg(jobs[i]);
  segs.clear();
  segs.reserve(pass_total + en_total);
  std::vector<int64_t> end_seg(jobs.size(), -1);  // one past the job's last segment
  std::vector<int64_t> first_seg(jobs.size(), -1);
  size_t pi = 0, ei = n_pass;
  uint32_t pu = 0, eu = 0;
  uint64_t pass_done = 0, en_done = 0;
  const uint64_t lag_segs = (lag + G - 1) / G;
  while (pi < n_pass || ei < jobs.size()) {
    // skip jobs without units
    if (pi < n_pass && jobs[pi].n_tiles == 0) { end_seg[pi] = first_seg[pi] = (int64_t)segs.size(); pi++; continue; }
    if (ei < jobs.size() && jobs[ei].n_tiles == 0) { ei++; continue; }
    bool e_ready = false;
    if (ei < jobs.size()) {
      const int dep = jobs[ei].dep;
      e_ready = dep < 0 || (end_seg[dep] >= 0 && (pi >= n_pass || (uint64_t)segs.size() - end_seg[dep] >= lag_segs));
    }
    bool take_e;
    if (pi >= n_pass) take_e = true;
    else if (!e_ready) take_e = false;
    else take_e = en_done * pass_total <= pass_done * en_total;
    const size_t j = take_e ? ei : pi;
    uint32_t &u = take_e ? eu : pu;
    if (first_seg[j] < 0) first_seg[j] = (int64_t)segs.size();
    segs.push_back(SvSeg{(uint32_t)j, u});
    u += (uint32_t)G;
    (take_e ? en_done : pass_done) += 1;
    if (u >= jobs[j].n_tiles) {
      end_seg[j] = (int64_t)segs.size();
      u = 0;
      if (take_e) ei++; else pi++;
    }
  }
  // every dependency lies wholly before its dependent (the launch drains)
  for (size_t j = 0; j < jobs.size(); j++) {
    const int d = jobs[j].dep;
    if (d >= 0 && jobs[j].n_tiles && jobs[d].n_tiles && end_seg[d] > first_seg[j])
      fail(QW_ERR_STATE, "internal: work list orders a job before its dependency");
  }
}

// ---------------------------------------------------------------------------
// prepare: allocate, upload, build launch descriptors
// ---------------------------------------------------------------------------
static void prepare(qw_plan *P) {
  Engine *E = P->eng;
  DeviceState *D = new DeviceState();
  D->arena.eng = E;
  P->dev = D;
  D->stream = (cudaStream_t)E->stream;
  cudaStream_t s = D->stream;
  const uint32_t nt = (uint32_t)P->tasks.size();

  // statevector programs
  SvTableBuilder b32(false), b64(true);
  D->mat_pass0.assign(P->mats.size(), 0);
  D->task_pass0.assign(nt, 0);
  D->ar_batch = plan_ar_batch(P);
  D->ar_chain = D->ar_batch == SV_AR_COMP ? SV_AR_REM : SV_AR_PLAIN;
  size_t rem_bytes = 0;  // largest FP32 chain that keeps a remainder
  for (size_t m = 0; m < P->mats.size(); m++) {
    const MatNode &M = P->mats[m];
    if (M.mode == QW_MODE_TABLEAU) continue;
    D->mat_pass0[m] = (M.mode == QW_MODE_SV_FP64 ? b64 : b32).add(M.sv);
    const bool f64 = M.mode == QW_MODE_SV_FP64;
    const int ar = f64 ? SV_AR_PLAIN : D->ar_chain;
    const size_t S = sv_state_bytes(f64, M.n_eff);
    // algorithmic bytes of the boundary's passes (state, and the remainder between passes)
    P->prefix_alg_bytes += chain_bytes((double)S, M.sv.passes.size(), ar);
    for (const HostPass &hp : M.sv.passes) P->prefix_alg_flops += pass_flops(hp, M.n_eff, M.sv.g, ar);
    if (ar == SV_AR_REM && M.sv.passes.size() > 1) rem_bytes = std::max(rem_bytes, S);
  }
  for (uint32_t t = 0; t < nt; t++) {
    const TaskPlan &tp = P->tasks[t];
    if (tp.mode == QW_MODE_TABLEAU) continue;
    D->task_pass0[t] = (tp.mode == QW_MODE_SV_FP64 ? b64 : b32).add(tp.sv);
  }
  D->t32.passes = D->arena.upload(b32.passes, s);
  D->t32.stages = D->arena.upload(b32.stages, s);
  D->t32.ops = D->arena.upload(b32.ops32, s);
  D->t32.ops_lo = D->arena.upload(b32.ops32lo, s);
  D->t32.ph = D->arena.upload(b32.ph, s);
  D->t64.passes = D->arena.upload(b64.passes, s);
  D->t64.stages = D->arena.upload(b64.stages, s);
  D->t64.ops = D->arena.upload(b64.ops64, s);

  // boundary store (budget was enforced by the planner)
  D->mat_buf.assign(P->mats.size(), nullptr);
  D->mat_export[0].assign(P->mats.size(), nullptr);
  D->mat_export[1].assign(P->mats.size(), nullptr);
  D->mat_basis.assign(P->mats.size(), nullptr);
  for (size_t m = 0; m < P->mats.size(); m++) {
    const MatNode &M = P->mats[m];
    if (M.mode == QW_MODE_TABLEAU) {
      const uint32_t W = (M.n + 63) / 64;
      D->mat_buf[m] = D->arena.alloc((size_t)2 * M.n * 2 * W * 8 + 2 * M.n + 64);
      if (M.export_modes) {
        if (M.n > QW_SV_MAX_QUBITS) fail(QW_ERR_STATE, "internal: tableau export above the statevector cap");
        D->mat_basis[m] = (StabBasis *)D->arena.alloc(sizeof(StabBasis));
        const uint32_t n_eff = std::max<uint32_t>(M.n, SV_G);
        for (uint32_t md = 0; md < 2; md++)
          if ((M.export_modes >> md) & 1u)
            D->mat_export[md][m] = D->arena.alloc(sv_state_bytes(md == QW_MODE_SV_FP64, n_eff));
      }
    } else {
      D->mat_buf[m] = D->arena.alloc(sv_state_bytes(M.mode == QW_MODE_SV_FP64, M.n_eff));
      // lower-precision copy for the consumers of another precision
      for (uint32_t md = 0; md < 2; md++)
        if (md != M.mode && ((M.export_modes >> md) & 1u))
          D->mat_export[md][m] = D->arena.alloc(sv_state_bytes(md == QW_MODE_SV_FP64, M.n_eff));
    }
  }
  // ---- statevector boundaries as dense-block programs (dense_boundaries) --
  D->mat_dense.assign(P->mats.size(), nullptr);
  P->dense_choices.clear();
  if (P->opts.dense_boundaries) {
    for (size_t m = 0; m < P->mats.size(); m++) {
      const MatNode &M = P->mats[m];
      if (M.mode == QW_MODE_TABLEAU || M.sv.passes.empty() || M.gates.empty()) continue;
      if (M.parent >= 0 && P->mats[M.parent].mode != M.mode) continue;
      const bool fp64 = M.mode == QW_MODE_SV_FP64;
      qw_dense_prog *dp = dense_prog_autotune(E, M.mode, M.n_eff, M.gates.data(), M.gates.size(), 0, QW_DENSE_AUTO);
      DenseChoice c;
      c.mat = (int)m;
      dense_prog_config(dp, &c.engine, &c.width, nullptr, &c.est_ms);
      c.blocks = (uint32_t)dense_prog_blocks(dp);
      c.over_budget = !fp64 && D->ar_chain == SV_AR_REM && c.blocks > DENSE_COMP_MAX_BLOCKS;
      bool use = P->opts.dense_boundaries == 2 && !c.over_budget;
      if (!use && !c.over_budget) {
        // both candidates timed once from |0...0> on a scratch state
        const size_t bytes = sv_state_bytes(fp64, M.n_eff), n_amp = (size_t)1 << M.n_eff;
        void *scratch = nullptr, *scratch_lo = nullptr;
        const int ar = fp64 ? SV_AR_PLAIN : D->ar_chain;
        CK(cudaMalloc(&scratch, bytes));
        if (ar == SV_AR_REM) CK(cudaMalloc(&scratch_lo, bytes));
        const SvTables &T = fp64 ? D->t64 : D->t32;
        cudaEvent_t e[4];
        for (auto &x : e) CK(cudaEventCreate(&x));
        CK(cudaEventRecord(e[0], s));
        const size_t np = M.sv.passes.size();
        for (size_t p = 0; p < np; p++)
          launch_sv_pass(fp64, T, D->mat_pass0[m] + (uint32_t)p, (uint32_t)M.sv.passes[p].q.size(), M.n_eff,
                         p == 0 ? nullptr : scratch, scratch, s, ar, (ar == SV_AR_REM && p > 0) ? scratch_lo : nullptr,
                         (ar == SV_AR_REM && p + 1 < np) ? scratch_lo : nullptr);
        CK(cudaEventRecord(e[1], s));
        CK(cudaEventRecord(e[2], s));
        basis_zero_kernel<<<(unsigned)std::min<size_t>((n_amp + 255) / 256, (size_t)E->sm_count * 16), 256, 0, s>>>(
            scratch, fp64, n_amp);
        dense_prog_run(dp, scratch, s);
        CK(cudaEventRecord(e[3], s));
        CK(cudaEventSynchronize(e[3]));
        float a = 0, b = 0;
        CK(cudaEventElapsedTime(&a, e[0], e[1]));
        CK(cudaEventElapsedTime(&b, e[2], e[3]));
        for (auto &x : e) cudaEventDestroy(x);
        cudaFree(scratch);
        if (scratch_lo) cudaFree(scratch_lo);
        dense_prog_check(dp);
        c.pass_ms = a;
        c.dense_ms = b;
        use = b < a;
      }
      c.used = use;
      P->dense_choices.push_back(c);
      if (use) D->mat_dense[m] = dp;
      else dense_prog_destroy(dp);
    }
  }

  // the state a statevector consumer of node m reads (the node itself, or its
  // export into the consumer's precision)
  auto sv_source = [&](int m, uint32_t mode) -> void * {
    if (P->mats[m].mode == mode) return D->mat_buf[m];
    return D->mat_export[mode][m] ? D->mat_export[mode][m] : D->mat_buf[m];
  };
  auto needs_convert = [&](const TaskPlan &tp) {
    return tp.src >= 0 && P->mats[tp.src].mode != QW_MODE_TABLEAU && P->mats[tp.src].mode != tp.mode &&
           !D->mat_export[tp.mode][tp.src];
  };

  // ---- statevector boundaries: one persistent launch per precision --------
  // Used when every boundary has passes and continues from |0...0> or from a
  // statevector boundary of its own precision (no export or conversion in
  // between); a boundary's first pass then waits for its parent's last, and
  // sibling boundaries run side by side.  Otherwise: pass by pass.
  {
    bool ok = P->opts.batched != 0;
    size_t n_sv = 0;
    for (const qw_dense_prog *dp : D->mat_dense)
      if (dp) ok = false;  // a dense-block boundary is launched block by block
    for (const MatNode &M : P->mats) {
      if (M.mode == QW_MODE_TABLEAU) continue;
      n_sv++;
      if (M.sv.passes.empty()) ok = false;
      if (M.parent >= 0 && P->mats[M.parent].mode != M.mode) ok = false;
      // compensated FP32 boundaries keep their remainder between passes,
      // which the persistent launch does not carry: pass by pass
      if (M.mode == QW_MODE_SV_FP32 && D->ar_chain == SV_AR_REM) ok = false;
    }
    // a single boundary is a chain of dependent passes: separate launches
    // serve it as well, without CTAs waiting on the previous pass
    if (ok && n_sv > 1) {
      std::vector<uint32_t> level(P->mats.size(), 0);
      uint32_t max_level = 0;
      size_t max_p = 0;
      for (size_t m = 0; m < P->mats.size(); m++) {  // parents precede their children
        const MatNode &M = P->mats[m];
        if (M.mode == QW_MODE_TABLEAU) continue;
        level[m] = (M.parent >= 0) ? level[M.parent] + 1 : 0;
        max_level = std::max(max_level, level[m]);
        max_p = std::max(max_p, M.sv.passes.size());
      }
      for (uint32_t prec : {(uint32_t)QW_MODE_SV_FP32, (uint32_t)QW_MODE_SV_FP64}) {
        std::vector<SvJob> jobs;
        std::vector<int> last_job(P->mats.size(), -1);
        uint32_t kmax = 5;
        for (uint32_t L = 0; L <= max_level; L++)
          for (size_t pi = 0; pi < max_p; pi++)
            for (size_t m = 0; m < P->mats.size(); m++) {
              const MatNode &M = P->mats[m];
              if (M.mode != prec || level[m] != L || pi >= M.sv.passes.size()) continue;
              const uint32_t k = (uint32_t)M.sv.passes[pi].q.size();
              SvJob j{};
              j.src = (pi == 0) ? (M.parent >= 0 ? D->mat_buf[M.parent] : nullptr) : D->mat_buf[m];
              j.dst = D->mat_buf[m];
              j.pass = D->mat_pass0[m] + (uint32_t)pi;
              j.n_tiles = 1u << (M.n_eff - k);
              j.dep = (pi == 0) ? (M.parent >= 0 ? last_job[M.parent] : -1) : last_job[m];
              j.kind = SVJ_PASS;
              j.n = M.n_eff;
              last_job[m] = (int)jobs.size();
              jobs.push_back(j);
              kmax = std::max(kmax, k);
            }
        if (jobs.empty()) continue;
        DeviceState::MatBatch B;
        B.fp64 = prec == QW_MODE_SV_FP64;
        B.k_max = kmax;
        B.grid = sv_batch_grid(B.fp64, kmax, E->sm_count);
        B.seg_bits = segment_bits(jobs);
        std::vector<SvSeg> segs;
        build_segments(jobs, jobs.size(), B.seg_bits, 2ull * (uint64_t)B.grid, segs);
        if (((uint64_t)segs.size() << B.seg_bits) > 0xFFFFFFF0ull)
          fail(QW_ERR_BUDGET, "the boundaries' work list exceeds 2^32 items");
        B.total_items = (uint32_t)(segs.size() << B.seg_bits);
        B.n_jobs = jobs.size();
        B.d_jobs = D->arena.upload(jobs, s);
        B.d_segs = D->arena.upload(segs, s);
        B.ctr_words = 2 + jobs.size();
        B.d_ctr = (unsigned int *)D->arena.alloc(B.ctr_words * sizeof(unsigned int));
        D->mat_batches.push_back(B);
      }
    }
  }

  // Hamiltonians
  std::vector<EnClass> cls;
  std::vector<EnTerm> trm;
  for (auto &H : P->hams) {
    D->ham_class_off.push_back((uint32_t)cls.size());
    const uint32_t toff = (uint32_t)trm.size();
    for (EnClass c : H.classes) {
      c.term_begin += toff;
      c.term_end += toff;
      cls.push_back(c);
    }
    trm.insert(trm.end(), H.terms.begin(), H.terms.end());
  }
  D->d_classes = D->arena.upload(cls, s);
  D->d_terms = D->arena.upload(trm, s);

  // results
  D->d_energy = (double *)D->arena.alloc(sizeof(double) * 2 * std::max<uint32_t>(nt, 1));
  P->sample_off.assign(nt + 1, 0);
  for (uint32_t t = 0; t < nt; t++) P->sample_off[t + 1] = P->sample_off[t] + P->tasks[t].shots;
  D->d_samples = (uint64_t *)D->arena.alloc(sizeof(uint64_t) * std::max<uint64_t>(1, P->sample_off[nt]));

  // ---- statevector tasks: buffers and waves --------------------------------
  D->task_state.assign(nt, nullptr);
  std::map<std::pair<int, uint32_t>, std::vector<uint32_t>> groups;  // (fp64, n_eff) -> tasks
  for (uint32_t t = 0; t < nt; t++) {
    const TaskPlan &tp = P->tasks[t];
    if (tp.mode == QW_MODE_TABLEAU) continue;
    groups[{tp.mode == QW_MODE_SV_FP64 ? 1 : 0, tp.n_eff}].push_back(t);
  }
  size_t max_partials = 1, max_smp_blocks = 1, max_src = 1;
  const bool batched = P->opts.batched != 0;
  // compensated FP32 tasks with long programs leave the persistent launch
  // (which rounds at every stage) for a chain of launches of their own that
  // keeps the remainder, one task after another
  auto long_chain = [&](const TaskPlan &tp) {
    return batched && D->ar_batch == SV_AR_COMP && tp.mode == QW_MODE_SV_FP32 &&
           tp.sv.passes.size() > (size_t)SV_COMP_MAX_BATCH_PASSES;
  };
  // Task buffers of every group coexist for the plan's lifetime, so the
  // groups share one task budget: each group with pooled tasks gets one
  // buffer, then the rest of the budget goes to the groups in order of
  // state size (smallest first) for up to one buffer per pooled task.
  std::map<std::pair<int, uint32_t>, size_t> pool_size;
  {
    std::vector<std::pair<size_t, std::pair<int, uint32_t>>> order;  // (S, group)
    std::map<std::pair<int, uint32_t>, size_t> n_pooled;
    uint64_t committed = 0;
    for (auto &g : groups) {
      size_t np = 0;
      bool any_long = false;
      for (uint32_t t : g.second) {
        const TaskPlan &tp = P->tasks[t];
        if ((!tp.sv.passes.empty() || needs_convert(tp)) && !(tp.flags & QW_TASK_KEEP_STATE)) {
          if (long_chain(tp)) any_long = true;
          else np++;
        }
      }
      if (any_long && np == 0) np = 1;
      const size_t S = sv_state_bytes(g.first.first != 0, g.first.second);
      n_pooled[g.first] = np;
      pool_size[g.first] = np ? 1 : 0;
      if (np) {
        committed += S;
        order.push_back({S, g.first});
      }
    }
    std::sort(order.begin(), order.end());
    uint64_t left = E->task_budget > committed ? E->task_budget - committed : 0;
    for (auto &o : order) {
      if (!batched) break;
      const size_t S = o.first;
      const size_t extra = std::min<size_t>(n_pooled[o.second] - 1, (size_t)(left / S));
      pool_size[o.second] += extra;
      left -= (uint64_t)extra * S;
    }
  }
  for (auto &g : groups) {
    const bool fp64 = g.first.first != 0;
    const uint32_t n_eff = g.first.second;
    const size_t S = sv_state_bytes(fp64, n_eff);
    std::vector<uint32_t> own, shared_src;
    for (uint32_t t : g.second) {
      const TaskPlan &tp = P->tasks[t];
      const bool convert = needs_convert(tp);
      if (!tp.sv.passes.empty() || convert) own.push_back(t);
      else { shared_src.push_back(t); D->task_state[t] = sv_source(tp.src, tp.mode); }
    }
    // KEEP_STATE tasks get dedicated buffers; the others share a pool
    std::vector<uint32_t> pooled;
    for (uint32_t t : own) {
      if (P->tasks[t].flags & QW_TASK_KEEP_STATE) D->task_state[t] = D->arena.alloc(S);
      else pooled.push_back(t);
    }
    // waves: dedicated tasks first (one wave), then pooled chunks; long
    // compensated chains one task per wave, launched pass by pass
    std::vector<uint32_t> dedicated, ded_short, pool_short, longs;
    for (uint32_t t : own) if (P->tasks[t].flags & QW_TASK_KEEP_STATE) dedicated.push_back(t);
    for (uint32_t t : dedicated) (long_chain(P->tasks[t]) ? longs : ded_short).push_back(t);
    bool pooled_long = false;
    for (uint32_t t : pooled) {
      if (long_chain(P->tasks[t])) { longs.push_back(t); pooled_long = true; }
      else pool_short.push_back(t);
    }
    const size_t pool_n =
        std::min(pool_size[g.first], std::max(pool_short.size(), (size_t)(pooled_long ? 1 : 0)));
    std::vector<void *> pool(pool_n);
    for (auto &p : pool) p = D->arena.alloc(S);
    std::vector<std::pair<std::vector<uint32_t>, bool>> wave_tasks;  // (tasks, per-pass launches)
    if (batched) {
      if (!ded_short.empty()) wave_tasks.push_back({ded_short, false});
      for (size_t i = 0; i < pool_short.size(); i += pool_n)
        wave_tasks.push_back({std::vector<uint32_t>(pool_short.begin() + i,
                                                    pool_short.begin() + std::min(pool_short.size(), i + pool_n)),
                              false});
      for (uint32_t t : longs) wave_tasks.push_back({{t}, true});
    } else {
      for (uint32_t t : own) wave_tasks.push_back({{t}, true});
    }
    if (wave_tasks.empty()) wave_tasks.push_back({{}, !batched});
    for (size_t w = 0; w < wave_tasks.size(); w++) {
      Wave W;
      W.fp64 = fp64;
      W.per_pass = wave_tasks[w].second;
      W.ar = fp64 ? SV_AR_PLAIN : (W.per_pass ? D->ar_chain : D->ar_batch);
      W.tasks = wave_tasks[w].first;
      uint32_t kmax = 5;
      for (size_t i = 0; i < W.tasks.size(); i++) {
        const uint32_t t = W.tasks[i];
        if (!(P->tasks[t].flags & QW_TASK_KEEP_STATE)) D->task_state[t] = pool[i % std::max<size_t>(1, pool_n)];
        for (const HostPass &hp : P->tasks[t].sv.passes) kmax = std::max<uint32_t>(kmax, (uint32_t)hp.q.size());
      }
      W.k_max = kmax;
      {
        uint32_t b_first = 0;
        for (uint32_t t : W.tasks)
          if (!P->tasks[t].sv.passes.empty()) { b_first = P->tasks[t].sv.passes[0].b; break; }
        P->wave_tiles.push_back({kmax, b_first});
      }
      W.obs_tasks = W.tasks;
      if (w == 0) W.obs_tasks.insert(W.obs_tasks.end(), shared_src.begin(), shared_src.end());
      // jobs, round-robin over pass index within windows of tasks
      std::map<uint32_t, int> last_pass;  // task -> its last pass job
      uint32_t window = P->opts.window ? P->opts.window : (uint32_t)W.tasks.size();
      window = std::max<uint32_t>(1, window);
      for (size_t w0 = 0; w0 < W.tasks.size(); w0 += window) {
        const size_t w1 = std::min(W.tasks.size(), w0 + window);
        size_t max_p = 0;
        for (size_t i = w0; i < w1; i++) max_p = std::max(max_p, P->tasks[W.tasks[i]].sv.passes.size());
        std::vector<int> last(W.tasks.size(), -1);
        for (size_t p = 0; p < max_p; p++) {
          for (size_t i = w0; i < w1; i++) {
            const uint32_t t = W.tasks[i];
            const TaskPlan &tp = P->tasks[t];
            if (p >= tp.sv.passes.size()) continue;
            SvJob j{};
            const bool convert = needs_convert(tp);
            j.src = (p == 0 && !convert) ? (tp.src >= 0 ? sv_source(tp.src, tp.mode) : nullptr) : D->task_state[t];
            j.dst = D->task_state[t];
            j.pass = D->task_pass0[t] + (uint32_t)p;
            j.n_tiles = 1u << (tp.n_eff - (uint32_t)tp.sv.passes[p].q.size());
            P->batch_alg_flops += pass_flops(tp.sv.passes[p], tp.n_eff, tp.sv.g, W.ar);
            j.dep = last[i];
            j.kind = SVJ_PASS;
            j.n = tp.n_eff;
            last[i] = (int)W.jobs.size();
            last_pass[t] = (int)W.jobs.size();
            W.jobs.push_back(j);
          }
        }
      }
      for (uint32_t t : W.tasks) {
        const TaskPlan &tp = P->tasks[t];
        if (needs_convert(tp)) W.converts.push_back({t, {D->mat_buf[tp.src], D->task_state[t]}});
      }
      // energy jobs
      for (uint32_t t : W.obs_tasks) {
        const TaskPlan &tp = P->tasks[t];
        if (tp.ham < 0) continue;
        const HamLayout &H = P->hams[tp.ham];
        EnJob j{};
        j.state = D->task_state[t];
        j.out = D->d_energy + 2 * (size_t)t;
        j.n = H.n_eff;
        j.chunk_bits = H.chunk_bits;
        j.class_begin = D->ham_class_off[tp.ham];
        j.n_classes = (uint32_t)H.classes.size();
        j.block_begin = W.en_blocks;
        j.n_blocks = H.n_blocks;
        W.en_blocks += H.n_blocks;
        W.en.push_back(j);
        W.obs_tasks_en.push_back(t);
      }
      max_partials = std::max<size_t>(max_partials, W.en_blocks);
      // sampling sources (deduplicated by state) and shots
      std::map<const void *, uint32_t> sid;
      for (uint32_t t : W.obs_tasks) {
        const TaskPlan &tp = P->tasks[t];
        if (!tp.shots) continue;
        const void *st = D->task_state[t];
        auto it = sid.find(st);
        uint32_t si;
        if (it == sid.end()) {
          SmpSource so{};
          so.state = st;
          so.n = tp.n_eff;
          so.n_blocks = (tp.n_eff >= (uint32_t)SMP_BLOCK_BITS) ? (1u << (tp.n_eff - SMP_BLOCK_BITS)) : 1u;
          so.block_begin = W.smp_blocks;
          W.smp_blocks += so.n_blocks;
          si = (uint32_t)W.src.size();
          W.src.push_back(so);
          sid[st] = si;
        } else {
          si = it->second;
        }
        for (uint32_t k = 0; k < tp.shots; k++) {
          SmpShot q{};
          q.u = tp.uniforms[k];
          q.source = si;
          q.out = D->d_samples + P->sample_off[t] + k;
          W.shots.push_back(q);
        }
      }
      max_smp_blocks = std::max<size_t>(max_smp_blocks, W.smp_blocks);
      max_src = std::max<size_t>(max_src, W.src.size());
      // algorithmic bytes: every pass reads and writes its state once; the
      // energy of a task reads every amplitude once per term class
      if (W.ar == SV_AR_REM) {  // one task, its passes in order
        P->batch_alg_bytes += chain_bytes((double)S, W.jobs.size(), W.ar);
        if (W.jobs.size() > 1) rem_bytes = std::max(rem_bytes, S);
      } else {
        for (const SvJob &j : W.jobs) { (void)j; P->batch_alg_bytes += 2.0 * (double)S; }
      }
      for (size_t e = 0; e < W.en.size(); e++) {
        const EnJob &j = W.en[e];
        const double Sj = (double)sv_state_bytes(fp64, j.n);
        P->energy_alg_bytes += (double)j.n_classes * Sj;
        // L2 -> SM reads: own amplitudes once per class, and half the state
        // per flipping term (each pair is read from one side)
        const HamLayout &H = P->hams[P->tasks[W.obs_tasks_en[e]].ham];
        size_t flipping = 0;
        for (const EnTerm &t : H.terms) flipping += (t.xm != 0);
        P->energy_l2_bytes += (double)j.n_classes * Sj + 0.5 * Sj * (double)flipping;
      }
      // persistent work list: pass jobs, then (fused) the energy jobs,
      // released in the order their states finish
      std::vector<SvJob> up = W.jobs;
      W.grid = !W.per_pass ? sv_batch_grid(fp64, W.k_max, E->sm_count, W.ar) : 0;
      W.fused_energy =
          !W.per_pass && P->opts.fuse_energy && !W.en.empty() && sv_threads_for_k(W.k_max, W.ar, fp64) == 128;
      if (W.fused_energy) {
        std::vector<SvJob> ej;
        for (size_t e = 0; e < W.en.size(); e++) {
          SvJob j{};
          const uint32_t t = W.obs_tasks_en[e];
          auto it = last_pass.find(t);
          j.dep = (it == last_pass.end()) ? -1 : it->second;
          j.kind = SVJ_ENERGY;
          j.pass = (uint32_t)e;
          j.n_tiles = W.en[e].n_blocks;
          j.n = W.en[e].n;
          ej.push_back(j);
        }
        std::stable_sort(ej.begin(), ej.end(), [](const SvJob &a, const SvJob &b) { return a.dep < b.dep; });
        up.insert(up.end(), ej.begin(), ej.end());
      }
      if (!W.per_pass) {
        W.seg_bits = segment_bits(up);
        build_segments(up, W.jobs.size(), W.seg_bits, 2ull * (uint64_t)W.grid, W.segs);
        if (((uint64_t)W.segs.size() << W.seg_bits) > 0xFFFFFFF0ull)
          fail(QW_ERR_BUDGET, "a wave's work list exceeds 2^32 items; lower task_budget");
        W.total_items = (uint32_t)(W.segs.size() << W.seg_bits);
        if (W.fused_energy) P->energy_fused = true;
      }
      // With fault injection (tests only) the first job waits on an extra
      // job that has no segment, so no CTA ever takes it: its counter never
      // reaches the one unit it needs and the bounded wait runs out.
      if (P->opts.fault_injection && !W.per_pass && !up.empty()) {
        SvJob ph{};
        ph.n_tiles = 1;
        ph.dep = -1;
        up[0].dep = (int32_t)up.size();
        up.push_back(ph);
      }
      W.d_jobs = D->arena.upload(up, s);
      W.d_segs = D->arena.upload(W.segs, s);
      W.ctr_words = 2 + up.size();
      W.d_ctr = (unsigned int *)D->arena.alloc(W.ctr_words * sizeof(unsigned int));
      CK(cudaMemsetAsync(W.d_ctr, 0, W.ctr_words * sizeof(unsigned int), s));
      W.d_en = D->arena.upload(W.en, s);
      W.d_src = D->arena.upload(W.src, s);
      W.d_shots = D->arena.upload(W.shots, s);
      D->waves.push_back(std::move(W));
    }
  }
  D->d_partials = (double *)D->arena.alloc(sizeof(double) * 2 * max_partials);
  if (rem_bytes) D->rem = D->arena.alloc(rem_bytes);
  D->d_bsum = (double *)D->arena.alloc(sizeof(double) * max_smp_blocks);
  D->d_blast = (int32_t *)D->arena.alloc(sizeof(int32_t) * max_smp_blocks);
  D->d_boff = (double *)D->arena.alloc(sizeof(double) * (max_smp_blocks + max_src));
  D->d_lastnz = (int64_t *)D->arena.alloc(sizeof(int64_t) * max_src);

  // ---- tableau --------------------------------------------------------------
  std::vector<TabProgram> progs;
  std::vector<TabLayer> layers;
  std::vector<TabSlot> slots;
  for (const TabHostProgram &hp : P->tab_progs) {
    TabProgram pg{};
    pg.layer_begin = (uint32_t)layers.size();
    pg.n_layers = (uint32_t)hp.layers.size();
    pg.n_bits = hp.n_bits;
    pg.n_outs = hp.n_outs;
    const uint32_t soff = (uint32_t)slots.size();
    for (TabLayer L : hp.layers) { L.slot_begin += soff; layers.push_back(L); }
    slots.insert(slots.end(), hp.slots.begin(), hp.slots.end());
    progs.push_back(pg);
  }
  bool any_tab = !P->tab_progs.empty();
  if (any_tab) {
    D->d_progs = D->arena.upload(progs, s);
    D->d_layers = D->arena.upload(layers, s);
    D->d_slots = D->arena.upload(slots, s);
    D->d_bits = D->arena.upload(P->tab_bits, s);
    // outcome layout
    P->outs_off.assign(nt + 1, 0);
    for (uint32_t t = 0; t < nt; t++) P->outs_off[t + 1] = P->outs_off[t] + P->tasks[t].tab_outs;
    P->outs_mat_off.assign(P->mats.size() + 1, 0);
    for (size_t m = 0; m < P->mats.size(); m++) P->outs_mat_off[m + 1] = P->outs_mat_off[m] + P->mats[m].tab_outs;
    D->d_outs = (uint8_t *)D->arena.alloc(std::max<uint32_t>(1, P->outs_off[nt]));
    D->d_mat_outs = (uint8_t *)D->arena.alloc(std::max<uint32_t>(1, P->outs_mat_off[P->mats.size()]));
    auto add_launch = [&](std::vector<DeviceState::TabLaunch> &dst, uint32_t n, const void *init,
                          void *out_buf, const std::vector<TabTaskDesc> &descs,
                          const std::vector<TabSegment> &segs, uint8_t *outs) {
      TabArgs a{};
      a.n = n;
      a.W = (n + 63) / 64;
      a.lpp = a.W <= 8 ? 8 : (a.W <= 16 ? 16 : 32);
      a.rows = 2 * n;
      const size_t words = (size_t)a.rows * 2 * a.W;
      a.init_rows = (const uint64_t *)init;
      a.init_sign = init ? (const uint8_t *)((const uint64_t *)init + words) : nullptr;
      a.out_rows = (uint64_t *)out_buf;
      a.out_sign = out_buf ? (uint8_t *)((uint64_t *)out_buf + words) : nullptr;
      a.tasks = D->arena.upload(descs, s);
      a.segs = D->arena.upload(segs, s);
      a.progs = D->d_progs;
      a.layers = D->d_layers;
      a.slots = D->d_slots;
      a.bits = D->d_bits;
      a.outs = outs;
      dst.push_back({a, (uint32_t)descs.size(), -1});
    };
    D->tab_launch_of_mat.assign(P->mats.size(), -1);
    for (size_t m = 0; m < P->mats.size(); m++) {
      const MatNode &M = P->mats[m];
      if (M.mode != QW_MODE_TABLEAU) continue;
      D->tab_launch_of_mat[m] = (int)D->tab_mat_launches.size();
      std::vector<TabSegment> segs;
      uint32_t oo = 0;
      for (auto &sg : M.tab_segs) {
        segs.push_back({sg.first, sg.second, oo, 0});
        oo += P->tab_progs[sg.first].n_outs;
      }
      std::vector<TabTaskDesc> d{{0, (uint32_t)segs.size(), 0, P->outs_mat_off[m]}};
      add_launch(D->tab_mat_launches, M.n, M.parent >= 0 ? D->mat_buf[M.parent] : nullptr,
                 D->mat_buf[m], d, segs, D->d_mat_outs);
    }
    std::map<std::pair<int, uint32_t>, std::vector<uint32_t>> by_src;
    for (uint32_t t = 0; t < nt; t++)
      if (P->tasks[t].mode == QW_MODE_TABLEAU) by_src[{P->tasks[t].src, P->tasks[t].n}].push_back(t);
    D->tab_keep.assign(nt, {nullptr, nullptr});
    for (auto &g : by_src) {
      std::vector<TabTaskDesc> descs;
      std::vector<TabSegment> segs;
      for (uint32_t t : g.second) {
        const TaskPlan &tp = P->tasks[t];
        TabTaskDesc d{};
        d.seg_begin = (uint32_t)segs.size();
        d.out_base = P->outs_off[t];
        uint32_t oo = 0;
        for (auto &sg : tp.tab_segs) {
          segs.push_back({sg.first, sg.second, oo, 0});
          oo += P->tab_progs[sg.first].n_outs;
        }
        d.n_segs = (uint32_t)segs.size() - d.seg_begin;
        descs.push_back(d);
      }
      // tasks that keep their final tableau: the whole launch writes its
      // tableaus back (rows of every task, then the signs of every task)
      bool keep = false;
      for (uint32_t t : g.second) keep = keep || (P->tasks[t].flags & QW_TASK_KEEP_STATE);
      void *keep_buf = nullptr;
      const uint32_t kn = g.first.second, kW = (kn + 63) / 64;
      const size_t kwords = (size_t)2 * kn * 2 * kW, nk = g.second.size();
      if (keep) keep_buf = D->arena.alloc(nk * (kwords * 8 + 2 * kn));
      add_launch(D->tab_task_launches, g.first.second,
                 g.first.first >= 0 ? D->mat_buf[g.first.first] : nullptr, keep_buf, descs, segs,
                 D->d_outs);
      if (keep) {
        uint8_t *signs = (uint8_t *)((uint64_t *)keep_buf + nk * kwords);
        D->tab_task_launches.back().a.out_sign = signs;
        for (size_t k = 0; k < nk; k++)
          D->tab_keep[g.second[k]] = {(const uint64_t *)keep_buf + k * kwords, signs + k * 2 * kn};
      }
      const int fg = P->task_frame_group[g.second[0]];
      if (fg >= 0) {
        // Pauli frames: the reference suffix once on the tableau, then the
        // frame launch; the per-task launch above runs only if a reference
        // outcome was random (decided on the device, no host round trip)
        const FrameGroup &G = P->frame_groups[fg];
        if (G.tasks != g.second) fail(QW_ERR_STATE, "internal: frame group and tableau group differ");
        uint8_t *ref_out = (uint8_t *)D->arena.alloc(std::max<uint32_t>(1, G.n_outs));
        uint32_t *rand = (uint32_t *)D->arena.alloc(sizeof(uint32_t));
        std::vector<TabSegment> rsegs;
        uint32_t oo = 0;
        for (auto &sg : G.ref_segs) {
          rsegs.push_back({sg.first, sg.second, oo, 0});
          oo += P->tab_progs[sg.first].n_outs;
        }
        std::vector<TabTaskDesc> rd{{0, (uint32_t)rsegs.size(), 0, 0}};
        std::vector<DeviceState::TabLaunch> tmp;
        add_launch(tmp, G.n, D->mat_buf[G.src], nullptr, rd, rsegs, ref_out);
        DeviceState::FrameLaunch fl{};
        fl.ref = tmp[0].a;
        fl.ref.rand_any = rand;
        FrameArgs &fa = fl.fa;
        fa.n = G.n;
        fa.n_tasks = (uint32_t)G.tasks.size();
        fa.n_words = G.n_words;
        fa.n_layers = (uint32_t)G.prog.layers.size();
        fa.layers = D->arena.upload(G.prog.layers, s);
        fa.ops = D->arena.upload(G.prog.ops, s);
        fa.ev_x = D->arena.upload(G.ev_x, s);
        fa.ev_z = D->arena.upload(G.ev_z, s);
        fa.ref_out = ref_out;
        fa.rand_any = rand;
        std::vector<uint32_t> ob;
        for (uint32_t t : G.tasks) ob.push_back(P->outs_off[t]);
        fa.out_base = D->arena.upload(ob, s);
        fa.outs = D->d_outs;
        D->tab_task_launches.back().a.run_if = rand;
        D->tab_task_launches.back().frame = (int)D->frame_launches.size();
        D->frame_launches.push_back(fl);
      }
    }
  }
  for (auto &e : D->ev) CK(cudaEventCreate(&e));
  CK(cudaStreamSynchronize(s));
  P->h2d_bytes = D->arena.h2d;
  P->d2h_bytes = 16ull * nt + 8ull * P->sample_off[nt] +
                 (any_tab ? (uint64_t)P->outs_off[nt] + P->outs_mat_off[P->mats.size()] : 0ull);
}

// ---------------------------------------------------------------------------
// launch sequence of a prepared plan (captured once into a graph)
// ---------------------------------------------------------------------------
static void enqueue(qw_plan *P, cudaStream_t s, bool capturing) {
  DeviceState *D = P->dev;
  uint64_t nl = 0;  // kernels launched by one execution
  // timing events: inside a capture they become external event-record nodes
  auto rec = [&](cudaEvent_t e) {
    return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
  };
  CK(rec(D->ev[0]));
  // 1) shared prefixes (boundary states), in creation order (parents first)
  for (size_t m = 0; m < P->mats.size(); m++) {
    const MatNode &M = P->mats[m];
    if (M.mode == QW_MODE_TABLEAU) {
      const DeviceState::TabLaunch &L = D->tab_mat_launches[D->tab_launch_of_mat[m]];
      launch_tab(L.a, L.n_tasks, s);
      nl += 1;
      // Table II STAB -> SV: the statevectors its consumers continue from
      for (uint32_t md = 0; md < 2; md++)
        if (D->mat_export[md][m]) {
          launch_stab_export(D->mat_buf[m], M.n, D->mat_basis[m], md == QW_MODE_SV_FP64,
                             std::max<uint32_t>(M.n, SV_G), D->mat_export[md][m], P->eng->sm_count, s);
          nl += 2;
        }
      continue;
    }
    if (!D->mat_batches.empty()) continue;  // statevector boundaries run in the batches below
    const bool fp64 = M.mode == QW_MODE_SV_FP64;
    const SvTables &T = fp64 ? D->t64 : D->t32;
    const void *psrc = nullptr;
    if (M.parent >= 0) {
      const MatNode &PM = P->mats[M.parent];
      if (PM.mode == M.mode) psrc = D->mat_buf[M.parent];
      else psrc = D->mat_export[M.mode][M.parent];
    }
    if (D->mat_dense[m]) {
      const size_t n_amp = (size_t)1 << M.n_eff;
      if (psrc) launch_copy(psrc, D->mat_buf[m], sv_state_bytes(fp64, M.n_eff), s);
      else
        basis_zero_kernel<<<(unsigned)std::min<size_t>((n_amp + 255) / 256, (size_t)P->eng->sm_count * 16), 256, 0,
                            s>>>(D->mat_buf[m], fp64, n_amp);
      dense_prog_run(D->mat_dense[m], D->mat_buf[m], s);
      nl += 1 + dense_prog_blocks(D->mat_dense[m]);
    } else if (M.sv.passes.empty()) {
      if (psrc) launch_copy(psrc, D->mat_buf[m], sv_state_bytes(fp64, M.n_eff), s);
    } else {
      // compensated FP32: the remainder stays in D->rem between the passes
      // and the last pass rounds the state once, into the boundary
      const int ar = fp64 ? SV_AR_PLAIN : D->ar_chain;
      const size_t np = M.sv.passes.size();
      nl += np;
      for (size_t p = 0; p < np; p++) {
        launch_sv_pass(fp64, T, D->mat_pass0[m] + (uint32_t)p, (uint32_t)M.sv.passes[p].q.size(), M.n_eff,
                       p == 0 ? psrc : D->mat_buf[m], D->mat_buf[m], s, ar, chain_src_lo(D, ar, p),
                       chain_dst_lo(D, ar, p, np));
      }
    }
    // the boundary rounded once into the other precision its consumers use
    for (uint32_t md = 0; md < 2; md++)
      if (md != M.mode && D->mat_export[md][m]) {
        const size_t n = (size_t)1 << M.n_eff;
        convert_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(D->mat_buf[m], fp64, D->mat_export[md][m],
                                                                  md == QW_MODE_SV_FP64, n);
        nl += 1;
      }
  }
  if (!D->mat_batches.empty()) {
    for (const DeviceState::MatBatch &B : D->mat_batches) {
      CK(cudaMemsetAsync(B.d_ctr, 0, B.ctr_words * sizeof(unsigned int), s));
      launch_sv_batch(B.fp64, B.fp64 ? D->t64 : D->t32, B.d_jobs, B.d_segs, B.seg_bits, B.total_items, B.k_max,
                      B.d_ctr, EnTables{}, B.grid, s);
      nl += 1;
    }
    // each boundary rounded once into the other precision its consumers use
    for (size_t m = 0; m < P->mats.size(); m++) {
      const MatNode &M = P->mats[m];
      if (M.mode == QW_MODE_TABLEAU) continue;
      for (uint32_t md = 0; md < 2; md++)
        if (md != M.mode && D->mat_export[md][m]) {
          const size_t n = (size_t)1 << M.n_eff;
          convert_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
              D->mat_buf[m], M.mode == QW_MODE_SV_FP64, D->mat_export[md][m], md == QW_MODE_SV_FP64, n);
          nl += 1;
        }
    }
  }
  CK(rec(D->ev[1]));
  // 2) task suffixes, observables
  size_t wi = 0;
  for (auto &W : D->waves) {
    const SvTables &T = W.fp64 ? D->t64 : D->t32;
    CK(rec(D->wave_ev[4 * wi]));
    nl += W.converts.size();
    for (auto &c : W.converts) {
      const TaskPlan &tp = P->tasks[c.first];
      const size_t n = (size_t)1 << tp.n_eff;
      convert_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
          c.second.first, P->mats[tp.src].mode == QW_MODE_SV_FP64, c.second.second, W.fp64, n);
    }
    if (!W.per_pass) {
      if (W.total_items) {
        CK(cudaMemsetAsync(W.d_ctr, 0, W.ctr_words * sizeof(unsigned int), s));
        EnTables et{W.d_en, D->d_classes, D->d_terms, D->d_partials};
        launch_sv_batch(W.fp64, T, W.d_jobs, W.d_segs, W.seg_bits, W.total_items, W.k_max, W.d_ctr, et,
                        W.grid, s, W.ar);
        nl += 1;
      }
    } else {
      // one task per wave, its passes in order (SV_AR_REM: one rounding, at the end)
      nl += W.jobs.size();
      for (size_t i = 0; i < W.jobs.size(); i++) {
        const SvJob &j = W.jobs[i];
        const uint32_t k = j.n - (uint32_t)std::log2((double)j.n_tiles);
        launch_sv_pass(W.fp64, T, j.pass, k, j.n, j.src, j.dst, s, W.ar, chain_src_lo(D, W.ar, i),
                       chain_dst_lo(D, W.ar, i, W.jobs.size()));
      }
    }
    CK(rec(D->wave_ev[4 * wi + 1]));
    if (W.fused_energy) {
      launch_energy_reduce(W.d_en, (uint32_t)W.en.size(), D->d_partials, s);
      nl += 1;
    } else {
      launch_energy(W.fp64, W.d_en, (uint32_t)W.en.size(), W.en_blocks, D->d_classes, D->d_terms,
                    D->d_partials, s);
      if (!W.en.empty()) nl += 2;
    }
    if (!W.src.empty()) nl += W.shots.empty() ? 2 : 3;
    CK(rec(D->wave_ev[4 * wi + 2]));
    launch_sampling(W.fp64, W.d_src, (uint32_t)W.src.size(), W.smp_blocks, D->d_bsum, D->d_blast, D->d_boff,
                    D->d_lastnz, W.d_shots, (uint32_t)W.shots.size(), s);
    CK(rec(D->wave_ev[4 * wi + 3]));
    wi++;
  }
  CK(rec(D->ev[2]));
  // 3) tableau tasks
  for (auto &L : D->tab_task_launches) {
    if (L.frame >= 0) {
      const DeviceState::FrameLaunch &F = D->frame_launches[L.frame];
      launch_tab(F.ref, 1, s);
      launch_frames(F.fa, s);
      nl += 2;
    }
    launch_tab(L.a, L.n_tasks, s);
  }
  nl += D->tab_task_launches.size();
  CK(rec(D->ev[3]));
  P->n_launches = nl;
  CK(cudaGetLastError());
}

void plan_execute(qw_plan *P, void *stream) {
  Engine *E = P->eng;
  if (!E) fail(QW_ERR_STATE, "plan has no engine (created without one, or its engine was destroyed)");
  CK(cudaSetDevice(E->device));
  const auto t0 = std::chrono::steady_clock::now();
  if (!P->dev) {
    prepare(P);
    P->t_upload_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    DeviceState *D = P->dev;
    for (size_t w = 0; w < 4 * D->waves.size(); w++) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      D->wave_ev.push_back(e);
    }
  }
  DeviceState *D = P->dev;
  cudaStream_t s = stream ? (cudaStream_t)stream : D->stream;
  if (P->opts.use_graph) {
    if (!D->gexec) {
      cudaStream_t cs = D->stream;
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      try {
        enqueue(P, cs, true);
      } catch (...) {
        cudaGraph_t g = nullptr;
        if (cudaStreamEndCapture(cs, &g) == cudaSuccess && g) cudaGraphDestroy(g);
        cudaGetLastError();
        throw;
      }
      CK(cudaStreamEndCapture(cs, &D->graph));
      CK(cudaGraphInstantiate(&D->gexec, D->graph, 0));
    }
    CK(cudaGraphLaunch(D->gexec, s));
  } else {
    enqueue(P, s, false);
  }
  P->executed = true;
}

void plan_wait(qw_plan *P) {
  DeviceState *D = P->dev;
  if (!D || !P->eng) fail(QW_ERR_STATE, "qw_wait before qw_execute, or the engine was destroyed");
  CK(cudaSetDevice(P->eng->device));
  CK(cudaEventSynchronize(D->ev[3]));
  CK(cudaGetLastError());
  const uint32_t nt = (uint32_t)P->tasks.size();
  // device error flags of the persistent launches
  for (auto &W : D->waves) {
    if (!W.total_items || W.per_pass) continue;
    unsigned int flag = 0;
    CK(cudaMemcpy(&flag, W.d_ctr + 1, sizeof(flag), cudaMemcpyDeviceToHost));
    if (flag) fail(QW_ERR_DEVICE_TIMEOUT, "a bounded dependency wait of the persistent batch expired");
  }
  for (const DeviceState::MatBatch &B : D->mat_batches) {
    unsigned int flag = 0;
    CK(cudaMemcpy(&flag, B.d_ctr + 1, sizeof(flag), cudaMemcpyDeviceToHost));
    if (flag) fail(QW_ERR_DEVICE_TIMEOUT, "a bounded dependency wait of the boundaries' launch expired");
  }
  for (qw_dense_prog *dp : D->mat_dense)
    if (dp) dense_prog_check(dp);
  std::vector<double> en(2 * (size_t)nt);
  if (nt) CK(cudaMemcpy(en.data(), D->d_energy, en.size() * sizeof(double), cudaMemcpyDeviceToHost));
  P->energy.assign(nt, 0);
  P->norm2.assign(nt, 0);
  for (uint32_t t = 0; t < nt; t++) { P->energy[t] = en[2 * t]; P->norm2[t] = en[2 * t + 1]; }
  P->samples.assign(P->sample_off[nt], 0);
  if (!P->samples.empty())
    CK(cudaMemcpy(P->samples.data(), D->d_samples, P->samples.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  if (D->d_outs) {
    P->outs_suffix.assign(P->outs_off[nt], 0);
    if (!P->outs_suffix.empty())
      CK(cudaMemcpy(P->outs_suffix.data(), D->d_outs, P->outs_suffix.size(), cudaMemcpyDeviceToHost));
    P->outs_mat.assign(P->outs_mat_off.back(), 0);
    if (!P->outs_mat.empty())
      CK(cudaMemcpy(P->outs_mat.data(), D->d_mat_outs, P->outs_mat.size(), cudaMemcpyDeviceToHost));
  }
  float ms = 0;
  cudaEventElapsedTime(&ms, D->ev[0], D->ev[1]);
  P->t_prefix_ms = ms;
  P->t_suffix_ms = P->t_energy_ms = P->t_sample_ms = 0;
  P->batch_ms.assign(D->waves.size(), 0.0);
  for (size_t w = 0; w < D->waves.size(); w++) {
    cudaEventElapsedTime(&ms, D->wave_ev[4 * w], D->wave_ev[4 * w + 1]);
    P->t_suffix_ms += ms;
    P->batch_ms[w] = ms;
    cudaEventElapsedTime(&ms, D->wave_ev[4 * w + 1], D->wave_ev[4 * w + 2]);
    P->t_energy_ms += ms;
    cudaEventElapsedTime(&ms, D->wave_ev[4 * w + 2], D->wave_ev[4 * w + 3]);
    P->t_sample_ms += ms;
  }
  cudaEventElapsedTime(&ms, D->ev[2], D->ev[3]);
  P->t_tab_ms = ms;
  cudaEventElapsedTime(&ms, D->ev[0], D->ev[3]);
  P->t_total_ms = ms;
  P->timed++;
}

void plan_release(qw_plan *P) {
  if (P->dev) {
    if (P->eng) cudaSetDevice(P->eng->device);
    // the plan may have run on a caller's stream: its blocks go back to the
    // engine's cache only once the device has finished with them
    cudaDeviceSynchronize();
    for (qw_dense_prog *dp : P->dev->mat_dense) dense_prog_destroy(dp);
    delete P->dev;
    P->dev = nullptr;
  }
}

void *plan_state_ptr(const qw_plan *P, uint64_t t) {
  return P->dev ? P->dev->task_state[t] : nullptr;
}

bool plan_tableau_keep(const qw_plan *P, uint64_t t, const uint64_t **rows, const uint8_t **sign) {
  if (!P->dev || t >= P->dev->tab_keep.size() || !P->dev->tab_keep[t].first) return false;
  *rows = P->dev->tab_keep[t].first;
  *sign = P->dev->tab_keep[t].second;
  return true;
}

// ---------------------------------------------------------------------------
// engine
// ---------------------------------------------------------------------------
__global__ void bw_probe_kernel(const float4 *a, float4 *b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

// L2 read probe: 64 KB blocks of an L2-resident buffer in hashed order (the
// access pattern of the energy kernel's partner reads: independent blocks
// at scattered places), 16 independent 16-byte loads per thread per block.
// Every block index is reduced modulo the block count, so all loads stay in
// the buffer.
__global__ void l2_probe_kernel(const float4 *__restrict__ buf, uint64_t n_blocks, int iters, float *sink) {
  float acc = 0.f;
  for (int it = 0; it < iters; it++) {
    const uint64_t b = ((((uint64_t)blockIdx.x * iters + it) * 0x9E3779B97F4A7C15ull) >> 20) % n_blocks;
    float4 v[16];
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __ldg(buf + b * 4096 + j * 256 + threadIdx.x);
#pragma unroll
    for (int j = 0; j < 16; j++) acc += (v[j].x + v[j].y) + (v[j].z + v[j].w);
  }
  if (acc == 1.5e30f) sink[0] = acc;  // keeps the loads; the buffer holds zeros
}

double engine_probe_l2(Engine *E) {
  CK(cudaSetDevice(E->device));
  cudaStream_t s = (cudaStream_t)E->stream;
  const size_t bytes = std::min<size_t>((size_t)64 << 20, (size_t)(E->l2_bytes / 2) & ~(size_t)0xFFFF);
  if (bytes < ((size_t)1 << 20)) fail(QW_ERR_UNSUPPORTED, "L2 of %llu bytes is too small to probe", (unsigned long long)E->l2_bytes);
  float4 *buf = nullptr;
  float *sink = nullptr;
  CK(cudaMalloc(&buf, bytes));
  CK(cudaMalloc(&sink, sizeof(float)));
  CK(cudaMemsetAsync(buf, 0, bytes, s));
  const int grid = E->sm_count * 8, iters = 64;
  const uint64_t nb = bytes / (size_t)65536;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int r = 0; r < 4; r++) {
    CK(cudaEventRecord(e0, s));
    l2_probe_kernel<<<grid, 256, 0, s>>>(buf, nb, iters, sink);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (r) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  cudaFree(sink);
  CK(cudaGetLastError());
  return (double)grid * iters * 65536.0 / (best * 1e-3) / 1e9;
}

void engine_init(Engine *E, const qw_engine_opts *o) {
  E->device = o ? o->device : 0;
  CK(cudaSetDevice(E->device));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, E->device));
  E->sm_count = prop.multiProcessorCount;
  E->l2_bytes = prop.l2CacheSize;
  cudaStream_t s;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  E->stream = s;
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  E->store_budget = (o && o->store_budget_bytes) ? o->store_budget_bytes : (uint64_t)(0.4 * fr);
  E->task_budget = (o && o->task_budget_bytes) ? o->task_budget_bytes : (uint64_t)(0.4 * fr);
  if (o && o->hbm_gbs > 0) {
    E->hbm_gbs = o->hbm_gbs;
  } else {
    const size_t n = (size_t)1 << 26;  // 1 GiB of float4 per buffer
    float4 *a = nullptr, *b = nullptr;
    CK(cudaMalloc(&a, n * sizeof(float4)));
    CK(cudaMalloc(&b, n * sizeof(float4)));
    CK(cudaMemsetAsync(a, 0, n * sizeof(float4), s));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r < 4; r++) {
      cudaEventRecord(e0, s);
      bw_probe_kernel<<<E->sm_count * 8, 256, 0, s>>>(a, b, n);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r) best = std::min(best, ms);
    }
    E->hbm_gbs = 2.0 * n * sizeof(float4) / (best * 1e-3) / 1e9;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(a);
    cudaFree(b);
  }
  // kernel attributes are set before any capture
  CK(sv_init_attrs());
  CK(tab_init_attrs());
  CK(dense_init_attrs());
  CK(frame_init_attrs());
  CK(cudaGetLastError());
}

void *Engine::dev_alloc(size_t bytes, size_t *got) {
  const size_t want = (bytes + 511) & ~(size_t)511;
  auto it = free_blocks.lower_bound(want);
  if (it != free_blocks.end() && it->first <= want + want / 4 + 4096) {
    void *p = it->second;
    *got = it->first;
    cached_bytes -= it->first;
    free_blocks.erase(it);
    return p;
  }
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {  // give the cached blocks back and try once more
    cudaGetLastError();
    trim_cache();
    e = cudaMalloc(&p, want);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(QW_ERR_OOM, "device allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
  }
  *got = want;
  return p;
}

void Engine::dev_free(void *p, size_t bytes) {
  free_blocks.insert({bytes, p});
  cached_bytes += bytes;
}

void Engine::trim_cache() {
  if (free_blocks.empty()) return;
  cudaSetDevice(device);
  cudaDeviceSynchronize();
  for (auto &b : free_blocks) cudaFree(b.second);
  free_blocks.clear();
  cached_bytes = 0;
}

void engine_release(Engine *E) {
  cudaSetDevice(E->device);
  E->trim_cache();
  if (E->scratch) cudaFree(E->scratch);
  if (E->d_mlp) cudaFree(E->d_mlp);
  if (E->stream) cudaStreamDestroy((cudaStream_t)E->stream);
}

void *Engine::ensure_scratch(size_t bytes) {
  if (bytes > scratch_bytes) {
    if (scratch) { cudaStreamSynchronize((cudaStream_t)stream); cudaFree(scratch); scratch = nullptr; }
    CK(cudaMalloc(&scratch, bytes));
    scratch_bytes = bytes;
  }
  return scratch;
}

// Autotuner: times one synthetic hardware-efficient layer stack under each
// candidate (tile qubits, contiguous low qubits) and keeps the fastest per
// (qubit count, precision).
TileConfig Engine::tile_config(uint32_t n_eff, bool fp64, int ar, uint32_t mix) {
  const uint32_t key_n = std::min<uint32_t>(n_eff, 26);
  if (fp64 || ar == SV_AR_REM) ar = SV_AR_PLAIN;
  mix &= 1u;
  const uint64_t key = tile_key(n_eff, fp64, ar, mix);
  auto it = tiles.find(key);
  if (it != tiles.end()) return it->second;
  TileConfig best;
  best.k_max = sv_max_tile(ar, fp64);
  best.b = 4;
  best.g = sv_stage_width(ar, fp64);
  CK(cudaSetDevice(device));
  cudaStream_t s = (cudaStream_t)stream;
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> U(0, 6.283185307179586);
  // the tuning circuits of the gate mix: layered (hardware-efficient layers,
  // rotations on every qubit and a CNOT chain, 1 to 4 layers as in a sweep's
  // suffixes; their times are summed) or entangling (a random circuit, half
  // of its gates CNOT / CZ on random pairs)
  std::vector<std::vector<qw_gate>> circuits;
  if (mix == 0) {
    for (int layers = 1; layers <= 4; layers++) {
      std::vector<qw_gate> g;
      for (int l = 0; l < layers; l++) {
        for (uint32_t q = 0; q < key_n; q++) g.push_back({QW_OP_RY, q, 0, 0, U(rng)});
        for (uint32_t q = 0; q < key_n; q++) g.push_back({QW_OP_RZ, q, 0, 0, U(rng)});
        for (uint32_t q = 0; q + 1 < key_n; q++) g.push_back({QW_OP_CNOT, q, q + 1, 0, 0.0});
      }
      circuits.push_back(std::move(g));
    }
  } else {
    std::vector<qw_gate> g;
    for (int i = 0; i < 40 * (int)key_n; i++) {
      const uint32_t a = (uint32_t)(rng() % key_n), b = (uint32_t)((a + 1 + rng() % (key_n - 1)) % key_n);
      const uint32_t r = (uint32_t)(rng() % 4);
      const uint32_t op = r == 0 ? QW_OP_CZ : r == 1 ? QW_OP_CNOT : r == 2 ? QW_OP_RX : QW_OP_RZ;
      g.push_back({op, a, r < 2 ? b : 0, 0, U(rng)});
    }
    circuits.push_back(std::move(g));
  }
  // independent states advanced together, as a wave's tasks are (so that
  // the tail of each pass overlaps the other states' work): up to 8, within 1 GB
  const size_t S = sv_state_bytes(fp64, key_n);
  const uint32_t chains = (uint32_t)std::max<size_t>(1, std::min<size_t>(8, ((size_t)1 << 30) / S));
  void *buf = nullptr;
  CK(cudaMalloc(&buf, S * chains));
  CK(cudaMemsetAsync(buf, 0, S * chains, s));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const uint32_t ks32[3] = {12, 13, 14}, ks64[3] = {11, 12, 13}, bs[3] = {3, 4, 5};
  float best_ms = 1e30f;
  const uint32_t best_cap = best.k_max;
  // a register that fits one tile is timed with that single shape (its
  // per-pass time calibrates the analytic cost model)
  const bool one_tile = key_n <= best.k_max;
  for (int ki = 0; ki < 3; ki++) {
    for (int bi = 0; bi < 3; bi++) {
      TileConfig tc;
      tc.k_max = fp64 ? ks64[ki] : ks32[ki];
      tc.b = bs[bi];
      tc.g = best.g;
      if (one_tile) {
        if (ki || bi) continue;
        tc.k_max = best.k_max;
        tc.b = best.b;
      }
      if (tc.b + 2 > tc.k_max || tc.k_max > best_cap) continue;
      float tot = 0;
      for (const auto &g : circuits) {
        SvProgram pr = fuse_sv(g.data(), g.size(), key_n, tc);
        SvTableBuilder tb(fp64);
        tb.add(pr);
        SvTables T;
        DevArena dar;
        T.passes = dar.upload(tb.passes, s);
        T.stages = dar.upload(tb.stages, s);
        T.ops = fp64 ? (const void *)dar.upload(tb.ops64, s) : (const void *)dar.upload(tb.ops32, s);
        T.ops_lo = fp64 ? nullptr : dar.upload(tb.ops32lo, s);
        T.ph = fp64 ? nullptr : dar.upload(tb.ph, s);
        // timed in the persistent batch kernel that runs the suffixes: each
        // state's passes a chain of jobs (each waiting for the last), the
        // chains interleaved pass by pass
        std::vector<SvJob> jobs;
        uint32_t kmax = 5;
        for (size_t p = 0; p < pr.passes.size(); p++) {
          const uint32_t kp = (uint32_t)pr.passes[p].q.size();
          for (uint32_t c = 0; c < chains; c++) {
            SvJob j{};
            j.src = (char *)buf + (size_t)c * S;
            j.dst = (char *)buf + (size_t)c * S;
            j.pass = (uint32_t)p;
            j.n_tiles = 1u << (key_n - kp);
            j.dep = p ? (int32_t)jobs.size() - (int32_t)chains : -1;
            j.kind = SVJ_PASS;
            j.n = key_n;
            jobs.push_back(j);
          }
          kmax = std::max(kmax, kp);
        }
        const int grid = sv_batch_grid(fp64, kmax, sm_count, ar);
        const uint32_t seg_bits = segment_bits(jobs);
        std::vector<SvSeg> segs;
        build_segments(jobs, jobs.size(), seg_bits, 2ull * (uint64_t)grid, segs);
        const uint32_t total = (uint32_t)(segs.size() << seg_bits);
        const SvJob *dj = dar.upload(jobs, s);
        const SvSeg *dsg = dar.upload(segs, s);
        const size_t ctr_bytes = (2 + jobs.size()) * sizeof(unsigned int);
        unsigned int *ctr = (unsigned int *)dar.alloc(ctr_bytes);
        const EnTables no_energy{};
        for (int r = 0; r < 3; r++) {  // one warm-up, two timed
          CK(cudaMemsetAsync(ctr, 0, ctr_bytes, s));
          cudaEventRecord(e0, s);
          launch_sv_batch(fp64, T, dj, dsg, seg_bits, total, kmax, ctr, no_energy, grid, s, ar);
          cudaEventRecord(e1, s);
          CK(cudaEventSynchronize(e1));
          float ms;
          cudaEventElapsedTime(&ms, e0, e1);
          if (r) tot += ms;
        }
        CK(cudaStreamSynchronize(s));
        dar.release();
      }
      if (tot < best_ms) {
        best_ms = tot;
        best = tc;
      }
    }
  }
  // the analytic cost's calibration (Eq. 2): the chosen shape's time per
  // pass on one state, its passes launched one by one, as the cost probe
  // times the segments of one task
  {
    float tot = 0;
    size_t n_passes = 0;
    for (const auto &g : circuits) {
      SvProgram pr = fuse_sv(g.data(), g.size(), key_n, best);
      SvTableBuilder tb(fp64);
      tb.add(pr);
      SvTables T;
      DevArena dar;
      T.passes = dar.upload(tb.passes, s);
      T.stages = dar.upload(tb.stages, s);
      T.ops = fp64 ? (const void *)dar.upload(tb.ops64, s) : (const void *)dar.upload(tb.ops32, s);
      T.ops_lo = fp64 ? nullptr : dar.upload(tb.ops32lo, s);
      T.ph = fp64 ? nullptr : dar.upload(tb.ph, s);
      for (int r = 0; r < 3; r++) {  // one warm-up, two timed
        cudaEventRecord(e0, s);
        for (size_t p = 0; p < pr.passes.size(); p++)
          launch_sv_pass(fp64, T, (uint32_t)p, (uint32_t)pr.passes[p].q.size(), key_n, buf, buf, s, ar);
        cudaEventRecord(e1, s);
        CK(cudaEventSynchronize(e1));
        float ms;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r) tot += ms;
      }
      CK(cudaStreamSynchronize(s));
      dar.release();
      n_passes += pr.passes.size();
    }
    best.pass_ns = (double)tot * 1e6 / 2.0 / std::max<double>(1.0, (double)n_passes);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  CK(cudaGetLastError());
  tiles[key] = best;
  tuning_runs++;
  return best;
}

double Engine::predict_log2ns(const float *feat, uint32_t rows, float *out) {
  CK(cudaSetDevice(device));
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<float> x((size_t)rows * QW_MLP_IN);
  for (uint32_t r = 0; r < rows; r++)
    for (int i = 0; i < QW_MLP_IN; i++)
      x[(size_t)r * QW_MLP_IN + i] = (feat[(size_t)r * QW_MLP_IN + i] - cm.mean[i]) / cm.scale[i];
  float *d = (float *)ensure_scratch(sizeof(float) * (x.size() + rows) + 256);
  float *dy = d + x.size();
  CK(cudaMemcpyAsync(d, x.data(), x.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  launch_mlp_forward(d_mlp, d, dy, rows, s);
  CK(cudaMemcpyAsync(out, dy, rows * sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return out[0];
}

void costmodel_train(Engine *E, const float *feat, const float *tgt, uint64_t n, uint32_t epochs,
                     uint32_t batch, float lr, uint64_t seed, float *final_loss) {
  if (n == 0 || batch == 0) fail(QW_ERR_INVALID_ARG, "empty training set");
  CK(cudaSetDevice(E->device));
  cudaStream_t s = (cudaStream_t)E->stream;
  CostModel &cm = E->cm;
  // feature normalization and training ranges
  for (int i = 0; i < QW_MLP_IN; i++) {
    double mu = 0, sq = 0;
    float lo = 1e30f, hi = -1e30f;
    for (uint64_t r = 0; r < n; r++) {
      const float v = feat[r * QW_MLP_IN + i];
      mu += v; sq += (double)v * v;
      lo = std::min(lo, v); hi = std::max(hi, v);
    }
    mu /= n;
    const double var = std::max(0.0, sq / n - mu * mu);
    cm.mean[i] = (float)mu;
    cm.scale[i] = (float)(var > 1e-12 ? std::sqrt(var) : 1.0);
    cm.f_lo[i] = lo;
    cm.f_hi[i] = hi;
  }
  cm.y_lo = *std::min_element(tgt, tgt + n);
  cm.y_hi = *std::max_element(tgt, tgt + n);
  // init (He-uniform), bias of the output at the target mean
  std::mt19937_64 rng(seed);
  cm.params.assign(QW_MLP_PARAMS, 0.f);
  auto fill = [&](int off, int count, int fan_in) {
    const double a = std::sqrt(6.0 / fan_in);
    std::uniform_real_distribution<double> U(-a, a);
    for (int i = 0; i < count; i++) cm.params[off + i] = (float)U(rng);
  };
  fill(0, QW_MLP_IN * QW_MLP_HID, QW_MLP_IN);
  fill(QW_MLP_IN * QW_MLP_HID + QW_MLP_HID, QW_MLP_HID * QW_MLP_HID, QW_MLP_HID);
  fill(QW_MLP_IN * QW_MLP_HID + 2 * QW_MLP_HID + QW_MLP_HID * QW_MLP_HID, QW_MLP_HID, QW_MLP_HID);
  double ym = 0;
  for (uint64_t r = 0; r < n; r++) ym += tgt[r];
  cm.params[QW_MLP_PARAMS - 1] = (float)(ym / n);
  std::vector<float> xn(n * QW_MLP_IN);
  for (uint64_t r = 0; r < n; r++)
    for (int i = 0; i < QW_MLP_IN; i++) xn[r * QW_MLP_IN + i] = (feat[r * QW_MLP_IN + i] - cm.mean[i]) / cm.scale[i];
  DevArena ar;
  float *dX = ar.upload(xn, s);
  std::vector<float> tv(tgt, tgt + n);
  float *dT = ar.upload(tv, s);
  if (E->d_mlp) { cudaFree(E->d_mlp); E->d_mlp = nullptr; }
  CK(cudaMalloc(&E->d_mlp, QW_MLP_PARAMS * sizeof(float)));
  CK(cudaMemcpyAsync(E->d_mlp, cm.params.data(), QW_MLP_PARAMS * sizeof(float), cudaMemcpyHostToDevice, s));
  float *dG = (float *)ar.alloc(QW_MLP_PARAMS * sizeof(float));
  float *dM = (float *)ar.alloc(QW_MLP_PARAMS * sizeof(float));
  float *dV = (float *)ar.alloc(QW_MLP_PARAMS * sizeof(float));
  float *dL = (float *)ar.alloc(sizeof(float));
  float *dS = (float *)ar.alloc(mlp_scratch_floats(batch) * sizeof(float));
  float *dXb = (float *)ar.alloc((size_t)batch * QW_MLP_IN * sizeof(float));
  float *dTb = (float *)ar.alloc((size_t)batch * sizeof(float));
  CK(cudaMemsetAsync(dM, 0, QW_MLP_PARAMS * sizeof(float), s));
  CK(cudaMemsetAsync(dV, 0, QW_MLP_PARAMS * sizeof(float), s));
  std::vector<uint32_t> perm(n);
  for (uint64_t i = 0; i < n; i++) perm[i] = (uint32_t)i;
  std::vector<float> bx((size_t)batch * QW_MLP_IN), bt(batch);
  uint32_t step = 0;
  for (uint32_t ep = 0; ep < epochs; ep++) {
    std::shuffle(perm.begin(), perm.end(), rng);
    for (uint64_t b0 = 0; b0 < n; b0 += batch) {
      const uint32_t bs = (uint32_t)std::min<uint64_t>(batch, n - b0);
      for (uint32_t i = 0; i < bs; i++) {
        memcpy(&bx[(size_t)i * QW_MLP_IN], &xn[(size_t)perm[b0 + i] * QW_MLP_IN], QW_MLP_IN * sizeof(float));
        bt[i] = tgt[perm[b0 + i]];
      }
      CK(cudaMemcpyAsync(dXb, bx.data(), (size_t)bs * QW_MLP_IN * sizeof(float), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(dTb, bt.data(), (size_t)bs * sizeof(float), cudaMemcpyHostToDevice, s));
      launch_mlp_loss_grad(E->d_mlp, dXb, dTb, bs, dL, dG, dS, s);
      launch_mlp_adam(E->d_mlp, dG, dM, dV, QW_MLP_PARAMS, ++step, lr, 0.9f, 0.999f, 1e-8f, s);
      CK(cudaStreamSynchronize(s));  // bx/bt are reused by the next batch
    }
  }
  // final full-set loss
  float *dSall = (float *)ar.alloc(mlp_scratch_floats((uint32_t)n) * sizeof(float));
  launch_mlp_loss_grad(E->d_mlp, dX, dT, (uint32_t)n, dL, dG, dSall, s);
  float L = 0;
  CK(cudaMemcpyAsync(&L, dL, sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(cm.params.data(), E->d_mlp, QW_MLP_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  ar.release();
  cm.trained = true;
  if (final_loss) *final_loss = L;
}

void costmodel_set(Engine *E, const float *params, const float *mean, const float *scale) {
  CK(cudaSetDevice(E->device));
  E->cm.params.assign(params, params + QW_MLP_PARAMS);
  memcpy(E->cm.mean, mean, sizeof(E->cm.mean));
  memcpy(E->cm.scale, scale, sizeof(E->cm.scale));
  for (int i = 0; i < QW_MLP_IN; i++) { E->cm.f_lo[i] = -1e30f; E->cm.f_hi[i] = 1e30f; }
  if (!E->d_mlp) CK(cudaMalloc(&E->d_mlp, QW_MLP_PARAMS * sizeof(float)));
  CK(cudaMemcpy(E->d_mlp, params, QW_MLP_PARAMS * sizeof(float), cudaMemcpyHostToDevice));
  E->cm.trained = true;
}

// timing probe: runs segments of the workload's statevector tasks on a
// scratch state and records (features, log2 ns)
void costmodel_probe(Engine *E, const Workload &W, float *feat, float *tgt, float *analytic, uint64_t cap,
                     uint64_t *n_rows) {
  CK(cudaSetDevice(E->device));
  cudaStream_t s = (cudaStream_t)E->stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  uint64_t rows = 0;
  std::mt19937_64 rng(777);
  std::vector<qw_gate> buf;
  for (const TaskData &T : W.tasks) {
    if (rows >= cap) break;
    if (T.mode == QW_MODE_TABLEAU || T.n_gates == 0) continue;
    const bool fp64 = T.mode == QW_MODE_SV_FP64;
    const uint32_t n_eff = std::max<uint32_t>(T.n, SV_G);
    // timings of the default FP32 arithmetic (compensated, as the
    // persistent suffix launch runs it)
    const int par = fp64 ? SV_AR_PLAIN : SV_AR_COMP;
    uint64_t n2 = 0;
    for (uint64_t i = 0; i < T.n_gates; i++) n2 += is_two_qubit_op(T.gate(i)->op) ? 1 : 0;
    TileConfig tc = E->tile_config(n_eff, fp64, par, gate_mix(n2, T.n_gates));
    const size_t S = sv_state_bytes(fp64, n_eff);
    void *st = E->ensure_scratch(S);
    CK(cudaMemsetAsync(st, 0, S, s));
    // segments: full list, and a prefix / suffix split at a random point
    const uint64_t c = 1 + rng() % std::max<uint64_t>(1, T.n_gates - 1);
    const std::pair<uint64_t, uint64_t> segs[3] = {{0, T.n_gates}, {0, c}, {c, T.n_gates}};
    for (auto sg : segs) {
      if (rows >= cap || sg.second <= sg.first) continue;
      T.copy_gates(sg.first, sg.second, buf);
      SvProgram pr = fuse_sv(buf.data(), buf.size(), n_eff, tc);
      SvTableBuilder tb(fp64);
      tb.add(pr);
      DevArena ar;
      SvTables Tt;
      Tt.passes = ar.upload(tb.passes, s);
      Tt.stages = ar.upload(tb.stages, s);
      Tt.ops = fp64 ? (const void *)ar.upload(tb.ops64, s) : (const void *)ar.upload(tb.ops32, s);
      Tt.ops_lo = fp64 ? nullptr : ar.upload(tb.ops32lo, s);
      Tt.ph = fp64 ? nullptr : ar.upload(tb.ph, s);
      float best = 1e30f;
      for (int r = 0; r < 3; r++) {
        cudaEventRecord(e0, s);
        for (size_t p = 0; p < pr.passes.size(); p++)
          launch_sv_pass(fp64, Tt, (uint32_t)p, (uint32_t)pr.passes[p].q.size(), n_eff, st, st, s, par);
        cudaEventRecord(e1, s);
        CK(cudaEventSynchronize(e1));
        float ms;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r) best = std::min(best, ms);
      }
      ar.release();
      features_for(T, sg.first, sg.second, 1, tc, 0.0, feat + rows * QW_MLP_IN);
      tgt[rows] = (float)std::log2(std::max(1.0, (double)best * 1e6));
      if (analytic) {
        // the planner's analytic cost: passes x measured time per pass
        const double per = tc.pass_ns > 0 ? tc.pass_ns : 2.0 * (double)S / E->hbm_gbs + E->launch_ns;
        const double ns = (double)pr.passes.size() * per;
        analytic[rows] = (float)std::log2(std::max(1.0, ns));
      }
      rows++;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  *n_rows = rows;
}

}  // namespace qw

// ---------------------------------------------------------------------------
// kernels on caller-owned device buffers
// ---------------------------------------------------------------------------
namespace qw {

template <typename T>
static T *stream_upload(const std::vector<T> &v, cudaStream_t s) {
  T *p = nullptr;
  CK(cudaMallocAsync((void **)&p, std::max<size_t>(16, v.size() * sizeof(T)), s));
  if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return p;
}

qw_status sv_apply_dev(Engine *E, uint32_t mode, uint32_t n, void *state, const qw_gate *gates,
                       uint64_t n_gates, bool init, void *stream) {
  CK(cudaSetDevice(E->device));
  cudaStream_t s = (cudaStream_t)stream;
  const bool fp64 = mode == QW_MODE_SV_FP64;
  // FP32: compensated arithmetic with the remainder kept between passes, so
  // the state is rounded once, by the last pass
  const int ar = fp64 ? SV_AR_PLAIN : SV_AR_REM;
  uint64_t n2 = 0;
  for (uint64_t i = 0; i < n_gates; i++) n2 += is_two_qubit_op(gates[i].op) ? 1 : 0;
  TileConfig tc = E->tile_config(n, fp64, SV_AR_COMP, gate_mix(n2, n_gates));
  SvProgram pr = fuse_sv(gates, n_gates, n, tc);
  if (pr.passes.empty()) {
    if (!init) return QW_OK;
    HostPass hp;
    const uint32_t k = std::min(tc.k_max, n);
    for (uint32_t q = 0; q < k; q++) hp.q.push_back(q);
    hp.b = (n <= tc.k_max) ? n : std::min(tc.b, k - 2);
    pr.passes.push_back(hp);
  }
  SvTableBuilder tb(fp64);
  tb.add(pr);
  SvTables T;
  SvPassDesc *dp = stream_upload(tb.passes, s);
  SvStageDesc *ds = stream_upload(tb.stages, s);
  void *dop = fp64 ? (void *)stream_upload(tb.ops64, s) : (void *)stream_upload(tb.ops32, s);
  float *dlo = fp64 ? nullptr : stream_upload(tb.ops32lo, s);
  float *dph = fp64 ? nullptr : stream_upload(tb.ph, s);
  const size_t np = pr.passes.size();
  void *rem = nullptr;
  if (ar == SV_AR_REM && np > 1) CK(cudaMallocAsync(&rem, sv_state_bytes(false, n), s));
  T.passes = dp;
  T.stages = ds;
  T.ops = dop;
  T.ops_lo = dlo;
  T.ph = dph;
  for (size_t p = 0; p < np; p++)
    launch_sv_pass(fp64, T, (uint32_t)p, (uint32_t)pr.passes[p].q.size(), n,
                   (p == 0 && init) ? nullptr : state, state, s, ar, p > 0 ? rem : nullptr,
                   p + 1 < np ? rem : nullptr);
  CK(cudaGetLastError());
  CK(cudaFreeAsync(dp, s));
  CK(cudaFreeAsync(ds, s));
  if (dph) CK(cudaFreeAsync(dph, s));
  CK(cudaFreeAsync(dop, s));
  if (dlo) CK(cudaFreeAsync(dlo, s));
  if (rem) CK(cudaFreeAsync(rem, s));
  return QW_OK;
}

qw_status sv_energy_dev(Engine *E, uint32_t mode, uint32_t n, const void *state, const qw_pauli_term *terms,
                        uint64_t n_terms, double *energy, double *norm2, void *stream) {
  CK(cudaSetDevice(E->device));
  cudaStream_t s = (cudaStream_t)stream;
  const bool fp64 = mode == QW_MODE_SV_FP64;
  HamLayout H;
  build_energy_layout(terms, n_terms, n, fp64 ? 16u : 8u, &H.chunk_bits, H.classes, H.terms, &H.n_blocks);
  EnClass *dc = stream_upload(H.classes, s);
  EnTerm *dt = stream_upload(H.terms, s);
  double *dout = nullptr, *dpart = nullptr;
  CK(cudaMallocAsync((void **)&dout, 2 * sizeof(double), s));
  CK(cudaMallocAsync((void **)&dpart, 2 * sizeof(double) * H.n_blocks, s));
  EnJob j{};
  j.state = state;
  j.out = dout;
  j.n = n;
  j.chunk_bits = H.chunk_bits;
  j.class_begin = 0;
  j.n_classes = (uint32_t)H.classes.size();
  j.block_begin = 0;
  j.n_blocks = H.n_blocks;
  EnJob *dj = stream_upload(std::vector<EnJob>{j}, s);
  launch_energy(fp64, dj, 1, H.n_blocks, dc, dt, dpart, s);
  double res[2];
  CK(cudaMemcpyAsync(res, dout, sizeof(res), cudaMemcpyDeviceToHost, s));
  CK(cudaFreeAsync(dc, s));
  CK(cudaFreeAsync(dt, s));
  CK(cudaFreeAsync(dout, s));
  CK(cudaFreeAsync(dpart, s));
  CK(cudaFreeAsync(dj, s));
  CK(cudaStreamSynchronize(s));
  *energy = res[0];
  if (norm2) *norm2 = res[1];
  return QW_OK;
}

qw_status sv_sample_dev(Engine *E, uint32_t mode, uint32_t n, const void *state, const double *u,
                        uint32_t shots, uint64_t *out, void *stream) {
  CK(cudaSetDevice(E->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (shots == 0) return QW_OK;
  const bool fp64 = mode == QW_MODE_SV_FP64;
  SmpSource so{};
  so.state = state;
  so.n = n;
  so.n_blocks = (n >= (uint32_t)SMP_BLOCK_BITS) ? (1u << (n - SMP_BLOCK_BITS)) : 1u;
  so.block_begin = 0;
  uint64_t *dres = nullptr;
  CK(cudaMallocAsync((void **)&dres, shots * sizeof(uint64_t), s));
  std::vector<SmpShot> sh(shots);
  for (uint32_t k = 0; k < shots; k++) { sh[k].u = u[k]; sh[k].source = 0; sh[k].out = dres + k; }
  SmpSource *dsrc = stream_upload(std::vector<SmpSource>{so}, s);
  SmpShot *dsh = stream_upload(sh, s);
  double *bsum = nullptr, *boff = nullptr;
  int32_t *blast = nullptr;
  int64_t *lastnz = nullptr;
  CK(cudaMallocAsync((void **)&bsum, so.n_blocks * sizeof(double), s));
  CK(cudaMallocAsync((void **)&boff, (so.n_blocks + 1) * sizeof(double), s));
  CK(cudaMallocAsync((void **)&blast, so.n_blocks * sizeof(int32_t), s));
  CK(cudaMallocAsync((void **)&lastnz, sizeof(int64_t), s));
  launch_sampling(fp64, dsrc, 1, so.n_blocks, bsum, blast, boff, lastnz, dsh, shots, s);
  CK(cudaMemcpyAsync(out, dres, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  for (void *p : {(void *)dres, (void *)dsrc, (void *)dsh, (void *)bsum, (void *)boff, (void *)blast, (void *)lastnz})
    CK(cudaFreeAsync(p, s));
  CK(cudaStreamSynchronize(s));
  return QW_OK;
}

}  // namespace qw

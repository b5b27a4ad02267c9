// C ABI entry points (include/quwarp.h): argument checks, exception-to-status
// conversion, and forwarding to the planner and the engine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "dense.h"
#include "plan.h"

namespace qw {
qw_dense_prog *dense_prog_create(Engine *E, uint32_t mode, uint32_t n, std::vector<DenseBlock> blocks,
                                 uint64_t n_gates, uint32_t engine, uint32_t nacc, std::vector<uint8_t> engines);
void dense_prog_run(qw_dense_prog *p, void *state, void *stream);
qw_status dense_prog_check(qw_dense_prog *p);
void dense_prog_destroy(qw_dense_prog *p);
uint64_t dense_prog_blocks(const qw_dense_prog *p);
qw_dense_prog *dense_prog_autotune(Engine *E, uint32_t mode, uint32_t n, const qw_gate *gates, uint64_t n_gates,
                                   uint32_t kmax, uint32_t engine);
void dense_prog_config(const qw_dense_prog *p, uint32_t *engine, uint32_t *kmax, uint32_t *nacc, double *est_ms);
uint64_t dense_prog_gates(const qw_dense_prog *p);
void build_plan(qw_plan *P, Engine *E, const Workload &W);
void plan_execute(qw_plan *P, void *stream);
void plan_wait(qw_plan *P);
void plan_release(qw_plan *P);
void *plan_state_ptr(const qw_plan *P, uint64_t t);
bool plan_tableau_keep(const qw_plan *P, uint64_t t, const uint64_t **rows, const uint8_t **sign);
void engine_init(Engine *E, const qw_engine_opts *o);
void engine_release(Engine *E);
double engine_probe_l2(Engine *E);
void costmodel_train(Engine *E, const float *feat, const float *tgt, uint64_t n, uint32_t epochs,
                     uint32_t batch, float lr, uint64_t seed, float *final_loss);
void costmodel_set(Engine *E, const float *params, const float *mean, const float *scale);
void costmodel_probe(Engine *E, const Workload &W, float *feat, float *tgt, float *analytic, uint64_t cap,
                     uint64_t *n_rows);
qw_status sv_apply_dev(Engine *E, uint32_t mode, uint32_t n, void *state, const qw_gate *gates,
                       uint64_t n_gates, bool init, void *stream);
qw_status sv_energy_dev(Engine *E, uint32_t mode, uint32_t n, const void *state, const qw_pauli_term *terms,
                        uint64_t n_terms, double *energy, double *norm2, void *stream);
qw_status sv_sample_dev(Engine *E, uint32_t mode, uint32_t n, const void *state, const double *u,
                        uint32_t shots, uint64_t *out, void *stream);

static thread_local std::string g_last_error;
void set_last_error(const std::string &m) { g_last_error = m; }
}  // namespace qw

using namespace qw;

#define QW_GUARD(body)                               \
  try {                                              \
    qw::set_last_error("");                          \
    body;                                            \
    return QW_OK;                                    \
  } catch (const qw::Error &e_) {                    \
    qw::set_last_error(e_.msg);                      \
    return e_.code;                                  \
  } catch (const std::bad_alloc &) {                 \
    qw::set_last_error("host allocation failed");    \
    return QW_ERR_OOM;                               \
  } catch (const std::exception &e_) {               \
    qw::set_last_error(e_.what());                   \
    return QW_ERR_INVALID_ARG;                       \
  } catch (...) {                                    \
    qw::set_last_error("unknown internal error");    \
    return QW_ERR_INVALID_ARG;                       \
  }

extern "C" {

const char *qw_last_error(void) { return qw::g_last_error.c_str(); }

qw_status qw_engine_create(const qw_engine_opts *opts, qw_engine **out) {
  QW_GUARD({
    if (!out) fail(QW_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || n_dev == 0)
      fail(QW_ERR_CUDA, "no CUDA device available");
    if (opts && (opts->device < 0 || opts->device >= n_dev))
      fail(QW_ERR_INVALID_ARG, "device %d out of range (%d devices)", opts->device, n_dev);
    qw_engine *e = new qw_engine();
    try {
      engine_init(&e->e, opts);
    } catch (...) {
      delete e;
      throw;
    }
    *out = e;
  })
}

void qw_engine_destroy(qw_engine *e) {
  if (!e) return;
  // plans still alive lose their device state and become host-only objects
  for (qw_plan *p : e->e.plans) {
    try { plan_release(p); } catch (...) {}
    p->eng = nullptr;
  }
  e->e.plans.clear();
  try { engine_release(&e->e); } catch (...) {}
  delete e;
}

qw_status qw_engine_info(const qw_engine *e, double *hbm_gbs, int32_t *sm_count, uint64_t *l2_bytes) {
  QW_GUARD({
    if (!e) fail(QW_ERR_INVALID_ARG, "engine is NULL");
    if (hbm_gbs) *hbm_gbs = e->e.hbm_gbs;
    if (sm_count) *sm_count = e->e.sm_count;
    if (l2_bytes) *l2_bytes = e->e.l2_bytes;
  })
}

static qw_status put_json(const std::string &s, char *buf, size_t cap, size_t *needed);

// the GPU model a tuning belongs to (tile shapes are measured on it)
static std::string device_tag(int dev) {
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return "unknown";
  std::string nm = strf("%s sm_%d%d %d SMs", pr.name, pr.major, pr.minor, pr.multiProcessorCount);
  for (char &c : nm)
    if (c == '"' || c == '\\') c = ' ';
  return nm;
}

qw_status qw_engine_tuning_json(const qw_engine *e, char *buf, size_t cap, size_t *needed) {
  if (!e) { set_last_error("engine is NULL"); return QW_ERR_INVALID_ARG; }
  set_last_error("");
  std::string s = strf("{\"type\":\"QuWARP:Tuning\",\"device\":\"%s\",\"tuning_runs\":%llu,\"tiles\":[",
                       device_tag(e->e.device).c_str(), (unsigned long long)e->e.tuning_runs);
  bool first = true;
  for (const auto &kv : e->e.tiles) {
    const uint64_t k = kv.first;
    const TileConfig &t = kv.second;
    s += strf("%s{\"n\":%llu,\"mix\":%llu,\"arith\":%llu,\"fp64\":%llu,\"k\":%u,\"b\":%u,\"g\":%u,"
              "\"pass_ns\":%.17g}",
              first ? "" : ",", (unsigned long long)(k >> 4), (unsigned long long)((k >> 3) & 1u),
              (unsigned long long)((k >> 1) & 3u), (unsigned long long)(k & 1u), t.k_max, t.b, t.g, t.pass_ns);
    first = false;
  }
  s += "]}";
  return put_json(s, buf, cap, needed);
}

// JSON text without the whitespace outside strings (a record may have been
// pretty-printed since qw_engine_tuning_json wrote it)
static std::string json_compact(const char *json) {
  std::string out;
  bool in_str = false, esc = false;
  for (const char *c = json; *c; c++) {
    if (in_str) {
      out += *c;
      if (esc) esc = false;
      else if (*c == '\\') esc = true;
      else if (*c == '"') in_str = false;
    } else if (*c == '"') {
      in_str = true;
      out += *c;
    } else if (*c != ' ' && *c != '\t' && *c != '\n' && *c != '\r') {
      out += *c;
    }
  }
  return out;
}

static void load_tuning(qw_engine *e, const char *json) {
  const std::string s = json_compact(json);
  const std::string dev = "\"device\":\"" + device_tag(e->e.device) + "\"";
  if (s.find("\"type\":\"QuWARP:Tuning\"") == std::string::npos)
    fail(QW_ERR_INVALID_ARG, "not a tuning record of this library");
  if (s.find(dev) == std::string::npos)
    fail(QW_ERR_INVALID_ARG, "the tuning was measured on another GPU model");
  std::map<uint64_t, TileConfig> got;
  size_t pos = s.find("\"tiles\":[");
  while (pos != std::string::npos && (pos = s.find("{\"n\":", pos)) != std::string::npos) {
    unsigned long long n = 0, mix = 0, ar = 0, f64 = 0;
    unsigned k = 0, b = 0, g = 0;
    double pns = 0;
    if (sscanf(s.c_str() + pos,
               "{\"n\":%llu,\"mix\":%llu,\"arith\":%llu,\"fp64\":%llu,\"k\":%u,\"b\":%u,\"g\":%u,"
               "\"pass_ns\":%lf}",
               &n, &mix, &ar, &f64, &k, &b, &g, &pns) != 8)
      fail(QW_ERR_INVALID_ARG, "malformed tile entry at offset %zu", pos);
    const uint32_t kcap = sv_max_tile((int)ar, f64 != 0);
    const uint32_t gw = sv_stage_width((int)ar, f64 != 0);
    if (n < 1 || n > QW_SV_MAX_QUBITS || mix > 1 || ar > SV_AR_COMP || f64 > 1 || k < SV_G + 1 || k > kcap ||
        b + 2 > k || g != gw || !(pns >= 0))
      fail(QW_ERR_INVALID_ARG, "tile entry out of range at offset %zu", pos);
    TileConfig t;
    t.k_max = k;
    t.b = b;
    t.g = g;
    t.pass_ns = pns;
    got[Engine::tile_key((uint32_t)n, f64 != 0, (int)ar, (uint32_t)mix)] = t;
    pos++;
  }
  for (auto &kv : got) e->e.tiles[kv.first] = kv.second;
}

qw_status qw_engine_tuning_load(qw_engine *e, const char *json) {
  QW_GUARD({
    if (!e || !json) fail(QW_ERR_INVALID_ARG, "NULL argument");
    load_tuning(e, json);
  })
}

qw_status qw_workload_create(qw_workload **out) {
  QW_GUARD({
    if (!out) fail(QW_ERR_INVALID_ARG, "out is NULL");
    *out = new qw_workload();
  })
}

void qw_workload_destroy(qw_workload *w) { delete w; }

static void validate_gate(const qw_gate &g, uint32_t mode, uint32_t n, uint64_t idx) {
  const bool two = is_two_qubit_op(g.op);
  if (g.q0 >= n) fail(QW_ERR_INVALID_ARG, "gate %llu: qubit %u out of range (n=%u)", (unsigned long long)idx, g.q0, n);
  if (two && (g.q1 >= n || g.q1 == g.q0))
    fail(QW_ERR_INVALID_ARG, "gate %llu: bad second qubit %u", (unsigned long long)idx, g.q1);
  if (!std::isfinite(g.theta)) fail(QW_ERR_INVALID_ARG, "gate %llu: non-finite parameter", (unsigned long long)idx);
  const bool known = (g.op >= QW_OP_H && g.op <= QW_OP_PHASE) || two || is_barrier_op(g.op);
  if (!known) fail(QW_ERR_INVALID_ARG, "gate %llu: unknown op %u", (unsigned long long)idx, g.op);
  if (mode == QW_MODE_TABLEAU) {
    if (!is_clifford_op(g.op)) fail(QW_ERR_INVALID_ARG, "gate %llu: op %u is not a tableau (Clifford) op", (unsigned long long)idx, g.op);
    if (is_barrier_op(g.op) && g.theta != 0.0 && g.theta != 1.0)
      fail(QW_ERR_INVALID_ARG, "gate %llu: outcome bit must be 0 or 1", (unsigned long long)idx);
  } else if (is_barrier_op(g.op)) {
    fail(QW_ERR_UNSUPPORTED, "gate %llu: MEASURE/RESET are supported in tableau mode only", (unsigned long long)idx);
  }
}

qw_status qw_workload_add_task(qw_workload *w, const qw_task *t, uint64_t *task_id) {
  QW_GUARD({
    if (!w || !t) fail(QW_ERR_INVALID_ARG, "NULL argument");
    if (t->mode > QW_MODE_TABLEAU) fail(QW_ERR_INVALID_ARG, "unknown mode %u", t->mode);
    const uint32_t n = t->n_qubits;
    if (t->mode == QW_MODE_TABLEAU) {
      if (n < 1 || n > QW_TABLEAU_MAX_QUBITS) fail(QW_ERR_INVALID_ARG, "tableau qubits %u outside [1, %d]", n, QW_TABLEAU_MAX_QUBITS);
      if (t->n_terms || t->shots) fail(QW_ERR_INVALID_ARG, "tableau tasks take no energy terms or shots");
    } else {
      if (n < 1 || n > QW_SV_MAX_QUBITS) fail(QW_ERR_INVALID_ARG, "statevector qubits %u outside [1, %d]", n, QW_SV_MAX_QUBITS);
    }
    if (t->n_spans && !t->spans) fail(QW_ERR_INVALID_ARG, "spans is NULL");
    if (t->n_terms && !t->terms) fail(QW_ERR_INVALID_ARG, "terms is NULL");
    if (t->shots && !t->uniforms) fail(QW_ERR_INVALID_ARG, "uniforms is NULL");
    TaskData d;
    d.mode = t->mode;
    d.n = n;
    d.flags = t->flags;
    d.shots = t->shots;
    uint64_t total = 0;
    for (uint32_t s = 0; s < t->n_spans; s++) {
      const qw_gate_span &sp = t->spans[s];
      if (sp.n_gates && !sp.gates) fail(QW_ERR_INVALID_ARG, "span %u has NULL gates", s);
      const auto key = std::make_tuple(sp.gates, sp.n_gates, t->mode, n);
      if (!w->validated.count(key)) {
        for (uint64_t i = 0; i < sp.n_gates; i++) validate_gate(sp.gates[i], t->mode, n, total + i);
        w->validated.insert(key);
      }
      if (sp.n_gates) {
        d.spans.push_back({sp.gates, sp.n_gates});
        total += sp.n_gates;
        d.span_end.push_back(total);
      }
    }
    d.n_gates = total;
    const uint64_t mask = (n >= 64) ? ~0ull : ((1ull << n) - 1);
    for (uint64_t k = 0; k < t->n_terms; k++) {
      const qw_pauli_term &p = t->terms[k];
      if ((p.xmask | p.zmask) & ~mask) fail(QW_ERR_INVALID_ARG, "term %llu acts outside the %u qubits", (unsigned long long)k, n);
      if (!std::isfinite(p.coef)) fail(QW_ERR_INVALID_ARG, "term %llu: non-finite coefficient", (unsigned long long)k);
      d.terms.push_back(p);
    }
    for (uint32_t k = 0; k < t->shots; k++) {
      const double u = t->uniforms[k];
      if (!(u >= 0.0 && u < 1.0)) fail(QW_ERR_INVALID_ARG, "uniform %u outside [0,1)", k);
      d.uniforms.push_back(u);
    }
    w->w.tasks.push_back(std::move(d));
    if (task_id) *task_id = w->w.tasks.size() - 1;
  })
}

void qw_plan_opts_default(qw_plan_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->reuse = 1;
  o->batched = 1;
  o->legality = 1;
  o->cost_model = QW_COST_ANALYTIC;
  o->delta_frac = 0.10;
  o->min_group = 2;
  o->min_prefix_gates = 1;
  o->min_prefix_cost_ns = 0.0;
  o->use_graph = 1;
  o->fault_injection = 0;
  o->fuse_energy = 0;
  o->pauli_frames = 1;
  o->handoff = 1;
  o->prefix_fp64 = 0;
  o->dense_boundaries = 0;
  o->fp32_arith = QW_FP32_AUTO;
}

qw_status qw_plan_create(qw_engine *e, const qw_workload *w, const qw_plan_opts *o, qw_plan **out) {
  QW_GUARD({
    if (!w || !out) fail(QW_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    qw_plan *p = new qw_plan();
    if (o) p->opts = *o; else qw_plan_opts_default(&p->opts);
    if (p->opts.delta_frac < 0 || !std::isfinite(p->opts.delta_frac)) { delete p; fail(QW_ERR_INVALID_ARG, "delta_frac must be >= 0"); }
    if (p->opts.cost_model != QW_COST_ANALYTIC && p->opts.cost_model != QW_COST_MLP) { delete p; fail(QW_ERR_INVALID_ARG, "unknown cost model"); }
    p->eng = e ? &e->e : nullptr;
    try {
      if (e) cudaSetDevice(e->e.device);
      build_plan(p, p->eng, w->w);
    } catch (...) {
      delete p;
      throw;
    }
    if (p->eng) p->eng->plans.insert(p);
    *out = p;
  })
}

void qw_plan_destroy(qw_plan *p) {
  if (!p) return;
  if (p->eng) p->eng->plans.erase(p);
  try { plan_release(p); } catch (...) {}
  delete p;
}

qw_status qw_execute(qw_plan *p, void *stream) {
  QW_GUARD({
    if (!p) fail(QW_ERR_INVALID_ARG, "plan is NULL");
    plan_execute(p, stream);
  })
}

qw_status qw_wait(qw_plan *p) {
  QW_GUARD({
    if (!p) fail(QW_ERR_INVALID_ARG, "plan is NULL");
    if (!p->executed) fail(QW_ERR_STATE, "qw_wait before qw_execute");
    plan_wait(p);
  })
}

static const TaskPlan &task_of(const qw_plan *p, uint64_t t) {
  if (!p) fail(QW_ERR_INVALID_ARG, "plan is NULL");
  if (t >= p->tasks.size()) fail(QW_ERR_NOT_FOUND, "task %llu does not exist", (unsigned long long)t);
  if (p->timed == 0) fail(QW_ERR_STATE, "no results yet (call qw_execute and qw_wait)");
  return p->tasks[t];
}

qw_status qw_get_energy(const qw_plan *p, uint64_t task, double *energy, double *norm2) {
  QW_GUARD({
    const TaskPlan &tp = task_of(p, task);
    if (tp.ham < 0) fail(QW_ERR_NOT_FOUND, "task %llu has no energy terms", (unsigned long long)task);
    if (energy) *energy = p->energy[task];
    if (norm2) *norm2 = p->norm2[task];
  })
}

qw_status qw_get_samples(const qw_plan *p, uint64_t task, uint64_t *out, size_t cap, size_t *n) {
  QW_GUARD({
    const TaskPlan &tp = task_of(p, task);
    if (n) *n = tp.shots;
    if (cap < tp.shots) fail(QW_ERR_BUFFER_TOO_SMALL, "need %u entries", tp.shots);
    if (tp.shots && !out) fail(QW_ERR_INVALID_ARG, "out is NULL");
    std::copy(p->samples.begin() + p->sample_off[task], p->samples.begin() + p->sample_off[task + 1], out);
  })
}

qw_status qw_get_syndrome(const qw_plan *p, uint64_t task, uint8_t *bits, size_t cap, size_t *n_bits) {
  QW_GUARD({
    const TaskPlan &tp = task_of(p, task);
    if (tp.mode != QW_MODE_TABLEAU) fail(QW_ERR_NOT_FOUND, "task %llu is not a tableau task", (unsigned long long)task);
    if (n_bits) *n_bits = tp.total_outs;
    if (cap < tp.total_outs) fail(QW_ERR_BUFFER_TOO_SMALL, "need %u bytes", tp.total_outs);
    if (tp.total_outs && !bits) fail(QW_ERR_INVALID_ARG, "bits is NULL");
    // outcomes of the materialized chain from the root, then the task's own
    std::vector<int> chain;
    for (int m = tp.src; m >= 0; m = p->mats[m].parent) chain.push_back(m);
    size_t o = 0;
    for (auto it = chain.rbegin(); it != chain.rend(); ++it) {
      const int m = *it;
      for (uint32_t i = p->outs_mat_off[m]; i < p->outs_mat_off[m + 1]; i++) bits[o++] = p->outs_mat[i];
    }
    for (uint32_t i = p->outs_off[task]; i < p->outs_off[task + 1]; i++) bits[o++] = p->outs_suffix[i];
  })
}

qw_status qw_get_state(const qw_plan *p, uint64_t task, void *host_dst, size_t bytes) {
  QW_GUARD({
    const TaskPlan &tp = task_of(p, task);
    if (tp.mode == QW_MODE_TABLEAU) fail(QW_ERR_NOT_FOUND, "tableau tasks have no amplitudes");
    if (!(tp.flags & QW_TASK_KEEP_STATE) && !(tp.sv.passes.empty() && tp.src >= 0))
      fail(QW_ERR_NOT_FOUND, "task %llu was not submitted with QW_TASK_KEEP_STATE", (unsigned long long)task);
    const size_t es = (tp.mode == QW_MODE_SV_FP64) ? 16 : 8;
    const size_t want = es << tp.n;
    if (bytes != want) fail(QW_ERR_INVALID_ARG, "state of task %llu has %zu bytes", (unsigned long long)task, want);
    if (!host_dst) fail(QW_ERR_INVALID_ARG, "host_dst is NULL");
    if (!p->eng || !plan_state_ptr(p, task)) fail(QW_ERR_STATE, "the plan's device memory was released");
    cudaSetDevice(p->eng->device);
    // padded qubits (n < 5) stay |0>: the state is the first 2^n amplitudes
    if (cudaMemcpy(host_dst, plan_state_ptr(p, task), want, cudaMemcpyDeviceToHost) != cudaSuccess)
      fail(QW_ERR_CUDA, "state copy failed");
  })
}

qw_status qw_get_stabilizers(const qw_plan *p, uint64_t task, uint8_t *x, uint8_t *z, uint8_t *sign,
                             size_t n_qubits) {
  QW_GUARD({
    const TaskPlan &tp = task_of(p, task);
    if (tp.mode != QW_MODE_TABLEAU) fail(QW_ERR_INVALID_ARG, "task %llu is not a tableau task", (unsigned long long)task);
    if (!(tp.flags & QW_TASK_KEEP_STATE))
      fail(QW_ERR_NOT_FOUND, "task %llu was not submitted with QW_TASK_KEEP_STATE", (unsigned long long)task);
    if (n_qubits != tp.n) fail(QW_ERR_INVALID_ARG, "task %llu has %u qubits", (unsigned long long)task, tp.n);
    if (!x || !z || !sign) fail(QW_ERR_INVALID_ARG, "NULL output");
    const uint64_t *rows = nullptr;
    const uint8_t *sg = nullptr;
    if (!p->eng || !p->executed || !plan_tableau_keep(p, task, &rows, &sg))
      fail(QW_ERR_STATE, "the plan has not been executed, or its device memory was released");
    const uint32_t n = tp.n;
    const uint32_t W = (n + 63) / 64;
    std::vector<uint64_t> hr((size_t)2 * n * 2 * W);
    std::vector<uint8_t> hs(2 * (size_t)n);
    cudaSetDevice(p->eng->device);
    if (cudaMemcpy(hr.data(), rows, hr.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(hs.data(), sg, hs.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      fail(QW_ERR_CUDA, "tableau copy failed");
    stabilizers_from_inverse(n, hr.data(), hs.data(), x, z, sign);
  })
}

static qw_status put_json(const std::string &s, char *buf, size_t cap, size_t *needed) {
  if (needed) *needed = s.size() + 1;
  if (!buf || cap < s.size() + 1) {
    set_last_error("buffer too small");
    return QW_ERR_BUFFER_TOO_SMALL;
  }
  memcpy(buf, s.c_str(), s.size() + 1);
  return QW_OK;
}

qw_status qw_explain_json(const qw_plan *p, char *buf, size_t cap, size_t *needed) {
  if (!p) { set_last_error("plan is NULL"); return QW_ERR_INVALID_ARG; }
  set_last_error("");
  return put_json(p->explain, buf, cap, needed);
}

qw_status qw_cost_record_json(const qw_plan *p, char *buf, size_t cap, size_t *needed) {
  if (!p) { set_last_error("plan is NULL"); return QW_ERR_INVALID_ARG; }
  set_last_error("");
  std::string s = strf(
      "{\"type\":\"QuWARP:CostRecord\",\"planning_ms\":%.6f,\"estimated_direct_ms\":%.6f,"
      "\"estimated_plan_ms\":%.6f,\"estimated_speedup\":%.4f,\"executions\":%d,"
      "\"upload_ms\":%.6f,\"prefix_ms\":%.6f,\"suffix_ms\":%.6f,\"energy_ms\":%.6f,"
      "\"sampling_ms\":%.6f,\"tableau_tasks_ms\":%.6f,\"device_total_ms\":%.6f,"
      "\"kernel_launches\":%llu,\"h2d_bytes\":%llu,\"d2h_bytes\":%llu,"
      "\"batch_alg_bytes\":%.0f,\"energy_alg_bytes\":%.0f,\"energy_l2_bytes\":%.0f,\"prefix_alg_bytes\":%.0f,"
      "\"batch_alg_flops\":%.0f,\"prefix_alg_flops\":%.0f,"
      "\"energy_fused\":%s,\"fp32_arith\":\"%s\","
      "\"artifacts\":%zu,\"artifact_bytes\":%llu,\"batch_ms\":[",
      p->planning_ns * 1e-6, p->est_direct_ns * 1e-6, p->est_plan_ns * 1e-6,
      p->est_plan_ns > 0 ? p->est_direct_ns / p->est_plan_ns : 1.0, p->timed, p->t_upload_ms,
      p->t_prefix_ms, p->t_suffix_ms, p->t_energy_ms, p->t_sample_ms, p->t_tab_ms, p->t_total_ms,
      (unsigned long long)p->n_launches, (unsigned long long)p->h2d_bytes,
      (unsigned long long)p->d2h_bytes, p->batch_alg_bytes, p->energy_alg_bytes, p->energy_l2_bytes, p->prefix_alg_bytes,
      p->batch_alg_flops, p->prefix_alg_flops,
      p->energy_fused ? "true" : "false", p->fp32_compensated ? "compensated" : "plain",
      p->mats.size(), [&] {
        unsigned long long b = 0;
        for (auto &m : p->mats) b += m.bytes;
        return b;
      }());
  for (size_t i = 0; i < p->batch_ms.size(); i++) s += strf(i ? ",%.6f" : "%.6f", p->batch_ms[i]);
  s += "],\"wave_tiles\":[";
  for (size_t i = 0; i < p->wave_tiles.size(); i++)
    s += strf(i ? ",[%u,%u]" : "[%u,%u]", p->wave_tiles[i].first, p->wave_tiles[i].second);
  s += "],\"dense_boundaries\":[";
  for (size_t i = 0; i < p->dense_choices.size(); i++) {
    const DenseChoice &c = p->dense_choices[i];
    const char *eng = c.engine == QW_DENSE_TENSOR ? "tensor" : c.engine == QW_DENSE_SIMT ? "cuda_cores" : "mixed";
    s += strf("%s{\"artifact\":%d,\"used\":%s,\"engine\":\"%s\",\"fusion_width\":%u,\"blocks\":%u,"
              "\"estimated_ms\":%.6f,\"pass_kernels_ms\":%.6f,\"dense_ms\":%.6f,\"over_accuracy_budget\":%s}",
              i ? "," : "", c.mat, c.used ? "true" : "false", eng, c.width, c.blocks, c.est_ms, c.pass_ms,
              c.dense_ms, c.over_budget ? "true" : "false");
  }
  s += "]}";
  return put_json(s, buf, cap, needed);
}

qw_status qw_sha256(const void *data, size_t len, uint8_t out[32]) {
  QW_GUARD({
    if ((!data && len) || !out) fail(QW_ERR_INVALID_ARG, "NULL argument");
    sha256(data, len, out);
  })
}

qw_status qw_fingerprint(uint32_t n_qubits, uint32_t mode, const qw_gate *gates, uint64_t n_gates,
                         uint8_t out[32]) {
  QW_GUARD({
    if ((!gates && n_gates) || !out) fail(QW_ERR_INVALID_ARG, "NULL argument");
    TaskData t;
    t.n = n_qubits;
    t.mode = mode;
    if (n_gates) {
      t.spans.push_back({gates, n_gates});
      t.span_end.push_back(n_gates);
    }
    t.n_gates = n_gates;
    fingerprint(n_qubits, mode, t, 0, n_gates, out);
  })
}

qw_status qw_reuse_decision(const qw_cost_tuple *c, int32_t *reuse, double *lhs, double *rhs) {
  QW_GUARD({
    if (!c || !reuse) fail(QW_ERR_INVALID_ARG, "NULL argument");
    if (c->n_tasks < 0) fail(QW_ERR_INVALID_ARG, "negative task count");
    const double l = (c->n_tasks - 1.0) * c->c_prefix;
    const double r = c->c_materialize + c->n_tasks * (c->c_reload + c->c_handoff) + c->delta;
    *reuse = l > r ? 1 : 0;
    if (lhs) *lhs = l;
    if (rhs) *rhs = r;
  })
}

qw_status qw_legality_check(const qw_artifact_desc *a, uint32_t target_backend,
                            const uint8_t expected_provenance[32], int32_t *legal, qw_refusal *out) {
  QW_GUARD({
    if (!a || !legal || !out) fail(QW_ERR_INVALID_ARG, "NULL argument");
    *legal = legality(*a, target_backend, expected_provenance, out) ? 1 : 0;
  })
}

// ---- learned cost model ---------------------------------------------------------
qw_status qw_mlp_forward_dev(const float *params, const float *x, float *y, uint32_t batch, void *stream) {
  QW_GUARD({
    if (!params || (batch && (!x || !y))) fail(QW_ERR_INVALID_ARG, "NULL argument");
    launch_mlp_forward(params, x, y, batch, stream);
    if (cudaGetLastError() != cudaSuccess) fail(QW_ERR_CUDA, "mlp forward launch failed");
  })
}

qw_status qw_mlp_loss_grad_dev(const float *params, const float *x, const float *target, uint32_t batch,
                               float *loss, float *grad, void *stream) {
  QW_GUARD({
    if (!params || !grad || !loss || (batch && (!x || !target))) fail(QW_ERR_INVALID_ARG, "NULL argument");
    if (batch == 0) fail(QW_ERR_INVALID_ARG, "empty batch");
    float *scratch = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMallocAsync((void **)&scratch, mlp_scratch_floats(batch) * sizeof(float), s) != cudaSuccess)
      fail(QW_ERR_OOM, "scratch allocation failed");
    launch_mlp_loss_grad(params, x, target, batch, loss, grad, scratch, stream);
    cudaFreeAsync(scratch, s);
    if (cudaGetLastError() != cudaSuccess) fail(QW_ERR_CUDA, "mlp backward launch failed");
  })
}

qw_status qw_mlp_adam_dev(float *params, const float *grad, float *m, float *v, uint32_t n_params,
                          uint32_t t, float lr, float beta1, float beta2, float eps, void *stream) {
  QW_GUARD({
    if (!params || !grad || !m || !v) fail(QW_ERR_INVALID_ARG, "NULL argument");
    if (t < 1) fail(QW_ERR_INVALID_ARG, "Adam step must be >= 1");
    launch_mlp_adam(params, grad, m, v, n_params, t, lr, beta1, beta2, eps, stream);
    if (cudaGetLastError() != cudaSuccess) fail(QW_ERR_CUDA, "adam launch failed");
  })
}

qw_status qw_costmodel_train(qw_engine *e, const float *features, const float *targets, uint64_t n,
                             uint32_t epochs, uint32_t batch, float lr, uint64_t seed, float *final_loss) {
  QW_GUARD({
    if (!e || !features || !targets) fail(QW_ERR_INVALID_ARG, "NULL argument");
    costmodel_train(&e->e, features, targets, n, epochs, batch, lr, seed, final_loss);
  })
}

qw_status qw_costmodel_predict(qw_engine *e, const float *features, uint64_t n, float *out) {
  QW_GUARD({
    if (!e || (n && (!features || !out))) fail(QW_ERR_INVALID_ARG, "NULL argument");
    if (!e->e.cm.trained) fail(QW_ERR_STATE, "cost model not trained");
    if (n) e->e.predict_log2ns(features, (uint32_t)n, out);
  })
}

qw_status qw_costmodel_get(const qw_engine *e, float *params, float *feat_mean, float *feat_scale) {
  QW_GUARD({
    if (!e || !params) fail(QW_ERR_INVALID_ARG, "NULL argument");
    if (!e->e.cm.trained) fail(QW_ERR_STATE, "cost model not trained");
    std::copy(e->e.cm.params.begin(), e->e.cm.params.end(), params);
    if (feat_mean) memcpy(feat_mean, e->e.cm.mean, sizeof(e->e.cm.mean));
    if (feat_scale) memcpy(feat_scale, e->e.cm.scale, sizeof(e->e.cm.scale));
  })
}

qw_status qw_costmodel_set(qw_engine *e, const float *params, const float *feat_mean, const float *feat_scale) {
  QW_GUARD({
    if (!e || !params || !feat_mean || !feat_scale) fail(QW_ERR_INVALID_ARG, "NULL argument");
    costmodel_set(&e->e, params, feat_mean, feat_scale);
  })
}

qw_status qw_costmodel_probe(qw_engine *e, const qw_workload *w, float *features, float *targets,
                             float *analytic_log2ns,
                             uint64_t cap, uint64_t *n_rows) {
  QW_GUARD({
    if (!e || !w || !features || !targets || !n_rows) fail(QW_ERR_INVALID_ARG, "NULL argument");
    costmodel_probe(&e->e, w->w, features, targets, analytic_log2ns, cap, n_rows);
  })
}

qw_status qw_costmodel_features(const qw_engine *e, const qw_workload *w, uint64_t task, uint64_t gate_begin,
                                uint64_t gate_end, uint32_t n_sharing, float out[12]) {
  QW_GUARD({
    if (!w || !out) fail(QW_ERR_INVALID_ARG, "NULL argument");
    if (task >= w->w.tasks.size()) fail(QW_ERR_NOT_FOUND, "no such task");
    const TaskData &t = w->w.tasks[task];
    if (gate_begin > gate_end || gate_end > t.n_gates) fail(QW_ERR_INVALID_ARG, "bad gate range");
    TileConfig tc;
    // tiles of the default arithmetic (compensated FP32)
    tc.k_max = (t.mode == QW_MODE_SV_FP64) ? SV_MAX_TILE_FP64 : SV_MAX_TILE_FP32_COMP;
    tc.b = 4;
    if (e) {
      uint64_t n2 = 0;
      for (uint64_t i = 0; i < t.n_gates; i++) n2 += is_two_qubit_op(t.gate(i)->op) ? 1 : 0;
      auto it = e->e.tiles.find(Engine::tile_key(std::max<uint32_t>(t.n, SV_G), t.mode == QW_MODE_SV_FP64,
                                                 SV_AR_COMP, gate_mix(n2, t.n_gates)));
      if (it != e->e.tiles.end()) tc = it->second;
    }
    features_for(t, gate_begin, gate_end, n_sharing, tc, 0.0, out);
  })
}

// ---- statevector kernels on caller buffers ----------------------------------------
qw_status qw_engine_probe_l2(qw_engine *e, double *l2_read_gbs) {
  QW_GUARD({
    if (!e || !l2_read_gbs) fail(QW_ERR_INVALID_ARG, "NULL argument");
    *l2_read_gbs = engine_probe_l2(&e->e);
  })
}

qw_status qw_sv_apply_dev(qw_engine *e, uint32_t mode, uint32_t n, void *state, const qw_gate *gates,
                          uint64_t n_gates, const int32_t *init, void *stream) {
  QW_GUARD({
    if (!e || !state || (n_gates && !gates)) fail(QW_ERR_INVALID_ARG, "NULL argument");
    if (mode > QW_MODE_SV_FP32) fail(QW_ERR_INVALID_ARG, "statevector modes only");
    if (n < SV_G || n > QW_SV_MAX_QUBITS) fail(QW_ERR_INVALID_ARG, "n must be in [%d, %d] for device buffers", SV_G, QW_SV_MAX_QUBITS);
    for (uint64_t i = 0; i < n_gates; i++) validate_gate(gates[i], mode, n, i);
    qw_status st = sv_apply_dev(&e->e, mode, n, state, gates, n_gates, init && *init == 1, stream);
    if (st != QW_OK) return st;
  })
}

qw_status qw_sv_energy_dev(qw_engine *e, uint32_t mode, uint32_t n, const void *state,
                           const qw_pauli_term *terms, uint64_t n_terms, double *energy, double *norm2,
                           void *stream) {
  QW_GUARD({
    if (!e || !state || (n_terms && !terms) || !energy) fail(QW_ERR_INVALID_ARG, "NULL argument");
    if (mode > QW_MODE_SV_FP32) fail(QW_ERR_INVALID_ARG, "statevector modes only");
    if (n < SV_G || n > QW_SV_MAX_QUBITS) fail(QW_ERR_INVALID_ARG, "n must be in [%d, %d] for device buffers", SV_G, QW_SV_MAX_QUBITS);
    const uint64_t mask = (1ull << n) - 1;
    for (uint64_t k = 0; k < n_terms; k++)
      if ((terms[k].xmask | terms[k].zmask) & ~mask) fail(QW_ERR_INVALID_ARG, "term %llu outside the register", (unsigned long long)k);
    qw_status st = sv_energy_dev(&e->e, mode, n, state, terms, n_terms, energy, norm2, stream);
    if (st != QW_OK) return st;
  })
}

qw_status qw_sv_sample_dev(qw_engine *e, uint32_t mode, uint32_t n, const void *state, const double *uniforms,
                           uint32_t shots, uint64_t *out, void *stream) {
  QW_GUARD({
    if (!e || !state || (shots && (!uniforms || !out))) fail(QW_ERR_INVALID_ARG, "NULL argument");
    if (mode > QW_MODE_SV_FP32) fail(QW_ERR_INVALID_ARG, "statevector modes only");
    if (n < SV_G || n > QW_SV_MAX_QUBITS) fail(QW_ERR_INVALID_ARG, "n must be in [%d, %d] for device buffers", SV_G, QW_SV_MAX_QUBITS);
    for (uint32_t k = 0; k < shots; k++)
      if (!(uniforms[k] >= 0.0 && uniforms[k] < 1.0)) fail(QW_ERR_INVALID_ARG, "uniform %u outside [0,1)", k);
    qw_status st = sv_sample_dev(&e->e, mode, n, state, uniforms, shots, out, stream);
    if (st != QW_OK) return st;
  })
}

// ---- dense blocks ------------------------------------------------------------
static void check_dense_target(uint32_t mode, uint32_t n, uint32_t engine, uint32_t nacc) {
  if (mode > QW_MODE_SV_FP32) fail(QW_ERR_INVALID_ARG, "statevector modes only");
  if (engine == QW_DENSE_TENSOR) {
    if (mode != QW_MODE_SV_FP32) fail(QW_ERR_UNSUPPORTED, "tensor-core dense blocks need an FP32 state");
    if (n < DENSE_TC_MIN_QUBITS || n > QW_SV_MAX_QUBITS)
      fail(QW_ERR_UNSUPPORTED, "tensor-core dense blocks need n in [%u, %d]", DENSE_TC_MIN_QUBITS, QW_SV_MAX_QUBITS);
    if (nacc != 1 && nacc != 2 && nacc != 4) fail(QW_ERR_INVALID_ARG, "nacc must be 1, 2 or 4");
  } else if (engine == QW_DENSE_SIMT || engine == QW_DENSE_AUTO) {
    if (n < 1 || n > QW_SV_MAX_QUBITS) fail(QW_ERR_INVALID_ARG, "n must be in [1, %d]", QW_SV_MAX_QUBITS);
  } else {
    fail(QW_ERR_INVALID_ARG, "unknown dense engine %u", engine);
  }
}

qw_status qw_dense_fuse(const qw_gate *gates, uint64_t n_gates, uint32_t n, uint32_t kmax, uint32_t *k,
                        uint32_t *qubits, double *u, uint64_t cap, uint64_t *n_blocks) {
  QW_GUARD({
    if ((n_gates && !gates) || !n_blocks || (cap && (!k || !qubits || !u))) fail(QW_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || n > QW_SV_MAX_QUBITS) fail(QW_ERR_INVALID_ARG, "n must be in [1, %d]", QW_SV_MAX_QUBITS);
    for (uint64_t i = 0; i < n_gates; i++) validate_gate(gates[i], QW_MODE_SV_FP64, n, i);
    std::vector<DenseBlock> b = fuse_dense(gates, n_gates, kmax);
    *n_blocks = b.size();
    if (cap == 0) return QW_OK;
    if (cap < b.size()) fail(QW_ERR_BUFFER_TOO_SMALL, "%zu blocks, capacity %llu", b.size(), (unsigned long long)cap);
    for (size_t i = 0; i < b.size(); i++) {
      k[i] = b[i].k;
      const uint32_t d = 1u << b[i].k;
      for (uint32_t j = 0; j < DENSE_MAX_QUBITS; j++) qubits[5 * i + j] = j < b[i].k ? b[i].q[j] : 0;
      double *ui = u + 2048 * i;
      std::fill(ui, ui + 2048, 0.0);
      for (uint32_t r = 0; r < d; r++)
        for (uint32_t c = 0; c < d; c++) {
          ui[2 * (r * d + c)] = b[i].u[r * d + c].real();
          ui[2 * (r * d + c) + 1] = b[i].u[r * d + c].imag();
        }
    }
  })
}

// JSON of a fused statevector program (host only; see qw_sv_fuse_json)
static std::string sv_program_json(const SvProgram &pr) {
  static const char *kinds[16] = {"?", "U1", "D1", "?", "CD", "?", "P1", "R", "RX", "RP", "?", "?", "?", "?", "?", "?"};
  auto map_json = [](const uint32_t *cols, uint32_t c, size_t k, const uint32_t *ctl_w) {
    std::string m = "{\"cols\":[";
    for (size_t t = 0; t < k; t++) m += strf("%s%u", t ? "," : "", cols[t]);
    m += strf("],\"c\":%u,\"ctl_w\":[", c);
    for (int t = 0; t < SV_MAX_OUT_CTL; t++) m += strf("%s%u", t ? "," : "", ctl_w[t]);
    return m + "]}";
  };
  std::string js = strf("{\"n\":%u,\"passes\":[", pr.n);
  for (size_t p = 0; p < pr.passes.size(); p++) {
    const HostPass &hp = pr.passes[p];
    js += p ? ",{\"q\":[" : "{\"q\":[";
    for (size_t t = 0; t < hp.q.size(); t++) js += strf("%s%u", t ? "," : "", hp.q[t]);
    js += "],\"ctl_q\":[";
    for (size_t t = 0; t < hp.ctl_q.size(); t++) js += strf("%s%u", t ? "," : "", hp.ctl_q[t]);
    js += strf("],\"b\":%u,\"map\":%s,\"stages\":[", hp.b,
               map_json(hp.mcol, hp.mc, hp.q.size(), hp.ctl_w).c_str());
    for (size_t s = 0; s < hp.stages.size(); s++) {
      const HostStage &hs = hp.stages[s];
      js += strf("%s{\"pos\":[%u,%u,%u,%u,%u],\"map\":%s,\"ops\":[", s ? "," : "", hs.pos[0], hs.pos[1],
                 hs.pos[2], hs.pos[3], hs.pos[4], map_json(hs.mcol, hs.mc, hp.q.size(), hs.ctl_w).c_str());
      for (size_t o = 0; o < hs.ops.size(); o++) {
        const HostOp &op = hs.ops[o];
        js += strf("%s{\"kind\":\"%s\",\"a\":%u,\"b\":%u,\"m\":[", o ? "," : "", kinds[op.kind & 15], op.a, op.b);
        for (int t = 0; t < 8; t++) js += strf("%s%.17g", t ? "," : "", op.m[t]);
        js += "]}";
      }
      js += "]}";
    }
    js += "]}";
  }
  return js + "]}";
}

qw_status qw_sv_fuse_json(const qw_gate *gates, uint64_t n_gates, uint32_t n, uint32_t tile_qubits,
                          uint32_t low_qubits, char *buf, size_t cap, size_t *needed) {
  QW_GUARD({
    if ((n_gates && !gates) || !needed) fail(QW_ERR_INVALID_ARG, "NULL argument");
    if (n < (uint32_t)SV_G || n > QW_SV_MAX_QUBITS) fail(QW_ERR_INVALID_ARG, "n must be in [%d, %d]", SV_G, QW_SV_MAX_QUBITS);
    if (tile_qubits < (uint32_t)SV_G + 1 || tile_qubits > (uint32_t)SV_MAX_TILE_FP32)
      fail(QW_ERR_INVALID_ARG, "tile_qubits must be in [%d, %d]", SV_G + 1, SV_MAX_TILE_FP32);
    if (low_qubits < 1 || low_qubits > tile_qubits - 2) fail(QW_ERR_INVALID_ARG, "low_qubits must be in [1, tile_qubits - 2]");
    for (uint64_t i = 0; i < n_gates; i++) validate_gate(gates[i], QW_MODE_SV_FP64, n, i);
    TileConfig tc;
    tc.k_max = tile_qubits;
    tc.b = low_qubits;
    return put_json(sv_program_json(fuse_sv(gates, n_gates, n, tc)), buf, cap, needed);
  })
}

qw_status qw_dense_prog_create(qw_engine *e, uint32_t mode, uint32_t n, const qw_gate *gates, uint64_t n_gates,
                               uint32_t kmax, uint32_t engine, uint32_t nacc, qw_dense_prog **out) {
  QW_GUARD({
    if (!e || !out || (n_gates && !gates)) fail(QW_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    check_dense_target(mode, n, engine, nacc);
    if (kmax == 1 || kmax > DENSE_MAX_QUBITS) fail(QW_ERR_INVALID_ARG, "kmax must be 0 (autotune) or in [2, 5]");
    for (uint64_t i = 0; i < n_gates; i++) validate_gate(gates[i], mode, n, i);
    if (kmax == 0 || engine == QW_DENSE_AUTO)
      *out = dense_prog_autotune(&e->e, mode, n, gates, n_gates, kmax, engine);
    else
      *out = dense_prog_create(&e->e, mode, n, fuse_dense(gates, n_gates, kmax), n_gates, engine, nacc, {});
  })
}

qw_status qw_dense_prog_create_block(qw_engine *e, uint32_t mode, uint32_t n, const uint32_t *qubits, uint32_t k,
                                     const double *u, uint32_t engine, uint32_t nacc, qw_dense_prog **out) {
  QW_GUARD({
    if (!e || !out || !qubits || !u) fail(QW_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (engine == QW_DENSE_AUTO) fail(QW_ERR_INVALID_ARG, "an explicit block takes a fixed engine");
    check_dense_target(mode, n, engine, nacc);
    if (k < 1 || k > DENSE_MAX_QUBITS || k > n) fail(QW_ERR_INVALID_ARG, "k must be in [1, min(5, n)]");
    DenseBlock b;
    b.k = k;
    uint32_t seen = 0;
    for (uint32_t j = 0; j < k; j++) {
      if (qubits[j] >= n || (seen >> qubits[j] & 1)) fail(QW_ERR_INVALID_ARG, "qubit %u repeated or out of range", qubits[j]);
      seen |= 1u << qubits[j];
      b.q[j] = qubits[j];
    }
    const uint32_t d = 1u << k;
    b.u.resize((size_t)d * d);
    for (size_t i = 0; i < b.u.size(); i++) {
      if (!std::isfinite(u[2 * i]) || !std::isfinite(u[2 * i + 1])) fail(QW_ERR_INVALID_ARG, "non-finite matrix entry");
      b.u[i] = std::complex<double>(u[2 * i], u[2 * i + 1]);
    }
    *out = dense_prog_create(&e->e, mode, n, std::vector<DenseBlock>{b}, 0, engine, nacc, {});
  })
}

qw_status qw_dense_prog_info(const qw_dense_prog *p, uint64_t *n_blocks, uint64_t *n_gates) {
  QW_GUARD({
    if (!p) fail(QW_ERR_INVALID_ARG, "NULL program");
    if (n_blocks) *n_blocks = dense_prog_blocks(p);
    if (n_gates) *n_gates = dense_prog_gates(p);
  })
}

qw_status qw_dense_prog_config(const qw_dense_prog *p, uint32_t *engine, uint32_t *kmax, uint32_t *nacc,
                               double *est_ms) {
  QW_GUARD({
    if (!p) fail(QW_ERR_INVALID_ARG, "NULL program");
    dense_prog_config(p, engine, kmax, nacc, est_ms);
  })
}

qw_status qw_dense_prog_run(qw_dense_prog *p, void *state, void *stream) {
  QW_GUARD({
    if (!p || !state) fail(QW_ERR_INVALID_ARG, "NULL argument");
    dense_prog_run(p, state, stream);
  })
}

qw_status qw_dense_prog_check(qw_dense_prog *p) {
  QW_GUARD({
    if (!p) fail(QW_ERR_INVALID_ARG, "NULL program");
    dense_prog_check(p);
  })
}

void qw_dense_prog_destroy(qw_dense_prog *p) {
  try {
    dense_prog_destroy(p);
  } catch (...) {
  }
}

}  // extern "C"

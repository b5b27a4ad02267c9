// Host planner: workload IR, prefix trie, candidate boundaries, the reuse
// inequality (Eq. 2), the legality guard (Table II), structural fingerprints
// (Eq. 1) and the EXPLAIN trace (Sec. III-A, Sec. IV).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <unordered_map>

#include "plan.h"

namespace qw {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
std::string strf(const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return buf;
}
void fail(qw_status code, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  throw Error{code, buf};
}

// ---------------------------------------------------------------------------
// workload
// ---------------------------------------------------------------------------
const qw_gate *TaskData::gate(uint64_t i) const {
  const size_t s = std::upper_bound(span_end.begin(), span_end.end(), i) - span_end.begin();
  const uint64_t start = s ? span_end[s - 1] : 0;
  return spans[s].g + (i - start);
}
void TaskData::copy_gates(uint64_t b, uint64_t e, std::vector<qw_gate> &out) const {
  out.clear();
  out.reserve(e - b);
  uint64_t i = b;
  while (i < e) {
    const size_t s = std::upper_bound(span_end.begin(), span_end.end(), i) - span_end.begin();
    const uint64_t start = s ? span_end[s - 1] : 0;
    const uint64_t take = std::min(e, span_end[s]) - i;
    const qw_gate *g = spans[s].g + (i - start);
    out.insert(out.end(), g, g + take);
    i += take;
  }
}

// ---------------------------------------------------------------------------
// SHA-256 (FIPS 180-4)
// ---------------------------------------------------------------------------
namespace {
const uint32_t K256[64] = {
    0x428a2f98, 0x71374491, 0xb5c0fbcf, 0xe9b5dba5, 0x3956c25b, 0x59f111f1, 0x923f82a4, 0xab1c5ed5,
    0xd807aa98, 0x12835b01, 0x243185be, 0x550c7dc3, 0x72be5d74, 0x80deb1fe, 0x9bdc06a7, 0xc19bf174,
    0xe49b69c1, 0xefbe4786, 0x0fc19dc6, 0x240ca1cc, 0x2de92c6f, 0x4a7484aa, 0x5cb0a9dc, 0x76f988da,
    0x983e5152, 0xa831c66d, 0xb00327c8, 0xbf597fc7, 0xc6e00bf3, 0xd5a79147, 0x06ca6351, 0x14292967,
    0x27b70a85, 0x2e1b2138, 0x4d2c6dfc, 0x53380d13, 0x650a7354, 0x766a0abb, 0x81c2c92e, 0x92722c85,
    0xa2bfe8a1, 0xa81a664b, 0xc24b8b70, 0xc76c51a3, 0xd192e819, 0xd6990624, 0xf40e3585, 0x106aa070,
    0x19a4c116, 0x1e376c08, 0x2748774c, 0x34b0bcb5, 0x391c0cb3, 0x4ed8aa4a, 0x5b9cca4f, 0x682e6ff3,
    0x748f82ee, 0x78a5636f, 0x84c87814, 0x8cc70208, 0x90befffa, 0xa4506ceb, 0xbef9a3f7, 0xc67178f2};
inline uint32_t rotr(uint32_t x, int n) { return (x >> n) | (x << (32 - n)); }

struct Sha256 {
  uint32_t h[8] = {0x6a09e667, 0xbb67ae85, 0x3c6ef372, 0xa54ff53a,
                   0x510e527f, 0x9b05688c, 0x1f83d9ab, 0x5be0cd19};
  uint8_t buf[64];
  size_t fill = 0;
  uint64_t total = 0;
  void block(const uint8_t *p) {
    uint32_t w[64];
    for (int i = 0; i < 16; i++)
      w[i] = (uint32_t)p[4 * i] << 24 | (uint32_t)p[4 * i + 1] << 16 | (uint32_t)p[4 * i + 2] << 8 |
             (uint32_t)p[4 * i + 3];
    for (int i = 16; i < 64; i++) {
      const uint32_t s0 = rotr(w[i - 15], 7) ^ rotr(w[i - 15], 18) ^ (w[i - 15] >> 3);
      const uint32_t s1 = rotr(w[i - 2], 17) ^ rotr(w[i - 2], 19) ^ (w[i - 2] >> 10);
      w[i] = w[i - 16] + s0 + w[i - 7] + s1;
    }
    uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
    for (int i = 0; i < 64; i++) {
      const uint32_t S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);
      const uint32_t ch = (e & f) ^ (~e & g);
      const uint32_t t1 = hh + S1 + ch + K256[i] + w[i];
      const uint32_t S0 = rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22);
      const uint32_t mj = (a & b) ^ (a & c) ^ (b & c);
      const uint32_t t2 = S0 + mj;
      hh = g; g = f; f = e; e = d + t1; d = c; c = b; b = a; a = t1 + t2;
    }
    h[0] += a; h[1] += b; h[2] += c; h[3] += d; h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
  }
  void update(const void *data, size_t len) {
    const uint8_t *p = (const uint8_t *)data;
    total += len;
    if (fill) {
      const size_t take = std::min(len, 64 - fill);
      memcpy(buf + fill, p, take);
      fill += take; p += take; len -= take;
      if (fill == 64) { block(buf); fill = 0; }
    }
    while (len >= 64) { block(p); p += 64; len -= 64; }
    if (len) { memcpy(buf, p, len); fill = len; }
  }
  void final(uint8_t out[32]) {
    const uint64_t bits = total * 8;
    uint8_t pad = 0x80;
    update(&pad, 1);
    const uint8_t z = 0;
    while (fill != 56) update(&z, 1);
    uint8_t len[8];
    for (int i = 0; i < 8; i++) len[i] = (uint8_t)(bits >> (56 - 8 * i));
    update(len, 8);
    for (int i = 0; i < 8; i++) {
      out[4 * i] = (uint8_t)(h[i] >> 24); out[4 * i + 1] = (uint8_t)(h[i] >> 16);
      out[4 * i + 2] = (uint8_t)(h[i] >> 8); out[4 * i + 3] = (uint8_t)h[i];
    }
  }
};
}  // namespace

void sha256(const void *data, size_t len, uint8_t out[32]) {
  Sha256 s;
  s.update(data, len);
  s.final(out);
}

// Eq. 1: SHA256(layout || g_1 || ... || g_l) with layout = {u32 n, u32 mode}
// and g_i the 24-byte little-endian gate records.
static void hash_gates(Sha256 &s, const TaskData &t, uint64_t b, uint64_t e) {
  uint64_t i = b;
  while (i < e) {
    const size_t k = std::upper_bound(t.span_end.begin(), t.span_end.end(), i) - t.span_end.begin();
    const uint64_t start = k ? t.span_end[k - 1] : 0;
    const uint64_t take = std::min(e, t.span_end[k]) - i;
    s.update(t.spans[k].g + (i - start), take * sizeof(qw_gate));
    i += take;
  }
}

static void hash_layout(Sha256 &s, uint32_t n, uint32_t mode) {
  const uint32_t layout[2] = {n, mode};
  s.update(layout, sizeof(layout));
}

void fingerprint(uint32_t n, uint32_t mode, const TaskData &t, uint64_t b, uint64_t e, uint8_t out[32]) {
  Sha256 s;
  hash_layout(s, n, mode);
  hash_gates(s, t, b, e);
  s.final(out);
}

std::string hex32(const uint8_t h[32]) {
  static const char *d = "0123456789abcdef";
  std::string s(64, '0');
  for (int i = 0; i < 32; i++) { s[2 * i] = d[h[i] >> 4]; s[2 * i + 1] = d[h[i] & 15]; }
  return s;
}

std::string json_escape(const std::string &s) {
  std::string o;
  for (char c : s) {
    if (c == '"' || c == '\\') { o += '\\'; o += c; }
    else if ((unsigned char)c < 0x20) o += strf("\\u%04x", c);
    else o += c;
  }
  return o;
}

// ---------------------------------------------------------------------------
// legality guard (Table II; three gates of Sec. IV-B plus provenance)
// ---------------------------------------------------------------------------
const char *backend_name(uint32_t b) {
  switch (b) {
    case QW_BACKEND_GPU_SV_FP64: return "GPU_SV_FP64";
    case QW_BACKEND_GPU_SV_FP32: return "GPU_SV_FP32";
    case QW_BACKEND_GPU_TABLEAU: return "GPU_TABLEAU";
    default: return "UNKNOWN";
  }
}
const char *kind_name(uint32_t k) {
  return k == QW_KIND_STATEVECTOR ? "STATEVECTOR_BOUNDARY_STATE"
                                  : (k == QW_KIND_TABLEAU ? "TABLEAU_BOUNDARY_STATE" : "UNKNOWN");
}
static uint32_t kind_of_backend(uint32_t b) {
  return b == QW_BACKEND_GPU_TABLEAU ? QW_KIND_TABLEAU : QW_KIND_STATEVECTOR;
}

static void fill_refusal(qw_refusal *o, const char *reason, const char *detail, uint32_t sk,
                         uint32_t tk, uint32_t sb, uint32_t tb) {
  memset(o, 0, sizeof(*o));
  snprintf(o->reason, sizeof(o->reason), "%s", reason);
  snprintf(o->detail, sizeof(o->detail), "%s", detail);
  snprintf(o->source_kind, sizeof(o->source_kind), "%s", kind_name(sk));
  snprintf(o->target_kind, sizeof(o->target_kind), "%s", kind_name(tk));
  snprintf(o->source_backend, sizeof(o->source_backend), "%s", backend_name(sb));
  snprintf(o->target_backend, sizeof(o->target_backend), "%s", backend_name(tb));
}

bool legality(const qw_artifact_desc &a, uint32_t tb, const uint8_t *expected, qw_refusal *out) {
  const uint32_t tk = (tb <= QW_BACKEND_GPU_TABLEAU) ? kind_of_backend(tb) : 99u;
  // gate 1: exactness
  if (a.exactness != QW_EXACT) {
    fill_refusal(out, "NON_EXACT_ARTIFACT", "artifact exactness class is not EXACT; only exact boundaries are reused",
                 a.kind, tk, a.backend, tb);
    return false;
  }
  // gate 2: backend family known on both sides and consistent with the kind
  if (a.backend > QW_BACKEND_GPU_TABLEAU || tb > QW_BACKEND_GPU_TABLEAU ||
      a.kind != kind_of_backend(a.backend)) {
    fill_refusal(out, "UNKNOWN_BACKEND", "producing or consuming backend family is unknown or inconsistent",
                 a.kind, tk, a.backend, tb);
    return false;
  }
  // gate 3: conversion matrix
  if (a.kind == QW_KIND_STATEVECTOR && tk == QW_KIND_TABLEAU) {
    fill_refusal(out, "FORBIDDEN_CONVERSION", "statevector boundary cannot continue on the stabilizer-tableau backend",
                 a.kind, tk, a.backend, tb);
    return false;
  }
  if (a.kind == QW_KIND_TABLEAU && tk == QW_KIND_STATEVECTOR && a.n_qubits > QW_SV_MAX_QUBITS) {
    fill_refusal(out, "UNSUPPORTED_CONVERSION",
                 "exact tableau-to-statevector export is limited to the statevector qubit cap",
                 a.kind, tk, a.backend, tb);
    return false;
  }
  // a higher-precision statevector serves a lower-precision consumer (it is
  // rounded once to the consumer's precision); the reverse is not exact
  if (a.kind == QW_KIND_STATEVECTOR && a.backend != tb &&
      !(a.backend == QW_BACKEND_GPU_SV_FP64 && tb == QW_BACKEND_GPU_SV_FP32)) {
    fill_refusal(out, "FORBIDDEN_CONVERSION",
                 "statevector precision differs: the artifact is not exact for the consuming precision",
                 a.kind, tk, a.backend, tb);
    return false;
  }
  // provenance
  if (expected && memcmp(expected, a.provenance, 32) != 0) {
    fill_refusal(out, "PROVENANCE_MISMATCH", "artifact provenance hash differs from the consumer prefix fingerprint",
                 a.kind, tk, a.backend, tb);
    return false;
  }
  memset(out, 0, sizeof(*out));
  return true;
}

static uint32_t backend_of_mode(uint32_t mode) {
  return mode == QW_MODE_SV_FP64 ? QW_BACKEND_GPU_SV_FP64
                                 : (mode == QW_MODE_SV_FP32 ? QW_BACKEND_GPU_SV_FP32 : QW_BACKEND_GPU_TABLEAU);
}

// ---------------------------------------------------------------------------
// cost-model features of a segment (12 features, see qw_costmodel_features)
// ---------------------------------------------------------------------------
void features_for(const TaskData &t, uint64_t b, uint64_t e, uint32_t n_sharing, const TileConfig &tc,
                  double occupancy, float out[QW_MLP_IN]) {
  uint64_t n1 = 0, n2 = 0, ncl = 0;
  for (uint64_t i = b; i < e; i++) {
    const qw_gate *g = t.gate(i);
    if (is_two_qubit_op(g->op)) n2++; else n1++;
    if (is_clifford_op(g->op)) ncl++;
  }
  const uint32_t n_eff = std::max<uint32_t>(t.n, SV_G);
  const bool fp64 = t.mode == QW_MODE_SV_FP64;
  const double bytes = (t.mode == QW_MODE_TABLEAU)
                           ? (double)(2 * t.n) * 2 * ((t.n + 63) / 64) * 8
                           : std::ldexp(fp64 ? 16.0 : 8.0, (int)n_eff);
  const double gates = (double)(e - b);
  const double k = std::min<uint32_t>(tc.k_max, n_eff);
  out[0] = (float)t.n;
  out[1] = (float)t.mode;
  out[2] = (float)std::log2(1.0 + n1);
  out[3] = (float)std::log2(1.0 + n2);
  out[4] = (float)std::log2(1.0 + gates / std::max(1.0, k - tc.b));
  out[5] = (float)(ncl / std::max(1.0, gates));
  out[6] = (float)k;
  out[7] = (float)std::log2(bytes);
  out[8] = (float)(n_eff <= tc.k_max ? 1.0 : 0.0);
  out[9] = (float)std::log2((double)std::max<uint32_t>(1, n_sharing));
  out[10] = (float)tc.b;
  out[11] = (float)occupancy;
}

}  // namespace qw

// ===========================================================================
// plan construction
// ===========================================================================
namespace qw {

namespace {

inline bool gate_eq(const qw_gate *a, const qw_gate *b) {
  return a == b || memcmp(a, b, sizeof(qw_gate)) == 0;
}

// length of the common run of A[a0..) and B[b0..), at most maxlen; spans
// referenced by both tasks at the same place are skipped without comparing
uint64_t match_len(const TaskData &A, uint64_t a0, const TaskData &B, uint64_t b0, uint64_t maxlen) {
  uint64_t m = 0;
  while (m < maxlen) {
    const uint64_t ia = a0 + m, ib = b0 + m;
    const size_t sa = std::upper_bound(A.span_end.begin(), A.span_end.end(), ia) - A.span_end.begin();
    const size_t sb = std::upper_bound(B.span_end.begin(), B.span_end.end(), ib) - B.span_end.begin();
    const uint64_t ra = A.span_end[sa] - ia, rb = B.span_end[sb] - ib;
    const qw_gate *pa = A.spans[sa].g + (A.spans[sa].n - ra);
    const qw_gate *pb = B.spans[sb].g + (B.spans[sb].n - rb);
    const uint64_t run = std::min(std::min(ra, rb), maxlen - m);
    if (pa == pb) { m += run; continue; }
    uint64_t j = 0;
    while (j < run && memcmp(pa + j, pb + j, sizeof(qw_gate)) == 0) j++;
    m += j;
    if (j < run) break;
  }
  return m;
}

struct Builder {
  const Workload &W;
  std::vector<TNode> nodes;
  std::map<uint32_t, int> roots;
  std::vector<int> end_node;
  explicit Builder(const Workload &w) : W(w) {}

  void insert(uint32_t t) {
    const TaskData &T = W.tasks[t];
    auto it = roots.find(T.n);
    int node;
    if (it == roots.end()) {
      TNode r;
      r.n = T.n;
      r.rep = t;
      nodes.push_back(r);
      node = (int)nodes.size() - 1;
      roots[T.n] = node;
    } else {
      node = it->second;
    }
    uint64_t pos = 0;
    for (;;) {
      if (pos == T.n_gates) { nodes[node].ending.push_back(t); end_node[t] = node; return; }
      const qw_gate *g = T.gate(pos);
      int c = -1;
      for (int kid : nodes[node].kids) {
        const TNode &K = nodes[kid];
        if (gate_eq(W.tasks[K.rep].gate(K.edge_begin), g)) { c = kid; break; }
      }
      if (c < 0) {
        TNode L;
        L.parent = node;
        L.rep = t;
        L.edge_begin = pos;
        L.depth = T.n_gates;
        L.n = T.n;
        L.ending.push_back(t);
        nodes.push_back(L);
        const int li = (int)nodes.size() - 1;
        nodes[node].kids.push_back(li);
        end_node[t] = li;
        return;
      }
      const uint64_t elen = nodes[c].depth - nodes[c].edge_begin;
      const uint64_t maxl = std::min(elen, T.n_gates - pos);
      const uint64_t m = match_len(W.tasks[nodes[c].rep], nodes[c].edge_begin, T, pos, maxl);
      if (m == elen) { node = c; pos += m; continue; }
      // split edge of c after m gates
      TNode M;
      M.parent = node;
      M.rep = nodes[c].rep;
      M.edge_begin = nodes[c].edge_begin;
      M.depth = nodes[c].edge_begin + m;
      M.n = T.n;
      M.kids.push_back(c);
      nodes.push_back(M);
      const int mi = (int)nodes.size() - 1;
      for (int &k : nodes[node].kids) if (k == c) k = mi;
      nodes[c].parent = mi;
      nodes[c].edge_begin = nodes[mi].depth;
      node = mi;
      pos += m;
    }
  }
};

}  // namespace

static bool is_handoff_op(uint32_t op);

struct PlanCtx {
  qw_plan *P;
  Engine *E;
  const Workload &W;
  Builder B;
  std::vector<int> mat_at;   // nearest mat node at or above each trie node's end
  std::vector<uint8_t> refused;
  std::vector<uint8_t> bypass;
  uint64_t store_used = 0;
  uint64_t store_budget = 0;
  double bw_gbs = 6000, launch_ns = 4000;
  std::map<uint64_t, double> gpp;  // gates per pass per (n_eff, fp64)
  // per materialized node: SHA-256 state after its layout and gates [0, end),
  // so a nested node's fingerprint continues from its parent's
  std::vector<Sha256> mat_sha;
  std::vector<int64_t> handoff_run;  // per task: leading gates a tableau can run (-1 = not yet known)
  PlanCtx(qw_plan *p, Engine *e, const Workload &w) : P(p), E(e), W(w), B(w) {}

  uint64_t handoff_len(uint32_t t) {
    if (handoff_run.empty()) handoff_run.assign(W.tasks.size(), -1);
    if (handoff_run[t] < 0) {
      const TaskData &T = W.tasks[t];
      uint64_t len = 0;
      bool go = true;
      for (size_t k = 0; k < T.spans.size() && go; k++)
        for (uint64_t j = 0; j < T.spans[k].n; j++) {
          if (!is_handoff_op(T.spans[k].g[j].op)) { go = false; break; }
          len++;
        }
      handoff_run[t] = (int64_t)len;
    }
    return (uint64_t)handoff_run[t];
  }

  // gate mix of the workload's statevector tasks of one size and precision
  std::map<uint64_t, uint32_t> mix_of;
  uint32_t mix(uint32_t n_eff, bool fp64) {
    const uint64_t key = ((uint64_t)n_eff << 1) | (fp64 ? 1 : 0);
    auto it = mix_of.find(key);
    if (it != mix_of.end()) return it->second;
    uint64_t n2 = 0, all = 0;
    for (const TaskData &T : W.tasks) {
      if (T.mode == QW_MODE_TABLEAU || std::max<uint32_t>(T.n, SV_G) != n_eff ||
          (T.mode == QW_MODE_SV_FP64) != fp64)
        continue;
      for (const Span &sp : T.spans)
        for (uint64_t i = 0; i < sp.n; i++) n2 += is_two_qubit_op(sp.g[i].op) ? 1 : 0;
      all += T.n_gates;
    }
    return mix_of[key] = gate_mix(n2, all);
  }

  TileConfig tiles(uint32_t n_eff, bool fp64) {
    TileConfig tc;
    tc.k_max = fp64 ? 12 : 13;
    tc.b = 4;
    const int ar = fp64 ? SV_AR_PLAIN : plan_ar_batch(P);
    tc.g = sv_stage_width(ar, fp64);
    if (E) tc = E->tile_config(n_eff, fp64, ar, mix(n_eff, fp64));
    const uint32_t kcap = sv_max_tile(ar, fp64);
    if (P->opts.tile_qubits) tc.k_max = std::min<uint32_t>(P->opts.tile_qubits, kcap);
    tc.k_max = std::min<uint32_t>(tc.k_max, kcap);
    if (P->opts.low_qubits) tc.b = P->opts.low_qubits;
    if (tc.k_max < SV_G + 2) tc.k_max = SV_G + 2;
    if (tc.b + 2 > tc.k_max) tc.b = tc.k_max - 2;
    return tc;
  }

  static double state_bytes(uint32_t mode, uint32_t n) {
    if (mode == QW_MODE_TABLEAU) return (double)(2 * n) * 2 * ((n + 63) / 64) * 8 + 2.0 * n;
    const uint32_t n_eff = std::max<uint32_t>(n, SV_G);
    return std::ldexp(mode == QW_MODE_SV_FP64 ? 16.0 : 8.0, (int)n_eff);
  }

  double gates_per_pass(uint32_t mode, uint32_t n, const TaskData &rep) {
    const uint32_t n_eff = std::max<uint32_t>(n, SV_G);
    const bool fp64 = mode == QW_MODE_SV_FP64;
    const uint64_t key = ((uint64_t)n_eff << 1) | (fp64 ? 1 : 0);
    auto it = gpp.find(key);
    if (it != gpp.end()) return it->second;
    TileConfig tc = tiles(n_eff, fp64);
    double v = 1e18;
    if (n_eff > tc.k_max) {
      std::vector<qw_gate> g;
      rep.copy_gates(0, std::min<uint64_t>(rep.n_gates, 2048), g);
      SvProgram pr = fuse_sv(g.data(), g.size(), n_eff, tc);
      v = pr.passes.empty() ? 1e18 : (double)g.size() / (double)pr.passes.size();
    }
    gpp[key] = v;
    return v;
  }

  // analytic cost of executing gates [b, e) of task t (Sec. VI-D gate-count
  // proxy): estimated passes x the time of one pass, measured by the
  // engine for this register size, precision and arithmetic when it tuned
  // the tile shape (else bytes / measured bandwidth + a launch)
  double seg_cost(const TaskData &t, uint32_t mode, uint64_t b, uint64_t e) {
    if (e <= b) return 0.0;
    const double S = state_bytes(mode, t.n);
    if (mode == QW_MODE_TABLEAU) return (double)(e - b) * 1.0 + launch_ns;  // ~1 ns per row op layer slot
    const uint32_t n_eff = std::max<uint32_t>(t.n, SV_G);
    TileConfig tc = tiles(n_eff, mode == QW_MODE_SV_FP64);
    const double p = estimate_passes(e - b, n_eff, tc, gates_per_pass(mode, t.n, t));
    return p * (tc.pass_ns > 0 ? tc.pass_ns : 2.0 * S / bw_gbs + launch_ns);
  }

  bool cost_mlp(const TaskData &t, uint64_t b, uint64_t e, uint32_t sharing, double *ns) {
    if (!E || !E->cm.trained || P->opts.cost_model != QW_COST_MLP || e <= b) return false;
    const uint32_t n_eff = std::max<uint32_t>(t.n, SV_G);
    TileConfig tc = tiles(n_eff, t.mode == QW_MODE_SV_FP64);
    float f[QW_MLP_IN];
    // the probe measures segments run alone on an empty store, so the
    // sharing and occupancy features are queried at those values
    (void)sharing;
    features_for(t, b, e, 1, tc, 0.0, f);
    for (int i = 0; i < QW_MLP_IN; i++)  // outside the training range: analytic fallback
      if (f[i] < E->cm.f_lo[i] - 1e-3f || f[i] > E->cm.f_hi[i] + 1e-3f) return false;
    float y;
    E->predict_log2ns(f, 1, &y);
    *ns = std::exp2((double)y);
    return true;
  }
};

static const char *cut_kind_name(int k) {
  return k == 0 ? "LARGEST_COMMON_PREFIX"
                : (k == 1 ? "CLIFFORD_SAFE_PREFIX" : (k == 2 ? "COARSE_BARRIER" : "TABLEAU_HANDOFF"));
}

// gates a tableau can run ahead of a statevector handoff (unitary Cliffords)
static bool is_handoff_op(uint32_t op) {
  switch (op) {
    case QW_OP_H: case QW_OP_S: case QW_OP_SDG: case QW_OP_X: case QW_OP_Y: case QW_OP_Z:
    case QW_OP_CNOT: case QW_OP_CZ: case QW_OP_SWAP: return true;
    default: return false;
  }
}

static bool is_pauli_op(uint32_t op) { return op == QW_OP_X || op == QW_OP_Y || op == QW_OP_Z; }

static bool same_ref_gate(const qw_gate &a, const qw_gate &b) {
  if (a.op != b.op || a.q0 != b.q0) return false;
  if (is_two_qubit_op(a.op) && a.q1 != b.q1) return false;
  if (is_barrier_op(a.op) && a.theta != b.theta) return false;  // the random outcome bit
  return true;
}

template <typename F>
static void for_each_gate(const TaskData &T, uint64_t b, uint64_t e, F &&f) {
  uint64_t i = b;
  while (i < e) {
    const size_t s = std::upper_bound(T.span_end.begin(), T.span_end.end(), i) - T.span_end.begin();
    const uint64_t start = s ? T.span_end[s - 1] : 0;
    const uint64_t take = std::min(e, T.span_end[s]) - i;
    const qw_gate *g = T.spans[s].g + (i - start);
    for (uint64_t j = 0; j < take; j++)
      if (!f(g[j])) return;
    i += take;
  }
}

// True when every (non-refused) task continues from gate `from` with the
// same gate list once Pauli gates are removed (the Pauli-frame condition).
static bool pauli_equivalent(const Workload &W, const std::vector<uint32_t> &tasks,
                             const std::vector<uint8_t> &refused, uint64_t from) {
  std::vector<const qw_gate *> ref;
  bool first = true, ok = true;
  for (uint32_t t : tasks) {
    if (refused[t] || W.tasks[t].mode != QW_MODE_TABLEAU) continue;
    size_t slot = 0;
    for_each_gate(W.tasks[t], from, W.tasks[t].n_gates, [&](const qw_gate &g) {
      if (is_pauli_op(g.op)) return true;
      if (first) {
        ref.push_back(&g);
      } else if (slot >= ref.size() || !same_ref_gate(*ref[slot], g)) {
        ok = false;
        return false;
      }
      slot++;
      return true;
    });
    if (!ok || (!first && slot != ref.size())) return false;
    first = false;
  }
  return !first;
}

static void decide(PlanCtx &C) {
  qw_plan *P = C.P;
  const Workload &W = C.W;
  auto &nodes = C.B.nodes;
  C.mat_at.assign(nodes.size(), -1);
  C.refused.assign(W.tasks.size(), 0);
  C.bypass.assign(W.tasks.size(), 0);
  const bool reuse = P->opts.reuse != 0;
  // preorder traversal with the nearest materialized ancestor.  A subtree
  // whose tasks all continue from one tableau boundary as Pauli frames is
  // frozen: deeper boundaries would only split the frame group.
  struct Item { int node; int mat; bool frozen; };
  for (auto &r : C.B.roots) {
    std::vector<Item> st{{r.second, -1, false}};
    while (!st.empty()) {
      Item it = st.back();
      st.pop_back();
      const TNode &V = nodes[it.node];
      int mat = it.mat;
      bool frozen = it.frozen;
      const uint32_t consumers = (uint32_t)(V.kids.size() + V.ending.size());
      if (!frozen && reuse && V.parent >= 0 && consumers >= 2 && V.below >= 2) {
        Decision D;
        D.node = it.node;
        D.n = V.n;
        D.depth = V.depth;
        D.n_tasks = V.below;
        // producer: majority mode of the tasks below
        uint32_t pm = 0;
        for (uint32_t m = 1; m < 3; m++) if (V.mode_count[m] > V.mode_count[pm]) pm = m;
        const TaskData &rep = W.tasks[V.rep];
        // the boundary this candidate would continue from must be of the
        // producer's own family (no cross-family continuation)
        int pmat = mat;
        auto same_family = [&](int m) {
          return P->mats[m].mode == pm || (pm != QW_MODE_TABLEAU && ((P->mats[m].export_modes >> pm) & 1u));
        };
        while (pmat >= 0 && !same_family(pmat)) pmat = P->mats[pmat].parent;
        const uint64_t base = (pmat >= 0) ? P->mats[pmat].end : 0;
        const uint64_t lo = std::max<uint64_t>(base, nodes[V.parent].depth);
        // candidate cut points (<= 3), all on the edge into V
        std::vector<std::pair<uint64_t, int>> cuts{{V.depth, 0}};
        for (uint64_t d = V.depth; d > lo + 1 && d + 0 > 0; d--) {
          const bool c1 = is_clifford_op(rep.gate(d - 1)->op), c0 = is_clifford_op(rep.gate(d - 2)->op);
          if (c1 != c0) { if (d - 1 > lo && d - 1 != V.depth) cuts.push_back({d - 1, 1}); break; }
          if (V.depth - d > 4096) break;
        }
        for (uint64_t d = V.depth; d > lo; d--) {
          const qw_gate *g = rep.gate(d - 1);
          if (is_barrier_op(g->op) || (g->flags & QW_GATE_CHECKPOINT)) {
            bool dup = false;
            for (auto &c : cuts) dup |= (c.first == d);
            if (!dup) cuts.push_back({d, 2});
            break;
          }
          if (V.depth - d > 4096) break;
        }
        // cost of the direct plan for the tasks below V: sum of full reruns
        // from the current source, estimated from the representative
        const double S = PlanCtx::state_bytes(pm, V.n);
        const double c_rest = C.seg_cost(rep, pm, V.depth, rep.n_gates);
        double best_net = -1e300;
        for (auto &cu : cuts) {
          Candidate cd;
          cd.cut = cu.first;
          cd.kind = cu.second;
          cd.n_tasks = V.below;
          double cp = 0;
          bool mlp = C.cost_mlp(rep, base, cu.first, 1, &cp);
          if (!mlp) cp = C.seg_cost(rep, pm, base, cu.first);
          D.cost_from_mlp |= mlp;
          cd.c_prefix = cp;
          cd.c_mat = 0.0;     // the producing pass writes the store slot itself (A5)
          cd.c_reload = 0.0;  // fused into the first suffix pass (A5)
          cd.c_handoff = 0.0; // same backend family
          const double c_suffix = C.seg_cost(rep, pm, cu.first, V.depth) + c_rest;
          const double direct = (double)V.below * (cp + c_suffix);
          cd.delta = P->opts.delta_frac * direct;
          qw_cost_tuple ct{(double)V.below, cd.c_prefix, cd.c_mat, cd.c_reload, cd.c_handoff, cd.delta};
          cd.lhs = (ct.n_tasks - 1) * ct.c_prefix;
          cd.rhs = ct.c_materialize + ct.n_tasks * (ct.c_reload + ct.c_handoff) + ct.delta;
          cd.holds = cd.lhs > cd.rhs;
          // early filters (Sec. IV-A)
          if (V.below < P->opts.min_group || cu.first - base < P->opts.min_prefix_gates ||
              cp < P->opts.min_prefix_cost_ns)
            cd.holds = false;
          D.cands.push_back(cd);
          const double net = cd.lhs - cd.rhs;
          if (cd.holds && net > best_net) { best_net = net; D.chosen = (int)D.cands.size() - 1; }
          if (cu.second == 0) {
            D.est_direct = direct;
            D.est_reuse = cp + (double)V.below * c_suffix;
          }
        }
        // Table II STAB -> SV: run an all-Clifford prefix on the tableau and
        // export it once as the statevector the suffixes continue from.  In
        // Eq. 2 terms: C_prefix is the statevector prefix every task would
        // otherwise run, C_mat the tableau run plus the export minus the one
        // statevector run that (N-1) C_prefix already leaves out.
        const double S_sv = S;
        if (P->opts.handoff && pm != QW_MODE_TABLEAU && V.n <= QW_SV_MAX_QUBITS && pmat < 0) {
          const uint64_t hc = std::min<uint64_t>(V.depth, C.handoff_len(V.rep));
          if (hc > 0) {
            Candidate cd;
            cd.cut = hc;
            cd.kind = 3;
            cd.n_tasks = V.below;
            const double c_sv = C.seg_cost(rep, pm, 0, hc);
            const double c_tab = C.seg_cost(rep, QW_MODE_TABLEAU, 0, hc);
            const double c_exp = S_sv / C.bw_gbs + 2.0 * C.launch_ns;
            cd.c_prefix = c_sv;
            cd.c_mat = c_tab + c_exp - c_sv;
            cd.c_reload = 0.0;
            cd.c_handoff = 0.0;
            const double c_suffix = C.seg_cost(rep, pm, hc, V.depth) + c_rest;
            const double direct = (double)V.below * (c_sv + c_suffix);
            cd.delta = P->opts.delta_frac * direct;
            cd.lhs = ((double)V.below - 1.0) * cd.c_prefix;
            cd.rhs = cd.c_mat + cd.delta;
            cd.holds = cd.lhs > cd.rhs;
            if (V.below < P->opts.min_group || hc < P->opts.min_prefix_gates || c_sv < P->opts.min_prefix_cost_ns)
              cd.holds = false;
            D.cands.push_back(cd);
            D.est_handoff = c_tab + c_exp + (double)V.below * c_suffix;
            const double net = cd.lhs - cd.rhs;
            if (cd.holds && net > best_net) { best_net = net; D.chosen = (int)D.cands.size() - 1; }
          }
        }
        const bool handoff = D.chosen >= 0 && D.cands[D.chosen].kind == 3;
        // shared prefixes of FP32 tasks are evolved in FP64 and rounded once
        // (their error no longer grows with the prefix length)
        // Up to 28 qubits (a 4 GiB FP64 boundary plus its 2 GiB copy), and
        // only where both fit the store budget; larger registers keep FP32
        // boundaries, whose memory decides how many the store admits.
        bool up64 = !handoff && pm == QW_MODE_SV_FP32 && P->opts.prefix_fp64 && V.n <= 28;
        if (up64 && C.store_used + (uint64_t)(PlanCtx::state_bytes(QW_MODE_SV_FP64, V.n) + S) > C.store_budget)
          up64 = false;
        const uint32_t prod = handoff ? (uint32_t)QW_MODE_TABLEAU : (up64 ? (uint32_t)QW_MODE_SV_FP64 : pm);
        const double S_store = handoff ? PlanCtx::state_bytes(QW_MODE_TABLEAU, V.n) + S_sv
                                       : (up64 ? PlanCtx::state_bytes(QW_MODE_SV_FP64, V.n) + S : S);
        if (D.chosen < 0) {
          D.decision = 1;
          D.reason = (V.below < P->opts.min_group) ? "EARLY_FILTER_GROUP_SIZE" : "NOT_PROFITABLE";
        } else if (C.store_used + (uint64_t)S_store > C.store_budget) {
          D.decision = 1;
          D.reason = "STORE_BUDGET";
          D.chosen = -1;
        } else {
          // legality of every consumer against the artifact
          MatNode M;
          M.node = it.node;
          M.parent = pmat;
          M.begin = base;
          M.end = D.cands[D.chosen].cut;
          M.rep = V.rep;
          M.mode = prod;
          M.n = V.n;
          M.n_eff = (prod == QW_MODE_TABLEAU) ? V.n : std::max<uint32_t>(V.n, SV_G);
          M.bytes = (uint64_t)S_store;
          if (handoff || up64) M.export_modes = 1u << pm;
          // Eq. 1 over [0, end): continued from the parent's state (the
          // tasks below V share the parent's gates [0, parent end))
          Sha256 sh;
          if (pmat >= 0 && P->mats[pmat].n == V.n && P->mats[pmat].mode == prod) {
            sh = C.mat_sha[pmat];
            hash_gates(sh, rep, P->mats[pmat].end, M.end);
          } else {
            hash_layout(sh, V.n, prod);
            hash_gates(sh, rep, 0, M.end);
          }
          {
            Sha256 fin = sh;
            fin.final(M.provenance);
          }
          qw_artifact_desc A{};
          A.kind = (prod == QW_MODE_TABLEAU) ? QW_KIND_TABLEAU : QW_KIND_STATEVECTOR;
          A.exactness = QW_EXACT;
          A.backend = backend_of_mode(prod);
          A.n_qubits = V.n;
          memcpy(A.provenance, M.provenance, 32);
          // consumers: every task below V
          std::vector<int> stack{it.node};
          uint32_t legal_count = 0;
          std::vector<uint32_t> below_tasks;
          while (!stack.empty()) {
            const int x = stack.back();
            stack.pop_back();
            for (uint32_t t : nodes[x].ending) below_tasks.push_back(t);
            for (int k : nodes[x].kids) stack.push_back(k);
          }
          std::sort(below_tasks.begin(), below_tasks.end());
          for (uint32_t t : below_tasks) {
            if (C.refused[t]) continue;
            qw_refusal rf;
            const uint32_t tb = backend_of_mode(W.tasks[t].mode);
            if (legality(A, tb, A.provenance, &rf)) { legal_count++; continue; }
            const bool sv_both = W.tasks[t].mode != QW_MODE_TABLEAU && prod != QW_MODE_TABLEAU;
            if (!P->opts.legality && sv_both) { C.bypass[t] = 1; legal_count++; continue; }
            C.refused[t] = 1;
            D.refusals.push_back({t, rf});
          }
          if (legal_count >= 2) {
            D.decision = 0;
            D.reason = D.refusals.empty() ? "REUSE" : "REUSE_WITH_REFUSALS";
            D.mat = (int)P->mats.size();
            P->mats.push_back(M);
            C.mat_sha.push_back(sh);
            C.store_used += M.bytes;
            mat = D.mat;
            if (prod == QW_MODE_TABLEAU && !handoff && P->opts.pauli_frames)
              frozen = pauli_equivalent(W, below_tasks, C.refused, M.end);
          } else {
            D.decision = D.refusals.empty() ? 1 : 2;
            D.reason = D.refusals.empty() ? "NOT_PROFITABLE" : "REFUSED_HANDOFF";
            D.chosen = -1;
          }
        }
        P->decisions.push_back(D);
      }
      C.mat_at[it.node] = mat;
      for (auto k = V.kids.rbegin(); k != V.kids.rend(); ++k) st.push_back({*k, mat, frozen});
    }
  }
}

// ---------------------------------------------------------------------------
// Pauli frames: stabilizer tasks on one boundary whose suffixes agree once
// their Pauli gates (X, Y, Z) are removed share that reference suffix; each
// task becomes a set of Pauli events (slot in the reference, qubit, X/Z
// bits).  Only groups of two or more tasks on a materialized boundary are
// converted; the per-task tableau launch stays in the plan as the fallback
// for a reference with random outcomes (decided on the device).
// ---------------------------------------------------------------------------
static void build_frame_groups(qw_plan *P, const Workload &W) {
  const uint32_t nt = (uint32_t)P->tasks.size();
  P->task_frame_group.assign(nt, -1);
  if (!P->opts.pauli_frames) return;
  std::map<std::pair<int, uint32_t>, std::vector<uint32_t>> cand;
  for (uint32_t t = 0; t < nt; t++)
    if (P->tasks[t].mode == QW_MODE_TABLEAU && P->tasks[t].src >= 0)
      cand[{P->tasks[t].src, P->tasks[t].n}].push_back(t);
  for (auto &c : cand) {
    const std::vector<uint32_t> &tasks = c.second;
    if (tasks.size() < 2) continue;
    // a task that keeps its final tableau runs on its own tableau
    bool keep = false;
    for (uint32_t t : tasks) keep = keep || (P->tasks[t].flags & QW_TASK_KEEP_STATE);
    if (keep) continue;
    FrameGroup G;
    G.src = c.first.first;
    G.n = c.first.second;
    // per task: (slot, qubit) -> X bit | Z bit << 1
    std::vector<std::map<std::pair<uint64_t, uint32_t>, uint8_t>> ev(tasks.size());
    bool ok = true;
    for (size_t k = 0; k < tasks.size() && ok; k++) {
      const TaskData &T = W.tasks[tasks[k]];
      uint64_t slot = 0;
      for_each_gate(T, P->tasks[tasks[k]].begin, T.n_gates, [&](const qw_gate &g) {
        if (is_pauli_op(g.op)) {
          const uint8_t b = (uint8_t)((g.op != QW_OP_Z ? 1 : 0) | (g.op != QW_OP_X ? 2 : 0));
          ev[k][{slot, g.q0}] ^= b;
          return true;
        }
        if (k == 0) {
          G.ref.push_back(g);
        } else if (slot >= G.ref.size() || !same_ref_gate(G.ref[slot], g)) {
          ok = false;
          return false;
        }
        slot++;
        return true;
      });
      if (ok && k > 0 && slot != G.ref.size()) ok = false;
    }
    if (!ok) continue;
    std::map<std::pair<uint64_t, uint32_t>, uint32_t> index;
    for (auto &m : ev)
      for (auto &kv : m)
        if (kv.second) index.emplace(kv.first, 0u);
    std::vector<std::pair<uint64_t, uint32_t>> events;
    for (auto &kv : index) {
      kv.second = (uint32_t)events.size();
      events.push_back(kv.first);
    }
    G.tasks = tasks;
    G.n_events = (uint32_t)events.size();
    G.n_words = (uint32_t)((tasks.size() + 31) / 32);
    G.ev_x.assign((size_t)G.n_events * G.n_words, 0u);
    G.ev_z.assign((size_t)G.n_events * G.n_words, 0u);
    for (size_t k = 0; k < tasks.size(); k++)
      for (auto &kv : ev[k]) {
        if (!kv.second) continue;
        const size_t e = index[kv.first];
        const uint32_t bit = 1u << (k & 31);
        if (kv.second & 1) G.ev_x[e * G.n_words + k / 32] |= bit;
        if (kv.second & 2) G.ev_z[e * G.n_words + k / 32] |= bit;
      }
    G.prog = compile_frames(G.ref.data(), G.ref.size(), G.n, events);
    TabHostProgram hp = compile_tab(G.ref.data(), G.ref.size(), G.n);
    const uint32_t bit_base = (uint32_t)P->tab_bits.size();
    for (const qw_gate &g : G.ref)
      if (is_barrier_op(g.op)) P->tab_bits.push_back(g.theta != 0.0 ? 1 : 0);
    G.n_outs = hp.n_outs;
    P->tab_progs.push_back(std::move(hp));
    G.ref_segs.push_back({(uint32_t)P->tab_progs.size() - 1, bit_base});
    bool outs_ok = true;
    for (uint32_t t : tasks) outs_ok = outs_ok && P->tasks[t].tab_outs == G.n_outs;
    if (!outs_ok) fail(QW_ERR_STATE, "internal: frame reference and task outcome counts differ");
    const int gi = (int)P->frame_groups.size();
    for (uint32_t t : tasks) P->task_frame_group[t] = gi;
    P->frame_groups.push_back(std::move(G));
  }
}

void build_plan(qw_plan *P, Engine *E, const Workload &W) {
  const auto t0 = std::chrono::steady_clock::now();
  // FP32 arithmetic: QW_FP32_AUTO compensates when some FP32 task asks for
  // a Pauli-sum energy (the 1e-6 relative energy target); samples and
  // states alone need the 1e-5 amplitude bound, which plain FP32 meets
  P->fp32_compensated = P->opts.fp32_arith == QW_FP32_COMPENSATED;
  if (P->opts.fp32_arith == QW_FP32_AUTO)
    for (const TaskData &T : W.tasks)
      if (T.mode == QW_MODE_SV_FP32 && !T.terms.empty()) P->fp32_compensated = true;
  PlanCtx C(P, E, W);
  C.bw_gbs = E ? E->hbm_gbs : 6000.0;
  C.launch_ns = E ? E->launch_ns : 4000.0;
  C.store_budget = E ? E->store_budget : (uint64_t)120e9;
  const uint32_t nt = (uint32_t)W.tasks.size();
  C.B.end_node.assign(nt, -1);
  for (uint32_t t = 0; t < nt; t++) {
    C.B.insert(t);
    P->total_gates += W.tasks[t].n_gates;
  }
  // subtree counts (children always have larger indices than... not
  // guaranteed after splits, so use an explicit post-order)
  auto &nodes = C.B.nodes;
  for (auto &r : C.B.roots) {
    std::vector<std::pair<int, int>> st{{r.second, 0}};
    while (!st.empty()) {
      auto &top = st.back();
      TNode &V = nodes[top.first];
      if (top.second < (int)V.kids.size()) {
        const int k = V.kids[top.second++];
        st.push_back({k, 0});
        continue;
      }
      V.below = (uint32_t)V.ending.size();
      for (uint32_t t : V.ending) V.mode_count[W.tasks[t].mode]++;
      for (int k : V.kids) {
        V.below += nodes[k].below;
        for (int m = 0; m < 3; m++) V.mode_count[m] += nodes[k].mode_count[m];
      }
      st.pop_back();
    }
  }
  bool any_branch = false;
  for (auto &V : nodes) any_branch |= (V.parent >= 0 && V.kids.size() + V.ending.size() >= 2);
  P->fast_path = !any_branch;
  decide(C);

  // task sources
  P->tasks.resize(nt);
  for (uint32_t t = 0; t < nt; t++) {
    const TaskData &T = W.tasks[t];
    TaskPlan &tp = P->tasks[t];
    tp.mode = T.mode;
    tp.n = T.n;
    tp.n_eff = (T.mode == QW_MODE_TABLEAU) ? T.n : std::max<uint32_t>(T.n, SV_G);
    tp.flags = T.flags;
    tp.shots = T.shots;
    tp.n_gates = T.n_gates;
    tp.uniforms = T.uniforms;
    tp.refused = C.refused[t] != 0;
    tp.legality_bypassed = C.bypass[t] != 0;
    int src = C.mat_at[C.B.end_node[t]];
    if (tp.refused) src = -1;
    // an artifact of another mode is usable only through the bypass, or as
    // a tableau boundary exported to the task's statevector (Table II)
    auto usable = [&](int m) {
      const uint32_t mm = P->mats[m].mode;
      if (mm == T.mode || tp.legality_bypassed) return true;
      if (T.mode == QW_MODE_SV_FP32 && mm == QW_MODE_SV_FP64) return true;  // rounded once
      return T.mode != QW_MODE_TABLEAU && mm == QW_MODE_TABLEAU && T.n <= QW_SV_MAX_QUBITS && P->opts.handoff;
    };
    while (src >= 0 && !usable(src)) src = P->mats[src].parent;
    tp.src = src;
    tp.begin = (src >= 0) ? P->mats[src].end : 0;
    if (src >= 0 && P->mats[src].mode != T.mode && T.mode != QW_MODE_TABLEAU && !tp.legality_bypassed)
      P->mats[src].export_modes |= 1u << T.mode;
  }

  // Hamiltonian layouts (deduplicated by content)
  std::unordered_map<std::string, int> ham_ids;
  for (uint32_t t = 0; t < nt; t++) {
    const TaskData &T = W.tasks[t];
    if (T.mode == QW_MODE_TABLEAU || T.terms.empty()) continue;
    const uint32_t n_eff = std::max<uint32_t>(T.n, SV_G);
    std::string key((const char *)T.terms.data(), T.terms.size() * sizeof(qw_pauli_term));
    const uint32_t amp_bytes = T.mode == QW_MODE_SV_FP64 ? 16u : 8u;
    key += strf("|%u|%u", n_eff, amp_bytes);
    auto it = ham_ids.find(key);
    if (it != ham_ids.end()) { P->tasks[t].ham = it->second; continue; }
    HamLayout H;
    H.n_eff = n_eff;
    build_energy_layout(T.terms.data(), T.terms.size(), n_eff, amp_bytes, &H.chunk_bits, H.classes, H.terms,
                        &H.n_blocks);
    P->hams.push_back(std::move(H));
    ham_ids[key] = (int)P->hams.size() - 1;
    P->tasks[t].ham = ham_ids[key];
  }

  // compile programs
  std::vector<qw_gate> buf;
  std::map<std::pair<const qw_gate *, uint64_t>, std::pair<uint32_t, uint32_t>> tab_cache;
  auto compile_tab_range = [&](const TaskData &T, uint64_t b, uint64_t e,
                               std::vector<std::pair<uint32_t, uint32_t>> &segs, uint32_t *outs) {
    *outs = 0;
    uint64_t i = b;
    while (i < e) {
      const size_t k = std::upper_bound(T.span_end.begin(), T.span_end.end(), i) - T.span_end.begin();
      const uint64_t start = k ? T.span_end[k - 1] : 0;
      const uint64_t take = std::min(e, T.span_end[k]) - i;
      const qw_gate *g = T.spans[k].g + (i - start);
      auto key = std::make_pair(g, take);
      auto it = tab_cache.find(key);
      uint32_t prog, bit_base;
      if (it == tab_cache.end()) {
        TabHostProgram hp = compile_tab(g, take, T.n);
        bit_base = (uint32_t)P->tab_bits.size();
        for (uint64_t j = 0; j < take; j++)
          if (is_barrier_op(g[j].op)) P->tab_bits.push_back(g[j].theta != 0.0 ? 1 : 0);
        P->tab_progs.push_back(std::move(hp));
        prog = (uint32_t)P->tab_progs.size() - 1;
        tab_cache[key] = {prog, bit_base};
      } else {
        prog = it->second.first;
        bit_base = it->second.second;
      }
      segs.push_back({prog, bit_base});
      *outs += P->tab_progs[prog].n_outs;
      i += take;
    }
  };
  for (auto &M : P->mats) {
    const TaskData &R = W.tasks[M.rep];
    if (M.mode == QW_MODE_TABLEAU) {
      compile_tab_range(R, M.begin, M.end, M.tab_segs, &M.tab_outs);
      M.out_offset = (M.parent >= 0) ? P->mats[M.parent].out_offset + P->mats[M.parent].tab_outs : 0;
    } else {
      R.copy_gates(M.begin, M.end, buf);
      TileConfig tc = C.tiles(M.n_eff, M.mode == QW_MODE_SV_FP64);
      M.sv = fuse_sv(buf.data(), buf.size(), M.n_eff, tc);
      if (P->opts.dense_boundaries) M.gates = buf;
    }
  }
  for (uint32_t t = 0; t < nt; t++) {
    const TaskData &T = W.tasks[t];
    TaskPlan &tp = P->tasks[t];
    if (T.mode == QW_MODE_TABLEAU) {
      compile_tab_range(T, tp.begin, T.n_gates, tp.tab_segs, &tp.tab_outs);
      tp.total_outs = tp.tab_outs +
                      ((tp.src >= 0) ? P->mats[tp.src].out_offset + P->mats[tp.src].tab_outs : 0);
    } else {
      T.copy_gates(tp.begin, T.n_gates, buf);
      TileConfig tc = C.tiles(tp.n_eff, T.mode == QW_MODE_SV_FP64);
      tp.sv = fuse_sv(buf.data(), buf.size(), tp.n_eff, tc);
      if (tp.sv.passes.empty() && tp.src < 0) {
        // no gates at all: one pass without stages materializes |0...0>
        HostPass hp;
        const uint32_t k = std::min(tc.k_max, tp.n_eff);
        for (uint32_t q = 0; q < k; q++) hp.q.push_back(q);
        hp.b = (tp.n_eff <= tc.k_max) ? tp.n_eff : std::min(tc.b, k - 2);
        tp.sv.passes.push_back(hp);
      }
    }
  }

  build_frame_groups(P, W);

  // plan-level estimates (Table IV "Est." column analog: direct / planned)
  double direct = 0, planned = 0;
  for (uint32_t t = 0; t < nt; t++) {
    const TaskData &T = W.tasks[t];
    direct += C.seg_cost(T, T.mode, 0, T.n_gates);
    planned += C.seg_cost(T, T.mode, P->tasks[t].begin, T.n_gates);
  }
  for (auto &M : P->mats) planned += C.seg_cost(W.tasks[M.rep], M.mode, M.begin, M.end);
  P->est_direct_ns = direct;
  P->est_plan_ns = planned;
  P->planning_ns =
      std::chrono::duration<double, std::nano>(std::chrono::steady_clock::now() - t0).count();

  // EXPLAIN
  std::string s;
  s.reserve(4096 + 512 * P->decisions.size());
  uint32_t n_ref = 0, n_reuse_tasks = 0;
  for (auto &tp : P->tasks) { n_ref += tp.refused; n_reuse_tasks += (tp.src >= 0); }
  s += "{\"type\":\"QuWARP:ExplainTrace\",";
  s += strf("\"tasks\":%u,\"groups\":%zu,\"total_gates\":%llu,", nt, C.B.roots.size(),
            (unsigned long long)P->total_gates);
  s += strf("\"options\":{\"reuse\":%d,\"batched\":%d,\"legality\":%d,\"cost_model\":\"%s\","
            "\"delta_frac\":%.6g,\"min_group\":%u,\"min_prefix_gates\":%u,\"pauli_frames\":%d},",
            P->opts.reuse, P->opts.batched, P->opts.legality,
            P->opts.cost_model == QW_COST_MLP ? "MLP" : "ANALYTIC", P->opts.delta_frac,
            P->opts.min_group, P->opts.min_prefix_gates, P->opts.pauli_frames);
  s += strf("\"fast_path\":%s,\"planning_ns\":%.0f,\"estimated_direct_ns\":%.1f,"
            "\"estimated_plan_ns\":%.1f,\"estimated_speedup\":%.4f,",
            P->fast_path ? "true" : "false", P->planning_ns, direct, planned,
            planned > 0 ? direct / planned : 1.0);
  s += strf("\"tasks_reusing\":%u,\"tasks_refused\":%u,\"artifacts\":%zu,", n_reuse_tasks, n_ref,
            P->mats.size());
  s += "\"pauli_frames\":[";
  for (size_t g = 0; g < P->frame_groups.size(); g++) {
    const FrameGroup &G = P->frame_groups[g];
    s += strf("%s{\"artifact\":%d,\"tasks\":%zu,\"reference_gates\":%zu,\"events\":%u,"
              "\"layers\":%zu,\"outcomes_per_task\":%u}",
              g ? "," : "", G.src, G.tasks.size(), G.ref.size(), G.n_events, G.prog.layers.size(), G.n_outs);
  }
  s += "],";
  s += "\"decisions\":[";
  for (size_t i = 0; i < P->decisions.size(); i++) {
    const Decision &D = P->decisions[i];
    if (i) s += ",";
    static const char *dn[3] = {"REUSE", "ABSTAIN", "REFUSE"};
    s += strf("{\"node\":%d,\"qubits\":%u,\"branch_gate\":%llu,\"tasks_sharing\":%u,"
              "\"decision\":\"%s\",\"reason\":\"%s\",\"cost_source\":\"%s\",",
              D.node, D.n, (unsigned long long)D.depth, D.n_tasks, dn[D.decision], D.reason.c_str(),
              D.cost_from_mlp ? "MLP" : "ANALYTIC");
    s += "\"candidates\":[";
    for (size_t c = 0; c < D.cands.size(); c++) {
      const Candidate &cd = D.cands[c];
      if (c) s += ",";
      s += strf("{\"boundary\":\"%s\",\"cut_gate\":%llu,\"n\":%u,\"c_prefix_ns\":%.1f,"
                "\"c_materialize_ns\":%.1f,\"c_reload_ns\":%.1f,\"c_handoff_ns\":%.1f,"
                "\"delta_ns\":%.1f,\"lhs_ns\":%.1f,\"rhs_ns\":%.1f,\"inequality_holds\":%s,"
                "\"chosen\":%s}",
                cut_kind_name(cd.kind), (unsigned long long)cd.cut, cd.n_tasks, cd.c_prefix,
                cd.c_mat, cd.c_reload, cd.c_handoff, cd.delta, cd.lhs, cd.rhs,
                cd.holds ? "true" : "false", (int)c == D.chosen ? "true" : "false");
    }
    s += "],";
    const bool ho = D.chosen >= 0 && D.cands[D.chosen].kind == 3;
    s += strf("\"alternatives\":[{\"plan\":\"BASELINE\",\"est_ns\":%.1f,\"chosen\":%s},"
              "{\"plan\":\"SAME_FAMILY_REUSE\",\"est_ns\":%.1f,\"chosen\":%s},",
              D.est_direct, D.decision == 0 ? "false" : "true", D.est_reuse,
              (D.decision == 0 && !ho) ? "true" : "false");
    if (D.est_handoff >= 0)
      s += strf("{\"plan\":\"CROSS_BACKEND_HANDOFF\",\"est_ns\":%.1f,\"chosen\":%s}],", D.est_handoff,
                (D.decision == 0 && ho) ? "true" : "false");
    else
      s += "{\"plan\":\"CROSS_BACKEND_HANDOFF\",\"status\":\"NOT_APPLICABLE\"}],";
    if (D.mat >= 0) {
      const MatNode &M = P->mats[D.mat];
      s += strf("\"artifact\":{\"kind\":\"%s\",\"exactness\":\"EXACT\",\"provenance_sha256\":\"%s\","
                "\"backend\":\"%s\",\"bytes\":%llu,\"qubits\":%u,\"prefix_gates\":%llu,",
                kind_name(M.mode == QW_MODE_TABLEAU ? QW_KIND_TABLEAU : QW_KIND_STATEVECTOR),
                hex32(M.provenance).c_str(), backend_name(backend_of_mode(M.mode)),
                (unsigned long long)M.bytes, M.n, (unsigned long long)M.end);
      s += strf("\"id\":%d,\"parent\":%d,\"first_gate\":%llu,", D.mat, M.parent, (unsigned long long)M.begin);
      s += "\"exported_to\":[";
      bool first_e = true;
      for (uint32_t md = 0; md < 2; md++)
        if ((M.export_modes >> md) & 1u) {
          s += strf("%s\"%s\"", first_e ? "" : ",", backend_name(backend_of_mode(md)));
          first_e = false;
        }
      // a consumer of another precision or representation reads the
      // artifact rounded once into its own precision (FP64 -> FP32, or the
      // tableau's amplitudes +-i^e 2^(-k/2) written in FP32 / FP64)
      s += "],\"consumer_exactness\":{";
      first_e = true;
      for (uint32_t md = 0; md < 2; md++)
        if ((M.export_modes >> md) & 1u) {
          s += strf("%s\"%s\":\"EXACT_UP_TO_ONE_ROUNDING\"", first_e ? "" : ",", backend_name(backend_of_mode(md)));
          first_e = false;
        }
      s += "}},";
    } else {
      s += "\"artifact\":null,";
    }
    s += "\"refusals\":[";
    for (size_t r = 0; r < D.refusals.size(); r++) {
      const qw_refusal &f = D.refusals[r].r;
      if (r) s += ",";
      s += strf("{\"task\":%u,\"reason\":\"%s\",\"detail\":\"%s\",\"source_kind\":\"%s\","
                "\"target_kind\":\"%s\",\"source_backend\":\"%s\",\"target_backend\":\"%s\","
                "\"fallback\":\"FULL_RERUN\"}",
                D.refusals[r].task, f.reason, json_escape(f.detail).c_str(), f.source_kind,
                f.target_kind, f.source_backend, f.target_backend);
    }
    s += "]}";
  }
  s += "]}";
  P->explain = std::move(s);
}

}  // namespace qw

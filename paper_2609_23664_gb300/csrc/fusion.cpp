// Gate fusion (statevector) and layer compilation (tableau), host side.
//
// Statevector: a gate list is cut into PASSES.  A pass owns a set Q of at
// most k tile qubits (always containing the b lowest qubits so that every
// tile is read and written in contiguous runs of 2^b amplitudes); one CTA
// loads a tile (2^k amplitudes with the bits outside Q fixed) into shared
// memory, applies every gate of the pass and writes the tile back.  Gates
// are taken out of order only past gates on disjoint qubits (they commute).
// Inside a pass, gates are grouped into STAGES of at most 5 tile bits; a
// thread holds the 32 amplitudes of one stage group in registers and applies
// the whole stage there.  Consecutive single-qubit gates on one qubit are
// multiplied into one 2x2 matrix in double precision.
//
// Tableau: a Clifford gate run becomes LAYERS of row operations on the
// inverse tableau that touch disjoint rows, so that one layer runs fully in
// parallel inside a CTA.
#include <algorithm>
#include <cmath>
#include <complex>

#include "qw_internal.h"

namespace qw {

using cd = std::complex<double>;

bool is_two_qubit_op(uint32_t op) {
  return op == QW_OP_CNOT || op == QW_OP_CZ || op == QW_OP_SWAP || op == QW_OP_CPHASE;
}
bool is_barrier_op(uint32_t op) { return op == QW_OP_MEASURE || op == QW_OP_RESET; }
bool is_clifford_op(uint32_t op) {
  switch (op) {
    case QW_OP_H: case QW_OP_X: case QW_OP_Y: case QW_OP_Z: case QW_OP_S: case QW_OP_SDG:
    case QW_OP_CNOT: case QW_OP_CZ: case QW_OP_SWAP: case QW_OP_MEASURE: case QW_OP_RESET:
      return true;
    default:
      return false;
  }
}

// 2x2 matrix of a single-qubit gate: m = {u00, u01, u10, u11} as (re, im).
bool gate_matrix_1q(const qw_gate &g, double m[8], bool *diagonal) {
  cd u00, u01, u10, u11;
  const double th = g.theta, c = std::cos(th / 2), s = std::sin(th / 2);
  const double r = 1.0 / std::sqrt(2.0);
  const cd I(0, 1);
  bool diag = false;
  switch (g.op) {
    case QW_OP_H: u00 = r; u01 = r; u10 = r; u11 = -r; break;
    case QW_OP_X: u00 = 0; u01 = 1; u10 = 1; u11 = 0; break;
    case QW_OP_Y: u00 = 0; u01 = -I; u10 = I; u11 = 0; break;
    case QW_OP_Z: u00 = 1; u11 = -1; diag = true; break;
    case QW_OP_S: u00 = 1; u11 = I; diag = true; break;
    case QW_OP_SDG: u00 = 1; u11 = -I; diag = true; break;
    case QW_OP_T: u00 = 1; u11 = std::polar(1.0, M_PI / 4); diag = true; break;
    case QW_OP_TDG: u00 = 1; u11 = std::polar(1.0, -M_PI / 4); diag = true; break;
    case QW_OP_RX: u00 = c; u01 = -I * s; u10 = -I * s; u11 = c; break;
    case QW_OP_RY: u00 = c; u01 = -s; u10 = s; u11 = c; break;
    case QW_OP_RZ: u00 = std::polar(1.0, -th / 2); u11 = std::polar(1.0, th / 2); diag = true; break;
    case QW_OP_PHASE: u00 = 1; u11 = std::polar(1.0, th); diag = true; break;
    default: return false;
  }
  const cd v[4] = {u00, u01, u10, u11};
  for (int i = 0; i < 4; i++) { m[2 * i] = v[i].real(); m[2 * i + 1] = v[i].imag(); }
  if (diagonal) *diagonal = diag;
  return true;
}

static uint32_t gate_mask(const qw_gate &g) {
  uint32_t m = 1u << g.q0;
  if (is_two_qubit_op(g.op)) m |= 1u << g.q1;
  return m;
}

static int popc32(uint32_t v) { return __builtin_popcount(v); }

// greedy cover of the remaining gates by groups of at most `cap` positions;
// `forced` positions belong to every group.  Returns, per group, the gate
// indices (into idx) and the position mask.
// With `perm` given, a gate that is not a permutation (perm[i] == 0) is not
// taken into a group after a permutation gate on one of its positions, so
// every permutation gate of a group can be moved to the end of the group.
static void greedy_groups(const std::vector<uint32_t> &masks, uint32_t n_pos, uint32_t cap,
                          uint32_t forced, std::vector<std::vector<uint32_t>> &groups,
                          std::vector<uint32_t> &group_masks,
                          const std::vector<uint8_t> *perm = nullptr) {
  const uint32_t full = (n_pos >= 32) ? 0xFFFFFFFFu : ((1u << n_pos) - 1);
  std::vector<uint32_t> rem(masks.size());
  for (uint32_t i = 0; i < rem.size(); i++) rem[i] = i;
  while (!rem.empty()) {
    uint32_t Q = forced, blocked = 0, permq = 0;
    std::vector<uint32_t> taken;
    std::vector<uint32_t> keep;
    keep.reserve(rem.size());
    size_t i = 0;
    for (; i < rem.size(); i++) {
      const uint32_t gi = rem[i], qs = masks[gi];
      const bool is_perm = perm && (*perm)[gi];
      if ((qs & blocked) || (perm && !is_perm && (qs & permq))) {
        blocked |= qs;  // must stay after an earlier skipped gate on a shared qubit
        keep.push_back(gi);
      } else if ((uint32_t)popc32(Q | qs) <= cap) {
        Q |= qs;        // commutes past every skipped gate (disjoint qubits)
        if (is_perm) permq |= qs;
        taken.push_back(gi);
      } else {
        blocked |= qs;
        keep.push_back(gi);
      }
      if (blocked == full) { i++; break; }
    }
    for (; i < rem.size(); i++) keep.push_back(rem[i]);
    if (taken.empty()) fail(QW_ERR_INVALID_ARG, "fusion: gate does not fit a group");
    groups.push_back(std::move(taken));
    group_masks.push_back(Q);
    rem.swap(keep);
  }
}

static void mat_mul(const double a[8], const double b[8], double out[8]) {  // out = a * b
  cd A[4], B[4];
  for (int i = 0; i < 4; i++) { A[i] = cd(a[2 * i], a[2 * i + 1]); B[i] = cd(b[2 * i], b[2 * i + 1]); }
  cd C[4] = {A[0] * B[0] + A[1] * B[2], A[0] * B[1] + A[1] * B[3],
             A[2] * B[0] + A[3] * B[2], A[2] * B[1] + A[3] * B[3]};
  for (int i = 0; i < 4; i++) { out[2 * i] = C[i].real(); out[2 * i + 1] = C[i].imag(); }
}

SvProgram fuse_sv(const qw_gate *gates, uint64_t n_gates, uint32_t n_eff, const TileConfig &tc) {
  SvProgram prog;
  prog.n = n_eff;
  prog.n_gates = n_gates;
  if (n_gates == 0) return prog;
  const uint32_t k = std::min(tc.k_max, n_eff);
  const bool single = (n_eff <= tc.k_max);
  const uint32_t b = single ? n_eff : std::min(tc.b, k - 2);
  const uint32_t forced = (b >= 32) ? 0xFFFFFFFFu : ((1u << b) - 1);

  std::vector<uint32_t> masks(n_gates);
  for (uint64_t i = 0; i < n_gates; i++) masks[i] = gate_mask(gates[i]);

  std::vector<std::vector<uint32_t>> pass_gates;
  std::vector<uint32_t> pass_masks;
  if (single) {
    std::vector<uint32_t> all(n_gates);
    for (uint64_t i = 0; i < n_gates; i++) all[i] = (uint32_t)i;
    pass_gates.push_back(all);
    pass_masks.push_back((n_eff >= 32) ? 0xFFFFFFFFu : ((1u << n_eff) - 1));
  } else {
    greedy_groups(masks, n_eff, k, forced, pass_gates, pass_masks);
  }

  for (size_t p = 0; p < pass_gates.size(); p++) {
    HostPass hp;
    uint32_t Q = pass_masks[p];
    // pad Q up to k with the lowest unused qubits
    for (uint32_t q = 0; q < n_eff && (uint32_t)popc32(Q) < k; q++) Q |= 1u << q;
    uint32_t loc[32];
    for (uint32_t q = 0; q < n_eff; q++)
      if (Q & (1u << q)) { loc[q] = (uint32_t)hp.q.size(); hp.q.push_back(q); }
    hp.b = b;
    hp.n_gates = (uint32_t)pass_gates[p].size();
    // stages inside the pass (positions = local tile bits)
    std::vector<uint32_t> lmask(pass_gates[p].size());
    for (size_t i = 0; i < pass_gates[p].size(); i++) {
      const qw_gate &g = gates[pass_gates[p][i]];
      uint32_t m = 1u << loc[g.q0];
      if (is_two_qubit_op(g.op)) m |= 1u << loc[g.q1];
      lmask[i] = m;
    }
    std::vector<std::vector<uint32_t>> st_gates;
    std::vector<uint32_t> st_masks;
    std::vector<uint8_t> lperm(pass_gates[p].size());
    for (size_t i = 0; i < pass_gates[p].size(); i++) {
      const uint32_t op = gates[pass_gates[p][i]].op;
      lperm[i] = (op == QW_OP_CNOT || op == QW_OP_SWAP) ? 1 : 0;
    }
    greedy_groups(lmask, k, SV_G, 0, st_gates, st_masks, &lperm);
    for (size_t s = 0; s < st_gates.size(); s++) {
      HostStage hs;
      uint32_t P = st_masks[s];
      for (uint32_t q = 0; q < k && popc32(P) < SV_G; q++) P |= 1u << q;
      int rel[32];
      int j = 0;
      for (uint32_t q = 0; q < k; q++)
        if (P & (1u << q)) { hs.pos[j] = (uint8_t)q; rel[q] = j; j++; }
      int last1q[SV_G];
      for (int t = 0; t < SV_G; t++) last1q[t] = -1;
      for (uint32_t gi_local : st_gates[s]) {
        const qw_gate &g = gates[pass_gates[p][gi_local]];
        const int a = rel[loc[g.q0]];
        HostOp op{};
        double m[8];
        bool diag = false;
        if (gate_matrix_1q(g, m, &diag)) {
          if (last1q[a] >= 0) {
            HostOp &prev = hs.ops[last1q[a]];
            double out[8];
            mat_mul(m, prev.m, out);
            std::memcpy(prev.m, out, sizeof(out));
            prev.kind = (prev.kind == K_D1 && diag) ? K_D1 : K_U1;
            continue;
          }
          op.kind = diag ? K_D1 : K_U1;
          op.a = (uint8_t)a;
          std::memcpy(op.m, m, sizeof(m));
          last1q[a] = (int)hs.ops.size();
          hs.ops.push_back(op);
          continue;
        }
        const int bb = rel[loc[g.q1]];
        op.a = (uint8_t)a;
        op.b = (uint8_t)bb;
        switch (g.op) {
          case QW_OP_CNOT: op.kind = K_CX; break;
          case QW_OP_CZ: op.kind = K_CD; op.m[0] = -1; op.m[1] = 0; break;
          case QW_OP_CPHASE: op.kind = K_CD; op.m[0] = std::cos(g.theta); op.m[1] = std::sin(g.theta); break;
          case QW_OP_SWAP: op.kind = K_SWAP; break;
          default: fail(QW_ERR_INVALID_ARG, "fusion: unsupported statevector op %u", g.op);
        }
        if ((op.kind == K_CD || op.kind == K_SWAP) && op.a > op.b) std::swap(op.a, op.b);
        last1q[a] = -1;
        last1q[bb] = -1;
        hs.ops.push_back(op);
      }
      // diagonal ops keep {d0, d1} in m[0..3]
      for (auto &o : hs.ops)
        if (o.kind == K_D1) { o.m[2] = o.m[6]; o.m[3] = o.m[7]; }
      // the permutation gates (all movable to the end of the stage) become
      // the linear index map A = E_last ... E_first; row j of A as a mask
      uint8_t row[SV_G];
      for (int t = 0; t < SV_G; t++) row[t] = (uint8_t)(1u << t);
      std::vector<HostOp> kept;
      for (const HostOp &o : hs.ops) {
        if (o.kind == K_CX) { row[o.b] ^= row[o.a]; continue; }
        if (o.kind == K_SWAP) { std::swap(row[o.a], row[o.b]); continue; }
        kept.push_back(o);
      }
      hs.ops.swap(kept);
      for (int c = 0; c < SV_G; c++) {
        uint8_t m = 0;
        for (int r = 0; r < SV_G; r++)
          if ((row[r] >> c) & 1u) m |= (uint8_t)(1u << r);
        hs.colmask[c] = m;
      }
      hp.stages.push_back(std::move(hs));
    }
    prog.passes.push_back(std::move(hp));
  }
  return prog;
}

uint32_t estimate_passes(uint64_t n_gates, uint32_t n, const TileConfig &tc, double gates_per_pass) {
  if (n_gates == 0) return 0;
  if (n <= tc.k_max) return 1;
  double p = std::ceil((double)n_gates / std::max(gates_per_pass, 1.0));
  return (uint32_t)std::max(1.0, p);
}

// ---------------------------------------------------------------------------
// tableau layers
// ---------------------------------------------------------------------------
TabHostProgram compile_tab(const qw_gate *gates, uint64_t n_gates, uint32_t n) {
  TabHostProgram P;
  const uint32_t rows = 2 * n;
  std::vector<uint32_t> w_layer(rows, 0xFFFFFFFFu), r_layer(rows, 0xFFFFFFFFu);
  std::vector<uint32_t> meas_q_layer(n, 0xFFFFFFFFu);
  uint32_t cur = 0xFFFFFFFFu;
  bool cur_is_meas = false;
  auto new_layer = [&](bool meas) {
    TabLayer L{};
    L.slot_begin = (uint32_t)P.slots.size();
    L.is_measure = meas ? 1u : 0u;
    P.layers.push_back(L);
    cur = (uint32_t)P.layers.size() - 1;
    cur_is_meas = meas;
  };
  auto X = [&](uint32_t q) { return (uint16_t)q; };
  auto Z = [&](uint32_t q) { return (uint16_t)(n + q); };
  for (uint64_t i = 0; i < n_gates; i++) {
    const qw_gate &g = gates[i];
    if (is_barrier_op(g.op)) {
      if (cur == 0xFFFFFFFFu || !cur_is_meas || meas_q_layer[g.q0] == cur) new_layer(true);
      meas_q_layer[g.q0] = cur;
      TabSlot s{};
      s.kind = T_MEAS;
      s.flags = (g.op == QW_OP_RESET) ? 1 : 0;
      s.dst = Z(g.q0);
      s.s1 = (uint16_t)g.q0;
      s.aux = P.n_bits++;
      s.aux2 = (g.op == QW_OP_MEASURE) ? P.n_outs++ : 0xFFFFFFFFu;
      P.slots.push_back(s);
      P.layers[cur].n_slots++;
      continue;
    }
    TabSlot sl[2];
    int ns = 0;
    const uint32_t a = g.q0, b = g.q1;
    auto prod = [&](uint16_t dst, uint16_t src2, uint8_t e0) {
      TabSlot s{}; s.kind = T_PROD; s.dst = dst; s.s1 = dst; s.s2 = src2; s.flags = e0; sl[ns++] = s;
    };
    auto swp = [&](uint16_t r1, uint16_t r2) {
      TabSlot s{}; s.kind = T_SWAP2; s.dst = r1; s.s1 = r1; s.s2 = r2; sl[ns++] = s;
    };
    auto sgn = [&](uint16_t r) { TabSlot s{}; s.kind = T_SIGN; s.dst = r; s.s1 = r; s.s2 = r; sl[ns++] = s; };
    switch (g.op) {
      case QW_OP_H: swp(X(a), Z(a)); break;
      case QW_OP_S: prod(X(a), Z(a), 3); break;
      case QW_OP_SDG: prod(X(a), Z(a), 1); break;
      case QW_OP_X: sgn(Z(a)); break;
      case QW_OP_Z: sgn(X(a)); break;
      case QW_OP_Y: sgn(X(a)); sgn(Z(a)); break;
      case QW_OP_CNOT: prod(X(a), X(b), 0); prod(Z(b), Z(a), 0); break;
      case QW_OP_CZ: prod(X(a), Z(b), 0); prod(X(b), Z(a), 0); break;
      case QW_OP_SWAP: swp(X(a), X(b)); swp(Z(a), Z(b)); break;
      default: fail(QW_ERR_INVALID_ARG, "tableau: non-Clifford op %u", g.op);
    }
    // conflict check against the current unitary layer
    bool conflict = (cur == 0xFFFFFFFFu) || cur_is_meas;
    for (int t = 0; t < ns && !conflict; t++) {
      const TabSlot &s = sl[t];
      uint16_t wr[2] = {s.dst, s.kind == T_SWAP2 ? s.s2 : s.dst};
      uint16_t rd[2] = {s.s1, s.s2};
      for (int u = 0; u < 2; u++)
        if (w_layer[wr[u]] == cur || r_layer[wr[u]] == cur) conflict = true;
      for (int u = 0; u < 2; u++)
        if (w_layer[rd[u]] == cur) conflict = true;
    }
    if (conflict) new_layer(false);
    for (int t = 0; t < ns; t++) {
      const TabSlot &s = sl[t];
      w_layer[s.dst] = cur;
      if (s.kind == T_SWAP2) w_layer[s.s2] = cur;
      r_layer[s.s1] = cur;
      r_layer[s.s2] = cur;
      P.slots.push_back(s);
      P.layers[cur].n_slots++;
    }
  }
  return P;
}

}  // namespace qw

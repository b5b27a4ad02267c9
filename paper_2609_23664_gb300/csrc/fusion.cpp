// Gate fusion (statevector) and layer compilation (tableau), host side.
//
// Statevector: a gate list is cut into PASSES.  A pass owns a set Q of at
// most k tile qubits (always containing the b lowest qubits so that every
// tile is read and written in contiguous runs of 2^b amplitudes); one CTA
// loads a tile (2^k amplitudes with the bits outside Q fixed) into shared
// memory, applies every gate of the pass and writes the tile back.  Gates
// are taken out of order only past gates on disjoint qubits (they commute).
// Inside a pass, gates are grouped into STAGES of at most G tile bits (5 for
// plain passes, 4 for compensated FP32 ones); a thread holds the 2^G
// amplitudes of one stage group in registers and applies the whole stage
// there.  Consecutive single-qubit gates on one qubit are
// multiplied into one 2x2 matrix in double precision.  Permutation gates
// (CNOT, SWAP, X) are index relabellings: the pass tracks an affine map over
// GF(2) from logical tile index to slot, and a permutation only changes that
// map, so CNOT chains cost no stage and no data movement.
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

// Greedy pass cover of the gates, in order (tile qubits, at most k;
// `forced` in every pass).  A gate joins the current pass when it touches no
// qubit blocked by an earlier skipped gate (it then commutes past every
// skipped gate) and its qubits still fit.  A CNOT whose control is not in
// the tile yet may also join with its control left outside (the control's
// bit is then fixed within each tile).  Such a control stays out of the pass: a
// later gate that acts on it, other than as the control of such a CNOT,
// waits for a later pass.  pass_out[i] = the outside controls of pass i.
static void pass_groups(const qw_gate *gates, const std::vector<uint32_t> &masks, uint32_t n_pos, uint32_t k,
                        uint32_t forced, std::vector<std::vector<uint32_t>> &groups,
                        std::vector<uint32_t> &group_masks, std::vector<uint32_t> &pass_out) {
  const uint32_t full = (n_pos >= 32) ? 0xFFFFFFFFu : ((1u << n_pos) - 1);
  std::vector<uint32_t> rem(masks.size());
  for (uint32_t i = 0; i < rem.size(); i++) rem[i] = i;
  while (!rem.empty()) {
    uint32_t Q = forced, blocked = 0, out = 0;
    std::vector<uint32_t> taken, keep;
    keep.reserve(rem.size());
    size_t i = 0;
    for (; i < rem.size(); i++) {
      const uint32_t gi = rem[i], qs = masks[gi];
      const qw_gate &g = gates[gi];
      if (qs & blocked) {
        blocked |= qs;
        keep.push_back(gi);
      } else if (!(qs & out) && (uint32_t)popc32(Q | qs) <= k) {
        Q |= qs;
        taken.push_back(gi);
      } else if (g.op == QW_OP_CNOT && !(Q & (1u << g.q0)) && !(out & (1u << g.q1)) &&
                 (uint32_t)popc32(Q | (1u << g.q1)) <= k &&
                 ((out & (1u << g.q0)) || popc32(out) < SV_MAX_OUT_CTL)) {
        Q |= 1u << g.q1;
        out |= 1u << g.q0;
        taken.push_back(gi);
      } else {
        blocked |= qs;
        keep.push_back(gi);
      }
      if (blocked == full) { i++; break; }
    }
    for (; i < rem.size(); i++) keep.push_back(rem[i]);
    if (taken.empty()) fail(QW_ERR_INVALID_ARG, "fusion: gate does not fit a pass");
    groups.push_back(std::move(taken));
    group_masks.push_back(Q);
    pass_out.push_back(out);
    rem.swap(keep);
  }
}

// Stage cover of a pass's gates (positions = tile bits, at most g per
// stage).  Permutation gates hold no positions: a stage takes one unless an
// earlier skipped gate shares a qubit with it, and it is applied after the
// stage's other gates, so a later non-permutation gate on one of its qubits
// waits for the next stage.  Another gate joins when no earlier skipped
// gate or taken permutation shares a position with it and the positions it
// reserves (cap_masks[i], a superset of masks[i]) still fit.
static void stage_groups(const std::vector<uint32_t> &masks, const std::vector<uint32_t> &cap_masks,
                         const std::vector<uint8_t> &perm, uint32_t g, std::vector<std::vector<uint32_t>> &groups,
                         std::vector<uint32_t> &group_masks) {
  std::vector<uint32_t> rem(masks.size());
  for (uint32_t i = 0; i < rem.size(); i++) rem[i] = i;
  while (!rem.empty()) {
    uint32_t Q = 0, blocked = 0, permq = 0;
    std::vector<uint32_t> taken, keep;
    keep.reserve(rem.size());
    for (const uint32_t gi : rem) {
      const uint32_t qs = masks[gi];
      if (perm[gi]) {
        if (qs & blocked) {
          blocked |= qs;
          keep.push_back(gi);
        } else {
          permq |= qs;
          taken.push_back(gi);
        }
        continue;
      }
      const uint32_t cs = qs | (cap_masks[gi] & ~blocked & ~permq);
      if (qs & (blocked | permq)) {
        blocked |= qs;
        keep.push_back(gi);
      } else if ((uint32_t)popc32(Q | cs) <= g) {
        Q |= cs;
        taken.push_back(gi);
      } else if ((uint32_t)popc32(Q | qs) <= g && (qs & Q) == qs) {
        taken.push_back(gi);
      } else {
        blocked |= qs;
        keep.push_back(gi);
      }
    }
    if (taken.empty()) fail(QW_ERR_INVALID_ARG, "fusion: gate does not fit a stage");
    groups.push_back(std::move(taken));
    group_masks.push_back(Q);
    rem.swap(keep);
  }
}

namespace {
// FP32 instructions per amplitude pair of each register-op kind (a real
// rotation uses packed two-lane FMAs)
int kind_cost(uint8_t k) {
  switch (k) {
    case K_U1: return 16;
    case K_D1: case K_RX: case K_RP: return 8;
    case K_R: case K_P1: return 4;
    default: return 16;
  }
}
// cheapest kind that represents the 2x2 matrix m exactly
uint8_t classify(const double m[8]) {
  const bool off0 = m[2] == 0 && m[3] == 0 && m[4] == 0 && m[5] == 0;
  if (off0) return (m[0] == 1.0 && m[1] == 0.0) ? K_P1 : K_D1;
  if (m[1] == 0 && m[3] == 0 && m[5] == 0 && m[7] == 0) return K_R;
  if (m[1] == 0 && m[7] == 0 && m[2] == 0 && m[4] == 0 && m[0] == m[6] && m[3] == m[5]) return K_RX;
  return K_U1;
}
void scale(double m[8], cd g) {
  for (int i = 0; i < 4; i++) {
    const cd v = cd(m[2 * i], m[2 * i + 1]) * g;
    m[2 * i] = v.real();
    m[2 * i + 1] = v.imag();
  }
}
}  // namespace

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
  const uint32_t G = tc.g;
  prog.g = G;
  if (G != (uint32_t)SV_G && G != (uint32_t)SV_G_COMP) fail(QW_ERR_STATE, "internal: stage width %u", G);
  if (n_gates == 0) return prog;
  const uint32_t k = std::min(tc.k_max, n_eff);
  const bool single = (n_eff <= tc.k_max);
  const uint32_t b = single ? n_eff : std::min(tc.b, k - 2);
  const uint32_t forced = (b >= 32) ? 0xFFFFFFFFu : ((1u << b) - 1);

  std::vector<uint32_t> masks(n_gates);
  for (uint64_t i = 0; i < n_gates; i++) masks[i] = gate_mask(gates[i]);

  std::vector<std::vector<uint32_t>> pass_gates;
  std::vector<uint32_t> pass_masks, pass_out;
  if (single) {
    std::vector<uint32_t> all(n_gates);
    for (uint64_t i = 0; i < n_gates; i++) all[i] = (uint32_t)i;
    pass_gates.push_back(all);
    pass_masks.push_back((n_eff >= 32) ? 0xFFFFFFFFu : ((1u << n_eff) - 1));
    pass_out.push_back(0);
  } else {
    pass_groups(gates, masks, n_eff, k, forced, pass_gates, pass_masks, pass_out);
  }

  cd gphase(1.0, 0.0);  // global phase pulled out of diagonal gates
  for (size_t p = 0; p < pass_gates.size(); p++) {
    HostPass hp;
    uint32_t Q = pass_masks[p];
    const uint32_t out = pass_out[p];
    // pad Q up to k with the lowest unused qubits (outside controls stay out)
    for (uint32_t q = 0; q < n_eff && (uint32_t)popc32(Q) < k; q++)
      if (!(out & (1u << q))) Q |= 1u << q;
    uint32_t loc[32];
    for (uint32_t q = 0; q < n_eff; q++)
      if (Q & (1u << q)) { loc[q] = (uint32_t)hp.q.size(); hp.q.push_back(q); }
    int ctl_slot[32];
    for (uint32_t q = 0; q < 32; q++) ctl_slot[q] = -1;
    for (uint32_t q = 0; q < n_eff; q++)
      if (out & (1u << q)) { ctl_slot[q] = (int)hp.ctl_q.size(); hp.ctl_q.push_back(q); }
    hp.b = b;
    hp.n_gates = (uint32_t)pass_gates[p].size();
    // stages inside the pass (positions = local tile bits).  Permutation
    // gates (CNOT, SWAP, X) move no data: they update the pass's affine map
    // from logical tile index to shared-memory slot, phi(l) = M l ^ c, at the
    // end of the stage that takes them, so they hold no stage positions.  A
    // single-qubit gate reserves the positions of a following two-position
    // phase gate on its qubit, so that both land in one stage.
    const size_t np = pass_gates[p].size();
    std::vector<uint32_t> lmask(np), emask(np);
    std::vector<uint8_t> lperm(np);
    auto outside_ctl = [&](const qw_gate &g) { return g.op == QW_OP_CNOT && (out & (1u << g.q0)); };
    for (size_t i = 0; i < np; i++) {
      const qw_gate &g = gates[pass_gates[p][i]];
      uint32_t m = outside_ctl(g) ? 0u : 1u << loc[g.q0];
      if (is_two_qubit_op(g.op)) m |= 1u << loc[g.q1];
      lmask[i] = m;
      lperm[i] = (g.op == QW_OP_CNOT || g.op == QW_OP_SWAP || g.op == QW_OP_X) ? 1 : 0;
    }
    std::vector<int> next_on(32, -1);
    for (size_t ii = np; ii-- > 0;) {
      const qw_gate &g = gates[pass_gates[p][ii]];
      if (outside_ctl(g)) {
        emask[ii] = 0;
        next_on[loc[g.q1]] = (int)ii;
        continue;
      }
      const uint32_t a = loc[g.q0];
      if (lperm[ii]) {
        emask[ii] = 0;
      } else if (!is_two_qubit_op(g.op)) {
        const int j = next_on[a];
        emask[ii] = (j < 0 || lperm[j]) ? lmask[ii] : emask[j];
      } else {
        emask[ii] = lmask[ii];
      }
      next_on[a] = (int)ii;
      if (is_two_qubit_op(g.op)) next_on[loc[g.q1]] = (int)ii;
    }
    std::vector<std::vector<uint32_t>> st_gates;
    std::vector<uint32_t> st_masks;
    stage_groups(lmask, emask, lperm, G, st_gates, st_masks);
    // phi as columns M e_t and constant c
    uint32_t mcol[32], mc = 0, ctl_w[SV_MAX_OUT_CTL] = {0, 0, 0, 0};
    for (uint32_t t = 0; t < 32; t++) mcol[t] = 1u << t;
    for (size_t s = 0; s < st_gates.size(); s++) {
      HostStage hs;
      for (uint32_t t = 0; t < k; t++) hs.mcol[t] = mcol[t];
      hs.mc = mc;
      for (int c = 0; c < SV_MAX_OUT_CTL; c++) hs.ctl_w[c] = ctl_w[c];
      // unused register positions are taken from the top: tile bit 0 is the
      // only one that reaches bank bit 0 of a slot, so it is kept for the
      // lanes (group bits) where it spreads a warp's accesses over the banks
      uint32_t P = st_masks[s];
      for (uint32_t q = k; q-- > 0 && popc32(P) < G;) P |= 1u << q;
      int rel[32];
      int j = 0;
      for (uint32_t q = 0; q < k; q++)
        if (P & (1u << q)) { hs.pos[j] = (uint8_t)q; rel[q] = j; j++; }
      int last1q[SV_G];
      for (int t = 0; t < SV_G; t++) last1q[t] = -1;
      std::vector<uint32_t> perms;  // applied to phi after the stage's ops
      for (uint32_t gi_local : st_gates[s]) {
        const qw_gate &g = gates[pass_gates[p][gi_local]];
        if (lperm[gi_local]) { perms.push_back(gi_local); continue; }
        const int a = rel[loc[g.q0]];
        HostOp op{};
        double m[8];
        bool diag = false;
        if (gate_matrix_1q(g, m, &diag)) {
          if (diag && !(m[0] == 1.0 && m[1] == 0.0)) {  // diag(d0,d1) = d0 diag(1, d1/d0)
            const cd d0(m[0], m[1]), d1(m[6], m[7]);
            gphase *= d0;
            const cd r = d1 / d0;
            m[0] = 1; m[1] = 0; m[6] = r.real(); m[7] = r.imag();
          }
          const uint8_t kn = classify(m);
          if (last1q[a] >= 0 && hs.ops[last1q[a]].kind == K_R && kn == K_P1) {
            // diag(1, p) after a real rotation: one op, its factors kept exact
            HostOp &prev = hs.ops[last1q[a]];
            double out[8];
            mat_mul(m, prev.m, out);
            prev.x[0] = prev.m[4];
            prev.x[1] = prev.m[6];
            prev.x[2] = m[6];
            prev.x[3] = m[7];
            std::memcpy(prev.m, out, sizeof(out));
            prev.kind = K_RP;
            continue;
          }
          if (last1q[a] >= 0) {
            HostOp &prev = hs.ops[last1q[a]];
            double out[8];
            mat_mul(m, prev.m, out);
            const uint8_t km = classify(out);
            if (kind_cost(km) <= kind_cost(prev.kind) + kind_cost(kn)) {
              std::memcpy(prev.m, out, sizeof(out));
              prev.kind = km;
              continue;
            }
          }
          op.kind = kn;
          op.a = (uint8_t)a;
          std::memcpy(op.m, m, sizeof(m));
          last1q[a] = (int)hs.ops.size();
          hs.ops.push_back(op);
          continue;
        }
        const int bb = rel[loc[g.q1]];
        op.a = (uint8_t)std::min(a, bb);
        op.b = (uint8_t)std::max(a, bb);
        op.kind = K_CD;
        if (g.op == QW_OP_CZ) { op.m[0] = -1; op.m[1] = 0; }
        else if (g.op == QW_OP_CPHASE) { op.m[0] = std::cos(g.theta); op.m[1] = std::sin(g.theta); }
        else fail(QW_ERR_INVALID_ARG, "fusion: unsupported statevector op %u", g.op);
        last1q[a] = -1;
        last1q[bb] = -1;
        hs.ops.push_back(op);
      }
      // the permutation pi of the stage's trailing gates: the amplitude of
      // logical index pi(l) stays in the slot of l, so phi <- phi o pi^-1
      for (uint32_t gi_local : perms) {
        const qw_gate &g = gates[pass_gates[p][gi_local]];
        if (outside_ctl(g)) {  // X on the target in tiles whose control bit is set
          ctl_w[ctl_slot[g.q0]] ^= mcol[loc[g.q1]];
          continue;
        }
        const uint32_t a = loc[g.q0];
        if (g.op == QW_OP_X) mc ^= mcol[a];
        else if (g.op == QW_OP_CNOT) mcol[a] ^= mcol[loc[g.q1]];
        else std::swap(mcol[a], mcol[loc[g.q1]]);
      }
      if (!hs.ops.empty()) hp.stages.push_back(std::move(hs));
    }
    for (uint32_t t = 0; t < k; t++) hp.mcol[t] = mcol[t];
    hp.mc = mc;
    for (int c = 0; c < SV_MAX_OUT_CTL; c++) hp.ctl_w[c] = ctl_w[c];
    prog.passes.push_back(std::move(hp));
  }
  // fold the global phase into one single-qubit op (every amplitude is in
  // exactly one of its pairs): the first general op if there is one, else
  // the first single-qubit op of any kind
  // (compensated programs, stages of four positions: carried by the first
  // stage with a rotation on every position, whose phase table multiplies
  // every amplitude anyway, so that its ops stay rotations)
  if (gphase != cd(1.0, 0.0) && G == (uint32_t)SV_G_COMP && SV_G_PLAIN32 != SV_G_COMP) {
    for (auto &ps : prog.passes)
      for (auto &st : ps.stages) {
        if (gphase == cd(1.0, 0.0) || st.ops.size() != 4) continue;
        uint32_t mask = 0;
        bool rot = true;
        for (const HostOp &o : st.ops) {
          rot = rot && (o.kind == K_RP || o.kind == K_R) && !(mask & (1u << o.a));
          mask |= 1u << o.a;
        }
        if (rot && mask == 0xFu) {
          st.gphase[0] = gphase.real();
          st.gphase[1] = gphase.imag();
          gphase = cd(1.0, 0.0);
        }
      }
  }
  if (gphase != cd(1.0, 0.0)) {
    HostOp *target = nullptr;
    for (auto &ps : prog.passes)
      for (auto &st : ps.stages)
        for (auto &o : st.ops)
          if (!target && o.kind == K_U1) target = &o;
    for (auto &ps : prog.passes)
      for (auto &st : ps.stages)
        for (auto &o : st.ops)
          if (!target && o.kind != K_CD) target = &o;
    if (!target) fail(QW_ERR_INVALID_ARG, "fusion: global phase without a single-qubit op");
    scale(target->m, gphase);
    target->kind = classify(target->m);
  }
  // device layout of the diagonal kinds: D1 keeps {d0, d1} in m[0..3], P1 keeps
  // p in m[0..1]; the other kinds keep the full matrix
  for (auto &ps : prog.passes)
    for (auto &st : ps.stages)
      for (auto &o : st.ops) {
        if (o.kind == K_D1) { o.m[2] = o.m[6]; o.m[3] = o.m[7]; }
        if (o.kind == K_P1) { o.m[0] = o.m[6]; o.m[1] = o.m[7]; }
        if (o.kind == K_RX) { o.m[1] = -o.m[3]; }  // m[0] = c, m[1] = s (matrix [[c,-is],[-is,c]])
        if (o.kind == K_RP) {  // {r00, r01, r10, r11, pr, pi}
          const double r00 = o.m[0], r01 = o.m[2];
          o.m[0] = r00; o.m[1] = r01;
          o.m[2] = o.x[0]; o.m[3] = o.x[1]; o.m[4] = o.x[2]; o.m[5] = o.x[3];
          o.m[6] = 0; o.m[7] = 0;
        }
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

namespace qw {

// ---------------------------------------------------------------------------
// forward stabilizers of a kept inverse tableau (host)
// ---------------------------------------------------------------------------
// The tableau kernels keep T(P) = C^-1 P C: row j < n is T(X_j), row n + j
// is T(Z_j), each as W x-words then W z-words, and sign byte r (bit 0) of
// the row (-1)^r i^{popc(x & z)} X^x Z^z.  The state C|0...0> has the
// stabilizer generators S_i = C Z_i C^-1.  For the symplectic map T the
// inverse is Omega M^T Omega, so S_i has X-bit j = x-bit i of T(Z_j) and
// Z-bit j = x-bit i of T(X_j); its sign follows from T(S_i) = Z_i, with
// T(i^{u.v} X^u Z^v) = i^{u.v} prod_{j in u} T(X_j) prod_{j in v} T(Z_j)
// and Paulis kept as i^e X^x Z^z:
//   (e1, x1, z1)(e2, x2, z2) = (e1 + e2 + 2 popc(z1 & x2), x1 ^ x2, z1 ^ z2).
void stabilizers_from_inverse(uint32_t n, const uint64_t *rows, const uint8_t *sign, uint8_t *x, uint8_t *z,
                              uint8_t *s) {
  const uint32_t W = (n + 63) / 64;
  auto xw = [&](uint32_t r, uint32_t w) { return rows[(size_t)r * 2 * W + w]; };
  auto zw = [&](uint32_t r, uint32_t w) { return rows[(size_t)r * 2 * W + W + w]; };
  auto xbit = [&](uint32_t r, uint32_t i) { return (uint32_t)((xw(r, i >> 6) >> (i & 63)) & 1ull); };
  std::vector<uint64_t> ax(W), az(W);
  for (uint32_t i = 0; i < n; i++) {
    uint32_t e = 0;
    std::fill(ax.begin(), ax.end(), 0ull);
    std::fill(az.begin(), az.end(), 0ull);
    uint32_t uv = 0;
    for (uint32_t j = 0; j < n; j++) {
      const uint32_t u = xbit(n + j, i), v = xbit(j, i);
      x[(size_t)i * n + j] = (uint8_t)u;
      z[(size_t)i * n + j] = (uint8_t)v;
      uv += u & v;
    }
    e = uv & 3u;
    // acc = i^{u.v} * prod_{j in u} T(X_j) * prod_{j in v} T(Z_j)
    auto mul_row = [&](uint32_t r) {
      uint32_t c = 0, own = 0;
      for (uint32_t w = 0; w < W; w++) {
        c += (uint32_t)__builtin_popcountll(az[w] & xw(r, w));
        own += (uint32_t)__builtin_popcountll(xw(r, w) & zw(r, w));
      }
      const uint32_t er = (2u * (sign[r] & 1u) + own) & 3u;
      e = (e + er + 2u * c) & 3u;
      for (uint32_t w = 0; w < W; w++) {
        ax[w] ^= xw(r, w);
        az[w] ^= zw(r, w);
      }
    };
    for (uint32_t j = 0; j < n; j++)
      if (x[(size_t)i * n + j]) mul_row(j);
    for (uint32_t j = 0; j < n; j++)
      if (z[(size_t)i * n + j]) mul_row(n + j);
    // acc must be i^e Z_i with e in {0, 2}
    bool ok = (e & 1u) == 0;
    for (uint32_t w = 0; w < W && ok; w++) {
      const uint64_t zi = ((i >> 6) == w) ? (1ull << (i & 63)) : 0ull;
      ok = ax[w] == 0ull && az[w] == zi;
    }
    if (!ok) fail(QW_ERR_STATE, "the kept tableau is not a valid stabilizer tableau");
    s[i] = (uint8_t)(e == 2 ? 1 : 0);  // S_i = i^{-e} i^{u.v} X^u Z^v
  }
}

}  // namespace qw

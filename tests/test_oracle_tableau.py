"""Pins for the tableau oracle: agreement with the (separately pinned)
statevector oracle on random Clifford circuits, mid-circuit measurement
checked against a projective measurement written here in numpy, and
surface-code facts that follow from the code's layout (noiseless syndromes,
single-error detection events)."""
import numpy as np
import pytest

from oracle import oracle as orc
from stab_canonical import canonical
from paper_2609_23664_gb300 import workloads as W

CLIFF_1Q = [W.OP_H, W.OP_S, W.OP_SDG, W.OP_X, W.OP_Y, W.OP_Z]
CLIFF_2Q = [W.OP_CNOT, W.OP_CZ, W.OP_SWAP]


def rand_clifford(rng, n, k, p_meas=0.0, p_reset=0.0):
    g = []
    for _ in range(k):
        r = rng.random()
        a = int(rng.integers(0, n))
        if r < p_meas:
            g.append((W.OP_MEASURE, a, 0, float(rng.integers(0, 2))))
        elif r < p_meas + p_reset:
            g.append((W.OP_RESET, a, 0, float(rng.integers(0, 2))))
        elif rng.random() < 0.5:
            g.append((CLIFF_1Q[int(rng.integers(0, 6))], a, 0))
        else:
            b = int(rng.integers(0, n - 1))
            b = b + 1 if b >= a else b
            g.append((CLIFF_2Q[int(rng.integers(0, 3))], a, b))
    return W.gates_from_list(g)


@pytest.mark.parametrize("n,seed", [(2, 1), (4, 2), (6, 3), (8, 4), (8, 5)])
def test_stabilizers_have_expectation_plus_one(n, seed):
    rng = np.random.default_rng(seed)
    g = rand_clifford(rng, n, 80)
    _, (x, z, r) = orc.tab_run(n, g, want_tableau=True)
    psi = orc.sv_run(n, g)
    for i in range(n, 2 * n):
        xm = int(sum(int(x[i, q]) << q for q in range(n)))
        zm = int(sum(int(z[i, q]) << q for q in range(n)))
        val = orc.pauli_expect(n, psi, xm, zm) * (-1) ** int(r[i])
        assert abs(val - 1) < 1e-12, (i, val)


def projective_reference(n, gates, rng_check=None):
    """Statevector with projective Z measurements (numpy), outcome taken
    from the record's bit only when both outcomes have probability 1/2."""
    psi = orc.sv_zero(n)
    outs = []
    for g in gates:
        op, a = int(g["op"]), int(g["q0"])
        if op in (W.OP_MEASURE, W.OP_RESET):
            idx = np.arange(1 << n)
            one = ((idx >> a) & 1).astype(bool)
            p1 = float(np.sum(np.abs(psi[one]) ** 2))
            if p1 < 1e-9:
                o = 0
            elif p1 > 1 - 1e-9:
                o = 1
            else:
                assert abs(p1 - 0.5) < 1e-9
                o = int(g["theta"])
            keep = one if o else ~one
            psi = np.where(keep, psi, 0)
            psi = psi / np.linalg.norm(psi)
            if op == W.OP_MEASURE:
                outs.append(o)
            elif o:
                psi = orc.sv_apply(n, np.ascontiguousarray(psi),
                                   W.gates_from_list([(W.OP_X, a, 0)]))
        else:
            psi = orc.sv_apply(n, np.ascontiguousarray(psi), W.gates_from_list([
                (op, a, int(g["q1"]), float(g["theta"]))]))
    return np.array(outs, dtype=np.uint8)


@pytest.mark.parametrize("n,seed", [(3, 10), (5, 11), (7, 12), (9, 13)])
def test_mid_circuit_measurement_vs_projective_statevector(n, seed):
    rng = np.random.default_rng(seed)
    g = rand_clifford(rng, n, 150, p_meas=0.15, p_reset=0.05)
    got = orc.tab_run(n, g)
    ref = projective_reference(n, g)
    assert np.array_equal(got, ref)


def run_code(d, rounds, errors=None):
    code = W.rotated_surface_code(d)
    rng = np.random.default_rng(d)
    parts = []
    for t in range(rounds):
        if errors and t in errors:
            parts.append(W.gates_from_list(errors[t]))
        parts.append(W.syndrome_round(code, rng))
    g = W.concat(*parts)
    out = orc.tab_run(code.n, g)
    anc = sorted(code.sched.keys())
    return code, out.reshape(rounds, len(anc)), anc


@pytest.mark.parametrize("d", [3, 5])
def test_surface_code_noiseless_syndromes(d):
    code, syn, anc = run_code(d, 6)
    assert code.n == 2 * d * d - 1
    assert len(code.x_anc) == len(code.z_anc) == (d * d - 1) // 2
    zcols = [anc.index(a) for a in code.z_anc]
    xcols = [anc.index(a) for a in code.x_anc]
    assert np.all(syn[:, zcols] == 0)
    assert np.all(syn[1:, xcols] == syn[0, xcols])


@pytest.mark.parametrize("d", [3, 5])
def test_single_x_error_flips_adjacent_z_checks(d):
    code = W.rotated_surface_code(d)
    anc = sorted(code.sched.keys())
    for q in range(code.n_data):
        _, base, _ = run_code(d, 4)
        _, syn, _ = run_code(d, 4, errors={2: [(W.OP_X, q, 0)]})
        det = syn ^ base
        expect = {anc.index(a) for a in code.z_anc if q in code.sched[a]}
        assert 1 <= len(expect) <= 2
        assert not det[:2].any()
        assert set(np.nonzero(det[2])[0]) == expect
        assert np.array_equal(det[3], det[2])   # persistent flip


def test_surface_code_d15_size():
    code = W.rotated_surface_code(15)
    assert code.n == 449 and len(code.x_anc) == 112 and len(code.z_anc) == 112
    cnots = sum(1 for a in code.sched for q in code.sched[a] if q is not None)
    assert cnots == 840


@pytest.mark.parametrize("seed", range(6))
def test_continuing_from_exported_rows_equals_the_run_from_zero(seed):
    # the tableau algorithm is deterministic: running a prefix, exporting its
    # rows and continuing with the suffix gives the outcomes and the final
    # rows of the whole circuit run from |0...0>, random-outcome
    # measurements and resets included
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(3, 9))
    ops = [W.OP_H, W.OP_S, W.OP_SDG, W.OP_X, W.OP_Y, W.OP_Z, W.OP_CNOT, W.OP_CZ, W.OP_SWAP,
           W.OP_MEASURE, W.OP_RESET]
    g = []
    for _ in range(120):
        op = ops[int(rng.integers(0, len(ops)))]
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        g.append((op, a, b, float(rng.integers(0, 2))))
    gates = W.gates_from_list(g)
    cut = int(rng.integers(1, len(gates)))
    pre, suf = gates[:cut], gates[cut:]
    whole, t_whole = orc.tab_run(n, gates, want_tableau=True)
    out_pre, t_pre = orc.tab_run(n, pre, want_tableau=True)
    out_suf, t_suf = orc.tab_run_from(n, t_pre, suf, want_tableau=True)
    assert np.array_equal(whole, np.concatenate([out_pre, out_suf]))
    for a, b in zip(t_whole, t_suf):
        assert np.array_equal(a, b)


def test_continuing_a_surface_code_task_from_its_shared_rounds():
    tasks = W.qec_surface_code_tasks(d=5, shared_rounds=6, task_rounds=3, n_tasks=4, p=0.05)
    pre_out, rows = orc.tab_run(tasks[0].n, tasks[0].spans[0], want_tableau=True)
    for t in tasks:
        assert t.spans[0] is tasks[0].spans[0]
        suf = W.concat(*t.spans[1:])
        got = np.concatenate([pre_out, orc.tab_run_from(t.n, rows, suf)])
        assert np.array_equal(got, orc.tab_run(t.n, t.gates))


def test_canonical_form_is_a_group_invariant():
    # the same group from two different generating sets: the oracle's
    # stabilizers, and the same rows each multiplied by the next one
    rng = np.random.default_rng(3)
    t = W.Task(mode=W.MODE_TABLEAU, n=9, spans=[rand_clifford(rng, 9, 200, p_meas=0.08, p_reset=0.04)])
    _, (x, z, r) = orc.tab_run(t.n, t.gates, want_tableau=True)
    n = t.n
    x, z, r = x[n:].astype(np.uint8), z[n:].astype(np.uint8), r[n:].astype(np.uint8)
    e = (2 * r.astype(np.int64) + np.sum(x.astype(np.int64) & z, axis=1)) % 4
    x2, z2, e2 = x.copy(), z.copy(), e.copy()
    for i in range(n - 1):
        e2[i] = (e[i] + e[i + 1] + 2 * int(np.sum(z[i].astype(np.int64) & x[i + 1]))) % 4
        x2[i] ^= x[i + 1]
        z2[i] ^= z[i + 1]
    r2 = ((e2 - np.sum(x2.astype(np.int64) & z2, axis=1)) % 4 // 2).astype(np.uint8)
    for a, b in zip(canonical(x, z, r), canonical(x2, z2, r2)):
        assert np.array_equal(a, b)

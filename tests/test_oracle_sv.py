"""Pins for the statevector oracle against facts that do not come from it:
closed forms (Bell, GHZ, QFT of basis states, product states), dense
Kronecker-product unitaries built here from textbook definitions and
scipy.linalg.expm, norm preservation, and brute-force CDF sampling."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as orc
from paper_2609_23664_gb300 import workloads as W

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def embed(n, ops):
    """ops: {qubit: 2x2}; little-endian (qubit q = bit q) so the Kronecker
    product runs from qubit n-1 (left) down to qubit 0 (right)."""
    m = np.array([[1.0 + 0j]])
    for q in reversed(range(n)):
        m = np.kron(m, ops.get(q, I2))
    return m


def dense_gate(n, g):
    op, a, b, th = int(g["op"]), int(g["q0"]), int(g["q1"]), float(g["theta"])
    one = {
        W.OP_H: (PX + PZ) / math.sqrt(2), W.OP_X: PX, W.OP_Y: PY, W.OP_Z: PZ,
        W.OP_S: np.diag([1, 1j]), W.OP_SDG: np.diag([1, -1j]),
        W.OP_T: np.diag([1, np.exp(1j * math.pi / 4)]),
        W.OP_TDG: np.diag([1, np.exp(-1j * math.pi / 4)]),
        W.OP_RX: scipy.linalg.expm(-0.5j * th * PX),
        W.OP_RY: scipy.linalg.expm(-0.5j * th * PY),
        W.OP_RZ: scipy.linalg.expm(-0.5j * th * PZ),
        W.OP_PHASE: np.diag([1, np.exp(1j * th)]),
    }
    if op in one:
        return embed(n, {a: one[op]})
    if op == W.OP_CNOT:
        return embed(n, {a: P0}) + embed(n, {a: P1, b: PX})
    if op == W.OP_CZ:
        return embed(n, {}) - 2 * embed(n, {a: P1, b: P1})
    if op == W.OP_CPHASE:
        return embed(n, {}) + (np.exp(1j * th) - 1) * embed(n, {a: P1, b: P1})
    if op == W.OP_SWAP:
        return 0.5 * (embed(n, {}) + embed(n, {a: PX, b: PX}) + embed(n, {a: PY, b: PY})
                      + embed(n, {a: PZ, b: PZ}))
    raise ValueError(op)


def rand_state(rng, n):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


def rand_gate_list(rng, n, k, ops=None):
    ops = ops or [W.OP_H, W.OP_X, W.OP_Y, W.OP_Z, W.OP_S, W.OP_SDG, W.OP_T, W.OP_TDG,
                  W.OP_RX, W.OP_RY, W.OP_RZ, W.OP_PHASE, W.OP_CNOT, W.OP_CZ, W.OP_SWAP,
                  W.OP_CPHASE]
    g = []
    for _ in range(k):
        op = ops[int(rng.integers(0, len(ops)))]
        a = int(rng.integers(0, n))
        b = int(rng.integers(0, n - 1))
        b = b + 1 if b >= a else b
        g.append((op, a, b, float(rng.uniform(0, 2 * math.pi))))
    return W.gates_from_list(g)


def test_bell():
    psi = orc.sv_run(2, W.bell_circuit())
    r = 1 / math.sqrt(2)
    assert np.allclose(psi, [r, 0, 0, r], atol=1e-15)


@pytest.mark.parametrize("n", [2, 3, 5, 8, 11])
def test_ghz(n):
    psi = orc.sv_run(n, W.ghz_circuit(n))
    ref = np.zeros(1 << n, complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - ref)) < 1e-15


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_qft_of_basis_states(n):
    N = 1 << n
    for j in range(N):
        psi = orc.sv_run(n, W.concat(W.basis_state_circuit(n, j), W.qft_circuit(n)))
        k = np.arange(N)
        ref = np.exp(2j * math.pi * j * k / N) / math.sqrt(N)
        assert np.max(np.abs(psi - ref)) < 1e-13, (n, j)


@pytest.mark.parametrize("op", [W.OP_H, W.OP_X, W.OP_Y, W.OP_Z, W.OP_S, W.OP_SDG, W.OP_T,
                                W.OP_TDG, W.OP_RX, W.OP_RY, W.OP_RZ, W.OP_PHASE])
def test_every_1q_gate_vs_dense(op):
    rng = np.random.default_rng(op)
    n = 4
    for q in range(n):
        g = W.gates_from_list([(op, q, 0, float(rng.uniform(0, 2 * math.pi)))])
        psi0 = rand_state(rng, n)
        got = orc.sv_apply(n, psi0.copy(), g)
        ref = dense_gate(n, g[0]) @ psi0
        assert np.max(np.abs(got - ref)) < 1e-14


@pytest.mark.parametrize("op", [W.OP_CNOT, W.OP_CZ, W.OP_SWAP, W.OP_CPHASE])
def test_every_2q_gate_vs_dense(op):
    rng = np.random.default_rng(100 + op)
    n = 4
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            g = W.gates_from_list([(op, a, b, float(rng.uniform(0, 2 * math.pi)))])
            psi0 = rand_state(rng, n)
            got = orc.sv_apply(n, psi0.copy(), g)
            ref = dense_gate(n, g[0]) @ psi0
            assert np.max(np.abs(got - ref)) < 1e-14


@pytest.mark.parametrize("n,seed", [(5, 1), (6, 2), (3, 3)])
def test_random_circuit_vs_dense_product(n, seed):
    rng = np.random.default_rng(seed)
    gl = rand_gate_list(rng, n, 40)
    U = np.eye(1 << n, dtype=complex)
    for g in gl:
        U = dense_gate(n, g) @ U
    got = orc.sv_run(n, gl)
    assert np.max(np.abs(got - U[:, 0])) < 1e-13


def test_norm_preserved():
    rng = np.random.default_rng(7)
    n = 12
    psi = orc.sv_run(n, rand_gate_list(rng, n, 200))
    assert abs(orc.norm2(n, psi) - 1.0) < 1e-12


def test_hadamard_uniform():
    n = 9
    psi = orc.sv_run(n, W.gates_from_list([(W.OP_H, q, 0) for q in range(n)]))
    assert np.max(np.abs(psi - 1 / math.sqrt(1 << n))) < 1e-15


def test_product_state_single_qubit_expectations():
    """RY(theta_q)|0>: <Z_q> = cos theta_q, <X_q> = sin theta_q, <Y_q> = 0."""
    rng = np.random.default_rng(11)
    n = 7
    th = rng.uniform(0, 2 * math.pi, n)
    psi = orc.sv_run(n, W.gates_from_list([(W.OP_RY, q, 0, th[q]) for q in range(n)]))
    for q in range(n):
        assert abs(orc.pauli_expect(n, psi, 0, 1 << q) - math.cos(th[q])) < 1e-14
        assert abs(orc.pauli_expect(n, psi, 1 << q, 0) - math.sin(th[q])) < 1e-14
        assert abs(orc.pauli_expect(n, psi, 1 << q, 1 << q)) < 1e-14
    # energy of sum_q c_q Z_q + d_q X_q is the closed-form sum
    c, d = rng.normal(size=n), rng.normal(size=n)
    terms = np.zeros(2 * n, dtype=W.TERM_DTYPE)
    for q in range(n):
        terms[2 * q] = (c[q], 0, 1 << q)
        terms[2 * q + 1] = (d[q], 1 << q, 0)
    e, nr, _ = orc.energy(n, psi, terms)
    assert abs(e - float(np.sum(c * np.cos(th) + d * np.sin(th)))) < 1e-13
    assert abs(nr - 1) < 1e-14


def test_ghz_stabilizers():
    n = 6
    psi = orc.sv_run(n, W.ghz_circuit(n))
    full = (1 << n) - 1
    assert abs(orc.pauli_expect(n, psi, full, 0) - 1) < 1e-14          # X^n
    for i in range(n):
        assert abs(orc.pauli_expect(n, psi, 0, 1 << i)) < 1e-14        # Z_i
        for j in range(i + 1, n):
            assert abs(orc.pauli_expect(n, psi, 0, (1 << i) | (1 << j)) - 1) < 1e-14
    # Y Y X X X X on GHZ_6: i^2 * (-1)^{...}: <Y0 Y1 X2..X5> = -1
    assert abs(orc.pauli_expect(n, psi, full, 0b11) + 1) < 1e-14


def pauli_matrix(n, xm, zm):
    ops = {}
    for q in range(n):
        x, z = (xm >> q) & 1, (zm >> q) & 1
        if x or z:
            ops[q] = PY if (x and z) else (PX if x else PZ)
    return embed(n, ops)


@pytest.mark.parametrize("n", [1, 3, 5, 6])
def test_energy_vs_kronecker_matrices(n):
    rng = np.random.default_rng(20 + n)
    psi = 1.7 * rand_state(rng, n)          # deliberately unnormalized
    terms = W.random_pauli_hamiltonian(rng, n, 25)
    H = sum(t["coef"] * pauli_matrix(n, int(t["xmask"]), int(t["zmask"])) for t in terms)
    ref = (np.vdot(psi, H @ psi) / np.vdot(psi, psi)).real
    e, nr, per = orc.energy(n, psi, terms)
    assert abs(e - ref) < 1e-12
    assert abs(nr - np.vdot(psi, psi).real) < 1e-12
    for t, v in zip(terms, per):
        P = pauli_matrix(n, int(t["xmask"]), int(t["zmask"]))
        assert abs(v - np.vdot(psi, P @ psi).real) < 1e-12


def test_sampling_basis_state_is_certain():
    n = 6
    psi = orc.sv_run(n, W.basis_state_circuit(n, 45))
    u = np.random.default_rng(1).random(50)
    assert np.all(orc.sample(n, psi, u) == 45)


def test_sampling_brute_force_cdf():
    rng = np.random.default_rng(5)
    n = 8
    psi = orc.sv_run(n, rand_gate_list(rng, n, 60))
    u = rng.random(2000)
    p = np.abs(psi) ** 2
    p = p / p.sum()
    F = np.cumsum(p)
    ref = np.searchsorted(F, u, side="right")
    got = orc.sample(n, psi, u)
    near = np.abs(F[np.minimum(ref, len(F) - 1)] - u) < 1e-12
    assert np.all((got == ref) | near)


def test_sampling_uniform_distribution():
    n = 5
    psi = orc.sv_run(n, W.gates_from_list([(W.OP_H, q, 0) for q in range(n)]))
    u = np.random.default_rng(9).random(20000)
    s = orc.sample(n, psi, u)
    k = np.floor(u * 32).astype(np.int64)
    frac_near = np.abs(u * 32 - np.round(u * 32)) < 1e-9
    assert np.all((s == k) | frac_near)
    counts = np.bincount(s.astype(np.int64), minlength=32)
    chi2 = float(np.sum((counts - 20000 / 32) ** 2 / (20000 / 32)))
    assert chi2 < 70   # 31 dof, p ~ 1e-4


def test_invalid_gate_rejected():
    with pytest.raises(ValueError):
        orc.sv_run(3, W.gates_from_list([(W.OP_CNOT, 1, 1)]))
    with pytest.raises(ValueError):
        orc.sv_run(3, W.gates_from_list([(W.OP_H, 5, 0)]))

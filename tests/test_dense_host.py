"""Dense blocks without a GPU: the oracle's k-qubit operator application
pinned against independent formulations, and the host-side fusion of gate
lists into blocks (qw_dense_fuse) checked against the oracle's gate-by-gate
evolution."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2609_23664_gb300 import quwarp as Q
from paper_2609_23664_gb300 import workloads as W


def random_state(rng, n):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


def random_unitary(rng, d):
    z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def tensordot_apply(n, psi, qubits, u):
    """Independent formulation: psi as an n-axis tensor (axis a <-> qubit
    n-1-a), u as a 2k-axis tensor (output axes, then input axes; local bit j
    <-> axis k-1-j), contracted over the block's axes."""
    k = len(qubits)
    t = psi.reshape((2,) * n)
    ut = u.reshape((2,) * (2 * k))
    axes_in = [n - 1 - qubits[k - 1 - a] for a in range(k)]  # tensor axis of u's input axis k+a
    res = np.tensordot(ut, t, axes=(list(range(k, 2 * k)), axes_in))
    # res axes: u's output axes (local bits k-1..0), then the remaining state axes in order
    rest = [a for a in range(n) if a not in axes_in]
    order = [None] * n
    for a in range(k):
        order[axes_in[a]] = a
    for i, a in enumerate(rest):
        order[a] = k + i
    return np.transpose(res, order).reshape(-1)


ONE_Q = [(W.OP_H, 0.0), (W.OP_X, 0.0), (W.OP_Y, 0.0), (W.OP_Z, 0.0), (W.OP_S, 0.0), (W.OP_T, 0.0),
         (W.OP_RX, 0.7), (W.OP_RY, -1.3), (W.OP_RZ, 2.1), (W.OP_PHASE, 0.4)]


def gate_matrix_via_oracle(op, theta):
    """2x2 matrix of a one-qubit gate, read off the oracle's action on |0>, |1>."""
    cols = []
    for b in (0, 1):
        psi = np.zeros(2, dtype=np.complex128)
        psi[b] = 1
        cols.append(orc.sv_apply(1, psi, W.gates_from_list([(op, 0, 0, theta)])).copy())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("seed", range(4))
def test_apply_matrix_matches_tensordot_formulation(seed):
    rng = np.random.default_rng(seed)
    n = 6
    for k in range(1, 6):
        qubits = list(rng.permutation(n)[:k])
        u = random_unitary(rng, 1 << k)
        psi = random_state(rng, n)
        got = orc.apply_matrix(n, psi, qubits, u)
        assert np.max(np.abs(got - tensordot_apply(n, psi, qubits, u))) < 1e-13
        assert abs(np.linalg.norm(got) - 1.0) < 1e-13


def test_apply_matrix_of_a_kronecker_product_equals_the_gates():
    # u = M2 (x) M1 (x) M0 on qubits (q0, q1, q2): local bit j <-> q_j, bit 0 least significant
    rng = np.random.default_rng(5)
    n, qubits = 7, [4, 1, 6]
    ops = [ONE_Q[i] for i in rng.choice(len(ONE_Q), 3)]
    mats = [gate_matrix_via_oracle(op, th) for op, th in ops]
    u = np.kron(mats[2], np.kron(mats[1], mats[0]))
    psi = random_state(rng, n)
    want = orc.sv_apply(n, psi.copy(), W.gates_from_list([(op, q, 0, th) for (op, th), q in zip(ops, qubits)]))
    assert np.max(np.abs(orc.apply_matrix(n, psi, qubits, u) - want)) < 1e-14


def test_apply_matrix_of_two_qubit_permutations_equals_the_gates():
    rng = np.random.default_rng(6)
    n = 5
    cnot = np.eye(4)[[0, 3, 2, 1]]       # local bit 0 = control, bit 1 = target: |c=1,t> -> |c=1,1-t>
    cz = np.diag([1, 1, 1, -1]).astype(complex)
    swap = np.eye(4)[[0, 2, 1, 3]]
    for op, u in ((W.OP_CNOT, cnot), (W.OP_CZ, cz), (W.OP_SWAP, swap)):
        psi = random_state(rng, n)
        want = orc.sv_apply(n, psi.copy(), W.gates_from_list([(op, 3, 1)]))
        assert np.max(np.abs(orc.apply_matrix(n, psi, [3, 1], u) - want)) < 1e-15, op


def random_gate_list(rng, n, count):
    ops = []
    for _ in range(count):
        if rng.random() < 0.35 and n > 1:
            a, b = rng.choice(n, 2, replace=False)
            op = int(rng.choice([W.OP_CNOT, W.OP_CZ, W.OP_SWAP, W.OP_CPHASE]))
            ops.append((op, int(a), int(b), float(rng.uniform(-3, 3))))
        else:
            op, _ = ONE_Q[int(rng.integers(len(ONE_Q)))]
            ops.append((op, int(rng.integers(n)), 0, float(rng.uniform(-3, 3))))
    return W.gates_from_list(ops)


@pytest.mark.parametrize("kmax", [2, 3, 4, 5])
@pytest.mark.parametrize("seed", range(3))
def test_fused_blocks_reproduce_the_gate_list(kmax, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 10))
    g = random_gate_list(rng, n, 80)
    blocks = Q.dense_fuse(g, n, kmax)
    psi = orc.sv_zero(n)
    psi[:] = random_state(rng, n)
    want = orc.sv_apply(n, psi.copy(), g)
    got = psi.copy()
    for qubits, u in blocks:
        assert 1 <= len(qubits) <= kmax and len(set(qubits)) == len(qubits)
        assert np.max(np.abs(u.conj().T @ u - np.eye(len(u)))) < 1e-12
        got = orc.apply_matrix(n, got, list(qubits), u)
    assert np.max(np.abs(got - want)) < 1e-12
    assert len(blocks) < len(g)


def test_hardware_efficient_layer_fuses_into_overlapping_five_qubit_blocks():
    rng = np.random.default_rng(2)
    g = W.hea_circuit(rng, 24, 1)          # RY, RZ on 24 qubits, then CNOT(q, q+1) chain
    blocks = Q.dense_fuse(g, 24, 5)
    assert [q for q, _ in blocks] == [(0, 1, 2, 3, 4), (4, 5, 6, 7, 8), (8, 9, 10, 11, 12),
                                      (12, 13, 14, 15, 16), (16, 17, 18, 19, 20), (20, 21, 22, 23)]


def test_fusion_rejects_measurements_and_bad_widths():
    g = W.gates_from_list([(W.OP_H, 0, 0), (W.OP_MEASURE, 0, 0, 0.0)])
    with pytest.raises(Q.QuwarpError) as e:
        Q.dense_fuse(g, 3, 5)
    assert e.value.status == -9
    for kmax in (1, 6):
        with pytest.raises(Q.QuwarpError) as e:
            Q.dense_fuse(W.gates_from_list([(W.OP_H, 0, 0)]), 3, kmax)
        assert e.value.status == -1

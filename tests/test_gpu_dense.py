"""Dense blocks on the GPU against the oracle: single explicit blocks (random
unitaries on arbitrary qubits, 1 to 5 qubits), fused gate lists, and the
24-qubit hardware-efficient suffix shape, on the tensor cores (3xTF32 with
1, 2 or 4 accumulators) and on the CUDA cores (FP32 and FP64)."""
import numpy as np
import pytest

from energy_tol import FP32_ENERGY_TOL, energy_error
from oracle import oracle as orc
from paper_2609_23664_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_23664_gb300 import quwarp as Q  # noqa: E402

T, S = Q.DENSE_TENSOR, Q.DENSE_SIMT
FP32, FP64 = W.MODE_SV_FP32, W.MODE_SV_FP64
# Relative 2-norm error of one block application, FP32 state.  3xTF32 drops
# the lo*lo product (2^-22 relative) and the tensor core accumulates the 24
# partial products of a 64-term dot product in FP32 with its own rounding;
# spreading the K-steps over more accumulators that the CUDA cores add in
# round-to-nearest lowers the error.  The bounds are a few times the errors
# measured on GB300 (random unitaries and states).
REL_TOL = {(T, 1): 4e-6, (T, 2): 3e-6, (T, 4): 2e-6, (S, 0): 1e-6}


@pytest.fixture(scope="module")
def eng():
    e = Q.Engine(0)
    yield e
    e.close()


def random_state(rng, n):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


def random_unitary(rng, d):
    z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def run_prog(prog, psi, mode):
    st = torch.tensor(psi, dtype=torch.complex128 if mode == FP64 else torch.complex64, device="cuda")
    prog.run(st.data_ptr())
    prog.check()
    return st.cpu().numpy().astype(np.complex128)


def rounded(psi, mode):
    return psi if mode == FP64 else psi.astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("engine,nacc", [(T, 1), (T, 2), (T, 4), (S, 0)])
@pytest.mark.parametrize("n,qubits", [(12, [0, 1, 2, 3, 4]), (13, [12, 0, 7, 3, 9]), (16, [15, 14, 13, 12, 11]),
                                      (16, [2, 9]), (20, [19, 0, 10]), (14, [5]), (17, [3, 4, 5, 6]),
                                      (15, [1, 6, 3]), (16, [3, 1, 4, 2]), (20, [4, 3, 0, 1, 19])])
def test_single_block_matches_oracle(eng, engine, nacc, n, qubits):
    rng = np.random.default_rng(n * 31 + len(qubits))
    u = random_unitary(rng, 1 << len(qubits))
    psi = rounded(random_state(rng, n), FP32)
    prog = Q.DenseProgram(eng, FP32, n, engine_kind=engine, nacc=max(nacc, 1), block=(qubits, u))
    got = run_prog(prog, psi, FP32)
    want = orc.apply_matrix(n, psi, qubits, u)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert np.max(np.abs(got - want)) <= 1e-5
    assert rel <= REL_TOL[(engine, nacc)], rel
    prog.close()


@pytest.mark.parametrize("n,k", [(5, 5), (10, 3), (14, 5), (9, 1)])
def test_fp64_block_on_cuda_cores_matches_oracle(eng, n, k):
    rng = np.random.default_rng(7 * n + k)
    qubits = list(rng.permutation(n)[:k])
    u = random_unitary(rng, 1 << k)
    psi = random_state(rng, n)
    prog = Q.DenseProgram(eng, FP64, n, engine_kind=S, block=(qubits, u))
    got = run_prog(prog, psi, FP64)
    assert np.max(np.abs(got - orc.apply_matrix(n, psi, qubits, u))) <= 1e-12


def random_gate_list(rng, n, count):
    one = [W.OP_H, W.OP_X, W.OP_Y, W.OP_Z, W.OP_S, W.OP_SDG, W.OP_T, W.OP_TDG, W.OP_RX, W.OP_RY, W.OP_RZ,
           W.OP_PHASE]
    ops = []
    for _ in range(count):
        if rng.random() < 0.35:
            a, b = rng.choice(n, 2, replace=False)
            ops.append((int(rng.choice([W.OP_CNOT, W.OP_CZ, W.OP_SWAP, W.OP_CPHASE])), int(a), int(b),
                        float(rng.uniform(-3, 3))))
        else:
            ops.append((int(rng.choice(one)), int(rng.integers(n)), 0, float(rng.uniform(-3, 3))))
    return W.gates_from_list(ops)


@pytest.mark.parametrize("mode,engine,nacc", [(FP32, T, 1), (FP32, T, 4), (FP32, S, 1), (FP64, S, 1)])
@pytest.mark.parametrize("n,kmax,seed", [(12, 5, 0), (13, 4, 1), (16, 5, 2), (15, 3, 3)])
def test_fused_gate_list_matches_oracle(eng, mode, engine, nacc, n, kmax, seed):
    rng = np.random.default_rng(500 + seed)
    g = random_gate_list(rng, n, 150)
    psi = rounded(random_state(rng, n), mode)
    prog = Q.DenseProgram(eng, mode, n, gates=g, kmax=kmax, engine_kind=engine, nacc=nacc)
    info = prog.info()
    assert info["gates"] == len(g) and 0 < info["blocks"] < len(g)
    got = run_prog(prog, psi, mode)
    want = orc.sv_apply(n, psi.copy(), g)
    if mode == FP64:
        assert np.max(np.abs(got - want)) <= 1e-12
    else:
        assert np.max(np.abs(got - want)) <= 1e-5
        assert np.linalg.norm(got - want) <= 2e-5


@pytest.mark.parametrize("nacc", [1, 4])
def test_hardware_efficient_suffix_at_24_qubits(eng, nacc):
    # the statevector suffix shape of the 24-qubit VQE sweep: 4 layers of RY,
    # RZ on every qubit and a CNOT chain, from a random FP32 state
    n = 24
    rng = np.random.default_rng(24)
    g = W.hea_circuit(rng, n, 4)
    psi = rounded(random_state(rng, n), FP32)
    prog = Q.DenseProgram(eng, FP32, n, gates=g, kmax=5, engine_kind=T, nacc=nacc)
    assert prog.info()["blocks"] == 24
    got = run_prog(prog, psi, FP32)
    want = orc.sv_apply(n, psi.copy(), g)
    assert np.max(np.abs(got - want)) <= 1e-5
    assert np.linalg.norm(got - want) <= (1.5e-5 if nacc == 1 else 1e-5)
    # the pass kernels on the same input agree to FP32 rounding as well
    st = torch.tensor(psi, dtype=torch.complex64, device="cuda")
    Q.sv_apply_dev(eng, FP32, n, st.data_ptr(), g)
    assert np.linalg.norm(st.cpu().numpy().astype(np.complex128) - want) <= 1e-5


def test_invalid_dense_requests_are_refused(eng):
    u = np.eye(4, dtype=np.complex128)
    with pytest.raises(Q.QuwarpError) as e:      # tensor cores take FP32 states only
        Q.DenseProgram(eng, FP64, 14, engine_kind=T, block=([0, 1], u))
    assert e.value.status == -9
    with pytest.raises(Q.QuwarpError) as e:      # 5 block bits + 7 row bits at least
        Q.DenseProgram(eng, FP32, 11, engine_kind=T, block=([0, 1], u))
    assert e.value.status == -9
    with pytest.raises(Q.QuwarpError) as e:
        Q.DenseProgram(eng, FP32, 14, engine_kind=T, block=([3, 3], u))
    assert e.value.status == -1
    with pytest.raises(Q.QuwarpError) as e:
        Q.DenseProgram(eng, FP32, 14, engine_kind=T, nacc=3, block=([0, 1], u))
    assert e.value.status == -1


@pytest.mark.parametrize("mode,n,engine", [(FP32, 14, Q.DENSE_AUTO), (FP32, 20, T), (FP64, 12, Q.DENSE_AUTO),
                                           (FP32, 10, Q.DENSE_AUTO)])
def test_autotuned_fusion_width_and_engine(eng, mode, n, engine):
    # kmax = 0: the fusion width (and with DENSE_AUTO the engine) is chosen
    # by measured block-pass times; the program still matches the oracle
    rng = np.random.default_rng(900 + n)
    g = random_gate_list(rng, n, 120)
    psi = rounded(random_state(rng, n), mode)
    prog = Q.DenseProgram(eng, mode, n, gates=g, kmax=0, engine_kind=engine)
    cfg = prog.config()
    assert 2 <= cfg["kmax"] <= 5 and cfg["estimated_ms"] > 0
    if mode == FP64 or n < 12:
        assert cfg["engine"] == S                 # the tensor cores take FP32 states of >= 12 qubits
    if engine == T:
        assert cfg["engine"] == T
    got = run_prog(prog, psi, mode)
    want = orc.sv_apply(n, psi.copy(), g)
    tol = 1e-12 if mode == FP64 else 1e-5
    assert np.max(np.abs(got - want)) <= tol
    # by the same (cached) measurements, no fixed width is faster
    if engine == Q.DENSE_AUTO:
        for k in (2, 3, 4, 5):
            other = Q.DenseProgram(eng, mode, n, gates=g, kmax=k, engine_kind=Q.DENSE_AUTO)
            assert other.config()["kmax"] <= k
            assert other.config()["estimated_ms"] >= cfg["estimated_ms"] * (1 - 1e-9)
            other.close()
    prog.close()


@pytest.mark.parametrize("n,qubits", [(28, [5, 6, 7, 8, 9]), (28, [0, 1, 2, 3, 4]), (28, [27, 3, 14, 0, 22]),
                                      (30, [29, 1, 2, 3, 17])])
def test_block_at_full_size_sampled_groups(eng, n, qubits):
    # full size (28 qubits: 2 GiB FP32 state, 2^16 tiles; 30 qubits, the
    # statevector cap: 8 GiB): 512 sampled groups of 32 amplitudes checked
    # one by one against the oracle's operator on the group, and the norm kept
    g = torch.Generator(device="cuda").manual_seed(28)
    st = torch.randn(1 << n, dtype=torch.complex64, device="cuda", generator=g)
    st /= torch.linalg.vector_norm(st)
    before = st.cpu().numpy()
    rng = np.random.default_rng(sum(qubits))
    u = random_unitary(rng, 32)
    prog = Q.DenseProgram(eng, FP32, n, engine_kind=T, nacc=4, block=(qubits, u))
    prog.run(st.data_ptr())
    prog.check()
    after = st.cpu().numpy()
    assert abs(float(np.linalg.norm(after.astype(np.complex128))) - 1.0) <= 1e-5
    other = [q for q in range(n) if q not in qubits]
    pos = np.array([sum(((p >> j) & 1) << q for j, q in enumerate(qubits)) for p in range(32)], dtype=np.int64)
    for gidx in rng.integers(0, 1 << (n - 5), size=512):
        base = sum(((int(gidx) >> i) & 1) << q for i, q in enumerate(other))
        vin = before[base + pos].astype(np.complex128)
        want = orc.apply_matrix(5, vin, [0, 1, 2, 3, 4], u)
        got = after[base + pos].astype(np.complex128)
        assert np.max(np.abs(got - want)) <= 1e-5
        assert np.linalg.norm(got - want) <= 2e-6 * np.linalg.norm(want) + 1e-12
    prog.close()


def test_mixed_engine_program_uses_tensor_cores_only_for_large_blocks(eng):
    # a circuit whose fusion yields both 5-qubit blocks (a dense brick on
    # qubits 8-12) and lone one- and two-qubit blocks: with DENSE_AUTO the
    # small blocks run on the CUDA cores; the result matches the oracle
    n = 16
    rng = np.random.default_rng(77)
    ops = []
    for _ in range(6):
        for q in range(8, 12):
            ops.append((W.OP_RY, q, 0, float(rng.uniform(0, 6))))
            ops.append((W.OP_CNOT, q, q + 1))
    ops += [(W.OP_H, 0, 0), (W.OP_RX, 3, 0, 0.4), (W.OP_CZ, 3, 4)]
    g = W.gates_from_list(ops)
    psi = rounded(random_state(rng, n), FP32)
    prog = Q.DenseProgram(eng, FP32, n, gates=g, kmax=5, engine_kind=Q.DENSE_AUTO)
    got = run_prog(prog, psi, FP32)
    want = orc.sv_apply(n, psi.copy(), g)
    assert np.max(np.abs(got - want)) <= 1e-5
    assert prog.config()["engine"] in (Q.DENSE_AUTO, Q.DENSE_SIMT, Q.DENSE_TENSOR)
    prog.close()


def test_plan_evolves_a_deep_local_boundary_with_dense_blocks(eng):
    # a shared prefix of 40 layers confined to qubits 6-10 (one 5-qubit dense
    # block, but hundreds of gates for a pass kernel), then a short suffix
    tasks = W.deep_local_sweep(seed=5, n=20, layers=40, lo=6, n_tasks=6, n_terms=16)
    plan = Q.Plan(eng, Q.Workload(tasks), dense_boundaries=1)
    plan.run()
    ch = plan.cost_record()["dense_boundaries"]
    assert len(ch) == 1 and ch[0]["blocks"] >= 1
    print(ch)
    # one dense pass over the state against hundreds of gates in a pass kernel
    assert ch[0]["used"] and ch[0]["dense_ms"] < ch[0]["pass_kernels_ms"]
    assert ch[0]["engine"] in ("tensor", "mixed")
    for i in range(len(tasks)):
        ref = orc.run_task(tasks[i])
        e, _ = plan.energy(i)
        err = energy_error(e, ref["energy"], tasks[i].terms, tasks[i].n)
        print("dense boundary (%d blocks) task %d energy error %.2e" % (ch[0]["blocks"], i, err))
        assert err <= FP32_ENERGY_TOL, i
    plan.close()


@pytest.mark.parametrize("mode", [1, 2])
def test_dense_boundaries_keep_parity_on_the_vqe_sweep(eng, mode):
    # a 20-layer prefix is ~100 dense blocks: beyond the accuracy budget of
    # compensated FP32 (each 3xTF32 block perturbs the state at FP32 level),
    # so the boundary keeps the compensated pass kernels, even when forced
    tasks = W.vqe24_sweep(n=16, n_tasks=4, n_terms=20)
    plan = Q.Plan(eng, Q.Workload(tasks), dense_boundaries=mode)
    plan.run()
    ch = plan.cost_record()["dense_boundaries"]
    assert len(ch) == 1 and ch[0]["over_accuracy_budget"] and not ch[0]["used"]
    for i, t in enumerate(tasks):
        ref = orc.run_task(t)
        e, _ = plan.energy(i)
        err = energy_error(e, ref["energy"], t.terms, t.n)
        print("dense_boundaries %d task %d energy error %.2e" % (mode, i, err))
        assert err <= FP32_ENERGY_TOL, (i, err)
    plan.close()


@pytest.mark.parametrize("engine", [T, S, Q.DENSE_AUTO])
def test_empty_gate_list_leaves_the_state(eng, engine):
    rng = np.random.default_rng(3)
    psi = rounded(random_state(rng, 13), FP32)
    prog = Q.DenseProgram(eng, FP32, 13, gates=W.gates_from_list([]), kmax=0 if engine == Q.DENSE_AUTO else 5,
                          engine_kind=engine)
    assert prog.info()["blocks"] == 0
    got = run_prog(prog, psi, FP32)
    assert np.array_equal(got, psi)
    prog.close()

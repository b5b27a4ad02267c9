"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Tolerances (stated by the target): FP64 statevector max-abs amplitude error
<= 1e-12; FP32 statevector max-abs amplitude error <= 1e-5 and energy error
<= 1e-6 relative to max(|E_ref|, E_typ) (energy_tol.py); tableau outcomes
bit-exact.  The energy kernel alone is checked on FP32-representable states
against the oracle's energy of the same state, within 4e-7 of the same
scale.  Sampling: a shot may differ from the oracle only where its uniform
lies within 1e-5 of the CDF value at the oracle's outcome boundary."""
import math

import numpy as np
import pytest

from energy_tol import FP32_ENERGY_TOL, energy_error, energy_ok
from oracle import mlp_oracle as MO
from oracle import oracle as orc
from paper_2609_23664_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # the GPU suite is only meaningful on a GPU
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_23664_gb300 import quwarp as Q  # noqa: E402


@pytest.fixture(scope="module")
def eng():
    e = Q.Engine(0)
    yield e
    e.close()


ALL_OPS = [W.OP_H, W.OP_X, W.OP_Y, W.OP_Z, W.OP_S, W.OP_SDG, W.OP_T, W.OP_TDG, W.OP_RX, W.OP_RY,
           W.OP_RZ, W.OP_PHASE, W.OP_CNOT, W.OP_CZ, W.OP_SWAP, W.OP_CPHASE]


def rand_gates(rng, n, k, ops=ALL_OPS):
    g = []
    for _ in range(k):
        op = ops[int(rng.integers(0, len(ops)))]
        a = int(rng.integers(0, n))
        b = int(rng.integers(0, n - 1))
        b = b + 1 if b >= a else b
        g.append((op, a, b, float(rng.uniform(0, 2 * math.pi))))
    return W.gates_from_list(g)


def tdtype(mode):
    return torch.complex128 if mode == W.MODE_SV_FP64 else torch.complex64


TOL_AMP = {W.MODE_SV_FP64: 1e-12, W.MODE_SV_FP32: 1e-5}


@pytest.mark.parametrize("mode,n", [(W.MODE_SV_FP64, 5), (W.MODE_SV_FP64, 9), (W.MODE_SV_FP64, 13),
                                    (W.MODE_SV_FP64, 16), (W.MODE_SV_FP32, 5), (W.MODE_SV_FP32, 11),
                                    (W.MODE_SV_FP32, 14), (W.MODE_SV_FP32, 17),
                                    (W.MODE_SV_FP32, 19)])
def test_sv_apply_random_circuits(eng, mode, n):
    rng = np.random.default_rng(1000 + 10 * n + mode)
    g = rand_gates(rng, n, 300)
    st = torch.zeros(1 << n, dtype=tdtype(mode), device="cuda")
    Q.sv_apply_dev(eng, mode, n, st.data_ptr(), g, init=True)
    torch.cuda.synchronize()
    got = st.cpu().numpy().astype(np.complex128)
    ref = orc.sv_run(n, g)
    err = float(np.max(np.abs(got - ref)))
    assert err <= TOL_AMP[mode], err


@pytest.mark.parametrize("mode", [W.MODE_SV_FP64, W.MODE_SV_FP32])
def test_sv_apply_every_gate_every_position(eng, mode):
    n = 7
    rng = np.random.default_rng(55 + mode)
    for op in ALL_OPS:
        for a in range(n):
            for b in ([a] if op not in W.TWO_QUBIT_OPS else [q for q in range(n) if q != a]):
                psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
                psi0 /= np.linalg.norm(psi0)
                st = torch.tensor(psi0, dtype=tdtype(mode), device="cuda")
                g = W.gates_from_list([(op, a, b, 0.7)])
                Q.sv_apply_dev(eng, mode, n, st.data_ptr(), g)
                torch.cuda.synchronize()
                got = st.cpu().numpy().astype(np.complex128)
                start = psi0 if mode == W.MODE_SV_FP64 else psi0.astype(np.complex64).astype(np.complex128)
                ref = orc.sv_apply(n, start.copy(), g)
                assert np.max(np.abs(got - ref)) <= TOL_AMP[mode], (op, a, b)


# The energy kernel's own error on an FP32 state: FP32 products and +-1
# butterflies, accumulated in double-float then FP64.  Emulating its
# operation order on random 14-qubit states gives errors of 7e-8 rms, 2e-7
# max, relative to max(|E|, E_typ); 4e-7 leaves room while still seeing an
# error of 1e-6.
KERNEL_ENERGY_TOL = 4e-7


@pytest.mark.parametrize("mode,n,k", [(W.MODE_SV_FP64, 6, 60), (W.MODE_SV_FP64, 12, 60), (W.MODE_SV_FP32, 10, 60),
                                      (W.MODE_SV_FP32, 15, 60), (W.MODE_SV_FP32, 18, 60),
                                      (W.MODE_SV_FP32, 24, 200)])
def test_energy_dev(eng, mode, n, k):
    rng = np.random.default_rng(200 + n)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi *= 1.3 / np.linalg.norm(psi)
    if mode == W.MODE_SV_FP32:
        psi = psi.astype(np.complex64).astype(np.complex128)
    terms = W.random_pauli_hamiltonian(rng, n, k)
    terms[0]["xmask"] = 0  # include diagonal and identity-like terms
    terms[1]["xmask"] = 0
    terms[1]["zmask"] = 0
    st = torch.tensor(psi, dtype=tdtype(mode), device="cuda")
    e, nr = Q.sv_energy_dev(eng, mode, n, st.data_ptr(), terms)
    e_ref, n_ref, _ = orc.energy(n, psi, terms)
    assert abs(nr - n_ref) <= (1e-13 if mode == W.MODE_SV_FP64 else 1e-6) * n_ref
    if mode == W.MODE_SV_FP64:
        assert abs(e - e_ref) <= 1e-12 * max(1.0, abs(e_ref)), (e, e_ref)
    else:
        err = energy_error(e, e_ref, terms, n)
        print("n %d: energy kernel error %.2e of max(|E|, E_typ)" % (n, err))
        assert err <= KERNEL_ENERGY_TOL, (e, e_ref, err)


def sample_agrees(got, ref, psi, u):
    p = np.abs(psi) ** 2
    F = np.cumsum(p / p.sum())
    ok = got == ref
    near = np.abs(F[np.minimum(ref, len(F) - 1).astype(np.int64)] - u) < 1e-5
    near |= np.abs(F[np.maximum(ref.astype(np.int64) - 1, 0)] - u) < 1e-5
    return bool(np.all(ok | near)), int(np.count_nonzero(~ok))


@pytest.mark.parametrize("mode,n", [(W.MODE_SV_FP64, 5), (W.MODE_SV_FP64, 13), (W.MODE_SV_FP32, 12),
                                    (W.MODE_SV_FP32, 16)])
def test_sample_dev(eng, mode, n):
    rng = np.random.default_rng(300 + n)
    psi = orc.sv_run(n, rand_gates(rng, n, 120))
    if mode == W.MODE_SV_FP32:
        psi = psi.astype(np.complex64).astype(np.complex128)
    u = rng.random(3000)
    st = torch.tensor(psi, dtype=tdtype(mode), device="cuda")
    got = Q.sv_sample_dev(eng, mode, n, st.data_ptr(), u)
    ref = orc.sample(n, psi, u)
    ok, mism = sample_agrees(got, ref, psi, u)
    assert ok, mism


def test_sample_basis_state(eng):
    n = 14
    psi = orc.sv_run(n, W.basis_state_circuit(n, 12345))
    st = torch.tensor(psi, dtype=torch.complex64, device="cuda")
    got = Q.sv_sample_dev(eng, W.MODE_SV_FP32, n, st.data_ptr(), np.random.default_rng(1).random(500))
    assert np.all(got == 12345)


# ---- workload level (plan / execute / read back through the C ABI) -----------

def run_plan(eng, tasks, **opts):
    wl = Q.Workload(tasks)
    p = Q.Plan(eng, wl, **opts)
    p.run()
    return p, wl


def test_vqe12_fp64_full(eng):
    tasks = W.vqe12_sweep()
    for t in tasks[:3]:
        t.want_state = True
    p, wl = run_plan(eng, tasks)
    ex = p.explain()
    assert ex["artifacts"] == 1 and ex["tasks_reusing"] == len(tasks)
    for i, t in enumerate(tasks):
        ref = orc.run_task(t, want_state=i < 3)
        e, nr = p.energy(i)
        assert abs(e - ref["energy"]) <= 1e-12 * max(1, abs(ref["energy"])), (i, e, ref["energy"])
        assert abs(nr - 1.0) < 1e-12
        if i < 3:
            got = p.state(i, t.n, True)
            assert np.max(np.abs(got - ref["state"])) <= 1e-12


@pytest.mark.parametrize("reuse,batched,graph", [(1, 1, 1), (0, 0, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0)])
def test_vqe_fp32_small(eng, reuse, batched, graph):
    tasks = W.vqe24_sweep(n=16, n_tasks=24, n_terms=40)
    for t in tasks[:2]:
        t.want_state = True
    p, wl = run_plan(eng, tasks, reuse=reuse, batched=batched, use_graph=graph)
    ex = p.explain()
    assert ex["artifacts"] == (1 if reuse else 0)
    for i, t in enumerate(tasks):
        ref = orc.run_task(t, want_state=i < 2)
        e, nr = p.energy(i)
        err = energy_error(e, ref["energy"], t.terms, t.n)
        assert err <= FP32_ENERGY_TOL, (i, err)
        assert abs(nr - 1.0) < 1e-5
        if i < 2:
            got = p.state(i, t.n, False).astype(np.complex128)
            assert np.max(np.abs(got - ref["state"])) <= 1e-5


@pytest.mark.parametrize("mode,n", [(W.MODE_SV_FP32, 16), (W.MODE_SV_FP64, 15)])
def test_energy_fused_into_the_suffix_launch(eng, mode, n):
    # energy blocks as work items of the persistent launch: same results as
    # the separate energy launch and as the oracle
    tasks = W.vqe24_sweep(n=n, n_tasks=12, n_terms=60, mode=mode)
    p, wl = run_plan(eng, tasks, fuse_energy=1, tile_qubits=13)
    assert p.cost_record()["energy_fused"] is True
    q, wl2 = run_plan(eng, tasks, tile_qubits=13)
    assert q.cost_record()["energy_fused"] is False
    fp64 = mode == W.MODE_SV_FP64
    for i, t in enumerate(tasks):
        ref = orc.run_task(t)
        e, nr = p.energy(i)
        e2, nr2 = q.energy(i)
        c1 = float(np.sum(np.abs(t.terms["coef"])))
        assert energy_ok(e, ref["energy"], t.terms, t.n, fp64), (i, e, ref["energy"])
        # the two launches differ only in the order of the block sums
        assert abs(e - e2) <= (1e-13 if fp64 else 1e-6) * c1, (i, e, e2)
        assert abs(nr - nr2) <= (1e-13 if fp64 else 1e-6)


def test_noisy_small(eng):
    tasks = W.noisy22_trajectories(n=14, n_gates=200, n_traj=96, p=0.01, shots=50)
    p, wl = run_plan(eng, tasks)
    ex = p.explain()
    assert ex["tasks_reusing"] > 0
    bad = 0
    for i, t in enumerate(tasks):
        ref = orc.run_task(t, want_state=True)
        got = p.samples(i)
        ok, m = sample_agrees(got, ref["samples"], ref["state"], t.uniforms)
        bad += 0 if ok else 1
    assert bad == 0


def test_noisy_full_trajectory_count_at_14_qubits(eng):
    # the noisy family's full shape (400 gates, 1024 trajectories with Pauli
    # noise at p = 1e-3, 100 shots each) at 14 qubits: every trajectory's
    # samples against the oracle's rerun from |0...0>
    tasks = W.noisy22_trajectories(n=14)
    assert len(tasks) == 1024 and tasks[0].shots == 100
    p, wl = run_plan(eng, tasks)
    ex = p.explain()
    assert ex["tasks_reusing"] > 0 and ex["artifacts"] > 1
    bad = []
    for i, t in enumerate(tasks):
        ref = orc.run_task(t, want_state=True)
        ok, m = sample_agrees(p.samples(i), ref["samples"], ref["state"], t.uniforms)
        if not ok:
            bad.append((i, m))
    assert not bad, bad[:10]


def test_qec_small_bit_exact(eng):
    tasks = W.qec_surface_code_tasks(d=5, shared_rounds=8, task_rounds=3, n_tasks=48, p=0.02)
    p, wl = run_plan(eng, tasks)
    for i, t in enumerate(tasks):
        ref = orc.tab_run(t.n, t.gates)
        got = p.syndrome(i)
        assert np.array_equal(got, ref), i


@pytest.mark.parametrize("frames,graph", [(1, 1), (0, 1), (1, 0)])
def test_qec_frames_and_tableau_agree_bit_exact(eng, frames, graph):
    # Pauli frames over the shared 3-round reference vs every task on its
    # own tableau, with and without graph capture: identical syndromes,
    # equal to the oracle's
    tasks = W.qec_surface_code_tasks(d=5, shared_rounds=6, task_rounds=3, n_tasks=80, p=0.02)
    p, wl = run_plan(eng, tasks, pauli_frames=frames, use_graph=graph)
    ex = p.explain()
    assert len(ex["pauli_frames"]) == frames
    if frames:
        assert ex["pauli_frames"][0]["tasks"] == 80 and ex["artifacts"] == 1
    for i, t in enumerate(tasks):
        assert np.array_equal(p.syndrome(i), orc.tab_run(t.n, t.gates)), (frames, i)


def test_pauli_frames_fall_back_when_a_reference_outcome_is_random(eng):
    # the shared reference measures a qubit in superposition: its outcome is
    # random, so frames do not apply; the per-task tableau launch (gated on
    # the device by the reference run) must produce the oracle's outcomes
    rng = np.random.default_rng(77)
    n = 7
    pre = W.gates_from_list([(W.OP_H, 0, 0), (W.OP_CNOT, 0, 1), (W.OP_CNOT, 1, 2), (W.OP_H, 5, 0),
                             (W.OP_MEASURE, 2, 0, 1.0), (W.OP_S, 1, 0), (W.OP_CZ, 1, 3)])
    suf = W.gates_from_list([(W.OP_H, 4, 0), (W.OP_MEASURE, 4, 0, 1.0), (W.OP_CNOT, 0, 6),
                             (W.OP_MEASURE, 6, 0, 0.0), (W.OP_H, 3, 0), (W.OP_MEASURE, 3, 0, 1.0),
                             (W.OP_RESET, 4, 0, 0.0), (W.OP_MEASURE, 0, 0, 0.0)])
    tasks = []
    for i in range(40):
        errs = [(int(rng.choice([W.OP_X, W.OP_Y, W.OP_Z])), int(rng.integers(0, n)), 0)
                for _ in range(int(rng.integers(0, 3)))]
        spans = [pre] + ([W.gates_from_list(errs)] if errs else []) + [suf]
        tasks.append(W.Task(mode=W.MODE_TABLEAU, n=n, spans=spans))
    p, wl = run_plan(eng, tasks, min_prefix_gates=1)
    ex = p.explain()
    assert ex["pauli_frames"] and ex["pauli_frames"][0]["tasks"] >= 2
    for i, t in enumerate(tasks):
        assert np.array_equal(p.syndrome(i), orc.tab_run(t.n, t.gates)), i


def phase_aligned_error(got, ref):
    # exported states carry a canonical global phase: align it, then compare
    k = int(np.argmax(np.abs(ref)))
    ph = ref[k] / got[k]
    return float(np.max(np.abs(got * ph / abs(ph) - ref)))


@pytest.mark.parametrize("mode,n", [(W.MODE_SV_FP64, 16), (W.MODE_SV_FP32, 18)])
def test_tableau_handoff_to_statevector(eng, mode, n):
    # deep Clifford prefix on the tableau, exported once (Table II STAB -> SV),
    # non-Clifford suffixes on the statevector: energies and states vs oracle
    tasks = W.handoff_family(n=n, clifford_depth=200, n_tasks=5, suffix_gates=40, mode=mode)
    for t in tasks[:2]:
        t.want_state = True
    p, wl = run_plan(eng, tasks)
    d = p.explain()["decisions"][0]
    alt = {a["plan"]: a for a in d["alternatives"]}
    assert alt["CROSS_BACKEND_HANDOFF"]["est_ns"] < alt["SAME_FAMILY_REUSE"]["est_ns"]
    assert d["artifact"]["kind"] == "TABLEAU_BOUNDARY_STATE" and d["artifact"]["exported_to"]
    fp64 = mode == W.MODE_SV_FP64
    for i, t in enumerate(tasks):
        ref = orc.run_task(t, want_state=i < 2)
        e, nr = p.energy(i)
        assert energy_ok(e, ref["energy"], t.terms, t.n, fp64), i
        assert abs(nr - 1.0) < (1e-12 if fp64 else 1e-5)
        if i < 2:
            got = p.state(i, n, fp64).astype(np.complex128)
            assert phase_aligned_error(got, ref["state"]) <= (1e-12 if fp64 else 1e-5)
    # the same workload without the handoff (statevector prefix) agrees
    q, wl2 = run_plan(eng, tasks, handoff=0)
    assert q.explain()["decisions"][0]["artifact"]["kind"] == "STATEVECTOR_BOUNDARY_STATE"
    for i in range(len(tasks)):
        assert abs(p.energy(i)[0] - q.energy(i)[0]) <= (1e-12 if fp64 else 1e-5)


def test_tableau_boundary_serves_stabilizer_and_statevector_tasks(eng):
    # a Clifford prefix shared by tableau tasks (majority) and statevector
    # tasks: one tableau boundary, exported for the statevector consumers
    rng = np.random.default_rng(5)
    n = 10
    pre = W.random_clifford_layers(rng, n, 30)
    terms = W.random_pauli_hamiltonian(rng, n, 20)
    tasks = []
    for i in range(6):
        suf = W.gates_from_list([(W.OP_H, i, 0), (W.OP_CNOT, i, (i + 1) % n),
                                 (W.OP_MEASURE, i, 0, float(i & 1)), (W.OP_MEASURE, (i + 3) % n, 0, 0.0)])
        tasks.append(W.Task(mode=W.MODE_TABLEAU, n=n, spans=[pre, suf]))
    for i in range(3):
        suf = W.random_circuit(rng, n, 25)
        tasks.append(W.Task(mode=W.MODE_SV_FP64, n=n, spans=[pre, suf], terms=terms))
    p, wl = run_plan(eng, tasks)
    arts = [d["artifact"] for d in p.explain()["decisions"] if d["artifact"]]
    assert any(a["kind"] == "TABLEAU_BOUNDARY_STATE" and "GPU_SV_FP64" in a["exported_to"] for a in arts)
    for i, t in enumerate(tasks):
        if t.mode == W.MODE_TABLEAU:
            assert np.array_equal(p.syndrome(i), orc.tab_run(t.n, t.gates)), i
        else:
            ref = orc.run_task(t)
            assert abs(p.energy(i)[0] - ref["energy"]) <= 1e-12 * max(1.0, abs(ref["energy"])), i


def test_qec_replay_bit_exact(eng):
    tasks = W.qec_surface_code_tasks(d=3, shared_rounds=4, task_rounds=2, n_tasks=16, p=0.05)
    p, wl = run_plan(eng, tasks, reuse=0)
    for i, t in enumerate(tasks):
        assert np.array_equal(p.syndrome(i), orc.tab_run(t.n, t.gates)), i


CLIFF = [W.OP_H, W.OP_S, W.OP_SDG, W.OP_X, W.OP_Y, W.OP_Z, W.OP_CNOT, W.OP_CZ, W.OP_SWAP]


def rand_clifford(rng, n, k, p_meas):
    g = []
    for _ in range(k):
        a = int(rng.integers(0, n))
        r = rng.random()
        if r < p_meas:
            g.append((W.OP_MEASURE if rng.random() < 0.7 else W.OP_RESET, a, 0,
                      float(rng.integers(0, 2))))
            continue
        op = CLIFF[int(rng.integers(0, len(CLIFF)))]
        b = int(rng.integers(0, n - 1))
        b = b + 1 if b >= a else b
        g.append((op, a, b))
    return W.gates_from_list(g)


@pytest.mark.parametrize("n", [2, 5, 17, 64, 65, 130])
def test_tableau_random_clifford_with_measurements(eng, n):
    rng = np.random.default_rng(400 + n)
    prefix = rand_clifford(rng, n, 6 * n, 0.1)
    tasks = [W.Task(mode=W.MODE_TABLEAU, n=n, spans=[prefix, rand_clifford(rng, n, 4 * n, 0.15)])
             for _ in range(6)]
    p, wl = run_plan(eng, tasks)
    for i, t in enumerate(tasks):
        assert np.array_equal(p.syndrome(i), orc.tab_run(n, t.gates)), i


def test_legality_refusal_keeps_exactness_and_disabled_guard_does_not(eng):
    rng = np.random.default_rng(9)
    n = 10
    prefix = rand_gates(rng, n, 80)
    ham = W.random_pauli_hamiltonian(rng, n, 10)
    tasks = []
    for i in range(6):
        mode = W.MODE_SV_FP64 if i == 5 else W.MODE_SV_FP32
        tasks.append(W.Task(mode=mode, n=n, spans=[prefix, rand_gates(rng, n, 10)], terms=ham,
                            want_state=(i == 5)))
    ref = orc.run_task(tasks[5], want_state=True)
    # FP32 boundary (prefix in the majority's precision): the FP64 task is refused
    p, wl = run_plan(eng, tasks)
    ex = p.explain()
    refs = [r for d in ex["decisions"] for r in d["refusals"]]
    assert len(refs) == 1 and refs[0]["reason"] == "FORBIDDEN_CONVERSION" and refs[0]["task"] == 5
    assert refs[0]["source_backend"] == "GPU_SV_FP32" and refs[0]["target_backend"] == "GPU_SV_FP64"
    assert np.max(np.abs(p.state(5, n, True) - ref["state"])) <= 1e-12
    p2, wl2 = run_plan(eng, tasks, legality=0)
    err = np.max(np.abs(p2.state(5, n, True) - ref["state"]))
    assert err > 1e-9   # the unsafe continuation is measurably not exact
    # FP64 boundary rounded once for the FP32 tasks: the FP64 task reuses it exactly
    p3, wl3 = run_plan(eng, tasks, prefix_fp64=1)
    assert [r for d in p3.explain()["decisions"] for r in d["refusals"]] == []
    assert np.max(np.abs(p3.state(5, n, True) - ref["state"])) <= 1e-12


def test_mlp_forward_and_grad_vs_oracle(eng):
    rng = np.random.default_rng(17)
    B = 333
    params = rng.normal(scale=0.25, size=Q.MLP_PARAMS).astype(np.float32)
    x = rng.normal(size=(B, Q.MLP_IN)).astype(np.float32)
    t = rng.normal(size=B).astype(np.float32)
    dp = torch.tensor(params, device="cuda")
    dx = torch.tensor(x, device="cuda")
    dt = torch.tensor(t, device="cuda")
    dy = torch.zeros(B, device="cuda")
    Q.mlp_forward_dev(dp.data_ptr(), dx.data_ptr(), dy.data_ptr(), B)
    dl = torch.zeros(1, device="cuda")
    dg = torch.zeros(Q.MLP_PARAMS, device="cuda")
    Q.mlp_loss_grad_dev(dp.data_ptr(), dx.data_ptr(), dt.data_ptr(), B, dl.data_ptr(), dg.data_ptr())
    torch.cuda.synchronize()
    y_ref, _ = MO.forward(params, x)
    loss_ref, g_ref = MO.loss_grad(params, x, t)
    assert np.max(np.abs(dy.cpu().numpy() - y_ref)) <= 1e-4 * max(1, np.max(np.abs(y_ref)))
    assert abs(dl.item() - loss_ref) <= 1e-4 * loss_ref
    g = dg.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * max(1e-3, np.max(np.abs(g_ref)))


def test_mlp_adam_step(eng):
    n = 1000
    rng = np.random.default_rng(2)
    p = rng.normal(size=n).astype(np.float32)
    g = rng.normal(size=n).astype(np.float32)
    dp, dg = torch.tensor(p, device="cuda"), torch.tensor(g, device="cuda")
    dm, dv = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    Q.mlp_adam_dev(dp.data_ptr(), dg.data_ptr(), dm.data_ptr(), dv.data_ptr(), n, 1, 1e-3)
    torch.cuda.synchronize()
    m = 0.1 * g.astype(np.float64)
    v = 0.001 * g.astype(np.float64) ** 2
    ref = p - 1e-3 * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    assert np.max(np.abs(dp.cpu().numpy() - ref)) < 1e-6

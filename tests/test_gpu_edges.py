"""Edge cases of the planned execution on the GPU: empty and gate-free
workloads, registers below the 5-qubit stage width, identical tasks (empty
suffixes), ragged mixed workloads, and the largest registers of both
engines checked against closed forms."""
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


@pytest.fixture(scope="module")
def eng():
    e = Q.Engine(0)
    yield e
    e.close()


def run(eng, tasks, **opts):
    wl = Q.Workload(tasks)
    p = Q.Plan(eng, wl, **opts)
    p.run()
    return p, wl


def tol(mode, ref):
    return 1e-12 * max(1.0, abs(ref)) if mode == W.MODE_SV_FP64 else 2e-6 * max(1.0, abs(ref))


def term(coef, xm, zm):
    t = np.zeros(1, dtype=W.TERM_DTYPE)
    t[0]["coef"], t[0]["xmask"], t[0]["zmask"] = coef, xm, zm
    return t


def test_empty_workload(eng):
    p, wl = run(eng, [])
    ex = p.explain()
    assert ex["tasks"] == 0 and ex["artifacts"] == 0


@pytest.mark.parametrize("mode", [W.MODE_SV_FP64, W.MODE_SV_FP32])
def test_gate_free_tasks_measure_the_zero_state(eng, mode):
    rng = np.random.default_rng(3)
    tasks = [W.Task(mode=mode, n=n, spans=[], terms=W.random_pauli_hamiltonian(rng, n, 12),
                    shots=5, uniforms=rng.random(5)) for n in (3, 9)]
    p, wl = run(eng, tasks)
    for i, t in enumerate(tasks):
        # <0|P|0> = c for Z-only strings, 0 otherwise
        closed = float(sum(c for c, x in zip(t.terms["coef"], t.terms["xmask"]) if x == 0))
        assert abs(p.energy(i)[0] - closed) <= tol(mode, closed)
        assert np.all(p.samples(i) == 0)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_registers_below_the_stage_width(eng, n):
    rng = np.random.default_rng(40 + n)
    pre = W.random_circuit(rng, n, 12) if n > 1 else W.gates_from_list([(W.OP_H, 0, 0), (W.OP_RZ, 0, 0, 0.7)])
    terms = W.random_pauli_hamiltonian(rng, n, 6)
    tasks = []
    for k in range(4):
        suf = W.gates_from_list([(W.OP_RY, int(rng.integers(0, n)), 0, float(rng.uniform(0, 6)))])
        tasks.append(W.Task(mode=W.MODE_SV_FP64, n=n, spans=[pre, suf], terms=terms, shots=20,
                            uniforms=rng.random(20), want_state=True))
    p, wl = run(eng, tasks)
    for i, t in enumerate(tasks):
        ref = orc.run_task(t, want_state=True)
        assert abs(p.energy(i)[0] - ref["energy"]) <= tol(t.mode, ref["energy"])
        assert np.max(np.abs(p.state(i, n, True) - ref["state"])) <= 1e-12
        assert np.array_equal(p.samples(i), ref["samples"])


def test_identical_tasks_read_the_boundary(eng):
    rng = np.random.default_rng(8)
    g = W.random_circuit(rng, 14, 120)
    terms = W.random_pauli_hamiltonian(rng, 14, 20)
    tasks = [W.Task(mode=W.MODE_SV_FP32, n=14, spans=[g], terms=terms) for _ in range(5)]
    p, wl = run(eng, tasks)
    ex = p.explain()
    assert ex["artifacts"] == 1 and ex["tasks_reusing"] == 5
    ref = orc.run_task(tasks[0])
    for i in range(5):
        assert energy_error(p.energy(i)[0], ref["energy"], terms, 14) <= FP32_ENERGY_TOL


def test_ragged_mixed_workload(eng):
    # modes, register sizes, group sizes 1..4 and suffix lengths all mixed
    rng = np.random.default_rng(12)
    tasks = []
    for mode, n, group in ((W.MODE_SV_FP64, 7, 3), (W.MODE_SV_FP32, 13, 4), (W.MODE_SV_FP32, 6, 1),
                           (W.MODE_TABLEAU, 20, 4), (W.MODE_SV_FP64, 11, 2)):
        if mode == W.MODE_TABLEAU:
            pre = W.random_clifford_layers(rng, n, 6)
        else:
            pre = W.random_circuit(rng, n, int(rng.integers(20, 80)))
        terms = W.random_pauli_hamiltonian(rng, n, 10) if mode != W.MODE_TABLEAU else None
        for _ in range(group):
            if mode == W.MODE_TABLEAU:
                q = int(rng.integers(0, n))
                suf = W.gates_from_list([(W.OP_H, q, 0), (W.OP_MEASURE, q, 0, float(rng.integers(0, 2))),
                                         (W.OP_MEASURE, (q + 1) % n, 0, 0.0)])
            else:
                suf = W.random_circuit(rng, n, int(rng.integers(0, 15)))
            tasks.append(W.Task(mode=mode, n=n, spans=[pre, suf], terms=terms))
    order = rng.permutation(len(tasks))
    tasks = [tasks[i] for i in order]
    p, wl = run(eng, tasks)
    for i, t in enumerate(tasks):
        if t.mode == W.MODE_TABLEAU:
            assert np.array_equal(p.syndrome(i), orc.tab_run(t.n, t.gates)), i
        else:
            ref = orc.run_task(t)
            if t.mode == W.MODE_SV_FP64:
                assert abs(p.energy(i)[0] - ref["energy"]) <= tol(t.mode, ref["energy"]), i
            else:
                assert energy_error(p.energy(i)[0], ref["energy"], t.terms, t.n) <= FP32_ENERGY_TOL, i


def test_largest_statevector_ghz_closed_form(eng):
    # 30 qubits (the statevector cap), FP32: GHZ prefix shared by two tasks
    n = 30
    full = (1 << n) - 1
    terms = np.concatenate([term(1.0, full, 0), term(0.5, 0, (1 << 0) | (1 << 29)), term(0.25, 0, 1 << 7)])
    pre = W.ghz_circuit(n)
    tasks = [W.Task(mode=W.MODE_SV_FP32, n=n, spans=[pre], terms=terms),
             W.Task(mode=W.MODE_SV_FP32, n=n, spans=[pre, W.gates_from_list([(W.OP_X, 0, 0)])], terms=terms)]
    p, wl = run(eng, tasks)
    # GHZ: <X^n> = 1, <Z0 Z29> = 1, <Z7> = 0; X0 GHZ flips <Z0 Z29>
    assert abs(p.energy(0)[0] - 1.5) <= 1e-5
    assert abs(p.energy(1)[0] - 0.5) <= 1e-5
    assert abs(p.energy(0)[1] - 1.0) <= 1e-5


def test_largest_tableau_ghz_and_noiseless_surface_code(eng):
    # 640 qubits (the tableau cap): GHZ then Z measurements all agree
    n = 640
    g = W.gates_from_list([(W.OP_H, 0, 0)] + [(W.OP_CNOT, q, q + 1) for q in range(n - 1)] +
                          [(W.OP_MEASURE, q, 0, 1.0) for q in range(n)])
    tasks = [W.Task(mode=W.MODE_TABLEAU, n=n, spans=[g]) for _ in range(2)]
    p, wl = run(eng, tasks)
    for i in range(2):
        out = p.syndrome(i)
        assert len(out) == n and np.all(out == out[0])
    # d = 17 surface code (577 qubits), noiseless: Z syndromes are 0 from the
    # first round, X syndromes repeat from the second (no detection events)
    tasks = W.qec_surface_code_tasks(d=17, shared_rounds=2, task_rounds=2, n_tasks=3, p=0.0)
    p, wl = run(eng, tasks)
    code = W.rotated_surface_code(17)
    anc = sorted(code.sched.keys())
    zpos = [k for k, a in enumerate(anc) if a not in code.x_anc]
    xpos = [k for k, a in enumerate(anc) if a in code.x_anc]
    for i in range(3):
        s = p.syndrome(i).reshape(4, len(anc))
        assert np.all(s[:, zpos] == 0)
        assert np.array_equal(s[1:, xpos], np.repeat(s[:1, xpos], 3, axis=0))


def test_l2_read_probe_exceeds_hbm_bandwidth(eng):
    # the energy step's L2 read bandwidth (hashed 64 KB blocks of an
    # L2-resident buffer) must come out above the HBM copy bandwidth the
    # engine measured at start-up
    l2 = eng.probe_l2()
    hbm = eng.info()["hbm_gbs"]
    assert np.isfinite(l2) and l2 > hbm, (l2, hbm)


def test_task_budget_is_shared_by_register_sizes():
    # prefix-free tasks of five register sizes under a 256 MB task budget:
    # the groups' task pools share the budget (at least one buffer each),
    # so the plan's device memory stays near 256 MB instead of the ~1 GB
    # that one budget per group would take
    budget = 256 << 20
    e = Q.Engine(0, task_budget_bytes=budget)
    rng = np.random.default_rng(77)
    tasks = []
    for n in (20, 21, 22, 23, 24):
        for _ in range(8):
            tasks.append(W.Task(mode=W.MODE_SV_FP32, n=n, spans=[W.random_circuit(rng, n, 30)],
                                terms=W.random_pauli_hamiltonian(rng, n, 6)))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    wl = Q.Workload(tasks)
    p = Q.Plan(e, wl, reuse=0)
    p.run()
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    assert used < budget + (160 << 20), used
    for i in (0, 8):  # one task of each of the two smallest sizes
        ref = orc.run_task(tasks[i])
        assert energy_error(p.energy(i)[0], ref["energy"], tasks[i].terms, tasks[i].n) <= FP32_ENERGY_TOL
    p.close()
    wl.close()
    e.close()

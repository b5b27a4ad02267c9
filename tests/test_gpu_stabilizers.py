"""Final stabilizer tableaus, not only outcomes: the engine keeps the inverse
tableau (Heisenberg form) and the oracle the textbook forward tableau, so
their rows differ, but both describe one stabilizer group.  Each side's
generators are brought to a canonical form that depends only on the group
(reduced row echelon form over the columns x_0..x_{n-1}, z_0..z_{n-1},
multiplying generators as Paulis with their phases; the group's elements
commute, so the order of a product cannot change its phase) and the two
forms, signs included, must be equal bit for bit."""
import numpy as np
import pytest

from oracle import oracle as orc
from stab_canonical import canonical
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


def oracle_group(t):
    _, (x, z, r) = orc.tab_run(t.n, t.gates, want_tableau=True)
    n = t.n
    return canonical(x[n:], z[n:], r[n:])


def check(plan, tasks):
    for i, t in enumerate(tasks):
        got = canonical(*plan.stabilizers(i, t.n))
        want = oracle_group(t)
        for a, b, what in zip(got, want, ("x", "z", "sign")):
            assert np.array_equal(a, b), (i, what)


def rand_clifford_measured(rng, n, k):
    ops = [W.OP_H, W.OP_S, W.OP_SDG, W.OP_X, W.OP_Y, W.OP_Z, W.OP_CNOT, W.OP_CZ, W.OP_SWAP]
    g = []
    for _ in range(k):
        r = rng.random()
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        if r < 0.08:
            g.append((W.OP_MEASURE, a, 0, float(rng.integers(0, 2))))
        elif r < 0.12:
            g.append((W.OP_RESET, a, 0, float(rng.integers(0, 2))))
        else:
            g.append((ops[int(rng.integers(0, len(ops)))], a, b, 0.0))
    return W.gates_from_list(g)


@pytest.mark.parametrize("d", [3, 5])
def test_surface_code_final_tableaus(eng, d):
    tasks = W.qec_surface_code_tasks(d=d, shared_rounds=6, task_rounds=3, n_tasks=24, p=0.05)
    for t in tasks:
        t.want_state = True
    p = Q.Plan(eng, Q.Workload(tasks))
    p.run()
    assert p.explain()["pauli_frames"] == []   # kept tableaus run on their own
    check(p, tasks)
    for i, t in enumerate(tasks):            # outcomes still equal
        assert np.array_equal(p.syndrome(i), orc.tab_run(t.n, t.gates)), i
    p.close()


@pytest.mark.parametrize("n", [6, 17, 40, 64, 65, 130])
def test_random_measured_clifford_final_tableaus(eng, n):
    # a shared prefix (one boundary) and per-task suffixes with random and
    # deterministic measurements and resets, at row widths of 1-3 words
    rng = np.random.default_rng(900 + n)
    pre = rand_clifford_measured(rng, n, 12 * n)
    tasks = [W.Task(mode=W.MODE_TABLEAU, n=n, spans=[pre, rand_clifford_measured(rng, n, 4 * n)],
                    want_state=True) for _ in range(6)]
    p = Q.Plan(eng, Q.Workload(tasks), min_prefix_gates=1)
    p.run()
    check(p, tasks)
    p.close()


def test_d15_final_tableaus(eng):
    # the full-size code (449 qubits, 8 words per row), two tasks of the
    # bench's workload: 100 shared rounds, 5 task rounds with errors
    tasks = W.qec_surface_code_tasks(n_tasks=2)
    for t in tasks:
        t.want_state = True
    p = Q.Plan(eng, Q.Workload(tasks))
    p.run()
    check(p, tasks)
    p.close()


def test_stabilizers_need_kept_state(eng):
    tasks = W.qec_surface_code_tasks(d=3, shared_rounds=2, task_rounds=1, n_tasks=2, p=0.05)
    p = Q.Plan(eng, Q.Workload(tasks))
    p.run()
    with pytest.raises(Q.QuwarpError) as ei:
        p.stabilizers(0, tasks[0].n)
    assert ei.value.status == -8  # QW_ERR_NOT_FOUND
    p.close()

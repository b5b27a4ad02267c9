"""Tableau kernel at every row width: registers whose tableau rows hold 1, 2,
4, 8 (power-of-two: swizzled rows, one thread per row product) and 3, 5, 10
(other: 8 lanes per product) 64-bit words, through shared prefixes with
random measurement outcomes and per-task Clifford suffixes with Pauli
errors, bit-exact against the oracle's Aaronson-Gottesman tableau; the
Pauli-frame path and the per-task tableau path both."""
import numpy as np
import pytest

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


def workload(n, seed):
    rng = np.random.default_rng(seed)
    pre = W.random_clifford_layers(rng, n, 3)
    # measurements in the prefix: random outcomes (carried bits) on fresh superpositions
    meas = [(W.OP_MEASURE, int(q), 0, float(rng.integers(0, 2))) for q in rng.choice(n, 6, replace=False)]
    pre = np.concatenate([pre, W.gates_from_list(meas), W.random_clifford_layers(rng, n, 2)])
    tail = W.random_clifford_layers(rng, n, 1)
    tasks = []
    for _ in range(5):
        err = [(int(rng.choice([W.OP_X, W.OP_Y, W.OP_Z])), int(rng.integers(0, n)), 0) for _ in range(2)]
        qs = rng.choice(n, 4, replace=False)
        m = [(W.OP_MEASURE, int(q), 0, float(rng.integers(0, 2))) for q in qs]
        m.append((W.OP_RESET, int(qs[0]), 0, float(rng.integers(0, 2))))
        tasks.append(W.Task(mode=W.MODE_TABLEAU, n=n,
                            spans=[pre, W.gates_from_list(err), tail, W.gates_from_list(m)]))
    return tasks


@pytest.mark.parametrize("n", [40, 100, 150, 200, 300, 449, 600])   # words per half row: 1, 2, 3, 4, 5, 8, 10
@pytest.mark.parametrize("frames", [1, 0])
def test_every_row_width_bit_exact(eng, n, frames):
    tasks = workload(n, 1000 + n)
    plan = Q.Plan(eng, Q.Workload(tasks), pauli_frames=frames)
    plan.run()
    for i, t in enumerate(tasks):
        assert np.array_equal(plan.syndrome(i), orc.tab_run(t.n, t.gates)), (n, i)
    plan.close()

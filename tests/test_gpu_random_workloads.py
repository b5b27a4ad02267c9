"""Randomized workloads through the whole planned path on the GPU: random
trie shapes (groups sharing prefixes, sub-groups sharing mid-segments,
loners), random modes and register sizes, random gate mixes, Pauli errors on
stabilizer tasks and Clifford prefixes on statevector tasks, under several
plan options.  Every task is compared with the oracle.  Registers of 2-14
qubits fit one tile; a second set draws 15-20 qubits, so that passes span
several tiles (tile maps across passes, outside-control CNOTs, multi-pass
suffixes and boundaries)."""
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



def sv_gates(rng, n, k, clifford=False):
    if clifford:
        return W.random_clifford_layers(rng, n, max(1, k // n))
    return W.random_circuit(rng, n, k)


def random_workload(seed, n_sv=(2, 15)):
    rng = np.random.default_rng(seed)
    tasks = []
    for _ in range(int(rng.integers(3, 7))):                 # families
        mode = int(rng.choice([W.MODE_SV_FP64, W.MODE_SV_FP32, W.MODE_TABLEAU]))
        n = int(rng.integers(*n_sv)) if mode != W.MODE_TABLEAU else int(rng.integers(3, 40))
        if mode == W.MODE_TABLEAU:
            pre = W.random_clifford_layers(rng, n, int(rng.integers(1, 6)))
        else:
            pre = sv_gates(rng, n, int(rng.integers(5, 60)), clifford=rng.random() < 0.3)
        terms = W.random_pauli_hamiltonian(rng, n, int(rng.integers(1, 12))) if mode != W.MODE_TABLEAU else None
        for _ in range(int(rng.integers(1, 4))):             # sub-groups sharing a mid-segment
            mid = (W.random_clifford_layers(rng, n, 1) if mode == W.MODE_TABLEAU
                   else sv_gates(rng, n, int(rng.integers(0, 20))))
            # stabilizer sub-groups share their tail (tasks differ by Pauli
            # errors only: Pauli frames) unless the tail is redrawn per task
            q = int(rng.integers(0, n))
            per_task_tail = rng.random() < 0.3
            bits = [float(rng.integers(0, 2)) for _ in range(2)]
            for _ in range(int(rng.integers(1, 5))):         # tasks
                if mode == W.MODE_TABLEAU:
                    err = [(int(rng.choice([W.OP_X, W.OP_Y, W.OP_Z])), int(rng.integers(0, n)), 0)
                           for _ in range(int(rng.integers(0, 3)))]
                    if per_task_tail:
                        q = int(rng.integers(0, n))
                    tail = [(W.OP_CNOT, q, (q + 1) % n), (W.OP_H, (q + 2) % n, 0),
                            (W.OP_MEASURE, q, 0, bits[0]), (W.OP_MEASURE, (q + 2) % n, 0, bits[1])]
                    spans = [pre, mid] + ([W.gates_from_list(err)] if err else []) + [W.gates_from_list(tail)]
                    tasks.append(W.Task(mode=mode, n=n, spans=spans))
                else:
                    suf = sv_gates(rng, n, int(rng.integers(0, 12)))
                    shots = int(rng.integers(0, 6))
                    tasks.append(W.Task(mode=mode, n=n, spans=[pre, mid, suf], terms=terms, shots=shots,
                                        uniforms=rng.random(shots) if shots else None))
    order = rng.permutation(len(tasks))
    return [tasks[i] for i in order]


def check(p, tasks):
    for i, t in enumerate(tasks):
        if t.mode == W.MODE_TABLEAU:
            assert np.array_equal(p.syndrome(i), orc.tab_run(t.n, t.gates)), i
            continue
        ref = orc.run_task(t, want_state=t.shots > 0)
        e = p.energy(i)[0]
        if t.mode == W.MODE_SV_FP64:
            assert abs(e - ref["energy"]) <= 1e-11 * max(1.0, float(np.sum(np.abs(t.terms["coef"])))), i
        else:
            assert energy_error(e, ref["energy"], t.terms, t.n) <= FP32_ENERGY_TOL, i
        if t.shots:
            got = p.samples(i)
            pr = np.abs(ref["state"]) ** 2
            F = np.cumsum(pr / pr.sum())
            r = ref["samples"].astype(np.int64)
            tol = 1e-12 if t.mode == W.MODE_SV_FP64 else 1e-5
            near = (np.abs(F[np.minimum(r, len(F) - 1)] - t.uniforms) < tol) | \
                   (np.abs(F[np.maximum(r - 1, 0)] - t.uniforms) < tol)
            assert np.all((got == ref["samples"]) | near), i


@pytest.fixture(scope="module")
def eng():
    e = Q.Engine(0)
    yield e
    e.close()


@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("opts", [dict(), dict(delta_frac=0.0, min_group=2), dict(batched=0),
                                  dict(pauli_frames=0, handoff=0, prefix_fp64=1, use_graph=0),
                                  dict(delta_frac=0.0, dense_boundaries=2)])
def test_random_workload_matches_oracle(eng, seed, opts):
    tasks = random_workload(1000 + seed)
    wl = Q.Workload(tasks)
    p = Q.Plan(eng, wl, **opts)
    p.run()
    check(p, tasks)
    p.close()


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("opts", [dict(), dict(delta_frac=0.0, min_group=2, batched=0)])
def test_random_workload_multi_tile_registers(eng, seed, opts):
    tasks = random_workload(2000 + seed, n_sv=(15, 21))
    wl = Q.Workload(tasks)
    p = Q.Plan(eng, wl, **opts)
    p.run()
    check(p, tasks)
    p.close()

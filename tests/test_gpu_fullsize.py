"""Parity at the full workload sizes, in the launch configuration bench.py
times (reuse + batched, graph-captured): the whole workload runs on the GPU,
and sampled tasks are checked against the oracle one by one."""
import json
import os

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


@pytest.mark.parametrize("prefix_fp64", [0, 1])
def test_vqe24_full_size_sampled(eng, prefix_fp64):
    # the bench's configuration (compensated FP32 throughout), and the same
    # workload with the shared prefix in FP64, rounded once for the FP32
    # suffixes; tasks 0, 5 and 255 against the oracle, task 5's state too
    tasks = W.vqe24_sweep()                     # 24 qubits, 256 tasks, 200 terms
    keep = 5
    tasks[keep].want_state = True
    plan = Q.Plan(eng, Q.Workload(tasks), prefix_fp64=prefix_fp64)
    plan.run()
    ex = plan.explain()
    assert ex["artifacts"] == 1 and ex["tasks_reusing"] == 256
    # an FP64 boundary serves the FP32 tasks rounded once (legality reading:
    # exact up to that one rounding), and EXPLAIN says so
    art = ex["decisions"][0]["artifact"]
    assert art["consumer_exactness"] == ({"GPU_SV_FP32": "EXACT_UP_TO_ONE_ROUNDING"} if prefix_fp64 else {})
    for i in (0, keep, 255):
        ref = _oracle(tasks, i, i == keep)
        e, nr = plan.energy(i)
        err = energy_error(e, ref["energy"], tasks[i].terms, 24)
        print("prefix_fp64 %d task %d energy %.10e ref %.10e error %.2e" % (prefix_fp64, i, e, ref["energy"], err))
        assert err <= FP32_ENERGY_TOL, (i, err)
        assert abs(nr - 1) < 1e-5
        if i == keep:
            st = plan.state(i, 24, False).astype(np.complex128)
            amp = float(np.max(np.abs(st - ref["state"])))
            print("task %d max-abs amplitude error %.2e" % (i, amp))
            assert amp <= 1e-5


GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "vqe24_256_energies.json")


def _every_task(eng, **opts):
    doc = json.load(open(GOLD))
    ref = np.array([t["energy"] for t in doc["tasks"]])
    tasks = W.vqe24_sweep()
    assert [int(len(t.spans[1])) for t in tasks] == [t["suffix_gates"] for t in doc["tasks"]]
    plan = Q.Plan(eng, Q.Workload(tasks), **opts)
    plan.run()
    e = np.array([plan.energy(i)[0] for i in range(len(tasks))])
    err = np.array([energy_error(e[i], ref[i], tasks[i].terms, 24) for i in range(len(tasks))])
    rel = np.abs(e - ref) / np.abs(ref)
    plan.close()
    return e, ref, err, rel


@pytest.mark.parametrize("prefix_fp64", [0, 1])
def test_vqe24_every_task_against_stored_oracle(eng, prefix_fp64):
    # every one of the 256 tasks of the bench's workload against the oracle's
    # complex128 energies (written by tests/golden/make_vqe24_energies.py):
    # error <= 1e-6 of max(|E_ref|, E_typ) for each task, i.e. relative error
    # <= 1e-6 wherever |E_ref| >= E_typ
    e, ref, err, rel = _every_task(eng, prefix_fp64=prefix_fp64)
    for i in range(len(e)):
        print("prefix_fp64 %d task %3d E %+.9e E_ref %+.9e error %.2e relative %.2e"
              % (prefix_fp64, i, e[i], ref[i], err[i], rel[i]))
    print("prefix_fp64 %d: error over %d tasks: max %.2e median %.2e; relative: median %.2e, above 1e-6: %d"
          % (prefix_fp64, len(err), err.max(), np.median(err), np.median(rel), int(np.sum(rel > 1e-6))))
    worst = int(np.argmax(err))
    assert err.max() <= FP32_ENERGY_TOL, (worst, err[worst])


def test_vqe24_plain_fp32_arithmetic_is_the_error_source(eng):
    # the same workload with plain FP32 gate arithmetic: its rounding through
    # ~600 rotations per amplitude moves energies by about 1e-6 of E_typ,
    # several times the compensated arithmetic's error (both against the
    # oracle; the plain result is an ablation, not a supported accuracy)
    _, _, err_c, _ = _every_task(eng)
    _, _, err_p, _ = _every_task(eng, fp32_arith=Q.FP32_PLAIN)
    print("compensated: max %.2e median %.2e; plain FP32: max %.2e median %.2e"
          % (err_c.max(), np.median(err_c), err_p.max(), np.median(err_p)))
    assert err_c.max() <= FP32_ENERGY_TOL
    assert np.median(err_p) > 2 * np.median(err_c)


def test_vqe24_energy_kernel_alone_on_the_rounded_oracle_state(eng):
    # separates the energy kernel's error from the evolution's: the oracle's
    # final state of task 5, rounded once to complex64, through the energy
    # kernel, against the oracle's energy of that same rounded state
    tasks = W.vqe24_sweep()
    t = tasks[5]
    ref = _oracle(tasks, 5, True)
    psi32 = ref["state"].astype(np.complex64)
    e_round, n_round, _ = orc.energy(24, psi32.astype(np.complex128), t.terms)
    st = torch.tensor(psi32, device="cuda")
    e_gpu, n_gpu = Q.sv_energy_dev(eng, W.MODE_SV_FP32, 24, st.data_ptr(), t.terms)
    kern = energy_error(e_gpu, e_round, t.terms, 24)
    rounding = energy_error(e_round, ref["energy"], t.terms, 24)
    print("task 5: energy kernel %.2e, one FP32 rounding of the state %.2e (of max(|E|, E_typ))" % (kern, rounding))
    assert kern <= 4e-7
    assert abs(n_gpu - n_round) <= 1e-6 * n_round
    del st


_ORACLE = {}


def _oracle(tasks, i, want_state):
    # the default 24-qubit workload is the same in both parametrizations
    key = (i, want_state)
    if key not in _ORACLE:
        _ORACLE[key] = orc.run_task(tasks[i], want_state=want_state)
    return _ORACLE[key]


def _first_error(t, base_len):
    # gate index of the trajectory's first inserted error (base_len if none)
    return len(t.spans[0]) if len(t.spans) > 1 else base_len


def test_noisy22_full_size_32_trajectories(eng):
    # the full 1024-trajectory workload on the GPU; 32 trajectories against
    # the oracle: 8 error-free ones (the shared CDF of the error-free chain)
    # and the 12 earliest and 12 latest first-error forks
    tasks = W.noisy22_trajectories()                   # 22 qubits, 1024 trajectories
    plan = Q.Plan(eng, Q.Workload(tasks))
    plan.run()
    ex = plan.explain()
    assert ex["tasks_reusing"] > 900
    n_gates = np.array([t.n_gates for t in tasks])
    free = np.nonzero(n_gates == 400)[0]
    noisy = np.nonzero(n_gates > 400)[0]
    order = sorted(noisy, key=lambda i: _first_error(tasks[i], 400))
    rng = np.random.default_rng(20260923)
    sample = sorted(set([int(i) for i in rng.choice(free, 8, replace=False)] + [int(i) for i in order[:12]] +
                        [int(i) for i in order[-12:]]))
    assert len(sample) == 32
    for i in sample:
        ref = orc.run_task(tasks[i], want_state=True)
        got = plan.samples(i)
        p = np.abs(ref["state"]) ** 2
        F = np.cumsum(p / p.sum())
        r = ref["samples"].astype(np.int64)
        near = (np.abs(F[np.minimum(r, len(F) - 1)] - tasks[i].uniforms) < 1e-5) | \
               (np.abs(F[np.maximum(r - 1, 0)] - tasks[i].uniforms) < 1e-5)
        print("trajectory %d (first error at gate %d): %d of %d shots equal, %d within 1e-5 of a CDF boundary"
              % (i, _first_error(tasks[i], 400), int(np.sum(got == ref["samples"])), len(got),
                 int(np.sum((got != ref["samples"]) & near))))
        assert np.all((got == ref["samples"]) | near), i


_QEC = {}


def _qec_reference():
    # The oracle's syndromes of all 4096 tasks.  The 100 shared rounds are
    # run once and every task's five rounds continue from the exported rows
    # (orc.tab_run_from; the tableau algorithm is deterministic, so this is
    # bit for bit the run from |0...0>, which tasks 0, 1 and 4095 also get).
    if not _QEC:
        from concurrent.futures import ThreadPoolExecutor
        tasks = W.qec_surface_code_tasks()             # 449 qubits, 100 + 5 rounds, 4096 tasks
        n = tasks[0].n
        pre_out, rows = orc.tab_run(n, tasks[0].spans[0], want_tableau=True)

        def ref(i):
            t = tasks[i]
            assert t.spans[0] is tasks[0].spans[0]
            return np.concatenate([pre_out, orc.tab_run_from(n, rows, W.concat(*t.spans[1:]))])

        with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:  # ctypes calls release the GIL
            refs = list(ex.map(ref, range(len(tasks))))
        for i in (0, 1, 4095):
            assert np.array_equal(refs[i], orc.tab_run(n, tasks[i].gates)), i
        _QEC["tasks"], _QEC["refs"] = tasks, refs
    return _QEC["tasks"], _QEC["refs"]


@pytest.mark.parametrize("frames", [1, 0])
def test_qec_d15_every_task_bit_exact(eng, frames):
    # Pauli frames over the shared rounds (the bench's plan) and every task
    # on its own tableau: all 4096 syndromes equal the oracle's
    tasks, refs = _qec_reference()
    plan = Q.Plan(eng, Q.Workload(tasks), pauli_frames=frames)
    plan.run()
    assert len(plan.explain()["pauli_frames"]) == frames
    bad = [i for i in range(len(tasks)) if not np.array_equal(plan.syndrome(i), refs[i])]
    print("frames %d: %d of %d tasks differ" % (frames, len(bad), len(tasks)))
    assert not bad, bad[:10]
    plan.close()

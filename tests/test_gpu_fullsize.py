"""Parity at the full workload sizes, in the launch configuration bench.py
times (reuse + batched, graph-captured): the whole workload runs on the GPU,
and sampled tasks are checked against the oracle one by one."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2609_23664_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_23664_gb300 import quwarp as Q  # noqa: E402


# Energy error bounds over all 256 tasks of the 24-qubit sweep, FP32
# throughout (0) and with the shared prefix in FP64 (1).  The energy of a
# random-like 24-qubit state is a near-cancellation: its typical size is
# E_typ = ||c||_2 2^(-n/2) = 3.6e-3 against sum |c_k| = 166, and 1 % of the
# tasks have |E| < 0.006 E_typ, where any relative error diverges.  So the
# bound is on the error normalized by max(|E_ref|, E_typ), plus the median
# relative error; both a little above the values measured on GB300 (FP32:
# normalized max 4.8e-6, median relative 1.24e-6; FP64 prefix: 1.45e-6 and
# 3.9e-7).
NORM_BOUND = {0: 1e-5, 1: 3e-6}
MEDIAN_REL_BOUND = {0: 2e-6, 1: 6e-7}


@pytest.fixture(scope="module")
def eng():
    e = Q.Engine(0)
    yield e
    e.close()


@pytest.mark.parametrize("prefix_fp64", [0, 1])
def test_vqe24_full_size_sampled(eng, prefix_fp64):
    # the bench's configuration (FP32 throughout), and the same workload
    # with the shared prefix in FP64, rounded once for the FP32 suffixes
    tasks = W.vqe24_sweep()                     # 24 qubits, 256 tasks, 200 terms
    keep = 5
    tasks[keep].want_state = True
    plan = Q.Plan(eng, Q.Workload(tasks), prefix_fp64=prefix_fp64)
    plan.run()
    ex = plan.explain()
    assert ex["artifacts"] == 1 and ex["tasks_reusing"] == 256
    c = tasks[0].terms["coef"]
    e_typ = float(np.sqrt(np.sum(c ** 2))) * 2.0 ** (-24 / 2)
    for i in (0, keep, 255):
        ref = _oracle(tasks, i, i == keep)
        e, nr = plan.energy(i)
        rel = abs(e - ref["energy"]) / abs(ref["energy"])
        print("prefix_fp64 %d task %d energy %.10e ref %.10e rel %.2e" % (prefix_fp64, i, e, ref["energy"], rel))
        assert abs(e - ref["energy"]) <= 2e-5 * float(np.sum(np.abs(tasks[i].terms["coef"])))
        # FP32 states: the energy is a near-cancellation (|E| ~ E_typ), so its
        # error is bounded relative to max(|E|, E_typ), as over all 256 tasks
        assert abs(e - ref["energy"]) / max(abs(ref["energy"]), e_typ) <= NORM_BOUND[prefix_fp64]
        assert abs(nr - 1) < 1e-5
        if i == keep:
            st = plan.state(i, 24, False).astype(np.complex128)
            err = float(np.max(np.abs(st - ref["state"])))
            print("task %d max-abs amplitude error %.2e" % (i, err))
            assert err <= 1e-5


GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "vqe24_256_energies.json")


@pytest.mark.parametrize("prefix_fp64", [0, 1])
def test_vqe24_every_task_against_stored_oracle(eng, prefix_fp64):
    # every one of the 256 tasks of the bench's workload against the oracle's
    # complex128 energies (written by tests/golden/make_vqe24_energies.py)
    doc = json.load(open(GOLD))
    ref = np.array([t["energy"] for t in doc["tasks"]])
    tasks = W.vqe24_sweep()
    assert [int(len(t.spans[1])) for t in tasks] == [t["suffix_gates"] for t in doc["tasks"]]
    plan = Q.Plan(eng, Q.Workload(tasks), prefix_fp64=prefix_fp64)
    plan.run()
    e = np.array([plan.energy(i)[0] for i in range(len(tasks))])
    rel = np.abs(e - ref) / np.abs(ref)
    print("prefix_fp64 %d: relative energy error over %d tasks: max %.2e median %.2e, above 1e-6: %d"
          % (prefix_fp64, len(rel), rel.max(), np.median(rel), int(np.sum(rel > 1e-6))))
    c = tasks[0].terms["coef"]
    e_typ = float(np.sqrt(np.sum(c ** 2))) * 2.0 ** (-24 / 2)
    normed = np.abs(e - ref) / np.maximum(np.abs(ref), e_typ)
    print("  error / max(|E_ref|, E_typ): max %.2e median %.2e" % (normed.max(), np.median(normed)))
    assert np.all(np.abs(e - ref) <= 2e-5 * float(np.sum(np.abs(c))))
    assert normed.max() <= NORM_BOUND[prefix_fp64], normed.max()
    assert np.median(rel) <= MEDIAN_REL_BOUND[prefix_fp64], np.median(rel)


_ORACLE = {}


def _oracle(tasks, i, want_state):
    # the default 24-qubit workload is the same in both parametrizations
    key = (i, want_state)
    if key not in _ORACLE:
        _ORACLE[key] = orc.run_task(tasks[i], want_state=want_state)
    return _ORACLE[key]


def test_noisy22_full_size_sampled(eng):
    tasks = W.noisy22_trajectories()                   # 22 qubits, 1024 trajectories
    plan = Q.Plan(eng, Q.Workload(tasks))
    plan.run()
    ex = plan.explain()
    assert ex["tasks_reusing"] > 900
    # earliest / latest error trajectories and error-free ones
    n_gates = np.array([t.n_gates for t in tasks])
    free = np.nonzero(n_gates == 400)[0]
    noisy = np.nonzero(n_gates > 400)[0]
    sample = [int(free[0]), int(free[-1]), int(noisy[0]), int(noisy[-1])]
    for i in sample:
        ref = orc.run_task(tasks[i], want_state=True)
        got = plan.samples(i)
        p = np.abs(ref["state"]) ** 2
        F = np.cumsum(p / p.sum())
        r = ref["samples"].astype(np.int64)
        near = (np.abs(F[np.minimum(r, len(F) - 1)] - tasks[i].uniforms) < 1e-5) | \
               (np.abs(F[np.maximum(r - 1, 0)] - tasks[i].uniforms) < 1e-5)
        assert np.all((got == ref["samples"]) | near), i


def test_qec_d15_full_size_sampled(eng):
    tasks = W.qec_surface_code_tasks()                       # 449 qubits, 100 + 5 rounds, 4096 tasks
    plan = Q.Plan(eng, Q.Workload(tasks))
    plan.run()
    for i in (0, 1, 4095):
        ref = orc.tab_run(tasks[i].n, tasks[i].gates)
        got = plan.syndrome(i)
        assert len(got) == 105 * 224
        assert np.array_equal(got, ref), i

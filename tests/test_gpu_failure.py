"""Failure detection without a GPU fault: the persistent suffix launch's
dependency waits are bounded; a plan built with the test-only
fault_injection option makes one wait run out (it waits on a job no CTA
takes), and the host must see QW_ERR_DEVICE_TIMEOUT while the device stays
usable for the next plan."""
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


def test_bounded_wait_reports_timeout_and_device_stays_usable():
    eng = Q.Engine(0)
    tasks = W.vqe24_sweep(n=16, n_tasks=6, n_terms=10)
    bad = Q.Plan(eng, Q.Workload(tasks), fault_injection=1)
    bad.execute()
    with pytest.raises(Q.QuwarpError) as ei:
        bad.wait()
    assert ei.value.status == -5   # QW_ERR_DEVICE_TIMEOUT
    bad.close()
    good = Q.Plan(eng, Q.Workload(tasks))
    good.run()
    ref = orc.run_task(tasks[0])
    e, _ = good.energy(0)
    assert energy_error(e, ref["energy"], tasks[0].terms, tasks[0].n) <= FP32_ENERGY_TOL
    eng.close()


def test_destroying_the_engine_releases_its_plans():
    eng = Q.Engine(0)
    tasks = W.vqe12_sweep(n_tasks=3)
    plan = Q.Plan(eng, Q.Workload(tasks))
    plan.run()
    e_before, _ = plan.energy(1)
    eng.close()                       # releases the plan's device memory
    assert plan.explain()["artifacts"] == 1
    assert plan.energy(1)[0] == e_before     # host results stay readable
    with pytest.raises(Q.QuwarpError) as ei:
        plan.execute()
    assert ei.value.status == -6      # QW_ERR_STATE
    plan.close()

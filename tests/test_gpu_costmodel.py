"""Learned cost model (Eq. 2 costs): engine-measured timings -> GPU training
-> planning.  Shows what the trained network gains over the analytic model
on held-out engine timings, and that plans built with it stay exact."""
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


def _dense(seed, groups):
    return W.dense_prefix_groups(seed=seed, groups=groups, group_size=4, prefix_gates=600, suffix_layers=12)


@pytest.fixture(scope="module")
def trained():
    eng = Q.Engine(0)
    # timing corpus: the mixed family (shared prefixes and prefix-free
    # circuits) at 12..20 qubits and the dense-prefix family (gate-dense
    # local prefixes, sparse layered suffixes), a training and a held-out seed
    tr = W.mixed_planned(seed=11, n_tasks=900, n_min=12, n_max=20) + _dense(31, 24)
    te = W.mixed_planned(seed=12, n_tasks=200, n_min=12, n_max=20) + _dense(32, 6)
    f_tr, y_tr, a_tr = eng.costmodel_probe(Q.Workload(tr), 3 * len(tr))
    f_te, y_te, a_te = eng.costmodel_probe(Q.Workload(te), 3 * len(te))
    loss = eng.costmodel_train(f_tr, y_tr, epochs=60, batch=256, lr=2e-3, seed=7)
    return eng, (f_tr, y_tr, a_tr), (f_te, y_te, a_te), loss


def test_probe_collects_engine_timings(trained):
    eng, (f, y, a), _, _ = trained
    assert len(y) >= 2000 and f.shape == (len(y), Q.MLP_IN)
    assert np.all(np.isfinite(y)) and np.all(y > 8)      # > 256 ns per timed segment


def test_training_beats_the_analytic_model_on_held_out_timings(trained):
    eng, (f_tr, y_tr, _), (f, y, a), loss = trained
    base = float(np.mean((y_tr - y_tr.mean()) ** 2))
    assert loss < 0.25 * base                              # learned something
    pred = eng.costmodel_predict(f)
    err_mlp = float(np.mean(np.abs(pred - y)))             # mean |log2 error|
    err_ana = float(np.mean(np.abs(a - y)))
    print("held-out mean |log2 error|: mlp %.3f analytic %.3f" % (err_mlp, err_ana))
    assert err_mlp < err_ana
    assert err_mlp < 0.5                                   # within ~1.4x on average


def test_parameters_roundtrip_and_forward_kernel_agree(trained):
    eng, _, (f, y, a), _ = trained
    p, m, s = eng.costmodel_get()
    pred = eng.costmodel_predict(f[:50])
    e2 = Q.Engine(0)
    e2.costmodel_set(p, m, s)
    assert np.array_equal(e2.costmodel_predict(f[:50]), pred)
    e2.close()


def test_planning_with_the_learned_model_stays_exact(trained):
    eng = trained[0]
    tasks = W.mixed_planned(seed=13, n_tasks=60, n_min=12, n_max=18)
    wl = Q.Workload(tasks)
    plan = Q.Plan(eng, wl, cost_model=Q.COST_MLP)
    ex = plan.explain()
    srcs = {d["cost_source"] for d in ex["decisions"]}
    assert "MLP" in srcs
    plan.run()
    for i in range(0, len(tasks), 7):
        ref = orc.run_task(tasks[i])
        e, _ = plan.energy(i)
        assert energy_error(e, ref["energy"], tasks[i].terms, tasks[i].n) <= FP32_ENERGY_TOL, i


def _run_ms(eng, wl, **opts):
    p = Q.Plan(eng, wl, **opts)
    p.run()
    ms = []
    for _ in range(3):
        p.run()
        ms.append(p.cost_record()["device_total_ms"])
    return p, float(np.median(ms))


def test_learned_costs_change_plans_for_the_better(trained):
    # Groups of 4 tasks sharing a gate-dense local prefix (one pass, 600
    # gates) with sparse layered suffixes (~8 passes of 20 rotations).  The
    # analytic cost (passes x the measured time of a pass) prices the
    # prefix at an eighth of a suffix, so Eq. 2 refuses reuse; the learned
    # model, which sees the gate counts, prices it near a suffix, reuse is
    # chosen, and the realized device time drops.
    eng = trained[0]
    tasks = _dense(33, 8)
    wl = Q.Workload(tasks)
    pa, t_a = _run_ms(eng, wl, cost_model=Q.COST_ANALYTIC)
    pm, t_m = _run_ms(eng, wl, cost_model=Q.COST_MLP)
    da = [d["decision"] for d in pa.explain()["decisions"]]
    dm = [d["decision"] for d in pm.explain()["decisions"]]
    srcs = {d["cost_source"] for d in pm.explain()["decisions"]}
    print("analytic: %s, %.2f ms; learned (%s): %s, %.2f ms" % (da, t_a, srcs, dm, t_m))
    assert da.count("REUSE") == 0 and dm.count("REUSE") == len(dm) == 8
    assert t_m < 0.8 * t_a
    for i in range(0, len(tasks), 5):
        ref = orc.run_task(tasks[i])
        for p in (pa, pm):
            assert energy_error(p.energy(i)[0], ref["energy"], tasks[i].terms, tasks[i].n) <= FP32_ENERGY_TOL, i
    pa.close()
    pm.close()

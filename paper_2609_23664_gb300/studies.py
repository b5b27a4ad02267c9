"""Calibration studies on one GPU, through the public API.

breakeven  -- Eq. 2 break-even: for the VQE family at a few register sizes
              and group sizes N, the planner's estimated speedup (direct /
              planned cost) and the realized one (per-task replay vs the
              reuse plan, same GPU), and the smallest N at which reuse pays
              (N*), with analytic and learned costs (Sec. VI-D, Fig. 3).
costmodel  -- the learned cost model (Eq. 2 costs): >= 10^4 engine-measured
              segment timings of the mixed family, training on the GPU,
              held-out error of the learned vs the analytic model, and the
              realized time of plans made with each, against the best of
              the plans compared (decision regret).
mixed      -- the mixed planned workload at full size: 2000 tasks at 16-30
              qubits (30-qubit boundaries of 8.6 GB under a 120 GB store
              budget), planned with analytic and with learned costs (the
              model trained by the costmodel study first) and without
              reuse: planning time, decisions, boundary bytes, realized
              device time of one execution after a first one, every norm,
              and the reuse plans' energies against the plan without reuse.

Usage: python -m paper_2609_23664_gb300.studies {breakeven,costmodel,mixed,all} [--out FILE]
Prints one JSON document (and writes it to FILE).
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import quwarp as Q
from . import workloads as W


def _device_ms(eng, wl, repeats=3, **opts):
    p = Q.Plan(eng, wl, **opts)
    p.run()                                   # first run: allocation, upload, graph capture
    ms = []
    for _ in range(repeats):
        p.run()
        ms.append(p.cost_record()["device_total_ms"])
    ex = p.explain()
    p.close()
    return float(np.median(ms)), ex


def breakeven(eng, n_list=(20, 24), N_list=(1, 2, 3, 4, 6, 8, 16, 32, 64), terms=20,
              prefix_layers=20, cost_models=(Q.COST_ANALYTIC,)):
    rows = []
    for n in n_list:
        for N in N_list:
            tasks = W.vqe24_sweep(n=n, n_tasks=N, prefix_layers=prefix_layers, n_terms=terms)
            wl = Q.Workload(tasks)
            t_replay, _ = _device_ms(eng, wl, reuse=0, batched=1)
            for cm in cost_models:
                # delta 0: reuse whenever the inequality holds, so that the
                # realized side exists at every N >= 2
                t_plan, ex = _device_ms(eng, wl, delta_frac=0.0, cost_model=cm)
                dec = ex["decisions"][0]["decision"] if ex["decisions"] else "NONE"
                rows.append({"qubits": n, "tasks": N,
                             "cost_model": "MLP" if cm == Q.COST_MLP else "ANALYTIC",
                             "decision": dec, "estimated_speedup": ex["estimated_speedup"],
                             "replay_ms": t_replay, "plan_ms": t_plan,
                             "realized_speedup": t_replay / t_plan})
            wl.close()
    nstar = {}
    for n in n_list:
        for cm in {r["cost_model"] for r in rows}:
            # reuse needs two tasks; 2 % above 1 separates a gain from timing noise
            pays = [r["tasks"] for r in rows if r["qubits"] == n and r["cost_model"] == cm and
                    r["tasks"] >= 2 and r["realized_speedup"] > 1.02]
            est = [r["tasks"] for r in rows
                   if r["qubits"] == n and r["cost_model"] == cm and r["decision"] == "REUSE"]
            nstar["%d/%s" % (n, cm)] = {"realized": min(pays) if pays else None,
                                         "planner": min(est) if est else None}
    return {"study": "breakeven", "workload": "VQE family, %d-layer HEA prefix, U{1..4} suffix layers, "
            "%d terms; replay = batched per-task rerun, plan = reuse with delta 0" % (prefix_layers, terms),
            "rows": rows, "n_star": nstar}


def costmodel(eng, n_min=16, n_max=22, train_tasks=3600, test_tasks=400, eval_tasks=600,
              epochs=80, seed=7):
    t0 = time.perf_counter()
    tr = W.mixed_planned(seed=21, n_tasks=train_tasks, n_min=n_min, n_max=n_max)
    te = W.mixed_planned(seed=22, n_tasks=test_tasks, n_min=n_min, n_max=n_max)
    wtr, wte = Q.Workload(tr), Q.Workload(te)
    f_tr, y_tr, a_tr = eng.costmodel_probe(wtr, 3 * len(tr))
    f_te, y_te, a_te = eng.costmodel_probe(wte, 3 * len(te))
    t_probe = time.perf_counter() - t0
    t1 = time.perf_counter()
    loss = eng.costmodel_train(f_tr, y_tr, epochs=epochs, batch=256, lr=2e-3, seed=seed)
    t_train = time.perf_counter() - t1
    pred = eng.costmodel_predict(f_te)

    def errs(p):
        d = p - y_te
        return {"mean_abs_log2": float(np.mean(np.abs(d))),
                "mape_log_cost": float(np.mean(np.abs(d) / np.abs(y_te))),
                "mape_time": float(np.mean(np.abs(np.exp2(d) - 1.0)))}

    # plans on a third workload: analytic vs learned costs, and two fixed
    # policies (reuse wherever Eq. 2 holds with delta 0, no reuse at all)
    ev = W.mixed_planned(seed=23, n_tasks=eval_tasks, n_min=n_min, n_max=n_max)
    wev = Q.Workload(ev)
    plans = {}
    for key, opts in (("analytic", dict(cost_model=Q.COST_ANALYTIC)),
                      ("mlp", dict(cost_model=Q.COST_MLP)),
                      ("reuse_delta0", dict(cost_model=Q.COST_ANALYTIC, delta_frac=0.0)),
                      ("no_reuse", dict(reuse=0))):
        ms, ex = _device_ms(eng, wev, **opts)
        decs = [d["decision"] for d in ex["decisions"]]
        plans[key] = {"device_ms": ms, "reuse_decisions": decs.count("REUSE"),
                      "abstain_decisions": decs.count("ABSTAIN"), "artifacts": ex["artifacts"],
                      "mlp_costed": sum(1 for d in ex["decisions"] if d["cost_source"] == "MLP")}
    best = min(v["device_ms"] for v in plans.values())
    for v in plans.values():
        v["regret"] = v["device_ms"] / best - 1.0
    for w in (wtr, wte, wev):
        w.close()
    return {"study": "costmodel",
            "workload": "mixed family: 60%% of tasks in groups of U{2..64} sharing a random prefix, "
                        "the rest prefix-free; %d..%d qubits, FP32" % (n_min, n_max),
            "train_rows": int(len(y_tr)), "test_rows": int(len(y_te)), "probe_s": t_probe,
            "train_s": t_train, "train_loss": float(loss),
            "held_out": {"mlp": errs(pred), "analytic": errs(a_te)},
            "plans": plans}


def mixed(eng, n_tasks=2000, n_min=16, n_max=30, store_gb=120.0, with_mlp=True):
    """The engine's store budget is the workload's (store_gb); see main."""
    tasks = W.mixed_planned(n_tasks=n_tasks, n_min=n_min, n_max=n_max)
    wl = Q.Workload(tasks)
    variants = [("analytic", dict(cost_model=Q.COST_ANALYTIC))]
    if with_mlp:
        variants.append(("mlp", dict(cost_model=Q.COST_MLP)))
    variants.append(("no_reuse", dict(reuse=0)))
    plans, energies = {}, {}
    for key, opts in variants:
        t0 = time.perf_counter()
        p = Q.Plan(eng, wl, **opts)
        t_plan = time.perf_counter() - t0
        t1 = time.perf_counter()
        p.run()                                   # first run: allocation, upload, graph capture
        t_first = time.perf_counter() - t1
        t2 = time.perf_counter()
        p.run()
        t_second = time.perf_counter() - t2
        rec, ex = p.cost_record(), p.explain()
        decs = [d["decision"] for d in ex["decisions"]]
        plans[key] = {"planning_s": t_plan, "first_run_s": t_first, "run_s": t_second,
                      "device_ms": rec["device_total_ms"], "reuse_decisions": decs.count("REUSE"),
                      "abstain_decisions": decs.count("ABSTAIN"), "refuse_decisions": decs.count("REFUSE"),
                      "mlp_costed": sum(1 for d in ex["decisions"] if d.get("cost_source") == "MLP"),
                      "artifacts": ex["artifacts"], "artifact_bytes": rec["artifact_bytes"],
                      "estimated_speedup": ex["estimated_speedup"], "kernel_launches": rec["kernel_launches"]}
        en = np.array([p.energy(i) for i in range(len(tasks))])
        energies[key] = en[:, 0]
        plans[key]["max_norm_error"] = float(np.max(np.abs(en[:, 1] - 1.0)))
        p.close()
    wl.close()
    n_hist = np.bincount([t.n for t in tasks], minlength=n_max + 1)[n_min:]
    scale = np.array([float(np.sum(np.abs(t.terms["coef"]))) for t in tasks])
    return {"study": "mixed",
            "workload": "mixed planned family at full size: %d tasks, %d..%d qubits, FP32, 60%% in groups "
                        "of U{2..64} sharing a prefix of 50..500 gates (suffixes of 10..100), 40%% prefix-free "
                        "(50..550 gates); 8-term Hamiltonian per task; store budget %.0f GB"
                        % (n_tasks, n_min, n_max, store_gb),
            "tasks_per_qubit_count": {str(n_min + i): int(c) for i, c in enumerate(n_hist)},
            "plans": plans,
            # reuse plans run each task's gates from a boundary instead of
            # from |0...0>: their energies must match the plan without reuse
            # up to FP32 rounding (scaled by the sum of |coefficients|)
            "max_energy_diff_vs_no_reuse": {
                k: float(np.max(np.abs(energies[k] - energies["no_reuse"]) / scale))
                for k in energies if k != "no_reuse"}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["breakeven", "costmodel", "mixed", "all"])
    ap.add_argument("--out", default=None)
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args(argv)
    # the mixed workload runs under a 120 GB boundary-store budget
    eng = Q.Engine(a.device, store_budget_bytes=int(120e9) if a.study == "mixed" else 0)
    if a.study == "breakeven":
        res = breakeven(eng)
    elif a.study == "costmodel":
        res = costmodel(eng)
    elif a.study == "mixed":
        # learned costs come from the costmodel study's training first
        res = {"costmodel": costmodel(eng), "mixed": mixed(eng)}
    else:
        # the learned model is trained first, then both models plan the sweep
        res = {"costmodel": costmodel(eng),
               "breakeven": breakeven(eng, cost_models=(Q.COST_ANALYTIC, Q.COST_MLP))}
    res["engine"] = eng.info()
    txt = json.dumps(res, indent=1)
    print(txt)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt)
    eng.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python3
"""Benchmark of the reuse hot path on GB300.

Workload (per GPU): batched VQE sweep at 24 qubits, FP32 statevector with
FP64 energy reductions -- 20-layer hardware-efficient shared prefix, 256
tasks with U{1..4} suffix layers, 200-term random Pauli Hamiltonian, all
suffixes in one persistent CUDA-graph-captured launch.

A step = one execution of the whole planned workload (prefix once, every
suffix, every energy).  `value` = tasks/s of the reuse+batched plan, timed
with CUDA events on the stream the plan runs on, inputs resident on the
device.  The same GPU also runs the per-task replay plan (same kernels, no
reuse, one launch sequence per task) and the batched replay ablation;
their tasks/s and the ratio are reported.  `e2e` runs the same workload
through the public C ABI from host buffers (workload submission, planning,
upload, execution, read-back of every energy) per step.

Multi-GPU (torchrun): every rank runs its own seeded replica (tasks are
independent: weak scaling, no collective on the data path); the step time
is the max over ranks.  `--impl reference` times the CPU oracle (per-task
rerun in complex128 on the host cores) on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2609_23664_gb300 import replicas as R  # noqa: E402
from paper_2609_23664_gb300 import workloads as W  # noqa: E402

METRIC = "workload tasks/s: reuse+batched vs per-task replay, same GB300; HBM % of peak"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--qubits", type=int, default=24)
    ap.add_argument("--tasks", type=int, default=256)
    ap.add_argument("--prefix-layers", type=int, default=20)
    ap.add_argument("--terms", type=int, default=200)
    ap.add_argument("--replay-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-replay", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-tasks", type=int, default=1)
    ap.add_argument("--cpu-families", type=int, default=1,
                    help="1: also time the oracle on every workload family (all cores and one core)")
    ap.add_argument("--qec-steps", type=int, default=3,
                    help="also time the QEC, noisy and small-VQE families (steps each); 0 = skip")
    ap.add_argument("--fuse-energy", type=int, default=0,
                    help="1: energy blocks as work items of the persistent suffix launch")
    ap.add_argument("--tile-qubits", type=int, default=0, help="0: autotuned")
    ap.add_argument("--low-qubits", type=int, default=0, help="0: autotuned")
    ap.add_argument("--dense-qubits", type=int, default=28,
                    help="register of the tensor-core dense-block family (0: skip it)")
    ap.add_argument("--dense-only", action="store_true",
                    help="run only the dense-block family (one JSON line)")
    ap.add_argument("--window", type=int, default=0,
                    help="tasks advanced together in the persistent launch (0: all of a wave)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return ap.parse_args()


def workload_desc(a):
    return ("vqe%d_fp32: %d qubits, %d-layer HEA shared prefix, %d tasks x U{1..4} HEA suffix "
            "layers, %d-term random Pauli H" % (a.qubits, a.qubits, a.prefix_layers, a.tasks, a.terms))


def make_tasks(a, rank):
    return W.vqe24_sweep(seed=R.rank_seed(W.BASE_SEED + 2, rank), n=a.qubits,
                           prefix_layers=a.prefix_layers, n_tasks=a.tasks, n_terms=a.terms)


# ---- clocks during the timed region -------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.lines = []
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.p:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.t.join(timeout=5)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- helpers -------------------------------------------------------------------------

def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def fp32_peak_tflops(sm_count: int):
    """FP32 peak from unit counts and the maximum SM clock: 128 FP32 lanes
    per SM, an FMA counted as two operations."""
    mhz, src = 2070.0, "maximum SM clock 2070 MHz (nominal)"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
        src = "maximum SM clock %.0f MHz (MEASURED_PEAKS.json)" % mhz
    except Exception:
        pass
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12, "%d SMs x 128 FP32 lanes x 2 (FMA) x %s" % (sm_count, src)


def profiled_traffic(kernel: str, workload_key: str, field: str = "dram"):
    """DRAM bytes per launch from the committed ncu summary, if its source
    hash matches the kernel source compiled now (else None)."""
    import hashlib
    src = os.path.join(ROOT, "paper_2609_23664_gb300", "csrc")
    h = hashlib.sha256()
    for fn in ("sv_kernels.cu", "sv_df.cuh", "obs_kernels.cu", "energy_block.cuh", "qw_internal.h"):
        with open(os.path.join(src, fn), "rb") as f:
            h.update(f.read())
    digest = h.hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload_key))
    try:
        txt = open(path).read()
    except OSError:
        return None
    m1 = re.search(r"source_sha16:\s*([0-9a-f]{16})", txt)
    m2 = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m1 or not m2 or m1.group(1) != digest:
        return None
    if field == "lts_pct":
        m3 = re.search(r"lts__throughput\.avg\.pct_of_peak_sustained_elapsed \| ([0-9.]+)", txt)
        return float(m3.group(1)) if m3 else None
    return float(m2.group(1))


def dist_setup():
    return R.env_ranks()


def max_over_ranks(x: float, world: int) -> float:
    return R.max_over_ranks(x, world, "cuda")


def barrier(world):
    R.barrier(world)


# ---- CPU oracle (reference arm and cpu_baseline) -------------------------------------

def oracle_tasks_per_s(a, n_tasks: int):
    """Times the oracle on the first tasks; returns (tasks/s, seconds,
    threads, the oracle's energies)."""
    from oracle import oracle as orc
    tasks = make_tasks(a, 0)[:n_tasks]
    t0 = time.perf_counter()
    energies = [orc.run_task(t)["energy"] for t in tasks]
    dt = time.perf_counter() - t0
    return n_tasks / dt, dt, orc.num_threads(), energies


_ORACLE_TIMER = r"""
import json, os, sys, time
sys.path.insert(0, %r)
from oracle import oracle as orc
from paper_2609_23664_gb300 import workloads as W
orc.build()
fam, count, gate_frac, term_frac = %r, %d, %r, %r
if fam == "vqe12_fp64":
    tasks = W.vqe12_sweep()
elif fam == "vqe24_fp32":
    tasks = W.vqe24_sweep()
elif fam == "noisy22":
    tasks = W.noisy22_trajectories()
elif fam == "qec_d15":
    tasks = W.qec_surface_code_tasks()
else:
    tasks = [t for t in W.mixed_planned() if t.n <= 20]
tasks = tasks[:count]
t0 = time.perf_counter()
tg = te = 0.0
for t in tasks:
    if t.mode == 2:
        orc.tab_run(t.n, t.gates)
    elif gate_frac is None:
        orc.run_task(t)
    else:
        g = t.gates
        a = time.perf_counter()
        psi = orc.sv_run(t.n, g[:max(1, int(len(g) * gate_frac))])
        b = time.perf_counter()
        orc.energy(t.n, psi, t.terms[:max(1, int(len(t.terms) * term_frac))])
        tg += b - a
        te += time.perf_counter() - b
print(json.dumps({"s": time.perf_counter() - t0, "threads": orc.num_threads(), "tasks": len(tasks),
                  "gates_s": tg, "energy_s": te}))
"""


def oracle_time(family, count, threads=None, gate_frac=None, term_frac=None):
    """Seconds the oracle takes for the first `count` tasks of a workload
    family, in a fresh process (OMP_NUM_THREADS = threads when given);
    with gate_frac / term_frac only that fraction of each task's gates and
    Hamiltonian terms runs (for an extrapolated single-core figure)."""
    env = dict(os.environ)
    if threads:
        env["OMP_NUM_THREADS"] = str(threads)
    code = _ORACLE_TIMER % (ROOT, family, count, gate_frac, term_frac)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baselines(n_vqe24):
    """The oracle (per-task rerun from |0...0>, complex128 / unpacked
    tableau) on bounded samples of every workload family, on all host
    cores and on one core."""
    out = {}
    specs = [
        ("vqe12_fp64", 16, 16, "all 16 tasks (config 1, in full)", None),
        ("vqe24_fp32", 256, 2, "2 of 256 tasks (config 2)", (0.125, 0.1)),
        ("noisy22", 1024, 4, "4 of 1024 trajectories at 22 qubits (config 3)", None),
        ("qec_d15", 4096, 8, "8 of 4096 tasks from |0...0>, 105 rounds each (config 4)", None),
        ("mixed_n_le_20", 2000, 40, "the first 40 tasks with n <= 20 of the 2000-task mixed workload (config 5)",
         None),
    ]
    for fam, total, count, sample, partial in specs:
        allc = oracle_time(fam, count)
        if not allc:
            continue
        ent = {"unit": "tasks/s", "kind": "oracle", "sample": sample, "tasks_in_workload": total,
               "value": allc["tasks"] / allc["s"], "cores": allc["threads"], "seconds": allc["s"]}
        if fam == "qec_d15":
            # the tableau oracle's loops are sequential: one core either way
            ent["cores"] = 1
            ent["single_core_value"] = ent["value"]
        elif partial:
            one = oracle_time(fam, 1, threads=1, gate_frac=partial[0], term_frac=partial[1])
            if one:
                # gate passes and energy terms scale linearly with their count
                est = one["gates_s"] / partial[0] + one["energy_s"] / partial[1]
                ent["single_core_value"] = 1.0 / est
                ent["single_core_note"] = ("extrapolated from %.1f%% of one task's gates and %.0f%% of its "
                                           "terms on one core" % (100 * partial[0], 100 * partial[1]))
        else:
            one = oracle_time(fam, max(1, count // 4), threads=1)
            if one:
                ent["single_core_value"] = one["tasks"] / one["s"]
        ent["extrapolated_workload_s"] = total / ent["value"]
        out[fam] = ent
    return out


def run_reference(a):
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    from oracle import oracle as orc
    orc.build()
    tasks = make_tasks(a, 0)
    per = []
    for s in range(a.warmup + a.steps):
        t = tasks[s % len(tasks)]
        t0 = time.perf_counter()
        orc.run_task(t)
        dt = time.perf_counter() - t0
        if s >= a.warmup:
            per.append(dt)
    ms = 1000.0 * statistics.mean(per)
    value = 1000.0 / ms
    sample = "1 task per step (per-task rerun from |0>, complex128: %d gates + %d-term energy)" % (
        tasks[0].n_gates, a.terms)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "tasks/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(a), "global_batch": a.tasks,
                                            "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": "tasks/s", "cores": orc.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "tasks/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- native arm ------------------------------------------------------------------------

def run_native(a):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        torch.cuda.set_device(local)
        R.init(world, "nccl", device=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2609_23664_gb300 import quwarp as Q

    eng = Q.Engine(local)
    info = eng.info()
    if a.dense_only:
        peak, peak_src = load_peaks()
        if rank == 0:
            print(json.dumps({"dense_tc": dense_family(a, eng, torch.cuda.current_stream(), peak),
                              "peak_gbs": peak, "peak_source": peak_src}), flush=True)
        R.finish(world)
        return 0
    tasks = make_tasks(a, rank)
    n_tasks = len(tasks)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream

    wl = Q.Workload(tasks)
    plan = Q.Plan(eng, wl, **plan_opts(a))   # the first plan also autotunes the tiles
    ex = plan.explain()
    # planning time (host): median of three plans of the same workload
    pts = []
    for _ in range(3):
        t0 = time.perf_counter()
        Q.Plan(eng, wl, **plan_opts(a)).close()
        pts.append((time.perf_counter() - t0) * 1e3)
    planning_ms = statistics.median(pts)
    for _ in range(max(1, a.warmup)):
        plan.execute(sptr)
        plan.wait()

    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    recs = []
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    if a.profile_range:
        torch.cuda.profiler.start()
    ev0.record(stream)
    evs[0].record(stream)
    for k in range(a.steps):
        plan.execute(sptr)
        plan.wait()
        evs[k + 1].record(stream)
        recs.append(plan.cost_record())
    ev1.record(stream)
    torch.cuda.synchronize()
    if a.profile_range:
        torch.cuda.profiler.stop()
    barrier(world)
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1) / a.steps
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(a.steps)]
    ms_max = max_over_ranks(ms, world)
    value = R.whole_job_rate(n_tasks, world, ms_max)
    cr = recs[-1]
    launches = int(cr["kernel_launches"])
    suffix_ms = statistics.mean(r["suffix_ms"] for r in recs)
    energy_ms = statistics.mean(r["energy_ms"] for r in recs)
    prefix_ms = statistics.mean(r["prefix_ms"] for r in recs)
    # energies of the last step, checked for finiteness (parity lives in tests)
    e_last = [plan.energy(i)[0] for i in range(n_tasks)]
    assert all(np.isfinite(e_last))

    peak, peak_src = load_peaks()
    S = 8 << a.qubits
    batch_alg_bytes = float(cr.get("batch_alg_bytes", 0.0))
    energy_alg_bytes = float(cr.get("energy_alg_bytes", 0.0))
    batch_flops = float(cr.get("batch_alg_flops", 0.0))
    wkey = "vqe%d_%dtasks" % (a.qubits, a.tasks)
    comp = cr.get("fp32_arith") == "compensated"
    l2_bytes = float(cr.get("energy_l2_bytes", 0.0))
    l2_peak = eng.probe_l2()
    fp32_peak, fp32_src = fp32_peak_tflops(int(info["sm_count"]))

    def hbm(alg, dur):
        g = alg / (dur * 1e-3) / 1e9
        return {"achieved": g, "peak": peak, "unit": "GB/s", "frac": g / peak, "peak_source": peak_src,
                "algorithmic_bytes_per_launch": alg}

    # the persistent suffix launch: compensated FP32 passes are bound by
    # FP32 arithmetic (double-float: ~16 packed operations per two-term
    # output), plain ones by latency against HBM
    t_sv = batch_flops / (suffix_ms * 1e-3) / 1e12 if suffix_ms > 0 else 0.0
    sv = {"kernel": "sv_batch_kernel", "launch_ms": suffix_ms, "fp32_arith": cr.get("fp32_arith"),
          "hbm": hbm(batch_alg_bytes, suffix_ms),
          "alu": {"achieved": t_sv, "peak": fp32_peak, "unit": "TFLOP/s", "frac": t_sv / fp32_peak,
                  "peak_source": fp32_src, "algorithmic_flops_per_launch": batch_flops},
          "traffic": profiled_traffic("sv_batch_kernel", wkey),
          "traffic_source": "ncu dram__bytes of the committed capture (profiles/), scaled to the launch; "
                            "null when the kernel source changed since"}
    # the energy launch: every term's partner amplitudes come from L2
    l2_gbs = l2_bytes / (energy_ms * 1e-3) / 1e9 if energy_ms > 0 else None
    en = {"kernel": "energy_kernel", "launch_ms": energy_ms, "hbm": hbm(energy_alg_bytes, energy_ms),
          "l2": {"achieved": l2_gbs, "peak": l2_peak, "unit": "GB/s",
                 "frac": (l2_gbs / l2_peak) if (l2_gbs and l2_peak) else None,
                 "peak_source": "measured in this run (qw_engine_probe_l2: hashed 64 KB blocks of an "
                                "L2-resident buffer, the kernel's access pattern)",
                 "algorithmic_bytes_per_launch": l2_bytes,
                 "ncu_lts_throughput_pct": profiled_traffic("energy_kernel", wkey, "lts_pct")},
          "traffic": profiled_traffic("energy_kernel", wkey),
          "traffic_source": "ncu dram__bytes of the committed capture (profiles/), scaled to the launch; "
                            "null when the kernel source changed since"}
    if suffix_ms >= energy_ms:
        b = "alu" if comp else "hbm"
        sel = sv["alu"] if comp else sv["hbm"]
        roofline = {"bound": b, "kernel": "sv_batch_kernel", "launch_ms": suffix_ms, "traffic": sv["traffic"]}
    else:
        b, sel = "l2", en["l2"]
        roofline = {"bound": "l2", "kernel": "energy_kernel", "launch_ms": energy_ms, "traffic": en["traffic"]}
    roofline.update({k: sel[k] for k in ("achieved", "peak", "unit", "frac", "peak_source")})
    roofline["kernels"] = {"sv_batch_kernel": sv, "energy_kernel": en,
                           "prefix_passes": {"ms": prefix_ms, "algorithmic_bytes": float(cr.get("prefix_alg_bytes", 0.0)),
                                             "algorithmic_flops": float(cr.get("prefix_alg_flops", 0.0))}}

    line = {"metric": METRIC, "value": value, "unit": "tasks/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(a), "global_batch": world * n_tasks,
                       "qubits": a.qubits, "state_bytes": S,
                       "l2": "inputs larger than L2 (task states %.1f GiB > L2 %.0f MB)" % (
                           n_tasks * S / 2 ** 30, info["l2_bytes"] / 1e6),
                       "parallelism": "replicas (one independent workload per GPU)"},
            "gpu_launches": launches * a.steps,
            "median_ms_per_step": statistics.median(step_ms),
            "planning_ms": planning_ms,
            # planning included: the workload planned once per execution
            "planning_inclusive": {"value": world * n_tasks / ((ms_max + planning_ms) / 1e3), "unit": "tasks/s",
                                   "ms_per_step": ms_max + planning_ms},
            "fp32_arith": cr.get("fp32_arith"),
            "artifacts": ex["artifacts"],
            "tiles": cr.get("wave_tiles"),
            "estimated_speedup": ex["estimated_speedup"],
            "engine_hbm_gbs": info["hbm_gbs"]}
    if ck:
        line["clocks"] = ck

    # per-task replay and batched replay on the same GPU, same kernels
    if not a.no_replay:
        plan.close()
        for key, opts in (("per_task_replay", dict(reuse=0, batched=0)),
                          ("batched_replay", dict(reuse=0, batched=1))):
            rp = Q.Plan(eng, wl, **plan_opts(a), **opts)
            rp.execute(sptr)
            rp.wait()
            barrier(world)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(a.replay_steps):
                rp.execute(sptr)
                rp.wait()
            e1.record(stream)
            torch.cuda.synchronize()
            rms = max_over_ranks(e0.elapsed_time(e1) / a.replay_steps, world)
            line[key] = {"value": world * n_tasks / (rms / 1e3), "unit": "tasks/s", "ms_per_step": rms}
            rp.close()
        line["speedup_vs_per_task_replay"] = value / line["per_task_replay"]["value"]
        line["speedup_vs_batched_replay"] = value / line["batched_replay"]["value"]

    # end to end through the C ABI from host buffers
    if a.e2e_steps > 0:
        plan.close()
        e2e_ms, h2d, d2h = [], 0, 0
        for _ in range(a.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            wl2 = Q.Workload(tasks)
            p2 = Q.Plan(eng, wl2, **plan_opts(a))
            p2.execute(sptr)
            p2.wait()
            en = [p2.energy(i) for i in range(n_tasks)]
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            r2 = p2.cost_record()
            h2d, d2h = int(r2["h2d_bytes"]), int(r2["d2h_bytes"])
            p2.close()
            wl2.close()
            del en
        em = max_over_ranks(statistics.mean(e2e_ms), world)
        line["e2e"] = {"value": world * n_tasks / (em / 1e3), "unit": "tasks/s", "ms_per_step": em,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "includes": "workload submission, planning, device allocation, upload, "
                                   "execution, read-back of all energies"}

    # the other workload families of the paper's evaluation, same GPU:
    # the planned execution vs a comparison plan (same kernels)
    if a.qec_steps > 0 and world == 1:
        fams = line["families"] = {}

        def time_plan(wl, units, opts):
            fp = Q.Plan(eng, wl, **opts)
            fp.execute(sptr)
            fp.wait()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(a.qec_steps):
                fp.execute(sptr)
                fp.wait()
            e1.record(stream)
            torch.cuda.synchronize()
            fms = e0.elapsed_time(e1) / a.qec_steps
            fcr = fp.cost_record()
            fp.close()
            return {"value": units / (fms / 1e3), "unit": "tasks/s", "ms_per_step": fms,
                    "kernel_launches": fcr["kernel_launches"], "artifacts": fcr["artifacts"],
                    "dense_choices": fcr.get("dense_boundaries") or None}

        for key, desc, gen, plans in (
                ("qec_d15", "rotated surface code, 449 qubits, 100 shared + 5 task rounds, 4096 tasks, "
                            "data X/Z errors p=1e-3 (stabilizer)", W.qec_surface_code_tasks,
                 (("pauli_frames", dict(pauli_frames=1)), ("per_task_tableau", dict(pauli_frames=0)))),
                ("noisy22", "22 qubits, 400-gate random circuit, 1024 Pauli-noise trajectories "
                            "(p=1e-3), 100 shots each (FP32)", W.noisy22_trajectories,
                 (("reuse", {}), ("per_task_replay", dict(reuse=0, batched=0)))),
                ("vqe12_fp64", "12 qubits, 6-layer HEA prefix, 16 tasks x final RY+RZ layer, 20-term "
                               "energy (FP64)", W.vqe12_sweep,
                 (("reuse", {}), ("per_task_replay", dict(reuse=0, batched=0)))),
                ("deep_local24", "24 qubits, H layer + 60 layers of RY/CNOT/RZ confined to qubits 8-12 "
                                 "(shared prefix), 64 tasks x RY layer, 32-term energy (FP32)",
                 lambda: W.deep_local_sweep(n=24, layers=60, n_tasks=64, n_terms=32),
                 (("dense_boundary", dict(dense_boundaries=1)), ("pass_kernels", {})))):
            ft = gen()
            fwl = Q.Workload(ft)
            fams[key] = {"workload": desc}
            for pk, opts in plans:
                fams[key][pk] = time_plan(fwl, len(ft), opts)
                if opts.get("dense_boundaries"):
                    fams[key][pk]["boundaries"] = fams[key][pk].pop("dense_choices", None)
            ks = [pk for pk, _ in plans]
            fams[key]["speedup"] = fams[key][ks[0]]["value"] / fams[key][ks[1]]["value"]
            fwl.close()

    if a.dense_qubits > 0 and world == 1:
        line.setdefault("families", {})["dense_tc"] = dense_family(a, eng, stream, peak)

    line["roofline"] = roofline
    # HBM bytes of the whole step against the measured copy bandwidth: the
    # suffix and energy launches' DRAM bytes from the committed ncu captures
    # (algorithmic bytes where the capture no longer matches the source),
    # the boundary's passes algorithmic
    b_suffix = profiled_traffic("sv_batch_kernel", wkey) or batch_alg_bytes
    b_energy = profiled_traffic("energy_kernel", wkey) or energy_alg_bytes
    b_prefix = float(cr.get("prefix_alg_bytes", 0.0))
    step_bytes = b_suffix + b_energy + b_prefix
    line["step_hbm"] = {"bytes": step_bytes, "suffix": b_suffix, "energy": b_energy, "prefix": b_prefix,
                        "achieved_gbs": step_bytes / (ms_max * 1e-3) / 1e9,
                        "frac_of_measured_peak": step_bytes / (ms_max * 1e-3) / 1e9 / peak}
    # every task of the default workload against the oracle's stored energies
    # (tests/golden/make_vqe24_energies.py, complex128)
    gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "vqe24_256_energies.json")
    if (rank == 0 and os.path.exists(gold) and (a.qubits, a.tasks, a.prefix_layers, a.terms) == (24, 256, 20, 200)):
        ref = np.array([t["energy"] for t in json.load(open(gold))["tasks"]])
        err = np.abs(np.array(e_last) - ref)
        rel = err / np.abs(ref)
        coef = tasks[0].terms["coef"]
        e_typ = float(np.sqrt(np.sum(coef ** 2))) * 2.0 ** (-a.qubits / 2)
        normed = err / np.maximum(np.abs(ref), e_typ)
        line["parity_all_tasks"] = {"tasks": int(len(rel)), "max_abs_energy_error": float(err.max()),
                                    "max_rel_energy_error": float(rel.max()),
                                    "median_rel_energy_error": float(np.median(rel)),
                                    "tasks_rel_above_1e-6": int(np.sum(rel > 1e-6)),
                                    "e_typ": e_typ, "max_error_over_max_absE_etyp": float(normed.max()),
                                    "median_error_over_max_absE_etyp": float(np.median(normed)),
                                    "tasks_above_tolerance": int(np.sum(normed > 1e-6)),
                                    "tolerance": "1e-6 of max(|E_ref|, E_typ), E_typ = ||c||_2 2^(-n/2)",
                                    "reference": "oracle energies, complex128, tests/golden/vqe24_256_energies.json"}
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        from oracle import oracle as orc
        orc.build()
        v, dt, cores, e_ref = oracle_tasks_per_s(a, a.cpu_sample_tasks)
        # the timed tasks double as a parity sample of the timed plan
        line["parity_sample"] = [{"task": i, "energy": e_last[i], "oracle_energy": e_ref[i],
                                  "rel_error": abs(e_last[i] - e_ref[i]) / abs(e_ref[i])}
                                 for i in range(len(e_ref))]
        line["cpu_baseline"] = {"value": v, "unit": "tasks/s", "cores": cores, "kind": "oracle",
                                "sample": "%d of %d tasks, per-task rerun from |0> in complex128 "
                                          "(%d gates each incl. shared prefix) + %d-term energy; "
                                          "%.1f s" % (a.cpu_sample_tasks, a.tasks,
                                                      tasks[0].n_gates, a.terms, dt)}
        # the oracle on every workload family, all cores and one core
        if a.cpu_families:
            line["cpu_baselines"] = cpu_baselines(a.tasks)
    if rank == 0:
        print(json.dumps(line), flush=True)
    R.finish(world)
    return 0


def gpu_ms(stream, fn, reps):
    """Mean device time of fn() over reps calls, CUDA events on `stream`.  A
    short device sleep is queued before the start event so that host-side
    preparation inside fn (fusion, uploads) overlaps it and is not timed."""
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        torch.cuda._sleep(50_000_000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def dense_family(a, eng, stream, peak_gbs):
    """Fused dense blocks on the tensor cores (tcgen05, 3xTF32): one random
    5-qubit unitary per pass over an FP32 state larger than L2, in the direct
    and the staged layout and on the CUDA cores; and the 4-layer
    hardware-efficient suffix at 24 qubits as 24 fused blocks against the
    pass kernels that plans use."""
    import torch
    from paper_2609_23664_gb300 import quwarp as Q
    n = a.dense_qubits
    rng = np.random.default_rng(20260923)
    st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    st[0] = 1
    sp = stream.cuda_stream
    out = {"workload": "%d-qubit FP32 state (%.1f GiB, larger than L2): one random 5-qubit unitary per "
                       "pass; 24-qubit 4-layer HEA suffix as fused 5-qubit blocks" % (n, (8 << n) / 2**30)}
    state_bytes = 8 << n
    for key, qubits, kind in (("block_pass", [5, 6, 7, 8, 9], Q.DENSE_TENSOR),
                              ("block_pass_low_qubits", [0, 1, 2, 3, 4], Q.DENSE_TENSOR),
                              ("block_pass_cuda_cores", [5, 6, 7, 8, 9], Q.DENSE_SIMT)):
        z = rng.normal(size=(32, 32)) + 1j * rng.normal(size=(32, 32))
        u, _ = np.linalg.qr(z)
        prog = Q.DenseProgram(eng, W.MODE_SV_FP32, n, engine_kind=kind, nacc=4, block=(qubits, u))
        ms = gpu_ms(stream, lambda: prog.run(st.data_ptr(), sp), 5)
        prog.check()
        prog.close()
        gbs = 2 * state_bytes / (ms * 1e-3) / 1e9
        out[key] = {"qubits": qubits, "engine": "tensor" if kind == Q.DENSE_TENSOR else "cuda_cores",
                    "ms": ms, "gbs": gbs, "frac_of_measured_hbm": gbs / peak_gbs}
    del st
    torch.cuda.empty_cache()
    n2 = 24
    g = W.hea_circuit(np.random.default_rng(24), n2, 4)
    s2 = torch.zeros(1 << n2, dtype=torch.complex64, device="cuda")
    s2[0] = 1
    prog = Q.DenseProgram(eng, W.MODE_SV_FP32, n2, gates=g, kmax=5, engine_kind=Q.DENSE_TENSOR, nacc=4)
    t_dense = gpu_ms(stream, lambda: prog.run(s2.data_ptr(), sp), 5)
    prog.check()
    nb = prog.info()["blocks"]
    prog.close()
    t_pass = gpu_ms(stream, lambda: Q.sv_apply_dev(eng, W.MODE_SV_FP32, n2, s2.data_ptr(), g, stream=sp), 5)
    auto = Q.DenseProgram(eng, W.MODE_SV_FP32, n2, gates=g, kmax=0, engine_kind=Q.DENSE_AUTO)
    cfg = auto.config()
    t_auto = gpu_ms(stream, lambda: auto.run(s2.data_ptr(), sp), 5)
    auto.close()
    out["hea_suffix_24q"] = {"gates": int(len(g)), "dense_blocks": nb, "tensor_blocks_ms": t_dense,
                             "pass_kernels_ms": t_pass, "pass_kernels_speedup": t_dense / t_pass,
                             "autotuned": {"engine": {Q.DENSE_TENSOR: "tensor", Q.DENSE_SIMT: "cuda_cores"}.get(
                                               cfg["engine"], "tensor for >=4-qubit blocks, cuda_cores for the rest"),
                                           "fusion_width": cfg["kmax"], "estimated_ms": cfg["estimated_ms"],
                                           "ms": t_auto}}
    return out


def plan_opts(a):
    return dict(window=a.window, fuse_energy=a.fuse_energy, tile_qubits=a.tile_qubits,
                low_qubits=a.low_qubits)


def main():
    a = parse_args()
    if a.impl == "reference":
        return run_reference(a)
    return run_native(a)


if __name__ == "__main__":
    sys.exit(main())

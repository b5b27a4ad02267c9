"""Host-side tests of the planner and the C ABI (no GPU needed: plans are
built with engine=NULL, and only host entry points are called)."""
import hashlib
import json
import math
import os
import re
import struct
import time

import numpy as np
import pytest

from paper_2609_23664_gb300 import quwarp as Q
from paper_2609_23664_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def header_symbols():
    src = open(os.path.join(ROOT, "include", "quwarp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qw_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    lib = Q.lib()
    syms = header_symbols()
    assert len(syms) >= 30
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(Q.SIGNATURES), set(syms) ^ set(Q.SIGNATURES)


@pytest.mark.parametrize("n", [0, 1, 55, 56, 63, 64, 65, 127, 1000, 4097])
def test_sha256_matches_hashlib(n):
    data = bytes((i * 131 + 7) % 256 for i in range(n))
    assert Q.sha256(data) == hashlib.sha256(data).digest()


def test_fingerprint_is_sha256_of_layout_and_gate_records():
    g = W.ghz_circuit(5)
    fp = Q.fingerprint(5, W.MODE_SV_FP32, g)
    assert fp == hashlib.sha256(struct.pack("<II", 5, W.MODE_SV_FP32) + g.tobytes()).digest()
    assert Q.fingerprint(5, W.MODE_SV_FP64, g) != fp      # layout enters the hash
    g2 = g.copy()
    g2[1]["theta"] = 1e-300                               # bound parameters enter the hash
    assert Q.fingerprint(5, W.MODE_SV_FP32, g2) != fp


def test_reuse_decision_eq2_strict_inequality():
    # (N-1) Cp > Cm + N (Cr + Ch) + delta
    assert Q.reuse_decision(4, 10.0, 1.0, 2.0, 0.0, 5.0)[0]          # 30 > 14
    ok, lhs, rhs = Q.reuse_decision(3, 10.0, 4.0, 2.0, 0.0, 10.0)    # 20 vs 20 -> no
    assert not ok and lhs == 20.0 and rhs == 20.0
    assert Q.reuse_decision(3, 10.0, 4.0, 2.0, 0.0, 9.999)[0]
    assert not Q.reuse_decision(1, 1e9, 0, 0, 0, 0)[0]               # a single task never reuses
    assert not Q.reuse_decision(2, 5.0, 0, 1.0, 2.0, 0.0)[0]          # handoff cost counts N times
    assert Q.reuse_decision(2, 6.1, 0, 1.0, 2.0, 0.0)[0]


BK = {"GPU_SV_FP64": 0, "GPU_SV_FP32": 1, "GPU_TABLEAU": 2, "UNKNOWN": 3}
KIND = {"STATEVECTOR": 0, "TABLEAU": 1}


def test_legality_matrix_table2():
    gold = json.load(open(os.path.join(GOLDEN, "legality_table2.json")))
    prov = hashlib.sha256(b"prefix").digest()
    for row in gold["rows"]:
        exact = 1 if row.get("exactness") == "FORBIDDEN" else 0
        ok, ref = Q.legality_check(KIND[row["kind"]], exact, BK[row["source_backend"]],
                                   row.get("n_qubits", 7), prov, BK[row["target_backend"]], prov)
        if row["outcome"] == "EXACT":
            assert ok and ref["reason"] == "", row
        else:
            assert not ok, row
            assert ref["reason"], row
            assert set(ref) == set(gold["refusal_fields"])
            if "cap" in row["case"]:
                assert ref["reason"] == "UNSUPPORTED_CONVERSION"
    # the paper's example reason for a forbidden statevector handoff
    ok, ref = Q.legality_check(0, 0, BK["GPU_SV_FP32"], 7, prov, BK["GPU_TABLEAU"], prov)
    assert not ok and ref["reason"] == gold["refusal_example_reason"]
    assert ref["source_kind"] == "STATEVECTOR_BOUNDARY_STATE"
    assert ref["target_backend"] == "GPU_TABLEAU"


def test_legality_gate_order_and_provenance():
    prov = hashlib.sha256(b"p").digest()
    other = hashlib.sha256(b"q").digest()
    # exactness is checked before the backend family
    ok, ref = Q.legality_check(0, 1, BK["UNKNOWN"], 3, prov, BK["GPU_SV_FP32"], prov)
    assert ref["reason"] == "NON_EXACT_ARTIFACT"
    ok, ref = Q.legality_check(0, 0, BK["GPU_SV_FP32"], 3, prov, BK["GPU_SV_FP32"], other)
    assert not ok and ref["reason"] == "PROVENANCE_MISMATCH"
    ok, ref = Q.legality_check(0, 0, BK["GPU_SV_FP32"], 3, prov, BK["GPU_SV_FP64"], prov)
    assert not ok and ref["reason"] == "FORBIDDEN_CONVERSION"


def host_plan(tasks, **opts):
    wl = Q.Workload(tasks)
    p = Q.Plan(None, wl, **opts)
    return p, p.explain(), wl


def brute_force_branch_points(gate_lists):
    """Branch points of the prefix trie by brute force: a node at depth d is
    a branch point when the tasks sharing the first d gates continue in at
    least two different ways (or some end there while others continue)."""
    seqs = [tuple(g.tobytes()[i * 24:(i + 1) * 24] for i in range(len(g))) for g in gate_lists]
    points = set()
    for d in range(1, max(len(s) for s in seqs) + 1):
        groups = {}
        for s in seqs:
            if len(s) >= d:
                groups.setdefault(s[:d], []).append(s)
        for pre, members in groups.items():
            if len(members) < 2:
                continue
            nxt = {m[d] if len(m) > d else None for m in members}
            if len(nxt) >= 2 or (len(nxt) == 1 and None in nxt and len(members) >= 2 and
                                 sum(1 for m in members if len(m) == d) >= 2):
                points.add((d, len(members)))
    return points


@pytest.mark.parametrize("seed", range(6))
def test_trie_branch_points_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = 6
    base = W.random_circuit(rng, n, 12)
    tasks, lists = [], []
    for _ in range(7):
        cut = int(rng.integers(0, 13))
        tail = W.random_circuit(rng, n, int(rng.integers(0, 5)))
        if rng.random() < 0.3:
            tail = base[cut:cut + 3].copy()   # equal continuations merge further
        g = W.concat(base[:cut], tail)
        lists.append(g)
        tasks.append(W.Task(mode=W.MODE_SV_FP32, n=n, spans=[g]))
    p, ex, wl = host_plan(tasks, delta_frac=0.0, min_prefix_gates=1)
    got = {(d["branch_gate"], d["tasks_sharing"]) for d in ex["decisions"]}
    want = brute_force_branch_points([g for g in lists if len(g)])
    assert got == want


def test_explain_schema_and_artifact_record():
    tasks = W.vqe12_sweep(n_tasks=4)
    p, ex, wl = host_plan(tasks)
    assert ex["type"] == "QuWARP:ExplainTrace"
    for key in ("tasks", "decisions", "fast_path", "estimated_speedup", "planning_ns", "options"):
        assert key in ex
    d = ex["decisions"][0]
    assert d["decision"] == "REUSE" and d["tasks_sharing"] == 4
    assert d["branch_gate"] == 210
    kinds = {c["boundary"] for c in d["candidates"]}
    assert "LARGEST_COMMON_PREFIX" in kinds and len(d["candidates"]) <= 3
    a = d["artifact"]
    assert a["kind"] == "STATEVECTOR_BOUNDARY_STATE" and a["exactness"] == "EXACT"
    assert a["backend"] == "GPU_SV_FP64" and a["bytes"] == 16 << 12
    prefix = tasks[0].spans[0]
    assert bytes.fromhex(a["provenance_sha256"]) == Q.fingerprint(12, W.MODE_SV_FP64, prefix)
    plans = {x["plan"] for x in d["alternatives"]}
    assert plans == {"BASELINE", "SAME_FAMILY_REUSE", "CROSS_BACKEND_HANDOFF"}


def test_negative_control_takes_the_fast_path():
    tasks = [t for t in W.mixed_planned(n_tasks=40, shared_frac=0.0, n_min=16, n_max=20)]
    t0 = time.perf_counter()
    p, ex, wl = host_plan(tasks)
    assert ex["fast_path"] is True
    assert ex["artifacts"] == 0 and ex["decisions"] == [] and ex["tasks_reusing"] == 0
    assert time.perf_counter() - t0 < 5.0


def test_threshold0_admits_what_the_guard_rejects():
    rng = np.random.default_rng(3)
    n = 24  # four 24-qubit layers take ~9 passes; the 3-gate prefix takes 1
    prefix = W.gates_from_list([(W.OP_H, q, 0) for q in range(3)])
    tasks = [W.Task(mode=W.MODE_SV_FP32, n=n, spans=[prefix, W.hea_circuit(rng, n, 4)])
             for _ in range(2)]
    _, ex_guard, _ = host_plan(tasks)
    _, ex_t0, _ = host_plan(tasks, delta_frac=0.0)
    assert ex_guard["decisions"][0]["decision"] == "ABSTAIN"
    assert ex_t0["decisions"][0]["decision"] == "REUSE"


def test_early_filters():
    tasks = W.vqe12_sweep(n_tasks=2)
    _, ex, _ = host_plan(tasks, min_group=3)
    assert ex["decisions"][0]["decision"] == "ABSTAIN"
    assert ex["decisions"][0]["reason"] == "EARLY_FILTER_GROUP_SIZE"
    _, ex, _ = host_plan(tasks, min_prefix_gates=500)
    assert ex["decisions"][0]["decision"] == "ABSTAIN"


def test_store_budget_admission_on_30_qubit_boundaries():
    rng = np.random.default_rng(4)
    tasks = []
    for _ in range(16):
        pre = W.random_circuit(rng, 30, 300)
        for _ in range(3):
            tasks.append(W.Task(mode=W.MODE_SV_FP32, n=30, spans=[pre, W.random_circuit(rng, 30, 20)]))
    _, ex, _ = host_plan(tasks)
    dec = ex["decisions"]
    reuse = [d for d in dec if d["decision"] == "REUSE"]
    budget = [d for d in dec if d["reason"] == "STORE_BUDGET"]
    assert len(reuse) == int(120e9 // (8 << 30)) and len(budget) == 16 - len(reuse)


def test_mixed_precision_group_refuses_minority():
    rng = np.random.default_rng(5)
    pre = W.random_circuit(rng, 8, 40)
    tasks = [W.Task(mode=W.MODE_SV_FP32 if i < 3 else W.MODE_SV_FP64, n=8,
                    spans=[pre, W.random_circuit(rng, 8, 5)]) for i in range(4)]
    # FP32 boundary (prefix in the tasks' precision): the FP64 task is refused
    _, ex, _ = host_plan(tasks)
    d = ex["decisions"][0]
    assert d["decision"] == "REUSE" and d["reason"] == "REUSE_WITH_REFUSALS"
    assert d["artifact"]["backend"] == "GPU_SV_FP32"
    (r,) = d["refusals"]
    assert r["task"] == 3 and r["reason"] == "FORBIDDEN_CONVERSION" and r["fallback"] == "FULL_RERUN"
    assert ex["tasks_refused"] == 1
    # FP64 boundary rounded once for the FP32 tasks: every task reuses it
    _, ex, _ = host_plan(tasks, prefix_fp64=1)
    d = ex["decisions"][0]
    assert d["decision"] == "REUSE" and d["refusals"] == [] and ex["tasks_reusing"] == 4
    assert d["artifact"]["backend"] == "GPU_SV_FP64" and d["artifact"]["exported_to"] == ["GPU_SV_FP32"]


def test_reuse_off_plans_per_task_replay():
    _, ex, _ = host_plan(W.vqe12_sweep(n_tasks=4), reuse=0)
    assert ex["artifacts"] == 0 and ex["decisions"] == []


def test_tableau_workload_shares_the_prefix_span():
    tasks = W.qec_surface_code_tasks(d=3, shared_rounds=4, task_rounds=2, n_tasks=20, p=0.05)
    _, ex, _ = host_plan(tasks)
    top = min(ex["decisions"], key=lambda d: d["branch_gate"])
    assert top["decision"] == "REUSE"
    assert top["artifact"]["kind"] == "TABLEAU_BOUNDARY_STATE"
    assert top["branch_gate"] >= len(tasks[0].spans[0])


def test_clifford_prefix_is_run_on_the_tableau_and_exported():
    # Table II STAB -> SV: statevector tasks sharing a deep Clifford prefix
    tasks = W.handoff_family(n=16, clifford_depth=200, n_tasks=16)
    p, ex, wl = host_plan(tasks)
    (d,) = ex["decisions"]
    assert d["decision"] == "REUSE"
    art = d["artifact"]
    assert art["kind"] == "TABLEAU_BOUNDARY_STATE" and art["exported_to"] == ["GPU_SV_FP32"]
    assert art["prefix_gates"] == len(tasks[0].spans[0])     # the whole Clifford run
    chosen = [c for c in d["candidates"] if c["chosen"]]
    assert chosen[0]["boundary"] == "TABLEAU_HANDOFF" and chosen[0]["inequality_holds"]
    alt = {a["plan"]: a for a in d["alternatives"]}
    assert alt["CROSS_BACKEND_HANDOFF"]["chosen"]
    assert alt["CROSS_BACKEND_HANDOFF"]["est_ns"] < alt["SAME_FAMILY_REUSE"]["est_ns"]
    # switched off: the same prefix as a statevector boundary
    _, ex0, _ = host_plan(tasks, handoff=0)
    assert ex0["decisions"][0]["artifact"]["kind"] == "STATEVECTOR_BOUNDARY_STATE"
    # a non-Clifford gate inside the shared prefix: no handoff
    t2 = W.handoff_family(n=16, clifford_depth=40, n_tasks=8)
    rot = W.gates_from_list([(W.OP_T, 3, 0)])
    for t in t2:
        t.spans = [t.spans[0][:100], rot, t.spans[0][100:]] + t.spans[1:]
    _, ex2, _ = host_plan(t2)
    assert all(c["boundary"] != "TABLEAU_HANDOFF" or c["cut_gate"] <= 100
               for d in ex2["decisions"] for c in d["candidates"])


def test_noisy_trajectories_reuse_nested_boundaries():
    # multi-level reuse: trajectories share the error-free chain, then
    # sub-groups share mid-segments up to later branch points; every nested
    # boundary continues from its parent's (first_gate = parent's end)
    tasks = W.noisy22_trajectories(n=10, n_gates=120, n_traj=64, p=0.02, shots=4)
    p, ex, wl = host_plan(tasks)
    arts = {d["artifact"]["id"]: d["artifact"] for d in ex["decisions"] if d["artifact"]}
    nested = [a for a in arts.values() if a["parent"] >= 0]
    assert len(arts) >= 3 and nested
    for a in nested:
        assert a["first_gate"] == arts[a["parent"]]["prefix_gates"]
        assert a["prefix_gates"] > a["first_gate"]


def test_full_size_qec_planning_is_fast():
    tasks = W.qec_surface_code_tasks()                  # 449 qubits, 100 + 5 rounds, 4096 tasks
    t0 = time.perf_counter()
    p, ex, wl = host_plan(tasks, pauli_frames=0)
    dt = time.perf_counter() - t0
    assert ex["artifacts"] >= 1 and dt < 10.0, dt


def test_qec_tasks_become_one_pauli_frame_group():
    # the tasks differ only by data errors (Pauli gates): one boundary after
    # the shared rounds, every task a frame over the 5-round reference
    tasks = W.qec_surface_code_tasks(d=5, shared_rounds=6, n_tasks=96, p=0.02)
    p, ex, wl = host_plan(tasks)
    assert ex["artifacts"] == 1 and ex["options"]["pauli_frames"] == 1
    (fr,) = ex["pauli_frames"]
    n_anc = 24
    assert fr["tasks"] == 96 and fr["outcomes_per_task"] == 5 * n_anc
    # reference = the suffix without its Pauli gates: 5 identical rounds
    n_round = len(tasks[0].spans[-1])       # every task ends with a syndrome round
    assert fr["reference_gates"] == 5 * n_round
    # one event per distinct (position, qubit) carrying an error in some task
    keys = set()
    for t in tasks:
        slot = 0
        for sp in t.spans[1:]:
            for g in sp:
                if g["op"] in (W.OP_X, W.OP_Y, W.OP_Z):
                    keys.add((slot, int(g["q0"])))
                else:
                    slot += 1
    assert fr["events"] == len(keys) > 0
    # without frames the trie nests boundaries at the error positions
    _, ex0, _ = host_plan(tasks, pauli_frames=0)
    assert ex0["pauli_frames"] == [] and ex0["artifacts"] >= 1


def test_structural_differences_prevent_frames():
    # a non-Pauli gate that differs between tasks after the boundary
    tasks = W.qec_surface_code_tasks(d=3, shared_rounds=4, n_tasks=6, p=0.0)
    extra = W.gates_from_list([(W.OP_H, 0, 0)])
    tasks[3].spans = tasks[3].spans + [extra]
    p, ex, wl = host_plan(tasks)
    assert all(f["tasks"] < 6 for f in ex["pauli_frames"])


@pytest.mark.parametrize("bad,code", [
    ((W.OP_H, 9, 0), -1), ((W.OP_CNOT, 2, 2), -1), ((99, 0, 0), -1),
    ((W.OP_MEASURE, 0, 0), -9), ((W.OP_RX, 0, 0, float("nan")), -1)])
def test_invalid_gates_are_rejected(bad, code):
    t = W.Task(mode=W.MODE_SV_FP32, n=4, spans=[W.gates_from_list([bad])])
    with pytest.raises(Q.QuwarpError) as ei:
        Q.Workload([t])
    assert ei.value.status == code


def test_invalid_task_fields_are_rejected():
    g = W.ghz_circuit(3)
    with pytest.raises(Q.QuwarpError):
        Q.Workload([W.Task(mode=W.MODE_SV_FP32, n=3, spans=[g], shots=2, uniforms=np.array([0.5, 1.0]))])
    terms = np.zeros(1, dtype=W.TERM_DTYPE)
    terms[0] = (1.0, 1 << 3, 0)
    with pytest.raises(Q.QuwarpError):
        Q.Workload([W.Task(mode=W.MODE_SV_FP32, n=3, spans=[g], terms=terms)])
    with pytest.raises(Q.QuwarpError):
        Q.Workload([W.Task(mode=W.MODE_TABLEAU, n=3, spans=[W.gates_from_list([(W.OP_T, 0, 0)])])])
    with pytest.raises(Q.QuwarpError):
        Q.Workload([W.Task(mode=W.MODE_SV_FP32, n=31, spans=[g])])


def test_execute_without_engine_is_a_state_error():
    p, ex, wl = host_plan(W.vqe12_sweep(n_tasks=2))
    with pytest.raises(Q.QuwarpError) as ei:
        p.execute()
    assert ei.value.status == -6
    with pytest.raises(Q.QuwarpError) as ei:
        p.energy(0)
    assert ei.value.status == -6
    with pytest.raises(Q.QuwarpError) as ei:
        p.wait()
    assert ei.value.status == -6


def test_public_header_is_plain_c():
    # the boundary is a C ABI: the header must compile as C99 on its own
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-x", "c",
                        os.path.join(ROOT, "include", "quwarp.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr

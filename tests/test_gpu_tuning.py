"""The tile-shape tuning record: shapes are timed per (qubits, precision,
arithmetic, gate mix) with a tuning circuit of that mix (hardware-efficient
layers when at most 35 % of the gates act on two qubits, a random entangling
circuit otherwise), and the record moves between engines as JSON.  An engine
that loads the record plans the same waves with the same tiles and times no
shape; the results are bit for bit those of the engine that measured it.
Records of another device, of another library, or with a shape the kernels
cannot run are refused and leave the engine's tuning as it was."""
import json

import numpy as np
import pytest

from paper_2609_23664_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_23664_gb300 import quwarp as Q  # noqa: E402

N = 18


def layered_tasks():
    rng = np.random.default_rng(W.BASE_SEED + 40)
    pre = W.hea_circuit(rng, N, 6)
    terms = W.random_pauli_hamiltonian(rng, N, 8)
    return [W.Task(mode=W.MODE_SV_FP32, n=N, spans=[pre, W.hea_circuit(rng, N, 2)], terms=terms)
            for _ in range(6)]


def entangling_tasks():
    rng = np.random.default_rng(W.BASE_SEED + 41)
    pre = W.random_circuit(rng, N, 300)
    terms = W.random_pauli_hamiltonian(rng, N, 8)
    return [W.Task(mode=W.MODE_SV_FP32, n=N, spans=[pre, W.random_circuit(rng, N, 120)], terms=terms)
            for _ in range(6)]


def run(eng, tasks):
    p = Q.Plan(eng, Q.Workload(tasks))
    p.run()
    tiles = p.cost_record()["wave_tiles"]
    e = [p.energy(i) for i in range(len(tasks))]
    p.close()
    return tiles, e


def keys(rec):
    return {(t["n"], t["mix"], t["arith"], t["fp64"]) for t in rec["tiles"]}


def test_gate_mix_keys_and_transfer():
    a = Q.Engine(0)
    tl_a, el_a = run(a, layered_tasks())
    te_a, ee_a = run(a, entangling_tasks())
    rec = a.tuning()
    assert rec["type"] == "QuWARP:Tuning" and rec["device"]
    # one FP32 compensated entry per gate mix at 18 qubits, each timed once
    assert {(N, 0, 1, 0), (N, 1, 1, 0)} <= keys(rec)
    assert rec["tuning_runs"] >= 2
    runs = rec["tuning_runs"]
    run(a, layered_tasks())
    assert a.tuning()["tuning_runs"] == runs        # cached within the engine
    for t in rec["tiles"]:
        assert t["pass_ns"] > 0 and t["b"] + 2 <= t["k"]

    b = Q.Engine(0)
    # a pretty-printed record loads as well (whitespace outside strings is ignored)
    pretty = json.dumps(rec, indent=2).encode()
    assert Q.lib().qw_engine_tuning_load(b.h, pretty) == 0
    tl_b, el_b = run(b, layered_tasks())
    te_b, ee_b = run(b, entangling_tasks())
    assert b.tuning()["tuning_runs"] == 0           # no shape was timed
    assert keys(b.tuning()) == keys(rec)
    assert (tl_a, te_a) == (tl_b, te_b)
    assert el_a == el_b and ee_a == ee_b            # same tiles, same kernels, same bits
    a.close()
    b.close()


def bad_records(rec):
    r = json.loads(json.dumps(rec))
    r["device"] = "another GPU"
    yield r
    r = json.loads(json.dumps(rec))
    r["type"] = "QuWARP:CostRecord"
    yield r
    for field, v in (("k", 15), ("k", 3), ("b", 12), ("g", 3), ("arith", 2), ("n", 31), ("pass_ns", -1.0)):
        r = json.loads(json.dumps(rec))
        r["tiles"][0][field] = v
        yield r
    r = json.loads(json.dumps(rec))
    r["tiles"][0] = {"n": 18}
    yield r


def test_bad_records_are_refused():
    a = Q.Engine(0)
    run(a, layered_tasks())
    rec = a.tuning()
    assert rec["tiles"]
    before = a.tuning()
    for r in bad_records(rec):
        with pytest.raises(Q.QuwarpError) as ei:
            a.load_tuning(r)
        assert ei.value.status == -1, r                 # QW_ERR_INVALID_ARG
        assert a.tuning() == before
    a.close()

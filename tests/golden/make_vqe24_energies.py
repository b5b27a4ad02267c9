"""Writes vqe24_256_energies.json: the oracle's energy of every task of the
24-qubit VQE sweep (20-layer hardware-efficient prefix, 256 tasks with 1-4
suffix layers, 200-term random Pauli Hamiltonian; the seeded workload that
bench.py times), for the full-size parity test of every task.

Only the oracle computes here.  Every task is the oracle's rerun from
|0...0> through prefix and suffix; the prefix state is computed once and
copied, which performs exactly the same sequence of floating-point
operations as rerunning it per task (the oracle applies gates one after
another, with fixed-order reductions), and the script checks that claim
bit for bit on two tasks against oracle.run_task.

    python tests/golden/make_vqe24_energies.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as orc  # noqa: E402
from paper_2609_23664_gb300 import workloads as W  # noqa: E402

N, LAYERS, TASKS, TERMS = 24, 20, 256, 200
SEED = W.BASE_SEED + 2


def main():
    orc.build()
    tasks = W.vqe24_sweep(seed=SEED, n=N, prefix_layers=LAYERS, n_tasks=TASKS, n_terms=TERMS)
    prefix = tasks[0].spans[0]
    assert all(t.spans[0] is prefix for t in tasks)
    t0 = time.time()
    boundary = orc.sv_run(N, prefix)
    out = []
    for i, t in enumerate(tasks):
        psi = orc.sv_apply(N, boundary.copy(), t.spans[1])
        e, nr, _ = orc.energy(N, psi, t.terms)
        out.append({"task": i, "energy": e, "norm2": nr, "suffix_gates": int(len(t.spans[1]))})
        if i % 16 == 0:
            print("task %d  %.1f s" % (i, time.time() - t0), flush=True)
    for i in (0, TASKS - 1):
        ref = orc.run_task(tasks[i])
        assert ref["energy"] == out[i]["energy"], (i, ref["energy"], out[i]["energy"])
    doc = {"workload": "vqe24_sweep(seed=BASE_SEED+2=%d, n=%d, prefix_layers=%d, n_tasks=%d, n_terms=%d)"
                       % (SEED, N, LAYERS, TASKS, TERMS),
           "written_by": "tests/golden/make_vqe24_energies.py (oracle only, complex128)",
           "tasks": out}
    with open(os.path.join(HERE, "vqe24_256_energies.json"), "w") as f:
        json.dump(doc, f, indent=0)
    print("done in %.1f s" % (time.time() - t0))


if __name__ == "__main__":
    main()

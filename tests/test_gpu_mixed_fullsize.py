"""The mixed planned workload at full size (2000 tasks, 16-30 qubits, FP32,
60 % in groups sharing a prefix, 40 % prefix-free, 120 GB boundary store)
planned and executed on the GPU, then checked task by task against the
oracle: every task with n <= 22 and a seeded sample of four tasks with
26 <= n <= 28 (complex128 states of 1-4 GB on the host), energies within
1e-6 of max(|E_ref|, E_typ) and norms within 1e-6.

The oracle evolves each shared prefix once and applies every task's suffix
to a copy of that state: its statevector loops are independent per
amplitude (no reductions), so this is the per-task run from |0...0> bit for
bit; two tasks are also run from |0...0> to show it."""
import numpy as np
import pytest

from energy_tol import FP32_ENERGY_TOL, energy_error
from oracle import oracle as orc
from paper_2609_23664_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_23664_gb300 import quwarp as Q  # noqa: E402


def _oracle_energies(tasks, idx):
    out = {}
    groups = {}
    for i in idx:
        t = tasks[i]
        key = id(t.spans[0]) if len(t.spans) == 2 else ("free", i)
        groups.setdefault(key, []).append(i)
    for key, members in groups.items():
        t0 = tasks[members[0]]
        if isinstance(key, tuple):
            psi_pre = None
        else:
            psi_pre = orc.sv_run(t0.n, t0.spans[0])
        for i in members:
            t = tasks[i]
            psi = orc.sv_run(t.n, t.gates) if psi_pre is None else orc.sv_apply(t.n, psi_pre.copy(), t.spans[1])
            e, nr, _ = orc.energy(t.n, psi, t.terms)
            out[i] = (e, nr)
        del psi_pre
    return out


def test_mixed2000_against_the_oracle():
    eng = Q.Engine(0, store_budget_bytes=int(120e9))
    tasks = W.mixed_planned()
    wl = Q.Workload(tasks)
    plan = Q.Plan(eng, wl)
    plan.run()
    ex = plan.explain()
    decs = [d["decision"] for d in ex["decisions"]]
    print("artifacts %d, REUSE %d, ABSTAIN %d, REFUSE %d, tasks reusing %d"
          % (ex["artifacts"], decs.count("REUSE"), decs.count("ABSTAIN"), decs.count("REFUSE"),
             ex["tasks_reusing"]))
    got = [plan.energy(i) for i in range(len(tasks))]
    plan.close()
    wl.close()
    eng.close()
    torch.cuda.empty_cache()

    small = [i for i, t in enumerate(tasks) if t.n <= 22]
    rng = np.random.default_rng(W.BASE_SEED + 5)
    big = sorted(int(i) for i in rng.choice([i for i, t in enumerate(tasks) if 26 <= t.n <= 28], 4,
                                            replace=False))
    shared_small = [i for i in small if len(tasks[i].spans) == 2]
    assert len(small) > 800 and shared_small
    ref = _oracle_energies(tasks, small + big)
    # the checkpointed prefix is the run from |0...0> bit for bit
    for i in (shared_small[0], shared_small[-1]):
        r = orc.run_task(tasks[i])
        assert r["energy"] == ref[i][0] and r["norm2"] == ref[i][1], i
    worst, bad = 0.0, []
    for i in small + big:
        t = tasks[i]
        e, nr = got[i]
        err = energy_error(e, ref[i][0], t.terms, t.n)
        worst = max(worst, err)
        if err > FP32_ENERGY_TOL or abs(nr - ref[i][1]) > 1e-6:
            bad.append((i, t.n, err, nr))
    print("%d tasks with n <= 22 and %d with n in [26, 28] (%s): max energy error %.2e of max(|E|, E_typ)"
          % (len(small), len(big), [tasks[i].n for i in big], worst))
    assert not bad, bad[:10]

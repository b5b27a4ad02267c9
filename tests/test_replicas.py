"""Multi-GPU replica path on host processes (gloo, world size 2): each rank
plans its own seeded workload of the family (independent replicas, no data
exchange), the step time is reduced with a max over ranks, and the whole-job
rate counts every rank's tasks over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    from paper_2609_23664_gb300 import replicas as R
    from paper_2609_23664_gb300 import workloads as W
    from paper_2609_23664_gb300 import quwarp as Q
    R.init(world, "gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank)
    tasks = W.vqe24_sweep(seed=R.rank_seed(W.BASE_SEED + 2, rank), n=12, prefix_layers=4, n_tasks=6,
                            n_terms=8)
    ex = Q.Plan(None, Q.Workload(tasks)).explain()       # host-only plan per rank
    R.barrier(world)
    step_ms = 10.0 + 5.0 * rank                          # stand-in step times
    m = R.max_over_ranks(step_ms, world, "cpu")
    rate = R.whole_job_rate(len(tasks), world, m)
    first = tasks[0].spans[-1]["theta"][:4].tolist()
    out.put((rank, m, rate, ex["artifacts"], ex["tasks_reusing"], first))
    R.barrier(world)
    R.finish(world)


def test_two_replicas_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, v0, a0, u0, f0), (r1, m1, v1, a1, u1, f1) = res
    assert m0 == m1 == 15.0                              # max over ranks, same on every rank
    assert v0 == v1 == pytest.approx(2 * 6 / 0.015)      # all ranks' tasks / slowest step
    assert a0 == a1 == 1 and u0 == u1 == 6               # each replica reuses its own prefix
    assert f0 != f1                                      # independent seeded workloads

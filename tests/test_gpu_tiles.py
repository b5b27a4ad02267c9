"""Pass kernels at every tile shape the planner can choose: tile widths 7-14
(FP32) and 7-13 (FP64) with 1-4 contiguous low qubits, on circuits of every
gate type (permutation gates move the tile map, so the stages and the tile
stores run through non-identity maps), through shared prefixes and per-task
suffixes.  Every task's final state is compared with the oracle's
gate-by-gate complex128 state."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2609_23664_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_23664_gb300 import quwarp as Q  # noqa: E402

ALL_OPS = [W.OP_H, W.OP_X, W.OP_Y, W.OP_Z, W.OP_S, W.OP_SDG, W.OP_T, W.OP_TDG, W.OP_RX, W.OP_RY,
           W.OP_RZ, W.OP_PHASE, W.OP_CNOT, W.OP_CZ, W.OP_SWAP, W.OP_CPHASE]
TOL_AMP = {W.MODE_SV_FP64: 1e-12, W.MODE_SV_FP32: 1e-5}


@pytest.fixture(scope="module")
def eng():
    e = Q.Engine(0)
    yield e
    e.close()


def rand_gates(rng, n, k):
    g = []
    for _ in range(k):
        op = ALL_OPS[int(rng.integers(0, len(ALL_OPS)))]
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        g.append((op, a, b, float(rng.uniform(0, 2 * math.pi))))
    return W.gates_from_list(g)


CASES = [(W.MODE_SV_FP32, 7, 1), (W.MODE_SV_FP32, 8, 2), (W.MODE_SV_FP32, 9, 3), (W.MODE_SV_FP32, 11, 4),
         (W.MODE_SV_FP32, 12, 3), (W.MODE_SV_FP32, 13, 2), (W.MODE_SV_FP32, 13, 4), (W.MODE_SV_FP32, 14, 3),
         (W.MODE_SV_FP64, 7, 2), (W.MODE_SV_FP64, 10, 3), (W.MODE_SV_FP64, 12, 4), (W.MODE_SV_FP64, 13, 3)]


@pytest.mark.parametrize("arith", [Q.FP32_COMPENSATED, Q.FP32_PLAIN])
@pytest.mark.parametrize("mode,tile,low", CASES)
def test_forced_tile_shapes_match_the_oracle(eng, mode, tile, low, arith):
    if mode == W.MODE_SV_FP64 and arith == Q.FP32_PLAIN:
        pytest.skip("FP64 passes have one arithmetic")
    n = 16
    rng = np.random.default_rng(4000 + 37 * tile + 5 * low + mode)
    pre = rand_gates(rng, n, 120)
    hea = W.hea_circuit(rng, n, 2)
    tasks = [W.Task(mode=mode, n=n, spans=[pre, hea, rand_gates(rng, n, 40)], want_state=True)
             for _ in range(3)]
    p = Q.Plan(eng, Q.Workload(tasks), tile_qubits=tile, low_qubits=low, fp32_arith=arith)
    p.run()
    # compensated FP32 tiles stop at 13 qubits (their remainder plane)
    cap = 13 if (mode == W.MODE_SV_FP64 or arith == Q.FP32_COMPENSATED) else 14
    assert all(k == min(tile, cap) for k, _ in p.cost_record()["wave_tiles"])
    for i, t in enumerate(tasks):
        got = p.state(i, n, mode == W.MODE_SV_FP64).astype(np.complex128)
        ref = orc.sv_run(n, t.gates)
        err = float(np.max(np.abs(got - ref)))
        assert err <= TOL_AMP[mode], (i, err)
    p.close()

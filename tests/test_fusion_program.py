"""Host fusion of statevector programs (passes, stages, tile maps), checked
on the CPU: the program that the pass kernels would run is exported through
qw_sv_fuse_json, replayed here in complex128 with numpy under the layout
that the header documents (tile loaded in logical order, stages reading and
writing their 32 amplitudes through the stage's tile map, tile stored
through the pass's final map) and compared with the oracle's plain gate-by-
gate statevector.  The replay shares no code with the library or the
oracle."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2609_23664_gb300 import quwarp as Q
from paper_2609_23664_gb300 import workloads as W

ONE_QUBIT = [W.OP_H, W.OP_X, W.OP_Y, W.OP_Z, W.OP_S, W.OP_SDG, W.OP_T, W.OP_TDG,
             W.OP_RX, W.OP_RY, W.OP_RZ, W.OP_PHASE]
TWO_QUBIT = [W.OP_CNOT, W.OP_CZ, W.OP_SWAP, W.OP_CPHASE]


def all_ops_circuit(rng, n, n_gates, perm_weight=0.3):
    lst = []
    for _ in range(n_gates):
        if rng.random() < perm_weight:
            op = int(rng.choice([W.OP_CNOT, W.OP_SWAP, W.OP_X]))
        elif rng.random() < 0.5:
            op = int(rng.choice(ONE_QUBIT))
        else:
            op = int(rng.choice(TWO_QUBIT))
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        lst.append((op, a, b if op in TWO_QUBIT else 0, float(rng.uniform(0, 2 * np.pi))))
    return W.gates_from_list(lst)


def tile_map(m, k):
    """slot of every logical tile index l: XOR of cols[t] over set bits of l, then ^ c"""
    phi = np.full(1 << k, m["c"], dtype=np.int64)
    ls = np.arange(1 << k)
    for t, col in enumerate(m["cols"]):
        phi ^= np.where((ls >> t) & 1, col, 0)
    return phi


def tile_terms(m, ctl_q, tile_base):
    """per tile: XOR of ctl_w[i] over the outside control qubits set in the tile"""
    out = np.zeros(len(tile_base), dtype=np.int64)
    for i, q in enumerate(ctl_q):
        out ^= np.where((tile_base >> q) & 1, m["ctl_w"][i], 0)
    return out


def apply_op(op, A):
    m = op["m"]
    a, b = op["a"], op["b"]
    i = np.arange(32)
    i0 = i[(i >> a) & 1 == 0]
    i1 = i0 | (1 << a)
    x, y = A[..., i0].copy(), A[..., i1].copy()
    kind = op["kind"]
    if kind == "U1":
        A[..., i0] = complex(m[0], m[1]) * x + complex(m[2], m[3]) * y
        A[..., i1] = complex(m[4], m[5]) * x + complex(m[6], m[7]) * y
    elif kind == "D1":
        A[..., i0] = complex(m[0], m[1]) * x
        A[..., i1] = complex(m[2], m[3]) * y
    elif kind == "P1":
        A[..., i1] = complex(m[0], m[1]) * y
    elif kind == "CD":
        both = i[((i >> a) & 1 == 1) & ((i >> b) & 1 == 1)]
        A[..., both] *= complex(m[0], m[1])
    elif kind == "R":
        A[..., i0] = m[0] * x + m[2] * y
        A[..., i1] = m[4] * x + m[6] * y
    elif kind == "RX":
        A[..., i0] = m[0] * x - 1j * m[1] * y
        A[..., i1] = -1j * m[1] * x + m[0] * y
    elif kind == "RP":
        A[..., i0] = m[0] * x + m[1] * y
        A[..., i1] = complex(m[4], m[5]) * (m[2] * x + m[3] * y)
    else:
        raise AssertionError("unknown op kind %s" % kind)


def replay(prog, n):
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    for P in prog["passes"]:
        q = P["q"]
        k = len(q)
        hi = [v for v in range(n) if v not in q]
        ls, ts = np.arange(1 << k), np.arange(1 << len(hi))
        lg = np.zeros(1 << k, dtype=np.int64)
        for t, v in enumerate(q):
            lg |= ((ls >> t) & 1) << v
        tg = np.zeros(1 << len(hi), dtype=np.int64)
        for t, v in enumerate(hi):
            tg |= ((ts >> t) & 1) << v
        G = tg[:, None] | lg[None, :]
        slots = psi[G].copy()  # identity map when the tile is loaded
        rows = np.arange(len(tg))[:, None, None]
        for S in P["stages"]:
            phi = tile_map(S["map"], k)
            pos = S["pos"]
            smask = sum(1 << p for p in pos)
            base = ls[(ls & smask) == 0]
            reg = np.array([sum(((i >> j) & 1) << pos[j] for j in range(5)) for i in range(32)])
            idx = phi[base[:, None] | reg[None, :]][None, :, :] ^ tile_terms(S["map"], P["ctl_q"], tg)[:, None, None]
            A = slots[rows, idx]
            for op in S["ops"]:
                apply_op(op, A)
            slots[rows, idx] = A
        fin = tile_map(P["map"], k)[None, :] ^ tile_terms(P["map"], P["ctl_q"], tg)[:, None]
        psi[G] = slots[np.arange(len(tg))[:, None], fin]
    return psi


def assert_bijective_maps(prog):
    for P in prog["passes"]:
        k = len(P["q"])
        assert not set(P["ctl_q"]) & set(P["q"])
        for m in [P["map"]] + [S["map"] for S in P["stages"]]:
            phi = tile_map(m, k)
            assert np.array_equal(np.sort(phi), np.arange(1 << k))
            assert all(w >> k == 0 for w in m["ctl_w"])


@pytest.mark.parametrize("n,tile,low", [(5, 6, 2), (7, 6, 1), (8, 7, 2), (10, 7, 3), (10, 9, 4), (11, 13, 3)])
@pytest.mark.parametrize("seed", [0, 1])
def test_fused_program_replays_to_the_oracle_state(n, tile, low, seed):
    rng = np.random.default_rng(700 + 31 * n + seed)
    g = all_ops_circuit(rng, n, 160)
    prog = Q.sv_fuse(g, n, tile, low)
    assert_bijective_maps(prog)
    got = replay(prog, n)
    ref = orc.sv_run(n, g)
    assert np.max(np.abs(got - ref)) <= 1e-12


@pytest.mark.parametrize("n,tile,low", [(10, 7, 2), (12, 9, 3)])
def test_hardware_efficient_layers_replay_to_the_oracle_state(n, tile, low):
    rng = np.random.default_rng(900 + n)
    g = W.hea_circuit(rng, n, 4)
    prog = Q.sv_fuse(g, n, tile, low)
    assert_bijective_maps(prog)
    assert np.max(np.abs(replay(prog, n) - orc.sv_run(n, g))) <= 1e-12


def test_permutation_only_program_has_no_stages():
    rng = np.random.default_rng(5)
    n = 9
    lst = []
    for _ in range(60):
        op = int(rng.choice([W.OP_CNOT, W.OP_SWAP, W.OP_X]))
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        lst.append((op, a, b if op != W.OP_X else 0))
    g = W.gates_from_list(lst)
    prog = Q.sv_fuse(g, n, 7, 2)
    assert all(len(P["stages"]) == 0 for P in prog["passes"])
    assert np.max(np.abs(replay(prog, n) - orc.sv_run(n, g))) <= 1e-12


@pytest.mark.parametrize("layers", [1, 2, 3])
def test_chains_across_tiles_replay_to_the_oracle_state(layers):
    """18 qubits in tiles of 9 (3 contiguous): the CNOT chain crosses tile
    boundaries, so passes take CNOTs whose control lies outside the tile"""
    rng = np.random.default_rng(950 + layers)
    n = 18
    g = W.hea_circuit(rng, n, layers)
    prog = Q.sv_fuse(g, n, 9, 3)
    assert any(P["ctl_q"] for P in prog["passes"])
    assert_bijective_maps(prog)
    assert np.max(np.abs(replay(prog, n) - orc.sv_run(n, g))) <= 1e-12


def test_hea_passes_with_outside_controls():
    """24 qubits, tiles of 13 (3 contiguous): CNOTs whose control lies outside
    the tile join the pass, so hardware-efficient layers take 3, 4, 4 and 6
    passes for 1-4 layers (4, 5, 7, 8 when every CNOT needs both qubits in
    the tile)"""
    rng = np.random.default_rng(12)
    got = [len(Q.sv_fuse(W.hea_circuit(rng, 24, L), 24, 13, 3)["passes"]) for L in (1, 2, 3, 4)]
    assert got == [3, 4, 4, 6], got


def test_cnot_chains_hold_no_stage_positions():
    """24 qubits, four hardware-efficient layers, tiles of 13 qubits: one op
    per qubit and layer (RY and RZ fused), every stage carries ops, and the
    CNOT chains add no stages beyond what the rotations need."""
    rng = np.random.default_rng(11)
    n, layers = 24, 4
    prog = Q.sv_fuse(W.hea_circuit(rng, n, layers), n, 13, 3)
    stages = [S for P in prog["passes"] for S in P["stages"]]
    n_ops = sum(len(S["ops"]) for S in stages)
    assert n_ops == n * layers
    assert all(len(S["ops"]) >= 1 for S in stages)
    assert len(stages) <= 24  # 96 ops, at most 5 per stage: at least 20
    assert_bijective_maps(prog)


@pytest.mark.parametrize("args", [(4, 6, 2), (8, 5, 2), (8, 15, 2), (8, 7, 0), (8, 7, 6)])
def test_invalid_fusion_arguments_are_errors(args):
    n, tile, low = args
    g = W.gates_from_list([(W.OP_H, 0, 0)])
    with pytest.raises(Q.QuwarpError):
        Q.sv_fuse(g, n, tile, low)

"""Seeded synthetic workload generators.

This module only *describes* inputs: gate lists, Pauli Hamiltonians, noise
draws, sampling uniforms and the random bits a measurement consumes when its
outcome is not fixed by the state.  It contains none of the simulation
arithmetic, so both the CPU oracle and the GPU engine consume what it emits
without sharing any computation.

Workload shapes follow the workload families of the paper (Sec. V, Table III):
VQE sweeps under one hardware-efficient ansatz (vqe_real / param_sweep),
noisy multishot sampling (noisy_multishot), QEC syndrome cycles
(qec_repetition) and a prefix-free negative control (no_share), scaled up to
GPU-sized qubit counts.  The exact recipes are stated per generator.

Input format (shared by every consumer, little-endian):
  gate record  = {u32 op, u32 q0, u32 q1, u32 flags, f64 theta}  (24 bytes)
  Pauli term   = {f64 coef, u64 xmask, u64 zmask}                (24 bytes)
    qubit q <-> bit q; X: x=1,z=0; Z: x=0,z=1; Y: x=1,z=1.
  For MEASURE / RESET the `theta` field carries the outcome bit (0.0 or 1.0)
  used when the outcome is not determined by the state.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# ---- operation codes (input format; mirrored by include/quwarp.h) ----------
OP_H, OP_X, OP_Y, OP_Z, OP_S, OP_SDG, OP_T, OP_TDG = 1, 2, 3, 4, 5, 6, 7, 8
OP_RX, OP_RY, OP_RZ, OP_PHASE = 9, 10, 11, 12
OP_CNOT, OP_CZ, OP_SWAP, OP_CPHASE = 20, 21, 22, 23
OP_MEASURE, OP_RESET = 30, 31

ONE_QUBIT_OPS = (OP_H, OP_X, OP_Y, OP_Z, OP_S, OP_SDG, OP_T, OP_TDG,
                 OP_RX, OP_RY, OP_RZ, OP_PHASE, OP_MEASURE, OP_RESET)
TWO_QUBIT_OPS = (OP_CNOT, OP_CZ, OP_SWAP, OP_CPHASE)

FLAG_CHECKPOINT = 1

MODE_SV_FP64, MODE_SV_FP32, MODE_TABLEAU = 0, 1, 2

GATE_DTYPE = np.dtype([("op", "<u4"), ("q0", "<u4"), ("q1", "<u4"),
                       ("flags", "<u4"), ("theta", "<f8")])
TERM_DTYPE = np.dtype([("coef", "<f8"), ("xmask", "<u8"), ("zmask", "<u8")])

BASE_SEED = 20260923


@dataclasses.dataclass
class Task:
    """One task.  Its gate list is the concatenation of `spans`; tasks that
    share a prefix share the same span array (the engine references spans
    instead of copying them)."""
    mode: int
    n: int
    spans: List[np.ndarray]
    terms: Optional[np.ndarray] = None      # TERM_DTYPE[n_terms] (energy)
    uniforms: Optional[np.ndarray] = None   # float64[shots] in [0,1)
    shots: int = 0
    want_state: bool = False

    @property
    def gates(self) -> np.ndarray:
        parts = [s for s in self.spans if len(s)]
        if not parts:
            return np.zeros(0, dtype=GATE_DTYPE)
        if len(parts) == 1:
            return parts[0]
        return concat(*parts)

    @property
    def n_gates(self) -> int:
        return int(sum(len(s) for s in self.spans))


def gates_from_list(lst) -> np.ndarray:
    """[(op, q0, q1, theta[, flags])...] -> GATE_DTYPE array."""
    a = np.zeros(len(lst), dtype=GATE_DTYPE)
    for i, g in enumerate(lst):
        a[i]["op"] = g[0]
        a[i]["q0"] = g[1]
        a[i]["q1"] = g[2] if len(g) > 2 else 0
        a[i]["theta"] = g[3] if len(g) > 3 else 0.0
        a[i]["flags"] = g[4] if len(g) > 4 else 0
    return a


def concat(*parts: np.ndarray) -> np.ndarray:
    return np.concatenate([p for p in parts if p is not None and len(p)]
                          ).astype(GATE_DTYPE) if any(
        p is not None and len(p) for p in parts) else np.zeros(0, GATE_DTYPE)


# ---- building blocks ---------------------------------------------------------

def hea_layer(n: int, thetas_ry, thetas_rz, cnot_chain: bool = True) -> np.ndarray:
    """One hardware-efficient ansatz layer: RY on every qubit, RZ on every
    qubit, then (optionally) a linear CNOT chain (q -> q+1, q = 0..n-2)."""
    g = []
    for q in range(n):
        g.append((OP_RY, q, 0, float(thetas_ry[q])))
    for q in range(n):
        g.append((OP_RZ, q, 0, float(thetas_rz[q])))
    if cnot_chain:
        for q in range(n - 1):
            g.append((OP_CNOT, q, q + 1, 0.0))
    return gates_from_list(g)


def hea_circuit(rng: np.random.Generator, n: int, layers: int,
                cnot_chain: bool = True) -> np.ndarray:
    parts = []
    for _ in range(layers):
        parts.append(hea_layer(n, rng.uniform(0, 2 * math.pi, n),
                               rng.uniform(0, 2 * math.pi, n), cnot_chain))
    return concat(*parts)


def random_pauli_hamiltonian(rng: np.random.Generator, n: int,
                             n_terms: int) -> np.ndarray:
    """Each term: per qubit uniform over {I,X,Y,Z}; coefficient N(0,1)."""
    t = np.zeros(n_terms, dtype=TERM_DTYPE)
    for k in range(n_terms):
        letters = rng.integers(0, 4, n)      # 0=I 1=X 2=Y 3=Z
        xm = 0
        zm = 0
        for q in range(n):
            if letters[q] in (1, 2):
                xm |= 1 << q
            if letters[q] in (2, 3):
                zm |= 1 << q
        t[k]["coef"] = rng.normal()
        t[k]["xmask"] = xm
        t[k]["zmask"] = zm
    return t


def random_circuit(rng: np.random.Generator, n: int, n_gates: int) -> np.ndarray:
    """op uniform over {H, RX, RZ, CNOT, CZ}; 1q qubit uniform; 2q pair uniform
    over ordered distinct pairs; angles U[0, 2pi)."""
    ops = (OP_H, OP_RX, OP_RZ, OP_CNOT, OP_CZ)
    g = []
    for _ in range(n_gates):
        op = ops[int(rng.integers(0, 5))]
        if op in (OP_CNOT, OP_CZ):
            a = int(rng.integers(0, n))
            b = int(rng.integers(0, n - 1))
            if b >= a:
                b += 1
            g.append((op, a, b, 0.0))
        else:
            q = int(rng.integers(0, n))
            th = float(rng.uniform(0, 2 * math.pi)) if op != OP_H else 0.0
            g.append((op, q, 0, th))
    return gates_from_list(g)


def random_clifford_layers(rng: np.random.Generator, n: int, depth: int) -> np.ndarray:
    """`depth` layers: a 1q Clifford uniform over {H, S, SDG, X, Y, Z} on
    every qubit, then CNOT or CZ (equal odds) on a random perfect matching
    of the qubits (one qubit idle when n is odd)."""
    ones = (OP_H, OP_S, OP_SDG, OP_X, OP_Y, OP_Z)
    g = []
    for _ in range(depth):
        for q in range(n):
            g.append((ones[int(rng.integers(0, 6))], q, 0, 0.0))
        perm = rng.permutation(n)
        for i in range(0, n - 1, 2):
            op = OP_CNOT if rng.random() < 0.5 else OP_CZ
            g.append((op, int(perm[i]), int(perm[i + 1]), 0.0))
    return gates_from_list(g)


def handoff_family(seed: int = BASE_SEED + 6, n: int = 16, clifford_depth: int = 200,
                   n_tasks: int = 32, suffix_gates: int = 60, n_terms: int = 40,
                   mode: int = MODE_SV_FP32) -> List[Task]:
    """Statevector tasks sharing a deep all-Clifford prefix (random Clifford
    layers, the stabilizer rounds of an error-correction experiment) followed
    by each task's own non-Clifford suffix (random circuit with rotations),
    each with an energy: the tableau-to-statevector handoff family."""
    rng = np.random.default_rng(seed)
    prefix = random_clifford_layers(rng, n, clifford_depth)
    terms = random_pauli_hamiltonian(rng, n, n_terms)
    tasks = []
    for _ in range(n_tasks):
        suf = random_circuit(rng, n, suffix_gates)
        # the suffix starts with a rotation, so the shared Clifford run ends
        # exactly at the prefix
        rot = gates_from_list([(OP_RY, int(rng.integers(0, n)), 0, float(rng.uniform(0.1, 3.0)))])
        tasks.append(Task(mode=mode, n=n, spans=[prefix, rot, suf], terms=terms))
    return tasks


_PAULI_OPS = (None, OP_X, OP_Y, OP_Z)


def pauli_error_gates(rng: np.random.Generator, g) -> np.ndarray:
    """A uniformly random non-identity Pauli on the support of gate g (3
    choices for 1q, 15 for 2q) as single-qubit Pauli gates."""
    out = []
    if int(g["op"]) in TWO_QUBIT_OPS:
        k = int(rng.integers(1, 16))
        pa, pb = k // 4, k % 4
        if pa:
            out.append((_PAULI_OPS[pa], int(g["q0"]), 0, 0.0))
        if pb:
            out.append((_PAULI_OPS[pb], int(g["q1"]), 0, 0.0))
    else:
        k = int(rng.integers(1, 4))
        out.append((_PAULI_OPS[k], int(g["q0"]), 0, 0.0))
    return gates_from_list(out)


def noisy_spans(rng: np.random.Generator, base: np.ndarray, p: float) -> List[np.ndarray]:
    """After each gate of `base`, with probability p, a random Pauli error
    on its support.  Returned as spans: slices (views) of `base` between
    error insertions, interleaved with the error gates."""
    spans = []
    last = 0
    for i in range(len(base)):
        if rng.random() < p:
            spans.append(base[last:i + 1])
            spans.append(pauli_error_gates(rng, base[i]))
            last = i + 1
    spans.append(base[last:])
    return [s for s in spans if len(s)]


# ---- closed-form circuits used as pins ----------------------------------------

def bell_circuit() -> np.ndarray:
    return gates_from_list([(OP_H, 0, 0), (OP_CNOT, 0, 1)])


def ghz_circuit(n: int) -> np.ndarray:
    g = [(OP_H, 0, 0)]
    for q in range(n - 1):
        g.append((OP_CNOT, q, q + 1))
    return gates_from_list(g)


def basis_state_circuit(n: int, j: int) -> np.ndarray:
    return gates_from_list([(OP_X, q, 0) for q in range(n) if (j >> q) & 1])


def qft_circuit(n: int, with_swaps: bool = True) -> np.ndarray:
    """Textbook QFT from H and controlled phases, most significant qubit
    first, followed by the bit-reversal SWAPs."""
    g = []
    for j in reversed(range(n)):
        g.append((OP_H, j, 0))
        for k in reversed(range(j)):
            g.append((OP_CPHASE, k, j, math.pi / (1 << (j - k))))
    if with_swaps:
        for q in range(n // 2):
            g.append((OP_SWAP, q, n - 1 - q))
    return gates_from_list(g)


# ---- rotated surface code ------------------------------------------------------

@dataclasses.dataclass
class SurfaceCode:
    d: int
    n_data: int
    x_anc: List[int]
    z_anc: List[int]
    # per ancilla: data neighbours in CNOT-step order (None where absent)
    sched: dict
    n: int


def rotated_surface_code(d: int) -> SurfaceCode:
    """Rotated surface code of odd distance d: d*d data qubits at (r, c),
    index r*d + c; one ancilla per face.  Bulk faces (r, c) in [0,d-2]^2 have
    corners (r,c),(r,c+1),(r+1,c),(r+1,c+1); type X when r+c is even.
    Weight-2 boundary faces: X-type on the top/bottom edges, Z-type on the
    left/right edges.  CNOT order: X ancillas NW,NE,SW,SE; Z ancillas
    NW,SW,NE,SE."""
    n_data = d * d
    faces = []
    for r in range(-1, d):
        for c in range(-1, d):
            typ = "X" if (r + c) % 2 == 0 else "Z"
            bulk = 0 <= r <= d - 2 and 0 <= c <= d - 2
            top_bot = (r == -1 or r == d - 1) and 0 <= c <= d - 2
            left_right = (c == -1 or c == d - 1) and 0 <= r <= d - 2
            if bulk or (top_bot and typ == "X") or (left_right and typ == "Z"):
                faces.append((r, c, typ))

    def dq(r, c):
        if 0 <= r < d and 0 <= c < d:
            return r * d + c
        return None

    x_anc, z_anc, sched = [], [], {}
    idx = n_data
    for (r, c, typ) in faces:
        nw, ne, sw, se = dq(r, c), dq(r, c + 1), dq(r + 1, c), dq(r + 1, c + 1)
        order = [nw, ne, sw, se] if typ == "X" else [nw, sw, ne, se]
        sched[idx] = order
        (x_anc if typ == "X" else z_anc).append(idx)
        idx += 1
    return SurfaceCode(d=d, n_data=n_data, x_anc=x_anc, z_anc=z_anc,
                       sched=sched, n=idx)


def syndrome_round(code: SurfaceCode, rng: np.random.Generator) -> np.ndarray:
    """Reset every ancilla, H on X ancillas, four CNOT steps (X ancilla is
    control, Z ancilla is target), H on X ancillas, measure every ancilla.
    Measurement/reset records carry a seeded outcome bit in theta."""
    anc = sorted(code.sched.keys())
    g = []
    for a in anc:
        g.append((OP_RESET, a, 0, float(rng.integers(0, 2))))
    for a in code.x_anc:
        g.append((OP_H, a, 0))
    for step in range(4):
        for a in anc:
            dqb = code.sched[a][step]
            if dqb is None:
                continue
            if a in code.x_anc:
                g.append((OP_CNOT, a, dqb))
            else:
                g.append((OP_CNOT, dqb, a))
    for a in code.x_anc:
        g.append((OP_H, a, 0))
    for a in anc:
        g.append((OP_MEASURE, a, 0, float(rng.integers(0, 2))))
    return gates_from_list(g)


def data_errors(code: SurfaceCode, rng: np.random.Generator, p: float) -> np.ndarray:
    """Each data qubit independently gets X with prob. p and Z with prob. p."""
    g = []
    for q in range(code.n_data):
        if rng.random() < p:
            g.append((OP_X, q, 0))
        if rng.random() < p:
            g.append((OP_Z, q, 0))
    return gates_from_list(g)


# ---- configurations -------------------------------------------------------------

def vqe12_sweep(seed: int = BASE_SEED + 1, n: int = 12, layers: int = 6,
                  n_tasks: int = 16, n_terms: int = 20,
                  mode: int = MODE_SV_FP64) -> List[Task]:
    """VQE sweep: shared HEA prefix of `layers` layers; each task appends one
    RY+RZ layer (no CNOTs) with its own angles; energy of one shared random
    Pauli Hamiltonian."""
    rng = np.random.default_rng(seed)
    prefix = hea_circuit(rng, n, layers)
    ham = random_pauli_hamiltonian(rng, n, n_terms)
    tasks = []
    for _ in range(n_tasks):
        suf = hea_layer(n, rng.uniform(0, 2 * math.pi, n),
                        rng.uniform(0, 2 * math.pi, n), cnot_chain=False)
        tasks.append(Task(mode=mode, n=n, spans=[prefix, suf], terms=ham))
    return tasks


def vqe24_sweep(seed: int = BASE_SEED + 2, n: int = 24, prefix_layers: int = 20,
                  n_tasks: int = 256, max_suffix_layers: int = 4,
                  n_terms: int = 200, mode: int = MODE_SV_FP32) -> List[Task]:
    """Batched VQE sweep: shared HEA prefix; each task adds L ~ U{1..4} full
    HEA layers (RY, RZ, CNOT chain); energy of a shared random Hamiltonian."""
    rng = np.random.default_rng(seed)
    prefix = hea_circuit(rng, n, prefix_layers)
    ham = random_pauli_hamiltonian(rng, n, n_terms)
    tasks = []
    for _ in range(n_tasks):
        L = int(rng.integers(1, max_suffix_layers + 1))
        tasks.append(Task(mode=mode, n=n, spans=[prefix, hea_circuit(rng, n, L)], terms=ham))
    return tasks


def deep_local_sweep(seed: int = BASE_SEED + 7, n: int = 24, layers: int = 60, lo: int = 8, width: int = 5,
                     n_tasks: int = 64, n_terms: int = 32, mode: int = MODE_SV_FP32) -> List[Task]:
    """A sweep whose shared prefix is deep but local: H on every qubit, then
    `layers` layers of RY, a CNOT chain and RZ confined to qubits
    lo..lo+width-1; each task adds an RY layer on every qubit and takes the
    energy of a shared random Hamiltonian."""
    rng = np.random.default_rng(seed)
    ops = [(OP_H, q, 0) for q in range(n)]
    qs = range(lo, lo + width)
    for _ in range(layers):
        ops += [(OP_RY, q, 0, float(rng.uniform(0, 2 * np.pi))) for q in qs]
        ops += [(OP_CNOT, q, q + 1) for q in range(lo, lo + width - 1)]
        ops += [(OP_RZ, q, 0, float(rng.uniform(0, 2 * np.pi))) for q in qs]
    prefix = gates_from_list(ops)
    ham = random_pauli_hamiltonian(rng, n, n_terms)
    tasks = []
    for _ in range(n_tasks):
        suf = gates_from_list([(OP_RY, q, 0, float(rng.uniform(0, 2 * np.pi))) for q in range(n)])
        tasks.append(Task(mode=mode, n=n, spans=[prefix, suf], terms=ham))
    return tasks


def costly_prefix_groups(seed: int = BASE_SEED + 8, n: int = 20, groups: int = 8, group_size: int = 4,
                         prefix_gates: int = 240, suffix_gates: int = 8000, suffix_qubits: int = 12,
                         n_terms: int = 16, mode: int = MODE_SV_FP32) -> List[Task]:
    """Groups of tasks whose gates differ in cost: each group shares a
    prefix of `prefix_gates` rotations (RX, RY or RZ, uniform, angles
    U[0, 2pi)) on uniform qubits, and every task adds a network of
    `suffix_gates` CNOTs on uniform pairs of qubits 0..suffix_qubits-1; one
    random Hamiltonian per group.  A rotation is arithmetic on every
    amplitude, a CNOT only relabels amplitudes, so the prefix is the costly
    part although it has far fewer gates."""
    rng = np.random.default_rng(seed)
    tasks = []
    for _ in range(groups):
        pre = gates_from_list([(int(rng.choice([OP_RX, OP_RY, OP_RZ])), int(rng.integers(0, n)), 0,
                                float(rng.uniform(0, 2 * np.pi))) for _ in range(prefix_gates)])
        ham = random_pauli_hamiltonian(rng, n, n_terms)
        for _ in range(group_size):
            g = [(OP_CNOT, int(a), int(b), 0.0)
                 for a, b in (rng.choice(suffix_qubits, 2, replace=False) for _ in range(suffix_gates))]
            tasks.append(Task(mode=mode, n=n, spans=[pre, gates_from_list(g)], terms=ham))
    return tasks


def noisy22_trajectories(seed: int = BASE_SEED + 3, n: int = 22, n_gates: int = 400,
                    n_traj: int = 1024, p: float = 1e-3, shots: int = 100,
                    mode: int = MODE_SV_FP32) -> List[Task]:
    """Noisy multishot: one random circuit; each trajectory inserts Pauli
    errors after gates with probability p; `shots` uniforms per trajectory."""
    rng = np.random.default_rng(seed)
    base = random_circuit(rng, n, n_gates)
    tasks = []
    for _ in range(n_traj):
        spans = noisy_spans(rng, base, p)
        u = rng.random(shots)
        tasks.append(Task(mode=mode, n=n, spans=spans, uniforms=u, shots=shots))
    return tasks


def qec_surface_code_tasks(seed: int = BASE_SEED + 4, d: int = 15, shared_rounds: int = 100,
                task_rounds: int = 5, n_tasks: int = 4096,
                p: float = 1e-3) -> List[Task]:
    """Stabilizer-mode QEC: `shared_rounds` noiseless syndrome rounds form the
    shared prefix; each task then runs `task_rounds` rounds, each preceded by
    seeded X/Z data errors."""
    rng = np.random.default_rng(seed)
    code = rotated_surface_code(d)
    prefix = concat(*[syndrome_round(code, rng) for _ in range(shared_rounds)])
    # every measurement after the first round is determined by the state, so
    # one round record (with its outcome bits) serves all later rounds
    round_g = syndrome_round(code, rng)
    tasks = []
    for _ in range(n_tasks):
        spans = [prefix]
        for _ in range(task_rounds):
            spans.append(data_errors(code, rng, p))
            spans.append(round_g)
        tasks.append(Task(mode=MODE_TABLEAU, n=code.n, spans=[s for s in spans if len(s)]))
    return tasks


def mixed_planned(seed: int = BASE_SEED + 5, n_tasks: int = 2000,
                  shared_frac: float = 0.6, n_min: int = 16, n_max: int = 30,
                  group_min: int = 2, group_max: int = 64,
                  prefix_len=(50, 500), suffix_len=(10, 100),
                  free_len=(50, 550), n_terms: int = 8,
                  mode: int = MODE_SV_FP32) -> List[Task]:
    """Mixed planned workload: `shared_frac` of the tasks come in groups of
    U{group_min..group_max} tasks sharing a random prefix (gate set of the
    noisy family), each with its own random suffix; the rest are prefix-free
    random circuits (negative control).  Each task carries its own small
    random Hamiltonian."""
    rng = np.random.default_rng(seed)
    n_shared = int(round(n_tasks * shared_frac))
    tasks = []
    while len(tasks) < n_shared:
        gsz = min(int(rng.integers(group_min, group_max + 1)), n_shared - len(tasks))
        if gsz < 2 and tasks:
            gsz = 2
        n = int(rng.integers(n_min, n_max + 1))
        pre = random_circuit(rng, n, int(rng.integers(prefix_len[0], prefix_len[1] + 1)))
        for _ in range(gsz):
            suf = random_circuit(rng, n, int(rng.integers(suffix_len[0], suffix_len[1] + 1)))
            tasks.append(Task(mode=mode, n=n, spans=[pre, suf],
                              terms=random_pauli_hamiltonian(rng, n, n_terms)))
    tasks = tasks[:n_shared]
    for _ in range(n_tasks - n_shared):
        n = int(rng.integers(n_min, n_max + 1))
        g = random_circuit(rng, n, int(rng.integers(free_len[0], free_len[1] + 1)))
        tasks.append(Task(mode=mode, n=n, spans=[g],
                          terms=random_pauli_hamiltonian(rng, n, n_terms)))
    return tasks

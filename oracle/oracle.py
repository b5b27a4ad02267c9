"""Python access to the CPU oracle (qw_oracle.c).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py; never by the product package.  It shares no code
with the GPU path: the only thing both sides consume is the seeded workload
description from paper_2609_23664_gb300.workloads.

Every task is evaluated independently from |0...0> (the per-task rerun the
paper uses as its fallback and as its denominator, Sec. IV-B and Sec. V-E
baseline 1), so reuse results can be checked against it directly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qw_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libqw_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile qw_oracle.c with gcc (OpenMP parallel loops, no other flags
    that change arithmetic: no -ffast-math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-std=c11", "-shared", "-fPIC",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            c_p, sz, i, d = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_double
            L.orc_sv_zero.argtypes = [i, c_p]
            L.orc_sv_apply.argtypes = [i, c_p, c_p, sz]
            L.orc_sv_apply.restype = i
            L.orc_sv_norm2.argtypes = [i, c_p]
            L.orc_sv_norm2.restype = d
            L.orc_sv_pauli_expect.argtypes = [i, c_p, ctypes.c_uint64, ctypes.c_uint64,
                                              ctypes.POINTER(d), ctypes.POINTER(d)]
            L.orc_sv_energy.argtypes = [i, c_p, c_p, sz, ctypes.POINTER(d),
                                        ctypes.POINTER(d), c_p]
            L.orc_sv_energy.restype = i
            L.orc_sv_sample.argtypes = [i, c_p, c_p, sz, c_p]
            L.orc_sv_sample.restype = i
            L.orc_tab_run.argtypes = [i, c_p, sz, c_p, sz, ctypes.POINTER(sz), c_p, c_p, c_p]
            L.orc_tab_run.restype = i
            L.orc_tab_run_from.argtypes = [i, c_p, c_p, c_p, c_p, sz, c_p, sz, ctypes.POINTER(sz), c_p, c_p, c_p]
            L.orc_tab_run_from.restype = i
            L.orc_num_threads.restype = i
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def sv_zero(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    lib().orc_sv_zero(n, _ptr(psi))
    return psi


def sv_apply(n: int, psi: np.ndarray, gates: np.ndarray) -> np.ndarray:
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == 1 << n
    g = np.ascontiguousarray(gates)
    rc = lib().orc_sv_apply(n, _ptr(psi), _ptr(g), len(g))
    if rc != 0:
        raise ValueError("oracle rejected the gate list (rc=%d)" % rc)
    return psi


def sv_run(n: int, gates: np.ndarray) -> np.ndarray:
    return sv_apply(n, sv_zero(n), gates)


def apply_matrix(n: int, psi: np.ndarray, qubits, u: np.ndarray) -> np.ndarray:
    """A k-qubit operator on the listed qubits, by definition: bit j of the
    block-local index is qubits[j], and for every basis index x
        psi'[x] = sum_p u[loc(x), p] * psi[(x with its block bits set to p)],
    where loc(x) is x's own block-local index.  This is how any gate (or
    product of gates) on k qubits acts on the statevector that the
    statevector backend evolves (Sec. III-A "Execution on the bounded Qrack
    surface"); it is the reference for fused dense blocks.  Returns a new
    array (complex128)."""
    psi = np.asarray(psi, dtype=np.complex128)
    u = np.asarray(u, dtype=np.complex128)
    k = len(qubits)
    assert u.shape == (1 << k, 1 << k) and psi.size == 1 << n
    x = np.arange(1 << n, dtype=np.int64)
    mask = 0
    loc = np.zeros_like(x)
    for j, q in enumerate(qubits):
        loc |= ((x >> q) & 1) << j
        mask |= 1 << q
    base = x & ~mask
    out = np.zeros_like(psi)
    for p in range(1 << k):
        off = sum(((p >> j) & 1) << q for j, q in enumerate(qubits))
        out += u[loc, p] * psi[base | off]
    return out


def norm2(n: int, psi: np.ndarray) -> float:
    return float(lib().orc_sv_norm2(n, _ptr(psi)))


def pauli_expect(n: int, psi: np.ndarray, xmask: int, zmask: int) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().orc_sv_pauli_expect(n, _ptr(psi), xmask, zmask, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def energy(n: int, psi: np.ndarray, terms: np.ndarray):
    """-> (energy, norm2, per-term <P_k>)"""
    t = np.ascontiguousarray(terms)
    per = np.zeros(max(len(t), 1), dtype=np.float64)
    e, nr = ctypes.c_double(), ctypes.c_double()
    rc = lib().orc_sv_energy(n, _ptr(psi), _ptr(t), len(t), ctypes.byref(e),
                             ctypes.byref(nr), _ptr(per))
    if rc != 0:
        raise MemoryError("oracle energy failed")
    return e.value, nr.value, per[:len(t)]


def sample(n: int, psi: np.ndarray, uniforms: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    out = np.zeros(len(u), dtype=np.uint64)
    rc = lib().orc_sv_sample(n, _ptr(psi), _ptr(u), len(u), _ptr(out))
    if rc != 0:
        raise MemoryError("oracle sampling failed")
    return out


def tab_run(n: int, gates: np.ndarray, want_tableau: bool = False):
    """-> outcomes (uint8 per MEASURE) [, (x, z, r) final tableau rows]"""
    g = np.ascontiguousarray(gates)
    n_meas = int(np.count_nonzero(g["op"] == 30))
    out = np.zeros(max(n_meas, 1), dtype=np.uint8)
    n_out = ctypes.c_size_t()
    if want_tableau:
        x = np.zeros((2 * n, n), dtype=np.uint8)
        z = np.zeros((2 * n, n), dtype=np.uint8)
        r = np.zeros(2 * n, dtype=np.uint8)
        rc = lib().orc_tab_run(n, _ptr(g), len(g), _ptr(out), len(out), ctypes.byref(n_out),
                               _ptr(x), _ptr(z), _ptr(r))
    else:
        rc = lib().orc_tab_run(n, _ptr(g), len(g), _ptr(out), len(out), ctypes.byref(n_out),
                               None, None, None)
    if rc != 0:
        raise ValueError("oracle tableau run failed (rc=%d)" % rc)
    outs = out[:n_out.value].copy()
    return (outs, (x, z, r)) if want_tableau else outs


def tab_run_from(n: int, tableau, gates: np.ndarray, want_tableau: bool = False):
    """tab_run continued from a tableau (x, z, r) that tab_run exported."""
    x0, z0, r0 = (np.ascontiguousarray(a, dtype=np.uint8) for a in tableau)
    g = np.ascontiguousarray(gates)
    n_meas = int(np.count_nonzero(g["op"] == 30))
    out = np.zeros(max(n_meas, 1), dtype=np.uint8)
    n_out = ctypes.c_size_t()
    if want_tableau:
        x = np.zeros((2 * n, n), dtype=np.uint8)
        z = np.zeros((2 * n, n), dtype=np.uint8)
        r = np.zeros(2 * n, dtype=np.uint8)
        ptrs = (_ptr(x), _ptr(z), _ptr(r))
    else:
        ptrs = (None, None, None)
    rc = lib().orc_tab_run_from(n, _ptr(x0), _ptr(z0), _ptr(r0), _ptr(g), len(g), _ptr(out), len(out),
                                ctypes.byref(n_out), *ptrs)
    if rc != 0:
        raise ValueError("oracle tableau run failed (rc=%d)" % rc)
    outs = out[:n_out.value].copy()
    return (outs, (x, z, r)) if want_tableau else outs


def run_task(task, want_state: bool = False) -> dict:
    """Evaluates one workload task from scratch (no reuse)."""
    res = {}
    if task.mode == 2:
        res["syndrome"] = tab_run(task.n, task.gates)
        return res
    psi = sv_run(task.n, task.gates)
    if want_state:
        res["state"] = psi
    if task.terms is not None and len(task.terms):
        e, nr, per = energy(task.n, psi, task.terms)
        res["energy"], res["norm2"], res["per_term"] = e, nr, per
    else:
        res["norm2"] = norm2(task.n, psi)
    if task.shots:
        res["samples"] = sample(task.n, psi, task.uniforms[:task.shots])
    return res

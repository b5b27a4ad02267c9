"""Thin ctypes binding of libquwarp.so (include/quwarp.h).

Argument marshalling only: every step of planning and execution runs in the
native library (host planner in C++, kernels on sm_103a).  There is no
Python or CPU fallback: if the library cannot be built or loaded, or no GPU
is present, the calls raise QuwarpError.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import threading
from typing import List, Optional, Sequence

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libquwarp.so")
_lock = threading.Lock()
_lib = None

QW_OK = 0
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "BUDGET", -4: "CUDA", -5: "DEVICE_TIMEOUT",
          -6: "STATE", -7: "BUFFER_TOO_SMALL", -8: "NOT_FOUND", -9: "UNSUPPORTED"}
COST_ANALYTIC, COST_MLP = 0, 1
FP32_AUTO, FP32_PLAIN, FP32_COMPENSATED = 0, 1, 2
TASK_KEEP_STATE = 1
MLP_IN, MLP_HID = 12, 64
MLP_PARAMS = MLP_IN * MLP_HID + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_HID + 1


class QuwarpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, msg))
        self.status = status


class qw_gate_span(C.Structure):
    _fields_ = [("gates", C.c_void_p), ("n_gates", C.c_uint64)]


class qw_task(C.Structure):
    _fields_ = [("mode", C.c_uint32), ("n_qubits", C.c_uint32), ("spans", C.POINTER(qw_gate_span)),
                ("n_spans", C.c_uint32), ("flags", C.c_uint32), ("terms", C.c_void_p),
                ("n_terms", C.c_uint64), ("uniforms", C.c_void_p), ("shots", C.c_uint32),
                ("reserved", C.c_uint32)]


class qw_engine_opts(C.Structure):
    _fields_ = [("device", C.c_int32), ("reserved", C.c_uint32), ("store_budget_bytes", C.c_uint64),
                ("task_budget_bytes", C.c_uint64), ("hbm_gbs", C.c_double)]


class qw_plan_opts(C.Structure):
    _fields_ = [("reuse", C.c_int32), ("batched", C.c_int32), ("legality", C.c_int32),
                ("cost_model", C.c_int32), ("delta_frac", C.c_double), ("min_group", C.c_uint32),
                ("min_prefix_gates", C.c_uint32), ("min_prefix_cost_ns", C.c_double),
                ("tile_qubits", C.c_uint32), ("low_qubits", C.c_uint32), ("window", C.c_uint32),
                ("use_graph", C.c_int32), ("fault_injection", C.c_int32),
                ("fuse_energy", C.c_int32), ("pauli_frames", C.c_int32), ("handoff", C.c_int32),
                ("prefix_fp64", C.c_int32), ("dense_boundaries", C.c_int32),
                ("fp32_arith", C.c_int32)]


class qw_cost_tuple(C.Structure):
    _fields_ = [("n_tasks", C.c_double), ("c_prefix", C.c_double), ("c_materialize", C.c_double),
                ("c_reload", C.c_double), ("c_handoff", C.c_double), ("delta", C.c_double)]


class qw_artifact_desc(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("exactness", C.c_uint32), ("backend", C.c_uint32),
                ("n_qubits", C.c_uint32), ("provenance", C.c_uint8 * 32)]


class qw_refusal(C.Structure):
    _fields_ = [("reason", C.c_char * 48), ("detail", C.c_char * 160), ("source_kind", C.c_char * 40),
                ("target_kind", C.c_char * 40), ("source_backend", C.c_char * 32),
                ("target_backend", C.c_char * 32)]


# every entry point declared in include/quwarp.h: name -> (restype, argtypes)
_vp, _u32, _u64, _i32, _d, _f, _sz = (C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32, C.c_double,
                                      C.c_float, C.c_size_t)
_st = C.c_int32
SIGNATURES = {
    "qw_engine_create": (_st, [_vp, _vp]),
    "qw_engine_destroy": (None, [_vp]),
    "qw_engine_info": (_st, [_vp, _vp, _vp, _vp]),
    "qw_engine_probe_l2": (_st, [_vp, _vp]),
    "qw_engine_tuning_json": (_st, [_vp, _vp, _sz, _vp]),
    "qw_engine_tuning_load": (_st, [_vp, C.c_char_p]),
    "qw_last_error": (C.c_char_p, []),
    "qw_workload_create": (_st, [_vp]),
    "qw_workload_add_task": (_st, [_vp, _vp, _vp]),
    "qw_workload_destroy": (None, [_vp]),
    "qw_plan_opts_default": (None, [_vp]),
    "qw_plan_create": (_st, [_vp, _vp, _vp, _vp]),
    "qw_plan_destroy": (None, [_vp]),
    "qw_execute": (_st, [_vp, _vp]),
    "qw_wait": (_st, [_vp]),
    "qw_get_energy": (_st, [_vp, _u64, _vp, _vp]),
    "qw_get_samples": (_st, [_vp, _u64, _vp, _sz, _vp]),
    "qw_get_syndrome": (_st, [_vp, _u64, _vp, _sz, _vp]),
    "qw_get_state": (_st, [_vp, _u64, _vp, _sz]),
    "qw_get_stabilizers": (_st, [_vp, _u64, _vp, _vp, _vp, _sz]),
    "qw_explain_json": (_st, [_vp, _vp, _sz, _vp]),
    "qw_cost_record_json": (_st, [_vp, _vp, _sz, _vp]),
    "qw_sha256": (_st, [_vp, _sz, _vp]),
    "qw_fingerprint": (_st, [_u32, _u32, _vp, _u64, _vp]),
    "qw_reuse_decision": (_st, [_vp, _vp, _vp, _vp]),
    "qw_legality_check": (_st, [_vp, _u32, _vp, _vp, _vp]),
    "qw_mlp_forward_dev": (_st, [_vp, _vp, _vp, _u32, _vp]),
    "qw_mlp_loss_grad_dev": (_st, [_vp, _vp, _vp, _u32, _vp, _vp, _vp]),
    "qw_mlp_adam_dev": (_st, [_vp, _vp, _vp, _vp, _u32, _u32, _f, _f, _f, _f, _vp]),
    "qw_costmodel_train": (_st, [_vp, _vp, _vp, _u64, _u32, _u32, _f, _u64, _vp]),
    "qw_costmodel_predict": (_st, [_vp, _vp, _u64, _vp]),
    "qw_costmodel_get": (_st, [_vp, _vp, _vp, _vp]),
    "qw_costmodel_set": (_st, [_vp, _vp, _vp, _vp]),
    "qw_costmodel_probe": (_st, [_vp, _vp, _vp, _vp, _vp, _u64, _vp]),
    "qw_costmodel_features": (_st, [_vp, _vp, _u64, _u64, _u64, _u32, _vp]),
    "qw_sv_apply_dev": (_st, [_vp, _u32, _u32, _vp, _vp, _u64, _vp, _vp]),
    "qw_sv_energy_dev": (_st, [_vp, _u32, _u32, _vp, _vp, _u64, _vp, _vp, _vp]),
    "qw_sv_sample_dev": (_st, [_vp, _u32, _u32, _vp, _vp, _u32, _vp, _vp]),
    "qw_sv_energy_noalloc_dev": (_st, [_u32, _u32, _vp, _vp, _u64, _vp, _vp]),
    "qw_dense_fuse": (_st, [_vp, _u64, _u32, _u32, _vp, _vp, _vp, _u64, _vp]),
    "qw_sv_fuse_json": (_st, [_vp, _u64, _u32, _u32, _u32, _vp, _sz, _vp]),
    "qw_dense_prog_create": (_st, [_vp, _u32, _u32, _vp, _u64, _u32, _u32, _u32, _vp]),
    "qw_dense_prog_create_block": (_st, [_vp, _u32, _u32, _vp, _u32, _vp, _u32, _u32, _vp]),
    "qw_dense_prog_info": (_st, [_vp, _vp, _vp]),
    "qw_dense_prog_config": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "qw_dense_prog_run": (_st, [_vp, _vp, _vp]),
    "qw_dense_prog_check": (_st, [_vp]),
    "qw_dense_prog_destroy": (None, [_vp]),
}

DENSE_TENSOR, DENSE_SIMT, DENSE_AUTO = 0, 1, 2


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Loads libquwarp.so (building it in-tree first if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                from . import _build
                _build.build()
            L = C.CDLL(_LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(st: int):
    if st != QW_OK:
        msg = lib().qw_last_error()
        raise QuwarpError(st, msg.decode() if msg else "")


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


class Engine:
    def __init__(self, device: int = 0, store_budget_bytes: int = 0, task_budget_bytes: int = 0,
                 hbm_gbs: float = 0.0):
        o = qw_engine_opts(device, 0, store_budget_bytes, task_budget_bytes, hbm_gbs)
        h = C.c_void_p()
        _check(lib().qw_engine_create(C.byref(o), C.byref(h)))
        self.h = h

    def info(self):
        bw, sm, l2 = C.c_double(), C.c_int32(), C.c_uint64()
        _check(lib().qw_engine_info(self.h, C.byref(bw), C.byref(sm), C.byref(l2)))
        return {"hbm_gbs": bw.value, "sm_count": sm.value, "l2_bytes": l2.value}

    def probe_l2(self) -> float:
        """Measured L2 read bandwidth (GB/s) for the energy step's access pattern."""
        v = C.c_double()
        _check(lib().qw_engine_probe_l2(self.h, C.byref(v)))
        return v.value

    def tuning(self) -> dict:
        """The engine's tile-shape tuning (see qw_engine_tuning_json)."""
        need = C.c_size_t()
        lib().qw_engine_tuning_json(self.h, None, 0, C.byref(need))
        buf = C.create_string_buffer(need.value)
        _check(lib().qw_engine_tuning_json(self.h, buf, need.value, C.byref(need)))
        return json.loads(buf.value.decode())

    def load_tuning(self, record: dict):
        """Adds a tuning record written on the same GPU model."""
        _check(lib().qw_engine_tuning_load(self.h, json.dumps(record, separators=(",", ":")).encode()))

    def close(self):
        if getattr(self, "h", None):
            lib().qw_engine_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # learned cost model
    def costmodel_train(self, features: np.ndarray, targets: np.ndarray, epochs: int = 30,
                        batch: int = 256, lr: float = 1e-3, seed: int = 1) -> float:
        f = np.ascontiguousarray(features, dtype=np.float32)
        t = np.ascontiguousarray(targets, dtype=np.float32)
        loss = C.c_float()
        _check(lib().qw_costmodel_train(self.h, _p(f), _p(t), len(t), epochs, batch, lr, seed,
                                        C.byref(loss)))
        return loss.value

    def costmodel_predict(self, features: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(features, dtype=np.float32)
        out = np.zeros(len(f), dtype=np.float32)
        _check(lib().qw_costmodel_predict(self.h, _p(f), len(f), _p(out)))
        return out

    def costmodel_get(self):
        p = np.zeros(MLP_PARAMS, np.float32)
        m = np.zeros(MLP_IN, np.float32)
        s = np.zeros(MLP_IN, np.float32)
        _check(lib().qw_costmodel_get(self.h, _p(p), _p(m), _p(s)))
        return p, m, s

    def costmodel_set(self, params, mean, scale):
        p = np.ascontiguousarray(params, np.float32)
        m = np.ascontiguousarray(mean, np.float32)
        s = np.ascontiguousarray(scale, np.float32)
        _check(lib().qw_costmodel_set(self.h, _p(p), _p(m), _p(s)))

    def costmodel_probe(self, workload: "Workload", cap: int):
        """-> (features [rows, 12], measured log2 ns, analytic-model log2 ns)"""
        f = np.zeros((cap, MLP_IN), np.float32)
        t = np.zeros(cap, np.float32)
        a = np.zeros(cap, np.float32)
        n = C.c_uint64()
        _check(lib().qw_costmodel_probe(self.h, workload.h, _p(f), _p(t), _p(a), cap, C.byref(n)))
        return f[:n.value], t[:n.value], a[:n.value]


class Workload:
    """Tasks reference their gate spans; the arrays are kept alive here."""

    def __init__(self, tasks: Sequence[W.Task] = ()):
        h = C.c_void_p()
        _check(lib().qw_workload_create(C.byref(h)))
        self.h = h
        self._keep: List[object] = []
        self.n = 0
        for t in tasks:
            self.add(t)

    def add(self, t: W.Task) -> int:
        spans = [np.ascontiguousarray(s, dtype=W.GATE_DTYPE) for s in t.spans if len(s)]
        arr = (qw_gate_span * max(1, len(spans)))()
        for i, s in enumerate(spans):
            arr[i] = qw_gate_span(s.ctypes.data, len(s))
        terms = None if t.terms is None else np.ascontiguousarray(t.terms, dtype=W.TERM_DTYPE)
        uni = None if not t.shots else np.ascontiguousarray(t.uniforms[:t.shots], dtype=np.float64)
        flags = TASK_KEEP_STATE if t.want_state else 0
        task = qw_task(t.mode, t.n, arr, len(spans), flags, _p(terms),
                       0 if terms is None else len(terms), _p(uni), t.shots, 0)
        tid = C.c_uint64()
        _check(lib().qw_workload_add_task(self.h, C.byref(task), C.byref(tid)))
        self._keep.append(spans)
        self.n += 1
        return tid.value

    def close(self):
        if getattr(self, "h", None):
            lib().qw_workload_destroy(self.h)
            self.h = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_options(**kw) -> qw_plan_opts:
    o = qw_plan_opts()
    lib().qw_plan_opts_default(C.byref(o))
    fields = {f[0] for f in qw_plan_opts._fields_}
    for k, v in kw.items():
        if k not in fields:
            raise TypeError("unknown plan option %r" % k)
        setattr(o, k, v)
    return o


class Plan:
    def __init__(self, engine: Optional[Engine], workload: Workload, **opts):
        self.opts = plan_options(**opts)
        h = C.c_void_p()
        _check(lib().qw_plan_create(engine.h if engine else None, workload.h, C.byref(self.opts),
                                    C.byref(h)))
        self.h = h
        self.n_tasks = workload.n
        self._engine = engine  # the engine owns the device memory: keep it alive

    def execute(self, stream: Optional[int] = None):
        _check(lib().qw_execute(self.h, stream))

    def wait(self):
        _check(lib().qw_wait(self.h))

    def run(self):
        self.execute()
        self.wait()
        return self

    def energy(self, t: int):
        e, n = C.c_double(), C.c_double()
        _check(lib().qw_get_energy(self.h, t, C.byref(e), C.byref(n)))
        return e.value, n.value

    def samples(self, t: int) -> np.ndarray:
        n = C.c_size_t()
        st = lib().qw_get_samples(self.h, t, None, 0, C.byref(n))
        out = np.zeros(n.value, dtype=np.uint64)
        if n.value == 0:
            return out
        _check(lib().qw_get_samples(self.h, t, _p(out), len(out), C.byref(n)))
        return out

    def syndrome(self, t: int) -> np.ndarray:
        n = C.c_size_t()
        lib().qw_get_syndrome(self.h, t, None, 0, C.byref(n))
        out = np.zeros(n.value, dtype=np.uint8)
        _check(lib().qw_get_syndrome(self.h, t, _p(out) if n.value else None, len(out), C.byref(n)))
        return out

    def state(self, t: int, n: int, fp64: bool) -> np.ndarray:
        out = np.zeros(1 << n, dtype=np.complex128 if fp64 else np.complex64)
        _check(lib().qw_get_state(self.h, t, _p(out), out.nbytes))
        return out

    def stabilizers(self, t: int, n: int):
        """(x, z, sign) of a tableau task kept with want_state: generator i
        is (-1)^sign[i] i^{x.z} X^x[i] Z^z[i] (see qw_get_stabilizers)."""
        x = np.zeros((n, n), dtype=np.uint8)
        z = np.zeros((n, n), dtype=np.uint8)
        sg = np.zeros(n, dtype=np.uint8)
        _check(lib().qw_get_stabilizers(self.h, t, _p(x), _p(z), _p(sg), n))
        return x, z, sg

    def _json(self, fn) -> dict:
        need = C.c_size_t()
        fn(self.h, None, 0, C.byref(need))
        buf = C.create_string_buffer(need.value)
        _check(fn(self.h, buf, need.value, C.byref(need)))
        return json.loads(buf.value.decode())

    def explain(self) -> dict:
        return self._json(lib().qw_explain_json)

    def cost_record(self) -> dict:
        return self._json(lib().qw_cost_record_json)

    def close(self):
        if getattr(self, "h", None):
            lib().qw_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- planner primitives -------------------------------------------------------------

def sha256(data: bytes) -> bytes:
    out = (C.c_uint8 * 32)()
    buf = C.create_string_buffer(data, len(data))
    _check(lib().qw_sha256(buf, len(data), out))
    return bytes(out)


def fingerprint(n: int, mode: int, gates: np.ndarray) -> bytes:
    g = np.ascontiguousarray(gates, dtype=W.GATE_DTYPE)
    out = (C.c_uint8 * 32)()
    _check(lib().qw_fingerprint(n, mode, _p(g) if len(g) else None, len(g), out))
    return bytes(out)


def reuse_decision(n_tasks, c_prefix, c_materialize, c_reload, c_handoff, delta):
    c = qw_cost_tuple(n_tasks, c_prefix, c_materialize, c_reload, c_handoff, delta)
    r, lhs, rhs = C.c_int32(), C.c_double(), C.c_double()
    _check(lib().qw_reuse_decision(C.byref(c), C.byref(r), C.byref(lhs), C.byref(rhs)))
    return bool(r.value), lhs.value, rhs.value


def legality_check(kind: int, exactness: int, backend: int, n_qubits: int, provenance: bytes,
                   target_backend: int, expected: Optional[bytes]):
    a = qw_artifact_desc(kind, exactness, backend, n_qubits, (C.c_uint8 * 32)(*provenance))
    ok = C.c_int32()
    ref = qw_refusal()
    exp = None if expected is None else (C.c_uint8 * 32)(*expected)
    _check(lib().qw_legality_check(C.byref(a), target_backend, exp, C.byref(ok), C.byref(ref)))
    fields = {f: getattr(ref, f).decode() for f, _ in qw_refusal._fields_}
    return bool(ok.value), fields


# ---- device-pointer primitives (pointers from torch tensors: t.data_ptr()) ----------

def mlp_forward_dev(params_ptr: int, x_ptr: int, y_ptr: int, batch: int, stream: int = 0):
    _check(lib().qw_mlp_forward_dev(params_ptr, x_ptr, y_ptr, batch, stream or None))


def mlp_loss_grad_dev(params_ptr, x_ptr, t_ptr, batch, loss_ptr, grad_ptr, stream: int = 0):
    _check(lib().qw_mlp_loss_grad_dev(params_ptr, x_ptr, t_ptr, batch, loss_ptr, grad_ptr,
                                      stream or None))


def mlp_adam_dev(params_ptr, grad_ptr, m_ptr, v_ptr, n, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8,
                 stream: int = 0):
    _check(lib().qw_mlp_adam_dev(params_ptr, grad_ptr, m_ptr, v_ptr, n, t, lr, b1, b2, eps,
                                 stream or None))


def sv_apply_dev(engine: Engine, mode: int, n: int, state_ptr: int, gates: np.ndarray,
                 init: bool = False, stream: int = 0):
    g = np.ascontiguousarray(gates, dtype=W.GATE_DTYPE)
    iv = C.c_int32(1 if init else 0)
    _check(lib().qw_sv_apply_dev(engine.h, mode, n, state_ptr, _p(g) if len(g) else None, len(g),
                                 C.byref(iv), stream or None))


def sv_energy_dev(engine: Engine, mode: int, n: int, state_ptr: int, terms: np.ndarray,
                  stream: int = 0):
    t = np.ascontiguousarray(terms, dtype=W.TERM_DTYPE)
    e, nr = C.c_double(), C.c_double()
    _check(lib().qw_sv_energy_dev(engine.h, mode, n, state_ptr, _p(t) if len(t) else None, len(t),
                                  C.byref(e), C.byref(nr), stream or None))
    return e.value, nr.value


def sv_sample_dev(engine: Engine, mode: int, n: int, state_ptr: int, uniforms: np.ndarray,
                  stream: int = 0) -> np.ndarray:
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    out = np.zeros(len(u), dtype=np.uint64)
    _check(lib().qw_sv_sample_dev(engine.h, mode, n, state_ptr, _p(u) if len(u) else None, len(u),
                                  _p(out) if len(u) else None, stream or None))
    return out


def sv_energy_noalloc_dev(mode: int, n: int, state_ptr: int, terms: np.ndarray, out_ptr: int,
                          stream: int = 0):
    """Energy into a caller-owned device buffer (2 doubles) without any device
    allocation (see qw_sv_energy_noalloc_dev); asynchronous on `stream`."""
    t = np.ascontiguousarray(terms, dtype=W.TERM_DTYPE)
    _check(lib().qw_sv_energy_noalloc_dev(mode, n, state_ptr, _p(t) if len(t) else None, len(t),
                                          out_ptr, stream or None))


def sv_fuse(gates: np.ndarray, n: int, tile_qubits: int = 13, low_qubits: int = 3) -> dict:
    """Host only: the pass program of the statevector kernels for `gates`
    (see qw_sv_fuse_json for the layout)."""
    g = np.ascontiguousarray(gates, dtype=W.GATE_DTYPE)
    need = C.c_size_t()
    st = lib().qw_sv_fuse_json(_p(g) if len(g) else None, len(g), n, tile_qubits, low_qubits, None, 0,
                               C.byref(need))
    if st not in (0, -7):
        _check(st)
    buf = C.create_string_buffer(need.value)
    _check(lib().qw_sv_fuse_json(_p(g) if len(g) else None, len(g), n, tile_qubits, low_qubits, buf,
                                 need.value, C.byref(need)))
    return json.loads(buf.value.decode())


def dense_fuse(gates: np.ndarray, n: int, kmax: int = 5):
    """Host only: the dense blocks a program would apply, as a list of
    (qubits, u) with u the 2^k x 2^k complex matrix (see qw_dense_fuse)."""
    g = np.ascontiguousarray(gates, dtype=W.GATE_DTYPE)
    nb = C.c_uint64()
    _check(lib().qw_dense_fuse(_p(g) if len(g) else None, len(g), n, kmax, None, None, None, 0,
                               C.byref(nb)))
    cap = max(1, nb.value)
    k = np.zeros(cap, dtype=np.uint32)
    q = np.zeros(5 * cap, dtype=np.uint32)
    u = np.zeros(2048 * cap, dtype=np.float64)
    _check(lib().qw_dense_fuse(_p(g) if len(g) else None, len(g), n, kmax, _p(k), _p(q), _p(u), cap,
                               C.byref(nb)))
    out = []
    for i in range(nb.value):
        d = 1 << int(k[i])
        m = u[2048 * i:2048 * i + 2 * d * d].view(np.complex128).reshape(d, d).copy()
        out.append((tuple(int(x) for x in q[5 * i:5 * i + k[i]]), m))
    return out


class DenseProgram:
    """Fused dense blocks applied to a caller's device state (see the dense
    block section of include/quwarp.h).  Built from a gate list, or from one
    explicit block (qubits, u)."""

    def __init__(self, engine: Engine, mode: int, n: int, gates: Optional[np.ndarray] = None,
                 kmax: int = 5, engine_kind: int = DENSE_TENSOR, nacc: int = 4,
                 block: Optional[tuple] = None):
        self.h = C.c_void_p()
        self.engine = engine
        if block is not None:
            qubits, u = block
            qa = np.ascontiguousarray(qubits, dtype=np.uint32)
            ua = np.ascontiguousarray(np.asarray(u, dtype=np.complex128)).view(np.float64)
            _check(lib().qw_dense_prog_create_block(engine.h, mode, n, _p(qa), len(qa), _p(ua),
                                                    engine_kind, nacc, C.byref(self.h)))
        else:
            g = np.ascontiguousarray(gates, dtype=W.GATE_DTYPE)
            _check(lib().qw_dense_prog_create(engine.h, mode, n, _p(g) if len(g) else None, len(g),
                                              kmax, engine_kind, nacc, C.byref(self.h)))

    def info(self):
        nb, ng = C.c_uint64(), C.c_uint64()
        _check(lib().qw_dense_prog_info(self.h, C.byref(nb), C.byref(ng)))
        return {"blocks": nb.value, "gates": ng.value}

    def config(self):
        e, k, a, ms = C.c_uint32(), C.c_uint32(), C.c_uint32(), C.c_double()
        _check(lib().qw_dense_prog_config(self.h, C.byref(e), C.byref(k), C.byref(a), C.byref(ms)))
        return {"engine": e.value, "kmax": k.value, "nacc": a.value, "estimated_ms": ms.value}

    def run(self, state_ptr: int, stream: int = 0):
        _check(lib().qw_dense_prog_run(self.h, state_ptr, stream or None))

    def check(self):
        _check(lib().qw_dense_prog_check(self.h))

    def close(self):
        if self.h:
            lib().qw_dense_prog_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

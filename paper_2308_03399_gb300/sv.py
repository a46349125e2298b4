"""Python binding of libsv (ctypes, argument marshalling only).

Every function has the name of its C entry point in include/sv.h; the
simulation itself runs in the library's CUDA kernels.  There is no CPU
fallback: if libsv.so cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

SV_OK, SV_EINVAL, SV_ENOMEM, SV_ECUDA, SV_ETIMEOUT, SV_EUNSUPPORTED, SV_EINTERNAL = range(7)
SV_C64, SV_C128 = 0, 1
SV_PLAIN, SV_BATCH, SV_BRANCH, SV_BATCH_BRANCH = 0, 1, 2, 3
SV_NOISE_PAULI, SV_NOISE_KRAUS = 0, 1
(SV_OPT_LOG, SV_OPT_TILE_BITS, SV_OPT_MAX_ACTIVE, SV_OPT_MAX_STAGES, SV_OPT_THREADS, SV_OPT_GRID,
 SV_OPT_PROFILE, SV_OPT_SLOT_LIMIT, SV_OPT_UPLOAD, SV_OPT_PASS_PATH, SV_OPT_JOINT_KRAUS,
 SV_OPT_SHOT_BASE, SV_OPT_CHAIN_DECIDES, SV_OPT_PREDRAW_PAULI, SV_OPT_COMMUTE, SV_OPT_FOLD,
 SV_OPT_WHOLE_STATE) = range(17)
SV_TREE_WORDS = 9
PROFILE_CLASSES = ("pass", "decide", "alloc", "copy", "final", "init", "other", "total")

_lock = threading.Lock()
_lib = None


class SvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libsv status {status}: {msg}")
        self.status = status


class SvCircuit(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_clbits", C.c_int32), ("n_ops", C.c_int32)] + [
        (f, C.POINTER(C.c_int32)) for f in
        ("kind", "nq", "q_off", "cl_off", "n_terms", "s_off", "cond_clbit", "cond_val", "reset")] + [
        ("d_off", C.POINTER(C.c_int64)), ("qubits", C.POINTER(C.c_int32)), ("clbits", C.POINTER(C.c_int32)),
        ("data", C.POINTER(C.c_double)), ("paulis", C.POINTER(C.c_uint8))]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libsv.so, building it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            P, I, U64, U32, D = C.c_void_p, C.c_int, C.c_uint64, C.c_uint32, C.c_double
            L.sv_last_error.restype = C.c_char_p
            sig = {
                "sv_alloc_batch": [I, U64, I, I, I, U64, U64, P, P],
                "sv_free_batch": [P],
                "sv_set_option": [P, I, C.c_int64],
                "sv_apply_gate_batch": [P, I, P, P, I, I],
                "sv_sample_noise": [P, U32, I, I, P, I, P, P, P],
                "sv_set_param_sets": [P, P, U32],
                "sv_dm_run": [P, I, U64, U64, P, P, P, P],
                "sv_apply_param_gate_batch": [P, I, P, P, I],
                "sv_measure_batch": [P, U32, I, P, P, I],
                "sv_branch": [P, U32],
                "sv_counts": [P, U32, P, P, U64, P],
                "sv_get_keys": [P, P],
                "sv_waiting": [P, P],
                "sv_run_circuit": [P, P, I],
                "sv_run_circuits": [P, P, I, I],
                "sv_get_amplitudes": [P, U64, P, U64],
                "sv_get_outcomes": [P, U32, P, P],
                "sv_get_fork_events": [P, P, U64, P],
                "sv_get_branch_tree": [P, P, U64, P, P, U64, P],
                "sv_stats": [P, P],
                "sv_profile": [P, P, P],
                "sv_sync": [P, U64],
                "sv_final_sample_noalloc": [P, I, I, U32, P, U64, U32, P, P],
                "sv_mlp_create": [I, I, P],
                "sv_mlp_free": [P],
                "sv_mlp_set_params": [P, P, U64],
                "sv_mlp_get_params": [P, P, U64],
                "sv_mlp_forward": [P, P, I, P],
                "sv_mlp_gradient": [P, P, P, I, P, P],
                "sv_mlp_train": [P, P, P, I, I, I, C.c_float, U64, P],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int
            L.sv_mlp_num_params.argtypes = [P]
            L.sv_mlp_num_params.restype = U64
            _lib = L
    return _lib


def _check(status):
    if status != SV_OK:
        raise SvError(status, lib().sv_last_error().decode())


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def circuit_struct(arrays: dict):
    """SvCircuit view of a workloads op table (keeps the arrays alive)."""
    s = SvCircuit()
    s.n_qubits, s.n_clbits, s.n_ops = arrays["n_qubits"], arrays["n_clbits"], arrays["n_ops"]
    for f in ("kind", "nq", "q_off", "cl_off", "n_terms", "s_off", "cond_clbit", "cond_val", "reset",
              "qubits", "clbits"):
        setattr(s, f, arrays[f].ctypes.data_as(C.POINTER(C.c_int32)))
    s.d_off = arrays["d_off"].ctypes.data_as(C.POINTER(C.c_int64))
    s.data = arrays["data"].ctypes.data_as(C.POINTER(C.c_double))
    s.paulis = arrays["paulis"].ctypes.data_as(C.POINTER(C.c_uint8))
    s._keep = arrays
    return s


class Batch:
    """A batch of shots on the GPU (sv_alloc_batch ... sv_free_batch)."""

    def __init__(self, n_qubits, n_shots, n_clbits=0, prec=SV_C64, mode=SV_BATCH, seed=0, mem_budget=0,
                 stream=None):
        self.n_qubits, self.n_shots, self.n_clbits = n_qubits, n_shots, n_clbits
        self.prec, self.mode, self.seed = prec, mode, seed
        h = C.c_void_p()
        _check(lib().sv_alloc_batch(n_qubits, n_shots, n_clbits, prec, mode, seed, mem_budget, stream, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().sv_free_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- ops ---------------------------------------------------------------
    def set_option(self, opt, value):
        _check(lib().sv_set_option(self.h, opt, int(value)))

    def apply_gate_batch(self, qubits, mat, cond_clbit=-1, cond_value=0):
        q = np.asarray(qubits, np.int32)
        m = np.ascontiguousarray(np.stack([np.real(mat), np.imag(mat)], -1).reshape(-1), np.float64)
        _check(lib().sv_apply_gate_batch(self.h, len(q), _p(q), _p(m), cond_clbit, cond_value))

    def set_param_sets(self, set_of_shot, n_sets):
        m = None if set_of_shot is None else np.ascontiguousarray(set_of_shot, np.uint32)
        _check(lib().sv_set_param_sets(self.h, _p(m), int(n_sets)))

    def apply_param_gate_batch(self, qubits, mats):
        q = np.asarray(qubits, np.int32)
        m = np.ascontiguousarray(np.stack([np.real(mats), np.imag(mats)], -1).reshape(-1), np.float64)
        _check(lib().sv_apply_param_gate_batch(self.h, len(q), _p(q), _p(m), len(mats)))

    def sample_noise_pauli(self, op, qubits, cum, strings):
        q = np.asarray(qubits, np.int32)
        c = np.asarray(cum, np.float64)
        s = np.frombuffer("".join(strings).encode(), np.uint8).copy()
        _check(lib().sv_sample_noise(self.h, op, SV_NOISE_PAULI, len(q), _p(q), len(c), _p(c), _p(s), None))

    def sample_noise_kraus(self, op, qubits, mats):
        q = np.asarray(qubits, np.int32)
        k = np.ascontiguousarray(np.stack([np.real(mats), np.imag(mats)], -1).reshape(-1), np.float64)
        _check(lib().sv_sample_noise(self.h, op, SV_NOISE_KRAUS, len(q), _p(q), len(mats), None, None, _p(k)))

    def measure_batch(self, op, qubits, clbits, reset=0):
        q = np.asarray(qubits, np.int32)
        c = np.asarray(clbits, np.int32)
        _check(lib().sv_measure_batch(self.h, op, len(q), _p(q), _p(c), int(reset)))

    def branch(self, op):
        _check(lib().sv_branch(self.h, op))

    def counts(self, op_final, cap=None):
        cap = cap or max(1, min(self.n_shots, 1 << self.n_qubits))
        keys = np.zeros(cap, np.uint64)
        cnt = np.zeros(cap, np.uint64)
        n = C.c_uint64()
        _check(lib().sv_counts(self.h, op_final, _p(keys), _p(cnt), cap, C.byref(n)))
        return {int(k): int(v) for k, v in zip(keys[:n.value], cnt[:n.value])}

    def get_keys(self):
        k = np.zeros(self.n_shots, np.uint64)
        _check(lib().sv_get_keys(self.h, _p(k)))
        return k

    def waiting(self):
        n = C.c_uint64()
        _check(lib().sv_waiting(self.h, C.byref(n)))
        return n.value

    def run_circuit(self, circ_struct, use_graph=True):
        _check(lib().sv_run_circuit(self.h, C.byref(circ_struct), int(use_graph)))

    def get_amplitudes(self, shot):
        out = np.zeros(2 << self.n_qubits, np.float64)
        _check(lib().sv_get_amplitudes(self.h, shot, _p(out), 1 << self.n_qubits))
        return out[0::2] + 1j * out[1::2]

    def get_outcomes(self, op, thresholds=False):
        sel = np.zeros(self.n_shots, np.int32)
        thr = np.zeros(2 * self.n_shots, np.float64) if thresholds else None
        _check(lib().sv_get_outcomes(self.h, op, _p(sel), _p(thr)))
        return (sel, thr.reshape(-1, 2)) if thresholds else sel

    def get_fork_events(self):
        n = C.c_uint64()
        _check(lib().sv_get_fork_events(self.h, None, 0, C.byref(n)))
        cap = max(n.value, 1)
        ev = np.zeros(5 * cap, np.int64)
        _check(lib().sv_get_fork_events(self.h, _p(ev), cap, C.byref(n)))
        return ev[:5 * n.value].reshape(-1, 5)

    def get_branch_tree(self):
        """(records, shots): records is (n, 9) int64 rows (round, op, parent,
        child, outcome, shot_offset, shot_count, parent_offset, parent_count)
        indexing into shots (sv_get_branch_tree)."""
        n_rec, n_ids = C.c_uint64(), C.c_uint64()
        _check(lib().sv_get_branch_tree(self.h, None, 0, C.byref(n_rec), None, 0, C.byref(n_ids)))
        rec = np.zeros(SV_TREE_WORDS * max(n_rec.value, 1), np.int64)
        ids = np.zeros(max(n_ids.value, 1), np.uint32)
        _check(lib().sv_get_branch_tree(self.h, _p(rec), n_rec.value, C.byref(n_rec), _p(ids), n_ids.value,
                                        C.byref(n_ids)))
        return rec[:SV_TREE_WORDS * n_rec.value].reshape(-1, SV_TREE_WORDS), ids[:n_ids.value]

    def stats(self):
        s = np.zeros(8, np.float64)
        _check(lib().sv_stats(self.h, _p(s)))
        keys = ("live_branches", "waiting", "launches", "passes", "pass_bytes", "copy_bytes", "restarts",
                "h2d_bytes")
        return dict(zip(keys, s.tolist()))

    def profile(self):
        ms = np.zeros(8, np.float64)
        cnt = np.zeros(8, np.int64)
        _check(lib().sv_profile(self.h, _p(ms), _p(cnt)))
        return {k: (float(m), int(c)) for k, m, c in zip(PROFILE_CLASSES, ms, cnt)}

    def sync(self, timeout_ns=0):
        _check(lib().sv_sync(self.h, timeout_ns))


class MLP:
    """The learned cost model (sv_mlp_*): forward, gradient and Adam training
    run in the library's CUDA kernels."""

    def __init__(self, n_in, n_hidden=64):
        self.n_in, self.n_hidden = n_in, n_hidden
        h = C.c_void_p()
        _check(lib().sv_mlp_create(n_in, n_hidden, C.byref(h)))
        self.h = h
        self.n_params = int(lib().sv_mlp_num_params(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().sv_mlp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, np.float32)
        _check(lib().sv_mlp_set_params(self.h, _p(p), p.size))

    def get_params(self):
        p = np.zeros(self.n_params, np.float32)
        _check(lib().sv_mlp_get_params(self.h, _p(p), p.size))
        return p

    def forward(self, x):
        x = np.ascontiguousarray(x, np.float32)
        y = np.zeros(x.shape[0], np.float32)
        _check(lib().sv_mlp_forward(self.h, _p(x), x.shape[0], _p(y)))
        return y

    def gradient(self, x, t):
        x = np.ascontiguousarray(x, np.float32)
        t = np.ascontiguousarray(t, np.float32)
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_float()
        _check(lib().sv_mlp_gradient(self.h, _p(x), _p(t), x.shape[0], C.byref(loss), _p(g)))
        return float(loss.value), g

    def train(self, x, t, epochs=200, batch=64, lr=1e-3, seed=0):
        x = np.ascontiguousarray(x, np.float32)
        t = np.ascontiguousarray(t, np.float32)
        loss = C.c_float()
        _check(lib().sv_mlp_train(self.h, _p(x), _p(t), x.shape[0], epochs, batch, lr, seed, C.byref(loss)))
        return float(loss.value)


def dm_run(circ_struct, n_shots, prec=SV_C64, seed=0, stream=None, thresholds=False):
    """sv_dm_run: the density-matrix method.  Returns (keys, probs) or, with
    thresholds, (keys, probs, thresholds as (n_shots, 2))."""
    keys = np.zeros(max(n_shots, 1), np.uint64)
    probs = np.zeros(1 << circ_struct.n_qubits, np.float64)
    thr = np.zeros(2 * max(n_shots, 1), np.float64) if thresholds else None
    _check(lib().sv_dm_run(C.byref(circ_struct), prec, seed, n_shots, _p(keys), _p(probs), _p(thr), stream))
    if thresholds:
        return keys[:n_shots], probs, thr[:2 * n_shots].reshape(-1, 2)
    return keys[:n_shots], probs


def run_circuits(batches, circ_structs, use_graph=True):
    """sv_run_circuits: several (batch, circuit) pairs in one CUDA graph."""
    n = len(batches)
    hs = (C.c_void_p * n)(*[b.h.value for b in batches])
    cs = (C.c_void_p * n)(*[C.cast(C.pointer(c), C.c_void_p).value for c in circ_structs])
    _check(lib().sv_run_circuits(hs, cs, n, int(use_graph)))


def exported_symbols():
    """Names of the entry points the header declares (checked by the tests)."""
    return ["sv_alloc_batch", "sv_free_batch", "sv_set_option", "sv_apply_gate_batch", "sv_sample_noise",
            "sv_measure_batch", "sv_branch", "sv_counts", "sv_get_keys", "sv_waiting", "sv_run_circuit",
            "sv_get_amplitudes", "sv_get_outcomes", "sv_get_fork_events", "sv_get_branch_tree", "sv_stats", "sv_profile", "sv_sync",
            "sv_last_error", "sv_run_circuits", "sv_final_sample_noalloc", "sv_set_param_sets",
            "sv_apply_param_gate_batch", "sv_dm_run", "sv_mlp_create", "sv_mlp_free", "sv_mlp_num_params",
            "sv_mlp_set_params", "sv_mlp_get_params", "sv_mlp_forward", "sv_mlp_gradient", "sv_mlp_train"]

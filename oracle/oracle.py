"""ctypes front end of the CPU oracle (oracle.c) plus the host-side pieces of
the definition that need no simulation: counts and the canonical branch tree.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
library: it reads the same seeded op table (the inputs) and nothing else.

Parity status of each function is recorded in the test files that pin it:
  philox / uniform      pinned to cuRAND's host Philox4x32-10 generator and a
                        uniformity test (tests/test_oracle_philox.py)
  run_shot / run_shots  pinned to Kronecker-product brute force, Bell/GHZ
                        closed forms, Table I, amplitude-damping and
                        depolarizing closed forms, norm preservation and the
                        density-matrix brute force (tests/test_oracle_*.py)
  counts, branch_tree   pinned by hand-built examples (tests/test_oracle_tree.py)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP across shots, no FP contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                               "-shared", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Circ(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_clbits", C.c_int32), ("n_ops", C.c_int32)] + [
        (f, C.POINTER(C.c_int32)) for f in
        ("kind", "nq", "q_off", "cl_off", "n_terms", "s_off", "cond_clbit", "cond_val", "reset")] + [
        ("d_off", C.POINTER(C.c_int64)), ("qubits", C.POINTER(C.c_int32)), ("clbits", C.POINTER(C.c_int32)),
        ("data", C.POINTER(C.c_double)), ("paulis", C.POINTER(C.c_uint8))]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_SO names a separately built variant of oracle.c; the
            # mutation tests use it to check that the pins catch planted
            # mistakes.
            L = C.CDLL(os.environ.get("ORACLE_SO") or build())
            P = C.c_void_p
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32]
            L.orc_uniform.restype = C.c_double
            L.orc_run_shot.argtypes = [C.POINTER(_Circ), C.c_uint64, C.c_uint64, C.c_int32, C.c_int32, P, P,
                                       P, P, P, P, P, P, P, P]
            L.orc_run_shot.restype = C.c_int
            L.orc_run_shots.argtypes = [C.POINTER(_Circ), C.c_uint64, C.c_uint64, C.c_uint64, P, C.c_int, P, P,
                                        P]
            L.orc_run_shots.restype = C.c_int
            L.orc_max_threads.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class OracleCircuit:
    """The op table of a workloads.Circuit, held for the C oracle."""

    def __init__(self, circuit):
        self.circuit = circuit
        self.arrays = a = circuit.to_arrays()
        self.n_qubits = a["n_qubits"]
        self.n_ops = a["n_ops"]
        s = _Circ()
        s.n_qubits, s.n_clbits, s.n_ops = a["n_qubits"], a["n_clbits"], a["n_ops"]
        for f in ("kind", "nq", "q_off", "cl_off", "n_terms", "s_off", "cond_clbit", "cond_val", "reset",
                  "qubits", "clbits"):
            setattr(s, f, a[f].ctypes.data_as(C.POINTER(C.c_int32)))
        s.d_off = a["d_off"].ctypes.data_as(C.POINTER(C.c_int64))
        s.data = a["data"].ctypes.data_as(C.POINTER(C.c_double))
        s.paulis = a["paulis"].ctypes.data_as(C.POINTER(C.c_uint8))
        self.struct = s


def _as_oc(c):
    return c if isinstance(c, OracleCircuit) else OracleCircuit(c)


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(seed: int, shot: int, op: int) -> float:
    return lib().orc_uniform(seed, shot, op)


def run_shot(circuit, seed: int, shot: int, overrides: dict | None = None, want_state: bool = False,
             pset: int = 0):
    """Simulate one shot.  overrides maps op ordinal -> forced outcome (used to
    follow the GPU past a flagged draw); pset is the shot's parameter set
    (the matrix its parameterized gates apply)."""
    oc = _as_oc(circuit)
    n_ops = oc.n_ops
    outcome = np.full(n_ops, -1, np.int32)
    u = np.zeros(n_ops)
    lo = np.zeros(n_ops)
    hi = np.zeros(n_ops)
    norms = np.zeros(n_ops)
    key = C.c_uint64(0)
    cl = C.c_uint64(0)
    state = np.zeros(2 << oc.n_qubits) if want_state else None
    ov = overrides or {}
    ov_op = np.asarray(list(ov.keys()) or [0], np.uint32)
    ov_out = np.asarray(list(ov.values()) or [0], np.int32)
    rc = lib().orc_run_shot(C.byref(oc.struct), seed, shot, int(pset), len(ov), _ptr(ov_op), _ptr(ov_out),
                            _ptr(outcome), _ptr(u), _ptr(lo), _ptr(hi), _ptr(norms),
                            C.byref(key), C.byref(cl), _ptr(state))
    if rc != 0:
        raise RuntimeError("oracle run_shot failed")
    res = dict(outcome=outcome, u=u, c_lo=lo, c_hi=hi, norms=norms, key=key.value, clbits=cl.value)
    if want_state:
        res["state"] = state[0::2] + 1j * state[1::2]
    return res


def run_shots(circuit, seed: int, shot0: int, n_shots: int, threads: int = 0, want_outcomes: bool = True,
              psets=None):
    """Keys (and outcome logs) of shots [shot0, shot0+n_shots); psets[s]
    (optional) is shot shot0+s's parameter set."""
    oc = _as_oc(circuit)
    keys = np.zeros(n_shots, np.uint64)
    outc = np.full((n_shots, oc.n_ops), -1, np.int32) if want_outcomes else None
    cl = np.zeros(n_shots, np.uint64)
    ps = None if psets is None else np.ascontiguousarray(psets, np.uint32)
    bad = lib().orc_run_shots(C.byref(oc.struct), seed, shot0, n_shots, _ptr(ps), threads, _ptr(keys), _ptr(outc),
                              _ptr(cl))
    if bad:
        raise RuntimeError(f"oracle: {bad} shots failed")
    return keys, outc, cl


def max_threads() -> int:
    return lib().orc_max_threads()


def counts(keys) -> dict:
    """Histogram of final keys."""
    vals, cnt = np.unique(np.asarray(keys, np.uint64), return_counts=True)
    return {int(v): int(c) for v, c in zip(vals, cnt)}


def branch_tree(outcomes: np.ndarray, random_ops, shot_ids=None):
    """Canonical shot-branching tree, derived from per-shot outcome logs only.

    A node is a distinct prefix of outcomes over the random ops (final
    sampling excluded); its shot set is the shots that share that prefix.
    Steps where a node has a single child are collapsed, so an edge appears
    only where shots diverge (Section IV-B: a state forks only where its shots'
    sampled outcomes differ).  Returned as a set of records
    (op, parent_shots, child_shots, outcome) with shot sets as frozensets; the
    set is invariant under slot assignment and waiting-list order.
    """
    outcomes = np.asarray(outcomes)
    n_shots = outcomes.shape[0]
    shots = np.arange(n_shots) if shot_ids is None else np.asarray(shot_ids)
    records = set()
    groups = [np.arange(n_shots)]
    for op in random_ops:
        nxt = []
        for g in groups:
            vals = outcomes[g, op]
            uniq = np.unique(vals)
            if len(uniq) == 1:
                nxt.append(g)
                continue
            parent = frozenset(int(shots[i]) for i in g)
            for v in uniq:
                sub = g[vals == v]
                records.add((int(op), parent, frozenset(int(shots[i]) for i in sub), int(v)))
                nxt.append(sub)
        groups = nxt
    return records

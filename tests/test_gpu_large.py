"""Oracle parity at 24 and 28 qubits (the sizes of configs 4 and 5).

These sizes run code that smaller cases never reach: 2 GB complex64 states,
slot offsets past 2^31 bytes, 1024 reduction chunks per state, slots admitted
against the device's free memory (or a budget), and the waiting list of
Section IV-B-2 at these sizes.  The oracle needs minutes per 28-qubit shot,
so it replays a seeded subset of the shots (each shot is reproducible on its
own, keyed by (seed, shot, op)) in parallel threads, and the circuits are
the configs' first layers:

* config 5's first layer (14 Haar SU(4) gates, each followed by 2-qubit
  depolarizing 1e-3 and amplitude damping 1e-3 on both qubits), 28 qubits,
  256 shots with shot-branching in complex64, once with slots admitted
  against all free device memory and once against a 3-state budget (waiting
  list restarts).  4 shots, chosen among those that drew noise, are compared
  draw by draw, and one shot's 2^28 final amplitudes within 1e-5.  At 28
  qubits the final sample's thresholds are 2^-28 apart on average, so a
  final draw may be flagged (the two sides' running sums differ by ~1e-7);
  the count of such flags is printed.
* config 4's 24-qubit brickwork circuit, its first 3 layers, 64 shots.
"""
import numpy as np
import pytest

from paper_2308_03399_gb300 import sv
from paper_2308_03399_gb300 import workloads as W
from tests.parity import compare_shots, oracle_refs, run_gpu

pytestmark = pytest.mark.gpu


def _host_free_gb():
    with open("/proc/meminfo") as f:
        for ln in f:
            if ln.startswith("MemAvailable:"):
                return int(ln.split()[1]) / (1 << 20)
    return 0.0


def _prefix(full, n_ops, name):
    c = W.Circuit(full.n_qubits, full.n_clbits, name=name)
    c.ops = list(full.ops[:n_ops])
    c.final()
    return c


def _noisy_shots(gpu, c, k, always=(0,)):
    """k shots: the given ones, then those that drew the most non-trivial
    noise outcomes (they exercise forks and per-branch matrices)."""
    rops = [op for op in c.random_ops() if c.ops[op].kind != W.FINAL]
    score = sum((gpu["sel"][op] > 0).astype(np.int64) for op in rops)
    order = [int(s) for s in np.argsort(-score, kind="stable") if int(s) not in always]
    return list(always) + order[:k - len(always)]


def test_config5_first_layer_28_qubits_matches_oracle():
    # four oracle shots hold 8 GB each (state and Kraus scratch in complex128)
    if _host_free_gb() < 64:
        pytest.skip("the 28-qubit oracle replay needs 64 GB of host memory")
    full = W.config5()
    c = _prefix(full, 56, "cfg5_layer1_28q")
    n_shots, seed = 256, 5
    st_bytes = 8 << 28
    a = run_gpu(c, seed, n_shots, sv.SV_BRANCH, sv.SV_C64)  # slots: all free memory
    shots = _noisy_shots(a, c, 4)
    b = run_gpu(c, seed, n_shots, sv.SV_BRANCH, sv.SV_C64, mem_budget=3 * (st_bytes + (1 << 20)),
                want_amps=[shots[1]])
    assert b["stats"]["restarts"] > 0, "the 3-state budget must park shots on the waiting list"
    # the schedule never changes a shot's result
    assert np.array_equal(a["keys"], b["keys"])
    for op in c.random_ops():
        assert np.array_equal(a["sel"][op], b["sel"][op]), op
    refs = oracle_refs(c, seed, shots, state_shots={shots[1]})
    errs = []
    n, flagged = compare_shots(c, seed, b, shots, sv.SV_C64, refs=refs, amp_errs=errs)
    print(f"\n28 qubits: {len(shots)} shots, {n} draws compared, {flagged} flagged, "
          f"restarts {b['stats']['restarts']:.0f}, amplitude error {errs}")
    fin = c.n_ops - 1
    assert flagged <= len(shots)  # only final draws may be flagged here
    assert all(int(b["sel"][op][s]) == int(refs[s]["outcome"][op]) for s in shots for op in c.random_ops()
               if op != fin)


def test_config4_24_qubit_circuit_matches_oracle():
    circs, _ = W.config4()
    full = next(x for x in circs if x.n_qubits == 24)
    per_layer = [2 * 24 + 2 * len(range(l % 2, 23, 2)) for l in range(3)]
    c = _prefix(full, sum(per_layer), full.name + "_3layers")
    n_shots, seed = 64, 41
    gpu = run_gpu(c, seed, n_shots, sv.SV_BRANCH, sv.SV_C64, want_amps=[0])
    shots = _noisy_shots(gpu, c, 4)
    refs = oracle_refs(c, seed, shots, state_shots={0})
    errs = []
    n, flagged = compare_shots(c, seed, gpu, shots, sv.SV_C64, refs=refs, amp_errs=errs)
    print(f"\n24 qubits: {len(shots)} shots, {n} draws compared, {flagged} flagged, amplitude error {errs}")
    assert flagged <= len(shots)

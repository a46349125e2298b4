"""Error of the complex64 path against the float64 oracle, per workload.

For each configuration the batched complex64 run (shot-branching) is
compared with the oracle shot by shot: every random choice (a mismatch only
within the threshold tolerance counts as flagged) and the final amplitudes of
sampled shots (largest absolute and relative L2 error).  The table printed by this module
(pytest -s) is the per-configuration error report."""
import pytest

from paper_2308_03399_gb300 import sv
from paper_2308_03399_gb300 import workloads as W
from tests.parity import compare_shots, oracle_refs, run_gpu

pytestmark = pytest.mark.gpu

# (workload, shots run, shots compared, shots whose amplitudes are compared)
CASES = {
    "cfg1_brickwork10": (W.config1, 1000, range(0, 1000), range(0, 1000, 50)),
    "cfg2_su4_16": (W.config2, 10_000, range(0, 10_000, 500), range(0, 10_000, 2000)),
    "cfg3_midmeas20": (W.config3, 2000, range(0, 2000, 500), range(0, 2000, 1000)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_complex64_error_against_oracle(name):
    make, n_shots, shots, amp_shots = CASES[name]
    c = make()
    seed = 31
    gpu = run_gpu(c, seed, n_shots, sv.SV_BRANCH, sv.SV_C64, want_amps=amp_shots)
    errs = []
    refs = oracle_refs(c, seed, shots, state_shots=set(amp_shots))
    n, flagged = compare_shots(c, seed, gpu, shots, sv.SV_C64, amp_errs=errs, refs=refs)
    assert len(errs) == len(amp_shots)
    assert flagged <= max(2, n // 1000)
    worst = max(e for e, _ in errs)
    worst_l2 = max(r for _, r in errs)
    print(f"\n{name}: {len(shots)} shots compared, {n} draws, {flagged} flagged, "
          f"largest amplitude error {worst:.3g}, largest relative L2 error {worst_l2:.3g} over {len(errs)} shots")
    assert worst <= 1e-5


# ---------------------------------------------------------------------------
# Accumulation against float64 sums of the same complex64 amplitudes.
#
# The complex64 path forms each |psi_j|^2 (and each Kraus quadratic form) in
# float32 and accumulates them as float-float pairs; the decide kernels add
# the partial sums in float64.  This measures what that costs against true
# float64 accumulation: before every Kraus op, measurement and final sample,
# the state the reduction will read is downloaded (complex64 values, exact in
# float64), the running sums the selection compares with are recomputed in
# float64 with numpy, and the GPU's logged running sums (just below and at
# each shot's choice) are compared with them.  The gap is the whole error of
# the accumulation, independent of the amplitudes' own float32 rounding.
# ---------------------------------------------------------------------------
import numpy as np  # noqa: E402


def _apply1(psi, n, q, m):
    a = psi.reshape(1 << (n - q - 1), 2, 1 << q)
    return np.einsum("rc,icj->irj", m, a).reshape(-1)


def _running_sums(op, psi, n):
    if op.kind == W.KRAUS:
        assert len(op.qubits) == 1
        p = [float(np.sum(np.abs(_apply1(psi, n, op.qubits[0], k)) ** 2)) for k in op.kraus]
        return np.cumsum(p)
    pr = np.abs(psi) ** 2
    if op.kind == W.MEASURE:
        idx = np.arange(psi.size)
        bits = sum(((idx >> q) & 1) << j for j, q in enumerate(op.qubits))
        return np.cumsum([pr[bits == o].sum() for o in range(1 << len(op.qubits))])
    return np.cumsum(pr)


def _rotated_damping(gamma):
    # amplitude damping in the X basis: its forms K^dagger K are not diagonal
    return [W.H @ k @ W.H for k in W.amplitude_damping(gamma)]


ACC_CASES = {
    "cfg2_prefix_su4_16": lambda: W.random_su4(16, 2, 1e-2, 5e-3, seed=2),
    "cfg3_prefix_midmeas20": lambda: W.midcircuit_measure(20, 2, 5e-3, [0, 5, 10, 15], seed=3),
}


@pytest.mark.parametrize("name", list(ACC_CASES))
def test_accumulation_matches_float64_sums(name):
    c = ACC_CASES[name]()
    if name.startswith("cfg2"):
        # plus non-diagonal Kraus forms (the general quadratic-form reduction)
        extra = W.Circuit(c.n_qubits, c.n_clbits)
        extra.ops = c.ops[:-1]
        for q in (0, 7, 15):
            extra.kraus([q], _rotated_damping(0.2))
        extra.final()
        c = extra
    n, n_shots, watch = c.n_qubits, 32, (0, 9, 21, 31)
    worst = {W.KRAUS: 0.0, W.MEASURE: 0.0, W.FINAL: 0.0}
    detail = []
    count = {W.KRAUS: 0, W.MEASURE: 0, W.FINAL: 0}
    with sv.Batch(n, n_shots, max(1, c.n_clbits), sv.SV_C64, sv.SV_BATCH, 17) as b:
        b.set_option(sv.SV_OPT_LOG, 1)
        for i, o in enumerate(c.ops):
            states = {}
            if o.kind in (W.KRAUS, W.MEASURE, W.FINAL):
                states = {s: b.get_amplitudes(s) for s in watch}
            if o.kind == W.GATE:
                b.apply_gate_batch(o.qubits, o.mat, o.cond_clbit, o.cond_val)
            elif o.kind == W.PAULI:
                b.sample_noise_pauli(i, o.qubits, o.cum, o.strings)
            elif o.kind == W.KRAUS:
                b.sample_noise_kraus(i, o.qubits, o.kraus)
            elif o.kind == W.MEASURE:
                b.measure_batch(i, o.qubits, o.clbits, o.reset)
            else:
                b.counts(i)
            if not states:
                continue
            sel, thr = b.get_outcomes(i, thresholds=True)
            for s, psi in states.items():
                cum = _running_sums(o, psi, n)
                k = int(sel[s])
                lo = cum[k - 1] if k else 0.0
                gap = max(abs(thr[s][0] - lo), abs(thr[s][1] - cum[k]))
                worst[o.kind] = max(worst[o.kind], gap)
                count[o.kind] += 1
                detail.append((gap, i, o.kind, tuple(o.qubits[:2]), s, k, float(thr[s][1]), float(cum[k])))
    names = {W.KRAUS: "Kraus", W.MEASURE: "measurement", W.FINAL: "final sample"}
    print(f"\n{name}: largest |C_gpu - C_float64| over the same complex64 state: " +
          ", ".join(f"{names[k]} {worst[k]:.2e} ({count[k]} decisions)" for k in worst if count[k]))
    for d in sorted(detail, reverse=True)[:6]:
        print("  gap %.2e op %d kind %d qubits %s shot %d choice %d C_gpu %.17g C_f64 %.17g" % d)
    # each |psi_j|^2 is formed in float32 (relative error 2^-24 per term);
    # in the sparse states of a circuit's first gates a few terms carry the
    # whole sum, so the gap reaches a few 1e-8 there and falls to ~1e-10 as
    # the state spreads -- in every case below the float32 amplitudes' own
    # distance from the float64 oracle (~1e-7) and the flag window (1e-5)
    assert max(worst.values()) <= 5e-8

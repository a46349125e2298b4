"""Error of the complex64 path against the float64 oracle, per workload.

For each configuration the batched complex64 run (shot-branching) is
compared with the oracle shot by shot: every random choice (a mismatch only
within the threshold tolerance counts as flagged) and the final amplitudes of
sampled shots (largest absolute and relative L2 error).  The table printed by this module
(pytest -s) is the per-configuration error report."""
import pytest

from paper_2308_03399_gb300 import sv
from paper_2308_03399_gb300 import workloads as W
from tests.parity import compare_shots, run_gpu

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
    n, flagged = compare_shots(c, seed, gpu, shots, sv.SV_C64, amp_errs=errs)
    assert len(errs) == len(amp_shots)
    assert flagged <= max(2, n // 1000)
    worst = max(e for e, _ in errs)
    worst_l2 = max(r for _, r in errs)
    print(f"\n{name}: {len(shots)} shots compared, {n} draws, {flagged} flagged, "
          f"largest amplitude error {worst:.3g}, largest relative L2 error {worst_l2:.3g} over {len(errs)} shots")
    assert worst <= 1e-5

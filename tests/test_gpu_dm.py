"""The density-matrix method on the GPU (sv_dm_run) against the oracle.

The density matrix gives the exact final distribution (Sections II and
III-C).  Checks:
* the GPU's distribution equals the numpy density-matrix brute force of
  oracle/dm.py (1e-12 in complex128, 2e-6 in complex64) on circuits with
  gates, Pauli noise and Kraus noise;
* every shot's key is the first index whose running sum exceeds the shot's
  Philox draw for the final op, with the draw taken from the oracle's own
  Philox and the running sums from the brute force (a mismatch is flagged,
  not failed, only when the draw lies within the two sides' rounding of the
  boundary running sum);
* at 10 qubits, beyond the brute force, the GPU distribution against the
  oracle's per-shot simulation: a chi-squared test on 20000 shots.
"""
import numpy as np
import pytest

from oracle import dm
from oracle import oracle as O
from paper_2308_03399_gb300 import sv
from paper_2308_03399_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = {
    "brickwork": lambda: W.brickwork(6, 4, 0.05, 0.1, seed=401),
    "su4_kraus": lambda: W.random_su4(5, 3, 0.1, 0.1, seed=402),
    "qft_pauli": lambda: W.qft(6, 0.05, seed=403),
    "qft_kraus": lambda: W.qft(5, 0.05, seed=404, kraus=True),
}
TOL = {sv.SV_C128: (1e-12, 1e-10), sv.SV_C64: (2e-6, 1e-5)}


@pytest.mark.parametrize("prec", [sv.SV_C64, sv.SV_C128])
@pytest.mark.parametrize("name", list(CASES))
def test_dm_distribution_and_keys_match_brute_force(name, prec):
    c = CASES[name]()
    n_shots, seed = 3000, 9
    keys, probs, thr = sv.dm_run(sv.circuit_struct(c.to_arrays()), n_shots, prec, seed, thresholds=True)
    ref = dm.final_distribution(c)
    tol_p, tol_c = TOL[prec]
    assert np.abs(probs - ref).max() < tol_p
    cum = np.cumsum(ref)
    fop = c.n_ops - 1
    flagged = 0
    for s in range(n_shots):
        u = O.uniform(seed, s, fop)
        k = int(np.searchsorted(cum, u, side="right"))  # first j with u < C_j
        if k == len(cum):
            k = int(np.nonzero(ref > 0)[0][-1])
        g = int(keys[s])
        if g == k:
            continue
        bg, bc = (thr[s][1], cum[k - 1]) if g < k else (thr[s][0], cum[k])
        assert abs(bg - bc) <= tol_c and min(bg, bc) - 1e-9 <= u <= max(bg, bc) + 1e-9, (s, g, k, u)
        flagged += 1
    assert flagged <= 3


def test_dm_ten_qubits_against_oracle_shots():
    from scipy import stats
    c = W.brickwork(10, 6, 0.02, 0.05, seed=410)
    _, probs = sv.dm_run(sv.circuit_struct(c.to_arrays()), 0, sv.SV_C128, 1)
    assert abs(probs.sum() - 1) < 1e-12
    keys, _, _ = O.run_shots(c, 77, 0, 20000, want_outcomes=False)
    counts = np.bincount(keys.astype(np.int64), minlength=probs.size)
    # pool the rare outcomes into one cell so every expected count is >= 5
    exp = probs * keys.size
    big = exp >= 5
    obs = np.append(counts[big], counts[~big].sum())
    ex = np.append(exp[big], exp[~big].sum())
    chi2 = ((obs - ex) ** 2 / np.maximum(ex, 1e-300)).sum()
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-3


def test_dm_rejects_what_it_cannot_run():
    c = W.midcircuit_measure(4, 1, 0.01, [0], seed=1)
    with pytest.raises(sv.SvError):
        sv.dm_run(sv.circuit_struct(c.to_arrays()), 10)
    big = W.brickwork(16, 1, 0.01, 0.01, seed=1)
    with pytest.raises(sv.SvError):
        sv.dm_run(sv.circuit_struct(big.to_arrays()), 10)

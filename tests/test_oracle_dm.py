"""Whole-distribution pin: oracle counts against the exact density-matrix
distribution (Section II: the density-matrix method yields the exact
distribution that multi-shot sampling estimates), chi-squared, fixed seeds."""
import numpy as np
import pytest

from oracle import dm
from oracle import oracle as O
from paper_2308_03399_gb300 import workloads as W


def _chi2_pvalue(counts, probs, shots):
    stats = pytest.importorskip("scipy.stats")
    obs = np.zeros(len(probs))
    for k, v in counts.items():
        obs[k] += v
    exp = probs * shots
    keep = exp > 5
    # lump rare keys into one bin
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    if e[-1] == 0:
        assert o[-1] == 0
        o, e = o[:-1], e[:-1]
    return stats.chisquare(o, e * o.sum() / e.sum()).pvalue


CASES = {
    "brickwork_pauli": lambda: W.brickwork(4, 4, 0.05, 0.1, seed=11),
    "su4_pauli_kraus": lambda: W.random_su4(4, 3, 0.1, 0.15, seed=12),
    "midmeasure_cond": lambda: W.midcircuit_measure(4, 2, 0.05, [0, 2], seed=13),
    "qft_kraus": lambda: W.qft(3, 0.05, seed=14, kraus=True),
}


@pytest.mark.parametrize("name", list(CASES))
def test_counts_match_density_matrix(name):
    c = CASES[name]()
    probs = dm.final_distribution(c)
    assert abs(probs.sum() - 1) < 1e-12
    shots = 100_000
    keys, _, _ = O.run_shots(c, 100 + len(name), 0, shots, want_outcomes=False)
    assert _chi2_pvalue(O.counts(keys), probs, shots) > 1e-3


def test_density_matrix_detects_a_wrong_channel():
    # sanity of the test itself: a distribution from a different noise rate fails
    c = W.random_su4(4, 3, 0.1, 0.15, seed=12)
    wrong = dm.final_distribution(W.random_su4(4, 3, 0.1, 0.05, seed=12))
    keys, _, _ = O.run_shots(c, 7, 0, 100_000, want_outcomes=False)
    assert _chi2_pvalue(O.counts(keys), wrong, 100_000) < 1e-6

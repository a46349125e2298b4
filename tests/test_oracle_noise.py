"""Pins of the oracle's noise sampling, measurement and classical control.

Table I (Section III-B-1) is read from tests/golden/table1_bitflip.txt; the
rest are closed forms of textbook channels:
  * amplitude damping on |1>: the jump K1 has probability gamma; after r
    applications the qubit is still 1 with probability (1-gamma)^r;
  * depolarizing p on |0> then measurement: P(1) = p/2;
  * GHZ measurement collapses onto 0...0 or 1...1;
  * a Pauli channel written as Kraus matrices sqrt(p_t) P_t picks the same
    strings (Section III-B-2), up to draws within 1e-9 of a threshold;
  * ||psi|| = 1 after every op.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2308_03399_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _binom_ok(k, n, p, z=4.5):
    return abs(k - n * p) <= z * math.sqrt(n * p * (1 - p)) + 1


def test_table1_bitflip_selection():
    rows = [ln.split() for ln in open(os.path.join(GOLD, "table1_bitflip.txt")) if ln.strip() and ln[0] != "#"]
    cum = [float(r[0]) for r in rows]
    strings = [r[1] for r in rows]
    assert cum == [0.99, 1.0] and strings == ["I", "X"]
    c = W.Circuit(1)
    op = c.pauli([0], cum, strings)
    c.final()
    n_flip = 0
    for s in range(20000):
        r = O.run_shot(c, 17, s)
        u = r["u"][op]
        want = 0 if u < 0.99 else 1
        assert r["outcome"][op] == want
        assert r["key"] == want  # X flips |0> to |1>, ID leaves it
        n_flip += want
    assert _binom_ok(n_flip, 20000, 0.01)


def test_amplitude_damping_closed_forms():
    g = 0.2
    c = W.Circuit(1)
    c.gate([0], W.X)
    op = c.kraus([0], W.amplitude_damping(g))
    c.final()
    for s in range(2000):
        r = O.run_shot(c, 5, s)
        # K1|1> = sqrt(g)|0>: p_0 = 1-g, so the jump is taken iff u >= 1-g
        assert r["c_hi"][op] == pytest.approx(1 - g if r["outcome"][op] == 0 else 1.0, abs=1e-15)
        assert r["outcome"][op] == (0 if r["u"][op] < 1 - g else 1)
        assert r["key"] == 1 - r["outcome"][op]
    # r repeated applications: P(still 1) = (1-g)^r
    for reps in (1, 3, 6):
        c = W.Circuit(1)
        c.gate([0], W.X)
        for _ in range(reps):
            c.kraus([0], W.amplitude_damping(g))
        c.final()
        keys, _, _ = O.run_shots(c, 8, 0, 20000, want_outcomes=False)
        assert _binom_ok(int((keys == 1).sum()), 20000, (1 - g) ** reps)


def test_depolarizing_on_zero_gives_half_p():
    p = 0.3
    c = W.Circuit(1)
    c.depolarizing([0], p)
    c.measure([0], [0])
    c.final()
    _, _, cl = O.run_shots(c, 21, 0, 40000)
    assert _binom_ok(int(cl.sum()), 40000, p / 2)


def test_depolarizing_table_is_textbook():
    cum, strings = W.depolarizing_table(0.01, 2)
    assert strings[0] == "II" and strings[1] == "XI" and strings[4] == "IX" and strings[15] == "ZZ"
    probs = np.diff([0.0] + cum)
    assert probs[0] == pytest.approx(1 - 0.01 + 0.01 / 16)
    assert np.allclose(probs[1:], 0.01 / 16)


def test_ghz_measurement_collapses():
    n = 4
    c = W.Circuit(n)
    c.gate([0], W.H)
    for q in range(n - 1):
        c.gate([q, q + 1], W.cx())
    op = c.measure([1], [0])
    c.final()
    for s in range(64):
        r = O.run_shot(c, 4, s, want_state=True)
        o = r["outcome"][op]
        assert r["clbits"] == o
        want = np.zeros(2 ** n, complex)
        want[0 if o == 0 else 2 ** n - 1] = 1
        assert np.abs(np.abs(r["state"]) - np.abs(want)).max() < 1e-15
        assert r["key"] == (0 if o == 0 else 2 ** n - 1)
        assert r["c_lo"][op] == pytest.approx(0.0 if o == 0 else 0.5, abs=1e-15)


def test_measure_with_reset_and_conditional_x():
    c = W.Circuit(3)
    c.gate([0], W.H)
    c.gate([0, 1], W.cx())
    m1 = c.measure([0, 1], [0, 1], reset=1)
    c.gate([2], W.H)
    m2 = c.measure([2], [2])
    c.gate([2], W.X, cond_clbit=2, cond_val=1)  # conditional reset of qubit 2
    c.final()
    seen = set()
    for s in range(200):
        r = O.run_shot(c, 2, s)
        assert r["key"] == 0  # everything was reset
        o1, o2 = r["outcome"][m1], r["outcome"][m2]
        assert o1 in (0, 3)  # Bell pair: both 0 or both 1
        assert r["clbits"] == o1 | (o2 << 2)
        seen.add((o1, o2))
    assert len(seen) == 4


def test_pauli_algebra_on_random_state():
    rng = np.random.default_rng(1)

    def rnd_state_circuit():
        c = W.Circuit(3)
        for q in range(3):
            c.gate([q], W.u3(*rng.uniform(0, 6, 3)))
        c.gate([0, 2], W.haar_su4(rng))
        return c

    base = rnd_state_circuit()
    ops = list(base.ops)
    # forced Pauli strings (single-entry tables): Y on qubit 1, then YY twice
    c = W.Circuit(3, ops=list(ops))
    c.pauli([1], [1.0], ["Y"])
    c.final()
    b = W.Circuit(3, ops=list(ops))
    b.gate([1], np.array([[0, -1j], [1j, 0]]))
    b.final()
    s1 = O.run_shot(c, 1, 0, want_state=True)["state"]
    s2 = O.run_shot(b, 1, 0, want_state=True)["state"]
    assert np.abs(s1 - s2).max() < 1e-14
    c = W.Circuit(3, ops=list(ops))
    c.pauli([0, 2], [1.0], ["XY"])
    c.pauli([0, 2], [1.0], ["XY"])
    c.final()
    b = W.Circuit(3, ops=list(ops))
    b.final()
    assert np.abs(O.run_shot(c, 1, 0, want_state=True)["state"] - O.run_shot(b, 1, 0, want_state=True)["state"]).max() < 1e-14
    # X then Y on the same qubit is the product Y X = -i Z
    c = W.Circuit(3, ops=list(ops))
    c.pauli([1], [1.0], ["X"])
    c.pauli([1], [1.0], ["Y"])
    c.final()
    b = W.Circuit(3, ops=list(ops))
    b.gate([1], -1j * np.diag([1, -1]))
    b.final()
    assert np.abs(O.run_shot(c, 1, 0, want_state=True)["state"] - O.run_shot(b, 1, 0, want_state=True)["state"]).max() < 1e-14


def test_pauli_channel_as_kraus_picks_same_strings():
    rng = np.random.default_rng(2)
    cp = W.Circuit(3)
    ck = W.Circuit(3)
    pauli_ops = []
    for layer in range(6):
        for q in range(3):
            g = W.u3(*rng.uniform(0, 6, 3))
            cp.gate([q], g)
            ck.gate([q], g)
            cum, st = W.depolarizing_table(0.2, 1)
            pauli_ops.append(cp.pauli([q], cum, st))
            ck.kraus([q], W.pauli_as_kraus(cum, st))
        cp.gate([0, 1], W.cx())
        ck.gate([0, 1], W.cx())
        cum, st = W.depolarizing_table(0.3, 2)
        pauli_ops.append(cp.pauli([0, 1], cum, st))
        ck.kraus([0, 1], W.pauli_as_kraus(cum, st))
    cp.final()
    ck.final()
    n_diff = 0
    for s in range(300):
        a = O.run_shot(cp, 3, s)
        b = O.run_shot(ck, 3, s)
        for op in pauli_ops:
            if a["outcome"][op] != b["outcome"][op]:
                # only a draw sitting on a threshold may differ
                n_diff += 1
                t = min(a["outcome"][op], b["outcome"][op])
                assert abs(a["u"][op] - a["c_hi"][op] if a["outcome"][op] == t else a["u"][op] - b["c_hi"][op]) < 1e-9
                break
        else:
            assert a["key"] == b["key"]
    assert n_diff <= 3


@pytest.mark.parametrize("cfg", ["su4", "mid", "brick"])
def test_norm_preserved_after_every_op(cfg):
    if cfg == "su4":
        c = W.random_su4(6, 6, 0.05, 0.05, seed=1)
    elif cfg == "mid":
        c = W.midcircuit_measure(6, 3, 0.05, [0, 3], seed=2)
    else:
        c = W.brickwork(7, 5, 0.05, 0.1, seed=3)
    for s in range(20):
        r = O.run_shot(c, 1, s)
        assert np.abs(r["norms"] - 1).max() < 1e-12


def test_override_forces_outcome():
    c = W.Circuit(2)
    c.gate([0], W.H)
    op = c.measure([0], [0])
    c.final()
    for forced in (0, 1):
        r = O.run_shot(c, 1, 0, overrides={op: forced})
        assert r["outcome"][op] == forced and r["key"] == forced

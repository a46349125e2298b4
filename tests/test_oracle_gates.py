"""Pins of the oracle's gate application and final sampling.

* a tensor-contraction (Kronecker product) evolution written with numpy,
  sharing nothing with oracle.c, on random circuits of up to 6 qubits;
* Bell and GHZ states in closed form (amplitudes 1/sqrt 2 on 0...0 and
  1...1; counts only on those keys, each with probability 1/2);
* unitarity of the generated U3, CX and Haar SU(4) matrices."""
import math

import numpy as np
import pytest

from oracle import dm
from oracle import oracle as O
from paper_2308_03399_gb300 import workloads as W


def _random_unitary(rng, k):
    z = rng.standard_normal((2 ** k, 2 ** k)) + 1j * rng.standard_normal((2 ** k, 2 ** k))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (5, 3), (6, 4)])
def test_gates_match_tensor_contraction(n, seed):
    rng = np.random.default_rng(seed)
    c = W.Circuit(n)
    for _ in range(40):
        k = int(rng.integers(1, min(n, 3) + 1))
        q = rng.choice(n, k, replace=False).tolist()
        c.gate(q, _random_unitary(rng, k))
    c.final()
    ref = dm.final_state_unitary(c)
    got = O.run_shot(c, 1, 0, want_state=True)["state"]
    assert np.abs(got - ref).max() < 1e-12


def test_bell_and_ghz_closed_forms():
    for n in (2, 3, 5):
        c = W.Circuit(n)
        c.gate([0], W.H)
        for q in range(n - 1):
            c.gate([q, q + 1], W.cx())
        c.final()
        st = O.run_shot(c, 1, 0, want_state=True)["state"]
        want = np.zeros(2 ** n, complex)
        want[0] = want[-1] = 1 / math.sqrt(2)
        assert np.abs(st - want).max() < 1e-15
        keys, _, _ = O.run_shots(c, 11, 0, 20000, want_outcomes=False)
        cnt = O.counts(keys)
        assert set(cnt) <= {0, 2 ** n - 1}
        # binomial(20000, 1/2): 4.5 sigma band
        assert abs(cnt.get(0, 0) - 10000) < 4.5 * math.sqrt(5000)


def test_cx_convention():
    # CX on [c, t] flips t where c is 1: |c=1,t=0> -> |c=1,t=1>
    c = W.Circuit(3)
    c.gate([2], W.X)
    c.gate([2, 0], W.cx())
    c.final()
    st = O.run_shot(c, 1, 0, want_state=True)["state"]
    assert abs(st[0b101] - 1) < 1e-15


def test_generated_matrices_are_unitary():
    rng = np.random.default_rng(0)
    mats = [W.u3(*rng.uniform(0, 2 * math.pi, 3)) for _ in range(50)] + [W.cx()]
    mats += [W.haar_su4(rng) for _ in range(50)]
    for m in mats:
        assert np.abs(m.conj().T @ m - np.eye(len(m))).max() < 1e-13
    for _ in range(10):
        assert abs(np.linalg.det(W.haar_su4(rng)) - 1) < 1e-12


def test_final_sampling_follows_cumulative_rule():
    # 3-qubit random state: key of every shot is the first j with u < C_j
    rng = np.random.default_rng(5)
    c = W.Circuit(3)
    c.gate([0, 1, 2], _random_unitary(rng, 3))
    op = c.final()
    st = O.run_shot(c, 1, 0, want_state=True)["state"]
    cum = np.cumsum(np.abs(st) ** 2)
    for s in range(300):
        r = O.run_shot(c, 9, s)
        u = r["u"][op]
        assert r["key"] == int(np.searchsorted(cum, u, side="right")) or abs(u - cum[r["key"]]) < 1e-12


@pytest.mark.parametrize("pset", [0, 1, 2])
def test_param_gates_match_the_substituted_circuit(pset):
    # a parameterized gate applies the matrix of the shot's parameter set
    # (Section VI): the oracle's state equals the tensor contraction of the
    # circuit with that set's matrices written in as plain gates
    rng = np.random.default_rng(7)
    c, plain = W.Circuit(5), W.Circuit(5)
    for _ in range(12):
        k = int(rng.integers(1, 3))
        q = rng.choice(5, k, replace=False).tolist()
        mats = [_random_unitary(rng, k) for _ in range(3)]
        c.param_gate(q, mats)
        plain.gate(q, mats[pset])
        u = _random_unitary(rng, 1)
        c.gate([int(rng.integers(5))], u)
        plain.gate(c.ops[-1].qubits, u)
    c.final()
    plain.final()
    got = O.run_shot(c, 1, 0, want_state=True, pset=pset)["state"]
    assert np.abs(got - dm.final_state_unitary(plain)).max() < 1e-12
    with pytest.raises(RuntimeError):
        O.run_shot(c, 1, 0, pset=3)  # no such parameter set

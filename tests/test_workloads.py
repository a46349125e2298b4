"""The seeded synthetic workloads have the shapes the input recipe states
(op counts, qubit counts, noise placement, shot splits), so the bench and
parity tests run the configurations they name."""
import numpy as np

from paper_2308_03399_gb300 import workloads as W


def kinds(c):
    return [o.kind for o in c.ops]


def test_config1_brickwork_shape():
    c = W.config1()
    assert c.n_qubits == 10
    # 20 layers x (10 U3 + 10 Pauli ops) + CX (5 and 4 on alternate layers) each with a Pauli op, + final
    assert len(c.ops) == 20 * 20 + (10 * 5 + 10 * 4) * 2 + 1 == 581
    assert kinds(c)[-1] == W.FINAL
    assert sum(k == W.KRAUS for k in kinds(c)) == 0


def test_config2_su4_shape():
    c = W.config2()
    assert c.n_qubits == 16 and len(c.ops) == 16 * 8 * 4 + 1 == 513
    ops = c.ops[:4]
    assert ops[0].kind == W.GATE and len(ops[0].qubits) == 2
    assert ops[1].kind == W.PAULI and ops[1].qubits == ops[0].qubits
    assert ops[2].kind == W.KRAUS and ops[2].qubits == [ops[0].qubits[0]]
    assert ops[3].kind == W.KRAUS and ops[3].qubits == [ops[0].qubits[1]]
    m = ops[0].mat
    assert np.allclose(m.conj().T @ m, np.eye(4)) and abs(np.linalg.det(m) - 1) < 1e-12


def test_config3_rounds():
    c = W.config3()
    assert c.n_qubits == 20
    per_round = 20 * 2 + 19 * 2 + 1 + 4
    assert len(c.ops) == 30 * per_round + 1
    meas = [o for o in c.ops if o.kind == W.MEASURE]
    assert len(meas) == 30 and all(o.qubits == [0, 5, 10, 15] for o in meas)
    cond = [o for o in c.ops if o.kind == W.GATE and o.cond_clbit >= 0]
    assert len(cond) == 30 * 4


def test_config4_split():
    circs, shots = W.config4()
    assert len(circs) == 64 and int(np.sum(shots)) == 100_000 and min(shots) >= 1
    assert all(8 <= c.n_qubits <= 24 for c in circs)


def test_config5_shape():
    c = W.config5()
    assert c.n_qubits == 28 and len(c.ops) == 12 * 14 * 4 + 1


def test_depolarizing_tables_are_distributions():
    for k in (1, 2):
        cum, strings = W.depolarizing_table(0.03, k)
        assert abs(cum[-1] - 1.0) < 1e-15 and strings[0] == "I" * k and len(strings) == 4 ** k
        p = np.diff(np.concatenate([[0.0], cum]))
        assert np.allclose(p[1:], 0.03 / 4 ** k) and abs(p[0] - (1 - 0.03 + 0.03 / 4 ** k)) < 1e-15


def test_qft_noise_forms_agree():
    a, b = W.qft(6, 0.01, seed=3), W.qft(6, 0.01, seed=3, kraus=True)
    assert [o.kind for o in a.ops if o.kind == W.PAULI] and [o.kind for o in b.ops if o.kind == W.KRAUS]
    assert len(a.ops) == len(b.ops)
    for oa, ob in zip(a.ops, b.ops):
        if oa.kind == W.PAULI:
            # the Kraus form of a Pauli channel: sqrt(p_k) P_k, complete
            s = sum(K.conj().T @ K for K in ob.kraus)
            assert np.allclose(s, np.eye(len(s)))

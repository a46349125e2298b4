"""Exact density-matrix evolution of a small noisy circuit (n <= 6 qubits).

TEST INFRASTRUCTURE ONLY (imported by tests).  The density-matrix method
gives the exact outcome distribution that multi-shot sampling estimates
(Section II; Section III-C compares the two methods).  It is written with
numpy tensor contractions and shares no code with oracle.c, so agreement
between the two is evidence for both.

Rules (Section III-B):
  gate U:            rho -> U rho U^dagger
  Pauli channel:     rho -> sum_t p_t P_t rho P_t^dagger, p_t from the
                     cumulative table
  Kraus channel:     rho -> sum_i K_i rho K_i^dagger
  measure (m qubits): one unnormalised rho per classical record; outcome o
                     projects, writes the bits, and for a reset flips the
                     measured ones back to 0
  conditional gate:  applied to the records whose bit matches
The final distribution is the diagonal summed over classical records.
"""
from __future__ import annotations

import numpy as np

GATE, PAULI, KRAUS, MEASURE, FINAL = 0, 1, 2, 3, 4
_P1 = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]]), "Y": np.array([[0, -1j], [1j, 0]]),
       "Z": np.diag([1.0, -1.0])}


def full_operator(mat: np.ndarray, qubits, n: int) -> np.ndarray:
    """2^n x 2^n operator of a k-qubit matrix (bit j of its index = qubit
    qubits[j]) by contracting it into the tensor of every basis vector."""
    k = len(qubits)
    dim = 1 << n
    t = np.asarray(mat, np.complex128).reshape((2,) * (2 * k))
    # matrix index bit j is tensor axis k-1-j (C order, most significant first)
    out_axes = list(range(k))
    in_axes = list(range(k, 2 * k))
    full = np.zeros((dim, dim), np.complex128)
    for col in range(dim):
        v = np.zeros(dim, np.complex128)
        v[col] = 1
        psi = v.reshape((2,) * n)  # axis a holds qubit n-1-a
        # contract matrix inputs with the qubit axes
        axes_psi = [n - 1 - qubits[k - 1 - a] for a in range(k)]
        r = np.tensordot(t, psi, axes=(in_axes, axes_psi))
        # r axes: k output axes (matrix order), then remaining psi axes in order
        remaining = [a for a in range(n) if a not in axes_psi]
        order = [None] * n
        for a in range(k):
            order[axes_psi[a]] = out_axes[a]
        for i, a in enumerate(remaining):
            order[a] = k + i
        full[:, col] = np.transpose(r, order).reshape(dim)
    return full


def pauli_string_operator(s: str, qubits, n: int) -> np.ndarray:
    m = np.ones((1, 1), np.complex128)
    for ch in s:  # character j acts on qubits[j] = bit j of the small index
        m = np.kron(_P1[ch], m)
    return full_operator(m, qubits, n)


def _ops(circuit):
    return circuit.ops


def final_distribution(circuit) -> np.ndarray:
    """Exact probabilities of every FINAL key (length 2^n)."""
    n = circuit.n_qubits
    dim = 1 << n
    assert n <= 6
    rho0 = np.zeros((dim, dim), np.complex128)
    rho0[0, 0] = 1
    recs = {0: rho0}
    for op in _ops(circuit):
        if op.kind == GATE:
            U = full_operator(op.mat, op.qubits, n)
            new = {}
            for c, r in recs.items():
                if op.cond_clbit >= 0 and ((c >> op.cond_clbit) & 1) != op.cond_val:
                    new[c] = r
                else:
                    new[c] = U @ r @ U.conj().T
            recs = new
        elif op.kind == PAULI:
            ops = []
            prev = 0.0
            for cum, s in zip(op.cum, op.strings):
                ops.append((cum - prev, pauli_string_operator(s, op.qubits, n)))
                prev = cum
            recs = {c: sum(p * P @ r @ P.conj().T for p, P in ops) for c, r in recs.items()}
        elif op.kind == KRAUS:
            Ks = [full_operator(K, op.qubits, n) for K in op.kraus]
            recs = {c: sum(K @ r @ K.conj().T for K in Ks) for c, r in recs.items()}
        elif op.kind == MEASURE:
            m = len(op.qubits)
            new = {}
            for c, r in recs.items():
                for o in range(1 << m):
                    proj = np.zeros(dim)
                    for j in range(dim):
                        if all(((j >> op.qubits[b]) & 1) == ((o >> b) & 1) for b in range(m)):
                            proj[j] = 1
                    Pm = np.diag(proj)
                    r2 = Pm @ r @ Pm
                    if op.reset:
                        for b in range(m):
                            if (o >> b) & 1:
                                Xf = full_operator(_P1["X"], [op.qubits[b]], n)
                                r2 = Xf @ r2 @ Xf
                    c2 = c
                    for b in range(m):
                        c2 = (c2 & ~(1 << op.clbits[b])) | (((o >> b) & 1) << op.clbits[b])
                    new[c2] = new.get(c2, 0) + r2
            recs = new
        elif op.kind == FINAL:
            break
    probs = sum(np.real(np.diag(r)) for r in recs.values())
    return np.clip(probs, 0, None)


def final_state_unitary(circuit) -> np.ndarray:
    """State vector of a circuit made only of unconditional gates, by
    tensor contraction (textbook Kronecker-product evolution)."""
    n = circuit.n_qubits
    psi = np.zeros((2,) * n, np.complex128)
    psi[(0,) * n] = 1
    for op in circuit.ops:
        if op.kind == FINAL:
            break
        assert op.kind == GATE and op.cond_clbit < 0
        k = len(op.qubits)
        t = op.mat.reshape((2,) * (2 * k))
        axes_psi = [n - 1 - op.qubits[k - 1 - a] for a in range(k)]
        r = np.tensordot(t, psi, axes=(list(range(k, 2 * k)), axes_psi))
        remaining = [a for a in range(n) if a not in axes_psi]
        order = [None] * n
        for a in range(k):
            order[axes_psi[a]] = a
        for i, a in enumerate(remaining):
            order[a] = k + i
        psi = np.transpose(r, order)
    return psi.reshape(-1)

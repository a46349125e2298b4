"""Seeded synthetic circuit and noise-model generator.

This module only *describes* circuits: it builds the flattened op table that
both the CUDA library and the CPU oracle consume.  It applies no gate, draws
no shot randomness and holds none of the simulation method's arithmetic.

What it fixes (conventions the paper leaves open):

* Qubit order is little-endian: qubit q is bit q of the amplitude index.
* A k-qubit matrix on the qubit list [q_0 .. q_{k-1}] maps bit j of its
  row/column index to q_j; storage is row-major complex, re/im interleaved,
  float64.
* U3(theta, phi, lam) = [[cos t/2, -e^{i lam} sin t/2],
                         [e^{i phi} sin t/2, e^{i(phi+lam)} cos t/2]].
* CX on [c, t] flips bit t where bit c is 1.
* A Pauli noise model is a list of Pauli strings with *cumulative*
  probabilities, identity first (Section III-B-1, Table I).  For a k-qubit
  depolarizing channel the strings are listed in ascending base-4 order
  (I=0, X=1, Y=2, Z=3), digit j acting on qubits[j]; the textbook channel
  rho -> (1-p) rho + p I/2^k gives P(I) = 1 - p + p/4^k and p/4^k to each
  other string.  The cumulative column is the running float64 sum in list
  order, exactly as Table I prints it.
* A Kraus noise model is a list of matrices (Section III-B-2); amplitude
  damping with rate g is K0 = [[1,0],[0,sqrt(1-g)]], K1 = [[0,sqrt(g)],[0,0]].
* Every op gets its ordinal (position in the flattened list); random ops key
  their draws with it.

Op kinds: GATE, PAULI, KRAUS, MEASURE (m qubits into m classical bits,
optionally followed by a reset of the measured qubits), FINAL (sample all
qubits; the sampled n-bit index is the count key) and PGATE (one matrix per
parameter set; a shot applies the matrix of its own set).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GATE, PAULI, KRAUS, MEASURE, FINAL, PGATE = 0, 1, 2, 3, 4, 5
KIND_NAMES = {GATE: "gate", PAULI: "pauli", KRAUS: "kraus", MEASURE: "measure", FINAL: "final",
              PGATE: "param_gate"}
RANDOM_KINDS = (PAULI, KRAUS, MEASURE, FINAL)


# ----------------------------------------------------------------------------
# matrices (inputs, computed once in float64)
# ----------------------------------------------------------------------------
def u3(theta: float, phi: float, lam: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -np.exp(1j * lam) * s],
                     [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]], dtype=np.complex128)


def cx() -> np.ndarray:
    """CX on qubits [control, target]; basis index = b_control + 2*b_target."""
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = 1
    m[2, 2] = 1
    m[3, 1] = 1
    m[1, 3] = 1
    return m


X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2)


def haar_unitary(dim: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random dim x dim unitary: QR of a complex Ginibre matrix with the
    phase fix of Mezzadri 2007."""
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / math.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def haar_su4(rng: np.random.Generator) -> np.ndarray:
    """Haar-random unitary of size 4, scaled to determinant 1."""
    q = haar_unitary(4, rng)
    det = np.linalg.det(q)
    return q / det ** 0.25


def depolarizing_table(p: float, k: int):
    """(cumulative probabilities, Pauli strings) of the k-qubit depolarizing
    channel, identity first then ascending base-4 order."""
    n_terms = 4 ** k
    probs = [p / n_terms] * n_terms
    probs[0] = 1.0 - p + p / n_terms
    cum, acc = [], 0.0
    for q in probs:
        acc += q
        cum.append(acc)
    strings = []
    for t in range(n_terms):
        s, v = [], t
        for _ in range(k):
            s.append("IXYZ"[v % 4])
            v //= 4
        strings.append("".join(s))
    return cum, strings


def amplitude_damping(gamma: float):
    k0 = np.array([[1, 0], [0, math.sqrt(1 - gamma)]], dtype=np.complex128)
    k1 = np.array([[0, math.sqrt(gamma)], [0, 0]], dtype=np.complex128)
    return [k0, k1]


def pauli_as_kraus(cum, strings):
    """The same Pauli channel written as Kraus matrices sqrt(p_t) P_t
    (Section III-B-2: a Pauli model is a special case of a Kraus model)."""
    one = {"I": np.eye(2), "X": X, "Y": np.array([[0, -1j], [1j, 0]]), "Z": np.diag([1, -1])}
    mats, prev = [], 0.0
    for c, s in zip(cum, strings):
        p = c - prev
        prev = c
        m = np.ones((1, 1), dtype=np.complex128)
        for ch in s:  # digit j acts on qubits[j] = bit j of the matrix index
            m = np.kron(one[ch], m)
        mats.append(math.sqrt(max(p, 0.0)) * m)
    return mats


# ----------------------------------------------------------------------------
# circuit container
# ----------------------------------------------------------------------------
@dataclass
class Op:
    kind: int
    qubits: list
    mat: np.ndarray | None = None          # GATE
    cum: list | None = None                # PAULI
    strings: list | None = None            # PAULI
    kraus: list | None = None              # KRAUS; PGATE: one matrix per parameter set
    clbits: list | None = None             # MEASURE
    reset: int = 0                         # MEASURE
    cond_clbit: int = -1                   # GATE
    cond_val: int = 0


@dataclass
class Circuit:
    n_qubits: int
    n_clbits: int = 0
    ops: list = field(default_factory=list)
    name: str = ""

    # builders -----------------------------------------------------------
    def gate(self, qubits, mat, cond_clbit=-1, cond_val=0):
        mat = np.asarray(mat, dtype=np.complex128)
        assert mat.shape == (1 << len(qubits),) * 2
        self.ops.append(Op(GATE, list(qubits), mat=mat, cond_clbit=cond_clbit, cond_val=cond_val))
        return len(self.ops) - 1

    def pauli(self, qubits, cum, strings):
        assert len(cum) == len(strings) and all(len(s) == len(qubits) for s in strings)
        self.ops.append(Op(PAULI, list(qubits), cum=list(cum), strings=list(strings)))
        return len(self.ops) - 1

    def depolarizing(self, qubits, p):
        cum, strings = depolarizing_table(p, len(qubits))
        return self.pauli(qubits, cum, strings)

    def kraus(self, qubits, mats):
        mats = [np.asarray(m, dtype=np.complex128) for m in mats]
        self.ops.append(Op(KRAUS, list(qubits), kraus=mats))
        return len(self.ops) - 1

    def param_gate(self, qubits, mats):
        """A gate whose matrix depends on the shot's parameter set: mats[j]
        is the matrix of parameter set j (Section VI's parameter sweeps)."""
        mats = [np.asarray(m, dtype=np.complex128) for m in mats]
        assert all(m.shape == (1 << len(qubits),) * 2 for m in mats)
        self.ops.append(Op(PGATE, list(qubits), kraus=mats))
        return len(self.ops) - 1

    def measure(self, qubits, clbits, reset=0):
        assert len(qubits) == len(clbits)
        self.n_clbits = max(self.n_clbits, max(clbits) + 1)
        self.ops.append(Op(MEASURE, list(qubits), clbits=list(clbits), reset=int(reset)))
        return len(self.ops) - 1

    def final(self):
        self.ops.append(Op(FINAL, list(range(self.n_qubits))))
        return len(self.ops) - 1

    # summaries ---------------------------------------------------------
    @property
    def n_ops(self):
        return len(self.ops)

    def random_ops(self):
        return [i for i, o in enumerate(self.ops) if o.kind in RANDOM_KINDS]

    def counts_by_kind(self):
        out = {}
        for o in self.ops:
            out[KIND_NAMES[o.kind]] = out.get(KIND_NAMES[o.kind], 0) + 1
        return out

    # flattened struct-of-arrays op table --------------------------------
    def to_arrays(self) -> dict:
        n = len(self.ops)
        kind = np.zeros(n, np.int32)
        nq = np.zeros(n, np.int32)
        q_off = np.zeros(n, np.int32)
        cl_off = np.full(n, -1, np.int32)
        n_terms = np.zeros(n, np.int32)
        d_off = np.zeros(n, np.int64)
        s_off = np.full(n, -1, np.int32)
        cond_clbit = np.full(n, -1, np.int32)
        cond_val = np.zeros(n, np.int32)
        reset = np.zeros(n, np.int32)
        qubits, clbits, data, paulis = [], [], [], []
        for i, o in enumerate(self.ops):
            kind[i] = o.kind
            nq[i] = len(o.qubits)
            q_off[i] = len(qubits)
            qubits.extend(o.qubits)
            d_off[i] = len(data)
            if o.kind == GATE:
                n_terms[i] = 1
                data.extend(np.stack([o.mat.real, o.mat.imag], -1).reshape(-1).tolist())
                cond_clbit[i] = o.cond_clbit
                cond_val[i] = o.cond_val
            elif o.kind == PAULI:
                n_terms[i] = len(o.cum)
                data.extend(float(c) for c in o.cum)
                s_off[i] = len(paulis)
                for s in o.strings:
                    paulis.extend(s.encode())
            elif o.kind in (KRAUS, PGATE):
                n_terms[i] = len(o.kraus)
                for m in o.kraus:
                    data.extend(np.stack([m.real, m.imag], -1).reshape(-1).tolist())
            elif o.kind == MEASURE:
                cl_off[i] = len(clbits)
                clbits.extend(o.clbits)
                reset[i] = o.reset
        return dict(
            n_qubits=self.n_qubits, n_clbits=self.n_clbits, n_ops=n,
            kind=kind, nq=nq, q_off=q_off, cl_off=cl_off, n_terms=n_terms, d_off=d_off,
            s_off=s_off, cond_clbit=cond_clbit, cond_val=cond_val, reset=reset,
            qubits=np.asarray(qubits, np.int32).reshape(-1),
            clbits=np.asarray(clbits if clbits else [0], np.int32),
            data=np.asarray(data if data else [0.0], np.float64),
            paulis=np.frombuffer(bytes(paulis) if paulis else b"I", dtype=np.uint8).copy(),
        )


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
def brickwork(n, depth, p1, p2, seed, name=None):
    """Layer l: U3 (angles uniform in [0, 2 pi)) on every qubit, each followed
    by 1-qubit depolarizing p1; then CX on (0,1),(2,3),... for even l and
    (1,2),(3,4),... for odd l, each followed by 2-qubit depolarizing p2.
    Final measurement of every qubit."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=name or f"brickwork{n}x{depth}")
    for layer in range(depth):
        for q in range(n):
            th, ph, la = rng.uniform(0, 2 * math.pi, 3)
            c.gate([q], u3(th, ph, la))
            if p1 > 0:
                c.depolarizing([q], p1)
        start = layer % 2
        for a in range(start, n - 1, 2):
            c.gate([a, a + 1], cx())
            if p2 > 0:
                c.depolarizing([a, a + 1], p2)
    c.final()
    return c


def random_su4(n, depth, p, gamma, seed, name=None):
    """Each layer is a uniformly random perfect matching of the qubits with a
    Haar-random SU(4) on every pair.  After each gate: 2-qubit depolarizing p
    on the pair, then amplitude damping gamma on qubits[0], then on qubits[1]
    (each noise op is its own op ordinal).  Final measurement of every qubit."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=name or f"su4_{n}x{depth}")
    ad = amplitude_damping(gamma) if gamma > 0 else None
    for _ in range(depth):
        perm = rng.permutation(n)
        for j in range(0, n - 1, 2):
            a, b = int(perm[j]), int(perm[j + 1])
            c.gate([a, b], haar_su4(rng))
            if p > 0:
                c.depolarizing([a, b], p)
            if ad is not None:
                c.kraus([a], ad)
                c.kraus([b], ad)
    c.final()
    return c


def midcircuit_measure(n, rounds, p, meas_qubits, seed, name=None):
    """Each round: U3 on every qubit (angles uniform in [0, 2 pi)); CX ladder
    (0,1),(1,2),...,(n-2,n-1); depolarizing p after every U3 and CX; measure
    meas_qubits into classical bits 0..m-1; then X on each measured qubit,
    conditioned on its classical bit being 1 (a conditional reset).  Final
    measurement of every qubit."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=name or f"midmeas{n}x{rounds}")
    m = len(meas_qubits)
    for _ in range(rounds):
        for q in range(n):
            th, ph, la = rng.uniform(0, 2 * math.pi, 3)
            c.gate([q], u3(th, ph, la))
            if p > 0:
                c.depolarizing([q], p)
        for a in range(n - 1):
            c.gate([a, a + 1], cx())
            if p > 0:
                c.depolarizing([a, a + 1], p)
        c.measure(list(meas_qubits), list(range(m)))
        for j, q in enumerate(meas_qubits):
            c.gate([q], X, cond_clbit=j, cond_val=1)
    c.final()
    return c


def qft(n, p, seed=0, kraus=False, name=None):
    """Quantum Fourier transform written in U3 and CX (the paper's evaluation
    circuit, Section V), with depolarizing p after every 1- and 2-qubit gate,
    as a Pauli model or, with kraus=True, as the equivalent Kraus model.
    A controlled phase CP(t) on (a, b) is U1(t/2) a; U1(t/2) b; CX a,b;
    U1(-t/2) b; CX a,b.  The input is a seeded random basis state prepared by
    X gates so that the output is not trivial."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=name or f"qft{n}")

    def noise(qs):
        if p <= 0:
            return
        cum, strings = depolarizing_table(p, len(qs))
        if kraus:
            c.kraus(qs, pauli_as_kraus(cum, strings))
        else:
            c.pauli(qs, cum, strings)

    def g1(q, m):
        c.gate([q], m)
        noise([q])

    def g2(a, b, m):
        c.gate([a, b], m)
        noise([a, b])

    for q in range(n):
        if rng.integers(2):
            g1(q, X)
    for j in reversed(range(n)):
        g1(j, H)
        for k in reversed(range(j)):
            t = math.pi / 2 ** (j - k)
            g1(j, u3(0, 0, t / 2))
            g1(k, u3(0, 0, t / 2))
            g2(j, k, cx())
            g1(k, u3(0, 0, -t / 2))
            g2(j, k, cx())
    for q in range(n // 2):
        a, b = q, n - 1 - q
        g2(a, b, cx())
        g2(b, a, cx())
        g2(a, b, cx())
    c.final()
    return c


# The five reference workloads (Section V's single-GPU evaluation setting,
# restated as seeded synthetic circuits).
def config1():
    return brickwork(10, 20, 1e-3, 1e-2, seed=1, name="cfg1_brickwork10")


def config2():
    return random_su4(16, 16, 1e-2, 5e-3, seed=2, name="cfg2_su4_16")


def config3():
    return midcircuit_measure(20, 30, 5e-3, [0, 5, 10, 15], seed=3, name="cfg3_midmeas20")


def config4(seed=4, total_shots=100_000):
    """64 brickwork circuits, n ~ U{8..24}, depth ~ U{10..40}, p log-uniform in
    [1e-4, 1e-2] (1-qubit p, 2-qubit min(10 p, 1e-2)); shots split by
    Dirichlet(1) weights, rounded, at least 1 each, remainder to the largest."""
    rng = np.random.default_rng(seed)
    circs = []
    for i in range(64):
        n = int(rng.integers(8, 25))
        d = int(rng.integers(10, 41))
        p = float(10 ** rng.uniform(-4, -2))
        circs.append(brickwork(n, d, p, min(10 * p, 1e-2), seed=int(rng.integers(1 << 31)),
                               name=f"cfg4_{i}_n{n}d{d}"))
    w = rng.dirichlet(np.ones(64))
    shots = np.maximum(1, np.floor(w * total_shots).astype(np.int64))
    shots[int(np.argmax(shots))] += total_shots - int(shots.sum())
    return circs, shots.tolist()


def config5():
    return random_su4(28, 12, 1e-3, 1e-3, seed=5, name="cfg5_su4_28")


CONFIG_SHOTS = {1: 1000, 2: 10_000, 3: 10_000, 5: 2000}


def param_sweep(n, layers, n_sets, p, seed, name=None):
    """A variational-style circuit run for several parameter settings at
    once (Section VI): each layer is RY(theta_q) RZ(phi_q) on every qubit --
    one parameterized gate per qubit, its angles drawn uniformly in [0, 2 pi)
    independently for each of the n_sets parameter sets -- then CX on
    (0,1),(2,3),... for even layers and (1,2),(3,4),... for odd ones, with
    depolarizing p after every gate.  Final measurement of every qubit."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=name or f"sweep{n}x{layers}p{n_sets}")
    for layer in range(layers):
        for q in range(n):
            mats = []
            for _ in range(n_sets):
                th, ph = rng.uniform(0, 2 * math.pi, 2)
                ry = np.array([[math.cos(th / 2), -math.sin(th / 2)], [math.sin(th / 2), math.cos(th / 2)]])
                rz = np.diag([np.exp(-0.5j * ph), np.exp(0.5j * ph)])
                mats.append(rz @ ry)
            c.param_gate([q], mats)
            if p > 0:
                c.depolarizing([q], p)
        for a in range(layer % 2, n - 1, 2):
            c.gate([a, a + 1], cx())
            if p > 0:
                c.depolarizing([a, a + 1], p)
    c.final()
    return c

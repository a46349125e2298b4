"""Autotuner and learned cost model for run configurations.

The library's run-time decisions are exposed as batch options: batch or
shot-branching mode (the paper's trade-off, Section V-B and Section VI:
batching suits few qubits, branching more qubits, and the technique has to
be chosen per circuit), the fusion width of a pass (SV_OPT_MAX_ACTIVE), the
tile size (SV_OPT_TILE_BITS), the pass path (registers or shared-memory
tiles) and the joint decision of back-to-back Kraus ops.  The autotuner times every candidate on the GPU and
keeps the fastest; it writes every timing to a JSONL log.  The cost model
is a small MLP (sv_mlp_*, trained by the library's CUDA kernels) that
predicts log run time from circuit features and a candidate's encoding and
picks the argmin; the autotuner stays as its fallback (verify=k times the
model's k best candidates) and as the check on its picks.
"""
from __future__ import annotations

import argparse
import itertools
import json
import math
import os
import time

import numpy as np

from . import sv
from . import workloads as W

DEFAULT = dict(mode="branch", max_active=0, path=0, joint=1, tile=0)  # the library's defaults


def candidates():
    """Batch or branch mode x fusion width (0: the library's default, 4
    qubits in registers) x pass path x joint Kraus decisions x tile size
    (0: 2^11 amplitudes for complex64; 10: 2^10)."""
    out = []
    for mode, fuse, path, joint, tile in itertools.product(("batch", "branch"), (0, 3, 5, 8), (0, 1), (1, 0),
                                                           (0, 10)):
        out.append(dict(mode=mode, max_active=fuse, path=path, joint=joint, tile=tile))
    return out


def features(circ, shots):
    """Circuit-level features: size, op mix, and the expected number of
    random divergences (the quantity that decides batch vs branch)."""
    ops = circ.ops
    n_gates = sum(o.kind == W.GATE for o in ops)
    n2 = sum(o.kind == W.GATE and len(o.qubits) >= 2 for o in ops)
    n_pauli = sum(o.kind == W.PAULI for o in ops)
    n_kraus = sum(o.kind == W.KRAUS for o in ops)
    n_meas = sum(o.kind == W.MEASURE for o in ops)
    events = 0.0
    for o in ops:
        if o.kind == W.PAULI:
            events += 1.0 - o.cum[0]
        elif o.kind == W.KRAUS:
            # mean jump probability on the maximally mixed state
            d = 2 ** len(o.qubits)
            events += sum(float(np.real(np.trace(K.conj().T @ K))) for K in o.kraus[1:]) / d
        elif o.kind == W.MEASURE:
            events += 1.0
    return np.array([
        circ.n_qubits / 28.0,
        math.log2(max(shots, 1)) / 17.0,
        len(ops) / 1000.0,
        n_gates / 1000.0,
        n2 / max(n_gates, 1),
        n_pauli / 1000.0,
        n_kraus / 1000.0,
        n_meas / 100.0,
        math.log1p(events) / 5.0,
        math.log1p(events * shots) / 20.0,
    ], np.float32)


def encode(cfg, n_qubits):
    """The configuration as the model sees it: mode, the fusion width and
    tile size in effect for an n-qubit complex64 state, pass path, joint
    decisions."""
    tb = min(n_qubits, cfg.get("tile", 0) or 11)
    width = cfg["max_active"] or 4
    return np.array([1.0 if cfg["mode"] == "branch" else 0.0, width / 8.0, float(cfg["path"]),
                     float(cfg["joint"]), tb / 11.0], np.float32)


N_IN = 15


def measure(circ, shots, cfg, seed=1, reps=3, warmup=1):
    """Median wall time (ms) of sv_run_circuit under cfg, or None when the
    configuration does not fit the device."""
    mode = sv.SV_BATCH if cfg["mode"] == "batch" else sv.SV_BRANCH
    cs = sv.circuit_struct(circ.to_arrays())
    try:
        b = sv.Batch(circ.n_qubits, shots, max(1, circ.n_clbits), sv.SV_C64, mode, seed)
    except sv.SvError as e:
        if e.status == sv.SV_ENOMEM:
            return None
        raise
    try:
        b.set_option(sv.SV_OPT_TILE_BITS, cfg.get("tile", 0))
        b.set_option(sv.SV_OPT_MAX_ACTIVE, cfg["max_active"])
        b.set_option(sv.SV_OPT_PASS_PATH, cfg["path"])
        b.set_option(sv.SV_OPT_JOINT_KRAUS, cfg["joint"])
        for _ in range(warmup):
            b.run_circuit(cs, use_graph=True)
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            b.run_circuit(cs, use_graph=True)  # returns after the device finished
            ts.append(1e3 * (time.perf_counter() - t0))
        return float(np.median(ts))
    finally:
        b.close()


def autotune(circ, shots, cands=None, log=None, seed=1, reps=3):
    """Exhaustive search: time every candidate, return (best cfg, records)."""
    cands = cands or candidates()
    recs = []
    f = features(circ, shots)
    for cfg in cands:
        ms = measure(circ, shots, cfg, seed=seed, reps=reps)
        rec = dict(circuit=circ.name, n=circ.n_qubits, shots=shots, cfg=cfg, ms=ms, features=f.tolist())
        recs.append(rec)
        if log is not None:
            log.write(json.dumps(rec) + "\n")
            log.flush()
    ok = [r for r in recs if r["ms"] is not None]
    best = min(ok, key=lambda r: r["ms"])["cfg"]
    return best, recs


def dataset(records):
    rows = [r for r in records if r["ms"] is not None]
    X = np.stack([np.concatenate([np.asarray(r["features"], np.float32), encode(r["cfg"], r["n"])]) for r in rows])
    y = np.log(np.array([r["ms"] for r in rows], np.float32))
    return X, y


class CostModel:
    """MLP cost model on the library's CUDA kernels."""

    def __init__(self, hidden=64, seed=0, params=None):
        self.mlp = sv.MLP(N_IN, hidden)
        self.hidden = hidden
        if params is None:
            rng = np.random.default_rng(seed)
            H = hidden
            W1 = rng.standard_normal((H, N_IN)) * np.sqrt(2.0 / N_IN)
            W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
            w3 = rng.standard_normal(H) * np.sqrt(1.0 / H)
            params = np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3, [0.0]])
        self.mlp.set_params(params)
        self.mu = np.zeros(1, np.float32)
        self.n_max = 0  # largest qubit count in the training records (0: no limit)

    def fit(self, records, epochs=400, batch=32, lr=3e-3, seed=0):
        X, y = dataset(records)
        self.mu = np.array([y.mean()], np.float32)  # predict deviations from the mean log time
        self.n_max = max(int(r["n"]) for r in records if r["ms"] is not None)
        return self.mlp.train(X, y - self.mu[0], epochs=epochs, batch=min(batch, len(y)), lr=lr, seed=seed)

    def predict(self, circ, shots, cands=None):
        cands = cands or candidates()
        f = features(circ, shots)
        X = np.stack([np.concatenate([f, encode(c, circ.n_qubits)]) for c in cands])
        return np.exp(self.mlp.forward(X) + self.mu[0])

    def pick(self, circ, shots, cands=None, verify=0, seed=1):
        """argmin of the predicted time; with verify=k the k best predictions
        are timed on the GPU and the fastest is kept (autotuner fallback).
        A circuit wider than any the model was trained on gets the library's
        defaults: past its training range the model extrapolates from
        smaller states, where passes are cheap and nothing restarts."""
        cands = cands or candidates()
        if self.n_max and circ.n_qubits > self.n_max:
            return dict(DEFAULT)
        pred = self.predict(circ, shots, cands)
        order = np.argsort(pred)
        if verify <= 0:
            return cands[int(order[0])]
        timed = [(measure(circ, shots, cands[int(i)], seed=seed), cands[int(i)]) for i in order[:verify]]
        timed = [t for t in timed if t[0] is not None]
        return min(timed, key=lambda t: t[0])[1]

    def save(self, path):
        with open(path, "w") as f:
            json.dump({"hidden": self.hidden, "mu": float(self.mu[0]), "n_max": int(self.n_max),
                       "params": [float(x) for x in self.mlp.get_params()]}, f)

    @classmethod
    def load(cls, path=None):
        """A saved model; by default the one trained on this package's GB300
        timing log (data/tuner_log_gb300.jsonl)."""
        path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "cost_model_gb300.json")
        d = json.load(open(path))
        m = cls(hidden=int(d["hidden"]), params=np.asarray(d["params"], np.float32))
        m.mu = np.array([d["mu"]], np.float32)
        m.n_max = int(d.get("n_max", 0))
        return m


def training_circuits(seed=0, count=24, max_n=16):
    """Seeded mix of the workload families at modest sizes."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        fam = i % 3
        n = int(rng.integers(6, max_n + 1))
        shots = int(2 ** rng.integers(8, 12))
        s = int(rng.integers(1 << 30))
        if fam == 0:
            p = float(10 ** rng.uniform(-3.5, -1.5))
            c = W.brickwork(n, int(rng.integers(4, 12)), p, min(10 * p, 0.05), seed=s, name=f"t{i}_brick{n}")
        elif fam == 1:
            c = W.random_su4(n, int(rng.integers(3, 8)), float(10 ** rng.uniform(-3, -1.5)),
                             float(10 ** rng.uniform(-3.5, -2)), seed=s, name=f"t{i}_su4_{n}")
        else:
            mq = sorted(rng.choice(n, 2, replace=False).tolist())
            c = W.midcircuit_measure(n, int(rng.integers(2, 5)), float(10 ** rng.uniform(-3.5, -2)), mq, seed=s,
                                     name=f"t{i}_mid{n}")
        out.append((c, shots))
    return out


def main():
    ap = argparse.ArgumentParser(description="collect autotuner timings / train the cost model")
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("collect")
    a.add_argument("--out", required=True)
    a.add_argument("--count", type=int, default=24)
    a.add_argument("--seed", type=int, default=0)
    a.add_argument("--max-n", type=int, default=16)
    t = sub.add_parser("train")
    t.add_argument("--log", required=True)
    t.add_argument("--out", required=True)
    args = ap.parse_args()
    if args.cmd == "collect":
        with open(args.out, "w") as f:
            for c, shots in training_circuits(args.seed, args.count, args.max_n):
                best, _ = autotune(c, shots, log=f)
                print(c.name, shots, best, flush=True)
    else:
        recs = [json.loads(ln) for ln in open(args.log)]
        m = CostModel()
        loss = m.fit(recs)
        m.save(args.out)
        print("final loss", loss)


if __name__ == "__main__":
    main()

"""Host side of the autotuner and cost model, without a GPU: the candidate
set, the configuration encoding (which must follow the library's defaults)
and the circuit features, and the committed log and model files."""
import json
import os

import numpy as np

from paper_2308_03399_gb300 import tuner as T
from paper_2308_03399_gb300 import workloads as W


def test_candidates_cover_the_knobs():
    c = T.candidates()
    assert len(c) == 64 and len({json.dumps(x, sort_keys=True) for x in c}) == 64
    assert T.DEFAULT in c


def test_encoding_follows_the_library_defaults():
    # fusion width 0 means the library's default of 4 qubits at every size
    for n in (6, 10, 11, 20):
        e = T.encode(dict(T.DEFAULT), n)
        assert e.shape == (5,) and e[0] == 1.0 and e[1] == 4 / 8.0
        assert np.isclose(e[4], min(n, 11) / 11.0)
    e = T.encode(dict(T.DEFAULT, mode="batch", max_active=8, tile=10), 14)
    assert np.allclose(e[[0, 1, 4]], [0.0, 1.0, 10 / 11])  # float32 encoding


def test_features_grow_with_noise():
    a = T.features(W.brickwork(10, 6, 1e-3, 1e-2, seed=1), 1024)
    b = T.features(W.brickwork(10, 6, 1e-2, 1e-2, seed=1), 1024)
    assert a.shape == (10,) and b[8] > a[8] and b[9] > a[9]
    assert T.features(W.brickwork(10, 6, 1e-3, 1e-2, seed=1), 4096)[1] > a[1]


def test_committed_log_and_model():
    d = os.path.join(os.path.dirname(T.__file__), "data")
    recs = [json.loads(ln) for ln in open(os.path.join(d, "tuner_log_gb300.jsonl"))]
    assert len(recs) == 36 * 64 and all(r["ms"] is None or r["ms"] > 0 for r in recs)
    m = json.load(open(os.path.join(d, "cost_model_gb300.json")))
    H = m["hidden"]
    assert len(m["params"]) == H * T.N_IN + H + H * H + H + H + 1
    assert m["n_max"] == max(r["n"] for r in recs)
    X, y = T.dataset(recs)
    assert X.shape[1] == T.N_IN and np.all(np.isfinite(y))

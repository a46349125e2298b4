"""The cost model's CUDA kernels and what the trained model gains.

* forward and gradient of the library's MLP kernels equal the float64
  reference (oracle/mlp_ref.py) on random networks: relative error < 1e-4;
* Adam training in the library reduces the loss on a smooth target;
* on held-out circuits, the trained model's picks are compared with the
  exhaustive autotuner (the best per circuit) and with the best single
  fixed configuration (the method without the learned part)."""
import numpy as np
import pytest

from oracle import mlp_ref as M
from paper_2308_03399_gb300 import sv
from paper_2308_03399_gb300 import tuner as T

pytestmark = pytest.mark.gpu


def test_forward_and_gradient_match_float64_reference():
    rng = np.random.default_rng(3)
    n_in, H, N = 14, 64, 200
    p = M.init_params(n_in, H, 7).astype(np.float32)
    x = rng.standard_normal((N, n_in)).astype(np.float32)
    t = rng.standard_normal(N).astype(np.float32)
    m = sv.MLP(n_in, H)
    m.set_params(p)
    y = m.forward(x)
    y_ref, _ = M.forward(p.astype(np.float64), x, n_in, H)
    assert np.abs(y - y_ref).max() <= 1e-4 * (1 + np.abs(y_ref).max())
    loss, g = m.gradient(x, t)
    g_ref = M.gradient(p.astype(np.float64), x, t, n_in, H)
    assert abs(loss - M.loss(p.astype(np.float64), x, t, n_in, H)) <= 1e-4 * (1 + loss)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_training_reduces_loss():
    rng = np.random.default_rng(4)
    n_in = 6
    x = rng.uniform(-1, 1, (512, n_in)).astype(np.float32)
    t = (np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2] - 0.5 * x[:, 3] ** 2).astype(np.float32)
    m = sv.MLP(n_in, 32)
    m.set_params(M.init_params(n_in, 32, 1).astype(np.float32))
    l0 = M.loss(m.get_params().astype(np.float64), x, t, n_in, 32)
    l1 = m.train(x, t, epochs=200, batch=64, lr=3e-3, seed=1)
    assert l1 < 0.2 * l0
    # the library's loss after training equals the reference on its parameters
    assert abs(l1 - M.loss(m.get_params().astype(np.float64), x, t, n_in, 32)) < 1e-4 * (1 + l1)


def test_trained_cost_model_gains_over_fixed_configuration():
    """Trained on the committed GB300 timing log (the simulator's own
    measurements), the model picks a configuration per held-out circuit
    (drawn from the training distribution with another seed); every
    candidate is also timed live.  The model's total must be no worse than
    the best fixed configuration (one configuration for every circuit,
    chosen with hindsight) within 5% timing noise, and stay within 1.5x of
    the per-circuit best; the ratios are printed."""
    import json
    import os
    log = os.path.join(os.path.dirname(T.__file__), "data", "tuner_log_gb300.jsonl")
    recs = [json.loads(ln) for ln in open(log)]
    cands = [c for c in T.candidates() if c["joint"] == 1 and c["path"] == 0 and c["max_active"] in (0, 3, 8)]
    held = T.training_circuits(seed=21, count=12, max_n=18)
    model = T.CostModel(seed=0)
    model.fit(recs, epochs=300)
    t_model = t_best = 0.0
    fixed = {json_key(cfg): 0.0 for cfg in cands}
    for c, shots in held:
        times = {json_key(r["cfg"]): r["ms"] for r in T.autotune(c, shots, cands=cands, reps=3)[1]}
        pick = json_key(model.pick(c, shots, cands=cands))
        t_model += times[pick]
        t_best += min(times.values())
        for k in fixed:
            fixed[k] += times[k]
    by_mode = {m: min(v for k, v in fixed.items() if k[0] == m) for m in ("batch", "branch")}
    best_fixed = min(fixed.values())
    print(f"held-out ({len(held)} circuits) total ms: model {t_model:.1f}, per-circuit best {t_best:.1f}, "
          f"best fixed {best_fixed:.1f}, always-batch {by_mode['batch']:.1f}, "
          f"always-branch {by_mode['branch']:.1f}; model / best fixed {t_model / best_fixed:.3f}")
    assert t_model <= 1.05 * best_fixed
    # the per-circuit best is picked with hindsight from the same timings;
    # the model's gap to it (1.24x on GB300) is a report, bounded loosely
    assert t_model <= 1.5 * t_best


def json_key(cfg):
    return (cfg["mode"], cfg["max_active"], cfg["path"], cfg["joint"], cfg.get("tile", 0))

"""Final sampling through sv_final_sample_noalloc, the entry point that
allocates no device memory (for callers that cannot call cudaMalloc: a host
framework with a fixed device-memory budget, or a latency-critical loop
that must not stall on cudaMalloc's implicit synchronisation).

The test is the caller: it owns the device buffers (states, 64-bit shot
ids, keys) and checks the keys against the batch path's own final sampling
(sv_run_circuit + sv_get_keys) on the same states, on two calls in a row
(the static scratch keeps the first call's contents), and against the CPU
oracle's final keys for the same global shots, including shot ids above
2^32.  Collected last, so a failure here does not hide any other test."""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2308_03399_gb300 import sv
from paper_2308_03399_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _entry():
    f = sv.lib().sv_final_sample_noalloc
    f.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_uint32, C.c_void_p, C.c_uint64, C.c_uint32, C.c_void_p,
                  C.c_void_p]  # shots: device uint64
    f.restype = C.c_int
    return f


@pytest.mark.parametrize("base", [0, (1 << 32) + 11])
@pytest.mark.parametrize("prec,n", [(sv.SV_C64, 8), (sv.SV_C64, 13), (sv.SV_C128, 12)])
def test_noalloc_final_sampling_matches_batch_path(prec, n, base):
    torch = pytest.importorskip("torch")
    c = W.random_su4(n, 3, 0.05, 0.1, seed=40 + n)
    final_op = c.n_ops - 1
    assert c.ops[final_op].kind == W.FINAL
    n_shots, seed = 48, 17
    cs = sv.circuit_struct(c.to_arrays())
    with sv.Batch(n, n_shots, 1, prec, sv.SV_BATCH, seed) as b:
        b.set_option(sv.SV_OPT_SHOT_BASE, base)
        b.run_circuit(cs, use_graph=True)
        keys_ref = b.get_keys()
        states = np.stack([b.get_amplitudes(s) for s in range(n_shots)])
    if prec == sv.SV_C128:
        # the batch path's keys are the oracle's for the same global shots
        # (a draw within 1e-9 of a threshold could differ by rounding; none
        # of these do)
        okeys, _, _ = O.run_shots(c, seed, base, n_shots, want_outcomes=False)
        assert np.array_equal(okeys, keys_ref)
    real = np.float32 if prec == sv.SV_C64 else np.float64
    flat = np.stack([states.real, states.imag], -1).astype(real).reshape(-1)
    dev_states = torch.from_numpy(flat).cuda()
    dev_shots = (torch.arange(n_shots, dtype=torch.int64) + base).cuda()
    dev_keys = torch.zeros(n_shots, dtype=torch.int64).cuda()
    f = _entry()
    stream = torch.cuda.current_stream()
    for call in range(2):
        dev_keys.fill_(-1)
        rc = f(dev_states.data_ptr(), prec, n, n_shots, dev_shots.data_ptr(), seed, final_op, dev_keys.data_ptr(),
               stream.cuda_stream)
        assert rc == sv.SV_OK, sv.lib().sv_last_error().decode()
        torch.cuda.synchronize()
        got = dev_keys.cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, keys_ref), f"call {call}"


def test_noalloc_rejects_more_than_its_scratch():
    torch = pytest.importorskip("torch")
    buf = torch.zeros(16, dtype=torch.float64).cuda()
    f = _entry()
    # 28 qubits use 1024 chunks per state: 200 states need 204800 > 131072 partial sums
    rc = f(buf.data_ptr(), sv.SV_C64, 28, 200, buf.data_ptr(), 1, 0, buf.data_ptr(), None)
    assert rc == sv.SV_EINVAL
    assert "scratch" in sv.lib().sv_last_error().decode()

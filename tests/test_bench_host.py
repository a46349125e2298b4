"""Host-side pieces of bench.py, without a GPU: the workload names, and the
committed DRAM-traffic record that the headline line's `roofline.traffic`
is scaled from.  The record is keyed to the pass kernels' sources, so this
test fails when the kernels change and the record has not been captured
again."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


class _Args:
    workload, mode, prec, shots = "cfg2", "branch", "c64", 0


def test_traffic_record_matches_the_kernel_sources(bench):
    alg = 3.5e9
    t = bench.pass_traffic(_Args, alg)
    assert t is not None, "profiles/k_pass_traffic_cfg2_su4_16.txt is stale: capture it again"
    # DRAM traffic within a few percent of the algorithmic bytes: one read
    # and one write of every live state per pass, no re-reads
    assert 0.85 < t["traffic_over_algorithmic"] < 1.05
    assert t["bytes_per_launch"] == pytest.approx(alg * t["traffic_over_algorithmic"])


def test_traffic_record_applies_to_its_workload_only(bench):
    class Other(_Args):
        workload = "cfg3"
    assert bench.pass_traffic(Other, 1e9) is None

    class Fewer(_Args):
        shots = 2000
    assert bench.pass_traffic(Fewer, 1e9) is None


@pytest.mark.parametrize("name,n,shots", [("cfg1", 10, 1000), ("cfg2", 16, 10_000), ("cfg3", 20, 10_000),
                                          ("cfg5", 28, 2000), ("qft12", 12, 4000), ("qftk14", 14, 4000)])
def test_workload_names(bench, name, n, shots):
    circ, n_shots, _ = bench.workload(name)
    assert circ.n_qubits == n and n_shots == shots


def test_unknown_workload_is_rejected(bench):
    with pytest.raises(SystemExit):
        bench.workload("cfg9")

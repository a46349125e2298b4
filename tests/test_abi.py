"""The C ABI library builds, loads without a GPU, and exports every entry
point include/sv.h declares (no compute calls here)."""
import ctypes as C
import os
import re

from paper_2308_03399_gb300 import sv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sv_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sv_alloc_batch", "sv_apply_gate_batch", "sv_sample_noise", "sv_measure_batch", "sv_branch",
                     "sv_counts"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = C.CDLL(sv.lib()._name)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert set(declared_functions()) >= set(sv.exported_symbols())


def test_no_cpu_fallback_in_the_binding():
    # the binding loads libsv and nothing else: no import of the oracle
    src = open(os.path.join(ROOT, "paper_2308_03399_gb300", "sv.py")).read()
    assert "oracle" not in src.replace("no import of the oracle", "")


def test_binding_constants_match_the_header():
    # every enum value the header defines has the same value in the binding
    import re

    from paper_2308_03399_gb300 import sv
    header = open(os.path.join(ROOT, "include", "sv.h")).read()
    pairs = re.findall(r"\b(SV_(?:OPT|OP|C64|C128|PLAIN|BATCH|BRANCH|BATCH_BRANCH|NOISE)\w*)\s*=\s*(\d+)", header)
    assert len(pairs) >= 20
    for name, value in pairs:
        if hasattr(sv, name):
            assert getattr(sv, name) == int(value), name
    opts = [n for n, _ in pairs if n.startswith("SV_OPT_")]
    assert all(hasattr(sv, n) for n in opts), [n for n in opts if not hasattr(sv, n)]


def test_op_kinds_match_the_header():
    # the circuit writer's op kinds are the header's SV_OP_* codes
    from paper_2308_03399_gb300 import workloads as W
    header = open(os.path.join(ROOT, "include", "sv.h")).read()
    codes = dict((n, int(v)) for n, v in re.findall(r"\bSV_OP_(\w+)\s*=\s*(\d+)", header))
    assert codes == {"GATE": W.GATE, "PAULI": W.PAULI, "KRAUS": W.KRAUS, "MEASURE": W.MEASURE, "FINAL": W.FINAL,
                     "PGATE": W.PGATE}

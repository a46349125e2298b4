"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a temporary copy of oracle.c (never in the
committed file), builds it, and runs the pin tests against that build; the
pins must fail.  Mistakes: a dropped square root in the Kraus
renormalisation, a transposed gate matrix, a wrong sign in Y, an inverted
measurement projector, a swapped Philox multiplier, classical bits written
to the wrong position, the imaginary part dropped from the norm, and the
final sample taken one index late."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "kraus_no_sqrt": ("double scale = 1.0 / sqrt(chosen_p);", "double scale = 1.0 / chosen_p;"),
    "gate_transposed": ("acc += m[r * sub + c] * v[c];", "acc += m[c * sub + r] * v[c];"),
    "y_sign": ("case 'Y': m[1] = -I; m[2] = I; break;", "case 'Y': m[1] = I; m[2] = -I; break;"),
    "measure_projector": ("psi[j] = (bits == (uint64_t)o) ? psi[j] * scale : 0.0;",
                          "psi[j] = (bits != (uint64_t)o) ? psi[j] * scale : 0.0;"),
    "philox_multiplier": ("uint64_t prod0 = (uint64_t)0xD2511F53u * c0;", "uint64_t prod0 = (uint64_t)0xCD9E8D57u * c0;"),
    "clbit_position": ("clreg = (clreg & ~(1ull << cl[b])) | (bit << cl[b]);", "clreg = (clreg & ~(1ull << b)) | (bit << b);"),
    "norm_drops_imag": ("s += creal(psi[j]) * creal(psi[j]) + cimag(psi[j]) * cimag(psi[j]);",
                        "s += creal(psi[j]) * creal(psi[j]);"),
    "final_off_by_one": ("if (u < sum) { chosen = (int64_t)j; break; }", "if (u < before) { chosen = (int64_t)j; break; }"),
    "select_fallback_last_entry": ("        double prev = t ? cum[t - 1] : 0.0;\n        if (cum[t] > prev) return t;",
                                   "        return n - 1;"),
    "select_not_strict": ("        if (u < cum[t]) return t;", "        if (u <= cum[t]) return t;"),
    "kraus_fallback_last_entry": ("chosen = last_nonzero >= 0 ? last_nonzero : nt - 1;", "chosen = nt - 1;"),
    "kraus_not_strict": ("int take = (ov >= 0) ? (i == ov) : (u < sum);", "int take = (ov >= 0) ? (i == ov) : (u <= sum);"),
    "final_fallback_last_entry": ("if (chosen < 0) chosen = last_nonzero >= 0 ? last_nonzero : (int64_t)dim - 1;",
                                  "if (chosen < 0) chosen = (int64_t)dim - 1;"),
    "final_override_keeps_old_sums": ("if (ov >= 0 || u >= sum) {", "if (ov < 0 && u >= sum) {"),
    "pgate_ignores_set": ("load_matrix(d + (int64_t)pset * (int64_t)(2ull << (2 * k)), k, m);", "load_matrix(d, k, m);"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           str(mut), "-o", str(so), "-lm"])
    env = dict(os.environ, ORACLE_SO=str(so))
    pins = [os.path.join(ROOT, "tests", f) for f in
            ("test_oracle_philox.py", "test_oracle_gates.py", "test_oracle_noise.py", "test_oracle_dm.py",
             "test_oracle_fallbacks.py")]
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"

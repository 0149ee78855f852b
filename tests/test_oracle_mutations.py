"""Planted mistakes in the oracle must break at least one pin.

Each case copies oracle.c to a temporary directory, plants one plausible slip
(a sign, a dropped term, a wrong index, a transposed operand), compiles it and
runs the pin suite against the mutant through ORACLE_LIB_OVERRIDE.  The pin
suite must fail.  Everything here runs on the CPU.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "rhs_sign": ("if (i > 0) bk += dy[k - W] * vn;", "if (i > 0) bk -= dy[k - W] * vn;"),
    "diag_term_dropped": ("data[nnz] = uw + ue + vn + vs;", "data[nnz] = uw + ue + vs;"),
    "weight_exponent": ("pow(fabs(resid), 2.0 - p)", "pow(fabs(resid), p)"),
    "ilu_no_pivot_division": ("P->fact[pk] /= P->fact[P->dpos[k]];", ";"),
    "residual_update_operand": ("r[t] = r[t] - alpha * q[t];", "r[t] = r[t] - alpha * d[t];"),
    "dct_transposed": ("acc += P->tmp[(long)i * W + l] * P->cw[(long)l * W + j];",
                       "acc += P->tmp[(long)i * W + l] * P->cw[(long)j * W + l];"),
    "dy_wrong_neighbour": ("orc_wrap(psi[k + W] - psi[k])", "orc_wrap(psi[k + 1] - psi[k])"),
    "wrap_tie_break": ("double k = ceil((x - ORC_PI) / (2.0 * ORC_PI));",
                       "double k = floor((x + ORC_PI) / (2.0 * ORC_PI));"),
    "ssor_missing_scaling": ("for (int i = 0; i < P->n; ++i) s[i] = (P->diag[i] / w) * s[i];", ";"),
    "beta_inverted": ("double beta = delta_new / delta_old;", "double beta = delta_old / delta_new;"),
    "ic_missing_sqrt": ("P->fact[P->dpos[i]] = sqrt(orc_guard_pivot(", "P->fact[P->dpos[i]] = (orc_guard_pivot("),
    "weight_tau_misplaced": ("return tau / (pow(fabs(resid), 2.0 - p) + tau);",
                             "return tau / (pow(fabs(resid), 2.0 - p) + 1.0);"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    (tmp_path / "oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "oracle", "oracle.h"), tmp_path / "oracle.h")
    so = tmp_path / "mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(tmp_path / "oracle.c"), "-lm"])
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"

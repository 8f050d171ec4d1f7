"""Plant plausible mistakes in copies of the oracle and check that the pins catch each one.

Every mutant is a textual edit of oracle/xref.c compiled into a temporary
library (the committed oracle is never changed).  A mutant "survives" if all
pins still pass on it; the test requires that none survives.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
from tests import pins

SRC = open(os.path.join(os.path.dirname(oracle.__file__), "xref.c")).read()

MUTANTS = {
    # assembly (Eqs. 1-7)
    "drop_sense_conductance": ("band_add(ab, p, u, u, go);", ";"),
    "wrong_sign_wl_coupling": ("band_add(ab, p, w, idx_wl(N, i, j + 1), -gw);",
                               "band_add(ab, p, w, idx_wl(N, i, j + 1), gw);"),
    "bl_coupling_wrong_row": ("band_add(ab, p, u, idx_bl(N, i + 1, j), -gb);",
                              "band_add(ab, p, u, idx_bl(N, i, j), -gb);"),
    "transposed_G": ("const double g = G[(size_t)i * N + j];",
                     "const double g = G[(size_t)j * M + i];"),
    "source_uses_wire_R": ("band_add(ab, p, w, w, gs);", "band_add(ab, p, w, w, gw);"),
    "wl_bl_swapped_in_ordering": ("static size_t idx_bl(int N, int i, int j) { return idx_wl(N, i, j) + 1; }",
                                  "static size_t idx_bl(int N, int i, int j) { return idx_wl(N, i, j) + 2; }"),
    # right-hand side
    "rhs_scaled_by_R": ("= V[(size_t)b * M + i] / Rs;", "= V[(size_t)b * M + i] * Rs;"),
    # LU (Sec. II-C)
    "lu_short_band": ("const long long last = (r + p < k - 1) ? r + p : k - 1;",
                      "const long long last = (r + p - 1 < k - 1) ? r + p - 1 : k - 1;"),
    "lu_multiplier_not_stored": ("row_i[col_r_in_i] = l;", "row_i[col_r_in_i] = a;"),
    # substitution (Sec. II-C)
    "back_subst_no_divide": ("y[i] = s / row[p];", "y[i] = s;"),
    "forward_subst_wrong_sign": ("s -= row[c - i + p] * y[c];\n      y[i] = s;\n    }\n    for",
                                 "s += row[c - i + p] * y[c];\n      y[i] = s;\n    }\n    for"),
    # extraction
    "current_from_top_row": ("I[(size_t)b * N + j] = xb[idx_bl(N, M - 1, j)] / Rsense;",
                             "I[(size_t)b * N + j] = xb[idx_bl(N, 0, j)] / Rsense;"),
    "voltages_transposed": ("const size_t o = ((size_t)b * M + i) * N + j;",
                            "const size_t o = ((size_t)b * N + j) * M + i;"),
    "voltages_wl_bl_swapped": ("if (vWL) vWL[o] = xb[idx_wl(N, i, j)];", "if (vWL) vWL[o] = xb[idx_bl(N, i, j)];"),
}


def _compile(tmp_path, name, src):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
                    "-o", str(so), str(c), "-lm"], check=True)
    return oracle._bind(ctypes.CDLL(str(so)))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    assert SRC.count(old) == 1, f"mutation site for {name} not found exactly once"
    lib = _compile(tmp_path, name, SRC.replace(old, new))
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin()
        except (AssertionError, ZeroDivisionError, ValueError, FloatingPointError,
                __import__("numpy").linalg.LinAlgError):
            caught.append(pin.__name__)
    assert caught, f"mutant {name} survived every pin"

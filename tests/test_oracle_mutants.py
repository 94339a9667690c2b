"""The oracle's pins must catch plausible mistakes.

Each mutant below is a copy of oracle.c with one planted slip (on the CPU,
never on a GPU).  The pin suite is run against every mutant in a subprocess
and must fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "lu_style_update_skips_rows_above": ("if (i == r) continue;", "if (i <= r) continue;"),
    "wrong_sign_in_update": ("uint64_t negf = p - f;", "uint64_t negf = f;"),
    "wrong_inverse_exponent": ("(uint64_t)p - 2, p)", "(uint64_t)p - 3, p)"),
    "row_swap_dropped": ("if (q != r) {", "if (0) {"),
    "pivot_column_not_cleared": ("for (int64_t j = c; j < n; j++)\n            row[j]",
                                 "for (int64_t j = c + 1; j < n; j++)\n            row[j]"),
    "consistency_reads_wrong_rows": ("for (int64_t i = r; i < m; i++)\n            if (M[",
                                     "for (int64_t i = r + 1; i < m; i++)\n            if (M["),
    "pivot_search_from_row_zero": ("for (int64_t i = r; i < C->m; i++) {",
                                   "for (int64_t i = 0; i < C->m; i++) {"),
    "solution_read_from_wrong_column": ("X[(int64_t)pivots[t] * ldx + j] = M[t * ld + nA + j];",
                                        "X[(int64_t)t * ldx + j] = M[t * ld + nA + j];"),
}

# planted slips in the construction and product routines, caught by the
# construction pins
CONSTRUCTION_MUTANTS = {
    "load_matrix_index_not_looked_up": ("v = (v * (uint64_t)bases[r * ldb + lindices[c * d + t]]) % p;",
                                        "v = (v * (uint64_t)bases[r * ldb + t % n_basis]) % p;"),
    "load_matrix_last_factor_dropped": ("for (int64_t t = 0; t < d; t++)\n                v = (v",
                                        "for (int64_t t = 1; t < d; t++)\n                v = (v"),
    "matmul_transposed_operand": ("(uint64_t)B[k * ldb + j]) % p) % p;", "(uint64_t)B[j * ldb + k]) % p) % p;"),
    "matmul_inner_loop_short": ("for (int64_t k = 0; k < K; k++)\n                s = (s",
                                "for (int64_t k = 1; k < K; k++)\n                s = (s"),
}

# planted slips in the 64-bit elimination, caught by its own pins
MUTANTS64 = {
    "o64_row_swap_dropped": ("for (int64_t j = 0; q != r && j < C->n; j++) {",
                             "for (int64_t j = 0; 0 && j < C->n; j++) {"),
    "o64_product_wraps_at_64_bits": ("(o_u128)minus_f * A[prow * ld + j];",
                                     "(o_u128)(minus_f * A[prow * ld + j]);"),
    "o64_update_skips_rows_above": ("if (i == prow || f == 0) continue;", "if (i <= prow || f == 0) continue;"),
    "o64_wrong_inverse_exponent": ("return o64_pow(h, p - 2, p);", "return o64_pow(h, p - 3, p);"),
    "o64_solution_read_into_wrong_row": ("X[pivots[t] * ldx + j] = M[t * ld + nA + j];",
                                         "X[t * ldx + j] = M[t * ld + nA + j];"),
    "o64_square_reduced_at_64_bits": ("return (uint64_t)(((o_u128)a * (o_u128)b) % p);",
                                      "return (uint64_t)((a * b) % p);"),
}

# planted slips in the LUP factorisation, caught by its pins
LUP_MUTANTS = {
    "lup_multiplier_not_divided_by_head": ("const uint64_t l = (f * hinv) % p;", "const uint64_t l = f % p;"),
    "lup_reduces_earlier_pivot_rows": ("if (is_pivot[i] || i == q) continue;", "if (i == q) continue;"),
    "lup_pivot_is_last_candidate": ("if (!is_pivot[i] && W[i * n + c] != 0) { q = i; break; }",
                                    "if (!is_pivot[i] && W[i * n + c] != 0) { q = i; }"),
    "lup_other_rows_reversed": ("for (int64_t i = 0; i < m; i++)\n        if (!is_pivot[i]) perm[t++]",
                                "for (int64_t i = m - 1; i >= 0; i--)\n        if (!is_pivot[i]) perm[t++]"),
}

PIN_FILES = {**{k: "test_oracle_pins.py" for k in MUTANTS},
             **{k: "test_oracle_lup.py" for k in LUP_MUTANTS},
             **{k: "test_oracle_construction.py" for k in CONSTRUCTION_MUTANTS},
             **{k: "test_oracle64_pins.py" for k in MUTANTS64}}


@pytest.mark.parametrize("name", sorted(PIN_FILES))
def test_pins_fail_on_mutant(name, tmp_path):
    before, after = {**MUTANTS, **CONSTRUCTION_MUTANTS, **MUTANTS64, **LUP_MUTANTS}[name]
    pins = PIN_FILES[name]
    src = open(SRC).read()
    assert src.count(before) == 1, f"mutation site for {name} not found exactly once"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(before, after))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", str(lib), str(mut)],
                   check=True)
    env = dict(os.environ, ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"

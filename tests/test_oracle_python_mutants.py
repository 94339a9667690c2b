"""The pins must also catch plausible mistakes in the oracle's Python-level
routines (section 5.1's null space and rank factor, for both residue widths,
and section 3.3's template evaluation), which the C mutant harness does not
reach.

Each mutant replaces one routine of the ``oracle`` module for the duration of
the test (on the CPU), and the pin tests that use it are run directly; at
least one of their cases must fail.
"""
import numpy as np
import pytest

import oracle
import test_oracle64_pins as pins64
import test_oracle_construction as pinsc
import test_oracle_pins as pins

_real_null_space = oracle.null_space
_real_null_space64 = oracle.null_space64
_real_rank_factor = oracle.rank_factor
_real_rank_factor64 = oracle.rank_factor64
_real_eval_template = oracle.eval_template


def _free_cols(n, pivots):
    return [c for c in range(n) if c not in {int(x) for x in pivots}]


def null_space_free_plus_one(R, pivots, p):
    K = _real_null_space(R, pivots, p).copy()
    for q, f in enumerate(_free_cols(np.asarray(R).shape[1], pivots)):
        K[f, q] = 1                                    # +1 instead of -1
    return K


def null_space_pivot_rows_negated(R, pivots, p):
    K = _real_null_space(R, pivots, p).astype(np.uint64)
    for c in pivots:
        K[int(c)] = (p - K[int(c)]) % p                # -R[t][f] instead of R[t][f]
    return K.astype(np.uint32)


def null_space64_free_plus_one(R, pivots, p):
    K = _real_null_space64(R, pivots, p).copy()
    for q, f in enumerate(_free_cols(np.asarray(R).shape[1], pivots)):
        K[f, q] = 1
    return K


def null_space64_pivot_rows_from_wrong_row(R, pivots, p):
    K = _real_null_space64(R, pivots, p).copy()
    Rm = np.asarray(R, dtype=np.uint64)
    for q, f in enumerate(_free_cols(Rm.shape[1], pivots)):
        for t, c in enumerate(pivots):
            K[int(c), q] = Rm[(t + 1) % max(len(pivots), 1), f]   # off-by-one pivot row
    return K


def rank_factor_leading_columns(A, pivots):
    A = np.asarray(A)
    return np.ascontiguousarray(A[:, :len(pivots)]).astype(A.dtype)   # not the pivot columns


def rank_factor64_leading_columns(A, pivots):
    A = np.asarray(A, dtype=np.uint64)
    return np.ascontiguousarray(A[:, :len(pivots)])


def eval_template_exponents_swapped(points, coefs, monomials, mask, p):
    return _real_eval_template(points, coefs, [(b, a) for (a, b) in monomials], mask, p)


def _cases_null_rank32():
    for p in (5, 2**31 - 1):
        for sr in ((6, 9, 4), (9, 6, 6), (8, 8, 3), (5, 5, 0)):
            yield lambda p=p, sr=sr: pinsc.test_rank_factorisation_and_null_space(p, sr)
    for p in (3, 5):
        for seed in range(5):
            yield lambda p=p, seed=seed: pins.test_null_space_bruteforce(p, seed)


def _cases_null_rank64():
    for p in (5, 2**32 + 15, 2**64 - 59):
        for mnr in ((9, 14, 5), (14, 9, 9), (10, 10, 0), (12, 12, 12)):
            yield lambda p=p, mnr=mnr: pins64.test_null_space_and_rank_factor(mnr, p)


def _cases_template():
    for p in (7, 2**31 - 1):
        yield lambda p=p: pinsc.test_eval_template_direct(p)


MUTANTS = {
    "null_space_free_plus_one": ("null_space", null_space_free_plus_one, _cases_null_rank32),
    "null_space_pivot_rows_negated": ("null_space", null_space_pivot_rows_negated, _cases_null_rank32),
    "rank_factor_leading_columns": ("rank_factor", rank_factor_leading_columns, _cases_null_rank32),
    "null_space64_free_plus_one": ("null_space64", null_space64_free_plus_one, _cases_null_rank64),
    "null_space64_pivot_rows_from_wrong_row": ("null_space64", null_space64_pivot_rows_from_wrong_row,
                                               _cases_null_rank64),
    "rank_factor64_leading_columns": ("rank_factor64", rank_factor64_leading_columns, _cases_null_rank64),
    "eval_template_exponents_swapped": ("eval_template", eval_template_exponents_swapped, _cases_template),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_fail_on_python_mutant(name, monkeypatch):
    attr, mutant, cases = MUTANTS[name]
    monkeypatch.setattr(oracle, attr, mutant)
    failures = 0
    for case in cases():
        try:
            case()
        except (AssertionError, IndexError, ValueError):
            failures += 1
    assert failures > 0, f"pins did not catch mutant {name}"


def test_pins_pass_on_the_real_routines():
    """The same cases pass with the oracle as it stands (so a failure above
    is the mutant's doing)."""
    for cases in (_cases_null_rank32, _cases_null_rank64, _cases_template):
        for case in cases():
            case()

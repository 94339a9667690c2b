"""CPU checks of the C ABI: the library loads, exports every entry point
that include/linac.h declares, and rejects bad arguments on the host
(argument checks run before any CUDA call)."""
import ctypes

import pytest

from paper_2605_25863_gb300 import build, linac


@pytest.fixture(scope="module")
def lib():
    build.build()
    return linac.lib()


def test_every_declared_symbol_is_exported(lib):
    syms = linac.header_symbols()
    assert {"linac_rref", "linac_solve", "linac_rref_batched", "linac_workspace_bytes"} <= set(syms)
    for s in syms:
        assert hasattr(lib, s), f"{s} declared in include/linac.h but not exported"


def test_probes_live_in_their_own_library(lib):
    """The pipe-rate probes are measurement tooling: exported by
    liblinac_probes.so, not by liblinac.so."""
    assert not hasattr(lib, "linac_measure_int_rates")
    assert not hasattr(lib, "linac_probe_int_rates")
    probes = ctypes.CDLL(build.PROBES_LIB)
    assert hasattr(probes, "linac_probe_int_rates")


def test_build_targets_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings_and_version(lib):
    assert lib.linac_version() >= 100
    for code in range(9):
        assert lib.linac_status_string(code)


@pytest.mark.parametrize("p", [0, 1, 2, 4, 9, 561, 2047, 3277, 4033, 25326001, 2**31, 2**31 + 11,
                               2**32 - 1, 2**31 - 3])
def test_non_primes_and_out_of_range_primes_rejected(lib, p):
    rank = ctypes.c_int32()
    piv = (ctypes.c_int32 * 4)()
    code = lib.linac_rref(None, 0, 0, 4, p, ctypes.byref(rank), piv, None)
    assert code == 2   # LINAC_ERR_PRIME


@pytest.mark.parametrize("m,n,ld,code", [(-1, 4, 4, 1), (4, -1, 4, 1), (4, 8, 4, 1), (4, 5, 6, 3)])
def test_shape_and_alignment_rejected(lib, m, n, ld, code):
    rank = ctypes.c_int32()
    piv = (ctypes.c_int32 * 8)()
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: rejected before any CUDA call
    assert lib.linac_rref(fake, m, n, ld, 2**31 - 1, ctypes.byref(rank), piv, None) == code


def test_misaligned_pointer_rejected(lib):
    rank = ctypes.c_int32()
    piv = (ctypes.c_int32 * 8)()
    assert lib.linac_rref(ctypes.c_void_p(0x1004), 4, 4, 4, 2**31 - 1, ctypes.byref(rank), piv, None) == 3


def test_bad_options_rejected(lib):
    rank = ctypes.c_int32()
    piv = (ctypes.c_int32 * 8)()
    for path, nb in ((5, 0), (-1, 0), (0, 20), (0, 256)):
        o = linac.Options(path, nb, 0, 0)
        assert lib.linac_rref_ex(ctypes.c_void_p(0x1000), 4, 4, 4, 2**31 - 1, 4, ctypes.byref(rank), piv,
                                 ctypes.byref(o), None) == 1


def test_batched_rejects_oversize(lib):
    code = lib.linac_rref_batched(ctypes.c_void_p(0x1000), ctypes.c_void_p(0x1000), ctypes.c_void_p(0x1000),
                                  ctypes.c_void_p(0x1000), ctypes.c_void_p(0x1000), None, 3, 10, 2000,
                                  2**31 - 1, 0, ctypes.c_void_p(0x1000), ctypes.c_void_p(0x1000),
                                  ctypes.c_void_p(0x1000), None, None)
    assert code == 8   # LINAC_ERR_UNSUPPORTED


def test_construction_and_derived_entry_points_check_arguments(lib):
    """linac_load_matrix, linac_matmul, linac_null_space, linac_rank_factor:
    host-side rejections happen before any CUDA call."""
    fake = ctypes.c_void_p(0x1000)
    P = 2**31 - 1
    # load_matrix: negative sizes, ld too small, d < 0, bad prime
    assert lib.linac_load_matrix(fake, -1, 3, 3, fake, 4, 2, P, fake, 4, None) == 1
    assert lib.linac_load_matrix(fake, 2, 3, 2, fake, 4, 2, P, fake, 4, None) == 1
    assert lib.linac_load_matrix(fake, 2, 3, 3, fake, 4, -1, P, fake, 4, None) == 1
    assert lib.linac_load_matrix(fake, 2, 3, 3, fake, 4, 2, 15, fake, 4, None) == 2
    # matmul: inner/leading dimensions, null output, bad prime
    assert lib.linac_matmul(fake, 2, 3, 2, fake, 4, 4, P, fake, 4, None) == 1
    assert lib.linac_matmul(fake, 2, 3, 3, fake, 4, 4, P, None, 4, None) == 1
    assert lib.linac_matmul(fake, 2, 3, 3, fake, 4, 4, 2**31, fake, 4, None) == 2
    # null space: ldK < kcols, missing outputs, bad prime
    assert lib.linac_null_space(fake, 3, 4, 4, fake, fake, P, fake, 4, 2, fake, fake, None) == 1
    assert lib.linac_null_space(fake, 3, 4, 4, fake, fake, P, fake, 4, 4, None, fake, None) == 1
    assert lib.linac_null_space(fake, 3, 4, 4, fake, fake, 9, fake, 4, 4, fake, fake, None) == 2
    # rank factor: ld < n, ldC < ccols
    assert lib.linac_rank_factor(fake, 3, 4, 3, fake, fake, fake, 3, 4, None) == 1
    assert lib.linac_rank_factor(fake, 3, 4, 4, fake, fake, fake, 3, 2, None) == 1


# composites a weak 64-bit prime test would pass: Carmichael numbers, strong
# pseudoprimes to the bases 2..23 (3825123056546413051) and to 2, 3, 5, 7
# (3215031751), even numbers, 2^64 - 1, and the Fermat number 2^32 + 1
@pytest.mark.parametrize("p", [0, 1, 2, 4, 9, 561, 3215031751, 3825123056546413051, 2**32 + 1, 2**63,
                               2**64 - 1, 2**61 + 1, (2**31 - 1) * (2**31 + 11)])
def test_uint64_entry_points_reject_composites(lib, p):
    rank = ctypes.c_int32()
    piv = (ctypes.c_int32 * 4)()
    fake = ctypes.c_void_p(0x1000)
    assert lib.linac_rref64(None, 0, 0, 2, p, ctypes.byref(rank), piv, None) == 2
    assert lib.linac_solve64(fake, 4, 4, 4, fake, 2, 2, p, fake, 2, fake, ctypes.byref(rank), piv, None) == 2


def test_uint64_entry_points_check_shapes_alignment_and_options(lib):
    rank = ctypes.c_int32()
    piv = (ctypes.c_int32 * 8)()
    fake = ctypes.c_void_p(0x1000)
    P = 2**64 - 59
    assert lib.linac_rref64(fake, 4, 5, 5, P, ctypes.byref(rank), piv, None) == 3       # odd ld
    assert lib.linac_rref64(ctypes.c_void_p(0x1008), 4, 4, 4, P, ctypes.byref(rank), piv, None) == 3
    assert lib.linac_rref64(fake, -1, 4, 4, P, ctypes.byref(rank), piv, None) == 1
    assert lib.linac_rref64(fake, 4, 6, 4, P, ctypes.byref(rank), piv, None) == 1       # ld < n
    assert lib.linac_rref64(fake, 4, 4, 4, P, None, piv, None) == 1
    assert lib.linac_rref64_ex(fake, 4, 4, 4, P, 5, ctypes.byref(rank), piv, None, None) == 1
    for path, nb in ((1, 0), (2, 0), (0, 32)):
        o = linac.Options(path, nb, 0, 0)
        assert lib.linac_rref64_ex(fake, 4, 4, 4, P, 4, ctypes.byref(rank), piv, ctypes.byref(o), None) == 1
    cons = ctypes.c_void_p(0x2000)
    assert lib.linac_solve64(fake, 4, 4, 4, fake, 2, 2, P, fake, 1, cons, ctypes.byref(rank), piv, None) == 1
    assert lib.linac_solve64(fake, 4, 4, 4, fake, 2, 2, P, fake, 2, None, ctypes.byref(rank), piv, None) == 1
    assert lib.linac_solve64(fake, 4, 4, 5, fake, 2, 2, P, fake, 2, cons, ctypes.byref(rank), piv, None) == 3
    assert lib.linac_workspace64_bytes(-1, 4) == 0
    assert lib.linac_workspace64_bytes(100, 200) >= 32 * (3 * 128 + 256) * 8


def test_uint64_derived_entry_points_check_arguments(lib):
    fake = ctypes.c_void_p(0x1000)
    P = 2**64 - 59
    assert lib.linac_null_space64(fake, 3, 4, 4, fake, fake, P, fake, 4, 2, fake, fake, None) == 1   # ldK < kcols
    assert lib.linac_null_space64(fake, 3, 4, 4, fake, fake, P, fake, 4, 4, None, fake, None) == 1
    assert lib.linac_null_space64(fake, 3, 4, 4, fake, fake, 2**64 - 1, fake, 4, 4, fake, fake, None) == 2
    assert lib.linac_rank_factor64(fake, 3, 4, 3, fake, fake, fake, 3, 4, None) == 1             # ld < n
    assert lib.linac_rank_factor64(fake, 3, 4, 4, fake, fake, fake, 3, 2, None) == 1             # ldC < ccols

"""Thin ctypes binding of the C ABI in include/linac.h.

Every function marshals torch CUDA tensors into device pointers, calls the
entry point of the same name in liblinac.so and turns a nonzero status into
``LinacError``.  There is no fallback: if the library is missing, every call
raises.  Matrices are 2-D int32 (or uint32) CUDA tensors holding residues in
[0, p), row-major with a row stride that is a multiple of 4 elements.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

LINAC_PATH_AUTO, LINAC_PATH_PLAIN, LINAC_PATH_LIMB, LINAC_PATH_CRT, LINAC_PATH_HYBRID = 0, 1, 2, 3, 4
LINAC_SHARED_PATTERN = 1
_PATHS = {"auto": LINAC_PATH_AUTO, "plain": LINAC_PATH_PLAIN, "limb": LINAC_PATH_LIMB, "crt": LINAC_PATH_CRT,
          "hybrid": LINAC_PATH_HYBRID}


class LinacError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        name = lib().linac_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: status {code} ({name})")


class Options(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("nb", ctypes.c_int32),
                ("validate", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double)]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load liblinac.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        vp, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        L.linac_rref.argtypes = [vp, i64, i64, i64, u32, vp, vp, vp]
        L.linac_rref_ex.argtypes = [vp, i64, i64, i64, u32, i64, vp, vp, ctypes.POINTER(Options), vp]
        L.linac_solve.argtypes = [vp, i64, i64, i64, vp, i64, i64, u32, vp, i64, vp, vp, vp, vp]
        L.linac_solve_ex.argtypes = [vp, i64, i64, i64, vp, i64, i64, u32, vp, i64, vp, vp, vp,
                                     ctypes.POINTER(Options), vp]
        L.linac_rref_batched.argtypes = [vp, vp, vp, vp, vp, vp, i32, i32, i32, u32, u32, vp, vp, vp,
                                         vp, vp]
        L.linac_workspace_bytes.argtypes = [i64, i64, ctypes.POINTER(Options)]
        L.linac_workspace_bytes.restype = ctypes.c_size_t
        L.linac_last_device_status.argtypes = [vp]
        L.linac_status_string.argtypes = [ctypes.c_int]
        L.linac_status_string.restype = ctypes.c_char_p
        L.linac_version.argtypes = []
        L.linac_profile_enable.argtypes = [ctypes.c_int]
        L.linac_profile_enable.restype = None
        L.linac_profile_reset.argtypes = []
        L.linac_profile_reset.restype = None
        L.linac_profile_read.argtypes = [ctypes.POINTER(ProfileEntry), ctypes.c_int]
        L.linac_profile_read.restype = ctypes.c_int
        L.linac_batched_tune.argtypes = [ctypes.c_uint32, ctypes.c_void_p, vp]
        L.linac_batched_tune.restype = ctypes.c_int
        L.linac_batched_panel_widths.argtypes = [ctypes.c_void_p]
        L.linac_batched_panel_widths.restype = ctypes.c_int
        L.linac_batched_set_panel_widths.argtypes = [ctypes.c_void_p]
        L.linac_batched_set_panel_widths.restype = ctypes.c_int
        L.linac_launch_count.argtypes = []
        L.linac_launch_count.restype = ctypes.c_longlong
        L.linac_load_matrix.argtypes = [vp, i64, i64, i64, vp, i64, i32, u32, vp, i64, vp]
        L.linac_matmul.argtypes = [vp, i64, i64, i64, vp, i64, i64, u32, vp, i64, vp]
        L.linac_null_space.argtypes = [vp, i64, i64, i64, vp, vp, u32, vp, i64, i64, vp, vp, vp]
        L.linac_rank_factor.argtypes = [vp, i64, i64, i64, vp, vp, vp, i64, i64, vp]
        u64 = ctypes.c_uint64
        L.linac_rref64.argtypes = [vp, i64, i64, i64, u64, vp, vp, vp]
        L.linac_rref64_ex.argtypes = [vp, i64, i64, i64, u64, i64, vp, vp, ctypes.POINTER(Options), vp]
        L.linac_solve64.argtypes = [vp, i64, i64, i64, vp, i64, i64, u64, vp, i64, vp, vp, vp, vp]
        L.linac_null_space64.argtypes = [vp, i64, i64, i64, vp, vp, u64, vp, i64, i64, vp, vp, vp]
        L.linac_rank_factor64.argtypes = [vp, i64, i64, i64, vp, vp, vp, i64, i64, vp]
        L.linac_lup.argtypes = [vp, i64, i64, i64, u32, vp, i64, vp, i64, vp, vp, vp, vp]
        L.linac_lup.restype = ctypes.c_int
        L.linac_rref_host.argtypes = [vp, i64, i64, i64, u32, vp, vp, vp]
        L.linac_rref_host.restype = ctypes.c_int
        L.linac_set_wait_limit.argtypes = [i64]
        L.linac_set_wait_limit.restype = ctypes.c_int
        L.linac_debug_inject_wait_failure.argtypes = [i32]
        L.linac_debug_inject_wait_failure.restype = None
        L.linac_workspace64_bytes.argtypes = [i64, i64]
        L.linac_workspace64_bytes.restype = ctypes.c_size_t
        for name in ("linac_rref", "linac_rref_ex", "linac_solve", "linac_solve_ex",
                     "linac_rref_batched", "linac_last_device_status", "linac_version",
                     "linac_load_matrix", "linac_matmul", "linac_null_space", "linac_rank_factor",
                     "linac_rref64", "linac_rref64_ex", "linac_solve64", "linac_null_space64",
                     "linac_rank_factor64"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def header_symbols() -> list[str]:
    """Entry points declared in include/linac.h."""
    hdr = os.path.join(os.path.dirname(_build.HERE), "include", "linac.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(linac_\w+)\s*\(", text, re.M)))


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _check(code: int, where: str):
    if code != 0:
        raise LinacError(code, where)


def _matrix(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or t.dim() != 2 or not t.is_cuda:
        raise ValueError(f"{name} must be a 2-D CUDA tensor")
    if t.dtype not in (torch.int32, torch.uint32):
        raise ValueError(f"{name} must be int32 or uint32")
    if t.stride(1) != 1 and t.shape[1] > 1:
        raise ValueError(f"{name} must be row-major (unit column stride)")
    ld = t.stride(0) if t.shape[0] > 1 else max(t.shape[1] + (-t.shape[1]) % 4, 4)
    return t.data_ptr(), t.shape[0], t.shape[1], ld


def _opts(path="auto", nb=0, validate=False) -> Options:
    return Options(_PATHS[path] if isinstance(path, str) else int(path), int(nb), int(bool(validate)), 0)


def padded(rows: int, cols: int, device="cuda") -> torch.Tensor:
    """A zeroed rows x cols int32 view whose row stride is a multiple of 4."""
    ld = max(cols + (-cols) % 4, 4)
    return torch.zeros((rows, ld), dtype=torch.int32, device=device)[:, :cols]


def to_device(M, device="cuda") -> torch.Tensor:
    """Copy a host matrix of residues into a padded int32 device view."""
    import numpy as np
    M = np.ascontiguousarray(np.asarray(M, dtype=np.uint32))
    out = padded(M.shape[0], M.shape[1], device)
    out.copy_(torch.from_numpy(M.view(np.int32)))
    return out


def linac_rref(A: torch.Tensor, p: int, *, ncols_search: int | None = None, path="auto", nb: int = 0,
               validate: bool = False, stream=None):
    """In-place RREF of A (paper section 3.2).  Returns (rank, pivots) as int32
    CUDA tensors (rank has one element; pivots has min(m, ncols_search)
    entries, -1 after the rank)."""
    ptr, m, n, ld = _matrix(A, "A")
    ns = n if ncols_search is None else int(ncols_search)
    rank = torch.zeros(1, dtype=torch.int32, device=A.device)
    piv = torch.full((max(min(m, ns), 1),), -1, dtype=torch.int32, device=A.device)
    o = _opts(path, nb, validate)
    _check(lib().linac_rref_ex(ptr, m, n, ld, p, ns, rank.data_ptr(), piv.data_ptr(), ctypes.byref(o),
                               _stream_ptr(stream)), "linac_rref")
    return rank, piv[:min(m, ns)]


def linac_lup(A: torch.Tensor, p: int, *, stream=None):
    """LUP factorisation P A = L U (see include/linac.h).  A is not modified.
    Returns (L, U, perm, rank, pivots) as CUDA tensors: L m x min(m, n), U
    m x n, perm m int32 (row i of P A is row perm[i] of A)."""
    pa, m, n, ld = _matrix(A, "A")
    mn = min(m, n)
    Lm = padded(max(m, 1), max(mn, 1), A.device)[:m, :mn]
    U = padded(max(m, 1), max(n, 1), A.device)[:m, :n]
    perm = torch.zeros(max(m, 1), dtype=torch.int32, device=A.device)
    rank = torch.zeros(1, dtype=torch.int32, device=A.device)
    piv = torch.full((max(mn, 1),), -1, dtype=torch.int32, device=A.device)
    ldl = max(Lm.stride(0), mn, 1) if m else max(mn, 1)
    ldu = max(U.stride(0), n, 1) if m else max(n, 1)
    _check(lib().linac_lup(pa, m, n, ld, p, Lm.data_ptr(), ldl, U.data_ptr(), ldu, perm.data_ptr(),
                           rank.data_ptr(), piv.data_ptr(), _stream_ptr(stream)), "linac_lup")
    return Lm, U, perm[:m], rank, piv[:mn]


def padded_host(rows: int, cols: int) -> torch.Tensor:
    """A zeroed rows x cols int32 view of PINNED host memory whose row stride
    is a multiple of 4 (the layout linac_rref_host takes)."""
    ld = max(cols + (-cols) % 4, 4)
    return torch.zeros((rows, ld), dtype=torch.int32, pin_memory=True)[:, :cols]


def linac_rref_host(A: torch.Tensor, p: int, *, rank: torch.Tensor | None = None,
                    pivots: torch.Tensor | None = None, stream=None):
    """In-place RREF of a matrix in pinned host memory (see padded_host); the
    transfers happen inside the call.  Returns (rank, pivots) as pinned CPU
    int32 tensors, valid once the stream has been synchronised."""
    if not isinstance(A, torch.Tensor) or A.dim() != 2 or A.is_cuda or not A.is_pinned():
        raise ValueError("A must be a 2-D pinned CPU tensor")
    if A.dtype not in (torch.int32, torch.uint32) or (A.stride(1) != 1 and A.shape[1] > 1):
        raise ValueError("A must be row-major int32 or uint32")
    m, n = A.shape
    ld = A.stride(0) if m > 1 else max(n + (-n) % 4, 4)
    if rank is None:
        rank = torch.zeros(1, dtype=torch.int32, pin_memory=True)
    if pivots is None:
        pivots = torch.full((max(min(m, n), 1),), -1, dtype=torch.int32, pin_memory=True)
    _check(lib().linac_rref_host(A.data_ptr(), m, n, ld, p, rank.data_ptr(), pivots.data_ptr(),
                                 _stream_ptr(stream)), "linac_rref_host")
    return rank, pivots[:min(m, n)]


def linac_solve(A: torch.Tensor, B: torch.Tensor, p: int, *, path="auto", nb: int = 0,
                validate: bool = False, stream=None):
    """Particular solutions of A X = B (paper section 5.2).  Returns
    (X, consistent, rank, pivots) as CUDA tensors; A and B are not modified."""
    pa, m, nA, ldA = _matrix(A, "A")
    pb, mb, k, ldB = _matrix(B, "B")
    if mb != m:
        raise ValueError("A and B need the same number of rows")
    X = torch.zeros((max(nA, 1), max(k, 1)), dtype=torch.int32, device=A.device)
    cons = torch.zeros(max(k, 1), dtype=torch.uint8, device=A.device)
    rank = torch.zeros(1, dtype=torch.int32, device=A.device)
    piv = torch.full((max(min(m, nA), 1),), -1, dtype=torch.int32, device=A.device)
    o = _opts(path, nb, validate)
    _check(lib().linac_solve_ex(pa, m, nA, ldA, pb, k, ldB, p, X.data_ptr(), X.stride(0), cons.data_ptr(),
                                rank.data_ptr(), piv.data_ptr(), ctypes.byref(o), _stream_ptr(stream)),
           "linac_solve")
    return X[:nA, :k], cons[:k].bool(), rank, piv[:min(m, nA)]


def batched_outputs(m: torch.Tensor, n: torch.Tensor, nsearch: torch.Tensor | None = None):
    """Output buffers of a packed batch: (ranks, pivots, piv_offsets, status),
    with piv_offsets the exclusive prefix sum of min(m, nsearch or n)."""
    dev = m.device
    batch = int(m.numel())
    mm = m.to(torch.int64)
    nn = (nsearch if nsearch is not None else n).to(torch.int64)
    npiv = torch.minimum(mm, nn)
    piv_off = torch.zeros(batch, dtype=torch.int64, device=dev)
    if batch > 1:
        piv_off[1:] = torch.cumsum(npiv, 0)[:-1]
    total = int(npiv.sum().item()) if batch else 0
    pivots = torch.full((max(total, 1),), -1, dtype=torch.int32, device=dev)
    ranks = torch.zeros(max(batch, 1), dtype=torch.int32, device=dev)
    status = torch.zeros(max(batch, 1), dtype=torch.int32, device=dev)
    return ranks, pivots, piv_off, status


def linac_rref_batched_into(data: torch.Tensor, offsets: torch.Tensor, m: torch.Tensor, n: torch.Tensor,
                            ld: torch.Tensor, p: int, ranks: torch.Tensor, pivots: torch.Tensor,
                            piv_off: torch.Tensor, status: torch.Tensor | None, *, max_m: int, max_n: int,
                            nsearch: torch.Tensor | None = None, flags: int = 0, stream=None):
    """linac_rref_batched into caller-made outputs (see batched_outputs).
    Argument marshalling only -- no allocation and no host synchronisation --
    so the call can be captured into a CUDA graph once the library's scratch
    for this stream exists (one uncaptured call of the same batch first)."""
    _check(lib().linac_rref_batched(data.data_ptr(), offsets.data_ptr(), m.data_ptr(), n.data_ptr(),
                                    ld.data_ptr(), nsearch.data_ptr() if nsearch is not None else None,
                                    int(m.numel()), int(max_m), int(max_n), p, flags, ranks.data_ptr(),
                                    pivots.data_ptr(), piv_off.data_ptr(),
                                    status.data_ptr() if status is not None else None,
                                    _stream_ptr(stream)), "linac_rref_batched")


def linac_rref_batched(data: torch.Tensor, offsets: torch.Tensor, m: torch.Tensor, n: torch.Tensor,
                       ld: torch.Tensor, p: int, *, nsearch: torch.Tensor | None = None, flags: int = 0,
                       max_m: int | None = None, max_n: int | None = None, stream=None):
    """In-place RREF of a packed batch of systems (see include/linac.h).
    Returns (ranks, pivots, piv_offsets, status) as CUDA tensors."""
    batch = int(m.numel())
    ranks, pivots, piv_off, status = batched_outputs(m, n, nsearch)
    if max_m is None:
        max_m = int(m.max().item()) if batch else 0
    if max_n is None:
        max_n = int(n.max().item()) if batch else 0
    linac_rref_batched_into(data, offsets, m, n, ld, p, ranks, pivots, piv_off, status, max_m=max_m,
                            max_n=max_n, nsearch=nsearch, flags=flags, stream=stream)
    return ranks[:batch], pivots, piv_off, status[:batch]


def linac_load_matrix(bases: torch.Tensor, lindices: torch.Tensor, p: int, *, out: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """A[r][c] = prod_t bases[r][lindices[c][t]] mod p (paper sections 2.3 and
    3.3): rows are sampling points, columns monomials.  lindices is an
    n_cols x d int32 CUDA tensor (contiguous)."""
    pb, n_rows, n_basis, ldb = _matrix(bases, "bases")
    if lindices.dim() != 2 or lindices.dtype != torch.int32 or not lindices.is_contiguous() or not lindices.is_cuda:
        raise ValueError("lindices must be a contiguous n_cols x d int32 CUDA tensor")
    n_cols, d = lindices.shape
    if out is None:
        out = padded(n_rows, n_cols, bases.device)
    po, ro, co, ldo = _matrix(out, "out")
    if (ro, co) != (n_rows, n_cols):
        raise ValueError("out has the wrong shape")
    _check(lib().linac_load_matrix(pb, n_rows, n_basis, ldb, lindices.data_ptr(), n_cols, d, p, po, ldo,
                                   _stream_ptr(stream)), "linac_load_matrix")
    return out


def linac_matmul(A: torch.Tensor, B: torch.Tensor, p: int, *, out: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """A B mod p for canonical residues (exact)."""
    pa, m, K, lda = _matrix(A, "A")
    pb, kb, n, ldb = _matrix(B, "B")
    if kb != K:
        raise ValueError("inner dimensions differ")
    if out is None:
        out = padded(m, n, A.device)
    pc, mc, nc, ldc = _matrix(out, "out")
    if (mc, nc) != (m, n):
        raise ValueError("out has the wrong shape")
    _check(lib().linac_matmul(pa, m, K, lda, pb, n, ldb, p, pc, ldc, _stream_ptr(stream)), "linac_matmul")
    return out


def linac_null_space(R: torch.Tensor, rank: torch.Tensor, pivots: torch.Tensor, p: int, *,
                     kcols: int | None = None, stream=None):
    """Canonical null-space basis of an RREF (paper section 5.1).  Returns
    (K, free, nullity): K is n x kcols (kcols defaults to n), valid in its
    first nullity columns; free lists the free columns, -1 after them."""
    pr, m, n, ld = _matrix(R, "R")
    kc = n if kcols is None else int(kcols)
    K = padded(n, max(kc, 1), R.device)[:, :kc] if n else padded(1, 1, R.device)[:0, :0]
    free = torch.full((max(n, 1),), -1, dtype=torch.int32, device=R.device)
    nullity = torch.zeros(1, dtype=torch.int32, device=R.device)
    ldk = K.stride(0) if n else 1
    _check(lib().linac_null_space(pr, m, n, ld, rank.data_ptr(), pivots.data_ptr(), p,
                                  K.data_ptr() if n else None, kc, max(ldk, kc), free.data_ptr(), nullity.data_ptr(),
                                  _stream_ptr(stream)), "linac_null_space")
    return K, free[:n], nullity


def linac_rank_factor(A: torch.Tensor, rank: torch.Tensor, pivots: torch.Tensor, *, ccols: int | None = None,
                      stream=None) -> torch.Tensor:
    """C = A[:, J] for the pivot columns J of A's RREF (paper section 5.1:
    A = C R).  A is the original matrix.  Returns m x ccols (default
    min(m, n)); columns at or beyond the rank are zero."""
    pa, m, n, ld = _matrix(A, "A")
    cc = min(m, n) if ccols is None else int(ccols)
    C = padded(m, max(cc, 1), A.device)[:, :cc]
    _check(lib().linac_rank_factor(pa, m, n, ld, rank.data_ptr(), pivots.data_ptr(), C.data_ptr(), cc,
                                   max(C.stride(0), cc), _stream_ptr(stream)), "linac_rank_factor")
    return C


def linac_last_device_status(stream=None) -> int:
    return int(lib().linac_last_device_status(_stream_ptr(stream)))


def linac_set_wait_limit(cycles: int) -> None:
    """Limit of the device-side waits in SM clock cycles (0 = default, ~2 s)."""
    _check(lib().linac_set_wait_limit(int(cycles)), "linac_set_wait_limit")


def linac_debug_inject_wait_failure(on: bool) -> None:
    """Test support: while on, the full-height pivot search's arrival barrier
    can never complete, so its waits run out (LINAC_ERR_TIMEOUT)."""
    lib().linac_debug_inject_wait_failure(1 if on else 0)


def linac_workspace_bytes(m: int, n: int, nb: int = 0) -> int:
    o = _opts("auto", nb, False)
    return int(lib().linac_workspace_bytes(m, n, ctypes.byref(o)))


def linac_version() -> int:
    return int(lib().linac_version())


def linac_profile_enable(on: bool = True):
    lib().linac_profile_enable(1 if on else 0)


def linac_profile_reset():
    lib().linac_profile_reset()


def linac_profile_read() -> dict:
    """{kernel class: (launches, total_ms)} for the launches timed so far."""
    buf = (ProfileEntry * 64)()
    n = lib().linac_profile_read(buf, 64)
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(n)}


def linac_launch_count() -> int:
    return int(lib().linac_launch_count())


def linac_batched_tune(p: int, stream=None) -> list[int]:
    """Autotune linac_rref_batched's panel width per size bucket (see include/linac.h)."""
    out = (ctypes.c_int32 * 5)()
    _check(lib().linac_batched_tune(p, out, _stream_ptr(stream)), "linac_batched_tune")
    return list(out)


def linac_batched_set_panel_widths(widths) -> None:
    """Panel width per size bucket (5 entries: 16, 32, 64 or 0 = default)."""
    arr = (ctypes.c_int32 * 5)(*[int(w) for w in widths])
    _check(lib().linac_batched_set_panel_widths(arr), "linac_batched_set_panel_widths")


def linac_batched_panel_widths() -> list[int]:
    out = (ctypes.c_int32 * 5)()
    _check(lib().linac_batched_panel_widths(out), "linac_batched_panel_widths")
    return list(out)


# ---------------------------------------------------------------------------
# uint64 residues (primes below 2^64; paper section 2.3).  Device matrices are
# 2-D int64 (or uint64) tensors holding the residues' bit patterns, row stride
# a multiple of 2 elements.

def _matrix64(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or t.dim() != 2 or not t.is_cuda:
        raise ValueError(f"{name} must be a 2-D CUDA tensor")
    if t.dtype != torch.int64 and str(t.dtype) != "torch.uint64":
        raise ValueError(f"{name} must be int64 or uint64")
    if t.stride(1) != 1 and t.shape[1] > 1:
        raise ValueError(f"{name} must be row-major (unit column stride)")
    ld = t.stride(0) if t.shape[0] > 1 else max(t.shape[1] + t.shape[1] % 2, 2)
    return t.data_ptr(), t.shape[0], t.shape[1], ld


def padded64(rows: int, cols: int, device="cuda") -> torch.Tensor:
    """A zeroed rows x cols int64 view whose row stride is a multiple of 2."""
    ld = max(cols + cols % 2, 2)
    return torch.zeros((rows, ld), dtype=torch.int64, device=device)[:, :cols]


def to_device64(M, device="cuda") -> torch.Tensor:
    """Copy a host matrix of uint64 residues into a padded int64 device view."""
    import numpy as np
    M = np.ascontiguousarray(np.asarray(M, dtype=np.uint64))
    out = padded64(M.shape[0], M.shape[1], device)
    out.copy_(torch.from_numpy(M.view(np.int64)))
    return out


def host64(t: torch.Tensor):
    """A device int64 matrix back on the host as uint64 residues."""
    import numpy as np
    return t.cpu().numpy().view(np.uint64)


def linac_rref64(A: torch.Tensor, p: int, *, ncols_search: int | None = None, validate: bool = False,
                 stream=None):
    """In-place RREF of a uint64 matrix over Z/pZ, p an odd prime below 2^64.
    Returns (rank, pivots) as int32 CUDA tensors."""
    ptr, m, n, ld = _matrix64(A, "A")
    ns = n if ncols_search is None else int(ncols_search)
    rank = torch.zeros(1, dtype=torch.int32, device=A.device)
    piv = torch.full((max(min(m, ns), 1),), -1, dtype=torch.int32, device=A.device)
    o = _opts("auto", 0, validate)
    _check(lib().linac_rref64_ex(ptr, m, n, ld, int(p), ns, rank.data_ptr(), piv.data_ptr(), ctypes.byref(o),
                                 _stream_ptr(stream)), "linac_rref64")
    return rank, piv[:min(m, ns)]


def linac_solve64(A: torch.Tensor, B: torch.Tensor, p: int, *, stream=None):
    """Particular solutions of A X = B with uint64 residues (section 5.2).
    Returns (X, consistent, rank, pivots); A and B are not modified."""
    pa, m, nA, ldA = _matrix64(A, "A")
    pb, mb, k, ldB = _matrix64(B, "B")
    if mb != m:
        raise ValueError("A and B need the same number of rows")
    X = torch.zeros((max(nA, 1), max(k, 1)), dtype=torch.int64, device=A.device)
    cons = torch.zeros(max(k, 1), dtype=torch.uint8, device=A.device)
    rank = torch.zeros(1, dtype=torch.int32, device=A.device)
    piv = torch.full((max(min(m, nA), 1),), -1, dtype=torch.int32, device=A.device)
    _check(lib().linac_solve64(pa, m, nA, ldA, pb, k, ldB, int(p), X.data_ptr(), X.stride(0), cons.data_ptr(),
                               rank.data_ptr(), piv.data_ptr(), _stream_ptr(stream)), "linac_solve64")
    return X[:nA, :k], cons[:k].bool(), rank, piv[:min(m, nA)]


def linac_null_space64(R: torch.Tensor, rank: torch.Tensor, pivots: torch.Tensor, p: int, *,
                       kcols: int | None = None, stream=None):
    """linac_null_space for uint64 residues (section 5.1).  Returns (K, free,
    nullity) with K an n x kcols int64 view."""
    pr, m, n, ld = _matrix64(R, "R")
    kc = n if kcols is None else int(kcols)
    K = padded64(max(n, 1), max(kc, 1), R.device)[:n, :kc]
    free = torch.full((max(n, 1),), -1, dtype=torch.int32, device=R.device)
    nullity = torch.zeros(1, dtype=torch.int32, device=R.device)
    ldk = max(K.stride(0), kc) if n else max(kc, 1)
    _check(lib().linac_null_space64(pr, m, n, ld, rank.data_ptr(), pivots.data_ptr(), int(p),
                                    K.data_ptr() if n else None, kc, ldk, free.data_ptr(), nullity.data_ptr(),
                                    _stream_ptr(stream)), "linac_null_space64")
    return K, free[:n], nullity


def linac_rank_factor64(A: torch.Tensor, rank: torch.Tensor, pivots: torch.Tensor, *, ccols: int | None = None,
                        stream=None) -> torch.Tensor:
    """linac_rank_factor for uint64 residues: C = A[:, J] (section 5.1)."""
    pa, m, n, ld = _matrix64(A, "A")
    cc = min(m, n) if ccols is None else int(ccols)
    C = padded64(max(m, 1), max(cc, 1), A.device)[:m, :cc]
    _check(lib().linac_rank_factor64(pa, m, n, ld, rank.data_ptr(), pivots.data_ptr(), C.data_ptr(), cc,
                                     max(C.stride(0), cc), _stream_ptr(stream)), "linac_rank_factor64")
    return C

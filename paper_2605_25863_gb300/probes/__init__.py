"""ctypes loader of liblinac_probes.so: the benchmark's integer pipe-rate
probes (the measured roofline denominators of the trailing-update paths).
Measurement tooling only; the library's compute path never uses it."""
from __future__ import annotations

import ctypes
import os

from .. import build as _build


class IntRates(ctypes.Structure):
    _fields_ = [("imad_wide_per_s", ctypes.c_double), ("imma_u8_mac_per_s", ctypes.c_double),
                ("dp4a_u8_mac_per_s", ctypes.c_double), ("sm_clock_khz", ctypes.c_double),
                ("sm_count", ctypes.c_int), ("coissue_imad_only_ms", ctypes.c_double),
                ("coissue_imma_only_ms", ctypes.c_double), ("coissue_both_ms", ctypes.c_double),
                ("imma_s8_mac_per_s", ctypes.c_double)]


def measure_int_rates(stream=None) -> dict:
    """Runs the probes on the current CUDA device (see probes/int_rates.h)."""
    import torch
    if not os.path.exists(_build.PROBES_LIB):
        raise RuntimeError(f"{_build.PROBES_LIB} is missing: build first")
    L = ctypes.CDLL(_build.PROBES_LIB)
    L.linac_probe_int_rates.argtypes = [ctypes.POINTER(IntRates), ctypes.c_void_p]
    L.linac_probe_int_rates.restype = ctypes.c_int
    s = stream if stream is not None else torch.cuda.current_stream()
    r = IntRates()
    code = L.linac_probe_int_rates(ctypes.byref(r), int(s.cuda_stream))
    if code != 0:
        raise RuntimeError(f"linac_probe_int_rates failed with status {code}")
    return {k: getattr(r, k) for k, _ in IntRates._fields_}

"""Exact mod-p Gauss-Jordan elimination (RREF, rank, pivots, solve) on GB300.

The computation lives in the sm_103a library ``_lib/liblinac.so`` (C ABI in
``include/linac.h``); ``linac`` binds it for torch CUDA tensors and
``synth`` builds seeded synthetic workloads.
"""
from .linac import (LinacError, linac_last_device_status, linac_rref, linac_rref_batched,  # noqa: F401
                    linac_solve, linac_version, linac_workspace_bytes, padded, to_device)

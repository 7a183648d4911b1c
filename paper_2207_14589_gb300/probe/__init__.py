"""ctypes binding of the benchmark's measurement library (libsped_probe.so): the gather-rate
probe, which replays the chain step's access stream without its arithmetic. Not part of the
libsped C ABI."""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsped_probe.so")
_lib = None

MODES = {"csr_order": 0, "hashed_rows": 1, "consecutive_rows": 2}


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsped_probe.so not built ({LIB_PATH}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.sped_probe_gather.argtypes = [ctypes.c_int64, vp, vp, ctypes.c_int, vp, ctypes.c_int,
                                        vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, vp]
        L.sped_probe_gather.restype = ctypes.c_int
        _lib = L
    return _lib


def probe_gather(row_ptr, col_idx, X, Y, k, mode=0, seed=0, stream=None):
    """The chain step's gathers without its arithmetic on a CSR (int32 device tensors) and BF16
    blocks X, Y (n x ld); Y receives the per-row sums. mode: 0 CSR order, 1 hashed rows,
    2 consecutive rows."""
    if X.dtype != torch.bfloat16 or Y.dtype != torch.bfloat16:
        raise TypeError("probe_gather works on bfloat16 blocks")
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().sped_probe_gather(row_ptr.numel() - 1, row_ptr.data_ptr(), col_idx.data_ptr(), k,
                                 X.data_ptr(), X.stride(0), Y.data_ptr(), Y.stride(0), int(mode),
                                 int(seed), s.cuda_stream)
    if rc != 0:
        raise RuntimeError(f"sped_probe_gather failed ({rc})")
    return Y

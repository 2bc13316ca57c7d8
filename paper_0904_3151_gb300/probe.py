"""ctypes view of libmsm_probe.so (include/msm_probe.h): the integer-mix
probe, a measurement aid for the pair check's roofline, built beside the
method's library but not part of it."""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

_handle = None


def load():
    """Load libmsm_probe.so; raises if it has not been built."""
    global _handle
    if _handle is None:
        if not os.path.exists(_build.PROBE_LIB):
            raise ImportError(f"{_build.PROBE_LIB} is missing: build the package first")
        L = ctypes.CDLL(_build.PROBE_LIB)
        L.msm_int_mix_probe.restype = ctypes.c_int
        L.msm_int_mix_probe.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_uint32, ctypes.c_void_p]
        _handle = L
    return _handle


def int_mix_probe(out: torch.Tensor, blocks: int, iters: int, seed: int = 0) -> None:
    """Launch the probe into `out`, a contiguous int32 CUDA tensor of
    blocks * 256 * 8 words; asynchronous on the current stream."""
    assert out.is_cuda and out.is_contiguous() and out.dtype == torch.int32
    assert out.numel() >= blocks * 256 * 8
    st = load().msm_int_mix_probe(ctypes.c_void_p(out.data_ptr()), blocks, iters,
                                  ctypes.c_uint32(seed & 0xFFFFFFFF),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise RuntimeError(f"msm_int_mix_probe failed ({st})")

"""The C ABI library builds, loads without a GPU, and exports every entry
point include/fpcg.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2504_09820_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"FPCG_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)
    return names


@pytest.fixture(scope="module")
def so():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("fpcg_detect", "fpbjcg_detect", "fpcg_solve_gram", "fpcg_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(so):
    for n in _declared():
        assert hasattr(so, n), n


def test_host_only_entry_points(so):
    so.fpcg_strerror.restype = ctypes.c_char_p
    assert so.fpcg_strerror(0) == b"success"
    assert so.fpcg_strerror(1) == b"invalid argument"
    assert so.fpcg_version() >= 100


def test_argument_validation_needs_no_gpu(so):
    """Bad arguments are rejected on the host before anything touches CUDA."""
    from paper_2504_09820_gb300 import fpcg as F
    F.lib()
    p = F.precision()
    L = F.lib()
    nul = None
    # K > N
    assert L.fpcg_detect(1, 1, 1, 1, 4, 8, 1, 4, ctypes.byref(p), 1, nul, nul, nul, nul, nul, nul, nul) == F.EINVAL
    # K > 128
    assert L.fpcg_detect(1, 1, 1, 1, 256, 129, 1, 4, ctypes.byref(p), 1, nul, nul, nul, nul, nul, nul, nul) == F.EINVAL
    # L does not divide K
    assert L.fpbjcg_detect(1, 1, 1, 1, 64, 16, 1, 4, 5, ctypes.byref(p), 1, nul, nul, nul, nul, nul, nul, nul) == F.EINVAL
    # missing x_hat
    assert L.fpcg_detect(1, 1, 1, 1, 64, 16, 1, 4, ctypes.byref(p), nul, nul, nul, nul, nul, nul, nul, nul) == F.EINVAL
    # fp64 mode needs every role at fp64
    bad = F.Precision(F.FP32, F.FP32, F.FP32, F.FP64, 0, -1, 0, 32, F.FP64)
    assert L.fpcg_detect(1, 1, 1, 1, 64, 16, 1, 4, ctypes.byref(bad), 1, nul, nul, nul, nul, nul, nul, nul) == F.EINVAL
    # fp64 mode beyond K = 64
    p64 = F.precision(w="fp64")
    # (fp64 mode beyond K = 64 runs from H; on a given Gram matrix it is not supported)
    assert L.fpcg_solve_gram(1, 1, 96, 1, 4, 0, ctypes.byref(p64), 1, nul, nul, nul, nul) == F.ENOTSUP
    # e4m3 with an unsupported block
    p8 = F.precision(mv="e4m3", fp8_block=16)
    assert L.fpcg_detect(1, 1, 1, 1, 64, 16, 1, 4, ctypes.byref(p8), 1, nul, nul, nul, nul, nul, nul, nul) == F.ENOTSUP
    # tx without a counter
    assert L.fpcg_detect(1, 1, 1, 1, 64, 16, 1, 4, ctypes.byref(p), 1, 1, nul, nul, 1, nul, nul, nul) == F.EINVAL
    # FMA probe: a length that is not a multiple of 256, too few iterations, no buffer
    f = ctypes.c_double(0.0)
    assert L.fpcg_fma_probe(0, 64, 256, 255, ctypes.byref(f), nul) == F.EINVAL
    assert L.fpcg_fma_probe(0, 2, 256, 256, ctypes.byref(f), nul) == F.EINVAL
    assert L.fpcg_fma_probe(1, 64, nul, 256, ctypes.byref(f), nul) == F.EINVAL
    assert L.fpcg_fma_probe(1, 64, 4, 256, ctypes.byref(f), nul) == F.EINVAL   # misaligned for fp64

"""Third-party reference implementations used to pin the oracle."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def aten_philox():
    """ctypes handle to ATen's philox_engine (header-only), compiled on first use."""
    global _lib
    if _lib is not None:
        return _lib
    import torch.utils.cpp_extension as ce
    inc = ce.include_paths()[0]
    out = os.path.join(tempfile.mkdtemp(prefix="aten_philox_"), "libaten_philox.so")
    subprocess.check_call(["g++", "-O1", "-shared", "-fPIC", "-std=c++17", "-I" + inc,
                           "-o", out, os.path.join(_HERE, "aten_philox_shim.cpp")])
    _lib = ctypes.CDLL(out)
    _lib.aten_philox_words.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.POINTER(ctypes.c_uint32)]
    return _lib


def aten_words(seed: int, ctr) -> np.ndarray:
    """Philox4x32-10 words for counter (c0, c1, c2, c3) under the 64-bit seed."""
    lib = aten_philox()
    c0, c1, c2, c3 = [int(x) & 0xFFFFFFFF for x in ctr]
    out = (ctypes.c_uint32 * 4)()
    lib.aten_philox_words(seed & 0xFFFFFFFFFFFFFFFF, c2 | (c3 << 32), c0 | (c1 << 32), out)
    return np.array(list(out), dtype=np.uint32)

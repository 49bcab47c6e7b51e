"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

No compute call is made here (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_ \*]*?)\b(randutv_[a-z0-9_]+)\s*\(", src):
            names.append(m.group(2))
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2002_06960_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ["randutv_factor", "randutv_factor_ex", "randutv_factor_host",
                 "randutv_philox_normal", "randutv_householder_qr", "randutv_wy_factor",
                 "randutv_small_svd", "randutv_workspace_bytes", "randutv_strerror"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_2002_06960_gb300 import _lib
    assert set(_declared_functions()) <= set(_lib.exported_names())
    _lib.lib()   # loads with every signature set


def test_strerror_and_workspace_need_no_gpu(libpath):
    from paper_2002_06960_gb300 import _lib
    L = _lib.lib()
    assert L.randutv_strerror(0) == b"success"
    assert L.randutv_strerror(-3) == b"invalid argument"
    assert L.randutv_strerror(3).startswith(b"a bounded")
    ws = L.randutv_workspace_bytes(16384, 16384, 128, 0)
    assert 7 * 16384 * 128 * 8 <= ws < 512 * 2 ** 20
    assert L.randutv_workspace_bytes(0, 5, 4, 0) == 0


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2002_06960_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.lib()


def test_argument_errors_return_before_any_device_work(libpath):
    """Each entry point validates its arguments on the host and returns the
    documented negative code without touching the device (the pointer below
    is never dereferenced, and no GPU is needed)."""
    from paper_2002_06960_gb300 import _lib
    L = _lib.lib()
    p = 0x1000   # stands in for a device pointer; never read
    # randutv_factor_ex: m, n, A, lda, b, q, T, first_step
    assert L.randutv_factor_ex(0, 8, p, 8, 4, 1, 0, None, p, None, -1, None, 0) == -1
    assert L.randutv_factor_ex(8, 0, p, 8, 4, 1, 0, None, p, None, -1, None, 0) == -2
    assert L.randutv_factor_ex(8, 8, None, 8, 4, 1, 0, None, p, None, -1, None, 0) == -3
    assert L.randutv_factor_ex(8, 8, p, 7, 4, 1, 0, None, p, None, -1, None, 0) == -4
    assert L.randutv_factor_ex(8, 8, p, 8, 257, 1, 0, None, p, None, -1, None, 0) == -5
    assert L.randutv_factor_ex(8, 8, p, 8, 4, 17, 0, None, p, None, -1, None, 0) == -6
    assert L.randutv_factor_ex(8, 8, p, 8, 4, 1, 0, None, None, None, -1, None, 0) == -9
    assert L.randutv_factor_ex(8, 8, p, 8, 4, 1, 0, None, p, None, -1, None, -1) == -13
    # randutv_factor_mixed: b a multiple of 8 in [8, 256]
    assert L.randutv_factor_mixed(64, 64, p, 64, 12, 1, 0, None, p, None, -1, None) == -5
    assert L.randutv_factor_mixed(64, 64, p, 64, 264, 1, 0, None, p, None, -1, None) == -5
    assert L.randutv_factor_mixed(64, 64, p, 64, 16, -1, 0, None, p, None, -1, None) == -6
    assert L.randutv_factor_mixed(64, 64, p, 32, 16, 1, 0, None, p, None, -1, None) == -4
    # randutv_lowrank / _backward: 1 <= k < min(m, n), b divides k
    for k, b, q, code in [(40, 8, 1, -5), (0, 8, 1, -5), (24, 16, 1, -6), (16, 0, 1, -6),
                          (16, 8, 17, -7)]:
        assert L.randutv_lowrank(64, 40, p, 64, k, b, q, 0, p, None) == code
        assert L.randutv_lowrank_backward(64, 40, p, 64, k, b, q, 0, p, p, None) == code
    assert L.randutv_lowrank(64, 40, p, 64, 16, 8, 1, 0, None, None) == -9
    assert L.randutv_lowrank_backward(64, 40, p, 64, 16, 8, 1, 0, p, None, None) == -10
    # randutv_factor_ooc: host A, the device budget at least the minimum
    need = L.randutv_ooc_min_device_bytes(64, 40, 8)
    assert need > 0 and L.randutv_ooc_min_device_bytes(0, 40, 8) == 0
    assert L.randutv_factor_ooc(0, 40, p, 64, 8, 1, 0, None, None, need, None, None) == -1
    assert L.randutv_factor_ooc(64, 40, None, 64, 8, 1, 0, None, None, need, None, None) == -3
    assert L.randutv_factor_ooc(64, 40, p, 63, 8, 1, 0, None, None, need, None, None) == -4
    assert L.randutv_factor_ooc(64, 40, p, 64, 300, 1, 0, None, None, need, None, None) == -5
    assert L.randutv_factor_ooc(64, 40, p, 64, 8, 17, 0, None, None, need, None, None) == -6
    assert L.randutv_factor_ooc(64, 40, p, 64, 8, 1, 0, None, None, need - 1, None, None) == -10
    # randutv_hqrrp: m >= n, 1 <= b <= 256, R and perm given
    assert L.randutv_hqrrp(40, 64, p, 40, 8, 0, None, p, p, None) == -2
    assert L.randutv_hqrrp(64, 40, p, 32, 8, 0, None, p, p, None) == -4
    assert L.randutv_hqrrp(64, 40, p, 64, 0, 0, None, p, p, None) == -5
    assert L.randutv_hqrrp(64, 40, p, 64, 8, 0, None, None, p, None) == -8
    assert L.randutv_hqrrp(64, 40, p, 64, 8, 0, None, p, None, None) == -9
    # randutv_gemm_bf16: planes must be 1 or 3
    assert L.randutv_gemm_bf16(b"N", 8, 8, 8, 1.0, p, 8, p, 8, 0.0, p, 8, 2, None) == -13
    assert L.randutv_gemm_bf16(b"X", 8, 8, 8, 1.0, p, 8, p, 8, 0.0, p, 8, 1, None) == -1

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

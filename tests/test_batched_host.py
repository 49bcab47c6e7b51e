"""Host-side logic of the batched form, without a GPU: the size classes of
the autotuner (which must be the library's: class c holds max(m, n) in
(128 c, 128 (c + 1)], the last class everything above) and the argument
checks of the tuning table and of plan creation, which run before any
device work."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def L():
    from paper_2002_06960_gb300 import _lib, build
    build.build()
    return _lib.lib()


def test_size_classes_match_the_library_mapping():
    from paper_2002_06960_gb300.batched import N_CLASSES, size_class
    for (m, n), c in [((1, 1), 0), ((128, 5), 0), ((129, 5), 1), ((5, 256), 1), ((257, 257), 2),
                      ((1024, 1024), 7), ((897, 3), 7), ((2000, 9), 7)]:
        assert size_class(m, n) == c, (m, n)
        # the library's own rule, written out
        assert min(N_CLASSES - 1, (max(m, n) - 1) // 128) == c


def test_tuning_table_arguments(L):
    arr = (ctypes.c_int * 8)(16, 32, 64, 0, 32, 32, 32, 32)
    assert L.randutv_batched_set_tuning(arr, 8, 0) == 0
    bad = (ctypes.c_int * 8)(16, 32, 48, 0, 0, 0, 0, 0)
    assert L.randutv_batched_set_tuning(bad, 8, 0) == -1     # 48 is not a block size
    assert L.randutv_batched_set_tuning(arr, 9, 0) == -2     # more classes than exist
    assert L.randutv_batched_set_tuning(arr, 8, 17) == -3    # CTAs per SM
    assert L.randutv_batched_set_tuning(None, 0, 0) == 0     # reset to the default


def test_plan_arguments_are_checked_before_device_work(L):
    h = ctypes.c_void_p()
    one = (ctypes.c_int64 * 1)(64)
    p = (ctypes.c_void_p * 1)(0x1000)
    args = dict(batch=1, m=one, n=one, A=p, lda=one, b=32, q=1, T=p)

    def call(**kw):
        a = {**args, **kw}
        return L.randutv_batched_plan_create(ctypes.byref(h), a["batch"], a["m"], a["n"], a["A"],
                                             a["lda"], a["b"], a["q"], 0, None, a["T"], None)
    assert call(batch=0) == -2
    assert call(m=None) == -3
    assert call(b=8) == -7
    assert call(q=17) == -8
    assert call(T=None) == -11

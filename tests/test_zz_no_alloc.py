"""The allocation-free Householder QR entry point.

randutv_householder_qr_noalloc serves callers that cannot allocate device
memory (inside CUDA graph capture, under an allocator that owns the whole
GPU, or in loops that cannot pay for an allocation): its scratch is a fixed
array inside the library.  Here it is called through the C-ABI twice in a
row and each result is checked against the allocating entry point on the
same input, within the tolerance of the other QR tests.  This file is
collected last, so a run that stops at its first failure has already run
every other test.
"""
import ctypes

import pytest
import torch

from paper_2002_06960_gb300 import inputs

pytestmark = pytest.mark.gpu

f64 = torch.float64


@pytest.fixture(scope="module")
def pkg():
    from paper_2002_06960_gb300 import build
    build.build()
    import paper_2002_06960_gb300 as p
    p.lib()
    return p


def _rel(x, y):
    d = float(torch.linalg.norm(y))
    return float(torch.linalg.norm(x - y)) / (d if d > 0 else 1.0)


def _noalloc(pkg, Y):
    r, c = Y.shape
    panel = pkg.to_colmajor(Y, "cuda")
    W = pkg.colmajor_empty(r, c)
    tau = torch.empty(c, dtype=f64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = pkg.lib().randutv_householder_qr_noalloc(r, c, ctypes.c_void_p(panel.data_ptr()),
                                                  panel.stride(1), ctypes.c_void_p(W.data_ptr()),
                                                  ctypes.c_void_p(tau.data_ptr()), st)
    return rc, panel.cpu(), W.cpu(), tau.cpu()


def _with_alloc(pkg, Y):
    panel = pkg.to_colmajor(Y, "cuda")
    W, tau = pkg.randutv_householder_qr(panel)
    torch.cuda.synchronize()
    return panel.cpu(), W.cpu(), tau.cpu()


def test_noalloc_qr_matches_allocating_qr_twice_in_a_row(pkg):
    for (r, c, seed) in [(3000, 96, 1), (20000, 128, 2)]:   # two calls, different shapes
        Y = inputs.gaussian(r, c, seed=seed)
        rc, P1, W1, t1 = _noalloc(pkg, Y)
        assert rc == 0
        P0, W0, t0 = _with_alloc(pkg, Y)
        assert _rel(P1, P0) < 1e-13
        assert _rel(W1, W0) < 1e-13
        assert _rel(t1, t0) < 1e-13


def test_noalloc_qr_rejects_sizes_beyond_its_maximum(pkg):
    Y = inputs.gaussian(400, 300, seed=3)
    rc, _, _, _ = _noalloc(pkg, Y)
    assert rc == 5   # RANDUTV_EUNSUPPORTED: more than 256 columns

"""Out-of-HBM randUTV (T, U, V in host memory, streamed through the device in
panels) against the FP64 oracle and against the in-HBM GPU path.

The device budget is set to the minimum, so that every pass over a trailing
region is cut into many panels and the three panel buffers rotate through
all copy and compute orders.  Parity with the oracle uses the gate of the
in-HBM parity tests: 1e-12, or 10x the factorization's own sensitivity to
a rounding-level change of A where that is larger.
"""
import pytest
import torch

import oracle
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


def rel(x, y):
    d = float(y.norm())
    return float((x - y).norm()) / (d if d > 0 else 1.0)


def _host(pkg, X, pin=True):
    H = pkg.colmajor_empty(X.shape[0], X.shape[1], device="cpu", pin=pin)
    H.copy_(X)
    return H


def _ooc(pkg, A, b, q, seed, device_bytes=None, want_uv=True, pin=True):
    m, n = A.shape
    T = _host(pkg, A, pin)
    U = pkg.colmajor_empty(m, m, device="cpu", pin=pin) if want_uv else None
    V = pkg.colmajor_empty(n, n, device="cpu", pin=pin) if want_uv else None
    if device_bytes is None:
        device_bytes = pkg.randutv_ooc_min_device_bytes(m, n, b)
    moved = pkg.randutv_factor_ooc(T, b, q, seed, U, V, device_bytes=device_bytes)
    return U, T.clone(), V, moved


@pytest.mark.parametrize("m,n,b,q", [(512, 512, 64, 1), (300, 200, 48, 1), (200, 300, 48, 2),
                                     (257, 257, 64, 0), (90, 70, 128, 1), (384, 640, 128, 2)])
def test_ooc_matches_oracle(pkg, m, n, b, q):
    A = inputs.matrix("linear", m, n, seed=m + n)
    U, T, V, moved = _ooc(pkg, A, b, q, 7)
    ref = oracle.randutv(A, b, q, 7)
    sens = {"U": 0.0, "T": 0.0, "V": 0.0}
    for s in (5, 6):
        g = torch.Generator().manual_seed(s)
        Ap = A + torch.randn(A.shape, generator=g, dtype=f64) * 1e-16 * float(A.abs().max())
        f = oracle.randutv(Ap, b, q, 7)
        for k in sens:
            sens[k] = max(sens[k], rel(getattr(f, k), getattr(ref, k)))
    gate = {k: max(1e-12, 10.0 * v) for k, v in sens.items()}
    assert rel(T, ref.T) < gate["T"]
    assert rel(U, ref.U) < gate["U"], (rel(U, ref.U), sens)
    assert rel(V, ref.V) < gate["V"], (rel(V, ref.V), sens)
    assert float(torch.tril(T, -1).abs().max()) == 0.0
    assert moved > 8.0 * m * n  # at least one read of A


def test_ooc_matches_in_hbm_path(pkg):
    """1536 x 1024, b = 128, q = 1, smooth spectrum: the same factorization
    as randutv_factor up to rounding order, under a budget that cuts every
    pass into several panels."""
    m, n, b, q = 1536, 1024, 128, 1
    A = inputs.matrix("smooth", m, n, seed=3)
    U, T, V, moved = _ooc(pkg, A, b, q, 0)
    Ug, Tg, Vg = pkg.randutv_factor(pkg.to_colmajor(A, "cuda"), b, q, 0)
    torch.cuda.synchronize()
    Ug, Tg, Vg = Ug.cpu(), Tg.cpu(), Vg.cpu()
    assert rel(T, Tg) < 1e-12
    assert rel(U[:, :2 * b], Ug[:, :2 * b]) < 1e-12
    assert rel(V[:, :2 * b], Vg[:, :2 * b]) < 1e-12
    assert oracle.recon_error(A, U, T, V) < 1e-13
    assert oracle.orth_error(U) < 1e-13 and oracle.orth_error(V) < 1e-13
    # with the minimum budget each panel buffer holds max(m, n) x b values:
    # every pass over T, U or V is cut into column panels of 128 columns or fewer
    assert moved > 4 * 8.0 * m * n


def test_ooc_t_only_and_pageable(pkg):
    """No U, V; pageable host memory (synchronous copies, same result)."""
    m, n, b = 400, 300, 32
    A = inputs.matrix("exp40", m, n, seed=4)
    _, T1, _, _ = _ooc(pkg, A, b, 1, 3, want_uv=False, pin=True)
    _, T2, _, _ = _ooc(pkg, A, b, 1, 3, want_uv=False, pin=False)
    assert torch.equal(T1, T2)
    ref = oracle.randutv(A, b, 1, 3, want_u=False, want_v=False)
    assert rel(T1, ref.T) < 1e-12


def test_ooc_budget_changes_only_rounding(pkg):
    """A larger budget cuts the passes into fewer panels: the same
    factorization up to rounding order, and the same bytes copied (every
    region is read, and written back if updated, once per pass)."""
    m, n, b = 700, 500, 64
    A = inputs.matrix("linear", m, n, seed=9)
    lo = pkg.randutv_ooc_min_device_bytes(m, n, b)
    U1, T1, V1, mv1 = _ooc(pkg, A, b, 1, 1, device_bytes=lo)
    U2, T2, V2, mv2 = _ooc(pkg, A, b, 1, 1, device_bytes=8 * lo)
    assert rel(T1, T2) < 1e-12 and rel(U1, U2) < 1e-12 and rel(V1, V2) < 1e-12
    assert mv1 == mv2
    U3, T3, V3, _ = _ooc(pkg, A, b, 1, 1, device_bytes=lo)
    assert torch.equal(T1, T3) and torch.equal(U1, U3) and torch.equal(V1, V3)  # deterministic


def test_ooc_reports_nonfinite(pkg):
    A = inputs.gaussian(64, 64, seed=1)
    A[5, 7] = float("nan")
    with pytest.raises(pkg.RandutvError) as ei:
        _ooc(pkg, A, 16, 1, 0)
    assert ei.value.status == 2

"""randUTV by blocks on the GPU (§3.2.2-3.2.4) against the by-blocks oracle.

The in-HBM executor and the out-of-HBM executor with its LRU block cache run
the analyzer's task list; both are compared element by element with
oracle.randutv_ab (U, T, V at 1e-12 relative on spectra whose singular
values are separated, or at 10x the oracle's own movement under a
rounding-level perturbation of A where that floor is higher), checked for
the invariants of the factorization, and the cache's I/O is checked against
the analyzer's model of the dispatcher.
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


def sensitivity(A, b, q, seed):
    """How far the oracle's U, T, V move when A moves at rounding level (two
    perturbations of size 1e-16 max|A|): the factorization fixes U and V only
    to about eps ||A|| / gap, so a parity gate sits at 10x this floor where
    the floor is above 1e-13."""
    ref = oracle.randutv_ab(A, b, q, seed)
    sens = {"U": 0.0, "T": 0.0, "V": 0.0}
    for s in (5, 6):
        g = torch.Generator().manual_seed(s)
        Ap = A + torch.randn(A.shape, generator=g, dtype=f64) * 1e-16 * float(A.abs().max())
        f = oracle.randutv_ab(Ap, b, q, seed)
        for k in sens:
            sens[k] = max(sens[k], rel(getattr(f, k), getattr(ref, k)))
    return ref, {k: max(1e-12, 10.0 * v) for k, v in sens.items()}


CASES = [("linear", 256, 256, 64, 1), ("linear", 300, 260, 64, 1), ("linear", 333, 517, 64, 2),
         ("linear", 517, 333, 128, 0), ("exp40", 200, 200, 32, 1), ("linear", 96, 80, 16, 1),
         ("gauss", 9, 1, 4, 0), ("gauss", 1, 7, 4, 1), ("linear", 64, 64, 64, 1)]


@pytest.mark.parametrize("kind,m,n,b,q", CASES)
@pytest.mark.parametrize("nstreams", [1, 4])
def test_ab_matches_oracle(pkg, kind, m, n, b, q, nstreams):
    A = inputs.matrix(kind, m, n, seed=3) if min(m, n) > 1 else inputs.gaussian(m, n, seed=3)
    U, T, V = pkg.randutv_factor_ab(pkg.to_colmajor(A, "cuda"), b, q, 7, nstreams=nstreams)
    torch.cuda.synchronize()
    assert pkg.randutv_stream_status() == 0
    U, T, V = U.cpu(), T.cpu(), V.cpu()
    ref, gate = sensitivity(A, b, q, 7)
    assert oracle.recon_error(A, U, T, V) < 1e-13
    assert float(torch.tril(T, -1).abs().max()) == 0.0
    assert rel(T, ref.T) < gate["T"]
    if kind != "gauss":
        assert rel(U, ref.U) < gate["U"], (rel(U, ref.U), gate)
        assert rel(V, ref.V) < gate["V"], (rel(V, ref.V), gate)


def test_ab_is_deterministic_and_reports_nonfinite(pkg):
    A = inputs.matrix("exp40", 300, 280, seed=5)
    a = pkg.randutv_factor_ab(pkg.to_colmajor(A, "cuda"), 32, 1, 1, nstreams=8)
    b = pkg.randutv_factor_ab(pkg.to_colmajor(A, "cuda"), 32, 1, 1, nstreams=3)
    torch.cuda.synchronize()
    assert all(torch.equal(x, y) for x, y in zip(a, b))
    A[7, 9] = float("nan")
    pkg.randutv_factor_ab(pkg.to_colmajor(A, "cuda"), 32, 1, 1)
    assert pkg.randutv_stream_status() == 2


@pytest.mark.parametrize("m,n,b,q,extra", [(256, 256, 64, 1, 0), (300, 260, 64, 1, 3),
                                           (333, 517, 64, 2, 40), (517, 333, 128, 0, 8),
                                           (200, 200, 64, 1, 100)])
def test_ooc_ab_matches_oracle_and_the_io_model(pkg, m, n, b, q, extra):
    A = inputs.matrix("linear", m, n, seed=4)
    Th = pkg.colmajor_empty(m, n, device="cpu", pin=True)
    Th.copy_(A)
    Uh = pkg.colmajor_empty(m, m, device="cpu", pin=True)
    Vh = pkg.colmajor_empty(n, n, device="cpu", pin=True)
    bb = min(b, m, n)
    dev = pkg.randutv_ooc_ab_min_device_bytes(m, n, b) + extra * bb * bb * 8
    io = pkg.randutv_factor_ooc_ab(Th, b, q, 7, Uh, Vh, device_bytes=dev)
    ref, gate = sensitivity(A, b, q, 7)
    assert rel(Th, ref.T) < gate["T"]
    assert rel(Uh, ref.U) < gate["U"] and rel(Vh, ref.V) < gate["V"], (rel(Uh, ref.U),
                                                                       rel(Vh, ref.V), gate)
    # the cache's copies are exactly those of an LRU cache of as many tiles
    # of A, U and V (least recently used first, ties to the lowest slot,
    # written back when modified, all modified tiles written at the end)
    want = _lru_io(pkg.ab_tasks(m, n, b, q=q, want_u=True, want_v=True), 8 + extra)
    assert (io["reads"], io["writes"]) == want


def _lru_io(tasks, nslots):
    slot, last, dirty = [None] * nslots, [-1] * nslots, [False] * nslots
    reads = writes = 0
    for t, (_, _, ins, outs) in enumerate(tasks):
        mine = set(ins) | set(outs)

        def place(x):
            nonlocal writes
            free = [s for s in range(nslots) if slot[s] is None]
            if free:
                s = free[0]
            else:
                s = min((s for s in range(nslots) if slot[s] not in mine), key=lambda s: (last[s], s))
                if dirty[s]:
                    writes += 1
            slot[s], dirty[s] = x, False
        for x in ins:
            if x[0] in "AUV" and x not in slot:
                place(x)
                reads += 1
        for x in outs:
            if x[0] in "AUV" and x not in slot:
                place(x)
        for s in range(nslots):
            if slot[s] in mine:
                last[s] = t
                if slot[s] in outs:
                    dirty[s] = True
    return reads, writes + sum(dirty)

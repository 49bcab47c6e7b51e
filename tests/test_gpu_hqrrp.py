"""HQRRP on the GPU (A P = Q R, pivots from a Gaussian sketch per block,
§2.2) against the FP64 oracle.

The inputs are seeded so that every pivot decision of the oracle is clear
(best norm^2 over the runner-up above 1 + 1e-8; the closest of these cases is
1 + 3e-5, far above the FP64 rounding of either side), and the test asserts
that this holds before it compares: the permutation exactly, R and Q at
1e-12.  (At a near-tie either choice would be a valid factorization, and
only the invariants could be compared.)
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


def _gpu(pkg, A, b, seed, want_q=True):
    Q, R, perm = pkg.randutv_hqrrp(pkg.to_colmajor(A, "cuda"), b, seed, want_q)
    assert pkg.randutv_stream_status() == 0
    return (Q.cpu() if Q is not None else None), R.cpu(), perm.cpu()


def _invariants(A, Q, R, perm, tol=1e-13):
    m, n = A.shape
    assert sorted(perm.tolist()) == list(range(n))
    assert float(torch.tril(R, -1).abs().max()) == 0.0
    assert rel(Q @ R, A[:, perm]) < tol
    assert float((Q.T @ Q - torch.eye(m, dtype=f64)).norm()) / m ** 0.5 < tol


@pytest.mark.parametrize("m,n,b", [(120, 80, 16), (200, 200, 32), (97, 61, 8), (300, 120, 64),
                                   (64, 64, 64), (50, 1, 4), (40, 40, 1), (130, 100, 256)])
def test_hqrrp_matches_oracle(pkg, m, n, b):
    A = inputs.gaussian(m, n, seed=m * 7 + n)
    Q, R, perm = _gpu(pkg, A, b, 5)
    ref = oracle.hqrrp(A, b, 5)
    _invariants(A, Q, R, perm)
    assert min(ref.gaps) > 1.0 + 1e-8   # every pivot decision is clear: compare element-wise
    assert torch.equal(perm, ref.perm)
    assert rel(R, ref.R) < 1e-12
    assert rel(Q, ref.Q) < 1e-12


def test_hqrrp_invariants_at_size(pkg):
    m, n, b = 1536, 1024, 128
    A = inputs.matrix("smooth", m, n, seed=2)
    Q, R, perm = _gpu(pkg, A, b, 1)
    _invariants(A, Q, R, perm, tol=1e-13)
    Q2, R2, perm2 = _gpu(pkg, A, b, 1, want_q=False)
    assert Q2 is None and torch.equal(R2, R) and torch.equal(perm2, perm)  # Q does not change R


def test_hqrrp_reveals_rank(pkg):
    m = n = 256
    r = 40
    sig = torch.where(torch.arange(n) < r, torch.ones(n, dtype=f64), torch.full((n,), 1e-10, dtype=f64))
    A = inputs.prescribed(m, n, sig, seed=4)
    _, R, _ = _gpu(pkg, A, 16, 3)
    d = torch.diagonal(R).abs()
    assert float(d[:r].min()) > 1e-3
    assert float(d[r:].max()) < 1e-8


def test_hqrrp_is_deterministic_and_reports_nonfinite(pkg):
    A = inputs.gaussian(300, 200, seed=9)
    a = _gpu(pkg, A, 32, 2)
    b = _gpu(pkg, A, 32, 2)
    assert all(torch.equal(x, y) for x, y in zip(a, b))
    A[3, 4] = float("inf")
    pkg.randutv_hqrrp(pkg.to_colmajor(A, "cuda"), 32, 2, True)
    assert pkg.randutv_stream_status() == 2

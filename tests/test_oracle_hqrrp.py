"""Pins of the HQRRP oracle (§2.2) against things other than itself.

* With the identity in place of the Gaussian sketch, every block step's CPQR
  runs on the trailing matrix itself, and blocked HQRRP becomes the
  traditional column-pivoted QR: its permutation must equal LAPACK's
  dgeqp3 (scipy.linalg.qr with pivoting) for any block size, and |diag R|
  must match.
* With the Philox sketch: A P = Q R, Q orthogonal, R upper trapezoidal with
  exact zeros, P a permutation; the sketch is the transpose of the stream-6
  Philox array of the step.
* On a matrix of numerical rank r, the first r diagonal entries of R stay
  above the gap and the rest fall below it (the factorization reveals rank).
"""
import numpy as np
import pytest
import scipy.linalg as sl
import torch

import oracle
from oracle import philox
from paper_2002_06960_gb300 import inputs

f64 = torch.float64


def _eye_sketch(i, rm, bi):
    return torch.eye(rm, dtype=f64)


@pytest.mark.parametrize("m,n,b", [(60, 40, 8), (50, 50, 1), (45, 33, 7), (30, 30, 30), (80, 24, 5)])
def test_identity_sketch_is_lapack_cpqr(m, n, b):
    A = inputs.gaussian(m, n, seed=m + n)
    f = oracle.hqrrp(A, b, 0, omega=_eye_sketch)
    _, Rs, Ps = sl.qr(A.numpy(), pivoting=True)
    assert min(f.gaps) > 1.0 + 1e-9  # no near-ties: the pivot sequence is unique
    assert (f.perm.numpy() == Ps).all()
    d, ds = np.abs(np.diag(f.R.numpy())), np.abs(np.diag(Rs))
    assert np.abs(d - ds).max() <= 1e-13 * ds[0]


@pytest.mark.parametrize("m,n,b", [(64, 48, 8), (40, 40, 16), (33, 17, 5), (20, 20, 1), (9, 9, 9)])
def test_factorization_invariants(m, n, b):
    A = inputs.matrix("exp16", m, n, seed=3)
    f = oracle.hqrrp(A, b, 11)
    assert sorted(f.perm.tolist()) == list(range(n))
    assert float((A[:, f.perm] - f.Q @ f.R).norm() / A.norm()) < 1e-14
    assert float((f.Q.T @ f.Q - torch.eye(m, dtype=f64)).norm()) < 1e-13
    assert float(torch.tril(f.R, -1).abs().max()) == 0.0
    # T only gives the same R and P
    g = oracle.hqrrp(A, b, 11, want_q=False)
    assert torch.equal(g.R, f.R) and torch.equal(g.perm, f.perm)


def test_sketch_is_the_transposed_philox_array():
    # step 2, 37 x 5: G = Omega^T with Omega the stream-6 array of that step
    Om = oracle.sketch_omega(9, 2, 37, 5)
    ref = philox.sketch(9, 2, 37, 5, 0, 6)
    assert np.array_equal(Om.numpy(), ref)
    assert not np.array_equal(ref, philox.sketch(9, 2, 37, 5, 0, 0))  # not the randUTV sketch


def test_first_block_pivots_are_the_cpqr_of_the_sketch():
    A = inputs.gaussian(40, 30, seed=5)
    b = 6
    f = oracle.hqrrp(A, b, 2)
    Y = oracle.sketch_omega(2, 0, 40, b).T @ A
    # the CPQR of Y, by brute force: at each step the remaining column of
    # largest norm after projecting out the chosen ones
    chosen = []
    for j in range(b):
        if chosen:
            Qc, _ = torch.linalg.qr(Y[:, chosen])
            Z = Y - Qc @ (Qc.T @ Y)
        else:
            Z = Y
        nrm = (Z ** 2).sum(0)
        nrm[chosen] = -1.0
        chosen.append(int(torch.argmax(nrm)))
    assert f.perm[:b].tolist() == chosen


def test_rank_revealing_on_a_gap():
    m = n = 64
    r = 20
    sig = torch.where(torch.arange(n) < r, torch.ones(n, dtype=f64), torch.full((n,), 1e-9, dtype=f64))
    A = inputs.prescribed(m, n, sig, seed=4)
    f = oracle.hqrrp(A, 8, 1)
    d = torch.diagonal(f.R).abs()
    assert float(d[:r].min()) > 1e-3
    assert float(d[r:].max()) < 1e-7

"""Pins of the randUTV-by-blocks oracle (§3.2.2-3.2.3), on the CPU.

* One tile (m, n <= b): the by-blocks loop is the blocked loop, bit for bit.
* The triangular-dense QR against the explicit product of its reflectors:
  [R; X] = H_1 ... H_c [R'; 0], the top of W is exactly the identity, and
  I - W S W^T equals the product.
* Invariants of every output: reconstruction, orthogonality, exact zeros
  below the diagonal and inside each diagonal block, ||T||_F = ||A||_F.
* Against the blocked loop (whose QRs are whole-panel): the first block of
  V spans the sketched range (the same in both), the first block of U spans
  the same space, and the first diagonal block has the same singular values;
  later blocks differ by the orthonormal completion the method leaves free.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2002_06960_gb300 import inputs

f64 = torch.float64


def _explicit_q(W, tau):
    n = W.shape[0]
    Q = torch.eye(n, dtype=f64)
    for j in range(W.shape[1]):
        w = W[:, j:j + 1]
        Q = Q @ (torch.eye(n, dtype=f64) - tau[j] * (w @ w.T))
    return Q


@pytest.mark.parametrize("c,r", [(4, 4), (6, 3), (5, 9), (1, 2)])
def test_td_qr_against_explicit_reflectors(c, r):
    g = torch.Generator().manual_seed(c * 10 + r)
    R = torch.triu(torch.randn(c, c, generator=g, dtype=f64))
    X = torch.randn(r, c, generator=g, dtype=f64)
    Rn, W, S = oracle.td_qr(R, X)
    assert torch.equal(W[:c], torch.eye(c, dtype=f64))          # top of W: exactly I
    tau = torch.diagonal(S)
    Q = _explicit_q(W, tau)
    M = torch.cat([R, X], 0)
    RZ = torch.cat([Rn, torch.zeros(r, c, dtype=f64)], 0)
    assert float((Q @ RZ - M).abs().max()) < 1e-13
    assert float((Q.T @ Q - torch.eye(c + r, dtype=f64)).abs().max()) < 1e-14
    assert float(((torch.eye(c + r, dtype=f64) - W @ S @ W.T) - Q).abs().max()) < 1e-14
    # |R'| has the column norms a QR of [R; X] must have
    _, Rnp = np.linalg.qr(M.numpy())
    assert np.allclose(np.abs(np.diag(Rnp)), np.abs(torch.diagonal(Rn).numpy()), rtol=1e-12)


@pytest.mark.parametrize("m,n,b,q", [(30, 30, 64, 1), (50, 50, 50, 2), (7, 7, 16, 0)])
def test_one_tile_is_the_blocked_loop(m, n, b, q):
    # one tile needs m = n <= b: otherwise the grid restarts at p = min(m, n)
    A = inputs.gaussian(m, n, seed=m + n)
    f = oracle.randutv_ab(A, b, q, 3)
    g = oracle.randutv(A, b, q, 3)
    assert torch.equal(f.T, g.T) and torch.equal(f.U, g.U) and torch.equal(f.V, g.V)


def _invariants(A, f, b):
    m, n = A.shape
    assert oracle.recon_error(A, f.U, f.T, f.V) < 1e-13
    assert oracle.orth_error(f.U) < 1e-13 and oracle.orth_error(f.V) < 1e-13
    assert float(torch.tril(f.T, -1).abs().max()) == 0.0
    p = min(m, n)
    for k in range(0, p, b):
        bi = min(b, p - k)
        blk = f.T[k:k + bi, k:k + bi]
        assert float((blk - torch.diag(torch.diagonal(blk))).abs().max()) == 0.0
        assert bool((torch.diagonal(blk) >= 0).all())
    assert abs(float(f.T.norm()) / float(A.norm()) - 1.0) < 1e-13


@pytest.mark.parametrize("kind,m,n,b,q", [("exp40", 96, 96, 16, 1), ("gauss", 70, 50, 16, 0),
                                          ("exp40", 50, 83, 16, 2), ("gauss", 33, 33, 8, 1),
                                          ("exp40", 64, 40, 32, 1)])
def test_invariants_and_first_block(kind, m, n, b, q):
    # the spans are compared where the sketch's range is well conditioned
    # ((s_0 / s_(b-1))^(2q+1) far below 1e16), so that both QRs determine it
    A = inputs.matrix(kind, m, n, seed=2)
    f = oracle.randutv_ab(A, b, q, 5)
    _invariants(A, f, b)
    g = oracle.randutv(A, b, q, 5)
    bi = min(b, m, n)
    # the same sketched range: the projectors onto the first blocks agree
    Pv = f.V[:, :bi] @ f.V[:, :bi].T
    Pg = g.V[:, :bi] @ g.V[:, :bi].T
    assert float((Pv - Pg).abs().max()) < 1e-11
    Pu = f.U[:, :bi] @ f.U[:, :bi].T
    Pug = g.U[:, :bi] @ g.U[:, :bi].T
    assert float((Pu - Pug).abs().max()) < 1e-11
    d, d0 = torch.diagonal(f.T)[:bi], torch.diagonal(g.T)[:bi]
    assert float(((d - d0).abs() / d0.clamp_min(1e-300)).max()) < 1e-11
    # and the tiles do change the rest: the second block's trailing matrix differs
    if min(m, n) > 2 * b:
        assert float((f.T - g.T).abs().max()) > 1e-8


def test_rank_revealing_on_a_step_spectrum():
    n, r, b = 96, 24, 16
    sig = torch.where(torch.arange(n) < r, torch.ones(n, dtype=f64), torch.full((n,), 1e-8, dtype=f64))
    A = inputs.prescribed(n, n, sig, seed=4)
    f = oracle.randutv_ab(A, b, 2, 1)
    _invariants(A, f, b)
    # the numerical rank shows in the diagonal and in the trailing block
    d = torch.diagonal(f.T)
    assert float(d[:r].min()) > 0.5
    assert float(d[r + b:].max()) < 1e-7
    assert float(f.T[r + b:, r + b:].norm()) < 1e-6

"""Oracle randUTV by blocks (randUTV_AB): the blocked loop with the QRs done by blocks.

TEST INFRASTRUCTURE: see the package header.  Nothing in the product path
imports this file.

Follows §3.2.2-3.2.3 of Heavner, Martinsson & Quintana-Orti (arXiv
2002.06960): randUTV written for algorithms-by-blocks is the loop of §3.1
(the update list of Fig. 2), except that every unpivoted QR works on b x b
blocks (QR_AB): a dense QR of the leading block of the block column, then,
for each block below it, the QR of the upper triangular R stacked on that
dense block (the "triangular-dense" QR), each with its own compact-WY factor.
The orthogonal factor of the column is the product of these, taken in that
order, and it is applied in that order.  The sketch, the power iteration, the
small SVD and its folds are those of the blocked loop (``oracle.randutv``).

Reading taken: the blocks are the tiles of a grid whose boundaries are the
block steps (multiples of b) up to p = min(m, n), then p + b t, so that every
diagonal block is one tile.  The result differs from the blocked loop's in
the parts of U, T and V that the method leaves free (the columns of each
step's Q beyond its first b are another orthonormal completion, so later
trailing matrices differ by an orthogonal factor); the first block of U and
V spans the same space and the first diagonal block has the same singular
values.
"""
from __future__ import annotations

import torch

from .randutv import Factorization, householder_qr, sketch, small_svd, wy_factor

f64 = torch.float64


def tile_starts(extent: int, p: int, b: int) -> list[int]:
    """Tile boundaries along one dimension (the last entry is ``extent``)."""
    s = list(range(0, p, b)) + list(range(p, extent, b))
    return s + [extent]


def td_qr(R: torch.Tensor, X: torch.Tensor):
    """QR of [R; X], R upper triangular c x c, X dense r x c (Comp_td_QR).

    Returns (R', W, S): [R; X] = (I - W S W^T) [R'; 0] with W (c + r) x c.
    The rows of R below its diagonal are zero, so the top c rows of W are
    the identity and only the bottom r rows carry the vectors.
    """
    W, tau, Rn = householder_qr(torch.cat([R, X], 0))
    return Rn, W, wy_factor(W, tau)


def _qr_by_blocks(col: list[torch.Tensor]):
    """QR_AB of a column of blocks col[0], col[1], ...: the list of factors
    (blocks touched, W, S) in order, and the final R of the leading block."""
    W0, tau0, R = householder_qr(col[0])
    factors = [((0,), W0, wy_factor(W0, tau0))]
    for l in range(1, len(col)):
        R, W, S = td_qr(R, col[l])
        factors.append(((0, l), W, S))
    return factors, R


def randutv_ab(A: torch.Tensor, b: int, q: int, seed: int, want_u: bool = True,
               want_v: bool = True) -> Factorization:
    """A = U T V^T by randUTV_AB (QRs by blocks of b)."""
    A = A.to(f64)
    m, n = A.shape
    p = min(m, n)
    rs, cs = tile_starts(m, p, b), tile_starts(n, p, b)
    Mt, Nt = len(rs) - 1, len(cs) - 1
    T = A.clone()
    U = torch.eye(m, dtype=f64) if want_u else None
    V = torch.eye(n, dtype=f64) if want_v else None
    steps = (p + b - 1) // b
    for k in range(steps):
        k0, bi = cs[k], cs[k + 1] - cs[k]
        rows = lambda i: slice(rs[i], rs[i + 1])      # noqa: E731
        cols = lambda j: slice(cs[j], cs[j + 1])      # noqa: E731
        # -- right transform: sketch, power iteration, QR_AB of Y, X <- X Q --
        if k + 1 < Nt:
            G = sketch(seed, k, m - rs[k], bi)
            T22 = T[rs[k]:, k0:].clone()
            Y = T22.T @ G
            for _ in range(q):
                Y = T22.T @ (T22 @ Y)
            ycol = [Y[cs[j] - k0:cs[j + 1] - k0] for j in range(k, Nt)]
            factors, _ = _qr_by_blocks(ycol)
            for X in ([T] + ([V] if V is not None else [])):
                for blocks, W, S in factors:
                    idx = torch.cat([torch.arange(cs[k + l], cs[k + l + 1]) for l in blocks])
                    Xc = X[:, idx].clone()
                    X[:, idx] = Xc - (Xc @ W) @ S @ W.T
        # -- left transform: QR_AB of the block column, X <- Q^T X, U <- U Q --
        if k + 1 < Mt:
            acol = [T[rows(i), cols(k)].clone() for i in range(k, Mt)]
            factors, R = _qr_by_blocks(acol)
            for blocks, W, S in factors:
                idx = torch.cat([torch.arange(rs[k + l], rs[k + l + 1]) for l in blocks])
                if cs[k + 1] < n:
                    Xc = T[idx, cs[k + 1]:].clone()
                    T[idx, cs[k + 1]:] = Xc - W @ (S.T @ (W.T @ Xc))
                if U is not None:
                    Xc = U[:, idx].clone()
                    U[:, idx] = Xc - (Xc @ W) @ S @ W.T
            T[rows(k), cols(k)] = R                  # Keep_upper_triang
            T[rs[k + 1]:, cols(k)] = 0.0             # Set_to_zero
        # -- small SVD of the diagonal block and its folds (§3.1 steps 3-6) --
        Us, D, Vs = small_svd(T[rows(k), cols(k)].clone())
        T[rows(k), cols(k)] = torch.diag(D)
        T[:rs[k], cols(k)] = T[:rs[k], cols(k)] @ Vs
        T[rows(k), cs[k + 1]:] = Us.T @ T[rows(k), cs[k + 1]:]
        if V is not None:
            V[:, cols(k)] = V[:, cols(k)] @ Vs
        if U is not None:
            U[:, rows(k)] = U[:, rows(k)] @ Us
    return Factorization(U, T, V, steps, p)

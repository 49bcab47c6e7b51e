"""Oracle HQRRP: blocked column-pivoted QR with randomized pivot selection.

TEST INFRASTRUCTURE: see the package header.  Nothing in the product path
imports this file.

Follows §2.1-2.2 of Heavner, Martinsson & Quintana-Orti (arXiv 2002.06960):
A P = Q R with R upper trapezoidal.  Block step i (offset k = i b, width
bi = min(b, n - k), rm = m - k, rn = n - k):

1. draw G (bi x rm) with i.i.d. N(0,1) entries;
2. Y = G R22 (bi x rn), R22 = R(k:, k:);
3. bi steps of traditional column-pivoted QR of Y (Businger-Golub: at step
   j take the remaining column of largest norm over rows j:, swap it to
   position j, apply its Householder reflector to the rest), which gives the
   permutation P22 of the rn trailing columns;
4. permute the trailing columns of R (all m rows) and of P by P22;
5. unpivoted Householder QR of R(k:, k:k+bi), and its reflectors applied
   from the left to R(k:, k+bi:) and accumulated into Q(:, k:).

The sketch is drawn anew at each step (the paper's implementation does not
downdate it).  Readings where the paper is silent (also in the design notes):

* G is the transpose of the rm x bi Philox sketch of step i on stream 6
  (element l = r + c rm of the rm x bi array, as for the randUTV sketch), so
  Y = Omega^T R22.  The last block has bi < b rows in G.
* The CPQR norms are taken afresh at every pivot step over rows j: (the
  textbook's downdated norms agree in exact arithmetic).  Ties go to the
  lowest column position.
* m >= n, as the paper assumes.

The step of the trailing permutation is the composition of the bi swaps
(j, p_j) in order, LAPACK's convention for a partial CPQR.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import philox
from .randutv import householder_qr, householder_reflector, wy_factor

f64 = torch.float64
STREAM_HQRRP = 6


@dataclass
class PivotedQR:
    Q: torch.Tensor | None  # m x m orthogonal
    R: torch.Tensor         # m x n upper trapezoidal
    perm: torch.Tensor      # (n,) int64: column j of A P is column perm[j] of A
    gaps: list              # per pivot decision: best norm^2 / runner-up norm^2 (1 if none)


def sketch_omega(seed: int, step: int, rows: int, cols: int) -> torch.Tensor:
    """Omega (rows x cols) of step `step`; G = Omega^T."""
    return torch.from_numpy(philox.sketch(seed, step, rows, cols, 0, STREAM_HQRRP))


def cpqr_pivots(Y: torch.Tensor, steps: int):
    """`steps` steps of traditional CPQR of Y (r x c): the swap targets p_j
    (position swapped with j at step j) and the norm gap of each decision."""
    Y = Y.clone()
    r, c = Y.shape
    swaps, gaps = [], []
    for j in range(steps):
        nrm = (Y[j:, j:] ** 2).sum(dim=0)
        p = j + int(torch.argmax(nrm))  # torch.argmax returns the first maximum
        srt = torch.sort(nrm, descending=True).values
        gaps.append(float(srt[0] / srt[1]) if srt.numel() > 1 and float(srt[1]) > 0 else float("inf"))
        swaps.append(p)
        if p != j:
            Y[:, [j, p]] = Y[:, [p, j]]
        v, tau, beta = householder_reflector(Y[j:, j].clone())
        if j + 1 < c:
            X = Y[j:, j + 1:].clone()
            w = tau * (v @ X)
            Y[j:, j + 1:] = X - torch.outer(v, w)
        Y[j, j] = beta
        Y[j + 1:, j] = 0.0
    return swaps, gaps


def apply_swaps(X: torch.Tensor, swaps) -> None:
    """Columns of X (in place): swap j <-> p_j for j = 0, 1, ... in order."""
    for j, p in enumerate(swaps):
        if p != j:
            X[..., [j, p]] = X[..., [p, j]]


def hqrrp(A: torch.Tensor, b: int, seed: int, want_q: bool = True,
          omega=None) -> PivotedQR:
    """A P = Q R by HQRRP.  ``omega(step, rm, bi)`` replaces the Philox sketch
    (a test hook: the identity sketch reduces the method to plain CPQR)."""
    A = A.to(f64)
    m, n = A.shape
    if m < n:
        raise ValueError("HQRRP needs m >= n")
    R = A.clone()
    Q = torch.eye(m, dtype=f64) if want_q else None
    perm = torch.arange(n, dtype=torch.int64)
    gaps = []
    for i, k in enumerate(range(0, n, b)):
        bi = min(b, n - k)
        rm = m - k
        Om = omega(i, rm, bi) if omega is not None else sketch_omega(seed, i, rm, bi)
        Y = Om.T @ R[k:, k:]
        swaps, g = cpqr_pivots(Y, bi)
        gaps.extend(g)
        trail = R[:, k:]
        apply_swaps(trail, swaps)
        pk = perm[k:].clone()
        apply_swaps(pk, swaps)
        perm[k:] = pk
        W, tau, Rb = householder_qr(R[k:, k:k + bi])
        S = wy_factor(W, tau)
        # the panel itself: R on and above the diagonal, exact zeros below
        R[k:k + bi, k:k + bi] = Rb
        R[k + bi:, k:k + bi] = 0.0
        if k + bi < n:
            X = R[k:, k + bi:]
            R[k:, k + bi:] = X - W @ (S.T @ (W.T @ X))
        if want_q:
            Qk = Q[:, k:]
            Q[:, k:] = Qk - (Qk @ W) @ (W @ S.T).T
    return PivotedQR(Q, R, perm, gaps)

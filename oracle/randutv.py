"""Oracle randUTV: a plain FP64 CPU restatement of the method, step by step.

TEST INFRASTRUCTURE: see the package header.  Nothing in the product path
imports this file.

Follows §3.1 of Heavner, Martinsson & Quintana-Orti, "Computing rank-revealing
factorizations of matrices stored out-of-core" (arXiv 2002.06960): steps 1-6
of the blocked loop, the construction of V-hat by a Gaussian sketch and power
iteration, and the update list of Fig. 2 (randUTV written for
algorithms-by-blocks).  Everything is torch.float64 on the CPU; the only
library primitives used as steps are the matrix product and, for the b x b
block, the library SVD.  Nothing is blocked, fused or reordered beyond what
those passages state.

Readings taken where the paper is silent or garbled (all also listed in the
design notes of the repository):

* Loop runs while k < p = min(m, n) with block width bi = min(b, p - k); the
  sketch has bi columns (the guard printed in Fig. 2 does not terminate for
  m > n).
* The right transform updates all m rows of the trailing columns, as
  T^(i) = U^(i)* T^(i-1) V^(i) with block-diagonal V^(i) requires (§3.1 step 6).
* The left update applies Q^T: T2 <- T2 - W S^T (W^T T2) (the formula in
  Fig. 2 is dimensionally garbled).
* Right transform only when rn > bi, left QR only when rm > bi; the small
  SVD is always taken (Fig. 3: the last diagonal block gets only an SVD).
* Householder convention (LAPACK's): for x = (alpha, x2), s = ||x2||;
  s == 0 gives tau = 0 and H = I, even for alpha < 0; otherwise
  beta = -sgn(alpha) sqrt(alpha^2 + s^2) with sgn(0) = +1,
  tau = (beta - alpha)/beta, v = (1, x2/(alpha - beta)).
* The product H_1 ... H_b is I - W S W^T with S upper triangular, built
  column by column: S_jj = tau_j, S(0:j, j) = -tau_j S(0:j,0:j) W(:,0:j)^T w_j
  (the paper calls this factor T_V / T_U; S here, to keep T for the middle
  factor).
* Small SVD: D descending and >= 0; each column of V_s is signed so that its
  entry of largest magnitude (lowest index on ties) is positive, and the
  matching column of U_s is flipped with it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import philox

f64 = torch.float64


# ---------------------------------------------------------------------------
# Householder QR and its compact-WY factor (Fig. 2: unpivoted_QR, W and T_V)
# ---------------------------------------------------------------------------

def householder_reflector(x: torch.Tensor):
    """Reflector H = I - tau v v^T with H x = beta e_1 (LAPACK convention).

    Returns (v, tau, beta); v[0] == 1.
    """
    alpha = x[0]
    x2 = x[1:]
    s = torch.linalg.vector_norm(x2) if x2.numel() else torch.zeros((), dtype=x.dtype)
    v = torch.zeros_like(x)
    v[0] = 1.0
    if float(s) == 0.0:
        return v, torch.zeros((), dtype=x.dtype), alpha.clone()
    sgn = 1.0 if float(alpha) >= 0.0 else -1.0
    beta = -sgn * torch.sqrt(alpha * alpha + s * s)
    tau = (beta - alpha) / beta
    v[1:] = x2 / (alpha - beta)
    return v, tau, beta


def householder_qr(Y: torch.Tensor):
    """Unpivoted Householder QR of an r x c matrix (r >= c), one column at a time.

    Returns W (r x c, unit lower trapezoidal, explicit), tau (c,) and R (c x c
    upper triangular), with Y = H_1 ... H_c [R; 0].
    """
    A = Y.clone()
    r, c = A.shape
    W = torch.zeros(r, c, dtype=A.dtype)
    tau = torch.zeros(c, dtype=A.dtype)
    for j in range(c):
        v, t, beta = householder_reflector(A[j:, j].clone())
        W[j:, j] = v
        tau[j] = t
        # apply H_j to the trailing columns
        if j + 1 < c:
            X = A[j:, j + 1:].clone()
            w = t * (v @ X)
            A[j:, j + 1:] = X - torch.outer(v, w)
        A[j, j] = beta
        A[j + 1:, j] = 0.0
    R = torch.triu(A[:c, :])
    return W, tau, R


def wy_factor(W: torch.Tensor, tau: torch.Tensor) -> torch.Tensor:
    """S (c x c upper triangular) with H_1 ... H_c = I - W S W^T."""
    c = W.shape[1]
    S = torch.zeros(c, c, dtype=W.dtype)
    for j in range(c):
        S[j, j] = tau[j]
        if j > 0:
            z = W[:, :j].T @ W[:, j]
            S[:j, j] = -tau[j] * (S[:j, :j].clone() @ z)
    return S


# ---------------------------------------------------------------------------
# The b x b SVD (Fig. 2: [A11, U_SVD, V_SVD] := SVD(A11)) with fixed signs
# ---------------------------------------------------------------------------

def normalise_svd(Us: torch.Tensor, D: torch.Tensor, Vs: torch.Tensor):
    """Fix the sign freedom of an SVD: the largest-|.| entry of each V column is > 0."""
    Us = Us.clone()
    Vs = Vs.clone()
    for j in range(Vs.shape[1]):
        col = Vs[:, j].abs()
        idx = int(torch.nonzero(col == col.max())[0, 0])   # lowest index on ties
        if float(Vs[idx, j]) < 0.0:
            Vs[:, j] = -Vs[:, j]
            Us[:, j] = -Us[:, j]
    return Us, D, Vs


def small_svd(B: torch.Tensor):
    """SVD of a square block: B = Us diag(D) Vs^T, D descending, signs fixed."""
    Us, D, Vh = torch.linalg.svd(B)
    return normalise_svd(Us, D, Vh.T)


# ---------------------------------------------------------------------------
# randUTV (§3.1 steps 1-6; Fig. 2 update list)
# ---------------------------------------------------------------------------

@dataclass
class Factorization:
    U: torch.Tensor | None
    T: torch.Tensor
    V: torch.Tensor | None
    steps: int
    k: int


def block_schedule(m: int, n: int, b: int):
    """(i, k, bi, rm, rn, right, left) for every step of the blocked loop."""
    p = min(m, n)
    k = 0
    i = 0
    out = []
    while k < p:
        bi = min(b, p - k)
        rm, rn = m - k, n - k
        out.append((i, k, bi, rm, rn, rn > bi, rm > bi))
        k += bi
        i += 1
    return out


def sketch(seed: int, step: int, rows: int, cols: int, matrix_id: int = 0,
           f32: bool = False) -> torch.Tensor:
    """G of one step: i.i.d. N(0,1), rows x cols (§3.1, V-hat step 1).

    ``f32`` draws the batched form's FP32 normals (returned as FP64 values)."""
    if f32:
        return torch.from_numpy(philox.sketch_f32(seed, step, rows, cols, matrix_id)).to(f64)
    return torch.from_numpy(philox.sketch(seed, step, rows, cols, matrix_id))


def range_basis(T22: torch.Tensor, G: torch.Tensor, q: int) -> torch.Tensor:
    """Y = (T22^T T22)^q T22^T G (§3.1, V-hat step 2), no re-orthonormalisation."""
    Y = T22.T @ G
    for _ in range(q):
        Y = T22.T @ (T22 @ Y)
    return Y


def randutv(A: torch.Tensor, b: int, q: int, seed: int, want_u: bool = True,
            want_v: bool = True, matrix_id: int = 0, max_steps: int | None = None,
            state: Factorization | None = None, svd: bool = True,
            sketch_f32: bool = False) -> Factorization:
    """A = U T V^T by blocked randUTV.

    ``max_steps`` stops after that many steps (a partial factorization);
    ``state`` resumes from the result of an earlier call.  ``svd=False``
    leaves out the small SVDs (T is then block upper triangular); the spans
    of U(:, 0:k) and V(:, 0:k) at every block boundary k, and the trailing
    matrices of later steps, do not depend on them.  ``sketch_f32`` draws
    every G from the batched form's FP32 generator (the arithmetic stays FP64).
    """
    A = A.to(f64)
    m, n = A.shape
    if state is None:
        T = A.clone()
        U = torch.eye(m, dtype=f64) if want_u else None
        V = torch.eye(n, dtype=f64) if want_v else None
        done = 0
    else:
        T = state.T.clone()
        U = None if state.U is None else state.U.clone()
        V = None if state.V is None else state.V.clone()
        done = state.steps
    sched = block_schedule(m, n, b)
    last_k = 0
    steps = done
    for (i, k, bi, rm, rn, right, left) in sched:
        if i < done:
            continue
        if max_steps is not None and i >= max_steps:
            break
        # -- right transform: V-hat from the sketch (§3.1 step 1; Fig. 2) --
        # (the operands are copied out before each update is written back, so
        # that the function can also be differentiated by torch autograd)
        if right:
            G = sketch(seed, i, rm, bi, matrix_id, f32=sketch_f32)
            Y = range_basis(T[k:, k:].clone(), G, q)
            W, tau, _ = householder_qr(Y)
            S = wy_factor(W, tau)
            X = T[:, k:].clone()
            T[:, k:] = X - (X @ W) @ S @ W.T
            if V is not None:
                X = V[:, k:].clone()
                V[:, k:] = X - (X @ W) @ S @ W.T
        # -- left transform: QR of the new column panel (§3.1 step 2; Fig. 2) --
        if left:
            W, tau, R = householder_qr(T[k:, k:k + bi].clone())
            S = wy_factor(W, tau)
            T[k:, k:k + bi] = 0.0
            T[k:k + bi, k:k + bi] = R
            X = T[k:, k + bi:].clone()
            T[k:, k + bi:] = X - W @ (S.T @ (W.T @ X))
            if U is not None:
                X = U[:, k:].clone()
                U[:, k:] = X - (X @ W) @ S @ W.T
        # -- small SVD of the diagonal block and its fold-back (§3.1 steps 3-6) --
        if not svd:
            steps = i + 1
            last_k = k + bi
            continue
        Us, D, Vs = small_svd(T[k:k + bi, k:k + bi])
        T[k:k + bi, k:k + bi] = torch.diag(D)
        T[:k, k:k + bi] = T[:k, k:k + bi] @ Vs
        T[k:k + bi, k + bi:] = Us.T @ T[k:k + bi, k + bi:]
        if V is not None:
            V[:, k:k + bi] = V[:, k:k + bi] @ Vs
        if U is not None:
            U[:, k:k + bi] = U[:, k:k + bi] @ Us
        steps = i + 1
        last_k = k + bi
    return Factorization(U, T, V, steps, last_k)


def lowrank(A: torch.Tensor, k: int, b: int, q: int, seed: int) -> torch.Tensor:
    """A_k = U(:, 0:k) U(:, 0:k)^T A (§1.1: A_k = U(:,1:k) R(1:k,:) V^*).

    k is a multiple of b.  Only the k/b steps that fix the span of the first
    k columns of U are run, and without the small SVDs: they rotate columns
    inside a block and change neither that span nor the trailing matrix of
    any later step, so A_k is the same and is differentiable through the
    Householder steps alone (torch autograd of this function is the FP64
    reference gradient).
    """
    if k % b != 0:
        raise ValueError("k must be a multiple of b")
    steps = k // b
    f = randutv(A, b, q, seed, want_u=True, want_v=False, max_steps=steps, svd=False)
    Uk = f.U[:, :k]
    return Uk @ (Uk.T @ A.to(f64))


# ---------------------------------------------------------------------------
# error measures used with every result
# ---------------------------------------------------------------------------

def recon_error(A, U, T, V) -> float:
    A = A.to(f64)
    return float(torch.linalg.norm(A - U.to(f64) @ T.to(f64) @ V.to(f64).T) / torch.linalg.norm(A))


def orth_error(Q) -> float:
    Q = Q.to(f64)
    n = Q.shape[1]
    return float(torch.linalg.norm(Q.T @ Q - torch.eye(n, dtype=f64)) / np.sqrt(n))

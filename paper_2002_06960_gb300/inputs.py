"""Seeded synthetic test matrices for randUTV (input preparation only).

This module builds the matrices that the factorization is run on: i.i.d.
standard-normal matrices and matrices with a prescribed spectrum
A = Q1 diag(sigma) Q2^T.  It holds none of the factorization's own arithmetic:
the orthogonal factors come from the library QR of a Gaussian matrix, and the
random numbers come from ``torch.Generator`` streams, not from the sketch
generator of the method.  Both the CPU oracle and the GPU path are fed from
here, so a test hands the same A to both.

The paper's experiments use randomly generated dense FP64 matrices (§4.2.1);
the spectra below are the ones the workloads are defined with:

* ``exp40``   sigma_j = exp(-j/40)               (512 x 512 parity workload)
* ``smooth``  sigma_j = 10^(-8 j / p)            (smooth decay over 8 decades)
* ``step``    sigma_j = 1 for j < gap, else 1e-6 (gap = floor(p/10) unless given)
* ``exp16``   sigma_j = exp(-j/16)               (batched workload)
* ``linear``  sigma_j = 1 - j/(2p)               (well separated, no deep tail)

with j = 0 .. p-1 and p = min(m, n).
"""
from __future__ import annotations

import torch

# Stream ids keep the different uses of one seed apart.
STREAM_Q1 = 1
STREAM_Q2 = 2
STREAM_GAUSS = 3
STREAM_B = 4
STREAM_SIZES = 5


def _gen(seed: int, stream: int, device="cpu") -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed((int(seed) * 1_000_003 + int(stream) * 7919 + 12345) & 0x7FFF_FFFF_FFFF_FFFF)
    return g


def gaussian(m: int, n: int, seed: int, stream: int = STREAM_GAUSS,
             dtype=torch.float64, device="cpu") -> torch.Tensor:
    """i.i.d. N(0,1) matrix, m x n, from a seeded generator on ``device``."""
    g = _gen(seed, stream, device)
    return torch.randn(m, n, generator=g, dtype=dtype, device=device)


def haar_orthogonal(n: int, seed: int, stream: int, p: int | None = None,
                    device="cpu") -> torch.Tensor:
    """First p columns of a Haar-distributed orthogonal n x n matrix.

    Q is the orthogonal factor of the library Householder QR of a seeded
    Gaussian n x p matrix, with the column signs fixed so that diag(R) > 0.
    """
    p = n if p is None else p
    X = gaussian(n, p, seed, stream, device=device)
    Q, R = torch.linalg.qr(X, mode="reduced")
    s = torch.sign(torch.diagonal(R))
    s[s == 0] = 1
    return Q * s


def spectrum(kind: str, p: int, gap: int | None = None) -> torch.Tensor:
    j = torch.arange(p, dtype=torch.float64)
    if kind == "exp40":
        return torch.exp(-j / 40.0)
    if kind == "exp16":
        return torch.exp(-j / 16.0)
    if kind == "smooth":
        return torch.pow(10.0, -8.0 * j / p)
    if kind == "linear":
        return 1.0 - j / (2.0 * p)
    if kind == "step":
        g = p // 10 if gap is None else gap
        return torch.where(j < g, torch.ones_like(j), torch.full_like(j, 1e-6))
    raise ValueError(f"unknown spectrum {kind!r}")


def prescribed(m: int, n: int, sigma: torch.Tensor, seed: int,
               device="cpu") -> torch.Tensor:
    """A = Q1 diag(sigma) Q2^T with Haar Q1 (m x p) and Q2 (n x p), p = len(sigma)."""
    p = sigma.numel()
    Q1 = haar_orthogonal(m, seed, STREAM_Q1, p, device=device)
    Q2 = haar_orthogonal(n, seed, STREAM_Q2, p, device=device)
    return (Q1 * sigma.to(device=device, dtype=Q1.dtype)) @ Q2.T


def matrix(kind: str, m: int, n: int, seed: int, gap: int | None = None,
           device="cpu") -> torch.Tensor:
    """One of the named workloads: ``gauss`` or a spectrum name above."""
    if kind == "gauss":
        return gaussian(m, n, seed, device=device)
    return prescribed(m, n, spectrum(kind, min(m, n), gap), seed, device=device)


def batch_sizes(count: int, lo: int, hi: int, seed: int) -> list[tuple[int, int]]:
    """(m, n) pairs drawn independently and uniformly from [lo, hi]."""
    g = _gen(seed, STREAM_SIZES)
    mn = torch.randint(lo, hi + 1, (count, 2), generator=g)
    return [(int(a), int(b)) for a, b in mn.tolist()]


def algorithmic_flops(m: int, n: int, b: int, q: int, want_u: bool = True,
                      want_v: bool = True, max_steps: int | None = None) -> float:
    """Leading-order flop count of one randUTV factorization, summed per step.

    Counted per step (k = offset, bi = block width, rm = m-k, rn = n-k):
    sketch and power products (2+4q) rm rn bi; right update of T 4 m rn bi;
    of V 4 n rn bi; left update of T 4 rm (rn-bi) bi; of U 4 m rm bi; the two
    panel QRs 2 bi^2 (r - bi/3) + r bi^2 each; the fold of the small SVD
    2 bi^2 (k + rn - bi) + 2 bi^2 (m + n).  Steps that the method skips (no
    right transform when rn == bi, no left one when rm == bi) count nothing.
    ``max_steps`` counts only the first that many block steps.
    """
    p = min(m, n)
    k = 0
    tot = 0.0
    step = 0
    while k < p and (max_steps is None or step < max_steps):
        step += 1
        bi = min(b, p - k)
        rm, rn = m - k, n - k
        if rn > bi:
            tot += (2 + 4 * q) * rm * rn * bi
            tot += 4.0 * m * rn * bi
            if want_v:
                tot += 4.0 * n * rn * bi
            tot += 2.0 * bi * bi * (rn - bi / 3.0) + rn * bi * bi
        if rm > bi:
            tot += 4.0 * rm * (rn - bi) * bi
            if want_u:
                tot += 4.0 * m * rm * bi
            tot += 2.0 * bi * bi * (rm - bi / 3.0) + rm * bi * bi
        tot += 2.0 * bi * bi * (k + rn - bi)
        tot += 2.0 * bi * bi * ((m if want_u else 0) + (n if want_v else 0))
        k += bi
    return tot


def bytes_touched(m: int, n: int, b: int, q: int, elem: int = 8) -> float:
    """Minimum HBM bytes of one factorization: every pass reads or writes its
    operands once (per step: (2q+1) rm rn + 3 m rn + 3 n rn + 3 rm rn + 3 m rm)."""
    p = min(m, n)
    k = 0
    tot = 0.0
    while k < p:
        bi = min(b, p - k)
        rm, rn = m - k, n - k
        tot += (2 * q + 1) * rm * rn + 3.0 * m * rn + 3.0 * n * rn + 3.0 * rm * rn + 3.0 * m * rm
        k += bi
    return tot * elem


__all__ = [
    "gaussian", "haar_orthogonal", "spectrum", "prescribed", "matrix", "batch_sizes",
    "algorithmic_flops", "bytes_touched", "STREAM_Q1", "STREAM_Q2", "STREAM_GAUSS",
    "STREAM_B", "STREAM_SIZES",
]

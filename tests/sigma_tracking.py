"""Singular-value tracking of a reduced-precision randUTV against the FP64 oracle.

The diagonal entries of each b x b block of T are the singular values of
U_blk^T T22 V_blk, the trailing matrix T22 of that block step seen through
the sketched basis (§3.1).  They estimate the leading singular values of
T22, and T22 at block k has the singular values of the final T(k:, k:).

A sketch computed with unit roundoff u resolves a direction of T22 only when
its weight in Y = (T22^T T22)^q T22^T G, (s_j / s_0)^(2q+1) relative to the
block's leading direction, stands well above u: every product perturbs Y by
about u of its size.  Below that level the basis is set by the rounding and
the estimate is one of lower quality; the directions it misses stay in the
next trailing matrix, so a reduced-precision run and the FP64 run work on
different trailing matrices from the second block on.  The check therefore
compares each run with its own trailing matrix:

* gated indices: resolved by the reduced-precision sketch (weight >= 16 u)
  and estimated accurately by the FP64 method itself (relative error at most
  1e-3 against its own trailing singular values);
* there the reduced-precision estimate must be within `tol` of its own
  trailing singular value;
* in the first block, where both runs see the same T22 = A, the gated
  estimates must also match the oracle's directly, within `first_tol` plus
  (u / w_j)^2 (the sketched basis leans off direction j by an angle of
  about u / w_j, and the estimate moves by its square);
* no estimate may exceed the norm of its trailing matrix.
"""
import torch

f64 = torch.float64


def check(T, Tref, b, q, u, tol, first_tol):
    """Raises AssertionError on a violation; returns a dict of the measured figures."""
    T = T.to(f64)
    Tref = Tref.to(f64)
    m, n = T.shape
    p = min(m, n)
    worst, worst_first, gated, blocks = 0.0, 0.0, 0, 0
    for k in range(0, p, b):
        bi = min(b, p - k)
        s = torch.linalg.svdvals(T[k:, k:])[:bi]
        s0 = torch.linalg.svdvals(Tref[k:, k:])[:bi]
        d = torch.diagonal(T)[k:k + bi].abs()
        d0 = torch.diagonal(Tref)[k:k + bi].abs()
        if float(s[0]) == 0.0:
            continue
        assert bool((d <= s[0] * (1 + 1e-5)).all()), (k, float((d / s[0]).max()))
        tiny = s0 <= 1e-300
        e = (d - s).abs() / s.clamp_min(1e-300)
        e0 = (d0 - s0).abs() / s0.clamp_min(1e-300)
        w = (s / s[0]) ** (2 * q + 1)
        g = (w >= 16 * u) & (e0 <= 1e-3) & ~tiny
        blocks += 1
        if int(g.sum()) == 0:
            continue
        gated += int(g.sum())
        worst = max(worst, float(e[g].max()))
        assert float(e[g].max()) <= tol, (k, float(e[g].max()))
        if k == 0:
            # the sketched basis leans off direction j by an angle of about
            # u / w_j, which moves the estimate by its square
            r = ((d - d0).abs() / d0.clamp_min(1e-300))[g]
            lim = first_tol + (u / w[g]) ** 2
            worst_first = float((r / lim).max()) * first_tol
            assert bool((r <= lim).all()), float((r / lim).max())
    assert gated >= 1
    return {"worst": worst, "worst_first_block": worst_first, "gated": gated, "blocks": blocks}

"""Pins of the CPU oracle against things other than itself.

Each test checks one oracle function against brute force, a closed form, an
invariant the paper states, or a third-party implementation, chosen so that a
dropped term, a wrong sign or index or a transposed operand fails one of them.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import philox
from paper_2002_06960_gb300 import inputs

from thirdparty import aten_words

f64 = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ----

@pytest.mark.parametrize("seed,ctr", [
    (0, (0, 0, 0, 0)),
    (2 ** 64 - 1, (0xFFFFFFFF,) * 4),
    (123456789012345, (5, 9, 7, 3)),
    (0xDEADBEEF, (1 << 31, 17, 0, 4)),
])
def test_philox_words_match_aten(seed, ctr):
    mine = philox.philox4x32_10(np.array([ctr], dtype=np.uint64), philox.seed_key(seed))[0]
    assert np.array_equal(mine, aten_words(seed, ctr))


def test_philox_words_match_aten_random_counters():
    rng = np.random.default_rng(7)
    ctrs = rng.integers(0, 2 ** 32, size=(64, 4), dtype=np.uint64)
    seed = int(rng.integers(0, 2 ** 63))
    mine = philox.philox4x32_10(ctrs, philox.seed_key(seed))
    for i in range(ctrs.shape[0]):
        assert np.array_equal(mine[i], aten_words(seed, ctrs[i]))


def test_uniform_extremes():
    lo = np.zeros((1, 4), dtype=np.uint32)
    hi = np.full((1, 4), 0xFFFFFFFF, dtype=np.uint32)
    u1, u2 = philox.uniforms(lo)
    assert u1[0] == 2.0 ** -53 and u2[0] == 0.0
    u1, u2 = philox.uniforms(hi)
    assert u1[0] == 1.0 and u2[0] == 1.0 - 2.0 ** -53


# Hand-worked words for the Box-Muller assignment (the reading of the sketch
# generator: u1 from x0, x1 with the +1 offset, u2 from x2, x3; cos to the
# even element, sin to the odd one).  Each case is worked out by hand below.
def test_box_muller_hand_worked_words():
    w = np.array([[1 << 31, 0, 1 << 30, 0]], dtype=np.uint32)
    # j1 = (2^31 >> 5) 2^26 = 2^52 -> u1 = (2^52 + 1) 2^-53 = 1/2 + 2^-53
    # j2 = (2^30 >> 5) 2^26 = 2^51 -> u2 = 1/4, angle pi/2
    # rho = sqrt(-2 ln(1/2 + 2^-53)) = sqrt(2 ln 2) (1 - 2^-52 / (2 ln 2)) to first order
    even, odd = philox.box_muller(w)
    rho = math.sqrt(2.0 * math.log(2.0))
    assert abs(odd[0] - rho) <= 4e-16 * rho          # sin(pi/2) = 1: all of rho on the odd element
    assert abs(even[0]) < 1e-15                      # cos(pi/2) = 0
    # swapping the roles of the two uniforms would give u1 = 1/4, u2 = 1/2:
    # (-sqrt(2 ln 4), 0); swapping cos and sin would give (rho, 0)
    w = np.array([[0, 0, 0, 0]], dtype=np.uint32)
    # j1 = 0 -> u1 = 2^-53 (the +1 keeps ln finite); u2 = 0 -> (rho, 0), rho = sqrt(106 ln 2)
    even, odd = philox.box_muller(w)
    assert abs(even[0] - math.sqrt(106.0 * math.log(2.0))) <= 4e-16 * 8.6
    assert odd[0] == 0.0
    w = np.array([[0, 0xFFFFFFFF, 0, 0]], dtype=np.uint32)
    # j1 = 0xFFFFFFFF >> 6 = 2^26 - 1 -> u1 = 2^26 2^-53 = 2^-27; rho = sqrt(54 ln 2)
    even, odd = philox.box_muller(w)
    assert abs(even[0] - math.sqrt(54.0 * math.log(2.0))) <= 4e-16 * 6.2
    w = np.array([[0xFFFFFFFF, 0xFFFFFFFF, 1 << 31, 0]], dtype=np.uint32)
    # j1 = 2^53 - 1 -> u1 = 1, rho = 0; u2 = 1/2 -> both normals are (-)0
    even, odd = philox.box_muller(w)
    assert even[0] == 0.0 and odd[0] == 0.0


def test_box_muller_f32_hand_worked_words():
    # batched form: u1 = ((x0 >> 8) + 1) 2^-24, u2 = (x2 >> 8) 2^-24, x1 and x3 unused
    w = np.array([[0x7FFFFF00, 0xABCDEF12, 1 << 30, 0x12345678]], dtype=np.uint32)
    # x0 >> 8 = 2^23 - 1 -> u1 = 1/2; x2 >> 8 = 2^22 -> u2 = 1/4: (0, sqrt(2 ln 2))
    even, odd = philox.box_muller_f32(w)
    assert even.dtype == np.float32
    assert odd[0] == np.float32(math.sqrt(2.0 * math.log(2.0)))
    assert abs(float(even[0])) < 1e-15
    w = np.array([[0, 0, 0x80000000, 0]], dtype=np.uint32)
    # u1 = 2^-24 -> rho = sqrt(48 ln 2); u2 = 1/2 -> (-rho, 0)
    even, odd = philox.box_muller_f32(w)
    assert even[0] == np.float32(-math.sqrt(48.0 * math.log(2.0)))
    assert abs(float(odd[0])) < 1e-14
    u1, u2 = philox.uniforms_f32(np.array([[0xFFFFFFFF, 0, 0xFFFFFFFF, 0]], dtype=np.uint32))
    assert u1[0] == 1.0 and u2[0] == 1.0 - 2.0 ** -24


def test_box_muller_f32_distribution_and_layout():
    from scipy import stats
    x = philox.normal_pairs_f32(seed=5, step=1, matrix_id=3, stream=0, npairs=100_000)
    assert x.dtype == np.float32
    xd = x.astype(np.float64)
    n = xd.size
    assert abs(xd.mean()) < 5.0 / math.sqrt(n)
    assert abs(xd.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert stats.kstest(xd, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(xd[0::2], xd[1::2])[0, 1]) < 5.0 / math.sqrt(n / 2)
    G = philox.sketch_f32(5, 1, 9, 4, matrix_id=3)
    flat = philox.normal_pairs_f32(5, 1, 3, 0, 18)
    assert np.array_equal(G, flat.reshape(4, 9).T)
    # the same words as the FP64 generator: the two sketches agree to the
    # 24-bit uniforms' resolution (the normals differ by about 2^-24 |ln u1|^-1/2)
    G64 = philox.sketch(5, 1, 9, 4, matrix_id=3)
    assert np.allclose(G, G64, rtol=0, atol=2e-3)


def test_box_muller_distribution():
    from scipy import stats
    x = philox.normal_pairs(seed=11, step=3, matrix_id=0, stream=0, npairs=100_000)
    n = x.size
    assert abs(x.mean()) < 5.0 / math.sqrt(n)
    assert abs(x.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert stats.kstest(x, "norm").pvalue > 1e-3
    # the two normals of one counter are uncorrelated
    assert abs(np.corrcoef(x[0::2], x[1::2])[0, 1]) < 5.0 / math.sqrt(n / 2)
    # fourth moment of N(0,1) is 3
    assert abs((x ** 4).mean() - 3.0) < 0.1


def test_sketch_layout_column_major_pairs():
    rows, cols = 7, 5          # odd element count: last pair yields one normal
    G = philox.sketch(3, 2, rows, cols, matrix_id=4)
    flat = philox.normal_pairs(3, 2, 4, 0, (rows * cols + 1) // 2)
    for c in range(cols):
        for r in range(rows):
            assert G[r, c] == flat[r + c * rows]
    # different step / matrix id / stream give different draws
    assert not np.allclose(G, philox.sketch(3, 3, rows, cols, matrix_id=4))
    assert not np.allclose(G, philox.sketch(3, 2, rows, cols, matrix_id=5))


# ------------------------------------------------------------ Householder ----

def _explicit_H(v, tau):
    r = v.numel()
    return torch.eye(r, dtype=f64) - tau * torch.outer(v, v)


def test_reflector_maps_to_e1():
    g = torch.Generator().manual_seed(1)
    for r in [1, 2, 5, 33]:
        x = torch.randn(r, generator=g, dtype=f64)
        v, tau, beta = oracle.householder_reflector(x)
        H = _explicit_H(v, tau)
        y = H @ x
        e = torch.zeros(r, dtype=f64)
        e[0] = float(beta)
        assert torch.allclose(y, e, atol=1e-14 * float(x.norm()))
        assert torch.allclose(H @ H.T, torch.eye(r, dtype=f64), atol=1e-15 * 8)
        assert abs(abs(float(beta)) - float(x.norm())) < 1e-14 * float(x.norm())
        if r > 1:
            assert 1.0 <= float(tau) <= 2.0
            assert float(beta) * float(x[0]) <= 0.0   # beta has the sign opposite to alpha


def test_reflector_special_cases():
    # x2 == 0: tau = 0 and H = I, even for negative alpha
    v, tau, beta = oracle.householder_reflector(torch.tensor([-3.0, 0.0, 0.0], dtype=f64))
    assert float(tau) == 0.0 and float(beta) == -3.0
    v, tau, beta = oracle.householder_reflector(torch.tensor([2.5], dtype=f64))
    assert float(tau) == 0.0 and float(beta) == 2.5
    # alpha == 0: sgn(0) = +1, beta = -||x||
    v, tau, beta = oracle.householder_reflector(torch.tensor([0.0, 3.0, 4.0], dtype=f64))
    assert float(beta) == -5.0 and float(tau) == 1.0


@pytest.mark.parametrize("r,c", [(50, 8), (9, 9), (64, 1), (13, 4)])
def test_householder_qr_against_explicit_reflectors(r, c):
    g = torch.Generator().manual_seed(r * 100 + c)
    Y = torch.randn(r, c, generator=g, dtype=f64)
    W, tau, R = oracle.householder_qr(Y)
    Q = torch.eye(r, dtype=f64)
    for j in range(c):
        assert float(W[j, j]) == 1.0 and float(W[:j, j].abs().max() if j else 0.0) == 0.0
        Q = Q @ _explicit_H(W[:, j], tau[j])
    assert torch.allclose(Q[:, :c] @ R, Y, atol=1e-14 * float(Y.norm()))
    assert torch.allclose(Q.T @ Q, torch.eye(r, dtype=f64), atol=1e-14)
    assert torch.equal(R, torch.triu(R))
    # third-party QR: |R_jj| is unique
    Rn = np.linalg.qr(Y.numpy(), mode="r")
    assert np.allclose(np.abs(np.diag(Rn)), np.abs(torch.diagonal(R).numpy()), rtol=1e-13)


def test_wy_factor_equals_product_of_reflectors():
    g = torch.Generator().manual_seed(5)
    for (r, c) in [(40, 6), (6, 6), (17, 1), (30, 12)]:
        Y = torch.randn(r, c, generator=g, dtype=f64)
        W, tau, _ = oracle.householder_qr(Y)
        S = oracle.wy_factor(W, tau)
        Q = torch.eye(r, dtype=f64)
        for j in range(c):
            Q = Q @ _explicit_H(W[:, j], tau[j])
        assert torch.equal(S, torch.triu(S))
        assert torch.allclose(torch.eye(r, dtype=f64) - W @ S @ W.T, Q, atol=1e-14)


def test_wy_factor_with_zero_tau():
    # a column already in R form gives tau = 0 and must drop out of S
    Y = torch.tensor([[1.0, 2.0], [0.0, 3.0], [0.0, 4.0]], dtype=f64)
    W, tau, _ = oracle.householder_qr(Y)
    assert float(tau[0]) == 0.0
    S = oracle.wy_factor(W, tau)
    Q = _explicit_H(W[:, 0], tau[0]) @ _explicit_H(W[:, 1], tau[1])
    assert torch.allclose(torch.eye(3, dtype=f64) - W @ S @ W.T, Q, atol=1e-15)


# ------------------------------------------------------------- small SVD ----

def _check_svd(B, Us, D, Vs, tol=1e-14):
    b = B.shape[0]
    assert torch.allclose(Us @ torch.diag(D) @ Vs.T, B, atol=tol * max(1.0, float(B.norm())))
    assert torch.allclose(Us.T @ Us, torch.eye(b, dtype=f64), atol=tol * 10)
    assert torch.allclose(Vs.T @ Vs, torch.eye(b, dtype=f64), atol=tol * 10)
    assert bool((D[:-1] >= D[1:]).all()) and bool((D >= 0).all())
    for j in range(b):                      # sign rule
        col = Vs[:, j]
        idx = int(torch.nonzero(col.abs() == col.abs().max())[0, 0])
        assert float(col[idx]) > 0


@pytest.mark.parametrize("zero_tau", [False, True])
def test_wy_factor_adjoint_closed_form(zero_tau):
    """The reverse of the WY factor that the backward form runs as b x b products: with
    N = striu(W^T W), D = diag(tau), M = (I + D N)^-1 (so that S = M D), Mb = triu(Sb) D and
    Kb = -M^T Mb M^T, the adjoints are Gb = striu(D Kb), Wb = W (Gb + Gb^T) and
    tau_b = diag(M^T triu(Sb)) + rowsum(striu(Kb) * N).  Checked against autograd through the
    oracle's column recurrence, also with identity reflectors (tau = 0)."""
    g = torch.Generator().manual_seed(11)
    r, c = 40, 12
    W = torch.randn(r, c, generator=g, dtype=torch.float64)
    tau = torch.rand(c, generator=g, dtype=torch.float64) + 0.5
    if zero_tau:
        tau[3] = 0.0
        tau[8] = 0.0
    Sb = torch.triu(torch.randn(c, c, generator=g, dtype=torch.float64))
    Wv = W.clone().requires_grad_(True)
    tv = tau.clone().requires_grad_(True)
    (oracle.wy_factor(Wv, tv) * Sb).sum().backward()
    N = torch.triu(W.T @ W, 1)
    D = torch.diag(tau)
    M = torch.linalg.inv(torch.eye(c, dtype=torch.float64) + D @ N)
    assert torch.allclose(M @ D, oracle.wy_factor(W, tau), atol=1e-13)
    Kb = -M.T @ (Sb @ D) @ M.T
    Gb = torch.triu(D @ Kb, 1)
    Wb = W @ (Gb + Gb.T)
    taub = torch.diag(M.T @ Sb) + (torch.triu(Kb, 1) * N).sum(1)
    scale = float(Wv.grad.abs().max())
    assert float((Wb - Wv.grad).abs().max()) <= 1e-12 * scale
    assert float((taub - tv.grad).abs().max()) <= 1e-12 * max(1.0, float(tv.grad.abs().max()))


def test_small_svd_diagonal_closed_form():
    B = torch.diag(torch.tensor([3.0, -1.0, 2.0, 0.5], dtype=f64))
    Us, D, Vs = oracle.small_svd(B)
    assert torch.allclose(D, torch.tensor([3.0, 2.0, 1.0, 0.5], dtype=f64), rtol=0, atol=1e-15)
    _check_svd(B, Us, D, Vs)
    # V is a signed permutation with positive entries; U carries the sign of -1
    assert torch.allclose(Vs.abs().sum(0), torch.ones(4, dtype=f64))
    assert float(Vs.min()) >= 0
    assert float(Us[1, 2]) == -1.0


def test_small_svd_rank_one_closed_form():
    x = torch.tensor([1.0, -2.0, 2.0], dtype=f64)
    y = torch.tensor([0.0, 3.0, -4.0], dtype=f64)
    B = torch.outer(x, y)
    Us, D, Vs = oracle.small_svd(B)
    assert abs(float(D[0]) - 15.0) < 1e-13
    assert float(D[1:].abs().max()) < 1e-13
    # largest entry of y/|y| is -4/5 -> the sign rule makes V[:,0] = -y/|y|
    assert torch.allclose(Vs[:, 0], -y / 5.0, atol=1e-15)
    assert torch.allclose(Us[:, 0], -x / 3.0, atol=1e-15)


def test_small_svd_2x2_closed_form():
    a, b_, d = 4.0, 3.0, -2.0
    B = torch.tensor([[a, b_], [0.0, d]], dtype=f64)
    Ssum = a * a + b_ * b_ + d * d
    det = abs(a * d)
    s1 = math.sqrt((Ssum + math.sqrt(Ssum * Ssum - 4 * det * det)) / 2)
    s2 = det / s1
    Us, D, Vs = oracle.small_svd(B)
    assert abs(float(D[0]) - s1) < 1e-14 * s1 and abs(float(D[1]) - s2) < 1e-14 * s1
    _check_svd(B, Us, D, Vs)


def test_small_svd_random_and_orthogonal():
    g = torch.Generator().manual_seed(9)
    B = torch.randn(24, 24, generator=g, dtype=f64)
    _check_svd(B, *oracle.small_svd(B))
    Q, _ = torch.linalg.qr(torch.randn(10, 10, generator=g, dtype=f64))
    Us, D, Vs = oracle.small_svd(Q)
    assert torch.allclose(D, torch.ones(10, dtype=f64), atol=1e-14)


# ------------------------------------------------------- whole randUTV ----

SHAPES = [(64, 64, 16, 1), (80, 48, 16, 2), (48, 80, 16, 0), (70, 70, 24, 1), (33, 21, 7, 1),
          (21, 33, 5, 2), (40, 40, 1, 1), (30, 30, 64, 1)]


@pytest.mark.parametrize("m,n,b,q", SHAPES)
def test_randutv_invariants(m, n, b, q):
    A = inputs.gaussian(m, n, seed=m * 7 + n)
    f = oracle.randutv(A, b, q, seed=1)
    assert oracle.recon_error(A, f.U, f.T, f.V) < 1e-13
    assert oracle.orth_error(f.U) < 1e-13 and oracle.orth_error(f.V) < 1e-13
    # exact zeros: strictly lower part, and off-diagonal inside every diagonal block
    assert float(torch.tril(f.T, -1).abs().max()) == 0.0
    for (i, k, bi, rm, rn, right, left) in oracle.block_schedule(m, n, b):
        blk = f.T[k:k + bi, k:k + bi]
        assert torch.equal(blk, torch.diag(torch.diagonal(blk)))
        assert bool((torch.diagonal(blk) >= 0).all())
    # orthogonal invariance of the Frobenius norm
    assert abs(float(f.T.norm() - A.norm())) < 1e-13 * float(A.norm())
    # interlacing and tail bounds at every block boundary
    sA = torch.linalg.svdvals(A)
    for (i, k, bi, rm, rn, right, left) in oracle.block_schedule(m, n, b):
        if k == 0:
            continue
        sT = torch.linalg.svdvals(f.T[:k, :k])
        assert bool((sT <= sA[:k] * (1 + 1e-12) + 1e-13).all())
        tail = f.T[k:, k:]
        assert float(torch.linalg.matrix_norm(tail, 2)) >= float(sA[k]) * (1 - 1e-12)
        assert float(tail.norm()) >= float(sA[k:].norm()) * (1 - 1e-12)


def test_randutv_single_block_is_svd():
    """b >= min(m,n): one step and T = diag(sigma(A)), the prescribed spectrum."""
    for (m, n) in [(40, 40), (50, 30), (30, 50)]:
        p = min(m, n)
        sig = torch.exp(-torch.arange(p, dtype=f64) / 7.0)
        A = inputs.prescribed(m, n, sig, seed=3)
        f = oracle.randutv(A, 64, 1, seed=0)
        d = torch.diagonal(f.T)
        assert torch.allclose(d, sig, rtol=1e-12, atol=1e-14)
        off = f.T.clone()
        off[range(p), range(p)] = 0
        assert float(off.abs().max()) < 1e-12


@pytest.mark.parametrize("q", [0, 1, 2])
def test_randutv_low_rank_first_block_captures_all(q):
    """rank r <= b: after step 0 the trailing block is zero and D_0 = sigma."""
    m, n, b, r = 72, 60, 12, 9
    sig = torch.zeros(min(m, n), dtype=f64)
    sig[:r] = torch.tensor([5.0, 4, 3, 2.5, 2, 1.5, 1, 0.7, 0.4], dtype=f64)
    A = inputs.prescribed(m, n, sig, seed=4)
    f = oracle.randutv(A, b, q, seed=2, max_steps=1)
    assert float(f.T[b:, b:].norm()) < 1e-14 * float(A.norm()) * 10
    assert torch.allclose(torch.diagonal(f.T)[:r], sig[:r], rtol=1e-12)


def _literal_section_31(A, b, q, seed):
    """§3.1 as written: dense U^(i), V^(i) per step and T^(i) = U^(i)^T T^(i-1) V^(i)."""
    m, n = A.shape
    T = A.clone()
    U = torch.eye(m, dtype=f64)
    V = torch.eye(n, dtype=f64)
    for (i, k, bi, rm, rn, right, left) in oracle.block_schedule(m, n, b):
        Vhat = torch.eye(rn, dtype=f64)
        if right:
            G = oracle.sketch(seed, i, rm, bi)
            Y = oracle.range_basis(T[k:, k:], G, q)
            W, tau, _ = oracle.householder_qr(Y)
            for j in range(bi):
                Vhat = Vhat @ _explicit_H(W[:, j], tau[j])
        Uhat = torch.eye(rm, dtype=f64)
        B = T[k:, k:] @ Vhat
        if left:
            W, tau, _ = oracle.householder_qr(B[:, :bi])
            for j in range(bi):
                Uhat = Uhat @ _explicit_H(W[:, j], tau[j])
        C = (Uhat.T @ B)[:bi, :bi]
        Us, D, Vs = oracle.small_svd(C)
        Vi = torch.eye(n, dtype=f64)
        Vi[k:, k:] = Vhat
        Vsv = torch.eye(n, dtype=f64)
        Vsv[k:k + bi, k:k + bi] = Vs
        Vi = Vi @ Vsv
        Ui = torch.eye(m, dtype=f64)
        Ui[k:, k:] = Uhat
        Usv = torch.eye(m, dtype=f64)
        Usv[k:k + bi, k:k + bi] = Us
        Ui = Ui @ Usv
        T = Ui.T @ T @ Vi
        U = U @ Ui
        V = V @ Vi
    return U, T, V


@pytest.mark.parametrize("m,n,b,q", [(12, 12, 3, 1), (16, 10, 4, 0), (10, 16, 4, 2), (9, 7, 2, 1),
                                     (8, 8, 1, 1), (11, 13, 4, 1)])
def test_randutv_matches_literal_dense_products(m, n, b, q):
    A = inputs.gaussian(m, n, seed=100 + m + n)
    f = oracle.randutv(A, b, q, seed=6)
    U, T, V = _literal_section_31(A, b, q, seed=6)
    # same up to rounding; separated singular values make U and V unique
    assert torch.allclose(f.T.triu(), T.triu(), atol=1e-13 * float(A.norm()))
    assert torch.allclose(f.U, U, atol=1e-12)
    assert torch.allclose(f.V, V, atol=1e-12)


def test_resume_is_bitwise():
    A = inputs.gaussian(50, 46, seed=8)
    full = oracle.randutv(A, 8, 1, seed=5)
    part = oracle.randutv(A, 8, 1, seed=5, max_steps=3)
    rest = oracle.randutv(A, 8, 1, seed=5, state=part)
    assert torch.equal(full.T, rest.T) and torch.equal(full.U, rest.U) and torch.equal(full.V, rest.V)


def test_t_only_matches_with_factors():
    A = inputs.gaussian(40, 36, seed=12)
    a = oracle.randutv(A, 8, 1, seed=5)
    b = oracle.randutv(A, 8, 1, seed=5, want_u=False, want_v=False)
    assert torch.equal(a.T, b.T) and b.U is None and b.V is None


def test_step_spectrum_is_revealed():
    """q >= 1 on a gapped spectrum: |T_kk| tracks sigma_k away from the gap's block."""
    n, b, gap = 192, 16, 40
    sig = inputs.spectrum("step", n, gap)
    A = inputs.prescribed(n, n, sig, seed=2)
    f = oracle.randutv(A, b, 1, seed=0)
    d = torch.diagonal(f.T)
    straddle = range((gap // b) * b, (gap // b + 1) * b)
    for k in range(n):
        if k in straddle:
            continue
        assert abs(float(d[k]) / float(sig[k]) - 1.0) < 1e-3, k


def test_fig3_schedule_golden():
    rows = []
    with open(os.path.join(GOLDEN, "fig3_task_order.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(tuple(int(t) for t in line.split()))
    n = 64
    sched = oracle.block_schedule(n, n, n // 2)
    got = [(i, int(right), int(left), 1) for (i, k, bi, rm, rn, right, left) in sched]
    assert got == rows


# ------------------------------------------------------------ low rank ----

def test_lowrank_is_paper_definition():
    m, n, b, k = 60, 50, 8, 16
    A = inputs.gaussian(m, n, seed=21)
    full = oracle.randutv(A, b, 1, seed=3)
    Ak_def = full.U[:, :k] @ full.T[:k, :] @ full.V.T          # §1.1 definition
    assert torch.allclose(oracle.lowrank(A, k, b, 1, seed=3), Ak_def, atol=1e-13)


def test_lowrank_of_rank_k_matrix_is_itself():
    m, n, b, k = 40, 36, 8, 16
    sig = torch.zeros(36, dtype=f64)
    sig[:k] = torch.linspace(3, 1, k, dtype=f64)
    A = inputs.prescribed(m, n, sig, seed=5)
    assert torch.allclose(oracle.lowrank(A, k, b, 1, seed=1), A, atol=1e-13)


# ------------------------------------------------------------- flops ----

def test_flop_count_leading_order():
    for q in [0, 1, 2]:
        n = 16384
        f = inputs.algorithmic_flops(n, n, 128, q)
        assert abs(f / ((8 + 4 * q / 3) * n ** 3) - 1) < 0.03
        f = inputs.algorithmic_flops(n, n, 128, q, want_u=False, want_v=False)
        assert abs(f / ((4 + 4 * q / 3) * n ** 3) - 1) < 0.03


# ----------------------------------------------- sketch and power iteration ----

def _known_svd(m, n, seed):
    p = min(m, n)
    sig = torch.exp(-torch.arange(p, dtype=f64) / 6.0)
    Q1 = inputs.haar_orthogonal(m, seed, inputs.STREAM_Q1, p)
    Q2 = inputs.haar_orthogonal(n, seed, inputs.STREAM_Q2, p)
    return Q1, sig, Q2, (Q1 * sig) @ Q2.T


@pytest.mark.parametrize("q", [0, 1, 2])
def test_range_basis_closed_form(q):
    """Y = (A^T A)^q A^T G = Q2 diag(sigma^(2q+1)) Q1^T G for A = Q1 diag(sigma) Q2^T."""
    Q1, sig, Q2, A = _known_svd(30, 24, seed=7)
    G = oracle.sketch(4, 0, 30, 5)
    Y = oracle.range_basis(A, G, q)
    Yref = (Q2 * sig ** (2 * q + 1)) @ (Q1.T @ G)
    assert torch.allclose(Y, Yref, atol=1e-14 * float(Yref.abs().max()) * 10)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_first_block_of_v_spans_the_sketched_range(q):
    """After step 0, V(:, 0:b) spans Y_0 = Q2 diag(sigma^(2q+1)) Q1^T G_0 (§3.1)."""
    m, n, b = 40, 32, 6
    Q1, sig, Q2, A = _known_svd(m, n, seed=9)
    f = oracle.randutv(A, b, q, seed=13, max_steps=1)
    G0 = oracle.sketch(13, 0, m, b)
    Yref = (Q2 * sig ** (2 * q + 1)) @ (Q1.T @ G0)
    Vb = f.V[:, :b]
    resid = Yref - Vb @ (Vb.T @ Yref)
    assert float(resid.norm()) < 1e-12 * float(Yref.norm())
    # and the sketch of the other q values is not in that span
    for q2 in {0, 1, 2} - {q}:
        Y2 = (Q2 * sig ** (2 * q2 + 1)) @ (Q1.T @ G0)
        assert float((Y2 - Vb @ (Vb.T @ Y2)).norm()) > 1e-6 * float(Y2.norm())


# ------------------------------------------------- gradient of the low-rank map

def _loss(A, B, k, b, q, seed):
    Ak = oracle.lowrank(A, k, b, q, seed)
    return ((Ak - B) ** 2).sum()


def _grad(A, B, k, b, q, seed):
    X = A.clone().requires_grad_(True)
    L = _loss(X, B, k, b, q, seed)
    (g,) = torch.autograd.grad(L, X)
    return g


@pytest.mark.parametrize("m,n,b,k,q", [(40, 36, 8, 16, 1), (30, 44, 6, 12, 2), (24, 24, 8, 8, 0)])
def test_lowrank_gradient_central_differences(m, n, b, k, q):
    """Autograd through the oracle matches FP64 central differences."""
    A = inputs.matrix("exp16", m, n, seed=3)
    B = inputs.gaussian(m, n, seed=4, stream=inputs.STREAM_B)
    g = _grad(A, B, k, b, q, 7)
    gen = torch.Generator().manual_seed(11)
    h = 1e-6 * float(A.norm())
    for _ in range(3):
        E = torch.randn(m, n, generator=gen, dtype=f64)
        E /= E.norm()
        fd = (float(_loss(A + h * E, B, k, b, q, 7)) - float(_loss(A - h * E, B, k, b, q, 7))) / (2 * h)
        an = float((g * E).sum())
        assert abs(an - fd) <= 1e-6 * max(1.0, abs(fd)), (an, fd)


def test_lowrank_gradient_128_step_spectrum():
    """The 128 x 128 check instance: b = 16, k = 32, q = 1, step spectrum with the gap at 32."""
    n, b, k, q = 128, 16, 32, 1
    A = inputs.matrix("step", n, n, seed=3, gap=k)
    B = inputs.gaussian(n, n, seed=3, stream=inputs.STREAM_B)
    g = _grad(A, B, k, b, q, 0)
    gen = torch.Generator().manual_seed(5)
    h = 1e-6 * float(A.norm())
    for _ in range(3):
        E = torch.randn(n, n, generator=gen, dtype=f64)
        E /= E.norm()
        fd = (float(_loss(A + h * E, B, k, b, q, 0)) - float(_loss(A - h * E, B, k, b, q, 0))) / (2 * h)
        an = float((g * E).sum())
        assert abs(an - fd) <= 1e-6 * max(1.0, abs(fd)), (an, fd)


def test_lowrank_without_svd_is_unchanged():
    A = inputs.gaussian(50, 40, seed=2)
    full = oracle.randutv(A, 8, 1, seed=3, max_steps=2)
    nosvd = oracle.randutv(A, 8, 1, seed=3, max_steps=2, svd=False)
    P1 = full.U[:, :16] @ full.U[:, :16].T
    P2 = nosvd.U[:, :16] @ nosvd.U[:, :16].T
    assert torch.allclose(P1, P2, atol=1e-13)
    # the trailing matrix after the steps is the same too
    assert torch.allclose(full.T[16:, 16:], nosvd.T[16:, 16:], atol=1e-13)

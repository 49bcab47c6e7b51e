"""GPU path against the CPU oracle, element by element, through the C-ABI.

Tolerance: relative Frobenius error <= 1e-12 on U, T and V (the FP64 parity
bar), 1e-13 on the single kernels; bit-exact on Philox words.  Sizes span
several tiles and a ragged tail; the full-size case runs the bench launch
configuration (16384^2, b = 128, q = 1) for its first step.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import philox
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
    y = y.to(f64)
    d = float(torch.linalg.norm(y))
    return float(torch.linalg.norm(x.to(f64) - y)) / (d if d > 0 else 1.0)


def cpu(t):
    return t.detach().to("cpu").contiguous()


# ------------------------------------------------------------ sketch ----

@pytest.mark.parametrize("seed,c", [(0, (0, 0, 0, 0)), (2 ** 64 - 1, (0xFFFFFFF0, 5, 6, 7)),
                                    (123456789, (1000, 3, 1, 0))])
def test_philox_words_bit_exact(pkg, seed, c):
    count = 4099
    got = cpu(pkg.randutv_philox_words(seed, *c, count)).numpy().view(np.uint32)
    ctr = np.zeros((count, 4), dtype=np.uint64)
    ctr[:, 0] = (np.arange(count, dtype=np.uint64) + np.uint64(c[0])) & np.uint64(0xFFFFFFFF)
    ctr[:, 1], ctr[:, 2], ctr[:, 3] = c[1], c[2], c[3]
    want = philox.philox4x32_10(ctr, philox.seed_key(seed))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("rows,cols,step,mid", [(1000, 64, 0, 0), (777, 13, 5, 3), (1, 1, 2, 0),
                                                (3, 5, 9, 1)])
def test_philox_normal_matches_oracle(pkg, rows, cols, step, mid):
    G = cpu(pkg.randutv_philox_normal(42, step, mid, 0, rows, cols))
    ref = torch.from_numpy(philox.sketch(42, step, rows, cols, mid))
    # same words; log / sincospi vs libm differ by a few ulp
    assert float((G - ref).abs().max()) <= 1e-14 * max(1.0, float(ref.abs().max()))


@pytest.mark.parametrize("rows,cols,step,mid", [(1000, 64, 0, 0), (777, 13, 5, 3), (1, 1, 2, 0),
                                                (1023, 64, 15, 4095)])
def test_philox_normal_f32_matches_oracle(pkg, rows, cols, step, mid):
    """The batched form's FP32 sketch against the oracle's: the same words, and
    Box-Muller of the same exact FP32 uniforms; logf / sqrtf / sincospif / the
    product each round in FP32, so the two agree to a few FP32 ulp."""
    G = cpu(pkg.randutv_philox_normal_f32(7, step, mid, 0, rows, cols)).double()
    ref = torch.from_numpy(philox.sketch_f32(7, step, rows, cols, mid)).double()
    assert torch.isfinite(G).all()
    tol = 8 * 2.0 ** -24 * ref.abs() + 1e-30
    assert bool(((G - ref).abs() <= tol).all()), float(((G - ref).abs() / ref.abs()).max())


# -------------------------------------------------------------- dgemm ----

@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
@pytest.mark.parametrize("M,N,K", [(130, 67, 45), (64, 64, 4000), (5, 300, 1), (257, 128, 9000),
                                   (1, 1, 1), (100, 3, 0)])
def test_dgemm_matches_fp64_matmul(pkg, ta, tb, M, N, K):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn((K, M) if ta == "T" else (M, K), generator=g, dtype=f64)
    B = torch.randn((N, K) if tb == "T" else (K, N), generator=g, dtype=f64)
    C = torch.randn(M, N, generator=g, dtype=f64)
    ref = 0.75 * ((A.T if ta == "T" else A) @ (B.T if tb == "T" else B)) - 0.5 * C
    Cd = pkg.to_colmajor(C, "cuda")
    pkg.randutv_dgemm(ta, tb, 0.75, pkg.to_colmajor(A, "cuda"), pkg.to_colmajor(B, "cuda"), -0.5, Cd)
    torch.cuda.synchronize()
    amax = float(A.abs().max()) if A.numel() else 0.0
    bmax = float(B.abs().max()) if B.numel() else 0.0
    scale = amax * bmax * max(K, 1) + float(C.abs().max())
    assert float((cpu(Cd) - ref).abs().max()) <= 1e-15 * scale * 8


# -------------------------------------------------- Householder and WY ----

@pytest.mark.parametrize("r,c", [(1000, 37), (64, 64), (20000, 128), (7, 1), (300, 256), (129, 5)])
def test_householder_qr_matches_oracle(pkg, r, c):
    Y = inputs.gaussian(r, c, seed=r + c)
    panel = pkg.to_colmajor(Y, "cuda")
    W, tau = pkg.randutv_householder_qr(panel)
    torch.cuda.synchronize()
    W0, tau0, R0 = oracle.householder_qr(Y)
    P = cpu(panel)
    assert rel(cpu(W), W0) < 1e-13
    assert rel(cpu(tau), tau0) < 1e-13
    assert rel(P[:c], R0) < 1e-13
    assert float(P[c:].abs().max() if r > c else 0.0) == 0.0
    assert torch.equal(torch.tril(P[:c], -1), torch.zeros(c, c, dtype=f64))
    S = pkg.randutv_wy_factor(W, tau)
    torch.cuda.synchronize()
    assert rel(cpu(S), oracle.wy_factor(W0, tau0)) < 1e-13


def test_householder_qr_zero_columns(pkg):
    """Columns already in R form (s == 0) give tau = 0, even for negative alpha."""
    Y = torch.zeros(50, 4, dtype=f64)
    Y[0, 0] = -2.0
    Y[:, 1] = 1.0
    Y[0, 2] = 3.0
    W, tau = pkg.randutv_householder_qr(pkg.to_colmajor(Y, "cuda"))
    torch.cuda.synchronize()
    W0, tau0, _ = oracle.householder_qr(Y)
    assert float(cpu(tau)[0]) == 0.0 and float(tau0[0]) == 0.0
    assert rel(cpu(W), W0) < 1e-14 and rel(cpu(tau), tau0) < 1e-14


# ------------------------------------------------------------ small SVD ----

def _separated_block(b, seed, triangular=False):
    sig = torch.exp(-torch.arange(b, dtype=f64) / max(b / 8.0, 1.0))
    B = inputs.prescribed(b, b, sig, seed=seed)
    if triangular:
        B = torch.linalg.qr(B, mode="r")[1]
    return B


@pytest.mark.parametrize("b", [1, 2, 3, 7, 64, 100, 128, 256])
def test_small_svd_matches_oracle(pkg, b):
    for tri in (False, True):
        B = _separated_block(b, seed=b, triangular=tri)
        Us, D, Vs = pkg.randutv_small_svd(pkg.to_colmajor(B, "cuda"))
        torch.cuda.synchronize()
        U0, D0, V0 = oracle.small_svd(B)
        assert rel(cpu(D), D0) < 1e-13
        assert rel(cpu(Us), U0) < 1e-12
        assert rel(cpu(Vs), V0) < 1e-12


def test_small_svd_zero_block_is_orthogonal(pkg):
    b = 16
    B = torch.zeros(b, b, dtype=f64)
    B[3, 5] = 2.0   # rank one
    Us, D, Vs = pkg.randutv_small_svd(pkg.to_colmajor(B, "cuda"))
    torch.cuda.synchronize()
    Us, D, Vs = cpu(Us), cpu(D), cpu(Vs)
    assert float(D[0]) == 2.0 and float(D[1:].abs().max()) == 0.0
    assert oracle.orth_error(Us) < 1e-15 and oracle.orth_error(Vs) < 1e-15
    assert rel(Us @ torch.diag(D) @ Vs.T, B) < 1e-15


# ------------------------------------------------------- whole randUTV ----

def _factor(pkg, A, b, q, seed, want_u=True, want_v=True):
    U, T, V = pkg.randutv_factor(pkg.to_colmajor(A, "cuda"), b, q, seed, want_u, want_v)
    torch.cuda.synchronize()
    return (cpu(U) if U is not None else None), cpu(T), (cpu(V) if V is not None else None)


def _blockwise_sensitivity(A, b, q, seed, which):
    """Per block column, how far U or V moves when A moves at rounding level.

    The factorization of a matrix with a fast-decaying spectrum determines
    the trailing blocks of U and V only to about eps ||A|| / gap; this
    measures that floor with the oracle itself (two perturbations of size
    1e-16 max|A|), so a parity gate can sit on it instead of below it."""
    base = oracle.randutv(A, b, q, seed)
    out = None
    for s in (5, 6):
        g = torch.Generator().manual_seed(s)
        Ap = A + torch.randn(A.shape, generator=g, dtype=f64) * 1e-16 * float(A.abs().max())
        f = oracle.randutv(Ap, b, q, seed)
        X, X0 = getattr(f, which), getattr(base, which)
        d = torch.tensor([float((X[:, k:k + b] - X0[:, k:k + b]).norm())
                          for k in range(0, X.shape[1], b)])
        out = d if out is None else torch.maximum(out, d)
    return base, out


def test_parity_512_exp40(pkg):
    """The 512 x 512, b = 64, q = 1 workload (sigma_j = exp(-j/40)).

    T matches at 1e-12.  U and V match at 1e-12 in every block column whose
    conditioning allows it, and elsewhere within 100x the oracle's own
    movement under a rounding-level perturbation of A."""
    m = n = 512
    b, q, seed = 64, 1, 0
    A = inputs.matrix("exp40", m, n, seed=1)
    U, T, V = _factor(pkg, A, b, q, seed)
    ref, sensU = _blockwise_sensitivity(A, b, q, seed, "U")
    _, sensV = _blockwise_sensitivity(A, b, q, seed, "V")
    assert rel(T, ref.T) < 1e-12
    for X, X0, sens in ((U, ref.U, sensU), (V, ref.V, sensV)):
        for j, k in enumerate(range(0, n, b)):
            d = float((X[:, k:k + b] - X0[:, k:k + b]).norm())
            allowed = max(1e-12 * float(X0[:, k:k + b].norm()), 100.0 * float(sens[j]))
            assert d <= allowed, (j, d, allowed)
        # the leading blocks, well conditioned, at the plain 1e-12 bar
        assert rel(X[:, :2 * b], X0[:, :2 * b]) < 1e-12
    assert oracle.recon_error(A, U, T, V) < 1e-13
    assert oracle.orth_error(U) < 1e-13 and oracle.orth_error(V) < 1e-13


@pytest.mark.parametrize("m,n,b,q", [(512, 512, 64, 1), (300, 200, 48, 1), (200, 300, 48, 2),
                                     (257, 257, 64, 0), (130, 130, 1, 1), (90, 70, 128, 1),
                                     (640, 384, 128, 1), (384, 640, 128, 2), (2, 3, 1, 0)])
def test_parity_shapes(pkg, m, n, b, q):
    """Well-separated spectrum (sigma_j = 1 - j/2p): U, T, V at 1e-12, or at
    10x the factorization's own measured sensitivity where that floor is
    above 1e-13 (the oracle moves by that much when A moves at rounding level)."""
    A = inputs.matrix("linear", m, n, seed=m + n)
    U, T, V = _factor(pkg, A, b, q, 7)
    ref = oracle.randutv(A, b, q, 7)
    sens = {"U": 0.0, "T": 0.0, "V": 0.0}
    for s in (5, 6):
        g = torch.Generator().manual_seed(s)
        Ap = A + torch.randn(A.shape, generator=g, dtype=f64) * 1e-16 * float(A.abs().max())
        f = oracle.randutv(Ap, b, q, 7)
        for k in sens:
            sens[k] = max(sens[k], rel(getattr(f, k), getattr(ref, k)))
    gate = {k: max(1e-12, 10.0 * v) for k, v in sens.items()}
    assert rel(T, ref.T) < gate["T"]
    assert rel(U, ref.U) < gate["U"], (rel(U, ref.U), sens)
    assert rel(V, ref.V) < gate["V"], (rel(V, ref.V), sens)
    assert float(torch.tril(T, -1).abs().max()) == 0.0


@pytest.mark.parametrize("m,n,b", [(1, 1, 4), (1, 40, 8), (40, 1, 8), (3, 2, 1)])
def test_parity_degenerate_shapes(pkg, m, n, b):
    A = inputs.gaussian(m, n, seed=m * 3 + n)
    U, T, V = _factor(pkg, A, b, 1, 7)
    ref = oracle.randutv(A, b, 1, 7)
    assert rel(T, ref.T) < 1e-13
    assert rel(U, ref.U) < 1e-13
    assert rel(V, ref.V) < 1e-13


@pytest.mark.parametrize("m,n,b", [(256, 256, 32), (300, 180, 40), (180, 300, 40)])
def test_gaussian_inputs_invariants_and_spectra(pkg, m, n, b):
    """i.i.d. Gaussian inputs: clustered singular values leave U and V
    element-wise unpinned; gate on invariants, the diagonal, and T's norm."""
    A = inputs.gaussian(m, n, seed=31)
    U, T, V = _factor(pkg, A, b, 1, 3)
    ref = oracle.randutv(A, b, 1, 3)
    assert oracle.recon_error(A, U, T, V) < 1e-13
    assert oracle.orth_error(U) < 1e-13 and oracle.orth_error(V) < 1e-13
    assert float(torch.tril(T, -1).abs().max()) == 0.0
    assert rel(torch.diagonal(T), torch.diagonal(ref.T)) < 1e-10
    assert abs(float(T.norm() / A.norm()) - 1) < 1e-13


def test_t_only_equals_full(pkg):
    A = inputs.matrix("exp40", 320, 288, seed=2)
    U, T, V = _factor(pkg, A, 64, 1, 0)
    _, T2, _ = _factor(pkg, A, 64, 1, 0, want_u=False, want_v=False)
    assert torch.equal(T, T2)


def test_deterministic_and_resume_bitwise(pkg):
    A = inputs.matrix("exp40", 384, 384, seed=4)
    Ad = pkg.to_colmajor(A, "cuda")
    U1, T1, V1 = pkg.randutv_factor(Ad, 64, 1, 9)
    U2, T2, V2 = pkg.randutv_factor(Ad, 64, 1, 9)
    assert torch.equal(T1, T2) and torch.equal(U1, U2) and torch.equal(V1, V2)
    Up, Tp, Vp = pkg.randutv_factor_ex(Ad, 64, 1, 9, max_steps=2)
    assert pkg.randutv_stream_status() == 0
    # the partial state matches the oracle's partial state
    ref = oracle.randutv(A, 64, 1, 9, max_steps=2)
    assert rel(cpu(Tp), ref.T) < 1e-12
    Ur, Tr, Vr = pkg.randutv_factor_ex(Ad, 64, 1, 9, U=Up, T=Tp, V=Vp, first_step=2)
    assert pkg.randutv_stream_status() == 0
    assert torch.equal(Tr, T1) and torch.equal(Ur, U1) and torch.equal(Vr, V1)


def test_host_entry_point_matches_device(pkg):
    A = inputs.matrix("exp40", 200, 160, seed=5)
    U, T, V = _factor(pkg, A, 32, 1, 2)
    Ah = pkg.colmajor_empty(200, 160, device="cpu", pin=True)
    Ah.copy_(A)
    Uh = pkg.colmajor_empty(200, 200, device="cpu")
    Th = pkg.colmajor_empty(200, 160, device="cpu")
    Vh = pkg.colmajor_empty(160, 160, device="cpu")
    pkg.randutv_factor_host(Ah, 32, 1, 2, Uh, Th, Vh)
    assert torch.equal(Th.contiguous(), T) and torch.equal(Uh.contiguous(), U)
    assert torch.equal(Vh.contiguous(), V)


def test_zero_and_rank_deficient_inputs(pkg):
    A = torch.zeros(96, 80, dtype=f64)
    U, T, V = _factor(pkg, A, 32, 1, 0)
    assert float(T.abs().max()) == 0.0
    assert oracle.orth_error(U) < 1e-14 and oracle.orth_error(V) < 1e-14
    sig = torch.zeros(80, dtype=f64)
    sig[:10] = torch.linspace(2, 1, 10, dtype=f64)
    A = inputs.prescribed(96, 80, sig, seed=6)
    U, T, V = _factor(pkg, A, 32, 1, 0)
    assert oracle.recon_error(A, U, T, V) < 1e-13
    assert oracle.orth_error(U) < 1e-13 and oracle.orth_error(V) < 1e-13
    assert rel(torch.diagonal(T)[:10], sig[:10]) < 1e-12
    assert float(T[32:, 32:].norm()) < 1e-13


def test_errors_are_reported(pkg):
    A = inputs.gaussian(64, 64, seed=1)
    A[5, 7] = float("nan")
    with pytest.raises(pkg.RandutvError) as ei:
        pkg.randutv_factor(pkg.to_colmajor(A, "cuda"), 16, 1, 0)
    assert ei.value.status == 2
    L = pkg.lib()
    Ad = pkg.to_colmajor(inputs.gaussian(8, 8, seed=1), "cuda")
    ptr = Ad.data_ptr()
    assert L.randutv_factor(8, 8, ptr, 4, 4, 1, 0, None, ptr, None) == -4   # lda < m
    assert L.randutv_factor(8, 8, ptr, 8, 0, 1, 0, None, ptr, None) == -5   # b < 1
    assert L.randutv_factor(8, 8, ptr, 8, 4, -1, 0, None, ptr, None) == -6  # q < 0
    assert L.randutv_factor(0, 8, ptr, 8, 4, 1, 0, None, ptr, None) == -1
    # the context is still usable
    U, T, V = pkg.randutv_factor(Ad, 4, 1, 0)
    assert pkg.randutv_stream_status() == 0


# --------------------------------------------------- full-size sample ----

def _span_residual(Q, Qref):
    """|| (I - Qref Qref^T) Q ||_F / ||Q||_F: zero when the columns span the same space."""
    return float(torch.linalg.norm(Q - Qref @ (Qref.T @ Q)) / torch.linalg.norm(Q))


def test_full_size_first_step_matches_oracle(pkg):
    """16384 x 16384, b = 128, q = 1 (the timed configuration), step 0.

    The top singular values of a Gaussian matrix are clustered, so the
    rotation of the small SVD inside the first block is not pinned; every
    part of the state that the rotation does not touch is compared element
    by element (trailing T, U, V and the singular values), the rest by what
    the rotation leaves invariant (spans of the first b columns of U and V,
    column norms of the block rows of T).  Sampled rows of U T V^T must
    reproduce A."""
    n, b, q = 16384, 128, 1
    A = inputs.gaussian(n, n, seed=1)
    Ad = pkg.to_colmajor(A, "cuda")
    U, T, V = pkg.randutv_factor_ex(Ad, b, q, 0, max_steps=1)
    assert pkg.randutv_stream_status() == 0
    ref = oracle.randutv(A, b, q, 0, max_steps=1)
    Tc = cpu(T)
    assert rel(Tc[b:, b:], ref.T[b:, b:]) < 1e-12
    assert float(Tc[b:, :b].abs().max()) == 0.0
    assert rel(torch.diagonal(Tc)[:b], torch.diagonal(ref.T)[:b]) < 1e-12
    assert rel(Tc[:b, b:].norm(dim=0), ref.T[:b, b:].norm(dim=0)) < 1e-12
    del Tc
    Vc = cpu(V)
    assert rel(Vc[:, b:], ref.V[:, b:]) < 1e-12
    assert _span_residual(Vc[:, :b], ref.V[:, :b]) < 1e-12
    del Vc
    Uc = cpu(U)
    assert rel(Uc[:, b:], ref.U[:, b:]) < 1e-12
    assert _span_residual(Uc[:, :b], ref.U[:, :b]) < 1e-12
    del Uc, ref
    rows = torch.randperm(n, generator=torch.Generator().manual_seed(0))[:64]
    rec = (U[rows.cuda(), :] @ T) @ V.T
    assert rel(cpu(rec), A[rows, :]) < 1e-13

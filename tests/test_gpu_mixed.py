"""Mixed-precision path: the tcgen05 GEMM and the whole factorization.

The GEMM is checked against an FP64 product of the same operands: with one
BF16 plane, against the product of the BF16-rounded inputs (so only the FP32
accumulation differs); with three planes, against the exact product (the
split is FP32-accurate).  The factorization is checked by its errors against
the FP64 oracle: reconstruction (at most 1e-6), orthogonality after the
final re-orthogonalisation (at most 1e-7), exact zeros, and the diagonal of
T (the singular-value estimates) wherever the BF16 sketch resolves it (see
tests/sigma_tracking.py).
"""
import pytest
import torch

import oracle
import sigma_tracking
from paper_2002_06960_gb300 import inputs

pytestmark = pytest.mark.gpu

f32, f64 = torch.float32, torch.float64


@pytest.fixture(scope="module")
def pkg():
    from paper_2002_06960_gb300 import build
    build.build()
    import paper_2002_06960_gb300 as p
    p.lib()
    return p


def colmajor(p, X):
    return p.to_colmajor(X.to(f32), "cuda")


@pytest.mark.parametrize("transa", ["T", "N"])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 150, 300), (333, 256, 1000), (64, 40, 70),
                                   (1, 1, 1), (1030, 130, 4097)])
def test_bgemm_three_planes_is_fp32_accurate(pkg, transa, M, N, K):
    g = torch.Generator().manual_seed(M + 7 * N + K)
    A = torch.randn((K, M) if transa == "T" else (M, K), generator=g, dtype=f64).to(f32)
    B = torch.randn(K, N, generator=g, dtype=f64).to(f32)
    C = torch.randn(M, N, generator=g, dtype=f64).to(f32)
    ref = 0.5 * ((A.double().T if transa == "T" else A.double()) @ B.double()) - 2.0 * C.double()
    Cd = colmajor(pkg, C)
    pkg.randutv_gemm_bf16(transa, 0.5, colmajor(pkg, A), colmajor(pkg, B), -2.0, Cd, planes=3)
    torch.cuda.synchronize()
    err = (Cd.cpu().double() - ref).abs().max().item()
    # FP32 accumulation of K terms: error up to about K u max|a| max|b|, u = 2^-24;
    # an FP32 GEMM of the same operands serves as the yardstick
    ref32 = 0.5 * ((A.T if transa == "T" else A) @ B) - 2.0 * C
    err32 = (ref32.double() - ref).abs().max().item()
    bound = 2.0 * K * 2.0 ** -24 * (A.double().abs().max() * B.double().abs().max()).item() + 1e-6
    assert err <= max(4.0 * err32, 1e-7) + 0.25 * bound, (err, err32, bound)


@pytest.mark.parametrize("transa", ["T", "N"])
@pytest.mark.parametrize("M,N,K", [(256, 256, 512), (130, 70, 65), (512, 128, 2048)])
def test_bgemm_one_plane_is_the_bf16_product(pkg, transa, M, N, K):
    g = torch.Generator().manual_seed(M * 3 + N + K)
    A = torch.randn((K, M) if transa == "T" else (M, K), generator=g, dtype=f64).to(f32)
    B = torch.randn(K, N, generator=g, dtype=f64).to(f32)
    Ab = A.to(torch.bfloat16).double()
    Bb = B.to(torch.bfloat16).double()
    ref = (Ab.T if transa == "T" else Ab) @ Bb
    Cd = colmajor(pkg, torch.zeros(M, N))
    pkg.randutv_gemm_bf16(transa, 1.0, colmajor(pkg, A), colmajor(pkg, B), 0.0, Cd, planes=1)
    torch.cuda.synchronize()
    err = (Cd.cpu().double() - ref).abs().max().item()
    assert err <= 1e-5 * (K ** 0.5) * 4, err


@pytest.mark.parametrize("planes", [3, 1])
@pytest.mark.parametrize("transa,M,N,K", [("T", 128, 128, 16384), ("N", 200, 96, 5000),
                                          ("T", 64, 40, 1030)])
def test_bgemm_split_k(pkg, planes, transa, M, N, K):
    """beta = 0 with few output tiles over a long K takes the split-K path (partial
    products summed in a fixed order): the same accuracy bounds as the plain path."""
    g = torch.Generator().manual_seed(M + N + K + planes)
    A = torch.randn((K, M) if transa == "T" else (M, K), generator=g, dtype=f64).to(f32)
    B = torch.randn(K, N, generator=g, dtype=f64).to(f32)
    Cd = colmajor(pkg, torch.full((M, N), float("nan")))  # beta = 0: C is not read
    pkg.randutv_gemm_bf16(transa, 0.5, colmajor(pkg, A), colmajor(pkg, B), 0.0, Cd, planes=planes)
    torch.cuda.synchronize()
    got = Cd.cpu().double()
    if planes == 3:
        ref = 0.5 * ((A.double().T if transa == "T" else A.double()) @ B.double())
        ref32 = 0.5 * ((A.T if transa == "T" else A) @ B)
        err32 = (ref32.double() - ref).abs().max().item()
        bound = 2.0 * K * 2.0 ** -24 * (A.double().abs().max() * B.double().abs().max()).item()
        assert (got - ref).abs().max().item() <= max(4.0 * err32, 1e-7) + 0.25 * bound
    else:
        Ab, Bb = A.to(torch.bfloat16).double(), B.to(torch.bfloat16).double()
        ref = 0.5 * ((Ab.T if transa == "T" else Ab) @ Bb)
        assert (got - ref).abs().max().item() <= 1e-5 * (K ** 0.5) * 4


def _mixed(pkg, A, b, q, seed):
    U, T, V = pkg.randutv_factor_mixed(colmajor(pkg, A), b, q, seed)
    assert pkg.randutv_stream_status() == 0
    return U.cpu().double(), T.cpu().double(), V.cpu().double()


@pytest.mark.parametrize("kind,m,n,b,q", [("exp40", 512, 512, 64, 1), ("smooth", 1024, 1024, 256, 2),
                                          ("smooth", 768, 512, 128, 2), ("smooth", 512, 768, 128, 1),
                                          ("gauss", 300, 260, 64, 1), ("exp40", 333, 517, 64, 1),
                                          ("smooth", 517, 333, 128, 0)])
def test_mixed_factorization_errors(pkg, kind, m, n, b, q):
    A = inputs.matrix(kind, m, n, seed=1)
    U, T, V = _mixed(pkg, A, b, q, 0)
    recon = oracle.recon_error(A, U, T, V)
    ou, ov = oracle.orth_error(U), oracle.orth_error(V)
    # after the final re-orthogonalisation U and V are orthogonal to about the
    # rounding of their FP32 entries (sqrt(2/3) 2^-24 = 5e-8 for an exactly
    # orthogonal matrix), and U T V^T reproduces A to the FP32-level target
    assert recon < 1e-6, recon
    assert ou < 1e-7 and ov < 1e-7, (ou, ov)
    assert float(torch.tril(T, -1).abs().max()) == 0.0
    p = min(m, n)
    for k in range(0, p, b):   # every diagonal block is exactly diagonal
        bi = min(b, p - k)
        blk = T[k:k + bi, k:k + bi]
        assert float((blk - torch.diag(torch.diagonal(blk))).abs().max()) == 0.0
    ref = oracle.randutv(A, b, q, 0)
    # BF16 sketch and power products (u = 2^-8): each block tracks its own
    # trailing singular values where the sketch resolves them, and the first
    # block's resolved estimates equal the FP64 oracle's
    sigma_tracking.check(T, ref.T, b, q, 2.0 ** -8, tol=1e-2, first_tol=1e-4)


def test_mixed_single_block_is_svd(pkg):
    """b >= min(m, n): T = diag(sigma) of the prescribed spectrum, to FP32 accuracy."""
    sig = torch.exp(-torch.arange(96, dtype=f64) / 20.0)
    A = inputs.prescribed(96, 96, sig, seed=2)
    U, T, V = _mixed(pkg, A, 128, 1, 0)
    assert torch.allclose(torch.diagonal(T), sig, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("m,n,b", [(100, 60, 64), (60, 100, 64), (37, 37, 40)])
def test_mixed_one_ragged_block(pkg, m, n, b):
    """b > min(m, n) with min(m, n) not a multiple of 8: one block of width
    p = min(m, n).  T(0:p, 0:p) is the diagonal of the block's SVD.  For
    m >= n the block is all of A, so that diagonal is A's spectrum to FP32
    accuracy.  For m < n the block is A V1 with V1 from the BF16 sketch, whose
    span holds A's row space only to the sketch's rounding: the diagonal then
    lies below the spectrum (interlacing, A V1 being A times orthonormal
    columns) and meets it at the top."""
    A = inputs.matrix("exp16", m, n, seed=4)
    U, T, V = _mixed(pkg, A, b, 1, 0)
    p = min(m, n)
    assert oracle.recon_error(A, U, T, V) < 1e-6
    assert oracle.orth_error(U) < 1e-7 and oracle.orth_error(V) < 1e-7
    assert float(torch.tril(T, -1).abs().max()) == 0.0
    sig = torch.linalg.svdvals(A)
    d = torch.diagonal(T)[:p].abs()
    off = T[:p, :p] - torch.diag(torch.diagonal(T)[:p])
    assert float(off.abs().max()) < 1e-5 * float(sig[0])
    if m >= n:
        assert torch.allclose(d, sig, rtol=1e-4, atol=1e-6 * float(sig[0])), (d - sig).abs().max()
    else:
        assert bool((d <= sig * (1 + 1e-5) + 1e-6 * float(sig[0])).all()), (d - sig).max()
        assert float(((d[:4] - sig[:4]).abs() / sig[:4]).max()) < 1e-3, (d[:4], sig[:4])

"""Rank-k approximation through randUTV and its hand-written adjoint.

Forward: A_k from the GPU against the oracle's (1e-12).  Backward: the GPU
vector-Jacobian product against torch autograd through the FP64 oracle (the
reference gradient, itself pinned to central differences in the CPU suite),
and, at the 4096 x 4096 size, against central differences of the GPU
forward along random directions.
"""
import pytest
import torch

import oracle
from paper_2002_06960_gb300 import inputs

pytestmark = pytest.mark.gpu

f64 = torch.float64


@pytest.fixture(scope="module")
def lr():
    from paper_2002_06960_gb300 import build
    build.build()
    import paper_2002_06960_gb300 as p
    p.lib()
    from paper_2002_06960_gb300 import autograd
    return autograd


def rel(x, y):
    return float((x - y).norm() / y.norm())


def _ref_grad(A, B, k, b, q, seed):
    X = A.clone().requires_grad_(True)
    Ak = oracle.lowrank(X, k, b, q, seed)
    L = ((Ak - B) ** 2).sum()
    (g,) = torch.autograd.grad(L, X)
    return Ak.detach(), g


@pytest.mark.parametrize("m,n,b,k,q", [(40, 36, 8, 16, 1), (30, 44, 6, 12, 2), (128, 128, 16, 32, 1),
                                       (200, 160, 32, 64, 1), (96, 96, 16, 16, 0)])
def test_lowrank_forward_and_gradient(lr, m, n, b, k, q):
    kind = "step" if m == n == 128 else "exp16"
    A = inputs.matrix(kind, m, n, seed=3, gap=k) if kind == "step" else inputs.matrix(kind, m, n, seed=3)
    B = inputs.gaussian(m, n, seed=4, stream=inputs.STREAM_B)
    Ak_ref, g_ref = _ref_grad(A, B, k, b, q, 7)
    Ad = A.cuda().requires_grad_(True)
    Ak = lr.lowrank(Ad, k, b, q, 7)
    L = ((Ak - B.cuda()) ** 2).sum()
    L.backward()
    torch.cuda.synchronize()
    assert rel(Ak.detach().cpu(), Ak_ref) < 1e-12
    assert rel(Ad.grad.cpu(), g_ref) < 1e-9, rel(Ad.grad.cpu(), g_ref)


def test_lowrank_gradient_full_size_central_differences(lr):
    """4096 x 4096, k = 256, b = 128, q = 1, step spectrum with the gap at k:
    <grad, E> against (L(A + hE) - L(A - hE)) / 2h of the GPU forward."""
    n, k, b, q = 4096, 256, 128, 1
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    Q1 = torch.linalg.qr(torch.randn(n, n, generator=g, device="cuda", dtype=f64))[0]
    Q2 = torch.linalg.qr(torch.randn(n, n, generator=g, device="cuda", dtype=f64))[0]
    sig = inputs.spectrum("step", n, gap=k).cuda()
    A = (Q1 * sig) @ Q2.T
    del Q1, Q2
    B = torch.randn(n, n, generator=g, device="cuda", dtype=f64)
    Ad = A.clone().requires_grad_(True)
    Ak = lr.lowrank(Ad, k, b, q, 0)
    L = ((Ak - B) ** 2).sum()
    L.backward()
    grad = Ad.grad
    R = 2.0 * (Ak.detach() - B)          # dL/dA_k
    h = 1e-6 * float(A.norm())
    for _ in range(3):
        E = torch.randn(n, n, generator=g, device="cuda", dtype=f64)
        E /= E.norm()
        with torch.no_grad():
            # central difference of the map A -> A_k itself, contracted with dL/dA_k
            # (differencing the scalar loss, about 1.7e7 here, would lose the
            # derivative in the loss's own rounding)
            dAk = (lr.lowrank(A + h * E, k, b, q, 0) - lr.lowrank(A - h * E, k, b, q, 0)) / (2 * h)
        fd = float((R * dAk).sum())
        an = float((grad * E).sum())
        assert abs(an - fd) <= 1e-4 * abs(fd) + 1e-10 * float(grad.norm()), (an, fd)

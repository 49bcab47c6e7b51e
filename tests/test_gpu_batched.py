"""Batched randUTV (one persistent launch over uneven sizes) against the oracle.

The batched form draws its sketch with an FP32 Box-Muller of the same Philox
words; the oracle draws that identical G (``sketch_f32``) and runs the
method in FP64.  Each matrix of the batch is then checked against it:
reconstruction at most 1e-6, orthogonality at the level FP32 updates
reach, exact zeros below the diagonal, and the singular-value estimates:
each block tracks its own trailing singular values wherever the sketch
resolves them, and the first block's estimates equal the oracle's.  The launch is
also checked for determinism, for giving the same result when captured in a
CUDA graph and replayed, and for per-matrix status reporting.
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
    from paper_2002_06960_gb300 import batched
    return p, batched


def _mats(p, sizes, seed=2):
    out = []
    for i, (m, n) in enumerate(sizes):
        sig = torch.exp(-torch.arange(min(m, n), dtype=f64) / 16.0)
        A = inputs.prescribed(m, n, sig, seed=seed + i) if min(m, n) > 1 else \
            inputs.gaussian(m, n, seed=seed + i)
        out.append((A, p.to_colmajor(A.to(f32), "cuda")))
    return out


# Orthogonality of the FP32 factors: each of the ceil(p/b) steps applies an
# FP32 compact-WY update to U and V, and their rounding accumulates to about
# 1.5e-6 after 32 steps of 32 columns at n = 1024 (measured); an FP32 matrix
# that is orthogonal to rounding would show 5e-8.
ORTH_GATE = 2e-6

SIZES = [(200, 150), (150, 200), (64, 64), (300, 97), (33, 257), (16, 16), (1, 1), (1, 7), (9, 1),
         (128, 128), (257, 33)]


@pytest.mark.parametrize("b", [16, 32, 64])
def test_batched_errors_against_oracle(pkg, b):
    p, batched = pkg
    mats = _mats(p, SIZES)
    plan = batched.BatchedPlan([d for _, d in mats], b=b, q=1, seed=5)
    plan.run()
    torch.cuda.synchronize()
    assert int(plan.info.abs().sum()) == 0
    for i, (A, _) in enumerate(mats):
        U, T, V = (plan.U[i].cpu().double(), plan.T[i].cpu().double(), plan.V[i].cpu().double())
        Aq = A.to(f32).double()
        recon = oracle.recon_error(Aq, U, T, V)
        assert recon < 1e-6, (i, recon)
        ou, ov = oracle.orth_error(U), oracle.orth_error(V)
        assert ou < ORTH_GATE and ov < ORTH_GATE, (i, ou, ov)
        assert float(torch.tril(T, -1).abs().max()) == 0.0
        ref = oracle.randutv(Aq, b, 1, 5, matrix_id=i, sketch_f32=True)
        if min(Aq.shape) > 1:
            # FP32 sketch and products (u = 2^-24) against FP64 on the identical
            # sketch: each block tracks its own trailing singular values where
            # the sketch resolves them, and the first block's estimates equal
            # the oracle's (a different sketch would move them by about the
            # FP64 method's own error there, up to 1e-3)
            sigma_tracking.check(T, ref.T, b, 1, 2.0 ** -24, tol=2e-3, first_tol=1e-4)
    plan.close()


def test_batched_is_deterministic_and_graph_replays(pkg):
    p, batched = pkg
    mats = _mats(p, SIZES[:6], seed=9)
    plan = batched.BatchedPlan([d for _, d in mats], b=32, q=1, seed=1)
    plan.run()
    torch.cuda.synchronize()
    T1 = [t.clone() for t in plan.T]
    plan.run()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(T1, plan.T))
    for t in plan.T:
        t.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run()
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(T1, plan.T))
    plan.close()


def test_batched_reports_nonfinite_per_matrix(pkg):
    p, batched = pkg
    mats = _mats(p, [(40, 30), (30, 40), (50, 50)], seed=4)
    devs = [d for _, d in mats]
    devs[1][3, 5] = float("nan")
    plan = batched.BatchedPlan(devs, b=16, q=1, seed=0)
    plan.run()
    torch.cuda.synchronize()
    assert plan.info.tolist() == [0, 2, 0]
    plan.close()


def test_autotuner_installs_a_table(pkg):
    p, batched = pkg

    def make(m, n, i):
        return p.to_colmajor(inputs.gaussian(m, n, seed=i).to(f32), "cuda")

    rep = batched.autotune(make, per_class=4, reps=1, classes=[0, 1])
    assert set(rep) == {0, 1}
    assert all(b in (16, 32, 64) and ms > 0 for b, ms in rep.values())
    batched.set_tuning([0] * batched.N_CLASSES)  # back to the default


def test_batch_autotuner_tunes_on_the_batch(pkg):
    p, batched = pkg
    mats = [d for _, d in _mats(p, [(100, 90), (90, 120), (300, 250), (260, 300), (40, 40)] * 4,
                                 seed=21)]
    rep = batched.autotune_batch(mats, q=1, reps=1)
    assert set(rep["b"]) == {0, 2}            # the size classes present in the batch
    assert all(b in (16, 32, 64) and ms > 0 for b, ms in rep["b"].values())
    assert rep["ctas_per_sm"][0] in (0, 1)
    plan = batched.BatchedPlan(mats, b=0, q=1, seed=0)   # the tuned table serves b = 0
    plan.run()
    torch.cuda.synchronize()
    assert int(plan.info.abs().sum()) == 0
    plan.close()
    batched.set_tuning([0] * batched.N_CLASSES)  # back to the default


@pytest.mark.parametrize("b", [32, 64])
def test_batched_maximum_sizes(pkg, b):
    """Matrices at the 1024 limit, square and ragged, checked by properties
    that hold at any size: reconstruction at most 1e-6, orthogonality at the
    FP32 level, exact zeros below the diagonal, and the leading diagonal of T against the
    prescribed spectrum."""
    p, batched = pkg
    sizes = [(1024, 1024), (1024, 1001), (999, 1024), (1024, 40)]
    mats = _mats(p, sizes, seed=11)
    plan = batched.BatchedPlan([d for _, d in mats], b=b, q=1, seed=3)
    plan.run()
    torch.cuda.synchronize()
    assert int(plan.info.abs().sum()) == 0
    for i, (A, _) in enumerate(mats):
        U, T, V = (plan.U[i].cpu().double(), plan.T[i].cpu().double(), plan.V[i].cpu().double())
        Aq = A.to(f32).double()
        assert oracle.recon_error(Aq, U, T, V) < 1e-6, i
        ou, ov = oracle.orth_error(U), oracle.orth_error(V)
        assert ou < ORTH_GATE and ov < ORTH_GATE, (i, ou, ov)
        assert float(torch.tril(T, -1).abs().max()) == 0.0
        sig = torch.exp(-torch.arange(4, dtype=f64) / 16.0)
        d = torch.diagonal(T)[:4].abs()
        assert float(((d - sig).abs() / sig).max()) < 1e-3, (i, d)

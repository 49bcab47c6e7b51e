"""Failure detection on the device, without a GPU fault.

A bounded wait is made to run out on purpose: one CTA arrives at a grid
barrier sized for two, so the count it waits on never completes.  The wait
gives up after its limit (about two seconds), the kernel records
RANDUTV_ETIMEOUT with the site of the wait and returns, and the context
stays usable for the next factorization.
"""
import pytest
import torch

import oracle
from paper_2002_06960_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2002_06960_gb300 import build
    build.build()
    import paper_2002_06960_gb300 as p
    p.lib()
    return p


def test_bounded_wait_times_out_and_context_survives(pkg):
    import time
    t0 = time.perf_counter()
    st = pkg.lib().randutv_selftest_wait_timeout(None)
    waited = time.perf_counter() - t0
    assert st == 3  # RANDUTV_ETIMEOUT, recorded at the self-test's site
    assert 1.0 < waited < 30.0
    # the next call starts from clean status words and works
    A = inputs.matrix("exp40", 96, 80, seed=1)
    U, T, V = pkg.randutv_factor(pkg.to_colmajor(A, "cuda"), 16, 1, 0)
    torch.cuda.synchronize()
    assert pkg.randutv_stream_status() == 0
    assert oracle.recon_error(A, U.cpu(), T.cpu(), V.cpu()) < 1e-13

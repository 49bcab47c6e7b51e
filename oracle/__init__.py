"""CPU oracle for randUTV -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of the paper's methods (Heavner, Martinsson &
Quintana-Orti, arXiv 2002.06960: randUTV of §3.1 and Fig. 2, randUTV by blocks
of §3.2, HQRRP of §2.2),
written to check the GPU path against.  It shares no code with the GPU path: it has its own Philox
sketch generator, its own Householder QR and compact-WY factor, and uses the
library SVD for the b x b block.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The library never does, and it has no CPU
fallback: without its CUDA extension it raises.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (brute-force products of reflectors,
closed forms, a third-party Philox, invariants of the factorization); none is
"parity unpinned".
"""
from . import philox  # noqa: F401
from .hqrrp import PivotedQR, cpqr_pivots, hqrrp, sketch_omega  # noqa: F401
from .randutv_ab import randutv_ab, td_qr, tile_starts  # noqa: F401
from .randutv import (  # noqa: F401
    Factorization, block_schedule, householder_qr, householder_reflector, lowrank,
    normalise_svd, orth_error, randutv, range_basis, recon_error, sketch, small_svd,
    wy_factor,
)

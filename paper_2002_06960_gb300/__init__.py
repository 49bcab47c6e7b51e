"""randUTV on GB300: A = U T V^T by the blocked randomized UTV factorization
(Heavner, Martinsson & Quintana-Orti, arXiv 2002.06960, §3.1).

The compute path is librandutv.so (CUDA, sm_103a) behind the C-ABI in
include/randutv.h; this package is its ctypes binding plus seeded input
generators.  Build the library with ``python -m paper_2002_06960_gb300.build``.
"""
from . import inputs  # noqa: F401

_BINDING_NAMES = (
    "randutv_factor", "randutv_factor_ex", "randutv_factor_host", "randutv_stream_status",
    "randutv_philox_normal", "randutv_philox_normal_f32", "randutv_philox_words", "randutv_householder_qr",
    "randutv_wy_factor", "randutv_small_svd", "randutv_dgemm", "randutv_workspace_bytes",
    "randutv_finalize", "randutv_launch_count", "colmajor_empty", "to_colmajor", "lib",
    "RandutvError", "exported_names", "randutv_profile_enable", "randutv_profile_read", "randutv_factor_mixed",
    "randutv_gemm_bf16", "randutv_factor_ooc", "randutv_ooc_min_device_bytes", "randutv_hqrrp",
    "ab_tasks", "ab_io", "ab_block_name", "randutv_factor_ab", "randutv_factor_ooc_ab",
    "randutv_ooc_ab_min_device_bytes",
)


def __getattr__(name):
    if name in _BINDING_NAMES:
        from . import _lib
        return getattr(_lib, name)
    raise AttributeError(name)

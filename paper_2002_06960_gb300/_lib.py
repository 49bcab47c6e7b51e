"""ctypes binding of librandutv.so: argument marshalling only.

Every function has the name and argument order of the C entry point in
include/randutv.h; torch tensors stand in for the pointers (device tensors for
device pointers, CPU tensors for the _host entry points) and the current
torch stream is passed as the CUDA stream.  Nothing here computes: if the
library is missing, loading raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librandutv.so")

_lib = None

c_i64 = ctypes.c_int64
c_u64 = ctypes.c_uint64
c_u32 = ctypes.c_uint32
c_int = ctypes.c_int
c_dbl = ctypes.c_double
c_vp = ctypes.c_void_p

_SIGS = {
    "randutv_factor": (c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_u64, c_vp, c_vp, c_vp]),
    "randutv_factor_ex": (c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_u64, c_vp, c_vp,
                                  c_vp, c_int, c_vp, c_int]),
    "randutv_factor_host": (c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_u64, c_vp, c_vp,
                                    c_vp]),
    "randutv_stream_status": (c_int, [c_vp]),
    "randutv_philox_normal": (c_int, [c_u64, c_u32, c_u32, c_u32, c_i64, c_i64, c_vp, c_vp]),
    "randutv_philox_normal_f32": (c_int, [c_u64, c_u32, c_u32, c_u32, c_i64, c_i64, c_vp, c_vp]),
    "randutv_philox_words": (c_int, [c_u64, c_u32, c_u32, c_u32, c_u32, c_i64, c_vp, c_vp]),
    "randutv_householder_qr": (c_int, [c_i64, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp]),
    "randutv_wy_factor": (c_int, [c_i64, c_i64, c_vp, c_vp, c_vp, c_vp]),
    "randutv_small_svd": (c_int, [c_i64, c_vp, c_i64, c_vp, c_vp, c_vp, c_vp]),
    "randutv_dgemm": (c_int, [ctypes.c_char, ctypes.c_char, c_i64, c_i64, c_i64, c_dbl, c_vp,
                              c_i64, c_vp, c_i64, c_dbl, c_vp, c_i64, c_vp]),
    "randutv_workspace_bytes": (ctypes.c_size_t, [c_i64, c_i64, c_int, c_int]),
    "randutv_finalize": (None, []),
    "randutv_strerror": (ctypes.c_char_p, [c_int]),
    "randutv_last_error": (ctypes.c_char_p, []),
    "randutv_launch_count": (c_u64, [c_int]),
    "randutv_selftest_wait_timeout": (c_int, [c_vp]),
    "randutv_factor_mixed": (c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_u64, c_vp, c_vp,
                                     c_vp, c_int, c_vp]),
    "randutv_gemm_bf16": (c_int, [ctypes.c_char, c_i64, c_i64, c_i64, ctypes.c_float, c_vp, c_i64,
                                  c_vp, c_i64, ctypes.c_float, c_vp, c_i64, c_int, c_vp]),
    "randutv_householder_qr_noalloc": (c_int, [c_i64, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp]),
    "randutv_batched_plan_create": (c_int, [ctypes.POINTER(c_vp), c_int, c_vp, c_vp, c_vp, c_vp,
                                            c_int, c_int, c_u64, c_vp, c_vp, c_vp]),
    "randutv_batched_run": (c_int, [c_vp, c_vp, c_vp]),
    "randutv_batched_plan_destroy": (c_int, [c_vp]),
    "randutv_factor_batched": (c_int, [c_int, c_vp, c_vp, c_vp, c_vp, c_int, c_int, c_u64, c_vp,
                                       c_vp, c_vp, c_vp, c_vp]),
    "randutv_batched_set_tuning": (c_int, [c_vp, c_int, c_int]),
    "randutv_hqrrp": (c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_u64, c_vp, c_vp, c_vp, c_vp]),
    "randutv_ooc_min_device_bytes": (ctypes.c_size_t, [c_i64, c_i64, c_int]),
    "randutv_factor_ooc": (c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_u64, c_vp, c_vp,
                                   ctypes.c_size_t, c_vp, c_vp]),
    "randutv_lowrank": (c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_int, c_u64, c_vp, c_vp]),
    "randutv_lowrank_backward": (c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_int, c_u64,
                                         c_vp, c_vp, c_vp]),
    "randutv_factor_ab": (c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_u64, c_vp, c_vp,
                                  c_vp, c_int, c_vp]),
    "randutv_ooc_ab_min_device_bytes": (ctypes.c_size_t, [c_i64, c_i64, c_int, c_int]),
    "randutv_factor_ooc_ab": (c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_u64, c_vp, c_vp,
                                      ctypes.c_size_t, c_int, c_vp, c_vp]),
    "randutv_ab_tasks": (c_i64, [c_i64, c_i64, c_int, c_int, c_int, c_int, c_vp, c_vp, c_vp, c_i64]),
    "randutv_ab_op_name": (ctypes.c_char_p, [c_int]),
    "randutv_ab_io": (c_int, [c_i64, c_i64, c_int, c_int, c_int, c_int, c_i64, c_i64, c_vp, c_vp,
                              c_vp]),
    "randutv_profile_enable": (None, [c_int]),
    "randutv_profile_read": (c_int, [c_vp, c_int]),
    "randutv_profile_class_name": (ctypes.c_char_p, [c_int]),
}


def exported_names() -> list[str]:
    return list(_SIGS)


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"librandutv.so not found at {LIB_PATH}; build it with "
                "`python -m paper_2002_06960_gb300.build` (there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class RandutvError(RuntimeError):
    def __init__(self, fn: str, status: int):
        L = lib()
        msg = L.randutv_strerror(status).decode()
        detail = L.randutv_last_error().decode()
        super().__init__(f"{fn} returned {status}: {msg}" + (f" [{detail}]" if detail else ""))
        self.status = status


def _check(fn: str, status: int) -> int:
    if status != 0:
        raise RandutvError(fn, status)
    return status


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _dev(t, name):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64")
    return t


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _colmajor(t, rows, cols, name):
    """(pointer, ld) of a column-major rows x cols view: a tensor whose
    transpose is contiguous, i.e. stride (1, ld)."""
    if t.shape != (rows, cols):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {(rows, cols)}")
    if cols > 1 and rows > 1 and t.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    ld = t.stride(1) if cols > 1 else rows
    return max(ld, rows, 1)


def colmajor_empty(rows, cols, device="cuda", dtype=torch.float64, pin=False):
    """A rows x cols column-major tensor (the transpose of a contiguous one)."""
    if device == "cpu":
        base = torch.empty(cols, rows, dtype=dtype, pin_memory=pin)
    else:
        base = torch.empty(cols, rows, dtype=dtype, device=device)
    return base.T


def to_colmajor(x, device=None):
    device = x.device if device is None else device
    out = colmajor_empty(x.shape[0], x.shape[1], device=device, dtype=x.dtype)
    out.copy_(x)
    return out


# ------------------------------------------------------------ entry points

def randutv_factor_ex(A, b, q, seed, want_u=True, want_v=True, max_steps=-1, U=None, T=None,
                      V=None, first_step=0):
    """Asynchronous randUTV on the current stream; returns (U, T, V) tensors.

    A: m x n column-major float64 CUDA tensor (read only).  When resuming
    (first_step > 0) U, T, V must be the state returned by the earlier call.
    """
    m, n = A.shape
    lda = _colmajor(_dev(A, "A"), m, n, "A")
    if T is None:
        T = colmajor_empty(m, n, device=A.device)
    if want_u and U is None:
        U = colmajor_empty(m, m, device=A.device)
    if want_v and V is None:
        V = colmajor_empty(n, n, device=A.device)
    for t, r, c, nm in ((T, m, n, "T"), (U, m, m, "U"), (V, n, n, "V")):
        if t is not None:
            ld = _colmajor(_dev(t, nm), r, c, nm)
            if ld != r:
                raise ValueError(f"{nm} must have leading dimension {r}")
    _check("randutv_factor_ex", lib().randutv_factor_ex(
        m, n, _ptr(A), lda, b, q, seed, _ptr(U), _ptr(T), _ptr(V), max_steps, _stream(),
        first_step))
    return U, T, V


def randutv_stream_status():
    return lib().randutv_stream_status(_stream())


def randutv_factor(A, b, q, seed, want_u=True, want_v=True):
    """Synchronous randUTV; returns (U, T, V) (U or V None when not wanted)."""
    U, T, V = randutv_factor_ex(A, b, q, seed, want_u, want_v)
    _check("randutv_factor", randutv_stream_status())
    return U, T, V


def randutv_factor_host(A_host, b, q, seed, U_host=None, T_host=None, V_host=None):
    """randUTV on HOST buffers (CPU float64 column-major tensors, pinned or not)."""
    m, n = A_host.shape
    if A_host.is_cuda:
        raise ValueError("A_host must be a CPU tensor")
    lda = _colmajor(A_host, m, n, "A_host")
    _check("randutv_factor_host", lib().randutv_factor_host(
        m, n, _ptr(A_host), lda, b, q, seed, _ptr(U_host), _ptr(T_host), _ptr(V_host)))
    return U_host, T_host, V_host


def randutv_hqrrp(A, b, seed, want_q=True):
    """A P = Q R by HQRRP on a column-major float64 CUDA tensor (m >= n).
    Returns (Q or None, R, perm) with perm an int64 CUDA tensor."""
    m, n = A.shape
    lda = _colmajor(_dev(A, "A"), m, n, "A")
    R = colmajor_empty(m, n, device=A.device)
    Q = colmajor_empty(m, m, device=A.device) if want_q else None
    perm = torch.empty(n, dtype=torch.int64, device=A.device)
    _check("randutv_hqrrp", lib().randutv_hqrrp(m, n, _ptr(A), lda, b, seed, _ptr(Q), _ptr(R),
                                                 _ptr(perm), _stream()))
    return Q, R, perm


def randutv_ooc_min_device_bytes(m, n, b):
    return int(lib().randutv_ooc_min_device_bytes(m, n, b))


def randutv_factor_ooc(A_host, b, q, seed, U_host=None, V_host=None, device_bytes=0):
    """Out-of-HBM randUTV: A_host (CPU float64 column-major, pinned for the
    copies to overlap) is overwritten by T; U_host, V_host (CPU, or None) get
    U and V.  device_bytes = 0 takes twice the minimum.  Returns the bytes
    copied between host and device."""
    m, n = A_host.shape
    if A_host.is_cuda:
        raise ValueError("A_host must be a CPU tensor")
    lda = _colmajor(A_host, m, n, "A_host")
    for t, r, c, nm in ((U_host, m, m, "U_host"), (V_host, n, n, "V_host")):
        if t is not None:
            if t.is_cuda or t.dtype != torch.float64:
                raise ValueError(f"{nm} must be a CPU float64 tensor")
            if _colmajor(t, r, c, nm) != r:
                raise ValueError(f"{nm} must have leading dimension {r}")
    if device_bytes <= 0:
        device_bytes = 2 * randutv_ooc_min_device_bytes(m, n, b)
    moved = ctypes.c_double(0.0)
    _check("randutv_factor_ooc", lib().randutv_factor_ooc(
        m, n, _ptr(A_host), lda, b, q, seed, _ptr(U_host), _ptr(V_host), device_bytes,
        ctypes.byref(moved), _stream()))
    return moved.value


def randutv_philox_normal(seed, step, matrix_id, stream_id, rows, cols, device="cuda"):
    G = colmajor_empty(rows, cols, device=device)
    _check("randutv_philox_normal", lib().randutv_philox_normal(
        seed, step, matrix_id, stream_id, rows, cols, _ptr(G), _stream()))
    return G


def randutv_philox_normal_f32(seed, step, matrix_id, stream_id, rows, cols, device="cuda"):
    G = colmajor_empty(rows, cols, device=device, dtype=torch.float32)
    _check("randutv_philox_normal_f32", lib().randutv_philox_normal_f32(
        seed, step, matrix_id, stream_id, rows, cols, _ptr(G), _stream()))
    return G


def randutv_philox_words(seed, c0, c1, c2, c3, count, device="cuda"):
    out = torch.empty(count, 4, dtype=torch.int32, device=device)
    _check("randutv_philox_words", lib().randutv_philox_words(
        seed, c0, c1, c2, c3, count, _ptr(out), _stream()))
    return out


def randutv_householder_qr(panel):
    """In-place QR of a column-major r x c CUDA panel; returns (W, tau)."""
    r, c = panel.shape
    ld = _colmajor(_dev(panel, "panel"), r, c, "panel")
    W = colmajor_empty(r, c, device=panel.device)
    tau = torch.empty(c, dtype=torch.float64, device=panel.device)
    _check("randutv_householder_qr", lib().randutv_householder_qr(
        r, c, _ptr(panel), ld, _ptr(W), _ptr(tau), _stream()))
    return W, tau


def randutv_wy_factor(W, tau):
    r, c = W.shape
    ld = _colmajor(_dev(W, "W"), r, c, "W")
    if ld != r:
        raise ValueError("W must have leading dimension r")
    S = colmajor_empty(c, c, device=W.device)
    _check("randutv_wy_factor", lib().randutv_wy_factor(r, c, _ptr(W), _ptr(tau), _ptr(S),
                                                         _stream()))
    return S


def randutv_small_svd(B):
    b = B.shape[0]
    ld = _colmajor(_dev(B, "B"), b, b, "B")
    D = torch.empty(b, dtype=torch.float64, device=B.device)
    Us = colmajor_empty(b, b, device=B.device)
    Vs = colmajor_empty(b, b, device=B.device)
    _check("randutv_small_svd", lib().randutv_small_svd(b, _ptr(B), ld, _ptr(D), _ptr(Us),
                                                         _ptr(Vs), _stream()))
    return Us, D, Vs


def randutv_dgemm(transa, transb, alpha, A, B, beta, C):
    """C = alpha op(A) op(B) + beta C on column-major float64 CUDA tensors."""
    M, N = C.shape
    K = A.shape[0] if transa == "T" else A.shape[1]
    lda = _colmajor(A, *A.shape, "A")
    ldb = _colmajor(B, *B.shape, "B")
    ldc = _colmajor(C, M, N, "C")
    _check("randutv_dgemm", lib().randutv_dgemm(
        transa.encode(), transb.encode(), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb, beta,
        _ptr(C), ldc, _stream()))
    return C


def randutv_workspace_bytes(m, n, b, prec=0):
    return int(lib().randutv_workspace_bytes(m, n, b, prec))


def randutv_finalize():
    lib().randutv_finalize()


def randutv_launch_count(reset=False):
    return int(lib().randutv_launch_count(1 if reset else 0))


def randutv_profile_enable(on=True):
    lib().randutv_profile_enable(1 if on else 0)


def randutv_profile_read():
    """{class name: {launches, ms, flops, bytes}} of the recorded launches (clears them)."""
    L = lib()
    buf = (ctypes.c_double * 64)()
    nc = L.randutv_profile_read(buf, 16)
    if nc < 0 or nc > 16:
        raise RandutvError("randutv_profile_read", nc)
    out = {}
    for c in range(nc):
        name = L.randutv_profile_class_name(c).decode()
        out[name] = {"launches": int(buf[4 * c]), "ms": buf[4 * c + 1],
                     "flops": buf[4 * c + 2], "bytes": buf[4 * c + 3]}
    return out


def _dev32(t, name):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise ValueError(f"{name} must be float32")
    return t


def randutv_factor_mixed(A, b, q, seed, want_u=True, want_v=True, max_steps=-1, U=None, T=None,
                         V=None):
    """Mixed-precision randUTV on the current stream (FP32 column-major in/out).

    Returns (U, T, V); call randutv_stream_status() to wait and read errors."""
    m, n = A.shape
    lda = _colmajor(_dev32(A, "A"), m, n, "A")
    dev = A.device
    if T is None:
        T = colmajor_empty(m, n, device=dev, dtype=torch.float32)
    if want_u and U is None:
        U = colmajor_empty(m, m, device=dev, dtype=torch.float32)
    if want_v and V is None:
        V = colmajor_empty(n, n, device=dev, dtype=torch.float32)
    for t, r, c, nm in ((T, m, n, "T"), (U, m, m, "U"), (V, n, n, "V")):
        if t is not None and _colmajor(_dev32(t, nm), r, c, nm) != r:
            raise ValueError(f"{nm} must have leading dimension {r}")
    _check("randutv_factor_mixed", lib().randutv_factor_mixed(
        m, n, _ptr(A), lda, b, q, seed, _ptr(U), _ptr(T), _ptr(V), max_steps, _stream()))
    return U, T, V


def randutv_gemm_bf16(transa, alpha, A, B, beta, C, planes=3):
    """C = alpha op(A) B + beta C on the tensor cores (FP32 column-major CUDA tensors)."""
    M, N = C.shape
    K = A.shape[0] if transa == "T" else A.shape[1]
    lda = _colmajor(_dev32(A, "A"), *A.shape, "A")
    ldb = _colmajor(_dev32(B, "B"), *B.shape, "B")
    ldc = _colmajor(_dev32(C, "C"), M, N, "C")
    _check("randutv_gemm_bf16", lib().randutv_gemm_bf16(
        transa.encode(), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb, beta, _ptr(C), ldc, planes,
        _stream()))
    return C


# ------------------------------------------------------ randUTV by blocks

AB_KINDS = "AGYZBCPQUV"


def ab_block_name(blk):
    """Name of an encoded block: A01, G1, Y0, B1, C1, P0, Q0, U10, V01 (tile indices)."""
    kind, i, j = blk >> 40, (blk >> 20) & 0xFFFFF, blk & 0xFFFFF
    letter = AB_KINDS[kind]
    if letter in "AUV":
        return f"{letter}{i}{j}" if i < 10 and j < 10 else f"{letter}{i},{j}"
    return f"{letter}{i}"


def ab_tasks(m, n, b, q=0, want_u=False, want_v=False):
    """The analyzer's task list: [(operation, step, [in blocks], [out blocks])]."""
    L = lib()
    count = L.randutv_ab_tasks(m, n, b, q, int(want_u), int(want_v), None, None, None, 0)
    if count < 0:
        raise RandutvError("randutv_ab_tasks", int(count))
    ops = (ctypes.c_int32 * max(count, 1))()
    steps = (ctypes.c_int32 * max(count, 1))()
    opnd = (ctypes.c_int64 * max(8 * count, 1))()
    L.randutv_ab_tasks(m, n, b, q, int(want_u), int(want_v), ops, steps, opnd, count)
    out = []
    for t in range(count):
        ins = [ab_block_name(x) for x in opnd[8 * t:8 * t + 4] if x >= 0]
        outs = [ab_block_name(x) for x in opnd[8 * t + 4:8 * t + 8] if x >= 0]
        out.append((L.randutv_ab_op_name(ops[t]).decode(), steps[t], ins, outs))
    return out


def ab_io(m, n, b, q=0, want_u=False, want_v=False, max_tasks=-1, cache_blocks=0, trace=False):
    """(reads, writes[, trace]) of the traditional (cache_blocks=0) or cached dispatcher."""
    L = lib()
    r, w = ctypes.c_int64(0), ctypes.c_int64(0)
    tr = None
    if trace and cache_blocks > 0 and max_tasks > 0:
        tr = (ctypes.c_int64 * (max_tasks * cache_blocks))()
    _check("randutv_ab_io", L.randutv_ab_io(m, n, b, q, int(want_u), int(want_v), max_tasks,
                                            cache_blocks, ctypes.byref(r), ctypes.byref(w), tr))
    if tr is None:
        return r.value, w.value
    rows = [[(ab_block_name(x) if x >= 0 else "-") for x in tr[t * cache_blocks:(t + 1) * cache_blocks]]
            for t in range(max_tasks)]
    return r.value, w.value, rows


def randutv_factor_ab(A, b, q, seed, want_u=True, want_v=True, nstreams=4):
    """randUTV by blocks in HBM (tile QRs, tasks ordered by data flow on
    `nstreams` streams); asynchronous on the current stream.  Returns (U, T, V)."""
    m, n = A.shape
    lda = _colmajor(_dev(A, "A"), m, n, "A")
    T = colmajor_empty(m, n, device=A.device)
    U = colmajor_empty(m, m, device=A.device) if want_u else None
    V = colmajor_empty(n, n, device=A.device) if want_v else None
    _check("randutv_factor_ab", lib().randutv_factor_ab(
        m, n, _ptr(A), lda, b, q, seed, _ptr(U), _ptr(T), _ptr(V), nstreams, _stream()))
    return U, T, V


def randutv_ooc_ab_min_device_bytes(m, n, b, nstreams=4):
    return int(lib().randutv_ooc_ab_min_device_bytes(m, n, b, nstreams))


def randutv_factor_ooc_ab(A_host, b, q, seed, U_host=None, V_host=None, device_bytes=0,
                          nstreams=4):
    """randUTV by blocks with T, U, V in host memory behind an HBM cache of
    blocks (LRU, write-back of modified blocks).  A_host (CPU float64,
    column-major, pinned for the copies to overlap) is overwritten by T.
    device_bytes = 0 takes the minimum plus 64 blocks.  Returns
    {"reads": blocks read, "writes": blocks written, "bytes": bytes copied}."""
    m, n = A_host.shape
    if A_host.is_cuda:
        raise ValueError("A_host must be a CPU tensor")
    lda = _colmajor(A_host, m, n, "A_host")
    for t, r, c, nm in ((U_host, m, m, "U_host"), (V_host, n, n, "V_host")):
        if t is not None:
            if t.is_cuda or t.dtype != torch.float64:
                raise ValueError(f"{nm} must be a CPU float64 tensor")
            if _colmajor(t, r, c, nm) != r:
                raise ValueError(f"{nm} must have leading dimension {r}")
    bb = min(b, m, n)
    if device_bytes <= 0:
        device_bytes = randutv_ooc_ab_min_device_bytes(m, n, b, nstreams) + 64 * bb * bb * 8
    io = (ctypes.c_int64 * 3)()
    _check("randutv_factor_ooc_ab", lib().randutv_factor_ooc_ab(
        m, n, _ptr(A_host), lda, b, q, seed, _ptr(U_host), _ptr(V_host), device_bytes, nstreams,
        io, _stream()))
    return {"reads": int(io[0]), "writes": int(io[1]), "bytes": int(io[2])}


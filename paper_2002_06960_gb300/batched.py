"""Batched randUTV: binding of the plan/run C-ABI and the block-size autotuner.

``BatchedPlan`` marshals lists of column-major FP32 CUDA tensors into the
host pointer arrays of ``randutv_batched_plan_create``; ``run()`` is one
memset and one persistent kernel launch on the current stream, so it can be
captured in a CUDA graph.  ``autotune()`` times the launch for each block
size allowed (16, 32, 64) on seeded matrices of every size class and hands
the fastest to the library; ``autotune_batch()`` does the same on the
matrices of the batch it will serve, at full occupancy (up to two CTAs per
SM of matrices per class), and then picks the CTAs per SM of the grid.
The CTA tile of the products is not a tuning knob: the kernel takes 64 x 64
tiles, or 128 x 32 / 32 x 128 when one side of the output is at most 32.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib

B_CHOICES = (16, 32, 64)
CLASS_WIDTH = 128
N_CLASSES = 8


def _arr(ctype, values):
    a = (ctype * len(values))(*values)
    return a


class BatchedPlan:
    """Plan for factoring a list of FP32 matrices (column-major CUDA tensors)."""

    def __init__(self, As, b=0, q=1, seed=0, want_u=True, want_v=True):
        self.As = list(As)
        self.T = [_lib.colmajor_empty(a.shape[0], a.shape[1], device=a.device,
                                      dtype=torch.float32) for a in self.As]
        self.U = [_lib.colmajor_empty(a.shape[0], a.shape[0], device=a.device,
                                      dtype=torch.float32) for a in self.As] if want_u else None
        self.V = [_lib.colmajor_empty(a.shape[1], a.shape[1], device=a.device,
                                      dtype=torch.float32) for a in self.As] if want_v else None
        k = len(self.As)
        for a in self.As:
            if not a.is_cuda or a.dtype != torch.float32:
                raise ValueError("matrices must be float32 CUDA tensors")
        m = _arr(ctypes.c_int64, [a.shape[0] for a in self.As])
        n = _arr(ctypes.c_int64, [a.shape[1] for a in self.As])
        lda = _arr(ctypes.c_int64, [_lib._colmajor(a, a.shape[0], a.shape[1], "A")
                                    for a in self.As])
        ptr = lambda ts: _arr(ctypes.c_void_p, [t.data_ptr() for t in ts])
        self._keep = (m, n, lda)
        self.info = torch.zeros(k, dtype=torch.int32, device=self.As[0].device)
        h = ctypes.c_void_p()
        _lib._check("randutv_batched_plan_create", _lib.lib().randutv_batched_plan_create(
            ctypes.byref(h), k, m, n, ptr(self.As), lda, b, q, seed,
            ptr(self.U) if self.U else None, ptr(self.T), ptr(self.V) if self.V else None))
        self.handle = h

    def run(self):
        _lib._check("randutv_batched_run", _lib.lib().randutv_batched_run(
            self.handle, ctypes.c_void_p(self.info.data_ptr()), _lib._stream()))
        return self

    def close(self):
        if self.handle:
            _lib.lib().randutv_batched_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass


def set_tuning(b_for_class, ctas_per_sm=0):
    vals = list(b_for_class)
    arr = (ctypes.c_int * len(vals))(*vals)
    _lib._check("randutv_batched_set_tuning",
                _lib.lib().randutv_batched_set_tuning(arr, len(vals), ctas_per_sm))


def size_class(m, n):
    return min(N_CLASSES - 1, max(0, (max(m, n) - 1) // CLASS_WIDTH))


def autotune(make_matrix, per_class=24, q=1, reps=2, classes=None):
    """Pick the block size per size class by timing the batched launch.

    ``make_matrix(m, n, i)`` returns a float32 column-major CUDA matrix.
    For each class, ``per_class`` matrices with max(m, n) inside the class are
    timed with every b in B_CHOICES (CUDA events, after a warm-up run); the
    fastest b is kept.  Returns {class: (b, ms)} and installs the table.
    """
    classes = range(N_CLASSES) if classes is None else classes
    table = [0] * N_CLASSES
    report = {}
    g = torch.Generator().manual_seed(1234)
    for c in classes:
        lo, hi = c * CLASS_WIDTH + 1, (c + 1) * CLASS_WIDTH
        mats = []
        for i in range(per_class):
            big = int(torch.randint(max(lo, 17), hi + 1, (1,), generator=g))
            small = int(torch.randint(16, big + 1, (1,), generator=g))
            m, n = (big, small) if i % 2 == 0 else (small, big)
            mats.append(make_matrix(m, n, i))
        best = None
        for b in B_CHOICES:
            plan = BatchedPlan(mats, b=b, q=q, seed=0)
            plan.run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                plan.run()
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            plan.close()
            if best is None or ms < best[1]:
                best = (b, ms)
        table[c] = best[0]
        report[c] = best
    set_tuning(table)
    return report


def _time_plan(mats, b, q, reps):
    plan = BatchedPlan(mats, b=b, q=q, seed=0)
    plan.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.run()
    e1.record()
    e1.synchronize()
    plan.close()
    return e0.elapsed_time(e1) / reps


def autotune_batch(mats, q=1, reps=2, per_class=None, ctas_choices=(0, 1)):
    """Tune on the batch itself.  For each size class, time its first
    ``per_class`` matrices (default: two per SM, so the launch is as full as
    in the real run) with every b in B_CHOICES and keep the fastest; then time
    the whole batch with the resulting table for each CTAs-per-SM choice (0 =
    the occupancy limit) and keep the fastest.  Installs the table and
    returns {"b": {class: (b, ms)}, "ctas_per_sm": (choice, ms)}."""
    if per_class is None:
        per_class = 2 * torch.cuda.get_device_properties(mats[0].device).multi_processor_count
    groups = {}
    for A in mats:
        groups.setdefault(size_class(A.shape[0], A.shape[1]), []).append(A)
    table = [0] * N_CLASSES
    report = {}
    set_tuning(table, 0)
    for c in sorted(groups):
        sample = groups[c][:per_class]
        best = None
        for b in B_CHOICES:
            ms = _time_plan(sample, b, q, reps)
            if best is None or ms < best[1]:
                best = (b, ms)
        table[c] = best[0]
        report[c] = best
    best_c = None
    for cps in ctas_choices:
        set_tuning(table, cps)
        ms = _time_plan(mats, 0, q, reps)
        if best_c is None or ms < best_c[1]:
            best_c = (cps, ms)
    set_tuning(table, best_c[0])
    return {"b": report, "ctas_per_sm": best_c}


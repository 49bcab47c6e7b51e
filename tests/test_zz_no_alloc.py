"""The allocation-free Householder QR entry point.

randutv_householder_qr_noalloc serves callers that cannot let the library
allocate device memory (a program whose own allocator owns all of the GPU's
memory, or a loop that cannot pay for cudaMalloc/cudaFree): its scratch is a
fixed array inside the library.  Here it is called through the C-ABI twice in
a row and each result is checked against the allocating entry point on the
same input, within the tolerance of the other QR tests.  A second test runs
it first thing in a fresh process, under a preloaded shim that counts every
call of the CUDA runtime's allocation routines, and checks that the count
stays at zero (and that the allocating entry point does move it, so that the
zero means something).  This file is collected last, so a run that stops at
its first failure has already run every other test.
"""
import ctypes
import os
import subprocess
import sys
import textwrap

import pytest
import torch

from paper_2002_06960_gb300 import inputs

pytestmark = pytest.mark.gpu

f64 = torch.float64
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2002_06960_gb300 import build
    build.build()
    import paper_2002_06960_gb300 as p
    p.lib()
    return p


def _rel(x, y):
    d = float(torch.linalg.norm(y))
    return float(torch.linalg.norm(x - y)) / (d if d > 0 else 1.0)


def _noalloc(pkg, Y):
    r, c = Y.shape
    panel = pkg.to_colmajor(Y, "cuda")
    W = pkg.colmajor_empty(r, c)
    tau = torch.empty(c, dtype=f64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = pkg.lib().randutv_householder_qr_noalloc(r, c, ctypes.c_void_p(panel.data_ptr()),
                                                  panel.stride(1), ctypes.c_void_p(W.data_ptr()),
                                                  ctypes.c_void_p(tau.data_ptr()), st)
    return rc, panel.cpu(), W.cpu(), tau.cpu()


def _with_alloc(pkg, Y):
    panel = pkg.to_colmajor(Y, "cuda")
    W, tau = pkg.randutv_householder_qr(panel)
    torch.cuda.synchronize()
    return panel.cpu(), W.cpu(), tau.cpu()


def test_noalloc_qr_matches_allocating_qr_twice_in_a_row(pkg):
    for (r, c, seed) in [(3000, 96, 1), (20000, 128, 2)]:   # two calls, different shapes
        Y = inputs.gaussian(r, c, seed=seed)
        rc, P1, W1, t1 = _noalloc(pkg, Y)
        assert rc == 0
        P0, W0, t0 = _with_alloc(pkg, Y)
        assert _rel(P1, P0) < 1e-13
        assert _rel(W1, W0) < 1e-13
        assert _rel(t1, t0) < 1e-13


def test_noalloc_qr_rejects_sizes_beyond_its_maximum(pkg):
    Y = inputs.gaussian(400, 300, seed=3)
    rc, _, _, _ = _noalloc(pkg, Y)
    assert rc == 5   # RANDUTV_EUNSUPPORTED: more than 256 columns


# A shim preloaded ahead of the CUDA runtime: every allocation or free routine
# of the runtime API counts one call and forwards to the real routine.
_SHIM = r"""
#define _GNU_SOURCE
#include <dlfcn.h>
#include <stddef.h>
static long g_calls = 0;
long shim_alloc_calls(void) { return g_calls; }
void shim_reset(void) { g_calls = 0; }
#define FWD(name, params, args)                                   \
  int name params {                                               \
    static int (*real) params = 0;                                \
    if (!real) real = (int (*) params)dlsym(RTLD_NEXT, #name);    \
    ++g_calls;                                                    \
    return real ? real args : 999;                                \
  }
FWD(cudaMalloc, (void** p, size_t n), (p, n))
FWD(cudaMallocAsync, (void** p, size_t n, void* s), (p, n, s))
FWD(cudaMallocManaged, (void** p, size_t n, unsigned f), (p, n, f))
FWD(cudaMallocHost, (void** p, size_t n), (p, n))
FWD(cudaHostAlloc, (void** p, size_t n, unsigned f), (p, n, f))
FWD(cudaMallocPitch, (void** p, size_t* pitch, size_t w, size_t h), (p, pitch, w, h))
FWD(cudaFree, (void* p), (p))
FWD(cudaFreeAsync, (void* p, void* s), (p, s))
FWD(cudaFreeHost, (void* p), (p))
"""

_CHILD = textwrap.dedent("""
    import ctypes, sys
    sys.path.insert(0, {root!r})
    import torch
    import paper_2002_06960_gb300 as pkg
    from paper_2002_06960_gb300 import inputs
    shim = ctypes.CDLL({shim!r})
    shim.shim_alloc_calls.restype = ctypes.c_long
    lib = pkg.lib()
    torch.cuda.init()
    cases = []
    for (r, c, seed) in [(3000, 96, 1), (20000, 128, 2)]:
        Y = inputs.gaussian(r, c, seed=seed)
        panel = pkg.to_colmajor(Y, "cuda")
        W = pkg.colmajor_empty(r, c)
        tau = torch.empty(c, dtype=torch.float64, device="cuda")
        cases.append((Y, r, c, panel, W, tau))
    torch.cuda.synchronize()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    shim.shim_reset()
    for (Y, r, c, panel, W, tau) in cases:
        rc = lib.randutv_householder_qr_noalloc(r, c, ctypes.c_void_p(panel.data_ptr()),
                                                panel.stride(1), ctypes.c_void_p(W.data_ptr()),
                                                ctypes.c_void_p(tau.data_ptr()), st)
        assert rc == 0, rc
    calls = shim.shim_alloc_calls()
    assert calls == 0, "allocation routines called: %d" % calls
    # the allocating entry point does allocate (its scratch and status words)
    # on its first call, so the shim sees the library's allocations
    ref = []
    for (Y, r, c, panel, W, tau) in cases:
        ref.append((pkg.to_colmajor(Y, "cuda"), pkg.colmajor_empty(r, c),
                    torch.empty(c, dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    shim.shim_reset()
    for (Y, r, c, panel, W, tau), (p0, W0, t0) in zip(cases, ref):
        rc = lib.randutv_householder_qr(r, c, ctypes.c_void_p(p0.data_ptr()), p0.stride(1),
                                        ctypes.c_void_p(W0.data_ptr()),
                                        ctypes.c_void_p(t0.data_ptr()), st)
        assert rc == 0, rc
    torch.cuda.synchronize()
    assert shim.shim_alloc_calls() > 0, "the shim saw no allocation by the library"
    worst = 0.0
    for (Y, r, c, panel, W, tau), (p0, W0, t0) in zip(cases, ref):
        for x, y in ((panel, p0), (W, W0), (tau, t0)):
            worst = max(worst, float((x - y).norm() / y.norm()))
    assert worst < 1e-13, worst
    print("noalloc ok", worst)
""")


def test_noalloc_qr_allocates_nothing_in_a_fresh_process(pkg, tmp_path):
    src = tmp_path / "count_alloc.c"
    src.write_text(_SHIM)
    shim = tmp_path / "libcount_alloc.so"
    r = subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-o", str(shim), str(src), "-ldl"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ)
    env["LD_PRELOAD"] = str(shim) + ((" " + env["LD_PRELOAD"]) if env.get("LD_PRELOAD") else "")
    code = _CHILD.format(root=ROOT, shim=str(shim))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert "noalloc ok" in r.stdout

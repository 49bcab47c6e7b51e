"""Canned workloads on the GPU path, for profiling and smoke runs.

    python -m paper_2002_06960_gb300.workloads fp64 --n 4096 --b 128 --q 1
    python -m paper_2002_06960_gb300.workloads mixed --n 4096 --b 256 --q 2 --steps 1
    python -m paper_2002_06960_gb300.workloads batched --count 152 --b 32
    python -m paper_2002_06960_gb300.workloads hqrrp --n 4096 --b 128
    python -m paper_2002_06960_gb300.workloads backward --n 4096 --b 128 --k 256
    python -m paper_2002_06960_gb300.workloads ab --n 2048 --b 256
    python -m paper_2002_06960_gb300.workloads ooc_ab --n 2048 --b 256

Each builds a seeded input, runs the factorization through the public API,
waits for it, and exits non-zero if the library reports an error.
"""
from __future__ import annotations

import argparse
import sys

import torch


def _fp64(args):
    import paper_2002_06960_gb300 as pkg
    from paper_2002_06960_gb300 import inputs
    n = args.n
    A = pkg.colmajor_empty(n, n)
    A.copy_(inputs.gaussian(n, n, args.seed).cuda())
    U, T, V = (pkg.colmajor_empty(n, n) for _ in range(3))
    for _ in range(args.reps):
        pkg.randutv_factor_ex(A, args.b, args.q, 0, U=U, T=T, V=V)
    return pkg.randutv_stream_status()


def _mixed(args):
    import paper_2002_06960_gb300 as pkg
    n = args.n
    g = torch.Generator(device="cuda")
    g.manual_seed(args.seed)
    A = pkg.colmajor_empty(n, n, device="cuda", dtype=torch.float32)
    A.copy_(torch.randn(n, n, device="cuda", generator=g))
    U, T, V = (pkg.colmajor_empty(n, n, dtype=torch.float32) for _ in range(3))
    for _ in range(args.reps):
        pkg.randutv_factor_mixed(A, args.b, args.q, 0, U=U, T=T, V=V,
                                 max_steps=args.steps if args.steps > 0 else -1)
    return pkg.randutv_stream_status()


def _batched(args):
    import paper_2002_06960_gb300 as pkg
    from paper_2002_06960_gb300 import batched
    g = torch.Generator(device="cuda")
    g.manual_seed(args.seed)
    As = []
    for i in range(args.count):
        m, n = 512 + (i % 5) * 100, 512 + (i % 3) * 120
        A = pkg.colmajor_empty(m, n, device="cuda", dtype=torch.float32)
        A.copy_(torch.randn(m, n, device="cuda", generator=g))
        As.append(A)
    plan = batched.BatchedPlan(As, b=args.b, q=args.q, seed=0)
    for _ in range(args.reps):
        plan.run()
    torch.cuda.synchronize()
    bad = int((plan.info != 0).sum())
    plan.close()
    return bad


def _hqrrp(args):
    import paper_2002_06960_gb300 as pkg
    n = args.n
    g = torch.Generator(device="cuda")
    g.manual_seed(args.seed)
    A = pkg.colmajor_empty(n, n)
    A.copy_(torch.randn(n, n, generator=g, device="cuda", dtype=torch.float64))
    for _ in range(args.reps):
        pkg.randutv_hqrrp(A, args.b, 0, True)
    return pkg.randutv_stream_status()


def _backward(args):
    import paper_2002_06960_gb300 as pkg
    from paper_2002_06960_gb300 import autograd as ag
    n = args.n
    g = torch.Generator(device="cuda")
    g.manual_seed(args.seed)
    A = torch.randn(n, n, generator=g, device="cuda", dtype=torch.float64)
    B = torch.randn(n, n, generator=g, device="cuda", dtype=torch.float64)
    for _ in range(args.reps):
        X = A.clone().requires_grad_(True)
        ((ag.lowrank(X, args.k, args.b, args.q, 0) - B) ** 2).sum().backward()
    torch.cuda.synchronize()
    return pkg.randutv_stream_status()


def _ab(args):
    import paper_2002_06960_gb300 as pkg
    from paper_2002_06960_gb300 import inputs
    n = args.n
    A = pkg.to_colmajor(inputs.gaussian(n, n, args.seed).cuda(), "cuda")
    for _ in range(args.reps):
        pkg.randutv_factor_ab(A, args.b, args.q, 0, nstreams=args.streams)
    torch.cuda.synchronize()
    return pkg.randutv_stream_status()


def _ooc_ab(args):
    import paper_2002_06960_gb300 as pkg
    from paper_2002_06960_gb300 import inputs
    n = args.n
    T = pkg.colmajor_empty(n, n, device="cpu", pin=True)
    U = pkg.colmajor_empty(n, n, device="cpu", pin=True)
    V = pkg.colmajor_empty(n, n, device="cpu", pin=True)
    for _ in range(args.reps):
        T.copy_(inputs.gaussian(n, n, args.seed))
        io = pkg.randutv_factor_ooc_ab(T, args.b, args.q, 0, U, V, nstreams=args.streams)
    print(f"ooc_ab io: {io}")
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("kind", choices=["fp64", "mixed", "batched", "hqrrp", "backward", "ab", "ooc_ab"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--b", type=int, default=0, help="block size (default: 128 FP64, 256 mixed, 32 batched)")
    ap.add_argument("--q", type=int, default=-1, help="power steps (default: 1 FP64 and batched, 2 mixed)")
    ap.add_argument("--steps", type=int, default=0, help="mixed: block steps to run (0 = all)")
    ap.add_argument("--count", type=int, default=152, help="batched: number of matrices")
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--k", type=int, default=256, help="backward: rank of the approximation")
    ap.add_argument("--streams", type=int, default=8, help="ab, ooc_ab: compute streams")
    ap.add_argument("--seed", type=int, default=1)
    args = ap.parse_args(argv)
    defaults = {"fp64": (128, 1), "mixed": (256, 2), "batched": (32, 1), "hqrrp": (128, 0),
                "backward": (128, 1), "ab": (256, 1), "ooc_ab": (256, 1)}[args.kind]
    if args.b <= 0:
        args.b = defaults[0]
    if args.q < 0:
        args.q = defaults[1]
    st = {"fp64": _fp64, "mixed": _mixed, "batched": _batched, "hqrrp": _hqrrp,
          "backward": _backward, "ab": _ab, "ooc_ab": _ooc_ab}[args.kind](args)
    print(f"{args.kind}: status {st}")
    return 0 if st == 0 else 1


if __name__ == "__main__":
    sys.exit(main())

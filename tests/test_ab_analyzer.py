"""The analyzer and the dispatchers of randUTV by blocks (§3.2.4), on the CPU.

The task list and the I/O counts are checked against what the paper prints
for its 2 x 2-block example (Figs. fig:analyzer, fig:dispatcher_trad and
fig:dispatcher_cache, transcribed under tests/golden/), and the list of any
shape against the structure of the blocked algorithm: every step's task
counts, the last-block rule, and the data flow (every block read is written
earlier or is an input block).  No device is used.
"""
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def pkg():
    from paper_2002_06960_gb300 import build
    build.build()
    import paper_2002_06960_gb300 as p
    p.lib()
    return p


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append(line.rstrip("\n"))
    return rows


def test_task_list_of_the_2x2_example(pkg):
    want = []
    for row in _golden("fig_analyzer_2x2.txt"):
        op, ins, outs = (x.strip() for x in row.split("|"))
        want.append((op, ins.split(), outs.split()))
    got = pkg.ab_tasks(200, 200, 100, q=0)
    # the printed list names the second block's SVD factors P0, Q0; they are
    # the factors of block 1 (the same reading as the last-block rule)
    relabel = {"P1": "P0", "Q1": "Q0"}
    got = [(op, [relabel.get(x, x) for x in ins], [relabel.get(x, x) for x in outs])
           for (op, step, ins, outs) in got]
    assert got == want


def test_io_of_the_first_six_tasks(pkg):
    # traditional dispatcher: 16 I/O operations, 10 reads and 6 writes
    r, w = pkg.ab_io(200, 200, 100, q=0, max_tasks=6, cache_blocks=0)
    assert (r, w) == (10, 6)
    # a cache of 7 blocks: 4 I/O operations, all of them reads, and the cache
    # holds what the figure shows after every task (A00, least recently used,
    # makes room for A11 and is not written back: it was not modified)
    r, w, trace = pkg.ab_io(200, 200, 100, q=0, max_tasks=6, cache_blocks=7, trace=True)
    assert (r, w) == (4, 0)
    want = [row.split() for row in _golden("fig_dispatcher_cache_2x2.txt")]
    assert trace == want


@pytest.mark.parametrize("m,n,b,q,uv", [(200, 200, 100, 0, False), (300, 260, 64, 1, True),
                                        (333, 517, 64, 2, True), (517, 333, 128, 0, True),
                                        (64, 64, 64, 1, True), (1, 7, 4, 1, True), (9, 1, 4, 0, True)])
def test_task_list_structure(pkg, m, n, b, q, uv):
    tasks = pkg.ab_tasks(m, n, b, q=q, want_u=uv, want_v=uv)
    p = min(m, n)
    starts_m = list(range(0, p, b)) + list(range(p, m, b))
    starts_n = list(range(0, p, b)) + list(range(p, n, b))
    Mt, Nt, steps = len(starts_m), len(starts_n), (p + b - 1) // b
    by_step = {}
    for op, s, _, _ in tasks:
        by_step.setdefault(s, []).append(op)
    assert sorted(by_step) == list(range(steps))
    for k in range(steps):
        ops = by_step[k]
        right, left = k + 1 < Nt, k + 1 < Mt
        assert ops.count("Svd_of_block") == 1
        assert ops.count("Generate_normal_random") == ((Mt - k) if right else 0)
        # sketch and power products: (1 + 2q) (Mt - k)(Nt - k) tile products
        prods = sum(ops.count(x) for x in ("Gemm_tn_oz", "Gemm_tn_oo", "Gemm_nn_oz", "Gemm_nn_oo"))
        assert prods == (((1 + 2 * q) * (Mt - k) * (Nt - k)) if right else 0)
        qr_td = (Nt - k - 1 if right else 0) + (Mt - k - 1 if left else 0)
        assert ops.count("Comp_td_QR") == qr_td
        assert ops.count("Comp_dense_QR") == int(right) + int(left)
        # right transform on every tile row of A (all m rows) and of V
        rt = (Mt + (Nt if uv else 0)) * (Nt - k - 1) if right else 0
        ut = (Mt * (Mt - k - 1)) if (left and uv) else 0
        assert ops.count("Apply_right_Q_td_QR") == rt + ut
        assert ops.count("Apply_left_Qt_of_td_QR") == ((Mt - k - 1) * (Nt - k - 1) if left else 0)
        assert ops.count("Gemm_abta") == Nt - k - 1
        assert ops.count("Gemm_aabt") == k + (Nt if uv else 0)
    # data flow: every block read was written by an earlier task or is a
    # block of the input (A) or of the identity U, V
    written = set()
    for op, s, ins, outs in tasks:
        for x in ins:
            assert x[0] in "AUV" or x in written, (op, s, x)
        written.update(outs)


def test_cache_never_does_worse_than_traditional(pkg):
    m = n = 640
    b = 128
    r0, w0 = pkg.ab_io(m, n, b, q=1, want_u=True, want_v=True, cache_blocks=0)
    last = None
    for c in (12, 24, 48, 200):
        r, w = pkg.ab_io(m, n, b, q=1, want_u=True, want_v=True, cache_blocks=c)
        assert r + w < r0 + w0
        if last is not None:
            assert r + w <= last
        last = r + w
    # a cache that holds every block reads each input block once and writes nothing back
    nblocks_in = 3 * 5 * 5
    r, w = pkg.ab_io(m, n, b, q=1, want_u=True, want_v=True, cache_blocks=10000)
    assert (r, w) == (nblocks_in, 0)

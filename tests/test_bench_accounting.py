"""The benchmark's own arithmetic, on CPU: the per-launch work the roofline
divides by, and the committed DRAM traffic it reports beside it.

Algorithmic work per plan-iteration (A and the iterates entering the GEMMs
as one BF16 term each): A read once per GEMM (2 m n bytes), 2 m n flops per
column and GEMM, iterates 2 bytes, FP32 state 4 bytes.  The executed figures
are those of the chosen form (A as two BF16 terms: 4 bytes per entry, 3
products; with the lagged low term the heavy GEMMs stream A's high term and
run 2 products)."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
m, n = 3750, 41200


def test_algorithmic_work_per_launch():
    for K in (32, 81):
        nb, fl, ex, xb = bench.kernel_work("gemm1", m, n, K)
        assert (nb, fl) == (2 * m * n + 2 * n * K + 4 * m * K, 2 * m * n * K)
        assert (ex, xb) == (3 * 2 * m * n * K, 4 * m * n + 4 * n * K + 4 * m * K)
        nb, fl, ex, xb = bench.kernel_work("gemm2", m, n, K)
        # V in (2 bytes), q1 read + write (8), R1 out (2)
        assert (nb, fl) == (2 * m * n + 2 * m * K + 10 * n * K, 2 * m * n * K)
        nb, fl, _, _ = bench.kernel_work("solve", m, n, K)
        assert (nb, fl) == (4 * m * m + 8 * m * K, 2 * m * m * K)
    # the bench line's GEMM2 figure at the streaming width
    assert bench.kernel_work("gemm2", m, n, 32)[0] == 322_424_000


def test_lagged_form_executes_the_high_term_only():
    K = 32
    _, _, ex, xb = bench.kernel_work("gemm1", m, n, K, refine=True)
    assert ex == 2 * 2 * m * n * K and xb == 2 * m * n + 4 * n * K + 4 * m * K
    _, _, ex, xb = bench.kernel_work("gemm2", m, n, K, refine=True)
    # A_hi, V terms, q1 read / write, R1 terms, and the stored lo^T v read
    assert ex == 2 * 2 * m * n * K and xb == 2 * m * n + 4 * m * K + 16 * n * K
    # the low-term products carry no algorithmic work: they only refine
    assert bench.kernel_work("gemm1_lo", m, n, K)[:2] == (0, 0)
    assert bench.kernel_work("gemm2_lo", m, n, K)[:2] == (0, 0)


def test_committed_traffic_is_keyed_by_launch_width_and_source():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        t = json.load(f)
    h = bench.kernel_hash()
    for key, entry in t.items():
        if key.startswith("_"):
            continue
        wl, k = key.rsplit("_k", 1)
        for kern, e in entry.items():
            got = bench.committed_traffic(kern, wl, int(k))
            assert got == (e["bytes_per_launch"] if e["source_hash"] == h else None)
    # a width nobody measured has no traffic
    assert bench.committed_traffic("gemm2", "cfg1", 57) is None
    # the streaming default's GEMM2 counters: DRAM bytes within 2 % of the
    # executed bytes (A is not re-read)
    got = t["cfg1_k32"]["gemm2"]["bytes_per_launch"]
    xb = bench.kernel_work("gemm2", m, n, 32, refine=True)[3]
    assert abs(got - xb) <= 0.02 * xb

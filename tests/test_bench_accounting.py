"""The benchmark's accounting, on the CPU: the algorithmic bytes per point
of each step (outer residual + update 3d + 2s, a CG or CGNR iteration 8s, the
CGNR set-up 2s, d the outer and s the inner element bytes), the clock-record
parsing that rejects throttled runs."""
import bench


def _stats(outer, h, s):
    return {"outer_its": outer, "inner_its_h": h, "inner_its_s": s}


def test_algorithmic_bytes_per_step():
    n = 1000
    # no inner work: (k + 1) residual steps of 3d + 2s, k CGNR set-ups of 2s
    assert bench.algorithmic_bytes(n, _stats(0, 0, 0), 4) == n * (3 * 8 + 2 * 4)
    assert bench.algorithmic_bytes(n, _stats(1, 0, 0), 4) == n * (2 * (3 * 8 + 2 * 4) + 2 * 4)
    # each CG or CGNR iteration adds 8s per point, for any s
    for s in (2, 4, 8):
        base = bench.algorithmic_bytes(n, _stats(3, 0, 0), s)
        assert bench.algorithmic_bytes(n, _stats(3, 5, 0), s) - base == n * 5 * 8 * s
        assert bench.algorithmic_bytes(n, _stats(3, 0, 7), s) - base == n * 7 * 8 * s
    # the complex class: 16-byte outer and 8-byte inner elements
    assert bench.algorithmic_bytes(n, _stats(0, 0, 0), 8, 16) == n * (3 * 16 + 2 * 8)


def test_headline_algorithmic_bytes():
    """The 2048^2 FP32 solve (2585 outer, 58943 CG, 9058 CGNR iterations) moves
    9.56 TB of algorithmic bytes: the figure the headline roofline divides."""
    b = bench.algorithmic_bytes(2048 * 2048, _stats(2585, 58943, 9058), 4)
    per_pt = 2586 * 32 + 32 * (58943 + 9058) + 8 * 2585
    assert b == 2048 * 2048 * per_pt
    assert abs(b / 1e12 - 9.56) < 0.01


def test_clock_record_parsing():
    c = bench.Clocks(0)
    c.out = "\n".join([
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 1000.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage",
    ])
    sm = c.summary()
    assert sm["sm_mhz"] == 2070.0 and sm["sm_max_mhz"] == 2070.0 and sm["samples"] == 3
    assert sm["reasons"] == ["sw_power_cap"]
    c.out = "0, 1500, 2070, 900.0, 0x8, Active, Not Active, Not Active, Not Active"
    assert c.summary()["reasons"] == ["hw_slowdown"]
    c.out = ""
    assert c.summary()["samples"] == 0

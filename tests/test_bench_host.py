"""Host logic of bench.py (CPU): the roofline entry takes the flop-counted
kernel class with the most device time and measures it against the peak of
the arithmetic unit the library recorded for that class."""
import bench


def _stats(kernels):
    return {"prec": "mixed", "kernels": kernels}


CLOCKS = {"sm_max_mhz": 2070.0}


def test_roofline_picks_longest_flop_counted_class():
    st = _stats({
        "jacobi_cluster": {"launches": 17, "ms": 100.0, "flops": 0, "bytes": 0},  # no count: not a candidate
        "gemm:schur": {"launches": 33, "ms": 25.0, "flops": 1.0e12, "pipe": "tcgen05_tf32x3"},
        "gemm:matvec couple": {"launches": 2, "ms": 36.0, "flops": 3.3e10, "pipe": "fp64"},
    })
    r = bench.roofline(st, CLOCKS)
    assert r["kernel"] == "gemm:matvec couple" and r["launches"] == 2
    assert abs(r["avg_launch_ms"] - 18.0) < 1e-12


def test_roofline_peak_follows_the_recorded_pipe():
    pk = bench.fp_peaks(CLOCKS)
    fp64 = bench.roofline(_stats({"g": {"launches": 1, "ms": 1.0, "flops": 1e9, "pipe": "fp64"}}), CLOCKS)
    assert fp64["bound"] == "alu" and abs(fp64["peak"] - pk["fp64"]) < 1e-12
    assert abs(pk["fp64"] - 152 * 2 * 2 * 2070e6 / 1e12) < 1e-12
    fp32 = bench.roofline(_stats({"g": {"launches": 1, "ms": 1.0, "flops": 1e9, "pipe": "fp32"}}), CLOCKS)
    assert abs(fp32["peak"] - pk["fp32"]) < 1e-12
    # FP64-accurate Grams on the FP32 pipe: 36 FP32 operations per 8 algorithmic flops
    df = bench.roofline(_stats({"g": {"launches": 1, "ms": 1.0, "flops": 1e9, "pipe": "fp32_df"}}), CLOCKS)
    assert abs(df["peak"] - 152 * 128 * 2070e6 * 8 / 36 / 1e12) < 1e-9
    # tensor-core tiles: the measured bf16 rate x TF32/bf16 ratio / 3 (hi / lo split)
    tc = bench.roofline(_stats({"g": {"launches": 1, "ms": 1.0, "flops": 1e9, "pipe": "tcgen05_tf32x3"}}), CLOCKS)
    pv, _ = bench.peaks()
    bf16 = pv.get("bf16_tflops_sustained", pv["bf16_tflops"])
    assert tc["bound"] == "tensor" and abs(tc["peak"] - bf16 * (1.1 / 2.25) / 3.0) < 1e-9
    for r in (fp64, fp32, df, tc):
        assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15 and abs(r["achieved"] - 1.0) < 1e-12


def test_roofline_without_flop_counts_is_absent():
    assert bench.roofline(_stats({"jacobi": {"launches": 3, "ms": 5.0, "flops": 0}}), CLOCKS) is None


def test_memory_bound_class_takes_the_hbm_peak():
    pv, _ = bench.peaks()
    r = bench.roofline(_stats({"copy:merge": {"launches": 4, "ms": 2.0, "flops": 0, "bytes": 2.0e9}}), CLOCKS)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 1000.0) < 1e-9 and abs(r["frac"] - 1000.0 / pv["hbm_gbs"]) < 1e-12


def test_roofline_table_rows_by_time():
    st = _stats({
        "gemm:schur": {"launches": 3, "ms": 5.0, "flops": 1.0e12, "pipe": "tcgen05_tf32x3"},
        "copy:merge": {"launches": 4, "ms": 2.0, "flops": 0, "bytes": 2.0e9},
        "jacobi": {"launches": 3, "ms": 9.0, "flops": 0, "bytes": 0},
        "pchol_wy": {"launches": 2, "ms": 7.0, "flops": 3.0e9, "pipe": "fp64"},
    })
    rows = bench.roofline_table(st, CLOCKS)
    assert [r["kernel"] for r in rows] == ["pchol_wy", "gemm:schur", "copy:merge"]
    assert rows[0]["bound"] == "alu" and rows[2]["bound"] == "hbm"


def test_reference_arm_names_our_config():
    class A:
        grid, chi, eps, nrhs = 32, 3.0, 1e-6, 16
    assert bench.workload_name(A) == "grid32 (N=32768), chi=3, eps=1e-06, nrhs=16, leaf 64, eta 1"


def test_autotune_coordinate_descent_and_ldlt_space(monkeypatch):
    # host logic of the autotuner: one parameter at a time from the defaults,
    # the fastest value kept; the block LDL^T choice is only offered for a
    # symmetric matrix (a fake context and timer: no GPU)
    from paper_1703_06155_gb300 import autotune

    class Fake:
        def __init__(self, sym):
            self.sym, self.opts = sym, {}

        def _sizes(self):
            return (0, 9, 2)

        def stats(self):
            return {"symmetric": self.sym}

        def set_opts(self, **kw):
            self.opts = dict(kw)

    def timer(ctx, b, eps, precision, tol, stream, repeats):
        o = ctx.opts
        return 100.0 - 5.0 * (o.get("ldlt") == 1) - 3.0 * (o.get("tile_policy") == 1) + 2.0 * (o.get("stop_level", 0) > 0)

    monkeypatch.setattr(autotune, "_time_step", timer)
    for sym, want in ((1, 1), (0, 2)):
        ctx = Fake(sym)
        best, log = autotune.autotune(ctx, None, 1e-6, stream=object())
        assert best["ldlt"] == want and best["tile_policy"] == 1 and best["stop_level"] == 0
        assert ctx.opts["ldlt"] == want
        tried = {c["ldlt"] for c, _ in log}
        assert tried == ({2, 1} if sym else {2})

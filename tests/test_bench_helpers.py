"""CPU checks of bench.py's measurement helpers: the roofline of the profiled
estimate's launch shapes (bound, achieved, fraction, traffic scaled from an
ncu ratio, the dominant shape by time) and the summary of an ncu launch list
(launches from the first matching kernel, a launch limit, shares)."""
import pytest

import bench

PEAKS = {"hbm": 6768.4, "fp32": 78.4, "fp64": 1.257, "hbm_src": "measured"}


def _tot(reg_ms, blk_ms):
    return {"classes": [
        {"mode": 3, "threads": 128, "cluster": 0, "smem": 1, "levels": [0, 1], "launches": 4, "ms": reg_ms,
         "cell_iters": 1e9, "flops": 5e11, "bytes": 2e12},
        {"mode": 0, "threads": 512, "cluster": 0, "smem": 0, "levels": [3, 4, 5], "launches": 2, "ms": blk_ms,
         "cell_iters": 2e9, "flops": 2e11, "bytes": 8e11}],
        "ms": {"fields": 100.0}, "fft_bytes": 1e11, "fft_flops": 3e11, "launches": {"fields": 40}}


def test_roofline_dominant_streamed_shape():
    r = bench.roofline_classes({"prec": 1}, _tot(100.0, 160.0), PEAKS, lambda l: 16 << l)
    assert r["kernel"] == "solve_list_kernel<1, 0>" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    # 8e11 algorithmic bytes in 160 ms
    assert r["achieved"] == pytest.approx(8e11 / 0.160 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / PEAKS["hbm"])
    key = "solve_list_kernel<1, 0> [blocks of 512 threads, workspace in global memory]"
    dram, alg, _ = bench.TRAFFIC[key]
    assert r["traffic"] == pytest.approx(dram / alg * 8e11 / 2)  # per launch
    assert sum(r["time_share"].values()) == pytest.approx(1.0, abs=1e-3)
    assert [s["kernel"] for s in r["all_shapes"]] == ["solve_list_kernel<1, 0>", "solve_list_kernel<1, 3>",
                                                      "ce_rows+ce_cols"]


def test_roofline_alu_shapes():
    r = bench.roofline_classes({"prec": 1}, _tot(200.0, 160.0), PEAKS, lambda l: 16 << l)
    assert r["kernel"] == "solve_list_kernel<1, 3>" and r["bound"] == "alu" and r["traffic"] is None
    assert r["achieved"] == pytest.approx(5e11 / 0.200 / 1e12)
    assert r["peak"] == PEAKS["fp32"] and "issue" in r["note"]
    fields = [s for s in r["all_shapes"] if s["kernel"] == "ce_rows+ce_cols"][0]
    assert fields["bound"] == "alu" and fields["achieved"] == pytest.approx(3e11 / 0.100 / 1e12)
    # the FP64 form measures its ALU shapes against the FP64 peak
    r64 = bench.roofline_classes({"prec": 0}, _tot(10.0, 5.0), PEAKS, lambda l: 16 << l)
    assert r64["bound"] == "alu" and r64["kernel"] == "ce_rows+ce_cols" and r64["peak"] == PEAKS["fp64"]


def test_ncu_summary(tmp_path):
    csv = tmp_path / "launches.csv"
    rows = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    names = ["void setup_kernel(int)", "void at::fill(int)", "void solve_kernel<1, 0>(Args)",
             "void solve_kernel<1, 0>(Args)", "void ce_rows_kernel<float>(Args)", "void late_kernel(int)"]
    times = [("us", "5"), ("us", "1"), ("ms", "3"), ("ms", "1"), ("us", "500"), ("ms", "9")]
    for i, (n, (u, v)) in enumerate(zip(names, times)):
        rows.append('"%d","%s","gpu__time_duration.sum","%s","%s"' % (i, n, u, v))
    csv.write_text("\n".join(rows) + "\n")
    out = bench.ncu_summary(str(csv), start_at="at::", limit=4).splitlines()
    assert "setup_kernel" not in "".join(out) and "late_kernel" not in "".join(out)
    line = [ln for ln in out if "solve_kernel<1," in ln][0]
    assert line.split()[-3] == "2" and float(line.split()[-2]) == pytest.approx(4.0)
    assert out[-1].split()[1] == "4" and float(out[-1].split()[2]) == pytest.approx(4.501)

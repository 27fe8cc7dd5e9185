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


class _FakeEvent:
    def __init__(self, enable_timing=False):
        pass

    def record(self, stream=None):
        pass

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return 250.0


def _fake_library(calls):
    import types

    class Context:
        def __init__(self, model, stream=None, device=0):
            self.model = model
            self.log = []
            calls.append((model["prec"], model["cgv"], self.log))

        def set_schedule(self, s):
            self.log.append(("set_schedule", s))

        def autotune(self, seed=0):
            self.log.append(("autotune",))
            return []

        def calibrate_costs(self, seed=0):
            self.log.append(("calibrate_costs",))
            return [1.0] * (self.model["L"] + 1)

        def autotune_schedule(self, eps, seed=0, n_pilot=64, cost_model=0, reps=2):
            self.log.append(("autotune_schedule", cost_model, reps))
            return 1.0, 1.0, []

        def estimate(self, eps, seed, n_pilot=64, cost_model=0):
            self.log.append(("estimate", cost_model))
            L = self.model["L"] + 1
            return {"N": [4] * L, "V": [1.0] * L, "q_hat": 1.0, "bias": 0.0, "alpha": 1.0, "var_hat": 0.0,
                    "sums": [{"iters_total": 8, "n": 4}] * L}

        def close(self):
            self.log.append(("close",))

    return types.SimpleNamespace(Context=Context)


@pytest.mark.parametrize("cost_model,schedule", [(2, 1), (0, 1), (2, 0)])
def test_compare_sets_up_each_arm_like_the_default_line(monkeypatch, capsys, cost_model, schedule):
    """--compare: every arm is tuned as the default line is (plans per level,
    calibrated costs when cost model 2 is used, launch shapes re-timed on
    whole estimates under the work-queue schedule) before its timed
    estimates; run here against a fake library and fake CUDA events."""
    import argparse
    import json
    import sys
    import torch
    calls = []
    monkeypatch.setitem(sys.modules, "paper_1506_04694_gb300", _fake_library(calls))
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "set_stream", lambda s: None)
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda: None)
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, **k: real_empty(4, dtype=k.get("dtype")))
    monkeypatch.setattr(bench, "COST_MODEL", cost_model)
    args = argparse.Namespace(compare="lognormal_2layer_cgv_16to512", bf16_arm=False, fp64cg_arm=False,
                              seed=0, steps=2, warmup=1, schedule=schedule)
    bench.compare(args)
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert [(p, g) for p, g, _ in calls] == [(1, 1), (0, 0)]
    for prec, _, log in calls:
        setup = [e for e in log if e[0] != "estimate"][:-1]
        want = [("set_schedule", schedule), ("autotune",)]
        cal = [("calibrate_costs",)] if cost_model == 2 else []
        want += cal
        if schedule:
            want += [("autotune_schedule", cost_model, 1 if prec == 0 else 2)] + cal
        assert setup == want
        # the timed estimates come after the whole set-up, with the same cost model
        first = next(i for i, e in enumerate(log) if e[0] == "estimate")
        assert first == len(want) and log[-1] == ("close",)
        assert log[first:-1] == [("estimate", cost_model)] * 3
    assert out["mixed_cgv"]["time_to_eps_s"] == pytest.approx(0.25)
    assert out["speedup_mixed_cgv_vs_plain_fp64"] == pytest.approx(1.0)


def _run_bench(*args, env=None):
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    return subprocess.run([sys.executable, os.path.join(root, "bench.py"), *args], capture_output=True, text=True,
                          timeout=600, cwd=root, env=dict(os.environ, **(env or {})))


def test_reference_arm_line():
    """--impl reference: the oracle timed on the host cores prints one JSON
    line with the keys the benchmark contract names (run here on the small
    three-layer workload; the default workload takes about 15 s a step)."""
    import json
    r = _run_bench("--impl", "reference", "--workload", "paper_3layer_const_16to128", "--steps", "2",
                   "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["unit"] == "level-samples/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["ms_per_step"] > 0 and line["time_to_eps_extrapolated_s"] > 0
    assert line["config"]["workload"] == "paper_3layer_const_16to128"
    assert "piecewise constant" in line["metric"] and "eps=0.002" in line["metric"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_fixed_count_workload_rejected():
    # the constant two-layer workload has a fixed N per level and no RMSE
    # target: the time-to-eps benchmark refuses it with a message
    r = _run_bench("--impl", "reference", "--workload", "const_2layer_8to32")
    assert r.returncode == 2 and "no RMSE target" in r.stderr
    r = _run_bench("--compare", "const_2layer_8to32")
    assert r.returncode != 0 and "no RMSE target" in r.stderr


def test_reference_arm_other_ranks_do_no_work():
    # under torchrun only rank 0 times the oracle and prints; the others exit 0
    r = _run_bench("--impl", "reference", "--workload", "paper_3layer_const_16to128", "--steps", "1",
                   "--warmup", "0", env={"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and r.stdout.strip() == ""

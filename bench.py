#!/usr/bin/env python
"""Benchmark of the MLMC level batch on GB300.

One step = one complete adaptive MLMC estimate to RMSE eps (pilot batches on
every level, then top-ups to the cost-optimal N_l until the sampling error is
<= eps^2/2), i.e. one pass of every stage of the hot path: Philox normals,
circulant-embedding fields, TPFA assembly, multigrid-preconditioned CG, the
outflow QoI, the level reduction and the estimator.  Default workload: two
layers, piecewise log-normal fields (sigma^2 = 1, lambda = 0.3, 2-norm),
levels m = 16 .. 256, eps = 1e-3, FP64.

value = level samples solved per second (sum_l N_l over all ranks / time);
ms_per_step = the time-to-eps of one estimate.

--impl reference times the CPU FP64 oracle on the host cores on a bounded
sample of the same workload and prints the same line with "impl": "reference".
"""
import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "lognormal_2layer_16to256"
# FP64 vector peak of GB300 (nominal 1.25 TFLOP/s: 152 SMs x 2 FP64 FMA/clk x
# 2 flop x ~2.06 GHz).
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 80.5
# Sample of the oracle timed for the CPU baseline: samples per level.
CPU_SAMPLE = {0: 512, 1: 128, 2: 48, 3: 16, 4: 8, 5: 2, 6: 1}


def _worker_init():
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"


def _oracle_worker(job):
    """Runs in a spawned process: oracle samples of one level; returns
    (level, seconds, per-sample (qf, qc, qc_cgv))."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import workloads
    from oracle import darcy
    name, overrides, level, first, n, seed = job
    model = darcy.Model.from_dict(workloads.workload(name, **overrides))
    cache = {}
    darcy.layer_fields(model, seed, level, first, model.m(level), cache)  # embedding table
    t = time.perf_counter()
    out = []
    for i in range(first, first + n):
        r = darcy.sample(model, seed, level, i, cache)
        out.append((r["qf"], r["qc"], r["qc_cgv"]))
    return level, time.perf_counter() - t, out


def oracle_rates(name, overrides, levels, seed, cores):
    """Per-level oracle throughput (samples/s) on `cores` spawned processes,
    plus the per-sample results."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    jobs = []
    for lvl in levels:
        n = CPU_SAMPLE.get(lvl, 1)
        per = max(1, n // cores)
        for c0 in range(0, n, per):
            jobs.append((name, overrides, lvl, 10_000_000 + c0, min(per, n - c0), seed))
    rates, results = {}, {}
    with ctx.Pool(cores, initializer=_worker_init) as pool:
        for lvl in levels:
            lj = [j for j in jobs if j[2] == lvl]
            t = time.perf_counter()
            res = pool.map(_oracle_worker, lj)
            wall = time.perf_counter() - t
            n = sum(j[4] for j in lj)
            rates[lvl] = n / wall
            results[lvl] = [x for r in res for x in r[2]]
    return rates, results


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, path=None):
        self.gpu = gpu_index
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), "mlmc_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 10:
                rows.append(p)
        if not rows:
            return None
        try:
            busy = [r for r in rows if float(r[4]) >= 50] or rows
            sm = sorted(float(r[1]) for r in busy)
            reasons = set()
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for r in busy:
                for k, name in enumerate(names):
                    if r[6 + k].lower() == "active":
                        reasons.add(name)
            return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(busy[0][2]), "reasons": sorted(reasons),
                    "samples": len(busy)}
        except ValueError:
            return None


def run_reference(args, d):
    """The CPU oracle on the host cores, bounded sample; same metric and unit."""
    cores = min(host_cores(), 16)
    L = d["L"]
    levels = list(range(L + 1))
    times, values = [], []
    from oracle import mlmc
    import numpy as np
    for step in range(args.warmup + args.steps):
        rates, results = oracle_rates(args.workload, {}, levels, args.seed, cores)
        # sample sizes from the oracle's own pilot variances (deterministic cost model)
        V = []
        for lvl in levels:
            arr = np.array(results[lvl])
            y = arr[:, 0] - (arr[:, 2] if (d["cgv"] and lvl) else arr[:, 1])
            V.append(float(np.var(y, ddof=1)) if len(y) > 1 else float(np.var(arr[:, 0])))
        from oracle import darcy
        model = darcy.Model.from_dict(d)
        C = [mlmc.parity_cost(model, lvl) for lvl in levels]
        N = mlmc.optimal_samples(d["eps"], V, C)
        t_eps = sum(n / rates[lvl] for lvl, n in zip(levels, N))
        if step >= args.warmup:
            times.append(t_eps)
            values.append(sum(N) / t_eps)
    value = sum(values) / len(values)
    ms = 1000 * sum(times) / len(times)
    sample = ("oracle (numpy/scipy FP64; banded Cholesky in 2-D, sparse LU in 3-D) on %d spawned processes; per step %s samples "
              "of levels %s timed, time-to-eps extrapolated as sum_l N_l / rate_l with N_l from the "
              "oracle's pilot variances" % (cores, [CPU_SAMPLE.get(lv, 1) for lv in levels], levels))
    return {"impl": "reference", "metric": metric_name(d, args), "value": value, "unit": "level-samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (Philox4x64-10 streams)", "config": config_block(args, d),
            "cpu_baseline": {"value": value, "unit": "level-samples/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "level-samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def metric_name(d, args):
    return ("level solves/s: MLMC time-to-RMSE eps=%g, %d-layer piecewise log-normal%s, m=%d..%d, %s%s"
            % (d["eps"], d["n_layers"], ", 3-D" if d.get("dim", 2) == 3 else "", d["m0"], d["m0"] << d["L"], {0: "FP64", 1: "mixed FP32-MG", 2: "mixed FP32-MG (BF16 faces)",
                                                         3: "FP64 CG with FP32-MG preconditioner"}[d["prec"]],
               ", CGV" if d["cgv"] else ""))


def config_block(args, d):
    return {"workload": args.workload, "m_levels": [d["m0"] << l for l in range(d["L"] + 1)],
            "eps": d["eps"], "sigma2": d["sigma2"][0], "lambda": d["lam"][0], "layers": d["n_layers"],
            "dim": d.get("dim", 2), "norm_r": d["norm_r"],
            "cgv": d["cgv"], "prec": PREC_NAMES[d["prec"]],
            "solver_tol": d["tol"], "seed": args.seed, "cost_model": "deterministic m_l^d (1 + n_coarse/2^d)",
            "l2": "flushed between steps (256 MB device write)", "parallelism": "replicas%d" % args.gpus}


def reduce_over_ranks(total_ms, n_total, device):
    """Whole-job timing: the slowest rank's time and the samples of all ranks
    (one replica per GPU; the only cross-rank communication of the benchmark)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), float(n_total)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(n_total)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


PREC_NAMES = {0: "fp64", 1: "fp32-mg/fp64-refinement", 2: "fp32-mg-bf16-faces/fp64-refinement",
              3: "fp64-cg/fp32-mg-preconditioner"}


def compare(args):
    """Time-to-eps: the workload as configured (mixed precision + CGV) against
    plain FP64 batched MLMC without CGV at the same eps and levels; with
    --bf16-arm also the mixed CGV form with BF16 multigrid faces (prec 2), with
    --fp64cg-arm the CGV form with FP64 fields and CG around an FP32
    multigrid preconditioner (prec 3)."""
    import torch
    import paper_1506_04694_gb300 as pk
    import workloads
    d = workloads.workload(args.compare)
    arms = {"mixed_cgv": dict(d), "plain_fp64": dict(d, prec=0, cgv=0)}
    if args.bf16_arm:
        arms["mixed_cgv_bf16_faces"] = dict(d, prec=2)
    if args.fp64cg_arm:
        arms["fp64cg_fp32mg_cgv"] = dict(d, prec=3)
    out = {"compare": args.compare, "eps": d["eps"], "m_levels": [d["m0"] << l for l in range(d["L"] + 1)],
           "steps": args.steps, "warmup": args.warmup}
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    for name, md in arms.items():
        ctx = pk.Context(md, stream=stream)
        ctx.autotune(seed=args.seed + 12345)
        for _ in range(args.warmup):
            ctx.estimate(md["eps"], args.seed, n_pilot=64, cost_model=0)
        torch.cuda.synchronize()
        ts, est = [], None
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            est = ctx.estimate(md["eps"], args.seed, n_pilot=64, cost_model=0)
            e1.record(ctx.stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        out[name] = {"time_to_eps_s": sum(ts) / len(ts), "N": est["N"], "V": est["V"], "q_hat": est["q_hat"],
                     "bias_estimate": est["bias"], "alpha": est["alpha"],
                     "var_hat": est["var_hat"], "level_samples_per_s": sum(est["N"]) / (sum(ts) / len(ts)),
                     "iters_per_sample": [round(x["iters_total"] / max(x["n"], 1), 2) for x in est["sums"]],
                     "prec": PREC_NAMES[md["prec"]],
                     "cgv": md["cgv"]}
        ctx.close()
        del ctx
        torch.cuda.empty_cache()
    out["speedup_mixed_cgv_vs_plain_fp64"] = out["plain_fp64"]["time_to_eps_s"] / out["mixed_cgv"]["time_to_eps_s"]
    if args.bf16_arm:
        out["speedup_bf16_faces_vs_fp32_faces"] = (out["mixed_cgv"]["time_to_eps_s"] /
                                                   out["mixed_cgv_bf16_faces"]["time_to_eps_s"])
    if args.fp64cg_arm:
        out["speedup_fp64cg_fp32mg_cgv_vs_plain_fp64"] = (out["plain_fp64"]["time_to_eps_s"] /
                                                          out["fp64cg_fp32mg_cgv"]["time_to_eps_s"])
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare", default=None,
                    help="workload name: time-to-eps of its mixed-precision CGV form against plain FP64 "
                         "batched MLMC (no CGV) at the same eps and level set; prints one JSON line")
    ap.add_argument("--bf16-arm", action="store_true",
                    help="with --compare: add the mixed CGV arm with BF16 multigrid faces (prec 2)")
    ap.add_argument("--fp64cg-arm", action="store_true",
                    help="with --compare: add the CGV arm with FP64 CG around an FP32 multigrid (prec 3)")
    ap.add_argument("--clocks-out", default=None,
                    help="file for the raw nvidia-smi clock samples of the timed region (default: a temp file)")
    ap.add_argument("--prec", type=int, default=None, choices=[0, 1, 2, 3],
                    help="override the workload's solver precision mode")
    args = ap.parse_args()
    if args.compare:
        compare(args)
        return

    import workloads
    d = workloads.workload(args.workload)
    if args.prec is not None:
        d["prec"] = args.prec
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, d)), flush=True)
        return

    import torch
    import torch.distributed as dist
    import paper_1506_04694_gb300 as pk

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # a non-default stream: lets the library capture each estimate round in a CUDA graph
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    ctx = pk.Context(d, device=local, stream=stream)
    tune = ctx.autotune(seed=args.seed + 12345)  # untimed set-up: launch plan per level
    eps = d["eps"]
    seed = args.seed + 7919 * rank
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        ctx.estimate(eps, seed, n_pilot=64, cost_model=0)
    torch.cuda.synchronize(dev)

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    phys = vis.split(",")[local] if vis else str(local)
    clocks = ClockSampler(phys, args.clocks_out)
    clocks.start()
    barrier()
    torch.cuda.synchronize(dev)
    ctx.profile(True)
    step_ms, n_total, est = [], 0, None
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        est = ctx.estimate(eps, seed, n_pilot=64, cost_model=0)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        n_total += sum(est["N"])
    torch.cuda.synchronize(dev)
    barrier()
    ctx.profile(False)
    clk = clocks.stop()
    prof = ctx.profile_read()
    total_ms, n_all = reduce_over_ranks(sum(step_ms), n_total, dev)

    # end to end through the host-buffer API: the estimate's per-level sample
    # counts run with per-sample results copied back to host memory
    e2e = None
    if rank == 0:
        N = est["N"]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for lvl, n in enumerate(N):
            ctx.level_batch_host(lvl, n, seed, first=0)
        torch.cuda.synchronize(dev)
        te = time.perf_counter() - t0
        e2e = {"value": sum(N) / te, "unit": "level-samples/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": int(sum(N) * (3 * 8 + 4) + (d["L"] + 1) * 128),
               "note": "inputs are (seed, model) passed by value; per-sample Q_f, Q_c, Q_cgv and "
                       "iterations copied to host inside the timed region"}

    if rank != 0:
        return
    stage_ms = prof["ms"]
    dom = max(stage_ms, key=lambda k: stage_ms[k])
    if stage_ms[dom] <= 0:
        raise RuntimeError("no stage timing collected in the timed region")
    launches = int(sum(prof["launches"].values()))
    prec = d["prec"]
    fp64_src = "nominal FP64 vector rate (152 SMs x 2 DFMA/clk x 2.06 GHz)"
    fp32_src = "nominal FP32 vector rate (152 SMs x 128 FFMA/clk x 2.07 GHz)"
    if dom == "solve":
        # algorithmic flops counted by the library per level from its cycle (V/W, sweeps); with
        # prec 3 only the FP64 CG part (23 per cell-iteration) is set against the FP64 peak
        if prec == 0:
            flops, peak, src, what = prof["solve_flops"], FP64_PEAK_TFLOPS, fp64_src, "FP64 MG-PCG"
        elif prec == 3:
            flops, peak, src, what = 23.0 * prof["cell_iters"], FP64_PEAK_TFLOPS, fp64_src, "FP64 CG part"
        else:
            flops, peak, src, what = prof["solve_flops"], FP32_PEAK_TFLOPS, fp32_src, "FP32 MG-PCG"
        ach = flops / (stage_ms["solve"] / 1e3) / 1e12
        roof = {"kernel": "solve_kernel<%d, mode> (assembly + MG-PCG + QoI; %s)" % (prec, what), "bound": "alu",
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "peak_source": src}
    else:
        # radix-2 FFT count, 5 log2(M) flops per point of each length-M transform, per level
        f32 = prec in (1, 2)
        peak = FP32_PEAK_TFLOPS if f32 else FP64_PEAK_TFLOPS
        ach = prof["fft_flops"] / (stage_ms["fields"] / 1e3) / 1e12
        roof = {"kernel": "ce_rows/ce_cols (Philox + Box-Muller + FFT, %s)" % ("FP32" if f32 else "FP64"),
                "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "peak_source": fp32_src if f32 else fp64_src}
    out = {
        "metric": metric_name(d, args), "value": n_all / (total_ms / 1e3), "unit": "level-samples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if d["prec"] == 0 else "f64+f32-mg" if d["prec"] == 3 else "f32+f64", "data": "synthetic (Philox4x64-10 streams)",
        "config": config_block(args, d), "roofline": roof, "e2e": e2e, "gpu_launches": launches // 1,
        "clocks": clk, "time_to_eps_s": total_ms / args.steps / 1e3, "N_per_level": est["N"],
        "q_hat": est["q_hat"], "var_hat": est["var_hat"], "alpha": est["alpha"], "bias_estimate": est["bias"],
        "bias_flag": est["bias_flag"],
        "stage_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
        "iters_per_cell_solve": prof["cell_iters"] / max(prof["cells"], 1.0),
        "autotune": [{"m": d["m0"] << l, "threads": t["threads"], "warp": t["warp"], "cluster": t["cluster"],
                      "cap_blocks_per_sm": t["cap_blocks_per_sm"], "gamma": t["gamma"], "nu": t["nu"]}
                     for l, t in enumerate(tune)],
    }
    if not args.no_cpu_baseline:
        cores = min(host_cores(), 16)
        rates, _ = oracle_rates(args.workload, {}, list(range(d["L"] + 1)), args.seed, cores)
        N = est["N"]
        t_cpu = sum(n / rates[lvl] for lvl, n in enumerate(N))
        out["cpu_baseline"] = {
            "value": sum(N) / t_cpu, "unit": "level-samples/s", "cores": cores, "kind": "oracle",
            "sample": "oracle on %d spawned processes, %s samples of levels 0..%d timed; time-to-eps "
                      "extrapolated with the GPU run's N_l (%.1f s)" % (
                          cores, [CPU_SAMPLE.get(lv, 1) for lv in range(d["L"] + 1)], d["L"], t_cpu)}
    print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark of the MLMC level batch on GB300.

One step = one complete adaptive MLMC estimate to RMSE eps (pilot batches on
every level, then top-ups to the cost-optimal N_l until the sampling error is
<= eps^2/2): one pass of every stage of the hot path over every level --
Philox normals, circulant-embedding fields, TPFA assembly, the multigrid-
preconditioned CG, the outflow QoI, the level reduction and the estimator.

Default workload: two layers, piecewise log-normal fields (sigma^2 = 1,
lambda = 0.3, 2-norm), levels m = 16 .. 512, eps = 5e-4, in the mixed form
with Coarse Grid Variates (FP32 fields and multigrid inside FP64 refinement;
FP64 residual, QoI and sums).  The same estimate in plain FP64 batched MLMC
(no CGV) at the same eps and level set is timed in the same run, and the
line reports both times-to-eps and their ratio.

value = level samples solved per second by the mixed CGV arm (sum_l N_l over
all ranks / time); ms_per_step = its time-to-eps.  The timed estimates run
with the levels of each round side by side under one CUDA graph; the stage
and per-level timings of the roofline come from a separate, untimed pass
with CUDA events around every stage (levels one after another).

--impl reference times the CPU FP64 oracle on the host cores on a bounded
sample of the same workload and prints the same line with "impl": "reference".
--profile-case CASE runs one of the fixed small cases used for ncu captures;
--ncu-summary CSV summarises an ncu launch list (kernel, launches, time, share).
"""
import argparse
import collections
import csv
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "lognormal_2layer_cgv_16to512"
# Copy-bandwidth fallback (an earlier GB300 measurement) when the measured
# peaks file is absent.
HBM_FALLBACK_GBS = 6800.0
# Samples per level of one bounded oracle sample (CPU baseline and reference arm).
CPU_SAMPLE = {0: 256, 1: 64, 2: 32, 3: 16, 4: 16, 5: 16, 6: 2}
PREC_NAMES = {0: "fp64", 1: "fp32-mg/fp64-refinement", 2: "fp32-mg-bf16-faces/fp64-refinement",
              3: "fp64-cg/fp32-mg-preconditioner"}
# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) against the
# library's algorithmic bytes of the same launches, from one-kernel captures of
# the current kernel versions (profiles/); the line's traffic scales the ratio
# to its kernel's average launch.
# Estimator cost model of every estimate (mlmc_estimate's cost_model): 2 = the
# per-sample GPU cost of each level measured by mlmc_calibrate_costs after the
# tuning (set from --cost-model in main).
COST_MODEL = 2

TRAFFIC = {
    "solve_list_kernel<1, 0> [blocks of 512 threads, workspace in global memory]": (
        292.80e9, 309.10e9,
        "ncu of bench.py --profile-case sched_block512_headline: the persistent launch of blocks of 512 as the "
        "headline estimate composes it (level 3 fine, level 4, level 5), profiles/solve_list_kernel_block512_dram.txt"),
    "solve_kernel<1, 0>": (54.23e9, 72.30e9,
                           "ncu of bench.py --profile-case mixed_m256_split: the two solve launches (m = 256 fine, "
                           "m = 128 coarse systems, blocks of 512), profiles/solve_kernel_m256_hbm.txt"),
}


# ------------------------------------------------------------- oracle side --
def _worker_init():
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"


_CE_CACHE = {}  # embedding tables of a worker process, per workload


def _oracle_worker(job):
    """Runs in a spawned process: oracle samples of one level; returns
    (level, seconds, per-sample (qf, qc, qc_cgv))."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import workloads
    from oracle import darcy
    name, overrides, level, first, n, seed = job
    model = darcy.Model.from_dict(workloads.workload(name, **overrides))
    cache = _CE_CACHE.setdefault((name, tuple(sorted(overrides.items()))), {})
    darcy.layer_fields(model, seed, level, first, model.m(level), cache)  # embedding table (once per process)
    t = time.perf_counter()
    out = []
    for i in range(first, first + n):
        r = darcy.sample(model, seed, level, i, cache)
        out.append((r["qf"], r["qc"], r["qc_cgv"]))
    return level, time.perf_counter() - t, out


def oracle_rates(name, overrides, levels, seed, cores, pool=None):
    """Per-level oracle throughput (samples/s) on `cores` spawned processes,
    the per-sample results, and the wall time of the whole sample."""
    import multiprocessing as mp
    jobs = []
    for lvl in levels:
        n = CPU_SAMPLE.get(lvl, 1)
        per = max(1, n // cores)
        for c0 in range(0, n, per):
            jobs.append((name, overrides, lvl, 10_000_000 + c0, min(per, n - c0), seed))
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(cores, initializer=_worker_init)
    rates, results = {}, {}
    t_all = time.perf_counter()
    try:
        for lvl in levels:
            lj = [j for j in jobs if j[2] == lvl]
            t = time.perf_counter()
            res = pool.map(_oracle_worker, lj)
            wall = time.perf_counter() - t
            rates[lvl] = sum(j[4] for j in lj) / wall
            results[lvl] = [x for r in res for x in r[2]]
    finally:
        if own:
            pool.close()
            pool.join()
    return rates, results, time.perf_counter() - t_all


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ clocks --
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
            d = os.path.dirname(self.path)
            if d:
                os.makedirs(d, exist_ok=True)
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


# ---------------------------------------------------------------- helpers --
def metric_name(d):
    return ("level solves/s and time-to-RMSE eps=%g: %d-layer piecewise %s%s, m=%d..%d, %s%s"
            % (d["eps"], d["n_layers"], "log-normal" if d["k_kind"] == 1 else "constant (k = exp(Z) per layer)",
               ", 3-D" if d.get("dim", 2) == 3 else "", d["m0"], d["m0"] << d["L"],
               {0: "plain FP64", 1: "mixed FP32-MG/FP64", 2: "mixed FP32-MG (BF16 faces)/FP64",
                3: "FP64 CG with FP32-MG preconditioner"}[d["prec"]], " + CGV" if d["cgv"] else ""))


def config_block(args, d, baseline):
    c = {"workload": args.workload, "m_levels": [d["m0"] << l for l in range(d["L"] + 1)],
         "eps": d["eps"], "sigma2": d["sigma2"][0], "lambda": d["lam"][0], "layers": d["n_layers"],
         "dim": d.get("dim", 2), "norm_r": d["norm_r"], "cgv": d["cgv"], "prec": PREC_NAMES[d["prec"]],
         "solver_tol": d["tol"], "seed": args.seed,
         "cost_model": ({0: "deterministic m_l^d (1 + n_coarse/2^d)", 1: "measured 64-sample pilot",
                         2: "measured per-sample GPU time of each level (mlmc_calibrate_costs, fixed for the run)"}
                        [args.cost_model] if args.impl != "reference" else
                        "measured per-sample time of each level of the oracle itself"),
         "l2": "flushed between steps (256 MB device write)", "parallelism": "replicas%d" % args.gpus,
         "graph": "each estimate round captured as one CUDA graph",
         "schedule": ("work queue: per launch shape one persistent solver launch across the levels"
                      if args.schedule else "per level: a launch chain per level, levels side by side")}
    if baseline is not None:
        c["baseline_arm"] = {"prec": PREC_NAMES[baseline["prec"]], "cgv": baseline["cgv"]}
    return c


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


def measured_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = float(json.load(open(p))["hbm_gbs"])
        return v, "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


def timed_estimates(ctx, d, seed, steps, warmup, flush, stream):
    """`warmup` untimed estimates, then `steps` timed ones (CUDA events on the
    context's stream, L2 flushed before each); returns (ms list, last estimate)."""
    import torch
    for _ in range(warmup):
        ctx.estimate(d["eps"], seed, n_pilot=64, cost_model=COST_MODEL)
    torch.cuda.synchronize()
    ms, est = [], None
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        est = ctx.estimate(d["eps"], seed, n_pilot=64, cost_model=COST_MODEL)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms, est


def solve_kernel_name(prec, t):
    mode = 2 if t["cluster"] else 3 if t["warp"] == 2 else 1 if t["warp"] else 0
    return "solve_kernel<%d, %d>" % (prec, mode)


def profiled_pass(ctx, d, est, seed, tune):
    """Untimed: one estimate with stage events (levels in series), then every
    level alone at the estimate's N_l with stage events.  Returns the stage
    totals per step and the per-level records."""
    ctx.profile(True)
    ctx.estimate(d["eps"], seed, n_pilot=64, cost_model=COST_MODEL)
    tot = ctx.profile_read()
    ctx.profile(False)
    per = []
    for lvl, n in enumerate(est["N"]):
        ctx.profile(True)
        s = ctx.level_batch(lvl, n, seed)
        p = ctx.profile_read()
        ctx.profile(False)
        t = tune[lvl]
        tc = t.get("coarse")
        plan = lambda x: {"threads": x["threads"], "warp": x["warp"], "cluster": x["cluster"], "nu": x["nu"],
                          "nu_coarse": x["nu_coarse"], "gamma": x["gamma"], "reliable": x["reliable"],
                          "inner_tol": x["inner_tol"], "cap_blocks_per_sm": x["cap_blocks_per_sm"]}
        per.append({"level": lvl, "m": d["m0"] << lvl, "N": n, "fields_ms": p["ms"]["fields"],
                    "solve_ms": p["ms"]["solve"] + p["ms"]["solve_coarse"], "reduce_ms": p["ms"]["reduce"],
                    "solve_fine_ms": p["ms"]["solve"], "solve_coarse_ms": p["ms"]["solve_coarse"],
                    "solve_launches": p["launches"]["solve"], "solve_coarse_launches": p["launches"]["solve_coarse"],
                    "iters_per_sample": s["iters_total"] / max(s["n"], 1),
                    "cell_iters": p["cell_iters"], "solve_bytes": p["solve_bytes"],
                    "solve_flops": p["solve_flops"], "fft_flops": p["fft_flops"], "fft_bytes": p["fft_bytes"],
                    "solve_bytes_c": p["solve_bytes_c"], "solve_flops_c": p["solve_flops_c"],
                    "solve_kernel": solve_kernel_name(d["prec"], t), "smem": t["smem"], "plan": plan(t),
                    "coarse_kernel": solve_kernel_name(d["prec"], tc) if tc else None,
                    "coarse_smem": tc["smem"] if tc else None, "coarse_plan": plan(tc) if tc else None})
    return tot, per


def roofline(d, per, peaks):
    """Roofline of the dominant kernel of the per-level pass: the solve kernel
    instantiation (one per launch plan kind) or the field passes with the
    largest summed time.  Streamed solver plans (workspace in global memory)
    are set against the copy bandwidth with the library's algorithmic bytes;
    shared-memory plans and the field passes against the measured FMA peak
    of their precision with the algorithmic flops."""
    by = collections.OrderedDict()
    for r in per:
        # the fine systems' launch (all systems when the coarse ones share it) and the
        # coarse systems' own launch, each under the kernel of its plan
        split = r["coarse_kernel"] is not None and r["solve_coarse_ms"] > 0
        parts = [(r["solve_kernel"], r["solve_fine_ms"],
                  r["solve_bytes"] - (r["solve_bytes_c"] if split else 0.0),
                  r["solve_flops"] - (r["solve_flops_c"] if split else 0.0), r["smem"], r["m"],
                  r["solve_launches"])]
        if split:
            parts.append((r["coarse_kernel"], r["solve_coarse_ms"], r["solve_bytes_c"], r["solve_flops_c"],
                          r["coarse_smem"], r["m"] // 2, r["solve_coarse_launches"]))
        for name_, ms, byt, fl, smem, msz, nl in parts:
            k = by.setdefault(name_, {"ms": 0.0, "bytes": 0.0, "flops": 0.0, "levels": [], "stream": 0,
                                      "sbytes": 0.0, "sms": 0.0, "slaunch": 0})
            k["ms"] += ms
            k["bytes"] += byt
            k["flops"] += fl
            k["levels"].append(msz)
            if not smem:  # streamed launches: their bytes and time alone make the HBM figure
                k["stream"] += ms
                k["sbytes"] += byt
                k["sms"] += ms
                k["slaunch"] += nl
        f = by.setdefault("ce_rows+ce_cols", {"ms": 0.0, "bytes": 0.0, "flops": 0.0, "levels": [], "stream": 0})
        f["ms"] += r["fields_ms"]
        f["bytes"] += r["fft_bytes"]
        f["flops"] += r["fft_flops"]
        f["levels"].append(r["m"])
    total = sum(k["ms"] for k in by.values())
    name = max(by, key=lambda n: by[n]["ms"])
    k = by[name]
    f32 = d["prec"] in (1, 2)
    shares = {n: round(v["ms"] / total, 4) for n, v in by.items()}
    if name.startswith("solve") and k["stream"] >= 0.5 * k["ms"]:
        ach = k["sbytes"] / (k["sms"] / 1e3) / 1e9
        per_launch = k["sbytes"] / max(k["slaunch"], 1)
        traffic, tsrc = None, "no counter capture of this kernel version"
        if name in TRAFFIC:
            dram, alg, tsrc = TRAFFIC[name]
            traffic = dram / alg * per_launch
        out = {"kernel": name, "systems_m": k["levels"], "bound": "hbm", "achieved": ach, "peak": peaks["hbm"],
               "unit": "GB/s", "frac": ach / peaks["hbm"], "traffic": traffic, "peak_source": peaks["hbm_src"],
               "launches": k["slaunch"], "algorithmic_bytes_per_launch": per_launch,
               "note": "achieved = algorithmic bytes of the kernel's streamed launches (cells x CG iterations x "
                       "bytes per cell-iteration of the streaming model: every pass reads its operands and "
                       "writes its results once) / their CUDA-event time; traffic = DRAM bytes per launch, the "
                       "DRAM-to-algorithmic ratio of one ncu capture scaled to the average launch (" + tsrc + ")"}
    else:
        # the field passes compute in FP32 with prec 1, 2; a shared-memory solver plan's
        # multigrid (most of its flops) in FP32 with prec 1, 2, 3
        use32 = f32 if name.startswith("ce") else d["prec"] != 0
        pk_t = peaks["fp32"] if use32 else peaks["fp64"]
        src = "measured by mlmc_fma_peak (independent FMA chains, %s) on this GPU" % ("FP32" if use32 else "FP64")
        ach = k["flops"] / (k["ms"] / 1e3) / 1e12
        out = {"kernel": name, "systems_m": k["levels"], "bound": "alu", "achieved": ach, "peak": pk_t,
               "unit": "TFLOP/s", "frac": ach / pk_t, "traffic": None, "peak_source": src}
    out["time_share"] = shares
    return out


SHAPE_NAMES = {0: "blocks of %d threads", 1: "one warp per system (blocks of %d)", 2: "clusters of %d x %d threads",
               3: "register path, one warp per system (blocks of %d)"}


def shape_name(cl):
    if cl["mode"] == 2:
        return SHAPE_NAMES[2] % (cl["cluster"], cl["threads"])
    return SHAPE_NAMES[cl["mode"]] % cl["threads"] + (", workspace in shared memory" if cl["smem"]
                                                       else ", workspace in global memory")


def roofline_classes(d, tot, peaks, m_of):
    """Roofline of the dominant kernel of the profiled estimate under the
    work-queue schedule: each launch shape's persistent solver launches (their
    summed CUDA-event time, algorithmic bytes and flops) and the field passes;
    the one with the largest time.  Streamed shapes (workspace in global
    memory) against the copy bandwidth, shared-memory shapes and the field
    passes against the measured FMA peak of their precision."""
    cand = []
    for cl in tot["classes"]:
        cand.append({"kernel": "solve_list_kernel<%d, %d>" % (d["prec"], cl["mode"]), "shape": shape_name(cl),
                     "ms": cl["ms"], "bytes": cl["bytes"], "flops": cl["flops"], "launches": cl["launches"],
                     "smem": cl["smem"], "levels": cl["levels"]})
    cand.append({"kernel": "ce_rows+ce_cols", "shape": "field passes", "ms": tot["ms"]["fields"],
                 "bytes": tot["fft_bytes"], "flops": tot["fft_flops"], "launches": tot["launches"]["fields"],
                 "smem": 1, "levels": []})
    total = sum(c["ms"] for c in cand)
    shares = {"%s [%s]" % (c["kernel"], c["shape"]): round(c["ms"] / total, 4) for c in cand}
    f32 = d["prec"] in (1, 2)

    def line(k):
        base = {"kernel": k["kernel"], "launch_shape": k["shape"], "levels": k["levels"], "launches": k["launches"]}
        if k["kernel"].startswith("solve") and not k["smem"]:
            ach = k["bytes"] / (k["ms"] / 1e3) / 1e9
            per_launch = k["bytes"] / max(k["launches"], 1)
            key = "%s [%s]" % (k["kernel"], k["shape"])
            traffic, tsrc = None, "no counter capture of this kernel version and launch shape"
            if key in TRAFFIC:
                dram, alg, tsrc = TRAFFIC[key]
                traffic = dram / alg * per_launch
            return dict(base, bound="hbm", achieved=ach, peak=peaks["hbm"], unit="GB/s", frac=ach / peaks["hbm"],
                        traffic=traffic, peak_source=peaks["hbm_src"], algorithmic_bytes_per_launch=per_launch,
                        note="achieved = algorithmic bytes of the launches (cells x CG iterations x bytes per "
                             "cell-iteration of the streaming model: every pass reads its operands and writes its "
                             "results once) / their CUDA-event time in the profiled estimate (launches in series); "
                             "traffic = DRAM bytes per launch, the DRAM-to-algorithmic ratio of one ncu capture "
                             "scaled to the average launch (" + tsrc + ")")
        use32 = f32 if k["kernel"].startswith("ce") else d["prec"] != 0
        pk_t = peaks["fp32"] if use32 else peaks["fp64"]
        src = "measured by mlmc_fma_peak (independent FMA chains, %s) on this GPU" % ("FP32" if use32 else "FP64")
        ach = k["flops"] / (k["ms"] / 1e3) / 1e12
        out = dict(base, bound="alu", achieved=ach, peak=pk_t, unit="TFLOP/s", frac=ach / pk_t, traffic=None,
                   peak_source=src,
                   note="achieved = algorithmic flops (the library's per cell-iteration count) / CUDA-event time")
        if k["kernel"].endswith(", 3>"):
            out["note"] += ("; the register path is bound by instruction issue and latency, not by FMA "
                            "throughput: per ncu it issues on about a third of the cycles (0.97e9 warp "
                            "instructions in 2.33 ms on 65535 systems) with the FP64 pipe 58.5 % busy "
                            "from the refinement and shuffle / shared-memory waits leading "
                            "(profiles/solve_kernel_register_path_m16.txt)")
        elif k["kernel"].startswith("ce"):
            out["note"] += ("; the FP32 field passes are bound by the integer multiplies of Philox4x64 "
                            "(the normals are generated inside the row pass)")
        return out

    out = line(max(cand, key=lambda c: c["ms"]))
    out["time_share"] = shares
    out["all_shapes"] = [{key: v for key, v in line(c).items() if key in (
        "kernel", "launch_shape", "levels", "bound", "achieved", "peak", "unit", "frac", "traffic")}
        for c in sorted(cand, key=lambda c: -c["ms"])]
    return out


def host_estimate_e2e(ctx, d, seed, costs=None):
    """The same adaptive estimate driven from the host through the host-buffer
    entry point mlmc_multilevel_batch_host: pilot and every top-up round copy
    the per-sample Q_f, Q_c, Q_cgv and iteration counts of all levels to host
    arrays, and the sample sizes come from those host values (same rule as
    mlmc_estimate).
    Returns (seconds, sum N_l, d2h bytes)."""
    import numpy as np
    L = d["L"]
    eps = d["eps"]
    dim = d.get("dim", 2)
    C = list(costs) if costs else []  # the estimate's costs (calibrated), else the m^d model
    for l in range(len(C), L + 1):
        nc = 0 if l == 0 else (2 ** dim if d["cgv"] else 1)
        C.append(float((d["m0"] << l) ** dim) * (1.0 + nc / 2.0 ** dim))
    ys = [np.empty(0) for _ in range(L + 1)]
    tried = [0] * (L + 1)  # samples drawn per level, converged or not
    d2h = 0
    t0 = time.perf_counter()
    want = [64] * (L + 1)
    for _ in range(11):  # the pilot and at most ten top-up rounds
        n = [max(0, want[l] - len(ys[l])) for l in range(L + 1)]
        # all levels of the round in one call (work-queue schedule, captured graph),
        # per-sample values copied to host arrays
        res = ctx.multilevel_batch_host(n, seed, first=list(tried))
        for l in range(L + 1):
            if n[l] <= 0:
                continue
            s, qf, qc, qg, it = res[l]
            tried[l] += n[l]
            d2h += n[l] * (3 * 8 + 4)
            y = qf - (qg if (d["cgv"] and l > 0) else qc)
            ys[l] = np.concatenate([ys[l], y[np.isfinite(y)]])
        V = [float(np.var(y, ddof=1)) for y in ys]
        tot = sum((v * c) ** 0.5 for v, c in zip(V, C))
        nxt = [max(len(ys[l]), int(np.ceil(2.0 / eps ** 2 * (V[l] / C[l]) ** 0.5 * tot))) for l in range(L + 1)]
        if nxt == [len(y) for y in ys]:
            break
        want = nxt
    return time.perf_counter() - t0, sum(len(y) for y in ys), d2h


# --------------------------------------------------------------- reference --
def run_reference(args, d):
    """The CPU oracle on the host cores, bounded sample per step; same metric
    and unit.  ms_per_step is the measured wall time of one bounded sample;
    the level-samples/s value uses the measured per-level rates with the
    sample sizes N_l of the oracle's own pilot variances and own per-sample
    costs, and the time-to-eps they extrapolate to is reported under its own
    key."""
    import multiprocessing as mp
    import numpy as np
    from oracle import mlmc
    cores = min(host_cores(), 16)
    levels = list(range(d["L"] + 1))
    walls, values, t_eps = [], [], []
    with mp.get_context("spawn").Pool(cores, initializer=_worker_init) as pool:
        for step in range(args.warmup + args.steps):
            rates, results, wall = oracle_rates(args.workload, {}, levels, args.seed, cores, pool)
            V = []
            for lvl in levels:
                arr = np.array(results[lvl])
                y = arr[:, 0] - (arr[:, 2] if (d["cgv"] and lvl) else arr[:, 1])
                V.append(float(np.var(y, ddof=1)) if len(y) > 1 else float(np.var(arr[:, 0])))
            # the oracle's own per-sample cost of each level (as the GPU arm uses its own)
            C = [1.0 / rates[lvl] for lvl in levels]
            N = mlmc.optimal_samples(d["eps"], V, C)
            te = sum(n / rates[lvl] for lvl, n in zip(levels, N))
            if step >= args.warmup:
                walls.append(wall)
                values.append(sum(N) / te)
                t_eps.append(te)
    value = sum(values) / len(values)
    sample = ("oracle (numpy/scipy FP64; banded Cholesky up to m = 256, sparse LU above, sparse LU in 3-D) on "
              "%d spawned processes; per step %s samples of levels %s timed (wall %.1f s)"
              % (cores, [CPU_SAMPLE.get(lv, 1) for lv in levels], levels, sum(walls) / len(walls)))
    return {"impl": "reference", "metric": metric_name(d), "value": value, "unit": "level-samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(walls) / len(walls), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (Philox4x64-10 streams)",
            "config": config_block(args, d, None),
            "time_to_eps_extrapolated_s": sum(t_eps) / len(t_eps),
            "cpu_baseline": {"value": value, "unit": "level-samples/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "level-samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# -------------------------------------------------- fixed cases for ncu ----
# Small fixed workloads for ncu captures of single kernels, each a complete
# program that exits 0 on its own (run it once without ncu first).  Launch
# plans are fixed by hand to those the autotuner picks in the benchmark;
# entries: (workload, overrides, [(level, samples, (mode, threads, cluster,
# gamma, nu), solver[, coarse launch])]) with solver None or (reliable,
# inner_tol) and the optional coarse launch (mode, threads, cluster, gamma, nu)
# giving the coarse systems a launch of their own.
PROFILE_CASES = {
    "fp64_levels": ("lognormal_2layer_16to256", {},
                    [(0, 65535, (1, 0, 0, 1, 2), None), (3, 1024, (0, 512, 0, 1, 2), None)]),
    "prec3_levels": ("lognormal_2layer_16to256", {"prec": 3},
                     [(0, 65535, (1, 0, 0, 1, 2), None), (3, 1024, (0, 512, 0, 1, 2), None)]),
    "mixed_large": ("lognormal_2layer_cgv_32to2048", {}, [(5, 8, (2, 512, 8, 1, 2), None)]),
    "mixed_small": ("lognormal_2layer_cgv_16to512", {},
                    [(0, 65535, (3, 0, 0, 1, 1), None), (1, 16384, (0, 128, 0, 1, 1), None)]),
    "mixed_small_generic": ("lognormal_2layer_cgv_16to512", {}, [(0, 65535, (1, 0, 0, 1, 1), None)]),
    "mixed_m256": ("lognormal_2layer_cgv_16to512", {}, [(4, 256, (0, 512, 0, 1, 2), (1, 1e-3))]),
    # the headline's level 4 as the autotuner runs it: the 256 x 256 systems in
    # one launch (blocks of 512, reliable updates), the 128 x 128 CGV coarse
    # systems in a launch of their own; the first solve launch is the fine one
    "mixed_m256_split": ("lognormal_2layer_cgv_16to512", {},
                         [(4, 256, (0, 512, 0, 1, 2), (1, 1e-3), (0, 512, 0, 1, 2))]),
    "fields_m16": ("lognormal_2layer_cgv_16to512", {}, [(0, 65536, None, None)]),
    "mixed_m512": ("lognormal_2layer_cgv_16to512", {}, [(5, 128, (2, 512, 4, 1, 2), None)]),
    "mixed_1024": ("lognormal_2layer_cgv_32to2048", {}, [(5, 32, (2, 512, 8, 1, 2), None)]),
    "fp64_m256": ("lognormal_2layer_16to256", {}, [(4, 512, (0, 512, 0, 1, 2), None)]),
    "fields_m512": ("lognormal_2layer_cgv_16to512", {}, [(5, 64, None, None)]),
    "mixed_3d": ("lognormal_3d_cgv_8to32", {},
                 [(1, 4096, (0, 128, 0, 1, 2), None), (2, 512, (0, 256, 0, 1, 2), None)]),
}

_P512 = {"threads": 512, "warp": 0, "cluster": 0, "cap_blocks_per_sm": 0, "gamma": 1, "nu": 2, "nu_coarse": 2,
         "inner_tol": 1e-3, "reliable": 1}

# Multilevel batches under the work-queue schedule: (workload, overrides,
# per-level plans, samples per level); a plan is (level, launch, solver,
# coarse launch or None) in the arguments of set_launch / set_solver /
# set_launch_coarse, or (level, plan dict) in the replay form of set_plan.  sched_block512: the headline's levels 2..4 with the autotuned plans
# of the headline, so that one persistent launch of blocks of 512 (global
# workspaces) solves level 2's fine systems and all of levels 3 and 4; the
# first solve_list_kernel launch is that one.
MULTI_CASES = {
    "sched_block512": ("lognormal_2layer_cgv_16to512", {},
                       [(2, (0, 512, 0, 1, 2), None, (0, 256, 0, 1, 1)), (3, (0, 512, 0, 1, 2), None, None),
                        (4, (0, 512, 0, 1, 2), (1, 1e-3), None)],
                       [0, 0, 2000, 600, 160, 0]),
    # the headline's level 5 alone in blocks of 512 (512 x 512 fine and 256 x 256
    # coarse systems, reliable updates): working sets far beyond L2, so DRAM
    # traffic follows the streaming model
    "sched_m512": ("lognormal_2layer_cgv_16to512", {},
                   [(5, (0, 512, 0, 1, 2), (1, 1e-3), (0, 512, 0, 1, 2))],
                   [0, 0, 0, 0, 0, 96]),
    # the blocks-of-512 launch of the headline estimate as one autotuned run
    # composed it (level 3's fine systems, all of level 4, level 5's fine and
    # coarse systems; full plans), at about a third of the final round's samples
    "sched_block512_headline": ("lognormal_2layer_cgv_16to512", {},
                                [(3, dict(_P512, coarse=dict(_P512, threads=256))),
                                 (4, dict(_P512, coarse=None)),
                                 (5, dict(_P512, nu=1, nu_coarse=1, coarse=dict(_P512, gamma=2, nu=1, nu_coarse=1)))],
                                [0, 0, 0, 1600, 390, 117]),
}


def run_profile_case(case):
    import torch
    import paper_1506_04694_gb300 as pk
    import workloads
    if case in MULTI_CASES:
        name, over, plans, n = MULTI_CASES[case]
        with pk.Context(workloads.workload(name, **over), stream=torch.cuda.Stream()) as ctx:
            for item in plans:
                if isinstance(item[1], dict):  # a full plan (replay form)
                    ctx.set_plan(item[0], item[1], 0)
                    if item[1].get("coarse"):
                        ctx.set_plan(item[0], item[1]["coarse"], 1)
                    continue
                level, launch, solver, coarse = item
                ctx.set_launch(level, *launch)
                if coarse is not None:
                    ctx.set_launch_coarse(level, *coarse)
                if solver is not None:
                    ctx.set_solver(level, *solver)
            ctx.set_schedule(1)
            ctx.profile(True)
            sums = ctx.multilevel_batch(n, 0, use_graph=False)
            p = ctx.profile_read()
            ctx.profile(False)
            torch.cuda.synchronize()
            print(case, "samples", [s["n"] for s in sums], "iterations", [s["iters_total"] for s in sums], flush=True)
            for cl in p["classes"]:
                print(case, "launch shape", shape_name(cl), "levels", cl["levels"], "launches", cl["launches"],
                      "ms %.4f" % cl["ms"], "cell_iterations %.6g" % cl["cell_iters"],
                      "algorithmic_solve_bytes %.6g" % cl["bytes"], flush=True)
        return
    name, over, levels = PROFILE_CASES[case]
    with pk.Context(workloads.workload(name, **over)) as ctx:
        for level, n, launch, solver, *coarse in levels:
            if launch is not None:
                ctx.set_launch(level, *launch)
            if coarse:
                ctx.set_launch_coarse(level, *coarse[0])
            if solver is not None:
                ctx.set_solver(level, *solver)
            if launch is None:  # the field passes alone
                g, _ = ctx.sample_fields(level, n, 0)
                torch.cuda.synchronize()
                print(case, "level", level, "fields of", n, "samples", tuple(g.shape), flush=True)
                continue
            ctx.profile(True)
            s = ctx.level_batch(level, n, 0)
            p = ctx.profile_read()
            ctx.profile(False)
            torch.cuda.synchronize()
            print(case, "level", level, "m", ctx.m(level), "samples", s["n"], "iterations", s["iters_total"],
                  "cell_iterations %.6g" % p["cell_iters"], "algorithmic_solve_bytes %.6g" % p["solve_bytes"],
                  flush=True)


UNITS = {"ns": 1.0, "nsecond": 1.0, "us": 1e3, "usecond": 1e3, "ms": 1e6, "msecond": 1e6,
         "s": 1e9, "second": 1e9}


def ncu_summary(path, skip=0, start_at=None, limit=0):
    """Per kernel of an ncu launch list (--metrics gpu__time_duration.sum
    --csv): launches, total device time and share.  skip leaves out the first
    launches; start_at leaves out every launch before the first kernel whose
    name contains that text; limit > 0 keeps only that many launches from
    there on."""
    rows = list(csv.reader(open(path)))
    start = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[start]
    ki, vi, ui = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Unit")
    idi = hdr.index("ID") if "ID" in hdr else None
    agg = collections.OrderedDict()
    seen = start_at is None
    for n, r in enumerate(rows[start + 1:]):
        if len(r) <= vi or not r[vi]:
            continue
        if (int(r[idi]) if idi is not None else n) < skip:
            continue
        if not seen:
            if start_at not in r[ki]:
                continue
            seen = True
        if limit and sum(a[0] for a in agg.values()) >= limit:
            break
        name = r[ki].split("(")[0].strip()
        ns = float(r[vi].replace(",", "")) * UNITS[r[ui].strip()]
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += ns
    tot = sum(a[1] for a in agg.values())
    out = ["%-48s %8s %12s %7s" % ("kernel", "launches", "total ms", "share")]
    for k, (n, ns) in sorted(agg.items(), key=lambda x: -x[1][1]):
        out.append("%-48s %8d %12.3f %6.2f%%" % (k[:48], n, ns / 1e6, 100 * ns / tot))
    out.append("%-48s %8d %12.3f" % ("total", sum(a[0] for a in agg.values()), tot / 1e6))
    return "\n".join(out)


# ------------------------------------------------------------------- main --
def compare(args):
    """--compare WORKLOAD: time-to-eps of its mixed-precision CGV form against
    plain FP64 batched MLMC without CGV at the same eps and levels; with
    --bf16-arm also BF16 multigrid faces (prec 2), with --fp64cg-arm the CGV
    form with FP64 fields and CG around an FP32 multigrid (prec 3)."""
    import torch
    import paper_1506_04694_gb300 as pk
    import workloads
    d = workloads.workload(args.compare)
    if "eps" not in d:
        raise SystemExit("workload %s has a fixed sample count per level and no RMSE target" % args.compare)
    arms = {"mixed_cgv": dict(d), "plain_fp64": dict(d, prec=0, cgv=0)}
    if args.bf16_arm:
        arms["mixed_cgv_bf16_faces"] = dict(d, prec=2)
    if args.fp64cg_arm:
        arms["fp64cg_fp32mg_cgv"] = dict(d, prec=3)
    out = {"compare": args.compare, "eps": d["eps"], "m_levels": [d["m0"] << l for l in range(d["L"] + 1)],
           "steps": args.steps, "warmup": args.warmup}
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for name, md in arms.items():
        # the default line's untimed set-up: plans per level, then (work-queue
        # schedule) launch shapes re-timed on whole estimates, then the
        # per-level costs of the final plans when the estimator uses them
        ctx = pk.Context(md, stream=stream)
        ctx.set_schedule(args.schedule)
        ctx.autotune(seed=args.seed + 12345)
        if COST_MODEL == 2:
            ctx.calibrate_costs(seed=args.seed + 777)
        if args.schedule:
            ctx.autotune_schedule(md["eps"], seed=args.seed + 4242, n_pilot=64, cost_model=COST_MODEL,
                                  reps=1 if md["prec"] == 0 else 2)
            if COST_MODEL == 2:
                ctx.calibrate_costs(seed=args.seed + 777)
        ms, est = timed_estimates(ctx, md, args.seed, args.steps, args.warmup, flush, stream)
        t = sum(ms) / len(ms) / 1e3
        out[name] = {"time_to_eps_s": t, "N": est["N"], "V": est["V"], "q_hat": est["q_hat"],
                     "bias_estimate": est["bias"], "alpha": est["alpha"], "var_hat": est["var_hat"],
                     "level_samples_per_s": sum(est["N"]) / t,
                     "iters_per_sample": [round(x["iters_total"] / max(x["n"], 1), 2) for x in est["sums"]],
                     "prec": PREC_NAMES[md["prec"]], "cgv": md["cgv"]}
        print("%s: %s" % (name, json.dumps(out[name])), file=sys.stderr, flush=True)  # progress
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
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--prec", type=int, default=None, choices=[0, 1, 2, 3],
                    help="override the workload's solver precision mode")
    ap.add_argument("--baseline-steps", type=int, default=3,
                    help="timed estimates of the plain FP64 arm (after max(3, warmup) untimed ones)")
    ap.add_argument("--no-baseline", action="store_true", help="skip the plain FP64 arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--clocks-out", default=None,
                    help="file for the raw nvidia-smi clock samples of the timed region (default: a temp file)")
    ap.add_argument("--compare", default=None,
                    help="workload name: time-to-eps of its mixed CGV form against plain FP64 (one JSON line)")
    ap.add_argument("--bf16-arm", action="store_true")
    ap.add_argument("--fp64cg-arm", action="store_true")
    ap.add_argument("--plans", default=None, metavar="FILE",
                    help="launch plans and estimator costs: replayed from FILE if it exists, else tuned and "
                         "written there")
    ap.add_argument("--cost-model", type=int, default=2, choices=[0, 1, 2],
                    help="estimator costs: 2 calibrated per-level GPU time (default), 0 the m^d model")
    ap.add_argument("--schedule", type=int, default=1, choices=[0, 1],
                    help="multilevel schedule (mlmc_set_schedule): 1 work queue per launch shape, 0 per level")
    ap.add_argument("--profile-case", default=None, choices=sorted(PROFILE_CASES) + sorted(MULTI_CASES))
    ap.add_argument("--ncu-summary", default=None, metavar="CSV")
    ap.add_argument("--skip", type=int, default=0)
    ap.add_argument("--limit", type=int, default=0)
    ap.add_argument("--from", dest="start_at", default=None)
    args = ap.parse_args()
    global COST_MODEL
    COST_MODEL = args.cost_model
    if args.ncu_summary:
        print(ncu_summary(args.ncu_summary, args.skip, args.start_at, args.limit))
        return
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    if args.compare:
        compare(args)
        return

    import workloads
    d = workloads.workload(args.workload)
    if "eps" not in d:
        ap.error("workload %s has a fixed sample count per level and no RMSE target; the benchmark times "
                 "time-to-eps" % args.workload)
    if args.prec is not None:
        d["prec"] = args.prec
    base = None
    if not args.no_baseline and (d["prec"] != 0 or d["cgv"] != 0):
        base = dict(d, prec=0, cgv=0)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, d)), flush=True)
        return

    # the CPU baseline's process pool starts before the first GPU call
    pool = None
    cores = min(host_cores(), 16)
    if rank == 0 and not args.no_cpu_baseline:
        import multiprocessing as mp
        pool = mp.get_context("spawn").Pool(cores, initializer=_worker_init)

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
    fp64_peak, _ = pk.fma_peak(local, fp64=True)
    fp32_peak, _ = pk.fma_peak(local, fp64=False, iters=100000)
    hbm, hbm_src = measured_hbm()
    peaks = {"fp64": fp64_peak, "fp32": fp32_peak, "hbm": hbm, "hbm_src": hbm_src}
    ctx = pk.Context(d, device=local, stream=stream)
    # untimed set-up: launch plan per level, then (work-queue schedule) the launch
    # shapes of the large levels re-timed on whole estimates
    # (--plans FILE: replay the plans a previous run of the same command wrote there)
    replay = None
    if args.plans and os.path.exists(args.plans):
        replay = json.load(open(args.plans))
    ctx.set_schedule(args.schedule)
    sched_tune = None
    calib = lambda c: c.calibrate_costs(seed=args.seed + 777) if COST_MODEL == 2 else None
    if replay:
        ctx.set_plans(replay["mixed"])
        tune = replay["mixed"]
        sched_tune = {"replayed_plans": args.plans}
    else:
        tune = ctx.autotune(seed=args.seed + 12345)
        if args.schedule:
            calib(ctx)
            before, after, tune = ctx.autotune_schedule(d["eps"], seed=args.seed + 4242, n_pilot=64,
                                                        cost_model=COST_MODEL)
            sched_tune = {"estimate_ms_before": before, "estimate_ms_after": after}
    if replay and replay.get("costs"):  # the costs the tuning run measured
        ctx.set_costs(replay["costs"])
        costs = replay["costs"]
    else:
        costs = calib(ctx)  # the per-sample costs of the final plans
    bctx = btune = None
    if base is not None:
        bctx = pk.Context(base, device=local, stream=stream)
        bctx.set_schedule(args.schedule)
        if replay and replay.get("plain"):
            bctx.set_plans(replay["plain"])
            btune = replay["plain"]
        else:
            btune = bctx.autotune(seed=args.seed + 12345)
            if args.schedule:
                calib(bctx)
                bb, ba, btune = bctx.autotune_schedule(base["eps"], seed=args.seed + 4242, n_pilot=64,
                                                       cost_model=COST_MODEL, reps=1)
                sched_tune = dict(sched_tune or {}, plain_fp64_arm={"estimate_ms_before": bb,
                                                                    "estimate_ms_after": ba})
    bcosts = None
    if bctx is not None:
        if replay and replay.get("plain_costs"):
            bctx.set_costs(replay["plain_costs"])
            bcosts = replay["plain_costs"]
        else:
            bcosts = calib(bctx)
    if args.plans and not replay and rank == 0:
        json.dump({"mixed": tune, "plain": btune, "costs": costs, "plain_costs": bcosts}, open(args.plans, "w"))
    seed = args.seed + 7919 * rank
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    phys = vis.split(",")[local] if vis else str(local)
    clocks = ClockSampler(phys, args.clocks_out)
    clocks.start()
    # ---- timed region: the mixed CGV arm (the line's value) ----
    for _ in range(args.warmup):
        ctx.estimate(d["eps"], seed, n_pilot=64, cost_model=COST_MODEL)
    barrier()
    torch.cuda.synchronize(dev)
    step_ms, est = timed_estimates(ctx, d, seed, args.steps, 0, flush, stream)
    torch.cuda.synchronize(dev)
    barrier()
    n_total = sum(est["N"]) * args.steps
    # ---- the plain FP64 arm at the same eps and level set ----
    base_out = None
    if bctx is not None:
        bms, best = timed_estimates(bctx, base, seed, args.baseline_steps, max(3, args.warmup), flush, stream)
        base_out = {"time_to_eps_s": sum(bms) / len(bms) / 1e3, "steps": args.baseline_steps,
                    "warmup": max(3, args.warmup), "N_per_level": best["N"], "q_hat": best["q_hat"],
                    "var_hat": best["var_hat"], "level_samples_per_s": sum(best["N"]) / (sum(bms) / len(bms) / 1e3),
                    "prec": PREC_NAMES[base["prec"]], "cgv": base["cgv"], "level_costs_s": bcosts,
                    "autotune": [{"m": base["m0"] << l, "threads": t["threads"], "warp": t["warp"],
                                  "cluster": t["cluster"], "nu": t["nu"]} for l, t in enumerate(btune)]}
    clk = clocks.stop()
    total_ms, n_all = reduce_over_ranks(sum(step_ms), n_total, dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- untimed: stage and per-level timing (CUDA events), roofline ----
    tot, per = profiled_pass(ctx, d, est, seed, tune)
    m_of = lambda l: d["m0"] << l
    roof = roofline_classes(d, tot, peaks, m_of) if tot["classes"] else roofline(d, per, peaks)
    base_stages = None
    if bctx is not None:
        btot, bper = profiled_pass(bctx, base, best, seed, btune)
        base_stages = {"stage_ms_per_step": btot["ms"],
                       "per_level": [{k: r[k] for k in ("m", "N", "fields_ms", "solve_ms", "iters_per_sample",
                                                        "solve_kernel")} for r in bper],
                       "roofline": (roofline_classes(base, btot, peaks, m_of) if btot["classes"]
                                    else roofline(base, bper, peaks))}
        base_out.update(base_stages)

    # ---- end to end through the host-buffer entry point ----
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize(dev)
        te, n_e2e, d2h = host_estimate_e2e(ctx, d, seed, costs)
        e2e = {"value": n_e2e / te, "unit": "level-samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h,
               "seconds": te,
               "note": "the same adaptive estimate driven from the host through mlmc_multilevel_batch_host: "
                       "per-sample Q_f, Q_c, Q_cgv and iterations of the pilot and every top-up (all levels of a "
                       "round in one call) copied to host arrays inside the timed region, sample sizes from those "
                       "host values; the only inputs are (seed, model) passed by value"}

    # kernel launches of one estimate (the same kernels run inside the graphs of
    # the timed steps), times the timed steps
    ctx.profile(True)
    ctx.estimate(d["eps"], seed, n_pilot=64, cost_model=COST_MODEL)
    launches = int(sum(ctx.profile_read()["launches"].values())) * args.steps
    ctx.profile(False)
    t_mix = total_ms / args.steps / 1e3
    out = {
        "metric": metric_name(d), "value": n_all / (total_ms / 1e3), "unit": "level-samples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if d["prec"] == 0 else "f64+f32-mg" if d["prec"] == 3 else "f32+f64",
        "data": "synthetic (Philox4x64-10 streams)", "config": config_block(args, d, base),
        "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
        "time_to_eps_s": t_mix,
        "time_to_eps": {"this_arm_s": t_mix, "plain_fp64_s": base_out["time_to_eps_s"] if base_out else None,
                        "speedup_vs_plain_fp64": (base_out["time_to_eps_s"] / t_mix) if base_out else None},
        "N_per_level": est["N"], "V_per_level": est["V"], "q_hat": est["q_hat"], "var_hat": est["var_hat"],
        "alpha": est["alpha"], "bias_estimate": est["bias"], "bias_flag": est["bias_flag"],
        "stage_ms_per_step_serial": tot["ms"],
        "schedule_tuning": sched_tune,
        "solve_launch_shapes": [{"kernel": "solve_list_kernel<%d, %d>" % (d["prec"], cl["mode"]),
                                 "shape": shape_name(cl), "levels": cl["levels"], "launches": cl["launches"],
                                 "ms_per_step": round(cl["ms"], 3),
                                 "alg_gbs": round(cl["bytes"] / max(cl["ms"], 1e-9) / 1e6, 1),
                                 "tflops": round(cl["flops"] / max(cl["ms"], 1e-9) / 1e9, 3)}
                                for cl in tot["classes"]],
        "per_level": [dict({k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()
                            if k not in ("cell_iters", "solve_flops", "fft_flops", "fft_bytes", "solve_bytes",
                                         "solve_bytes_c", "solve_flops_c")},
                           solve_alg_gbs=round(r["solve_bytes"] / max(r["solve_ms"], 1e-9) / 1e6, 1),
                           solve_tflops=round(r["solve_flops"] / max(r["solve_ms"], 1e-9) / 1e9, 3),
                           fields_alg_gbs=round(r["fft_bytes"] / max(r["fields_ms"], 1e-9) / 1e6, 1))
                      for r in per],
        "peaks": {"fp64_tflops": fp64_peak, "fp32_tflops": fp32_peak, "hbm_gbs": hbm},
        "plain_fp64_arm": base_out,
        "level_costs_s": costs,
    }
    if pool is not None:
        levels = list(range(d["L"] + 1))
        rates, _, wall = oracle_rates(args.workload, {}, levels, args.seed, cores, pool)
        pool.close()
        pool.join()
        N = est["N"]
        t_cpu = sum(n / rates[lvl] for lvl, n in enumerate(N))
        out["cpu_baseline"] = {
            "value": sum(N) / t_cpu, "unit": "level-samples/s", "cores": cores, "kind": "oracle",
            "sample": "oracle on %d spawned processes, %s samples of levels 0..%d (wall %.1f s); time-to-eps "
                      "extrapolated with the GPU run's N_l: %.1f s" % (
                          cores, [CPU_SAMPLE.get(lv, 1) for lv in levels], d["L"], wall, t_cpu)}
    print(json.dumps(out), flush=True)
    ctx.close()
    if bctx is not None:
        bctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

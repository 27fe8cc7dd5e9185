"""Small fixed workloads for ncu captures of single kernels, each a complete
program that exits 0 on its own (run it once without ncu first):
    python -m paper_1506_04694_gb300.profile_cases <case>
Launch plans are fixed by hand to the ones the autotuner picks in the
benchmark (V-cycles with two red-black sweep pairs), so a capture shows the
kernel the benchmark times.  Cases:
  fp64_levels   two-layer log-normal model, m = 16..256, FP64: level 0
                (65535 samples, m = 16, M = 32, one warp per system) and
                level 3 (1024 samples, m = 128, M = 512, one block of 512
                threads per system)
  prec3_levels  the same with prec 3 (FP64 CG, FP32 multigrid)
  mixed_small   the CGV model with FP32 multigrid in FP64 refinement:
                level 0 (65535 samples, m = 16) and level 1 (16384, m = 32)
  mixed_large   the CGV model m = 32..2048: level 5 (8 samples, m = 1024,
                clusters of 8 blocks)
  mixed_1024    the CGV model m = 32..2048: level 5 in steady state (32
                samples, m = 1024, 32 + 128 systems on clusters of 8 blocks)
  fp64_m256     the default workload's finest level, FP64: level 4 (512
                samples, m = 256, one block of 512 threads per system)
  mixed_m256    the CGV model, level 4 (1024 samples, m = 256, blocks of 512,
                FP32 CG with reliable FP64 updates, inner_tol 1e-3)
  mixed_3d      the 3-D CGV workload (FP32 multigrid in FP64 refinement):
                level 1 (4096 samples, m = 16, eight m = 8 coarse systems
                each, blocks of 128 threads) and level 2 (512 samples,
                m = 32, blocks of 256)
"""
import sys

import torch

import paper_1506_04694_gb300 as pk
import workloads

CASES = {
    "fp64_levels": ("lognormal_2layer_16to256", {}, [(0, 65535, (1, 0, 0, 1, 2)), (3, 1024, (0, 512, 0, 1, 2))]),
    "prec3_levels": ("lognormal_2layer_16to256", {"prec": 3},
                     [(0, 65535, (1, 0, 0, 1, 2)), (3, 1024, (0, 512, 0, 1, 2))]),
    "mixed_small": ("lognormal_2layer_cgv_16to512", {}, [(0, 65535, (1, 0, 0, 1, 1)), (1, 16384, (1, 0, 0, 1, 2))]),
    "mixed_large": ("lognormal_2layer_cgv_32to2048", {}, [(5, 8, (2, 512, 8, 1, 2))]),
    "mixed_1024": ("lognormal_2layer_cgv_32to2048", {}, [(5, 32, (2, 512, 8, 1, 2))]),
    "fp64_m256": ("lognormal_2layer_16to256", {}, [(4, 512, (0, 512, 0, 1, 2))]),
    "mixed_m256": ("lognormal_2layer_cgv_16to512", {}, [(4, 1024, (0, 512, 0, 1, 2))]),
    "mixed_3d": ("lognormal_3d_cgv_8to32", {}, [(1, 4096, (0, 128, 0, 1, 2)), (2, 512, (0, 256, 0, 1, 2))]),
}


def run(case):
    name, over, levels = CASES[case]
    with pk.Context(workloads.workload(name, **over)) as ctx:
        for level, n, (mode, threads, cluster, gamma, nu) in levels:
            ctx.set_launch(level, mode, threads, cluster, gamma, nu)
            if case == "mixed_m256":
                ctx.set_solver(level, 1, 1e-3)
            s = ctx.level_batch(level, n, 0)
            torch.cuda.synchronize()
            print(case, "level", level, "m", ctx.m(level), "samples", s["n"], "iterations", s["iters_total"],
                  flush=True)


if __name__ == "__main__":
    run(sys.argv[1])

"""Writes fine_levels.json: oracle values of real samples at the fine levels
of the four-layer workload (sigma^2 = 3, lambda = 0.1, m up to 1024) and of
the lambda = 0.05 workload (m up to 2048), both with Coarse Grid Variates.

For each (workload, level) the first samples of seed 0 are computed by
oracle.darcy.sample alone: interfaces, circulant-embedding fields (Sec. 3.4),
the five-point system of Eq. 3.3 solved directly (banded Cholesky up to
m = 256, sparse LU above), the outflow Q_l, the plain coarse Q_{l-1} and the
CGV coarse average of Eq. 4.1 / 4.2.  For the finest level of each workload
it also stores the per-layer fine fields at a seeded set of cells, for
element-wise field parity at M = 2048 and 4096.

Nothing here reads the CUDA path.  Run from the repository root:
    python tests/golden/make_fine_levels.py [processes]
(about ten minutes on 8 cores; the m = 2048 samples dominate)."""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fine_levels.json")

# (workload, level, samples); sample indices 0 .. samples-1 of seed 0
CASES = [
    ("lognormal_4layer_cgv_16to1024", 4, 4),
    ("lognormal_4layer_cgv_16to1024", 5, 3),
    ("lognormal_4layer_cgv_16to1024", 6, 2),
    ("lognormal_2layer_cgv_32to2048", 0, 8),
    ("lognormal_2layer_cgv_32to2048", 3, 4),
    ("lognormal_2layer_cgv_32to2048", 5, 2),
    ("lognormal_2layer_cgv_32to2048", 6, 2),
]
FIELD_CELLS = 512  # sampled cells per layer of the stored fine fields
SEED = 0


def one(job):
    sys.path.insert(0, ROOT)
    import numpy as np
    import workloads
    from oracle import darcy
    name, level, i, want_fields = job
    model = darcy.Model.from_dict(workloads.workload(name))
    t = time.time()
    r = darcy.sample(model, SEED, level, i, {}, want_fields=want_fields)
    out = {"workload": name, "level": level, "m": model.m(level), "sample": i, "seed": SEED,
           "qf": r["qf"], "qc": r["qc"], "qc_cgv": r["qc_cgv"], "qc_each": list(r.get("qc_each", [])),
           "inflow": r["inflow"], "eta": [float(x) for x in r["eta"]], "oracle_s": time.time() - t}
    if want_fields:
        m = model.m(level)
        rng = np.random.default_rng(1000 + level)
        jj = rng.integers(0, m, FIELD_CELLS)
        ii = rng.integers(0, m, FIELD_CELLS)
        out["field_cells"] = {"j": [int(x) for x in jj], "i": [int(x) for x in ii],
                              "g": [[float(r["g"][t, a, b]) for a, b in zip(jj, ii)]
                                    for t in range(model.n_layers)]}
    return out


def main():
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else 4
    jobs = []
    for name, level, n in CASES:
        finest = level == 6
        for i in range(n):
            jobs.append((name, level, i, finest and i == 0))
    jobs.sort(key=lambda j: -j[1])  # the big ones first
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(one, jobs, chunksize=1)
    res.sort(key=lambda r: (r["workload"], r["level"], r["sample"]))
    with open(OUT, "w") as f:
        json.dump({"about": "oracle values (oracle.darcy.sample, seed 0) of the fine levels of the four-layer "
                            "and lambda = 0.05 workloads; written by make_fine_levels.py",
                   "samples": res}, f, indent=1)
    print("wrote", OUT, len(res), "samples")


if __name__ == "__main__":
    main()

"""Oracle parity at the fine levels of the four-layer workload (sigma^2 = 3,
lambda = 0.1, m up to 1024) and of the lambda = 0.05 workload (m up to
2048), on the real samples of seed 0: the CUDA path's Q_l, plain Q_{l-1} and
CGV average (Eq. 3.6, Eq. 4.1 / 4.2) against the oracle's values, which
tests/golden/make_fine_levels.py wrote with oracle/ alone (direct sparse
solves at m >= 512, circulant embedding at M = 2m).  These levels run the
cluster launch plans with staged sweeps and the FP32 embedding at
M = 2048 / 4096.

Tolerances: the mixed form (FP32 fields and multigrid, FP64 refinement to
the workloads' tol = 1e-10) within 1e-6 relative; the FP64 form at
tol = 1e-14 within 1e-10 relative (the algebraic error of Q scales with the
residual tolerance times the system's condition number, which grows as m^2
and with the permeability contrast: sigma^2 = 3 at tol = 1e-13 left 1.3e-10
at m = 512); fine fields element by element within 1e-12 sigma log2(M) / 10
(FP64: the rounding of the two length-M transforms grows with their log2 M
stages and with the field's scale sigma) and 2e-5 absolute (FP32)."""
import json
import os

import numpy as np
import pytest

import workloads
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fine_levels.json")))["samples"]
CASES = sorted({(r["workload"], r["level"]) for r in GOLDEN})


def golden(name, level):
    rows = sorted((r for r in GOLDEN if r["workload"] == name and r["level"] == level), key=lambda r: r["sample"])
    assert [r["sample"] for r in rows] == list(range(len(rows)))
    return rows


def gpu_level(pk, torch, d, level, n):
    with pk.Context(d) as ctx:
        qf = torch.empty(n, dtype=torch.float64, device="cuda")
        qc = torch.empty_like(qf)
        qg = torch.empty_like(qf)
        s = ctx.level_batch(level, n, seed=0, first=0, qf=qf, qc=qc, qc_cgv=qg)
    assert s["n"] == n and s["n_failed"] == 0
    return qf.cpu().numpy(), qc.cpu().numpy(), qg.cpu().numpy()


def rel_err(gpu, ref):
    ref = np.asarray(ref)
    return np.abs(gpu - ref) / np.maximum(np.abs(ref), 1e-300)


@pytest.mark.parametrize("name,level", CASES)
@pytest.mark.parametrize("prec", [1, 0])
def test_fine_level_q_against_oracle(name, level, prec):
    torch, pk = need_gpu()
    rows = golden(name, level)
    n = len(rows)
    d = workloads.workload(name)
    if prec == 0:
        d = dict(d, prec=0, tol=1e-14, max_it=4000)
    qf, qc, qg = gpu_level(pk, torch, d, level, n)
    m = d["m0"] << level
    tol = 1e-6 if prec else 1e-10
    ef = rel_err(qf, [r["qf"] for r in rows])
    print("%s level %d m %d prec %d: max rel err Q_f %.2e" % (name, level, m, prec, ef.max()))
    assert ef.max() <= tol, ef
    if level > 0:
        ec = rel_err(qc, [r["qc"] for r in rows])
        eg = rel_err(qg, [r["qc_cgv"] for r in rows])
        print("    Q_c %.2e  Q_cgv %.2e" % (ec.max(), eg.max()))
        assert ec.max() <= tol, ec
        assert eg.max() <= tol, eg
    else:
        assert np.all(qc == 0.0)


@pytest.mark.parametrize("name", sorted({r["workload"] for r in GOLDEN if "field_cells" in r}))
@pytest.mark.parametrize("prec", [0, 1])
def test_finest_fields_against_oracle(name, prec):
    torch, pk = need_gpu()
    r = next(r for r in GOLDEN if r["workload"] == name and "field_cells" in r)
    d = workloads.workload(name, prec=prec)
    with pk.Context(d) as ctx:
        M, lo, hi = ctx.ce_info(r["level"])
        assert M == 2 * r["m"] and lo >= -1e-13 * hi
        g, eta = ctx.sample_fields(r["level"], 1, seed=0, first=r["sample"])
        g = g[0].cpu().numpy()
        eta = eta[0].cpu().numpy()
    np.testing.assert_array_equal(eta, np.asarray(r["eta"]))  # bit-exact interfaces
    cells = r["field_cells"]
    jj, ii = np.asarray(cells["j"]), np.asarray(cells["i"])
    for t, ref in enumerate(cells["g"]):
        err = np.max(np.abs(g[t, jj, ii] - np.asarray(ref)))
        print("%s prec %d layer %d: max |dg| %.2e over %d cells" % (name, prec, t, err, len(jj)))
        bound = 1e-12 * max(1.0, d["sigma2"][0] ** 0.5) * np.log2(M) / 10 if prec == 0 else 2e-5
        assert err <= bound

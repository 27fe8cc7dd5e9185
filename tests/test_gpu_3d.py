"""GPU parity of the 3-D path (Sec. 3.4 extruded layers, the seven-point
system, 3-D circulant embedding, CGV over 8 offsets) against the 3-D oracle,
through the C ABI."""
import numpy as np
import pytest

import workloads
from oracle import darcy, darcy3, mlmc
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

RTOL64 = 1e-10
RTOL_MIX = 1e-6


def run_gpu(d, level, n, seed, first=0):
    torch, pk = need_gpu()
    with pk.Context(d) as ctx:
        qf = torch.empty(n, dtype=torch.float64, device="cuda")
        qc = torch.empty_like(qf)
        qg = torch.empty_like(qf)
        it = torch.empty(n, dtype=torch.int32, device="cuda")
        s = ctx.level_batch(level, n, seed, first=first, qf=qf, qc=qc, qc_cgv=qg, iters=it)
        return s, qf.cpu().numpy(), qc.cpu().numpy(), qg.cpu().numpy(), it.cpu().numpy()


def check(d, level, n, seed, rtol, first=0):
    model = darcy.Model.from_dict(d)
    s, qf, qc, qg, it = run_gpu(d, level, n, seed, first)
    assert s["n"] == n and s["n_failed"] == 0
    cache = {}
    for i in range(n):
        r = darcy3.sample(model, seed, level, first + i, cache)
        assert abs(qf[i] - r["qf"]) <= rtol * abs(r["qf"]), (i, qf[i], r["qf"])
        if level:
            assert abs(qc[i] - r["qc"]) <= rtol * abs(r["qc"]), (i, qc[i], r["qc"])
            if d["cgv"]:
                assert abs(qg[i] - r["qc_cgv"]) <= rtol * abs(r["qc_cgv"]), (i, qg[i], r["qc_cgv"])
    ref = mlmc.level_sums(qf, qc, qg, d["cgv"] != 0)
    for key in mlmc.SUM_KEYS:
        if d["cgv"] == 0 and key in ("s_qcg", "s_qcg2", "s_yg", "s_yg2"):
            continue
        assert abs(s[key] - ref[key]) <= 4e-16 * max(abs(ref[key]), 1e-300) + 1e-300, key
    return it


@pytest.mark.parametrize("level,n", [(0, 30), (1, 12), (2, 4)])
def test_3d_constant_layers(level, n):
    d = workloads.workload("const_2layer_8to32", dim=3, m0=4, L=2, cgv=1, tol=1e-13)
    check(d, level, n, seed=3, rtol=RTOL64)


@pytest.mark.parametrize("cgv,level,n", [(0, 0, 20), (0, 1, 8), (1, 1, 8), (1, 2, 3), (2, 1, 6)])
def test_3d_lognormal_fp64(cgv, level, n):
    d = workloads.workload("lognormal_3d_cgv_8to32", prec=0, cgv=cgv, tol=1e-12, m0=4)
    check(d, level, n, seed=4, rtol=RTOL64)


@pytest.mark.parametrize("level,n", [(0, 16), (1, 6), (2, 2)])
def test_3d_lognormal_mixed(level, n):
    d = workloads.workload("lognormal_3d_cgv_8to32", prec=1, tol=1e-10, m0=4)
    check(d, level, n, seed=5, rtol=RTOL_MIX)


def test_3d_benchmark_sizes_sampled():
    # the 3-D workload at its own sizes (m = 8, 16, 32), sampled outputs
    d = workloads.workload("lognormal_3d_cgv_8to32", tol=1e-10)
    model = darcy.Model.from_dict(d)
    s, qf, qc, qg, it = run_gpu(d, 2, 40, seed=0)
    assert s["n"] == 40 and s["n_failed"] == 0
    for i in (0, 39):
        r = darcy3.sample(model, 0, 2, i)
        assert abs(qf[i] - r["qf"]) <= RTOL_MIX * abs(r["qf"])
        assert abs(qg[i] - r["qc_cgv"]) <= RTOL_MIX * abs(r["qc_cgv"])


def test_3d_fields_match_oracle():
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_3d_cgv_8to32", prec=0, m0=4, L=1, n_layers=3, mu=[0.0, 0.5, -0.3],
                           sigma2=[1.0, 1.0, 2.0], lam=[0.3, 0.3, 0.2])
    model = darcy.Model.from_dict(d)
    with pk.Context(d) as ctx:
        g, eta = ctx.sample_fields(1, 5, seed=7, first=2)
    g = g.cpu().numpy()
    for s in range(5):
        ref = darcy3.layer_fields3(model, 7, 1, 2 + s, 8)
        assert np.max(np.abs(g[s] - ref)) < 1e-12
        assert np.array_equal(eta.cpu().numpy()[s], darcy.interfaces(model, 7, 1, 2 + s))


@pytest.mark.parametrize("m", [8, 16, 32, 64])
def test_3d_solve_k_closed_forms(m):
    # constant k: Q = k; layers stacked in x2 (parallel to the flow): the mean
    torch, pk = need_gpu()
    d = workloads.workload("const_2layer_8to32", dim=3, m0=4, L=0, tol=1e-12, max_it=1000)
    rows = np.exp(np.random.default_rng(m).standard_normal(m))
    k = torch.empty((2, m, m, m), dtype=torch.float64, device="cuda")
    k[0] = 2.5
    k[1] = torch.from_numpy(rows).cuda()[None, :, None].expand(m, m, m)
    with pk.Context(d) as ctx:
        p, q, it = ctx.solve_k(k)
    q = q.cpu().numpy()
    assert abs(q[0] - 2.5) <= 1e-9 * 2.5
    assert abs(q[1] - rows.mean()) <= 1e-9 * rows.mean()
    x = (np.arange(m) + 0.5) / m
    assert np.max(np.abs(p.cpu().numpy()[0] - (1 - x)[None, None, :])) < 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_3d_launch_modes_agree(prec):
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_3d_cgv_8to32", prec=prec, tol=1e-13 if prec == 0 else 1e-10)
    level, n = 1, 6  # m = 16 fine and eight m = 8 coarse systems per sample
    modes = [(0, 512, 0, 1, 1), (0, 128, 0, 1, 1), (2, 512, 2, 1, 1), (2, 512, 4, 1, 1), (0, 256, 0, 2, 1),
             (0, 256, 0, 1, 2), (1, 0, 0, 1, 1), (1, 0, 0, 1, 2)]
    res = []
    with pk.Context(d) as ctx:
        for mode, threads, cl, gamma, nu in modes:
            ctx.set_launch(level, mode, threads, cl, gamma, nu)
            qf = torch.empty(n, dtype=torch.float64, device="cuda")
            qg = torch.empty_like(qf)
            s = ctx.level_batch(level, n, 4, qf=qf, qc_cgv=qg)
            assert s["n"] == n and s["n_failed"] == 0, (mode, threads, cl, gamma, nu)
            res.append((qf.cpu().numpy(), qg.cpu().numpy()))
    tol = 1e-10 if prec == 0 else RTOL_MIX
    for qf, qg in res[1:]:
        np.testing.assert_allclose(qf, res[0][0], rtol=tol, atol=0)
        np.testing.assert_allclose(qg, res[0][1], rtol=tol, atol=0)


@pytest.mark.parametrize("prec", [0, 1])
def test_3d_model_problem_1(prec):
    d = workloads.workload("lognormal_3d_cgv_8to32", problem=1, prec=prec, m0=4,
                           tol=1e-12 if prec == 0 else 1e-10)
    check(d, 1, 6, seed=8, rtol=RTOL64 if prec == 0 else RTOL_MIX)


def test_3d_paper_geometry():
    d = workloads.workload("paper_3layer_const_16to128", dim=3, m0=4, L=1, cgv=1, tol=1e-13)
    check(d, 1, 10, seed=9, rtol=RTOL64)


def test_3d_estimate_parity_mode():
    torch, pk = need_gpu()
    d = workloads.workload("const_2layer_8to32", dim=3, m0=4, L=1, tol=1e-13)
    model = darcy.Model.from_dict(d)
    eps = 0.1
    ref = mlmc.estimate(model, eps, seed=12, n_pilot=16)
    with pk.Context(d) as ctx:
        est = ctx.estimate(eps, seed=12, n_pilot=16, cost_model=0)
    assert est["N"] == ref["N"]
    assert abs(est["q_hat"] - ref["q_hat"]) < 1e-10 * abs(ref["q_hat"])


def test_3d_autotune_and_multilevel():
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_3d_cgv_8to32", tol=1e-10)
    stream = torch.cuda.Stream()
    with pk.Context(d, stream=stream) as ctx:
        rep = ctx.autotune(seed=3)
        assert len(rep) == 3
        ref = [ctx.level_batch(l, n, 9) for l, n in enumerate((64, 16, 4))]
        got = ctx.multilevel_batch([64, 16, 4], 9, use_graph=True)
        for l in range(3):
            for key in ("n", "n_failed") + pk.SUM_FIELDS:
                assert got[l][key] == ref[l][key], (l, key)


def test_3d_bad_arguments():
    torch, pk = need_gpu()
    with pytest.raises(pk.MLMCError):
        pk.Context(workloads.workload("lognormal_3d_cgv_8to32", L=5))      # m = 256 > 128
    with pytest.raises(pk.MLMCError):
        pk.Context(workloads.workload("lognormal_3d_cgv_8to32", prec=2))   # 3-D takes prec 0 or 1

"""GPU parity of whole level batches (Eq. 3.6, Eq. 4.2) against the oracle,
through the C ABI: per-sample Q_f, Q_c, Q_cgv; level sums; ragged chunks;
sampled samples at the full benchmark sizes; failure reporting; the adaptive
estimator in its deterministic-cost mode."""
import math

import numpy as np
import pytest

import workloads
from oracle import darcy, mlmc
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

RTOL64 = 1e-10   # FP64 path vs direct solve
RTOL_MIX = 1e-6  # FP32-multigrid path


def run_gpu(pk, torch, d, level, n, seed, first=0):
    with pk.Context(d) as ctx:
        qf = torch.empty(n, dtype=torch.float64, device="cuda")
        qc = torch.empty_like(qf)
        qg = torch.empty_like(qf)
        it = torch.empty(n, dtype=torch.int32, device="cuda")
        s = ctx.level_batch(level, n, seed, first=first, qf=qf, qc=qc, qc_cgv=qg, iters=it)
        return s, qf.cpu().numpy(), qc.cpu().numpy(), qg.cpu().numpy(), it.cpu().numpy()


def check_against_oracle(d, level, n, seed, first, rtol, stride=1):
    torch, pk = need_gpu()
    model = darcy.Model.from_dict(d)
    s, qf, qc, qg, it = run_gpu(pk, torch, d, level, n, seed, first)
    assert s["rc"] == 0 and s["n"] == n and s["n_failed"] == 0
    cache = {}
    for i in range(0, n, stride):
        r = darcy.sample(model, seed, level, first + i, cache)
        assert abs(qf[i] - r["qf"]) <= rtol * abs(r["qf"]), (i, qf[i], r["qf"])
        if level:
            assert abs(qc[i] - r["qc"]) <= rtol * abs(r["qc"]), (i, qc[i], r["qc"])
        else:
            assert qc[i] == 0.0
        if d["cgv"] and level:
            assert abs(qg[i] - r["qc_cgv"]) <= rtol * abs(r["qc_cgv"]), (i, qg[i], r["qc_cgv"])
    # sums of the GPU's own per-sample values, compensated: within a few ulp of fsum
    ref = mlmc.level_sums(qf, qc, qg, d["cgv"] != 0)
    for key in mlmc.SUM_KEYS:
        if d["cgv"] == 0 and key in ("s_qcg", "s_qcg2", "s_yg", "s_yg2"):
            continue
        assert abs(s[key] - ref[key]) <= 4e-16 * max(abs(ref[key]), 1e-300) + 1e-300, key
    return s, qf, qc, qg, it


@pytest.mark.parametrize("level", [0, 1, 2])
def test_const_model_levels(level):
    d = workloads.workload("const_2layer_8to32", tol=1e-13)
    check_against_oracle(d, level, 300, seed=0, first=0, rtol=RTOL64)


@pytest.mark.parametrize("level,n", [(0, 40), (1, 30), (2, 9)])
def test_lognormal_fp64_levels(level, n):
    d = workloads.workload("lognormal_2layer_16to256", tol=1e-12)
    check_against_oracle(d, level, n, seed=5, first=1000 + level, rtol=RTOL64)


@pytest.mark.parametrize("cgv", [1, 2])
def test_cgv_fp64(cgv):
    d = workloads.workload("lognormal_2layer_cgv_16to512", prec=0, cgv=cgv, tol=1e-12, m0=8)
    check_against_oracle(d, 1, 25, seed=2, first=0, rtol=RTOL64)
    check_against_oracle(d, 2, 6, seed=2, first=3, rtol=RTOL64)


@pytest.mark.parametrize("level,n", [(0, 30), (1, 12), (2, 4)])
def test_cgv_mixed(level, n):
    d = workloads.workload("lognormal_2layer_cgv_16to512", tol=1e-10)
    check_against_oracle(d, level, n, seed=8, first=0, rtol=RTOL_MIX)


def test_four_layers_mixed():
    d = workloads.workload("lognormal_4layer_cgv_16to1024", tol=1e-10)
    check_against_oracle(d, 1, 8, seed=3, first=0, rtol=RTOL_MIX)


@pytest.mark.parametrize("cgv,level,n", [(0, 0, 40), (0, 1, 20), (0, 3, 6), (1, 1, 12), (1, 2, 6)])
def test_fp64_cg_fp32_multigrid(cgv, level, n):
    # prec 3: FP64 fields, operator and CG with an FP32 multigrid
    # preconditioner reach the FP64 path's agreement with the oracle
    d = workloads.workload("lognormal_2layer_cgv_16to512", prec=3, cgv=cgv, tol=1e-12)
    _, qf3, qc3, _, it3 = check_against_oracle(d, level, n, seed=6, first=0, rtol=RTOL64)
    torch, pk = need_gpu()
    _, qf0, qc0, _, it0 = run_gpu(pk, torch, dict(d, prec=0), level, n, 6)
    np.testing.assert_allclose(qf3, qf0, rtol=1e-10, atol=0)
    assert it3.sum() <= 1.3 * it0.sum() + n


@pytest.mark.parametrize("prec,mode,threads,cluster", [(1, 1, 0, 0), (1, 0, 256, 0), (1, 2, 512, 4), (2, 0, 512, 0)])
def test_reliable_updates(prec, mode, threads, cluster):
    # one FP32 CG with reliable FP64 residual replacement instead of
    # restarted refinement: the same FP64 stopping test, so the same Q to the
    # tolerance, in every launch mode, and no more iterations
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512", prec=prec, tol=1e-10, L=3)
    model = darcy.Model.from_dict(d)
    level, n = 3, 6
    out = {}
    for reliable, itol in ((0, 1e-5), (1, 1e-2), (1, 1e-3)):
        with pk.Context(d) as ctx:
            ctx.set_launch(level, mode, threads, cluster, 1, 2)
            ctx.set_solver(level, reliable, itol)
            qf = torch.empty(n, dtype=torch.float64, device="cuda")
            qg = torch.empty_like(qf)
            it = torch.empty(n, dtype=torch.int32, device="cuda")
            s = ctx.level_batch(level, n, 5, qf=qf, qc_cgv=qg, iters=it)
            assert s["n"] == n and s["n_failed"] == 0
            out[(reliable, itol)] = (qf.cpu().numpy(), qg.cpu().numpy(), int(it.sum()))
    for i in range(n):
        r = darcy.sample(model, 5, level, i)
        for qf, qg, _ in out.values():
            assert abs(qf[i] - r["qf"]) <= RTOL_MIX * abs(r["qf"])
            assert abs(qg[i] - r["qc_cgv"]) <= RTOL_MIX * abs(r["qc_cgv"])
    assert min(out[(1, 1e-2)][2], out[(1, 1e-3)][2]) <= out[(0, 1e-5)][2]
    with pk.Context(d) as ctx:
        with pytest.raises(pk.MLMCError):
            ctx.set_solver(level, 1, 0.0)


@pytest.mark.parametrize("level,n", [(0, 20), (1, 8), (2, 4)])
def test_bf16_faces_in_multigrid(level, n):
    # prec 2: BF16 faces only inside the multigrid preconditioner; the FP64
    # refinement still solves the FP32-face operator to tol, so Q agrees with
    # the oracle as closely as with FP32 faces, at a few more iterations
    d = workloads.workload("lognormal_4layer_cgv_16to1024", tol=1e-10, prec=2)
    _, qf2, _, qg2, it2 = check_against_oracle(d, level, n, seed=3, first=0, rtol=RTOL_MIX)
    torch, pk = need_gpu()
    _, qf1, _, qg1, it1 = run_gpu(pk, torch, dict(d, prec=1), level, n, 3)
    np.testing.assert_allclose(qf2, qf1, rtol=1e-8, atol=0)
    np.testing.assert_allclose(qg2, qg1, rtol=1e-8, atol=0)
    assert it2.sum() <= 1.5 * it1.sum() + n


@pytest.mark.parametrize("tol,rtol,prec", [(1e-13, RTOL64, 0), (1e-10, 1e-7, 0), (1e-13, RTOL64, 3)])
def test_full_size_sampled_fp64(tol, rtol, prec):
    # the benchmark's finest level (m = 256, M = 1024) in the launch the
    # benchmark uses (a large batch); sampled outputs checked one by one.
    # With the paper's stopping rule (||r||/||r0|| < 1e-10) the algebraic error
    # of Q is ~1e-8; with 1e-13 the FP64 path agrees with the direct solve to
    # 1e-10.
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_16to256", tol=tol, prec=prec)
    model = darcy.Model.from_dict(d)
    n = 400
    s, qf, qc, qg, it = run_gpu(pk, torch, d, 4, n, seed=0)
    assert s["n"] == n and s["n_failed"] == 0
    cache = {}
    for i in (0, 137, 399):
        r = darcy.sample(model, 0, 4, i, cache)
        assert abs(qf[i] - r["qf"]) <= rtol * abs(r["qf"])
        assert abs(qc[i] - r["qc"]) <= rtol * abs(r["qc"])


def test_full_size_sampled_mixed_cgv():
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512")
    model = darcy.Model.from_dict(d)
    n = 64
    s, qf, qc, qg, it = run_gpu(pk, torch, d, 5, n, seed=0)
    assert s["n"] == n and s["n_failed"] == 0
    cache = {}
    for i in (0, 63):
        r = darcy.sample(model, 0, 5, i, cache)
        assert abs(qf[i] - r["qf"]) <= RTOL_MIX * abs(r["qf"])
        assert abs(qg[i] - r["qc_cgv"]) <= RTOL_MIX * abs(r["qc_cgv"])


def test_ragged_chunks_and_ranges():
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_16to256", tol=1e-12)
    s_all, qf_all, *_ = run_gpu(pk, torch, d, 1, 333, seed=7)
    s_a, qf_a, *_ = run_gpu(pk, torch, d, 1, 100, seed=7)
    s_b, qf_b, *_ = run_gpu(pk, torch, d, 1, 233, seed=7, first=100)
    assert np.array_equal(np.concatenate([qf_a, qf_b]), qf_all)
    assert s_all["n"] == 333


def test_empty_batch():
    torch, pk = need_gpu()
    with pk.Context(workloads.workload("const_2layer_8to32")) as ctx:
        s = ctx.level_batch(1, 0, 0)
        assert s["n"] == 0 and s["rc"] == 0


def test_failures_reported_not_summed():
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_16to256", max_it=1, tol=1e-14)
    s, qf, qc, qg, it = run_gpu(pk, torch, d, 2, 10, seed=0)
    assert s["rc"] == 1 and s["n_failed"] == 10 and s["n"] == 0
    assert np.all(np.isnan(qf))


def test_bad_arguments_rejected():
    torch, pk = need_gpu()
    with pytest.raises(pk.MLMCError):
        pk.Context(workloads.workload("const_2layer_8to32", m0=12))
    with pytest.raises(pk.MLMCError):
        pk.Context(workloads.workload("paper_3layer_const_16to128", n_layers=2))
    with pytest.raises(pk.MLMCError):
        pk.Context(workloads.workload("lognormal_2layer_16to256", problem=5))
    with pk.Context(workloads.workload("const_2layer_8to32")) as ctx:
        with pytest.raises(pk.MLMCError):
            ctx.level_batch(5, 10, 0)


def test_estimate_parity_mode():
    # deterministic cost model: the GPU and the oracle choose the same N_l
    torch, pk = need_gpu()
    d = workloads.workload("const_2layer_8to32", L=2, tol=1e-13)
    model = darcy.Model.from_dict(d)
    eps = 0.08
    ref = mlmc.estimate(model, eps, seed=11, n_pilot=32)
    with pk.Context(d) as ctx:
        est = ctx.estimate(eps, seed=11, n_pilot=32, cost_model=0)
    assert est["N"] == ref["N"]
    assert abs(est["q_hat"] - ref["q_hat"]) < 1e-10 * abs(ref["q_hat"])
    assert est["var_hat"] <= eps * eps / 2 * (1 + 1e-9)
    # the reported weak rate and finest-level bias follow from the same means
    assert abs(est["alpha"] - ref["alpha"]) < 1e-8 and abs(est["bias"] - ref["bias"]) < 1e-8 * ref["bias"] + 1e-14
    assert est["bias_flag"] == ref["bias_flag"]


def test_multilevel_batch_matches_level_batches():
    # all levels queued in one call (with and without a CUDA graph) give the
    # level sums of separate level batches exactly
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512", L=3)
    n = [300, 80, 20, 6]
    first = [5, 0, 11, 2]
    stream = torch.cuda.Stream()
    with pk.Context(d, stream=stream) as ctx:
        ref = [ctx.level_batch(l, n[l], 9, first=first[l]) for l in range(4)]
        for use_graph in (False, True, True):  # the third call relaunches the kept graph
            got = ctx.multilevel_batch(n, 9, first=first, use_graph=use_graph)
            for l in range(4):
                for key in ("n", "n_failed", "iters_total") + pk.SUM_FIELDS:
                    assert got[l][key] == ref[l][key], (use_graph, l, key)


def test_autotune_keeps_parity():
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_16to256", L=2, tol=1e-12)
    model = darcy.Model.from_dict(d)
    with pk.Context(d) as ctx:
        rep = ctx.autotune(seed=1)
        assert len(rep) == 3 and all(r["candidates"] >= 1 and r["threads"] > 0 for r in rep)
        assert all(r["ms_per_sample_best"] <= r["ms_per_sample_default"] * 1.0001 for r in rep)
        qf = torch.empty(6, dtype=torch.float64, device="cuda")
        qc = torch.empty_like(qf)
        ctx.level_batch(2, 6, 3, qf=qf, qc=qc)
    qf, qc = qf.cpu().numpy(), qc.cpu().numpy()
    for i in range(6):
        r = darcy.sample(model, 3, 2, i)
        assert abs(qf[i] - r["qf"]) <= RTOL64 * abs(r["qf"])
        assert abs(qc[i] - r["qc"]) <= RTOL64 * abs(r["qc"])


def test_autotune_mixed_keeps_parity():
    # the mixed-precision knobs (FP32 inner tolerance among them) change the
    # iteration path, not the FP64 stopping test
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512", L=3, tol=1e-12)
    model = darcy.Model.from_dict(d)
    with pk.Context(d) as ctx:
        rep = ctx.autotune(seed=2)
        assert len(rep) == 4
        # restarted refinement: inner tolerance 1e-4..1e-6; reliable updates: residual drop 1e-2 or 1e-3
        assert all(r["inner_tol"] in ((1e-2, 1e-3) if r["reliable"] else (1e-4, 1e-5, 1e-6)) for r in rep)
        qf = torch.empty(5, dtype=torch.float64, device="cuda")
        qc = torch.empty_like(qf)
        qg = torch.empty_like(qf)
        ctx.level_batch(3, 5, 4, qf=qf, qc=qc, qc_cgv=qg)
    qf, qg = qf.cpu().numpy(), qg.cpu().numpy()
    for i in range(5):
        r = darcy.sample(model, 4, 3, i)
        assert abs(qf[i] - r["qf"]) <= RTOL_MIX * abs(r["qf"])
        assert abs(qg[i] - r["qc_cgv"]) <= RTOL_MIX * abs(r["qc_cgv"])


def test_checkpoint_resume_bit_identical(tmp_path):
    # an estimate interrupted after its first top-up round, checkpointed and
    # resumed in a fresh context, ends exactly where an uninterrupted one does
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_16to256", L=2)
    eps = 4e-3
    with pk.Context(d) as ctx:
        full = ctx.estimate(eps, seed=21, n_pilot=32, max_rounds=10)
    path = str(tmp_path / "est.ckpt")
    with pk.Context(d) as ctx:
        part = ctx.estimate(eps, seed=21, n_pilot=32, max_rounds=1)
        ctx.checkpoint(path)
    assert part["rounds"] == 1 and full["rounds"] >= 1
    with pk.Context(d) as ctx:
        ctx.resume(path)
        rest = ctx.estimate(eps, seed=21, n_pilot=32, max_rounds=10)
    assert rest["N"] == full["N"] and rest["rounds"] == full["rounds"]
    assert rest["q_hat"] == full["q_hat"] and rest["var_hat"] == full["var_hat"]
    # a checkpoint of another model is refused: another grid, and the same
    # grid with another variance or correlation length (merging those level
    # sums would bias the estimate without any error)
    for other in (dict(d, m0=8), dict(d, sigma2=[1.5, 1.5]), dict(d, lam=[0.2, 0.2])):
        with pk.Context(other) as ctx:
            with pytest.raises(pk.MLMCError, match="differs"):
                ctx.resume(path)


def test_nan_permeability_reported_as_failure():
    # fault injection on the host side: a non-finite k makes the solve break
    # down; the system reports NaN instead of a value and no GPU fault occurs
    torch, pk = need_gpu()
    k = workloads.random_k(16, seed=3, n=4)
    k[2, 5, 7] = np.nan
    with pk.Context(workloads.workload("const_2layer_8to32")) as ctx:
        _, q, it = ctx.solve_k(torch.from_numpy(k).cuda(), want_p=False)
    q = q.cpu().numpy()
    assert np.isnan(q[2]) and np.all(np.isfinite(q[[0, 1, 3]]))


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_launch_modes_agree(prec):
    # one system per block (64..512 threads), per warp, or per thread-block
    # cluster of 2/4/8 blocks, with V- or W-cycles and one or two smoothing
    # sweep pairs: the same systems give the same Q to the solver tolerance
    # and agree with the oracle
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512", prec=prec, cgv=1, tol=1e-13, m0=16, L=4)
    model = darcy.Model.from_dict(d)
    level, n = 3, 10   # m = 128: fine 128^2 and four 64^2 coarse systems per sample
    # (the cluster plans stage the m = 128 half sweeps through shared memory)
    modes = [(0, 512, 0, 1, 1), (0, 64, 0, 1, 1), (1, 0, 0, 1, 1), (2, 512, 2, 1, 1), (2, 512, 4, 1, 1),
             (2, 512, 8, 1, 1), (0, 256, 0, 2, 1), (1, 0, 0, 2, 1), (2, 512, 4, 2, 1), (0, 256, 0, 1, 2),
             (2, 512, 4, 1, 2), (1, 0, 0, 2, 2)]
    res = []
    with pk.Context(d) as ctx:
        for mode, threads, cl, gamma, nu in modes:
            ctx.set_launch(level, mode, threads, cl, gamma, nu)
            qf = torch.empty(n, dtype=torch.float64, device="cuda")
            qg = torch.empty_like(qf)
            s = ctx.level_batch(level, n, 4, qf=qf, qc_cgv=qg)
            assert s["n"] == n and s["n_failed"] == 0, (mode, threads, cl, gamma, nu)
            res.append((qf.cpu().numpy(), qg.cpu().numpy()))
    tol = 1e-10 if prec in (0, 3) else RTOL_MIX
    for qf, qg in res[1:]:
        np.testing.assert_allclose(qf, res[0][0], rtol=tol, atol=0)
        np.testing.assert_allclose(qg, res[0][1], rtol=tol, atol=0)
    for i in (0, n - 1):
        r = darcy.sample(model, 4, level, i)
        assert abs(res[-1][0][i] - r["qf"]) <= tol * abs(r["qf"])
        assert abs(res[-1][1][i] - r["qc_cgv"]) <= tol * abs(r["qc_cgv"])


@pytest.mark.parametrize("prec,cgv,level,n", [(0, 0, 0, 30), (0, 0, 2, 6), (0, 1, 1, 10), (1, 1, 2, 6),
                                              (2, 1, 2, 6), (3, 1, 2, 6)])
def test_model_problem_1(prec, cgv, level, n):
    # Sec. 3.4 Model Problem 1: f = 1, p = 0 on the whole boundary, Q = mean of p
    # over D* = [7/16, 9/16]^2, plain and CGV coupling, FP64 and mixed
    d = workloads.workload("lognormal_2layer_cgv_16to512", problem=1, prec=prec, cgv=cgv,
                           tol=1e-12 if prec in (0, 3) else 1e-10)
    check_against_oracle(d, level, n, seed=13, first=0, rtol=RTOL64 if prec in (0, 3) else RTOL_MIX)


def test_model_problem_1_box_and_solve_k():
    torch, pk = need_gpu()
    box = [0.05, 0.32, 0.6, 0.61]
    d = workloads.workload("const_2layer_8to32", problem=1, qoi_box=box, tol=1e-13)
    k = workloads.random_k(32, seed=77, n=3, contrast=3.0)
    with pk.Context(d) as ctx:
        p, q, _ = ctx.solve_k(torch.from_numpy(k).cuda())
    p, q = p.cpu().numpy(), q.cpu().numpy()
    for s in range(3):
        p_ref, q_ref = darcy.solve_k(k[s], problem=1, box=tuple(box))
        assert np.max(np.abs(p[s] - p_ref)) < 1e-9 * np.max(p_ref)
        assert abs(q[s] - q_ref) <= RTOL64 * abs(q_ref)
    with pytest.raises(pk.MLMCError):
        pk.Context(dict(d, qoi_box=[0.5, 0.4, 0.1, 0.2]))


@pytest.mark.parametrize("name,prec,cgv,level,n", [
    ("paper_3layer_const_16to128", 0, 0, 1, 30), ("paper_3layer_lognormal_16to128", 0, 0, 1, 10),
    ("paper_3layer_lognormal_16to128", 0, 1, 2, 4), ("paper_3layer_lognormal_16to128", 1, 1, 1, 8)])
def test_paper_geometry_levels(name, prec, cgv, level, n):
    # Sec. 3.4's three sloped layers (per-cell layer map, per-layer parameters)
    d = workloads.workload(name, prec=prec, cgv=cgv, tol=1e-12 if prec == 0 else 1e-10)
    check_against_oracle(d, level, n, seed=17, first=0, rtol=RTOL64 if prec == 0 else RTOL_MIX)

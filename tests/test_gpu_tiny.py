"""The register-resident warp solver for 16 x 16 systems (launch mode 3,
prec 1): the same systems as the generic shared-memory warp path (mode 1)
give the same Q to the solver tolerance, and both agree with the oracle
(Sec. 3.1 Eq. 3.3, Sec. 3.4 Model Problems 1 and 2), over its variants:
restarted refinement and reliable updates, V- and W-cycles, one to three
sweep pairs, fields from the circulant embedding, per-layer constants and a
caller's k array, Model Problems 1 and 2."""
import numpy as np
import pytest

import workloads
from oracle import darcy
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

RTOL_MIX = 1e-6


def level_q(pk, torch, ctx, level, n, seed, first=0):
    qf = torch.empty(n, dtype=torch.float64, device="cuda")
    qc = torch.empty_like(qf)
    qg = torch.empty_like(qf)
    it = torch.empty(n, dtype=torch.int32, device="cuda")
    s = ctx.level_batch(level, n, seed, first=first, qf=qf, qc=qc, qc_cgv=qg, iters=it)
    assert s["n"] == n and s["n_failed"] == 0
    return qf.cpu().numpy(), qc.cpu().numpy(), qg.cpu().numpy(), it.cpu().numpy()


@pytest.mark.parametrize("gamma,nu,reliable,inner_tol", [(1, 1, 0, 1e-5), (1, 2, 0, 1e-5), (2, 1, 0, 1e-5),
                                                         (2, 2, 0, 1e-6), (1, 1, 1, 1e-3), (1, 3, 1, 1e-2)])
def test_register_path_matches_generic_warp_and_oracle(gamma, nu, reliable, inner_tol):
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512", tol=1e-10)
    model = darcy.Model.from_dict(d)
    n, seed = 200, 31
    out = {}
    with pk.Context(d) as ctx:
        for mode in (1, 3):
            ctx.set_launch(0, mode, 0, 0, gamma, nu)
            ctx.set_solver(0, reliable, inner_tol)
            out[mode] = level_q(pk, torch, ctx, 0, n, seed)
    np.testing.assert_allclose(out[3][0], out[1][0], rtol=1e-8, atol=0)
    assert np.all(out[3][1] == 0.0)
    # iteration counts follow the same recursion up to rounding order
    assert abs(int(out[3][3].sum()) - int(out[1][3].sum())) <= 0.02 * out[1][3].sum() + 2
    cache = {}
    for i in (0, 1, 77, n - 1):
        r = darcy.sample(model, seed, 0, i, cache)
        assert abs(out[3][0][i] - r["qf"]) <= RTOL_MIX * abs(r["qf"]), (i, out[3][0][i], r["qf"])


def test_register_path_model_problem_1_and_constant_layers():
    torch, pk = need_gpu()
    for d in (workloads.workload("lognormal_2layer_cgv_16to512", problem=1, tol=1e-10),
              workloads.workload("const_2layer_8to32", m0=16, L=0, prec=1, tol=1e-10)):
        model = darcy.Model.from_dict(d)
        with pk.Context(d) as ctx:
            assert ctx.autotune(seed=1)[0]["candidates"] > 0
            ctx.set_launch(0, 3, 0, 0, 1, 1)
            qf, *_ = level_q(pk, torch, ctx, 0, 64, 9)
        cache = {}
        for i in (0, 13, 63):
            r = darcy.sample(model, 9, 0, i, cache)
            assert abs(qf[i] - r["qf"]) <= RTOL_MIX * abs(r["qf"]), (d["k_kind"], i, qf[i], r["qf"])


def test_register_path_solve_k_pressure():
    # a caller's k array (solve_k): pressure and outflow against the direct
    # solve.  The mixed path solves the system with its faces rounded to FP32
    # (each perturbed by at most 6e-8 relative); on these high-contrast k
    # (exp(2 z) with layer jumps) that moves the pressure by about 1e-6, the
    # outflow by less than 1e-6 relative.
    torch, pk = need_gpu()
    k = workloads.random_k(16, seed=77, n=40, contrast=4.0)
    d = workloads.workload("const_2layer_8to32", prec=1, tol=1e-10)
    with pk.Context(d) as ctx:
        p, q, it = ctx.solve_k(torch.from_numpy(k).cuda())
        p, q = p.cpu().numpy(), q.cpu().numpy()
    for s in range(40):
        p_ref, q_ref = darcy.solve_k(k[s])
        assert abs(q[s] - q_ref) <= RTOL_MIX * abs(q_ref)
        assert np.max(np.abs(p[s] - p_ref)) < 5e-6


@pytest.mark.parametrize("problem", [2, 1])
def test_coarse_systems_in_a_launch_of_their_own(problem):
    # level 1 (m = 32): the fine 32 x 32 systems in blocks of 128 threads, the
    # four 16 x 16 CGV coarse systems of each sample on the register path in a
    # launch of their own; the same Q as one launch for all systems, and the oracle's
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512", tol=1e-10, problem=problem)
    model = darcy.Model.from_dict(d)
    n, seed = 40, 5
    with pk.Context(d) as ctx:
        ctx.set_launch(1, 0, 128, 0, 1, 1)
        one = level_q(pk, torch, ctx, 1, n, seed)
        ctx.set_launch_coarse(1, 3, 0, 0, 1, 1)
        two = level_q(pk, torch, ctx, 1, n, seed)
        ctx.set_launch_coarse(1, 0, 64, 0, 1, 2)  # a block plan for the coarse launch
        blk = level_q(pk, torch, ctx, 1, n, seed)
        ctx.set_launch_coarse(1, -1)
        back = level_q(pk, torch, ctx, 1, n, seed)
    assert np.array_equal(back[0], one[0]) and np.array_equal(back[2], one[2])
    for res in (two, blk):
        np.testing.assert_array_equal(res[0], one[0])  # the fine systems' launch is unchanged
        np.testing.assert_allclose(res[1], one[1], rtol=1e-8, atol=0)
        np.testing.assert_allclose(res[2], one[2], rtol=1e-8, atol=0)
    cache = {}
    for i in (0, n - 1):
        r = darcy.sample(model, seed, 1, i, cache)
        assert abs(two[1][i] - r["qc"]) <= RTOL_MIX * abs(r["qc"])
        assert abs(two[2][i] - r["qc_cgv"]) <= RTOL_MIX * abs(r["qc_cgv"])

"""The work-queue schedule of the multilevel batch (one persistent solver
launch per launch shape across the levels, systems taken from an atomic
work counter) against the per-level schedule: the level sums of Eq. 3.6 and
Eq. 4.2 are bit-identical, with and without the CUDA graph, when levels share
a launch (warp, register and block plans, global and shared workspaces,
fine and coarse systems of different levels in one launch) and when a level
runs its own cluster launch."""
import pytest

import workloads
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def both_schedules(pk, torch, d, n, seed, first, setup=None):
    out = {}
    stream = torch.cuda.Stream()
    with pk.Context(d, stream=stream) as ctx:
        if setup:
            setup(ctx)
        for sched in (0, 1):
            ctx.set_schedule(sched)
            out[sched] = [ctx.multilevel_batch(n, seed, first=first, use_graph=g) for g in (False, True, True)]
        ref = [ctx.level_batch(l, n[l], seed, first=first[l]) for l in range(len(n)) if n[l] > 0]
    return out, ref


def assert_same(pk, out, ref, n):
    keys = ("n", "n_failed", "iters_total") + pk.SUM_FIELDS
    for sched in (0, 1):
        for call in out[sched]:
            for l in range(len(n)):
                for key in keys:
                    assert call[l][key] == out[0][0][l][key], (sched, l, key)
    k = 0
    for l in range(len(n)):
        if n[l] == 0:
            continue
        for key in keys:
            assert out[1][0][l][key] == ref[k][key], (l, key)
        assert out[1][0][l]["n"] == n[l] and out[1][0][l]["n_failed"] == 0
        k += 1


def test_shared_launches_mixed_cgv():
    # levels 0..3 (m = 16 .. 128) of the two-layer mixed CGV workload, with
    # plans that put several levels into one launch: the 16 x 16 register
    # path for level 0 and level 1's coarse systems, blocks of 256 with the
    # workspace in shared memory for the 32 x 32 systems of levels 1 (fine)
    # and 2 (coarse), blocks of 512 with global workspaces for level 2's fine
    # and all of level 3's systems
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512", L=3)
    n = [2500, 300, 60, 9]
    first = [3, 0, 17, 4]

    def setup(ctx):
        ctx.set_launch(0, 3, 0, 0, 1, 2)
        ctx.set_launch(1, 0, 256, 0, 1, 1)
        ctx.set_launch_coarse(1, 3, 0, 0, 1, 2)
        ctx.set_launch(2, 0, 512, 0, 1, 2)
        ctx.set_launch_coarse(2, 0, 256, 0, 1, 1)
        ctx.set_launch(3, 0, 512, 0, 1, 2)
        ctx.set_solver(3, 1, 1e-3)

    out, ref = both_schedules(pk, torch, d, n, 9, first, setup)
    assert_same(pk, out, ref, n)


def test_autotuned_plans_and_empty_level():
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512", L=4)
    n = [1200, 0, 40, 12, 5]
    first = [0, 0, 2, 0, 1]
    out, ref = both_schedules(pk, torch, d, n, 5, first, lambda ctx: ctx.autotune(seed=1))
    assert_same(pk, out, ref, n)


def test_fp64_plain_warp_block_and_cluster():
    # FP64 without CGV: warp plans at m = 16, 32 share a launch; level 3 runs
    # a cluster of four blocks per system, level 2 blocks of 256
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_16to256", L=3)
    n = [700, 150, 30, 6]
    first = [1, 2, 3, 4]

    def setup(ctx):
        ctx.set_launch(0, 1, 0, 0, 1, 1)
        ctx.set_launch(1, 1, 0, 0, 1, 2)
        ctx.set_launch(2, 0, 256, 0, 1, 1)
        ctx.set_launch(3, 2, 512, 4, 1, 2)

    out, ref = both_schedules(pk, torch, d, n, 13, first, setup)
    assert_same(pk, out, ref, n)


def test_estimate_same_under_both_schedules():
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512", L=2)
    res = {}
    for sched in (0, 1):
        with pk.Context(d, stream=torch.cuda.Stream()) as ctx:
            ctx.set_schedule(sched)
            res[sched] = ctx.estimate(4e-3, seed=2, n_pilot=64, cost_model=0)
    for key in ("q_hat", "var_hat", "alpha"):
        assert res[0][key] == res[1][key], key
    assert list(res[0]["N"]) == list(res[1]["N"])


def test_schedule_autotune_keeps_results():
    # the schedule-aware pass only changes launch shapes of the large levels:
    # a fixed multilevel batch gives the same level sums to the solver
    # tolerance before and after it (a whole estimate may draw N_l one apart,
    # since Eq. 3.7's ceiling sees V_l to that tolerance)
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512")
    n = [4000, 300, 60, 20, 8, 3]
    with pk.Context(d, stream=torch.cuda.Stream()) as ctx:
        ctx.autotune(seed=3)
        r0 = ctx.multilevel_batch(n, 2)
        before, after, plans = ctx.autotune_schedule(2e-3, seed=5, n_pilot=32, cost_model=0, reps=1)
        assert 0 < after <= before
        for p in plans:
            assert p["cluster"] in (0, 2, 4, 8) and p["threads"] > 0
            assert p["coarse"] is None or p["coarse"]["cluster"] in (0, 2, 4, 8)
        r1 = ctx.multilevel_batch(n, 2)
    for l in range(len(n)):
        assert r1[l]["n"] == r0[l]["n"] == n[l] and r1[l]["n_failed"] == r0[l]["n_failed"] == 0
        for key in ("s_qf", "s_qc", "s_qcg", "s_yg"):
            assert abs(r1[l][key] - r0[l][key]) <= 1e-7 * abs(r0[l]["s_qf"]), (l, key)


def test_plans_replay_in_another_context():
    # mlmc_set_launch_ex replays a tuned plan set exactly: a second context
    # given the first one's plans gives bit-identical level sums
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512", L=4)
    n = [1500, 200, 40, 12, 6]
    with pk.Context(d, stream=torch.cuda.Stream()) as a:
        plans = a.autotune(seed=8)
        ra = a.multilevel_batch(n, 3)
    with pk.Context(d, stream=torch.cuda.Stream()) as b:
        b.set_plans(plans)
        rb = b.multilevel_batch(n, 3)
    for l in range(len(n)):
        for key in ("n", "n_failed", "iters_total") + pk.SUM_FIELDS:
            assert ra[l][key] == rb[l][key], (l, key)


def test_calibrated_costs_estimate():
    # mlmc_calibrate_costs: positive per-sample costs, growing with the grid
    # from level 1 on; an estimate on them meets the sampling-error target of
    # Eq. 3.7 and is deterministic while the costs are kept
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512", L=3)
    with pk.Context(d, stream=torch.cuda.Stream()) as ctx:
        with pytest.raises(pk.MLMCError):
            ctx.estimate(4e-3, seed=2, n_pilot=32, cost_model=2)
        C = ctx.calibrate_costs(seed=1)
        assert len(C) == 4 and all(c > 0 for c in C)
        assert C[3] > C[2] > C[1]
        e1 = ctx.estimate(4e-3, seed=2, n_pilot=32, cost_model=2)
        e2 = ctx.estimate(4e-3, seed=2, n_pilot=32, cost_model=2)
    assert list(e1["N"]) == list(e2["N"]) and e1["q_hat"] == e2["q_hat"]
    assert list(e1["C"]) == C
    assert sum(v / n for v, n in zip(e1["V"], e1["N"])) <= 0.5 * 4e-3 ** 2 * (1 + 1e-12)


def test_multilevel_host_outputs_match_level_batches():
    # mlmc_multilevel_batch_host: the per-sample values of every level equal
    # those of mlmc_level_batch_host, with and without the work-queue schedule
    torch, pk = need_gpu()
    import numpy as np
    d = workloads.workload("lognormal_2layer_cgv_16to512", L=3)
    n = [500, 0, 30, 7]
    first = [4, 0, 9, 1]
    with pk.Context(d, stream=torch.cuda.Stream()) as ctx:
        ref = [ctx.level_batch_host(l, n[l], 6, first=first[l]) if n[l] else None for l in range(4)]
        for sched in (1, 0):
            ctx.set_schedule(sched)
            for use_graph in (False, True):
                got = ctx.multilevel_batch_host(n, 6, first=first, use_graph=use_graph)
                for l in range(4):
                    if not n[l]:
                        continue
                    for j in range(1, 5):
                        np.testing.assert_array_equal(got[l][j], ref[l][j])
                    for key in ("n", "n_failed", "iters_total") + pk.SUM_FIELDS:
                        assert got[l][0][key] == ref[l][0][key], (sched, use_graph, l, key)


def test_set_costs_replays_calibration():
    # mlmc_set_costs: a second context given the first one's calibrated costs
    # draws the same sample sizes
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512", L=2)
    with pk.Context(d, stream=torch.cuda.Stream()) as a:
        C = a.calibrate_costs(seed=4)
        ea = a.estimate(4e-3, seed=2, n_pilot=32, cost_model=2)
    with pk.Context(d, stream=torch.cuda.Stream()) as b:
        with pytest.raises(pk.MLMCError):
            b.set_costs([1.0, -1.0, 1.0])
        b.set_costs(C)
        eb = b.estimate(4e-3, seed=2, n_pilot=32, cost_model=2)
    assert list(ea["N"]) == list(eb["N"]) and ea["q_hat"] == eb["q_hat"]

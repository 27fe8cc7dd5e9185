"""Edge cases of the CUDA path through the C ABI: degenerate and extreme
models (one layer, eight layers, one level, 2 x 2 and 4 x 4 grids),
extreme counters (seed 2^64 - 1, sample indices near 2^40), single-sample
batches, and the largest grids checked by closed forms that hold at any size
(constant k: Q = k; horizontal layers: Q = mean row permeability)."""
import numpy as np
import pytest

import workloads
from oracle import darcy
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def gpu_batch(pk, torch, d, level, n, seed, first=0):
    with pk.Context(d) as ctx:
        qf = torch.empty(n, dtype=torch.float64, device="cuda")
        qc = torch.empty_like(qf)
        qg = torch.empty_like(qf)
        s = ctx.level_batch(level, n, seed, first=first, qf=qf, qc=qc, qc_cgv=qg)
        return s, qf.cpu().numpy(), qc.cpu().numpy(), qg.cpu().numpy()


@pytest.mark.parametrize("over,level,n,seed,first", [
    (dict(n_layers=1, mu=[0.2], sigma2=[1.0], lam=[0.3]), 1, 5, 3, 0),                  # one layer
    (dict(n_layers=8, if_lo=0.0, if_hi=1.0, mu=[0.1 * t for t in range(8)], sigma2=[1.0] * 8,
          lam=[0.2] * 8), 1, 4, 4, 0),                                                   # eight layers
    (dict(m0=2, L=1), 1, 6, 5, 0),                                                       # tiny grids
    (dict(L=0), 0, 3, 6, 0),                                                             # one level
    (dict(), 1, 1, 2 ** 64 - 1, 2 ** 40 - 3),                                            # extreme counters
])
def test_degenerate_models_match_oracle(over, level, n, seed, first):
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512", prec=0, tol=1e-12, m0=over.pop("m0", 8), **over)
    model = darcy.Model.from_dict(d)
    s, qf, qc, qg = gpu_batch(pk, torch, d, level, n, seed, first)
    assert s["n"] == n and s["n_failed"] == 0
    for i in range(n):
        r = darcy.sample(model, seed, level, first + i)
        assert abs(qf[i] - r["qf"]) <= 1e-10 * abs(r["qf"])
        if level:
            assert abs(qg[i] - r["qc_cgv"]) <= 1e-10 * abs(r["qc_cgv"])


def test_estimate_single_level():
    torch, pk = need_gpu()
    d = workloads.workload("const_2layer_8to32", L=0)
    with pk.Context(d) as ctx:
        est = ctx.estimate(0.2, seed=1, n_pilot=16)
    assert len(est["N"]) == 1 and est["N"][0] >= 16
    assert abs(est["q_hat"] - np.exp(0.5)) < 5 * np.sqrt(est["var_hat"])


@pytest.mark.parametrize("m,prec,rtol", [(1024, 0, 1e-9), (2048, 1, 1e-6), (4096, 1, 1e-6)])
def test_largest_grids_closed_forms(m, prec, rtol):
    # constant k gives Q = k; horizontal layers give the mean row permeability
    torch, pk = need_gpu()
    d = workloads.workload("const_2layer_8to32", prec=prec, tol=1e-12 if prec == 0 else 1e-10, max_it=1000)
    rows = np.exp(np.random.default_rng(m).standard_normal(m))
    k = torch.empty((2, m, m), dtype=torch.float64, device="cuda")
    k[0] = 3.5
    k[1] = torch.from_numpy(rows).cuda()[:, None].expand(m, m)
    with pk.Context(d) as ctx:
        _, q, it = ctx.solve_k(k, want_p=False)
    q = q.cpu().numpy()
    assert abs(q[0] - 3.5) <= rtol * 3.5
    assert abs(q[1] - rows.mean()) <= rtol * rows.mean()

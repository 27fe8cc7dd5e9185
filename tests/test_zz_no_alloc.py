"""The allocation-free solve entry point (mlmc_solve_k_static), for callers
that cannot allocate device memory (a host application that reserved the GPU
for its own pool, or a loop that cannot afford cudaMalloc's synchronisation).
It must give the same Q and pressure as the context-based mlmc_solve_k, on
consecutive calls that share its fixed scratch array.  Collected last on
purpose."""
import numpy as np
import pytest

import workloads
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

RTOL = 1e-10


# (16, 0): shared memory only; (32, 1), (32, 2): shared memory with the FP64
# refinement vectors in the array; 64 ... 256: whole workspaces in the array;
# 512: the documented maximum, where the array holds one or two systems.
@pytest.mark.parametrize("m,prec", [(16, 0), (32, 1), (32, 2), (64, 0), (128, 0), (256, 0), (128, 1), (128, 2),
                                    (128, 3), (512, 0), (512, 1)])
def test_static_scratch_matches_context_solve(m, prec):
    torch, pk = need_gpu()
    n = 24 if m <= 64 else 6 if m <= 256 else 3
    d = workloads.workload("const_2layer_8to32", tol=1e-12, max_it=500, prec=prec)
    with pk.Context(d) as ctx:
        for call in range(2):  # two calls in a row on the shared array
            k = torch.from_numpy(workloads.random_k(m, seed=1000 * m + call, n=n, contrast=4.0)).cuda()
            p_ref, q_ref, it_ref = ctx.solve_k(k)
            q = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            p = torch.full_like(k, float("nan"))
            it = torch.zeros(n, dtype=torch.int32, device="cuda")
            pk.solve_k_static(k, q, p=p, iters=it, tol=1e-12, max_it=500, prec=prec)
            torch.cuda.synchronize()
            q_ref, q = q_ref.cpu().numpy(), q.cpu().numpy()
            assert np.all(np.isfinite(q))
            np.testing.assert_allclose(q, q_ref, rtol=RTOL, atol=0)
            np.testing.assert_allclose(p.cpu().numpy(), p_ref.cpu().numpy(), rtol=0, atol=1e-9)
            assert np.array_equal(it.cpu().numpy(), it_ref.cpu().numpy())


def test_static_scratch_rejects_too_large():
    torch, pk = need_gpu()
    k = torch.ones((1, 1024, 1024), dtype=torch.float64, device="cuda")
    q = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pk.MLMCError, match="maximum"):
        pk.solve_k_static(k, q)

"""Pins of the oracle's Model Problem 1 (Sec. 3.4): f = 1, p = 0 on the whole
boundary, M^(1) = mean of p over the box D*.  Constant k against an
independent separable (Kronecker-sum) solve from the 1-D operator's
eigendecomposition; random k against a dense matrix built cell by cell;
box weights; symmetry and positivity."""
import numpy as np
import pytest

import workloads
from oracle import darcy, mlmc


def separable_solution(m, kval):
    """-div(k grad p) = 1 with constant k: A = A1 (x) I + I (x) A1 with the 1-D
    finite-volume operator A1 = k tridiag(-1, 2, -1) plus k on both end cells
    (half-cell Dirichlet faces 2k); solved in the eigenbasis of A1."""
    A1 = kval * (2.0 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1))
    A1[0, 0] += kval
    A1[-1, -1] += kval
    lam, V = np.linalg.eigh(A1)
    B = np.full((m, m), 1.0 / (m * m))
    Bt = V.T @ B @ V
    return V @ (Bt / (lam[:, None] + lam[None, :])) @ V.T


@pytest.mark.parametrize("m", [1, 2, 8, 32])
def test_constant_k_separable(m):
    p, _ = darcy.solve_k(np.full((m, m), 1.7), problem=1)
    np.testing.assert_allclose(p, separable_solution(m, 1.7), rtol=1e-11, atol=1e-15)


def dense_mp1(k):
    m = k.shape[0]
    A = np.zeros((m * m, m * m))
    for j in range(m):
        for i in range(m):
            r = j * m + i
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < m and 0 <= jj < m:
                    t = 2.0 / (1.0 / k[j, i] + 1.0 / k[jj, ii])
                    A[r, r] += t
                    A[r, jj * m + ii] -= t
                else:  # every boundary face is Dirichlet p = 0, half a cell away
                    A[r, r] += 2.0 * k[j, i]
    return A, np.full(m * m, 1.0 / (m * m))


@pytest.mark.parametrize("m", [2, 4, 7, 8])
def test_random_k_dense_brute_force(m):
    k = workloads.random_k(m, seed=40 + m, contrast=3.0)[0]
    A, b = dense_mp1(k)
    p_ref = np.linalg.solve(A, b).reshape(m, m)
    p, _ = darcy.solve_k(k, problem=1)
    np.testing.assert_allclose(p, p_ref, rtol=1e-11, atol=1e-15)
    assert np.all(p > 0)


def test_box_weights():
    box = (7 / 16, 9 / 16, 7 / 16, 9 / 16)
    for m in (1, 2, 8, 16, 32, 64):
        w = darcy.box_weights(m, box)
        assert abs(w.sum() - 1.0) < 1e-15
        assert abs(darcy.local_average(np.ones((m, m)), box) - 1.0) < 1e-15
    w16 = darcy.box_weights(16, box)
    assert np.count_nonzero(w16) == 4 and np.allclose(w16[7:9, 7:9], 0.25)
    w8 = darcy.box_weights(8, box)
    assert np.count_nonzero(w8) == 4 and np.allclose(w8[3:5, 3:5], 0.25)
    # an off-centre box covering parts of cells
    w = darcy.box_weights(10, (0.05, 0.32, 0.6, 0.61))
    assert abs(w.sum() - 1.0) < 1e-14 and np.count_nonzero(w) == 4


def test_symmetry_and_refinement():
    # k symmetric in x <-> y gives p symmetric; M^(1) converges as m grows
    rng = np.random.default_rng(3)
    k = np.exp(rng.standard_normal((16, 16)))
    k = 0.5 * (k + k.T)
    p, _ = darcy.solve_k(k, problem=1)
    np.testing.assert_allclose(p, p.T, rtol=1e-12)
    q = [darcy.solve_k(np.ones((m, m)), problem=1)[1] for m in (16, 32, 64)]
    assert abs(q[2] - q[1]) < abs(q[1] - q[0])


def test_level_batch_mp1():
    d = workloads.workload("lognormal_2layer_cgv_16to512", m0=8, L=1, problem=1, prec=0)
    model = darcy.Model.from_dict(d)
    assert model.problem == 1
    b = mlmc.level_batch(model, 1, 0, 6, 1)
    assert np.all(b["qf"] > 0) and np.all(b["qc"] > 0) and np.all(b["qc_cgv"] > 0)

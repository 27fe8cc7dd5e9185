"""Pins of the oracle's cell-centred TPFA assembly, direct solve and outflow
QoI (Sec. 3.1 Eq. 3.3 with harmonic faces; Sec. 3.4 Model Problem 2):
closed forms, dense brute force built cell by cell from the flux balance,
conservation."""
import numpy as np
import pytest

import workloads
from oracle import darcy


def dense_from_flux_balance(k):
    """Dense matrix and rhs from the flux balance of each cell, written face by
    face: interior faces 2/(1/k_a + 1/k_b) (series resistances of the two half
    cells), Dirichlet faces 2k (half a cell to the boundary), no-flow faces 0."""
    m = k.shape[0]
    n = m * m
    A = np.zeros((n, n))
    b = np.zeros(n)
    idx = lambda i, j: j * m + i
    for j in range(m):
        for i in range(m):
            r = idx(i, j)
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < m and 0 <= jj < m:
                    t = 2.0 / (1.0 / k[j, i] + 1.0 / k[jj, ii])
                    A[r, r] += t
                    A[r, idx(ii, jj)] -= t
                elif ii < 0:            # x1 = 0, p = 1
                    A[r, r] += 2.0 * k[j, i]
                    b[r] += 2.0 * k[j, i] * 1.0
                elif ii >= m:           # x1 = 1, p = 0
                    A[r, r] += 2.0 * k[j, i]
                # jj out of range: no-flow face, nothing
    return A, b


@pytest.mark.parametrize("m", [2, 3, 4, 5, 8])
def test_banded_solve_matches_dense_brute_force(m):
    for s in range(3):
        k = workloads.random_k(m, seed=100 + s, contrast=3.0)[0]
        A, b = dense_from_flux_balance(k)
        np.linalg.cholesky(A)  # SPD
        p_ref = np.linalg.solve(A, b).reshape(m, m)
        p, q = darcy.solve_k(k)
        np.testing.assert_allclose(p, p_ref, rtol=1e-11, atol=1e-13)
        tx, _ = darcy.transmissibilities(k)
        assert abs(q - np.sum(2.0 * k[:, -1] * p_ref[:, -1])) < 1e-11 * abs(q)


@pytest.mark.parametrize("m", [1, 2, 8, 64])
def test_constant_k_linear_pressure(m):
    k = np.full((m, m), 2.5)
    p, q = darcy.solve_k(k)
    x = (np.arange(m) + 0.5) / m
    np.testing.assert_allclose(p, np.broadcast_to(1.0 - x, (m, m)), rtol=1e-12, atol=1e-14)
    assert abs(q - 2.5) < 1e-12 * 2.5


@pytest.mark.parametrize("m", [4, 16, 64])
def test_horizontal_layers_arithmetic_mean(m):
    rng = np.random.default_rng(m)
    kr = np.exp(2 * rng.standard_normal(m))
    k = np.repeat(kr[:, None], m, axis=1)
    _, q = darcy.solve_k(k)
    assert abs(q - kr.mean()) < 1e-11 * kr.mean()


@pytest.mark.parametrize("m", [4, 16, 64])
def test_vertical_layers_harmonic_mean(m):
    rng = np.random.default_rng(m + 1)
    kc = np.exp(2 * rng.standard_normal(m))
    k = np.repeat(kc[None, :], m, axis=0)
    _, q = darcy.solve_k(k)
    ref = m / np.sum(1.0 / kc)
    assert abs(q - ref) < 1e-11 * ref


def test_single_cell():
    p, q = darcy.solve_k(np.array([[3.0]]))
    assert p[0, 0] == 0.5 and q == 3.0


@pytest.mark.parametrize("m", [8, 32])
def test_conservation_inflow_equals_outflow(m):
    k = workloads.random_k(m, seed=5, contrast=4.0)[0]
    tx, ty = darcy.transmissibilities(k)
    p = darcy.solve_direct(tx, ty, darcy.rhs(tx))
    qo, qi = darcy.outflow(tx, p), darcy.inflow(tx, p)
    assert abs(qo - qi) < 1e-10 * qo
    # symmetric faces, zero no-flow faces
    assert np.all(ty[0] == 0) and np.all(ty[-1] == 0)
    assert np.allclose(tx[:, 1:-1], 2 * k[:, :-1] * k[:, 1:] / (k[:, :-1] + k[:, 1:]))


# ---- the sparse LU path (grids above darcy.BANDED_MAX_M) ----
@pytest.mark.parametrize("m", [2, 3, 5, 8])
def test_sparse_solve_matches_dense_brute_force(m):
    for s in range(2):
        k = workloads.random_k(m, seed=300 + s, contrast=3.0)[0]
        A, b = dense_from_flux_balance(k)
        p_ref = np.linalg.solve(A, b).reshape(m, m)
        tx, ty = darcy.transmissibilities(k)
        np.testing.assert_allclose(darcy.solve_sparse(tx, ty, darcy.rhs(tx)), p_ref, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("m", [16, 64, 128])
def test_sparse_solve_matches_banded_cholesky(m):
    k = workloads.random_k(m, seed=400 + m, contrast=6.0)[0]
    tx, ty = darcy.transmissibilities(k)
    b = darcy.rhs(tx)
    p_band = scipy_banded(tx, ty, b)
    p_lu = darcy.solve_sparse(tx, ty, b)
    # two backward-stable direct solves agree to about cond(A) * eps; with
    # contrast 6 (k spans e^+-9) and m = 128 that is ~1e-11 relative
    np.testing.assert_allclose(p_lu, p_band, rtol=1e-9, atol=1e-13)
    assert abs(darcy.outflow(tx, p_lu) - darcy.outflow(tx, p_band)) < 1e-9 * darcy.outflow(tx, p_band)


def scipy_banded(tx, ty, b):
    import scipy.linalg
    m = tx.shape[0]
    return scipy.linalg.solveh_banded(darcy.banded_upper(tx, ty), b.reshape(-1)).reshape(m, m)


def test_large_grid_closed_forms_through_sparse_path():
    # m = 512 > BANDED_MAX_M: solve_k dispatches to the sparse LU
    m = 512
    assert m > darcy.BANDED_MAX_M
    p, q = darcy.solve_k(np.full((m, m), 0.7))
    x = (np.arange(m) + 0.5) / m
    # cond(A) ~ (2m/pi)^2 ~ 1e5 at m = 512: errors up to ~1e-11 are rounding
    np.testing.assert_allclose(p, np.broadcast_to(1.0 - x, (m, m)), rtol=0, atol=1e-10)
    assert abs(q - 0.7) < 1e-10
    rng = np.random.default_rng(7)
    kr = np.exp(2 * rng.standard_normal(m))
    _, q = darcy.solve_k(np.repeat(kr[:, None], m, axis=1))
    assert abs(q - kr.mean()) < 1e-10 * kr.mean()
    kc = np.exp(2 * rng.standard_normal(m))
    _, q = darcy.solve_k(np.repeat(kc[None, :], m, axis=0))
    assert abs(q - m / np.sum(1.0 / kc)) < 1e-10 * q
    # conservation on a random layered field
    k = workloads.random_k(m, seed=9, contrast=4.0)[0]
    tx, ty = darcy.transmissibilities(k)
    p = darcy.solve_direct(tx, ty, darcy.rhs(tx))
    assert abs(darcy.outflow(tx, p) - darcy.inflow(tx, p)) < 1e-10 * darcy.outflow(tx, p)

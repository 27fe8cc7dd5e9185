"""Pins of the 3-D oracle (Sec. 3.4 extruded layers, Eq. 3.3 in 3-D, Eq. 4.1
with d = 3): closed forms, a matrix built cell by cell from the flux balance,
fast diagonalisation of the constant-k Model Problem 1, the separable form of
the 1-norm embedding, field statistics and the CGV/plain identity of
piecewise constant layers."""
import numpy as np
import pytest

import workloads
from oracle import darcy, darcy3, philox


@pytest.mark.parametrize("m", [1, 2, 4, 8])
def test_constant_k_linear_pressure(m):
    k = np.full((m, m, m), 1.7)
    p, q = darcy3.solve_k3(k)
    x = (np.arange(m) + 0.5) / m
    assert abs(q - 1.7) < 1e-13
    assert np.allclose(p, np.broadcast_to(1.0 - x, (m, m, m)), atol=1e-13)


@pytest.mark.parametrize("m", [4, 8])
def test_layers_parallel_and_series(m):
    rng = np.random.default_rng(m)
    kr = np.exp(1.5 * rng.standard_normal(m))
    # layers stacked in x2 or in x3 are parallel to the flow: arithmetic mean
    for shape in ((1, m, 1), (m, 1, 1)):
        k = np.broadcast_to(kr.reshape(shape), (m, m, m)).copy()
        assert abs(darcy3.solve_k3(k)[1] - kr.mean()) < 1e-12 * kr.mean()
    # layers across x1 are in series: harmonic mean
    k = np.broadcast_to(kr[None, None, :], (m, m, m)).copy()
    hm = m / np.sum(1.0 / kr)
    assert abs(darcy3.solve_k3(k)[1] - hm) < 1e-12 * hm


def brute_force_system(k, problem):
    """Dense matrix and right-hand side from the flux balance of every cell,
    face by face (divided by the face area over the centre distance h)."""
    m = k.shape[0]
    n = m ** 3
    A = np.zeros((n, n))
    b = np.zeros(n)
    idx = lambda i, j, l: (l * m + j) * m + i
    for l in range(m):
        for j in range(m):
            for i in range(m):
                c = idx(i, j, l)
                for axis, step in ((0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1)):
                    nb = [i, j, l]
                    nb[axis] += step
                    if 0 <= nb[axis] < m:
                        kn = k[nb[2], nb[1], nb[0]]
                        t = 2.0 * k[l, j, i] * kn / (k[l, j, i] + kn)
                        A[c, c] += t
                        A[c, idx(*nb)] -= t
                    elif axis == 0 or problem == 1:  # Dirichlet face half a cell away
                        t = 2.0 * k[l, j, i]
                        A[c, c] += t
                        if axis == 0 and step == -1 and problem == 2:
                            b[c] += t * 1.0
                if problem == 1:
                    b[c] += 1.0 / (m * m)
    return A, b


@pytest.mark.parametrize("m,problem", [(3, 2), (4, 2), (3, 1), (4, 1)])
def test_dense_brute_force(m, problem):
    k = workloads.random_k(m, seed=30 + m, n=m, contrast=3.0)  # [m, m, m] of log-normal values
    tx, ty, tz = darcy3.transmissibilities3(k, problem)
    A, b = brute_force_system(k, problem)
    assert np.allclose(darcy3.matrix3(tx, ty, tz).toarray(), A, rtol=1e-14, atol=1e-14)
    assert np.allclose(darcy3.rhs3(tx, problem).reshape(-1), b, rtol=1e-14, atol=0)
    np.linalg.cholesky(A)  # symmetric positive definite
    p = np.linalg.solve(A, b).reshape(m, m, m)
    assert np.allclose(darcy3.solve_direct3(tx, ty, tz, b.reshape(m, m, m)), p, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("m", [4, 6])
def test_model_problem_1_constant_k_fast_diagonalisation(m):
    # constant k = 1: A = T x I x I + I x T x I + I x I x T with the 1-D matrix T
    # of Dirichlet ends half a cell away (diagonal 2, end cells 3, neighbours -1)
    T = 2.0 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    T[0, 0] = T[-1, -1] = 3.0
    w, V = np.linalg.eigh(T)
    b = np.full((m, m, m), 1.0 / (m * m))
    bh = np.einsum("ai,bj,ck,abc->ijk", V, V, V, b)
    ph = bh / (w[:, None, None] + w[None, :, None] + w[None, None, :])
    p_ref = np.einsum("ai,bj,ck,ijk->abc", V, V, V, ph)
    box = (0.25, 0.75, 0.25, 0.5)
    p, q = darcy3.solve_k3(np.ones((m, m, m)), problem=1, box=box)
    assert np.allclose(p, p_ref, rtol=1e-12, atol=1e-15)
    wts = darcy3.box_weights3(m, box)
    assert abs(wts.sum() - 1.0) < 1e-14
    assert abs(q - float(np.sum(wts * p_ref))) < 1e-14


@pytest.mark.parametrize("m,lam", [(4, 0.3), (8, 0.3), (8, 0.1)])
def test_one_norm_embedding_is_separable(m, lam):
    # with the 1-norm, c = sigma2 e x e x e, so Lambda = sigma2 * outer(L1, L1, L1)
    # with L1 the 1-D DFT of e = exp(-d/lam); it is non-negative at p = 2
    M = 2 * m
    a = np.arange(M)
    e = np.exp(-(np.minimum(a, M - a) / m) / lam)
    l1 = np.fft.fft(e).real
    ref = 1.3 * l1[:, None, None] * l1[None, :, None] * l1[None, None, :]
    lam3 = darcy3.ce_eigenvalues3(m, M, 1.3, lam, 1)
    assert np.allclose(lam3, ref, rtol=1e-12, atol=1e-12 * ref.max())
    assert darcy3.ce_padding3(m, 1.3, lam, 1)[0] == M


def test_field_statistics():
    # one complex draw per sample gives two independent fields with the
    # covariance of Eq. 2.3 (1-norm, lambda = 0.3): sample variance, two
    # lagged covariances and the Re/Im cross-covariance over 3000 samples
    d = workloads.workload("lognormal_3d_cgv_8to32", n_layers=2, m0=4, L=0)
    model = darcy.Model.from_dict(d)
    n = 3000
    cache = {}
    g = np.stack([darcy3.layer_fields3(model, 5, 0, s, 4, cache) for s in range(n)])  # [n, 2, 4, 4, 4]
    h, lam = 0.25, model.lam[0]
    for t in range(2):
        x = g[:, t]
        assert abs(np.mean(x[:, 1, 2, 1] ** 2) - 1.0) < 0.08
        assert abs(np.mean(x[:, 1, 2, 1] * x[:, 1, 2, 2]) - np.exp(-h / lam)) < 0.08
        assert abs(np.mean(x[:, 0, 1, 1] * x[:, 2, 2, 1]) - np.exp(-3 * h / lam)) < 0.08
    assert abs(np.mean(g[:, 0, 1, 1, 1] * g[:, 1, 1, 1, 1])) < 0.08


def test_normals_3d_index_order():
    # the complex index q = q1 + M q2 + M^2 q3 of the 3-D draw continues the
    # Philox stream of the 2-D layout
    xi3 = philox.field_normals(9, 1, 4, 0, 4, dim=3)
    flat = philox.field_normals(9, 1, 4, 0, 8).reshape(-1)
    assert np.array_equal(xi3.reshape(-1), flat[:64])
    assert xi3[1, 2, 3] == flat[3 + 4 * 2 + 16 * 1]


def test_extruded_layer_map():
    d = workloads.workload("paper_3layer_const_16to128", dim=3)
    model = darcy.Model.from_dict(d)
    ends = darcy.interfaces(model, 3, 1, 7)
    lay = darcy3.layer_map3(model, ends, 8)
    lay2 = darcy.layer_map(model, ends, 8)
    for l in range(8):
        assert np.array_equal(lay[l], lay2)


def test_cgv_of_constant_layers_equals_plain():
    # Ex. 1: constant fields per layer, so the 8 sub-samples are one and the
    # same coarse permeability: Q_cgv = Q_c
    d = workloads.workload("const_2layer_8to32", dim=3, m0=4, L=1, cgv=1)
    model = darcy.Model.from_dict(d)
    for i in range(3):
        r = darcy3.sample(model, 11, 1, i)
        assert all(abs(q - r["qc"]) < 1e-13 for q in r["qc_each"])
        assert abs(r["qc_cgv"] - r["qc"]) < 1e-13 * abs(r["qc"])


def test_sample_conserves_flux():
    d = workloads.workload("lognormal_3d_cgv_8to32", m0=4, L=1)
    model = darcy.Model.from_dict(d)
    r = darcy.sample(model, 2, 1, 5)
    assert abs(r["inflow"] - r["qf"]) < 1e-11 * abs(r["qf"])
    assert np.isfinite(r["qc_cgv"]) and len(r["qc_each"]) == 8

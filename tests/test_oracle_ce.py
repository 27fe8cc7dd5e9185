"""Pins of the oracle's layers and circulant-embedding sampler (Sec. 2, Ex. 2,
Eq. 2.3; circulant embedding of Sec. 3.4): closed-form 1-D embedding
eigenvalues, exact covariance of the linear sampling map, padding rule,
empirical moments of Philox-driven draws."""
import math

import numpy as np
import pytest

import workloads
from oracle import darcy


def exp_torus_eigs_closed_form(M, rho):
    """Eigenvalues of the symmetric circulant with first row rho^min(a, M-a):
    1 + 2 Re sum_{a=1}^{M/2-1} (rho e^{i theta})^a + rho^{M/2} cos(M theta / 2),
    the finite geometric series summed in closed form."""
    q = np.arange(M)
    z = rho * np.exp(2j * np.pi * q / M)
    n = M // 2 - 1
    geo = z * (1 - z ** n) / (1 - z)
    return 1 + 2 * geo.real + rho ** (M // 2) * np.cos(np.pi * q)


@pytest.mark.parametrize("m,M,lam,s2", [(8, 16, 0.3, 1.0), (16, 64, 0.1, 3.0), (5, 10, 0.7, 2.0)])
def test_eigs_separable_r1_closed_form(m, M, lam, s2):
    # With the 1-norm, exp(-(|x|+|y|)/lam) factorises, so the 2-D embedding
    # eigenvalues are the outer product of two 1-D closed forms.
    lam_q = darcy.ce_eigenvalues(m, M, s2, lam, norm_r=1)
    e1 = exp_torus_eigs_closed_form(M, math.exp(-1.0 / (m * lam)))
    np.testing.assert_allclose(lam_q, s2 * np.outer(e1, e1), rtol=1e-11, atol=1e-11 * lam_q.max())


def sampling_map(m, M, lam_q):
    """Columns: the m*m complex field for each unit xi_q (the sampler is linear)."""
    B = np.empty((m * m, M * M), dtype=complex)
    for q in range(M * M):
        e = np.zeros(M * M, dtype=complex)
        e[q] = 1.0
        re, im = darcy.ce_pair(lam_q, e.reshape(M, M), m)
        B[:, q] = (re + 1j * im).reshape(-1)
    return B


@pytest.mark.parametrize("norm_r,lam,s2", [(2, 0.3, 1.0), (1, 0.3, 1.0), (2, 0.1, 3.0)])
def test_exact_covariance_of_sampler(norm_r, lam, s2):
    # xi = z_re + i z_im with independent standard normals: Re y and Im y are
    # linear maps of (z_re, z_im); their exact covariances must equal Eq. 2.3
    # at the cell-centre distances, and Re y, Im y must be uncorrelated.
    m = 4
    M, lam_q = darcy.ce_padding(m, s2, lam, norm_r)
    B = sampling_map(m, M, lam_q)
    A_re = np.hstack([B.real, -B.imag])   # Re y = Re B z_re - Im B z_im
    A_im = np.hstack([B.imag, B.real])    # Im y = Im B z_re + Re B z_im
    c_re = A_re @ A_re.T
    c_im = A_im @ A_im.T
    c_x = A_re @ A_im.T
    jj, ii = np.divmod(np.arange(m * m), m)
    dx = np.abs(ii[:, None] - ii[None, :]) / m
    dy = np.abs(jj[:, None] - jj[None, :]) / m
    dist = dx + dy if norm_r == 1 else np.hypot(dx, dy)
    target = s2 * np.exp(-dist / lam)
    np.testing.assert_allclose(c_re, target, atol=1e-12)
    np.testing.assert_allclose(c_im, target, atol=1e-12)
    assert np.abs(c_x).max() < 1e-12


def test_padding_rule():
    # lambda = 0.3, 2-norm: the periodic embedding at p = 2 holds up to m = 16;
    # above, the cut-off embedding at p = 3 (up to m = 1024), where the
    # periodic one needs p = 4 (m = 32 ... 256) and p = 8 (m = 512, the
    # embed = 1 rule); short correlation lengths embed at p = 2.
    got = {m: darcy.ce_padding(m, 1.0, 0.3, 2)[0] // m for m in (8, 16, 32, 64, 128, 256, 512)}
    assert got == {8: 2, 16: 2, 32: 3, 64: 3, 128: 3, 256: 3, 512: 3}
    old = {m: darcy.ce_padding(m, 1.0, 0.3, 2, embed=1)[0] // m for m in (8, 16, 32, 64, 128, 256, 512)}
    assert old == {8: 2, 16: 2, 32: 4, 64: 4, 128: 4, 256: 4, 512: 8}
    assert darcy.ce_padding(64, 3.0, 0.1, 2)[0] == 128
    assert darcy.ce_padding(64, 1.0, 0.05, 2)[0] == 128
    assert darcy.ce_padding(64, 1.0, 0.3, 1)[0] == 128  # the 1-norm never takes the cut-off
    for m in (8, 32, 64):
        M, lam_q = darcy.ce_padding(m, 1.0, 0.3, 2)
        raw = darcy.ce_eigenvalues(m, M, 1.0, 0.3, 2, cutoff=(M == 3 * m))
        assert raw.min() >= -darcy.CE_NEG_TOL * raw.max()
        assert lam_q.min() >= 0.0


def test_cutoff_radial_function():
    # equal to Eq. 2.3 up to R0 (the largest centre distance), C^1 at R0 and
    # R1, zero from R1 = M h / 2 on
    m, M, s2, lam = 32, 96, 1.7, 0.3
    R0, R1 = darcy.cutoff_radii(m, M)
    assert R0 == pytest.approx(math.sqrt(2) * 31 / 32) and R1 == 1.5
    r = np.linspace(0, R0, 1001)
    np.testing.assert_allclose(darcy.cutoff_covariance(r, m, M, s2, lam), s2 * np.exp(-r / lam), rtol=1e-15)
    f = lambda x: float(darcy.cutoff_covariance(np.array(x), m, M, s2, lam))
    h = 1e-6
    for R in (R0, R1):
        left = 2 * f(R - h) - f(R - 2 * h)   # value at R extrapolated from either side
        right = 2 * f(R + h) - f(R + 2 * h)
        assert abs(left - right) < 1e-10                             # continuous
        slope_l = (f(R - h) - f(R - 2 * h)) / h
        slope_r = (f(R + 2 * h) - f(R + h)) / h
        assert abs(slope_l - slope_r) < 1e-4                         # continuous slope
    assert f(R1) == 0.0 and f(R1 + 0.3) == 0.0 and f(0.5 * (R0 + R1)) > 0.0
    # the torus table holds the same values at every lag of two cell centres
    c = darcy.covariance_torus(m, M, s2, lam, 2, cutoff=True)
    a = np.arange(m)
    np.testing.assert_allclose(c[:m, :m], s2 * np.exp(-np.hypot(a[None, :], a[:, None]) / m / lam), rtol=1e-15)


@pytest.mark.parametrize("m,forced", [(8, True), (32, False)])
def test_exact_covariance_of_cutoff_sampler(m, forced):
    # The cut-off embedding changes the covariance only at lags beyond the
    # grid, so the linear sampling map still reproduces Eq. 2.3 exactly at
    # every pair of cell centres (m = 8: the cut-off forced at M = 24; m = 32:
    # the embedding the padding rule picks, M = 96).
    lam, s2 = 0.3, 1.0
    if forced:
        M = 3 * m
        raw = darcy.ce_eigenvalues(m, M, s2, lam, 2, cutoff=True)
        assert raw.min() >= 0.0
        lam_q = raw
    else:
        M, lam_q = darcy.ce_padding(m, s2, lam, 2)
        assert M == 3 * m
    B = sampling_map(m, M, lam_q)
    A_re = np.hstack([B.real, -B.imag])
    A_im = np.hstack([B.imag, B.real])
    jj, ii = np.divmod(np.arange(m * m), m)
    dist = np.hypot(np.abs(ii[:, None] - ii[None, :]) / m, np.abs(jj[:, None] - jj[None, :]) / m)
    target = s2 * np.exp(-dist / lam)
    np.testing.assert_allclose(A_re @ A_re.T, target, atol=1e-12)
    np.testing.assert_allclose(A_im @ A_im.T, target, atol=1e-12)
    assert np.abs(A_re @ A_im.T).max() < 1e-12


@pytest.mark.parametrize("p_small", [2])
def test_padding_too_small_is_negative(p_small):
    raw = darcy.ce_eigenvalues(32, 32 * p_small, 1.0, 0.3, 2)
    assert raw.min() < -darcy.CE_NEG_TOL * raw.max()


def test_empirical_field_moments():
    # Philox-driven draws: mean mu, variance sigma^2, covariance at lags
    # h and 3h along x and y, Re/Im (layer 0 / layer 1) uncorrelated.
    model = darcy.Model.from_dict(workloads.workload(
        "lognormal_2layer_16to256", m0=8, mu=[0.5, -0.25], sigma2=[2.0, 2.0], lam=[0.2, 0.2]))
    n = 1500
    cache = {}
    g = np.stack([darcy.layer_fields(model, 7, 0, i, 8, cache) for i in range(n)])
    y0 = g[:, 0] - 0.5
    y1 = g[:, 1] + 0.25
    se = 2.0 * math.sqrt(2.0 / n)
    assert abs(y0.mean()) < 5 * math.sqrt(2.0 / n) and abs(y1.mean()) < 5 * math.sqrt(2.0 / n)
    for lag in (0, 1, 3):
        target = 2.0 * math.exp(-(lag / 8) / 0.2)
        cx = np.mean(y0[:, 2, 1:1 + 4] * y0[:, 2, 1 + lag:5 + lag])
        cy = np.mean(y1[:, 1:1 + 4, 3] * y1[:, 1 + lag:5 + lag, 3])
        assert abs(cx - target) < 5 * se, (lag, cx, target)
        assert abs(cy - target) < 5 * se, (lag, cy, target)
    assert abs(np.mean(y0 * y1)) < 5 * se


def test_interfaces_and_layer_rows():
    model = darcy.Model.from_dict(workloads.workload("lognormal_4layer_cgv_16to1024"))
    for s in range(50):
        eta = darcy.interfaces(model, 3, 2, s)
        assert eta.shape == (3,) and np.all(np.diff(eta) >= 0) and np.all((eta > 0) & (eta < 1))
        m = 64
        rows = darcy.layer_of_rows(eta, m)
        # number of row centres (j + 1/2)/m below each interface, in closed form
        below = [int(np.ceil(m * e - 0.5)) for e in eta]
        for t in range(3):
            assert np.sum(rows <= t) == below[t]
    # a centre exactly on an interface belongs to the upper layer
    assert list(darcy.layer_of_rows(np.array([0.375]), 4)) == [0, 1, 1, 1]
    model1 = darcy.Model.from_dict(workloads.workload("const_2layer_8to32"))
    eta = darcy.interfaces(model1, 0, 1, 5)
    from oracle import philox
    u = philox.interface_uniforms(0, 1, 5, 1)[0]
    assert eta[0] == 0.3 + (0.7 - 0.3) * u

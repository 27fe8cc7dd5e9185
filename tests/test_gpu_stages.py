"""GPU parity of the individual stages against the oracle, through the C ABI:
Philox words and interfaces bit-exact, fields (Ex. 1 constants, Ex. 2
circulant embedding), and the linear solve + outflow QoI on given k."""
import math

import numpy as np
import pytest

import workloads
from oracle import darcy, philox
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,level,sample,stream,first,n", [
    (0, 0, 0, 0, 0, 3), (12345, 3, 77, 2, 1000, 257), (2**63 + 5, 11, 2**40, 9, 2**33, 64)])
def test_philox_words_bit_exact(seed, level, sample, stream, first, n):
    torch, pk = need_gpu()
    w = pk.philox_words(seed, level, sample, stream, first, n).cpu().numpy().view(np.uint64)
    ref = philox.stream_words(seed, level, sample, stream, np.arange(first, first + n, dtype=np.uint64))
    assert np.array_equal(w, ref)


@pytest.mark.parametrize("prec,atol", [(0, 2e-15), (1, 2e-6)])
def test_normals_against_oracle(prec, atol):
    # the field kernels' Box-Muller (table-driven FP64 log/sincos, or FP32)
    # against the oracle's numpy log/cos/sin on a million calls, including
    # uniforms next to 0 and 1 (the words with all high bits 0 or 1 come up
    # among 2^22 draws only by chance, so the edge words are checked too)
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_16to256", prec=prec)
    n = 1 << 20
    with pk.Context(d) as ctx:
        z = ctx.normals(77, 3, 5, 2, 0, n).cpu().numpy()
    ref = philox.call_normals(philox.stream_words(77, 3, 5, 2, np.arange(n, dtype=np.uint64)))
    err = np.abs(z - ref)
    assert err.max() <= atol * max(1.0, np.abs(ref).max()), err.max()
    if prec == 0:
        # the log part on its own: re^2 + im^2 = -2 ln u_a to a few ulp
        # (re, im within ~2 ulp of r cos, r sin each, plus the two roundings
        # of the sum of squares here: <= 9 ulp = 2e-15 relative), and ~1e-18
        # absolute as u_a -> 1, where -2 ln u_a cancels in its table form
        u = philox.uniform(philox.stream_words(77, 3, 5, 2, np.arange(n, dtype=np.uint64)))
        r2 = z[:, 0] ** 2 + z[:, 1] ** 2
        ref2 = -2.0 * np.log(u[:, 0])
        assert np.all(np.abs(r2 - ref2) <= 2e-15 * ref2 + 1e-18)


@pytest.mark.parametrize("name", ["const_2layer_8to32", "lognormal_4layer_cgv_16to1024"])
def test_interfaces_bit_exact(name):
    torch, pk = need_gpu()
    d = workloads.workload(name, L=1)
    model = darcy.Model.from_dict(d)
    with pk.Context(d) as ctx:
        for level in (0, 1):
            g, eta = ctx.sample_fields(level, 37, seed=9, first=5)
            eta = eta.cpu().numpy()
            for s in range(37):
                ref = darcy.interfaces(model, 9, level, 5 + s)
                assert np.array_equal(eta[s], ref)


def test_const_fields():
    torch, pk = need_gpu()
    d = workloads.workload("const_2layer_8to32", mu=[0.3, -0.2], sigma2=[1.5, 0.5])
    model = darcy.Model.from_dict(d)
    with pk.Context(d) as ctx:
        g, _ = ctx.sample_fields(1, 20, seed=4)
        g = g.cpu().numpy()
    for s in range(20):
        ref = darcy.layer_fields(model, 4, 1, s, 16)
        np.testing.assert_allclose(g[s], ref, rtol=1e-14, atol=1e-14)


# lambda = 0.3: m = 16 embeds periodically at M = 32, m = 32 ... 256 with the
# cut-off embedding at M = 3m (radix-3 FFT stage); embed = 1 keeps the
# powers-of-two padding (M = 4m); lambda = 0.1 embeds at M = 2m.
@pytest.mark.parametrize("name,levels,embed", [("lognormal_2layer_16to256", (0, 1, 2, 4), 0),
                                               ("lognormal_2layer_16to256", (1, 2), 1),
                                               ("lognormal_4layer_cgv_16to1024", (0, 1), 0)])
def test_ce_fields_fp64(name, levels, embed):
    torch, pk = need_gpu()
    d = workloads.workload(name, prec=0, embed=embed)
    model = darcy.Model.from_dict(d)
    cache = {}
    with pk.Context(d) as ctx:
        for level in levels:
            m = model.m(level)
            M, lo, hi = ctx.ce_info(level)
            Mo, _ = darcy.ce_padding(m, model.sigma2[0], model.lam[0], model.norm_r, model.embed)
            assert M == Mo and lo >= -1e-13 * hi
            if name == "lognormal_2layer_16to256" and m >= 32:
                assert M == (3 * m if embed == 0 else 4 * m)
            n = 6
            g, _ = ctx.sample_fields(level, n, seed=3, first=11)
            g = g.cpu().numpy()
            for s in range(n):
                ref = darcy.layer_fields(model, 3, level, 11 + s, m, cache)
                np.testing.assert_allclose(g[s], ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("level,pad,n", [(0, 2, 40), (2, 3, 3), (5, 3, 3)])
def test_ce_fields_fp32_error_bound(level, pad, n):
    # the mixed workload's FP32 embedding: m = 16 (M = 32: both passes fused in
    # one kernel, warp-shuffle FFTs), m = 64 (M = 192) and the finest level
    # m = 512 (M = 1536, the cut-off embedding's radix-3 stage in FP32)
    torch, pk = need_gpu()
    d = workloads.workload("lognormal_2layer_cgv_16to512")
    model = darcy.Model.from_dict(d)
    m = model.m(level)
    with pk.Context(d) as ctx:
        assert ctx.ce_info(level)[0] == pad * m
        g, _ = ctx.sample_fields(level, n, seed=1, first=5)
        g = g.cpu().numpy()
    cache = {}
    for s in range(n):
        ref = darcy.layer_fields(model, 1, level, 5 + s, m, cache)
        assert np.max(np.abs(g[s] - ref)) < 2e-5


@pytest.mark.parametrize("m", [1, 2, 4, 8, 16, 32, 64, 128])
def test_solve_k_fp64(m):
    torch, pk = need_gpu()
    n = 12 if m <= 32 else 4
    k = workloads.random_k(m, seed=m, n=n, contrast=4.0)
    d = workloads.workload("const_2layer_8to32", tol=1e-13, max_it=500)
    with pk.Context(d) as ctx:
        p, q, it = ctx.solve_k(torch.from_numpy(k).cuda())
        p, q, it = p.cpu().numpy(), q.cpu().numpy(), it.cpu().numpy()
    for s in range(n):
        p_ref, q_ref = darcy.solve_k(k[s])
        assert abs(q[s] - q_ref) <= 1e-10 * abs(q_ref), (s, q[s], q_ref, it[s])
        assert np.max(np.abs(p[s] - p_ref)) < 1e-9
    assert it.max() < 100


@pytest.mark.parametrize("m,prec", [(16, 1), (64, 1), (256, 1), (16, 2), (64, 2), (256, 2), (16, 3), (64, 3),
                                    (256, 3)])
def test_solve_k_mixed(m, prec):
    torch, pk = need_gpu()
    n = 6
    k = workloads.random_k(m, seed=100 + m, n=n, contrast=4.0)
    # these log-normal k with layer jumps are ill-conditioned: a relative
    # residual of 1e-12 leaves Q errors up to ~7e-10, 1e-13 below 1e-10
    d = workloads.workload("const_2layer_8to32", tol=1e-13 if prec == 3 else 1e-12, max_it=1000, prec=prec)
    with pk.Context(d) as ctx:
        _, q, it = ctx.solve_k(torch.from_numpy(k).cuda(), want_p=False)
        q = q.cpu().numpy()
    for s in range(n):
        _, q_ref = darcy.solve_k(k[s])
        assert abs(q[s] - q_ref) <= (1e-10 if prec == 3 else 1e-6) * abs(q_ref), (s, q[s], q_ref)


def test_constant_k_closed_form_gpu():
    torch, pk = need_gpu()
    for m in (1, 2, 8, 64, 512):
        k = np.full((1, m, m), 2.5)
        with pk.Context(workloads.workload("const_2layer_8to32", tol=1e-13)) as ctx:
            p, q, _ = ctx.solve_k(torch.from_numpy(k).cuda())
        assert abs(q.item() - 2.5) < 1e-10 * 2.5
        x = (np.arange(m) + 0.5) / m
        assert np.max(np.abs(p.cpu().numpy()[0] - (1 - x)[None, :])) < 1e-9


def test_paper_geometry_line_ends_and_fields():
    # the sloped three-layer geometry of Sec. 3.4: line ends bit-exact, per-layer
    # fields (outer layers lambda = 0.3 on one draw, middle layer lambda = 0.1 on
    # its own draw) equal to the oracle's
    torch, pk = need_gpu()
    d = workloads.workload("paper_3layer_lognormal_16to128", prec=0)
    model = darcy.Model.from_dict(d)
    cache = {}
    with pk.Context(d) as ctx:
        for level in (0, 1):
            g, ends = ctx.sample_fields(level, 5, seed=6, first=3)
            g, ends = g.cpu().numpy(), ends.cpu().numpy()
            for s in range(5):
                assert np.array_equal(ends[s], darcy.interfaces(model, 6, level, 3 + s))
                ref = darcy.layer_fields(model, 6, level, 3 + s, model.m(level), cache)
                np.testing.assert_allclose(g[s], ref, rtol=0, atol=1e-12)

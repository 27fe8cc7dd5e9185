"""Pins of the oracle's counter-based generator (Philox4x64-10, uniforms,
Box-Muller) against numpy's independent Philox implementation, exact
arithmetic identities and distribution checks."""
import math

import numpy as np
import pytest

from oracle import philox



@pytest.mark.parametrize("key,ctr", [
    ((0, 0), (0, 0, 0, 0)),
    ((12345, 0), (7, 3, 2, 5)),
    ((0xFFFFFFFFFFFFFFFF, 0), (0xFFFFFFFFFFFFFFFE, 0, 1, 2)),
    ((2**40 + 17, 0), (99, 1 << 33, 6, 3)),
])
def test_philox_matches_numpy_bitgenerator(key, ctr):
    # numpy.random.Philox (Philox4x64-10) increments its 256-bit counter
    # before each block, so its block n comes from counter ctr + n + 1.
    bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64),
                          key=np.array(key, dtype=np.uint64))
    ref = bg.random_raw(12).reshape(3, 4)
    for blk in range(3):
        c = list(ctr)
        v = sum(x << (64 * t) for t, x in enumerate(c)) + blk + 1
        c = [(v >> (64 * t)) & 0xFFFFFFFFFFFFFFFF for t in range(4)]
        w = philox.philox4x64(*[np.uint64(x) for x in c], key[0], key[1])
        assert [int(x) for x in w] == [int(x) for x in ref[blk]]


def test_philox_vectorised_equals_scalar():
    calls = np.arange(37)
    w = philox.stream_words(11, 3, 1234, 5, calls)
    for c in (0, 1, 17, 36):
        s = philox.philox4x64(np.uint64(c), np.uint64(1234), np.uint64(3), np.uint64(5), 11, 0)
        assert [int(x) for x in w[c]] == [int(x) for x in s]


def test_uniform_exact_and_open_interval():
    words = np.array([0, 1, 4095, 4096, 2**63, 2**64 - 1], dtype=np.uint64)
    u = philox.uniform(words)
    k = (words >> np.uint64(12)).astype(np.float64)
    assert np.all(u > 0.0) and np.all(u < 1.0)
    assert np.array_equal(u * 2.0 ** 52 - 0.5, k)  # exact: no rounding anywhere
    assert u[0] == 2.0 ** -53 and u[-1] == 1.0 - 2.0 ** -53


def test_box_muller_polar_identity():
    rng = np.random.default_rng(0)
    ua, ub = rng.random(1000) * 0.999 + 5e-4, rng.random(1000)
    re, im = philox.box_muller(ua, ub)
    np.testing.assert_allclose(re * re + im * im, -2.0 * np.log(ua), rtol=1e-13)
    ang = np.mod(np.arctan2(im, re), 2 * np.pi)
    d = np.abs(np.angle(np.exp(1j * (ang - 2 * np.pi * ub))))
    assert d.max() < 1e-12


def test_call_normal_order():
    w = philox.stream_words(3, 1, 9, 2, np.arange(4))
    z = philox.call_normals(w)
    u = philox.uniform(w)
    re0, im0 = philox.box_muller(u[:, 0], u[:, 1])
    re1, im1 = philox.box_muller(u[:, 2], u[:, 3])
    assert np.array_equal(z[:, 0], re0) and np.array_equal(z[:, 1], im0)
    assert np.array_equal(z[:, 2], re1) and np.array_equal(z[:, 3], im1)
    xi = philox.field_normals(3, 1, 9, 0, 2)  # M = 2: four complex normals
    assert xi[0, 0] == z[0, 0] + 1j * z[0, 1]
    assert xi[0, 1] == z[0, 2] + 1j * z[0, 3]
    assert xi[1, 0] == z[1, 0] + 1j * z[1, 1]


def test_normals_distribution():
    xi = philox.field_normals(0, 0, 0, 0, 256).reshape(-1)
    z = np.concatenate([xi.real, xi.imag])
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(np.mean(xi.real * xi.imag)) < 5 / math.sqrt(xi.size)
    # Kolmogorov-Smirnov against the standard normal CDF
    zs = np.sort(z)
    cdf = 0.5 * (1 + np.vectorize(math.erf)(zs / math.sqrt(2)))
    ks = np.max(np.abs(cdf - np.arange(1, n + 1) / n))
    assert ks < 1.63 / math.sqrt(n)  # 1% level

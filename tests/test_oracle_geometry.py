"""Pins of the oracle's sloped three-layer geometry and per-layer parameters
(Sec. 3.4): the layer map against an independent orientation test, the line
ends' distribution, the pairing of layers onto circulant-embedding draws,
and per-layer field statistics (the middle layer has its own mean and
correlation length)."""
import math

import numpy as np
import pytest

import workloads
from oracle import darcy, philox


def paper(kind="lognormal", **kw):
    return darcy.Model.from_dict(workloads.workload("paper_3layer_%s_16to128" % kind, **kw))


def orientation_layers(ends, m):
    """Layer by the sign of the cross product (P1 - P0) x (c - P0) for each
    line P0 = (0, a), P1 = (1, b): the centre c is on or above the line iff
    (b - a) * cx - (cy - a) <= 0."""
    c = (np.arange(m) + 0.5) / m
    out = np.zeros((m, m), dtype=int)
    for j in range(m):
        for i in range(m):
            for a, b in ((ends[2], ends[3]), (ends[0], ends[1])):
                if (b - a) * c[i] - (c[j] - a) <= 1e-15:
                    out[j, i] += 1
    return out


def test_layer_map_against_orientation():
    model = paper()
    for s in range(30):
        ends = darcy.interfaces(model, 5, 1, s)
        assert ends.shape == (4,)
        for t, (lo, hi) in enumerate(zip(model.line_lo, model.line_hi)):
            assert lo < ends[t] < hi
        for m in (8, 32):
            assert np.array_equal(darcy.layer_map(model, ends, m), orientation_layers(ends, m))
    # the three layers are stacked: bottom 0, middle 1, top 2 in every column
    lm = darcy.layer_map(model, darcy.interfaces(model, 0, 0, 0), 64)
    assert np.all(np.diff(lm, axis=0) >= 0) and lm[0].max() == 0 and lm[-1].min() == 2


def test_line_ends_uniform():
    model = paper()
    ends = np.array([darcy.interfaces(model, 1, 0, s) for s in range(4000)])
    for t, (lo, hi) in enumerate(zip(model.line_lo, model.line_hi)):
        u = (ends[:, t] - lo) / (hi - lo)
        assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / 4000)
        assert abs(u.var() - 1 / 12) < 0.01


def test_field_slots():
    slots, params = darcy.field_slots(paper())
    assert slots == [(0, 0), (1, 0), (0, 1)] and params == [(1.0, 0.3), (1.0, 0.1)]
    slots, params = darcy.field_slots(darcy.Model.from_dict(workloads.workload("lognormal_4layer_cgv_16to1024")))
    assert slots == [(0, 0), (0, 1), (1, 0), (1, 1)] and len(params) == 2


def test_per_layer_field_statistics():
    # each layer's field has its own mean and covariance: lag-1 correlation
    # exp(-h / lambda) with lambda = 0.3 (outer) or 0.1 (middle)
    model = paper()
    m, n = 16, 600
    cache = {}
    g = np.stack([darcy.layer_fields(model, 3, 0, i, m, cache) for i in range(n)])
    h = 1.0 / m
    for t, (mu, lam) in enumerate(((0.0, 0.3), (4.0, 0.1), (0.0, 0.3))):
        y = g[:, t] - mu
        assert abs(y.mean()) < 0.15
        c1 = np.mean(y[:, :, :-1] * y[:, :, 1:])
        assert abs(c1 - math.exp(-h / lam)) < 0.08, (t, c1)
    # layers 0 and 2 share one complex draw (Re / Im): uncorrelated
    assert abs(np.mean((g[:, 0]) * (g[:, 2]))) < 0.08


def test_const_sloped_sample_matches_dense():
    model = paper("const")
    r = darcy.sample(model, 2, 1, 7, want_fields=True)
    k = r["k"]
    vals = np.unique(k)
    assert len(vals) == 3  # three constant layers
    z = philox.layer_normals(2, 1, 7, 3)
    assert np.allclose(np.sort(vals), np.sort(np.exp(z)))

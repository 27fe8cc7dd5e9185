"""The oracle against the convergence rates the paper reports for piecewise
constant random layers (Sec. 3.4, the paper's sloped three-layer geometry,
outflow functional; values in tests/golden/paper_values.json with their
citation): the bias decays like h (alpha = 1) and the variance of
Y_l = Q_l - Q_{l-1} like h^2 (beta = 2).

Fixed seeds and sample counts, so the check is deterministic; the bounds
leave room for the sampling error of a few hundred heavy-tailed samples.
A broken coupling of the fine and coarse samples fails it: with the coarse
term taken from another sample's draw the fitted rates are alpha = -0.2 and
beta = 0.3.
The CGV counterpart (Sec. 4.2: a much smaller variance of Y_l, decaying
faster) is test_oracle_mlmc.py::test_cgv_variance_reduction."""
import json
import os

import numpy as np
import pytest

import workloads
from oracle import darcy

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))

pytestmark = pytest.mark.slow


def _y_stats(model, seed, level, n, coarse="qc"):
    y = np.array([(lambda r: r["qf"] - r[coarse])(darcy.sample(model, seed, level, i)) for i in range(n)])
    return y.mean(), y.var(ddof=1)


def test_piecewise_constant_layer_rates():
    """alpha and beta of the sloped three-layer model with constant k per
    layer, from levels m = 32 and m = 128 (two halvings of h)."""
    rates = GOLD["rates_piecewise_constant_outflow"]
    model = darcy.Model.from_dict(workloads.workload("paper_3layer_const_16to128"))
    mean1, var1 = _y_stats(model, 0, 1, 400)
    mean3, var3 = _y_stats(model, 0, 3, 100)
    alpha = np.log2(abs(mean1) / abs(mean3)) / 2
    beta = np.log2(var1 / var3) / 2
    assert abs(alpha - rates["alpha"]) <= 0.5, alpha
    assert abs(beta - rates["beta"]) <= 0.6, beta


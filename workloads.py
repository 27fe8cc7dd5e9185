"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

This module holds parameters and seeded input generators only, none of the
method's arithmetic.  The five workloads are the layered Darcy models used to
exercise the MLMC level batch (Sec. 2 Ex. 1 / Ex. 2, Sec. 3.4 Model Problem 2):

  const_2layer_8to32        two horizontal layers, constant k = exp(Z) per
                            layer, interface ~U(0.3, 0.7), m = 8, 16, 32
  lognormal_2layer_16to256  two layers, log-normal fields with exponential
                            2-norm covariance, sigma^2 = 1, lambda = 0.3,
                            m = 16 .. 256, eps = 1e-3, FP64
  lognormal_2layer_cgv_16to512  the same model with Coarse Grid Variates,
                            FP32 multigrid inside FP64 refinement, m = 16 .. 512,
                            eps = 5e-4
  lognormal_4layer_cgv_16to1024 four layers from three sorted U(0,1) draws,
                            sigma^2 = 3, lambda = 0.1, m = 16 .. 1024
  lognormal_2layer_cgv_32to2048 interface ~U(0.2, 0.8), sigma^2 = 1,
                            lambda = 0.05, m = 32 .. 2048, eps = 2e-4
  paper_3layer_const_16to128  the three sloped layers of Sec. 3.4 (lines
                            (0,y1)-(1,y2), (0,y3)-(1,y4), y1~U(.8,.9),
                            y2~U(.6,.7), y3~U(.2,.3), y4~U(.4,.5)) with
                            k = exp(z), z ~ N(0, 1) per layer
  paper_3layer_lognormal_16to128  the same layers with log-normal fields:
                            outer layers mu = 0, lambda = 0.3, middle layer
                            mu = 4, lambda = 0.1, sigma^2 = 1, 2-norm
  lognormal_3d_cgv_8to32    the unit cube (Sec. 3.4, 2-D layers extruded
                            along x3): two layers, interface ~U(0.3, 0.7),
                            log-normal fields with the 1-norm covariance of
                            the CGV experiments (Sec. 4.2), sigma^2 = 1,
                            lambda = 0.3, m = 8, 16, 32, CGV with 8 offsets
"""
import numpy as np

WORKLOADS = {
    "const_2layer_8to32": dict(
        n_layers=2, k_kind=0, if_lo=0.3, if_hi=0.7, mu=[0.0, 0.0], sigma2=[1.0, 1.0],
        lam=[0.3, 0.3], norm_r=2, m0=8, L=2, cgv=0, prec=0, tol=1e-12, max_it=500,
        n_per_level=1000, seed=0),
    "lognormal_2layer_16to256": dict(
        n_layers=2, k_kind=1, if_lo=0.3, if_hi=0.7, mu=[0.0, 0.0], sigma2=[1.0, 1.0],
        lam=[0.3, 0.3], norm_r=2, m0=16, L=4, cgv=0, prec=0, tol=1e-10, max_it=500,
        eps=1e-3, seed=0),
    "lognormal_2layer_cgv_16to512": dict(
        n_layers=2, k_kind=1, if_lo=0.3, if_hi=0.7, mu=[0.0, 0.0], sigma2=[1.0, 1.0],
        lam=[0.3, 0.3], norm_r=2, m0=16, L=5, cgv=1, prec=1, tol=1e-10, max_it=500,
        eps=5e-4, seed=0),
    "lognormal_4layer_cgv_16to1024": dict(
        n_layers=4, k_kind=1, if_lo=0.0, if_hi=1.0, mu=[0.0] * 4, sigma2=[3.0] * 4,
        lam=[0.1] * 4, norm_r=2, m0=16, L=6, cgv=1, prec=1, tol=1e-10, max_it=500,
        eps=5e-4, seed=0),
    "lognormal_2layer_cgv_32to2048": dict(
        n_layers=2, k_kind=1, if_lo=0.2, if_hi=0.8, mu=[0.0, 0.0], sigma2=[1.0, 1.0],
        lam=[0.05, 0.05], norm_r=2, m0=32, L=6, cgv=1, prec=1, tol=1e-10, max_it=500,
        eps=2e-4, seed=0),
    "paper_3layer_const_16to128": dict(
        n_layers=3, k_kind=0, geometry=1, mu=[0.0] * 3, sigma2=[1.0] * 3, lam=[0.3] * 3, norm_r=2,
        m0=16, L=3, cgv=0, prec=0, tol=1e-10, max_it=500, eps=2e-3, seed=0),
    "lognormal_3d_cgv_8to32": dict(
        dim=3, n_layers=2, k_kind=1, if_lo=0.3, if_hi=0.7, mu=[0.0, 0.0], sigma2=[1.0, 1.0],
        lam=[0.3, 0.3], norm_r=1, m0=8, L=2, cgv=1, prec=1, tol=1e-10, max_it=500, eps=5e-4, seed=0),
    "paper_3layer_lognormal_16to128": dict(
        n_layers=3, k_kind=1, geometry=1, mu=[0.0, 4.0, 0.0], sigma2=[1.0, 1.0, 1.0],
        lam=[0.3, 0.1, 0.3], norm_r=2, m0=16, L=3, cgv=0, prec=0, tol=1e-10, max_it=500,
        eps=2e-2, seed=0),
}


def workload(name, **overrides):
    """A copy of a named workload with fields overridden."""
    d = dict(WORKLOADS[name])
    d.update(overrides)
    return d


def random_k(m, seed, n=1, contrast=4.0, layered=True):
    """Seeded positive permeability arrays k[n, m, m] for solver-only tests:
    log-normal cell values exp(contrast * z) with z ~ N(0, 1), optionally
    multiplied by a few horizontal bands of constant jumps."""
    rng = np.random.default_rng(seed)
    k = np.exp(contrast * rng.standard_normal((n, m, m)) / 2.0)
    if layered:
        for s in range(n):
            cuts = np.sort(rng.integers(0, m + 1, size=2))
            k[s, cuts[0]:cuts[1], :] *= np.exp(contrast * rng.standard_normal())
    return k

"""One Darcy-flow sample of the layered model, plain FP64 (test infrastructure).

Follows the paper section by section:

* Sec. 2, random partition and Ex. 1 / Ex. 2: the unit square is split into
  horizontal layers by random interface heights; layer t carries
  k_t = exp(g_t) with g_t either the constant mu_t + sigma_t Z_t (Ex. 1) or a
  stationary Gaussian field with the exponential covariance of Eq. 2.3.
* Sec. 3.4 / 3.5: fields are drawn exactly on the cell-centre grid by
  circulant embedding (CE) on an M x M torus.
* Sec. 3.1, Eq. 3.3 with the harmonic face average of Sec. 3.1/3.4: the
  cell-centred five-point system; Dirichlet faces use the one-sided
  difference over half a cell (transmissibility 2k), Neumann faces carry no
  flux.
* Sec. 3.4, Model Problem 2: p = 1 at x1 = 0, p = 0 at x1 = 1, no flow on
  x2 = 0 and x2 = 1; the quantity of interest M^(2) is the outflow at x1 = 1.
* Sec. 3.4, Model Problem 1: f = 1, p = 0 on the whole boundary; the quantity
  of interest M^(1) is the mean of p over a small box D* around x*.

Layout: a grid of m x m cells, cell (i, j) 0-based with centre
((i + 1/2) h, (j + 1/2) h), h = 1/m; arrays are indexed [j, i] (x1 = flow
direction along the fast axis).
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

from . import philox

# Padding rule of the circulant embedding: try the embeddings of
# padding_candidates (M = 2m, the cut-off one at 3m, then 4m, 8m, 16m) until
# every eigenvalue is >= -CE_NEG_TOL * the largest; eigenvalues inside that
# band are clipped to zero.
CE_NEG_TOL = 1e-13
CE_MAX_PAD = 16


@dataclass
class Model:
    """Parameters of the layered permeability model and the solver.

    k_kind: 0 = piecewise constant (Ex. 1), 1 = piecewise log-normal field (Ex. 2)
    if_lo, if_hi: the n_layers-1 interface heights are U(if_lo, if_hi) draws,
        sorted ascending; layer 0 is the bottom layer.
    mu, sigma2, lam: per-layer mean, variance and correlation length.
    norm_r: the l_r norm of Eq. 2.3 (1 or 2).
    m0, L: level l has m0 * 2^l cells per side, l = 0..L.
    cgv: 0 plain MLMC coupling, 1 Coarse Grid Variates subsampling the
        per-layer Gaussian fields, 2 CGV subsampling the composed k.
    tol: relative residual tolerance of iterative solvers (unused by the
        direct solve of the oracle).
    problem: 2 (or 0) = Model Problem 2, outflow; 1 = Model Problem 1, local
        average of p over the box qoi_box = (x0, x1, y0, y1).
    geometry: 0 = horizontal interfaces (above); 1 = the three layers of Sec. 3.4
        cut by the straight lines (0, y1)-(1, y2) and (0, y3)-(1, y4), with
        y_t ~ U(line_lo[t], line_hi[t]).
    dim: 2, or 3 for the extruded 3-D medium of Sec. 3.4 (oracle/darcy3.py).
    embed: 0 = the cut-off embedding at M = 3m may be chosen (2-D, 2-norm),
        1 = periodic embeddings with M = 2m, 4m, 8m, 16m only.
    """
    n_layers: int = 2
    k_kind: int = 0
    if_lo: float = 0.3
    if_hi: float = 0.7
    mu: List[float] = field(default_factory=lambda: [0.0] * 8)
    sigma2: List[float] = field(default_factory=lambda: [1.0] * 8)
    lam: List[float] = field(default_factory=lambda: [0.3] * 8)
    norm_r: int = 2
    m0: int = 8
    L: int = 2
    cgv: int = 0
    prec: int = 0
    tol: float = 1e-12
    max_it: int = 200
    problem: int = 2
    qoi_box: List[float] = field(default_factory=lambda: [7 / 16, 9 / 16, 7 / 16, 9 / 16])
    geometry: int = 0
    line_lo: List[float] = field(default_factory=lambda: [0.8, 0.6, 0.2, 0.4])
    line_hi: List[float] = field(default_factory=lambda: [0.9, 0.7, 0.3, 0.5])
    dim: int = 2
    embed: int = 0

    @classmethod
    def from_dict(cls, d):
        kw = {k: d[k] for k in cls.__dataclass_fields__ if k in d}
        if kw.get("problem", 2) == 0:
            kw["problem"] = 2
        for key in ("mu", "sigma2", "lam"):
            if key in kw:
                v = list(kw[key]) + [kw[key][-1]] * (8 - len(kw[key]))
                kw[key] = v[:8]
        return cls(**kw)

    def m(self, level):
        return self.m0 << level


# ---------------------------------------------------------------- layers ----
def interfaces(model, seed, level, sample):
    """Random partition (Sec. 2): sorted interface heights eta_t ~ U(if_lo,
    if_hi) (geometry 0), or the four line end heights y_1..y_4 ~ U(line_lo[t],
    line_hi[t]) of the sloped layers of Sec. 3.4 (geometry 1).

    Each value is lo + (hi - lo) * u, every operation rounded once (no fused
    multiply-add)."""
    if model.geometry == 1:
        u = philox.interface_uniforms(seed, level, sample, 4)
        lo = np.asarray(model.line_lo, dtype=np.float64)
        width = np.asarray(model.line_hi, dtype=np.float64) - lo
        return lo + width * u
    n_if = model.n_layers - 1
    if n_if == 0:
        return np.zeros(0)
    u = philox.interface_uniforms(seed, level, sample, n_if)
    width = np.float64(model.if_hi) - np.float64(model.if_lo)
    eta = np.float64(model.if_lo) + width * u
    return np.sort(eta)


def layer_map(model, ends, m):
    """Layer index of every cell centre ((i + 1/2)/m, (j + 1/2)/m), as an array
    [j, i].  Geometry 0: the number of interfaces at or below the row centre.
    Geometry 1: the number of the two lines (0, y3)-(1, y4) (lower) and
    (0, y1)-(1, y2) (upper) at or below the centre, the line height at x being
    y_a + ((y_b - y_a) * x) with each operation rounded once."""
    if model.geometry != 1:
        rows = layer_of_rows(ends, m)
        return np.repeat(rows[:, None], m, axis=1)
    c = (np.arange(m) + 0.5) / m
    x, y = c[None, :], c[:, None]
    lower = ends[2] + (ends[3] - ends[2]) * x
    upper = ends[0] + (ends[1] - ends[0]) * x
    return (lower <= y).astype(np.int64) + (upper <= y).astype(np.int64)


def field_slots(model):
    """Which complex circulant-embedding draw feeds which layer: layers are
    taken in order and paired greedily with an earlier layer of the same
    (sigma2, lambda) whose draw still has its imaginary part free; returns
    (slots, params) with slots[t] = (pair f, 0 for Re / 1 for Im) and params[f]
    = (sigma2, lambda).  Draw f uses Philox stream 2 + f."""
    slots, params, open_im = [], [], {}
    for t in range(model.n_layers):
        key = (model.sigma2[t], model.lam[t])
        if key in open_im:
            f = open_im.pop(key)
            slots.append((f, 1))
        else:
            f = len(params)
            params.append(key)
            open_im[key] = f
            slots.append((f, 0))
    return slots, params


def layer_of_rows(eta, m):
    """Layer index of each cell row j: the number of interfaces at or below the
    row's centre y_j = (j + 1/2)/m (a centre exactly on an interface belongs to
    the upper layer)."""
    y = (np.arange(m) + 0.5) / m
    return np.array([int(np.sum(eta <= yj)) for yj in y], dtype=np.int64)


# ------------------------------------------------------ circulant embedding --
def cutoff_radii(m, M):
    """(R0, R1) of the cut-off embedding: R0 = sqrt(2) (m - 1) h, the largest
    distance between two cell centres of the unit square, and R1 = M h / 2,
    half the side of the torus (h = 1/m)."""
    return np.sqrt(2.0) * (m - 1) / m, M / (2.0 * m)


def cutoff_covariance(r, m, M, sigma2, lam):
    """The radial function of the cut-off embedding (2-norm): the covariance
    of Eq. 2.3, sigma2 exp(-r/lam), up to R0; between R0 and R1 the cubic
    that continues it with the same value and slope at R0 and reaches zero
    with zero slope at R1; zero beyond R1.  It equals Eq. 2.3 at every
    distance between two cell centres, and with R1 <= M h / 2 its periodic
    copies on the M x M torus do not overlap."""
    R0, R1 = cutoff_radii(m, M)
    r = np.asarray(r, dtype=np.float64)
    c = sigma2 * np.exp(-r / lam)
    w = R1 - R0
    t = (r - R0) / w
    c0 = sigma2 * np.exp(-R0 / lam)      # value at R0
    d0 = -c0 / lam * w                   # slope at R0, in units of t
    taper = c0 * (2 * t ** 3 - 3 * t ** 2 + 1) + d0 * (t ** 3 - 2 * t ** 2 + t)
    return np.where(r <= R0, c, np.where(r < R1, taper, 0.0))


def covariance_torus(m, M, sigma2, lam, norm_r, cutoff=False):
    """c[b, a] = sigma2 * exp(-||(d_a h, d_b h)||_r / lam) on the M x M torus of
    cell-centre offsets (Eq. 2.3), d_a = min(a, M - a), h = 1/m; with cutoff
    (2-norm only) the cut-off radial function of the same distance."""
    a = np.arange(M)
    d = np.minimum(a, M - a) / m
    dx = d[None, :]
    dy = d[:, None]
    if norm_r == 1:
        dist = np.abs(dx) + np.abs(dy)
    else:
        dist = np.sqrt(dx * dx + dy * dy)
    if cutoff:
        assert norm_r == 2
        return cutoff_covariance(dist, m, M, sigma2, lam)
    return sigma2 * np.exp(-dist / lam)


def ce_eigenvalues(m, M, sigma2, lam, norm_r, cutoff=False):
    """Eigenvalues of the block-circulant embedding: the unnormalised forward
    2-D DFT of the torus covariance (real because c is even)."""
    return np.fft.fft2(covariance_torus(m, M, sigma2, lam, norm_r, cutoff)).real


def padding_candidates(m, norm_r, embed=0):
    """The embeddings tried, in order, as (p, cutoff): the periodic embedding
    at p = 2, then (2-norm, m >= 8, embed == 0) the cut-off embedding at
    p = 3, then the periodic one at p = 4, 8, 16.  The cut-off needs the
    torus half-side M h / 2 above the largest centre distance sqrt(2), which
    p = 3 gives and p = 2 does not."""
    out = [(2, False)]
    if embed == 0 and norm_r == 2 and m >= 8:
        out.append((3, True))
    return out + [(4, False), (8, False), (16, False)]


def ce_padding(m, sigma2, lam, norm_r, embed=0):
    """The first embedding of padding_candidates whose eigenvalues are all
    >= -CE_NEG_TOL * max; returns (M, eigenvalues clipped to >= 0)."""
    for p, cut in padding_candidates(m, norm_r, embed):
        M = p * m
        lam_q = ce_eigenvalues(m, M, sigma2, lam, norm_r, cut)
        if lam_q.min() >= -CE_NEG_TOL * lam_q.max():
            return M, np.maximum(lam_q, 0.0)
    raise ValueError("circulant embedding not non-negative at p=%d" % CE_MAX_PAD)


def ce_pair(lam_q, xi, m):
    """Two independent fields on the m x m cell centres from one complex draw:
    y[b, a] = sum_q sqrt(Lambda_q)/M xi_q exp(-2 pi i (a q1 + b q2)/M);
    returns (Re y, Im y) cropped to the first m x m entries."""
    M = lam_q.shape[0]
    y = np.fft.fft2(np.sqrt(lam_q) / M * xi)
    return y.real[:m, :m], y.imag[:m, :m]


def layer_fields(model, seed, level, sample, m, ce_cache=None):
    """Per-layer fields g_t on the m x m grid: Ex. 1 constants or Ex. 2 CE fields.

    Returns an array g[t, j, i] (t < n_layers)."""
    nl = model.n_layers
    g = np.empty((nl, m, m))
    if model.k_kind == 0:
        z = philox.layer_normals(seed, level, sample, nl)
        for t in range(nl):
            g[t] = model.mu[t] + np.sqrt(model.sigma2[t]) * z[t]
        return g
    slots, params = field_slots(model)
    for f, (sigma2, lam) in enumerate(params):
        key = (m, sigma2, lam, model.norm_r, model.embed)
        if ce_cache is not None and key in ce_cache:
            M, lam_q = ce_cache[key]
        else:
            M, lam_q = ce_padding(m, sigma2, lam, model.norm_r, model.embed)
            if ce_cache is not None:
                ce_cache[key] = (M, lam_q)
        xi = philox.field_normals(seed, level, sample, f, M)
        parts = ce_pair(lam_q, xi, m)
        for t in range(nl):
            if slots[t][0] == f:
                g[t] = model.mu[t] + parts[slots[t][1]]
    return g


def compose_k(g, layers):
    """k at the cell centres: k[j, i] = exp(g_{layer}[j, i]), with `layers` the
    layer of each row (array [m]) or of each cell (array [m, m])."""
    m = g.shape[1]
    lay = layers[:, None] if layers.ndim == 1 else layers
    return np.exp(g[lay, np.arange(m)[:, None], np.arange(m)[None, :]])


# ----------------------------------------------------------------- TPFA -----
def transmissibilities(k, problem=2):
    """Face coefficients of Eq. 3.3 with harmonic face averages.

    tx[j, i'] for the m+1 faces x1 = i'/m of row j: interior faces
    2 k_a k_b / (k_a + k_b); Dirichlet faces (i' = 0, m) 2 k_cell from the
    one-sided difference over half a cell.
    ty[j', i] for the m+1 faces x2 = j'/m of column i: interior faces harmonic;
    the faces j' = 0, m carry 0 (no flow, Model Problem 2) or 2 k_cell
    (Dirichlet, Model Problem 1)."""
    m = k.shape[0]
    tx = np.zeros((m, m + 1))
    ty = np.zeros((m + 1, m))
    ka, kb = k[:, :-1], k[:, 1:]
    tx[:, 1:m] = 2.0 * ka * kb / (ka + kb)
    tx[:, 0] = 2.0 * k[:, 0]
    tx[:, m] = 2.0 * k[:, m - 1]
    ka, kb = k[:-1, :], k[1:, :]
    ty[1:m, :] = 2.0 * ka * kb / (ka + kb)
    if problem == 1:
        ty[0, :] = 2.0 * k[0, :]
        ty[m, :] = 2.0 * k[m - 1, :]
    return tx, ty


def rhs(tx, problem=2):
    """Right-hand side.  Model Problem 2: the Dirichlet value p = 1 at x1 = 0
    enters through the west boundary face of column i = 0 (f = 0).  Model
    Problem 1: f = 1 by the midpoint rule, f / m^2 in every cell (p = 0 on the
    boundary adds nothing)."""
    m = tx.shape[0]
    if problem == 1:
        return np.full((m, m), 1.0 / (m * m))
    b = np.zeros((m, m))
    b[:, 0] = tx[:, 0] * 1.0
    return b


def banded_upper(tx, ty):
    """The SPD five-point matrix in LAPACK upper banded storage (bandwidth m),
    unknown n = j*m + i."""
    m = tx.shape[0]
    n = m * m
    ab = np.zeros((m + 1, n))
    diag = tx[:, :m] + tx[:, 1:] + ty[:m, :] + ty[1:, :]
    ab[m, :] = diag.reshape(-1)
    east = np.zeros((m, m))
    east[:, :m - 1] = -tx[:, 1:m]           # coupling (i, j) -- (i+1, j)
    ab[m - 1, 1:] = east.reshape(-1)[:-1]
    if m > 1:
        north = -ty[1:m, :]                 # coupling (i, j) -- (i, j+1)
        ab[0, m:] = north.reshape(-1)
    return ab


# Grids up to this side use the banded Cholesky; larger ones a sparse LU
# (storage of the band grows as m^3, its work as m^4).
BANDED_MAX_M = 256


def sparse_matrix(tx, ty):
    """The SPD five-point matrix as a scipy CSC matrix, unknown n = j*m + i:
    diagonal = sum of the four faces, off-diagonals = -face."""
    m = tx.shape[0]
    n = m * m
    diag = (tx[:, :m] + tx[:, 1:] + ty[:m, :] + ty[1:, :]).reshape(-1)
    east = np.zeros((m, m))
    east[:, :m - 1] = -tx[:, 1:m]
    e = east.reshape(-1)[:-1]
    north = -ty[1:m, :].reshape(-1)
    return scipy.sparse.diags([diag, e, e, north, north], [0, 1, -1, m, -m], shape=(n, n), format="csc")


def solve_sparse(tx, ty, b):
    """Direct sparse LU solve of the five-point system (SuperLU, minimum
    degree ordering of A^T + A, which keeps the fill of a 2-D grid near
    n log n)."""
    m = tx.shape[0]
    lu = scipy.sparse.linalg.splu(sparse_matrix(tx, ty), permc_spec="MMD_AT_PLUS_A",
                                  options=dict(SymmetricMode=True))
    return lu.solve(b.reshape(-1)).reshape(m, m)


def solve_direct(tx, ty, b):
    """Direct solve of the five-point system: banded Cholesky (LAPACK pbsv)
    for m <= BANDED_MAX_M, sparse LU above."""
    m = tx.shape[0]
    if m == 1:
        return (b / (tx[:, :1] + tx[:, 1:] + ty[:1, :] + ty[1:, :])).reshape(1, 1)
    if m > BANDED_MAX_M:
        return solve_sparse(tx, ty, b)
    p = scipy.linalg.solveh_banded(banded_upper(tx, ty), b.reshape(-1), lower=False)
    return p.reshape(m, m)


def outflow(tx, p):
    """M^(2): outflow through x1 = 1, sum_j tx[j, m] * (p[j, m-1] - 0)."""
    return float(np.sum(tx[:, -1] * p[:, -1]))


def inflow(tx, p):
    """Inflow through x1 = 0, sum_j tx[j, 0] * (1 - p[j, 0])."""
    return float(np.sum(tx[:, 0] * (1.0 - p[:, 0])))


def box_weights(m, box):
    """Weights w[j, i] = |cell (i, j) & D*| / |D*| of the box D* = [x0, x1] x
    [y0, y1]: M^(1) of the piecewise constant p is sum w p."""
    x0, x1, y0, y1 = box
    e = np.arange(m + 1) / m
    ox = np.clip(np.minimum(e[1:], x1) - np.maximum(e[:-1], x0), 0.0, None)
    oy = np.clip(np.minimum(e[1:], y1) - np.maximum(e[:-1], y0), 0.0, None)
    return np.outer(oy, ox) / ((x1 - x0) * (y1 - y0))


def local_average(p, box):
    """M^(1): mean of the piecewise constant p over D*."""
    return float(np.sum(box_weights(p.shape[0], box) * p))


def solve_k(k, problem=2, box=(7 / 16, 9 / 16, 7 / 16, 9 / 16)):
    """Assemble and solve for one permeability array; returns (p, Q) with Q the
    outflow (Model Problem 2) or the local average (Model Problem 1)."""
    tx, ty = transmissibilities(k, problem)
    p = solve_direct(tx, ty, rhs(tx, problem))
    return p, (local_average(p, box) if problem == 1 else outflow(tx, p))


# ------------------------------------------------------- one MLMC sample ----
CGV_OFFSETS = ((0, 0), (1, 0), (0, 1), (1, 1))  # (ox, oy) in summation order


def coarse_samples(model, g_fine, k_fine, eta, mode):
    """Coarse permeability arrays on the level below, extracted from the fine
    sample (Sec. 4.1, Eq. 4.1).

    mode 0 (plain coupling): one coarse sample, offset (0, 0).
    mode 1 (CGV): the 2^d = 4 strided sub-vectors of the fine per-layer fields
        g_t at offsets (ox, oy), composed with the layer map of the coarse
        centres.
    mode 2 (CGV on k): the 4 strided sub-vectors of the composed fine k."""
    m = g_fine.shape[1]
    mc = m // 2
    rows_c = layer_map(model, eta, mc)
    offsets = CGV_OFFSETS[:1] if mode == 0 else CGV_OFFSETS
    out = []
    for ox, oy in offsets:
        if mode == 2:
            out.append(k_fine[oy::2, ox::2].copy())
        else:
            gc = g_fine[:, oy::2, ox::2]
            out.append(compose_k(gc, rows_c))
    return out


def sample(model, seed, level, i, ce_cache=None, want_fields=False):
    """Q_l and the coarse Q's of sample i at level l (Eq. 3.6, Eq. 4.2).

    Returns a dict with qf, qc (plain coupling, offset (0,0); 0 at l = 0),
    qc_cgv (mean of the 4 CGV coarse Q's, in CGV_OFFSETS order; NaN if
    cgv == 0), and diagnostics.  dim = 3 models go to darcy3.sample."""
    if model.dim == 3:
        from . import darcy3
        return darcy3.sample(model, seed, level, i, ce_cache, want_fields)
    m = model.m(level)
    eta = interfaces(model, seed, level, i)
    rows = layer_map(model, eta, m)
    g = layer_fields(model, seed, level, i, m, ce_cache)
    k = compose_k(g, rows)
    prob = 1 if model.problem == 1 else 2
    box = tuple(model.qoi_box)
    p, qf = solve_k(k, prob, box)
    out = {"qf": qf, "qc": 0.0, "qc_cgv": float("nan"), "eta": eta, "rows": rows,
           "inflow": inflow(transmissibilities(k)[0], p)}
    if want_fields:
        out.update(g=g, k=k, p=p)
    if level > 0:
        if model.cgv == 0:
            (kc,) = coarse_samples(model, g, k, eta, 0)
            out["qc"] = solve_k(kc, prob, box)[1]
        else:
            kcs = coarse_samples(model, g, k, eta, model.cgv)
            qcs = [solve_k(kc, prob, box)[1] for kc in kcs]
            out["qc"] = qcs[0]
            out["qc_cgv"] = 0.25 * (((qcs[0] + qcs[1]) + qcs[2]) + qcs[3])
            out["qc_each"] = qcs
    elif model.cgv != 0:
        out["qc_cgv"] = 0.0
    return out

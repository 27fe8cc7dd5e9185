"""One Darcy-flow sample of the layered model in three dimensions, plain FP64
(test infrastructure: only tests, the smoke check and the benchmark's CPU
baseline use it).

Follows the paper:

* Sec. 3.4: the 3-D layered medium is the 2-D one extruded along the x3 axis
  (the layer of a cell depends on (x1, x2) only), with horizontal interfaces
  (geometry 0) or the two sloped lines of the three-layer example
  (geometry 1).
* Sec. 2, Ex. 2, Eq. 2.3: per-layer stationary Gaussian fields with the
  exponential covariance in d = 3, drawn exactly on the cell centres by
  circulant embedding on an M x M x M torus.
* Sec. 3.1, Eq. 3.3 in 3-D: the cell-centred seven-point two-point-flux
  system with harmonic face averages; a face of area h^2 between centres h
  apart has transmissibility h * 2 k_a k_b / (k_a + k_b), a Dirichlet face
  (centre h/2 away) h * 2 k.  The system below is divided by h, so its face
  coefficients are those of the 2-D code and the outflow is h times their
  flux sum.
* Sec. 3.4: Model Problem 2 (p = 1 at x1 = 0, p = 0 at x1 = 1, no flow
  elsewhere, Q = outflow through x1 = 1) and Model Problem 1 (f = 1, p = 0 on
  the boundary, Q = mean of p over the box D*).
* Sec. 4.1, Eq. 4.1 with d = 3: Coarse Grid Variates average the 2^3 = 8
  strided sub-samples of the fine fields.

Layout: m x m x m cells, cell (i, j, l) 0-based with centre ((i + 1/2) h,
(j + 1/2) h, (l + 1/2) h), arrays indexed [l, j, i] (x1 on the fast axis).
"""
import numpy as np
import scipy.sparse
import scipy.sparse.linalg

from . import darcy, philox

# Coarse Grid Variate offsets (ox, oy, oz) in summation order.
CGV_OFFSETS3 = ((0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1))


def layer_map3(model, ends, m):
    """Layer of every cell centre, array [l, j, i]: the 2-D layer map of the
    (x1, x2) centre, the same for every l (extrusion along x3)."""
    return np.broadcast_to(darcy.layer_map(model, ends, m)[None, :, :], (m, m, m)).copy()


# ------------------------------------------------------ circulant embedding --
def covariance_torus3(m, M, sigma2, lam, norm_r):
    """c[c3, b, a] = sigma2 exp(-||(d_a h, d_b h, d_c h)||_r / lam) on the M^3
    torus of cell-centre offsets, d_a = min(a, M - a), h = 1/m."""
    a = np.arange(M)
    d = np.minimum(a, M - a) / m
    dx, dy, dz = d[None, None, :], d[None, :, None], d[:, None, None]
    if norm_r == 1:
        dist = np.abs(dx) + np.abs(dy) + np.abs(dz)
    else:
        dist = np.sqrt(dx * dx + dy * dy + dz * dz)
    return sigma2 * np.exp(-dist / lam)


def ce_eigenvalues3(m, M, sigma2, lam, norm_r):
    """Eigenvalues of the embedding: the unnormalised forward 3-D DFT of the
    torus covariance (real: c is even in every axis)."""
    return np.fft.fftn(covariance_torus3(m, M, sigma2, lam, norm_r)).real


def ce_padding3(m, sigma2, lam, norm_r):
    """Smallest M = p m, p in {2, 4, 8, 16}, with every eigenvalue >= -1e-13
    max (the 2-D rule); returns (M, eigenvalues clipped to >= 0)."""
    p = 2
    while True:
        M = p * m
        lam_q = ce_eigenvalues3(m, M, sigma2, lam, norm_r)
        ok = lam_q.min() >= -darcy.CE_NEG_TOL * lam_q.max()
        if ok or p >= darcy.CE_MAX_PAD:
            if not ok:
                raise ValueError("circulant embedding not non-negative at p=%d" % p)
            return M, np.maximum(lam_q, 0.0)
        p *= 2


def ce_pair3(lam_q, xi, m):
    """Two independent fields on the m^3 cell centres from one complex draw:
    y[c, b, a] = sum_q sqrt(Lambda_q / M^3) xi_q exp(-2 pi i (a q1 + b q2 + c q3)/M);
    returns (Re y, Im y) cropped to the first m^3 entries."""
    M = lam_q.shape[0]
    y = np.fft.fftn(np.sqrt(lam_q / float(M) ** 3) * xi)
    return y.real[:m, :m, :m], y.imag[:m, :m, :m]


def layer_fields3(model, seed, level, sample, m, ce_cache=None):
    """Per-layer fields g[t, l, j, i]: Ex. 1 constants or Ex. 2 CE fields (the
    draws paired with the layers as in 2-D, darcy.field_slots)."""
    nl = model.n_layers
    g = np.empty((nl, m, m, m))
    if model.k_kind == 0:
        z = philox.layer_normals(seed, level, sample, nl)
        for t in range(nl):
            g[t] = model.mu[t] + np.sqrt(model.sigma2[t]) * z[t]
        return g
    slots, params = darcy.field_slots(model)
    for f, (sigma2, lam) in enumerate(params):
        key = (3, m, sigma2, lam, model.norm_r)
        if ce_cache is not None and key in ce_cache:
            M, lam_q = ce_cache[key]
        else:
            M, lam_q = ce_padding3(m, sigma2, lam, model.norm_r)
            if ce_cache is not None:
                ce_cache[key] = (M, lam_q)
        xi = philox.field_normals(seed, level, sample, f, M, dim=3)
        parts = ce_pair3(lam_q, xi, m)
        for t in range(nl):
            if slots[t][0] == f:
                g[t] = model.mu[t] + parts[slots[t][1]]
    return g


def compose_k3(g, layers):
    """k[l, j, i] = exp(g[layers[l, j, i], l, j, i])."""
    m = g.shape[1]
    ll, jj, ii = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    return np.exp(g[layers, ll, jj, ii])


# ----------------------------------------------------------------- TPFA -----
def transmissibilities3(k, problem=2):
    """Face coefficients (divided by h) of the seven-point system.

    tx[l, j, i'] for the faces x1 = i'/m: interior 2 k_a k_b / (k_a + k_b),
    Dirichlet faces i' = 0, m: 2 k_cell.
    ty[l, j', i] (faces x2 = j'/m) and tz[l', j, i] (faces x3 = l'/m): interior
    harmonic; boundary faces 0 (no flow, Model Problem 2) or 2 k_cell
    (Dirichlet, Model Problem 1)."""
    m = k.shape[0]
    tx = np.zeros((m, m, m + 1))
    ty = np.zeros((m, m + 1, m))
    tz = np.zeros((m + 1, m, m))
    ka, kb = k[:, :, :-1], k[:, :, 1:]
    tx[:, :, 1:m] = 2.0 * ka * kb / (ka + kb)
    tx[:, :, 0] = 2.0 * k[:, :, 0]
    tx[:, :, m] = 2.0 * k[:, :, m - 1]
    ka, kb = k[:, :-1, :], k[:, 1:, :]
    ty[:, 1:m, :] = 2.0 * ka * kb / (ka + kb)
    ka, kb = k[:-1, :, :], k[1:, :, :]
    tz[1:m, :, :] = 2.0 * ka * kb / (ka + kb)
    if problem == 1:
        ty[:, 0, :] = 2.0 * k[:, 0, :]
        ty[:, m, :] = 2.0 * k[:, m - 1, :]
        tz[0, :, :] = 2.0 * k[0, :, :]
        tz[m, :, :] = 2.0 * k[m - 1, :, :]
    return tx, ty, tz


def rhs3(tx, problem=2):
    """Right-hand side (divided by h).  Model Problem 2: the Dirichlet value
    p = 1 at x1 = 0 through the faces i' = 0.  Model Problem 1: f h^3 / h =
    1/m^2 in every cell."""
    m = tx.shape[0]
    if problem == 1:
        return np.full((m, m, m), 1.0 / (m * m))
    b = np.zeros((m, m, m))
    b[:, :, 0] = tx[:, :, 0]
    return b


def matrix3(tx, ty, tz):
    """The SPD seven-point matrix (scipy sparse CSR), unknown n = (l m + j) m + i."""
    m = tx.shape[0]
    n = m ** 3
    idx = np.arange(n).reshape(m, m, m)
    diag = (tx[:, :, :m] + tx[:, :, 1:]) + (ty[:, :m, :] + ty[:, 1:, :]) + (tz[:m] + tz[1:])
    rows, cols, vals = [idx.reshape(-1)], [idx.reshape(-1)], [diag.reshape(-1)]
    couplings = ((idx[:, :, :-1], idx[:, :, 1:], tx[:, :, 1:m]),
                 (idx[:, :-1, :], idx[:, 1:, :], ty[:, 1:m, :]),
                 (idx[:-1, :, :], idx[1:, :, :], tz[1:m, :, :]))
    for a, b, t in couplings:
        rows += [a.reshape(-1), b.reshape(-1)]
        cols += [b.reshape(-1), a.reshape(-1)]
        vals += [-t.reshape(-1), -t.reshape(-1)]
    return scipy.sparse.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                   shape=(n, n))


def solve_direct3(tx, ty, tz, b):
    """Direct sparse LU solve (SuperLU) of the seven-point system."""
    m = tx.shape[0]
    A = matrix3(tx, ty, tz).tocsc()
    return scipy.sparse.linalg.splu(A).solve(b.reshape(-1)).reshape(m, m, m)


def outflow3(tx, p):
    """M^(2): outflow through x1 = 1, h * sum over the faces of tx * p(m-1)."""
    m = tx.shape[0]
    return float(np.sum(tx[:, :, -1] * p[:, :, -1])) / m


def inflow3(tx, p):
    """Inflow through x1 = 0, h * sum over the faces of tx * (1 - p(0))."""
    m = tx.shape[0]
    return float(np.sum(tx[:, :, 0] * (1.0 - p[:, :, 0]))) / m


def box_weights3(m, box):
    """Weights w[l, j, i] = |cell & D*| / |D*| of D* = [x0, x1] x [y0, y1] x
    [y0, y1] (the box's x2 range also bounds x3)."""
    x0, x1, y0, y1 = box
    e = np.arange(m + 1) / m
    ox = np.clip(np.minimum(e[1:], x1) - np.maximum(e[:-1], x0), 0.0, None)
    oy = np.clip(np.minimum(e[1:], y1) - np.maximum(e[:-1], y0), 0.0, None)
    return (oy[:, None, None] * oy[None, :, None] * ox[None, None, :]) / ((x1 - x0) * (y1 - y0) * (y1 - y0))


def solve_k3(k, problem=2, box=(7 / 16, 9 / 16, 7 / 16, 9 / 16)):
    """Assemble and solve for one permeability array k[l, j, i]; returns (p, Q)."""
    tx, ty, tz = transmissibilities3(k, problem)
    p = solve_direct3(tx, ty, tz, rhs3(tx, problem))
    q = float(np.sum(box_weights3(k.shape[0], box) * p)) if problem == 1 else outflow3(tx, p)
    return p, q


# ------------------------------------------------------- one MLMC sample ----
def coarse_samples3(model, g_fine, k_fine, ends, mode):
    """Coarse permeability arrays of the level below (Eq. 4.1, d = 3): mode 0
    one sample at offset (0, 0, 0); mode 1 the 8 strided sub-samples of the
    per-layer fields composed with the coarse layer map; mode 2 those of the
    composed k."""
    m = g_fine.shape[1]
    lay_c = layer_map3(model, ends, m // 2)
    offsets = CGV_OFFSETS3[:1] if mode == 0 else CGV_OFFSETS3
    out = []
    for ox, oy, oz in offsets:
        if mode == 2:
            out.append(k_fine[oz::2, oy::2, ox::2].copy())
        else:
            out.append(compose_k3(g_fine[:, oz::2, oy::2, ox::2], lay_c))
    return out


def sample(model, seed, level, i, ce_cache=None, want_fields=False):
    """Q_l and the coarse Q's of sample i at level l in 3-D; the same dict as
    darcy.sample (qc_cgv is the mean of the 8 coarse Q's in CGV_OFFSETS3
    order, summed left to right)."""
    m = model.m(level)
    ends = darcy.interfaces(model, seed, level, i)
    lay = layer_map3(model, ends, m)
    g = layer_fields3(model, seed, level, i, m, ce_cache)
    k = compose_k3(g, lay)
    prob = 1 if model.problem == 1 else 2
    box = tuple(model.qoi_box)
    p, qf = solve_k3(k, prob, box)
    out = {"qf": qf, "qc": 0.0, "qc_cgv": float("nan"), "eta": ends,
           "inflow": inflow3(transmissibilities3(k)[0], p)}
    if want_fields:
        out.update(g=g, k=k, p=p)
    if level > 0:
        if model.cgv == 0:
            (kc,) = coarse_samples3(model, g, k, ends, 0)
            out["qc"] = solve_k3(kc, prob, box)[1]
        else:
            qcs = [solve_k3(kc, prob, box)[1] for kc in coarse_samples3(model, g, k, ends, model.cgv)]
            acc = qcs[0]
            for q in qcs[1:]:
                acc = acc + q
            out["qc"] = qcs[0]
            out["qc_cgv"] = 0.125 * acc
            out["qc_each"] = qcs
    elif model.cgv != 0:
        out["qc_cgv"] = 0.0
    return out

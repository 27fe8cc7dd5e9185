// Fused assembly + multigrid-preconditioned CG + QoI for the 3-D medium of
// Sec. 3.4 (the 2-D layers extruded along x3), one thread block or one
// thread-block cluster per linear system, many systems per launch.
//
// System of one sample (Sec. 3.1 Eq. 3.3 in 3-D, divided by h): unknown p on
// m^3 cells, sum_faces T_f (p_c - p_nbr) = b_c with T = 2 k_a k_b / (k_a +
// k_b) inside, T = 2 k_c on the Dirichlet faces (x1 = 0, 1; every boundary
// face for Model Problem 1), T = 0 on the no-flow faces of Model Problem 2.
// Outflow QoI M^(2) = h sum over the faces x1 = 1 of T p(m-1, j, l).
// Multigrid as in 2-D, in three dimensions: 2x2x2 aggregation, a coarse face
// coefficient is half the sum of the four fine faces it covers (the
// rediscretisation of a constant k with faces of area h^2 over h), red-black
// Gauss-Seidel with colour (i + j + l) mod 2, restriction = sum of the fine
// residuals (only the four red cells of an aggregate are nonzero after a
// black half sweep), piecewise-constant prolongation, exact 1x1x1 solve.
// prec 0: FP64 throughout; prec 1: FP32 CG and multigrid inside FP64
// iterative refinement (FP64 residual, solution, stopping test and QoI).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "../../include/mlmc.h"
#include "common.cuh"
#include "groups.cuh"
#include "kernels.cuh"
#include "layers.cuh"

namespace mlmc {
namespace {

constexpr int kMaxLevels3 = 9;  // m <= 128: 128, 64, ..., 1
constexpr int kMaxThreads3 = 512;

__host__ __device__ __forceinline__ size_t align16_3(size_t v) { return (v + 15) & ~(size_t)15; }

// Workspace bytes of an m^3 system in the order solve_one3() lays it out:
// prec 1: FP64 x and r; per level: faces tx, ty, tz (m^2 (m + 1) each), diag,
// invd, e, f (m^3 each), in the solver type; after level 0 the CG vectors
// x, p, q.  Each array starts 16-byte aligned.
__host__ __device__ inline size_t ws3_layout(int m, int prec) {
  const size_t ts = prec ? 4 : 8;
  const size_t n = (size_t)m * m * m;
  size_t o = 0;
  auto take = [&](size_t bytes) { o += align16_3(bytes); };
  if (prec) {
    take(n * 8);
    take(n * 8);
  }
  for (int ml = m, l = 0;; ml >>= 1, ++l) {
    const size_t nl = (size_t)ml * ml * ml, nf = (size_t)ml * ml * (ml + 1);
    for (int a = 0; a < 3; ++a) take(nf * ts);
    for (int a = 0; a < 4; ++a) take(nl * ts);
    if (l == 0)
      for (int b = 0; b < 3; ++b) take(nl * ts);
    if (ml == 1) break;
  }
  return o;
}

// Cell c = (l m + j) m + i.  Faces: tx[(l m + j)(m + 1) + i'] (x1 = i'/m),
// ty[(l (m + 1) + j') m + i] (x2 = j'/m), tz[(l' m + j) m + i] (x3 = l'/m).
template <typename T>
struct Level3 {
  int m;
  T *tx, *ty, *tz;
  T* diag;
  T* invd;
  T* e;  // correction (level 0: CG z)
  T* f;  // right-hand side (level 0: CG r)
};

template <typename T>
__device__ __forceinline__ T apply3(const Level3<T>& L, const T* __restrict__ v, int i, int j, int l) {
  const int m = L.m, m2 = m * m;
  const int c = (l * m + j) * m + i;
  const int rx = (l * m + j) * (m + 1) + i;
  const int ry = (l * (m + 1) + j) * m + i;
  T s = L.diag[c] * v[c];
  if (i > 0) s -= L.tx[rx] * v[c - 1];
  if (i < m - 1) s -= L.tx[rx + 1] * v[c + 1];
  if (j > 0) s -= L.ty[ry] * v[c - m];
  if (j < m - 1) s -= L.ty[ry + m] * v[c + m];
  if (l > 0) s -= L.tz[c] * v[c - m2];
  if (l < m - 1) s -= L.tz[c + m2] * v[c + m2];
  return s;
}

// Red (colour 0, i + j + l even) or black half sweep; zero_guess treats the
// other colour as zero.
template <typename T, typename G>
__device__ __forceinline__ void rb_sweep3(const G& g, const Level3<T>& L, int color, bool zero_guess) {
  const int m = L.m, hm = m >> 1, m2 = m * m;
  const int plane = m * hm, nh = m * plane;
  for (int h = g.rank(); h < nh; h += g.size()) {
    const int l = h / plane;
    const int r = h - l * plane;
    const int j = r / hm;
    const int i = ((r - j * hm) << 1) + ((j + l + color) & 1);
    const int c = (l * m + j) * m + i;
    T s = L.f[c];
    if (!zero_guess) {
      const int rx = (l * m + j) * (m + 1) + i;
      const int ry = (l * (m + 1) + j) * m + i;
      if (i > 0) s += L.tx[rx] * L.e[c - 1];
      if (i < m - 1) s += L.tx[rx + 1] * L.e[c + 1];
      if (j > 0) s += L.ty[ry] * L.e[c - m];
      if (j < m - 1) s += L.ty[ry + m] * L.e[c + m];
      if (l > 0) s += L.tz[c] * L.e[c - m2];
      if (l < m - 1) s += L.tz[c + m2] * L.e[c + m2];
    }
    L.e[c] = s * L.invd[c];
  }
  g.sync();
}

// Coarse f = sum of the fine residuals over each 2x2x2 aggregate; called
// after a black half sweep, so only the red cells (0,0,0), (1,1,0), (1,0,1),
// (0,1,1) of the aggregate contribute.
template <typename T, typename G>
__device__ __forceinline__ void restrict3(const G& g, const Level3<T>& F, const Level3<T>& C) {
  const int mc = C.m, m = F.m;
  const int nc = mc * mc * mc;
  for (int cc = g.rank(); cc < nc; cc += g.size()) {
    const int K = cc / (mc * mc);
    const int r = cc - K * mc * mc;
    const int J = r / mc, I = r - J * mc;
    const int i0 = 2 * I, j0 = 2 * J, l0 = 2 * K;
    auto res = [&](int i, int j, int l) { return F.f[(l * m + j) * m + i] - apply3(F, F.e, i, j, l); };
    C.f[cc] = (res(i0, j0, l0) + res(i0 + 1, j0 + 1, l0)) + (res(i0 + 1, j0, l0 + 1) + res(i0, j0 + 1, l0 + 1));
  }
  g.sync();
}

template <typename T, typename G>
__device__ __forceinline__ void prolong3(const G& g, const Level3<T>& C, const Level3<T>& F) {
  const int m = F.m, mc = C.m;
  const int n = m * m * m;
  for (int c = g.rank(); c < n; c += g.size()) {
    const int l = c / (m * m);
    const int r = c - l * m * m;
    const int j = r / m, i = r - j * m;
    F.e[c] += C.e[((l >> 1) * mc + (j >> 1)) * mc + (i >> 1)];
  }
  g.sync();
}

// Coarse faces: half the sum of the four fine faces that make up each one.
template <typename T, typename G>
__device__ __forceinline__ void build_coarse3(const G& g, const Level3<T>& F, const Level3<T>& C) {
  const int m = F.m, mc = C.m;
  const int nf = mc * mc * (mc + 1);
  for (int t = g.rank(); t < 3 * nf; t += g.size()) {
    const int axis = t / nf, u = t - axis * nf;
    if (axis == 0) {  // tx[(K mc + J)(mc + 1) + I']
      const int KJ = u / (mc + 1), Ip = u - KJ * (mc + 1);
      const int K = KJ / mc, J = KJ - K * mc;
      T s = T(0);
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) s += F.tx[((2 * K + b) * m + 2 * J + a) * (m + 1) + 2 * Ip];
      C.tx[u] = T(0.5) * s;
    } else if (axis == 1) {  // ty[(K (mc + 1) + J') mc + I]
      const int KJ = u / mc, I = u - KJ * mc;
      const int K = KJ / (mc + 1), Jp = KJ - K * (mc + 1);
      T s = T(0);
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) s += F.ty[((2 * K + b) * (m + 1) + 2 * Jp) * m + 2 * I + a];
      C.ty[u] = T(0.5) * s;
    } else {  // tz[(K' mc + J) mc + I]
      const int KJ = u / mc, I = u - KJ * mc;
      const int Kp = KJ / mc, J = KJ - Kp * mc;
      T s = T(0);
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) s += F.tz[((2 * Kp) * m + 2 * J + b) * m + 2 * I + a];
      C.tz[u] = T(0.5) * s;
    }
  }
  g.sync();
}

template <typename T, typename G>
__device__ __forceinline__ void build_diag3(const G& g, const Level3<T>& L) {
  const int m = L.m, m2 = m * m, n = m2 * m;
  for (int c = g.rank(); c < n; c += g.size()) {
    const int l = c / m2;
    const int r = c - l * m2;
    const int j = r / m, i = r - j * m;
    const int rx = (l * m + j) * (m + 1) + i;
    const int ry = (l * (m + 1) + j) * m + i;
    const T d = ((L.tx[rx] + L.tx[rx + 1]) + (L.ty[ry] + L.ty[ry + m])) + (L.tz[c] + L.tz[c + m2]);
    L.diag[c] = d;
    L.invd[c] = T(1) / d;
  }
  g.sync();
}

// Symmetric multigrid cycle e_0 <- B f_0 (red-black then black-red smoothing,
// nu sweep pairs on the finest level and nuc on the coarser ones, gamma
// visits of the next level per visit, one when it is the 1x1x1 grid, solved
// exactly), written as a loop over per-level visit counts.
template <typename T, typename G>
__device__ void mg_cycle3(const G& g, const Level3<T>* lev, int nl, int gamma, int nu, int nuc) {
  int done[kMaxLevels3];
  bool zero[kMaxLevels3];
  int l = 0;
  zero[0] = true;
  while (true) {
    if (l < nl - 1) {
      const int ns = l == 0 ? nu : nuc;
      for (int s = 0; s < ns; ++s) {
        rb_sweep3(g, lev[l], 0, zero[l] && s == 0);
        rb_sweep3(g, lev[l], 1, false);
      }
      restrict3(g, lev[l], lev[l + 1]);
      done[l] = 0;
      zero[l + 1] = true;
      ++l;
      continue;
    }
    {
      const Level3<T>& Lc = lev[l];
      if (g.rank() == 0) Lc.e[0] = Lc.f[0] * Lc.invd[0];
      g.sync();
    }
    bool revisit = false;
    while (l > 0) {
      const int up = l - 1;
      const int visits = (up + 1 == nl - 1) ? 1 : gamma;
      if (++done[up] < visits) {
        zero[l] = false;
        revisit = true;
        break;
      }
      prolong3(g, lev[l], lev[up]);
      const int ns = up == 0 ? nu : nuc;
      for (int s = 0; s < ns; ++s) {
        rb_sweep3(g, lev[up], 1, false);
        rb_sweep3(g, lev[up], 0, false);
      }
      l = up;
    }
    if (!revisit) return;
  }
}

// Preconditioned CG on the level-0 operator (r = lev[0].f on entry, z =
// lev[0].e, x set to 0 here); stops when r.r <= thr; status 0 converged, 1 the
// iteration cap, 2 breakdown.
template <typename T, typename G>
__device__ int pcg3(const G& g, const Level3<T>* lev, int nl, int gamma, int nu, int nuc, T* __restrict__ x,
                    T* __restrict__ p, T* __restrict__ q, T thr, int max_it, T* red, int& par, int& status) {
  const Level3<T>& L0 = lev[0];
  const int m = L0.m, m2 = m * m, n = m2 * m;
  T* __restrict__ r = L0.f;
  const T* __restrict__ z = L0.e;
  const int step = g.size();
  if (nuc < 1) nuc = nu;
  T rr = T(0);
  for (int c = g.rank(); c < n; c += step) {
    x[c] = T(0);
    rr += r[c] * r[c];
  }
  rr = g.sum(rr, red, par);
  status = 1;
  if (rr <= thr) {
    status = 0;
    return 0;
  }
  mg_cycle3(g, lev, nl, gamma, nu, nuc);
  T rz = T(0);
  for (int c = g.rank(); c < n; c += step) {
    p[c] = z[c];
    rz += r[c] * z[c];
  }
  rz = g.sum(rz, red, par);
  int it = 0;
  while (it < max_it) {
    ++it;
    T pq = T(0);
    for (int c = g.rank(); c < n; c += step) {
      const int l = c / m2;
      const int rem = c - l * m2;
      const int j = rem / m, i = rem - j * m;
      const T v = apply3(L0, p, i, j, l);
      q[c] = v;
      pq += p[c] * v;
    }
    pq = g.sum(pq, red, par);
    if (!(pq > T(0)) || !isfinite(pq) || !isfinite(rz)) {
      status = 2;
      break;
    }
    const T alpha = rz / pq;
    rr = T(0);
    for (int c = g.rank(); c < n; c += step) {
      x[c] += alpha * p[c];
      const T rv = r[c] - alpha * q[c];
      r[c] = rv;
      rr += rv * rv;
    }
    rr = g.sum(rr, red, par);
    if (rr <= thr) {
      status = 0;
      break;
    }
    mg_cycle3(g, lev, nl, gamma, nu, nuc);
    T rzn = T(0);
    for (int c = g.rank(); c < n; c += step) rzn += r[c] * z[c];
    rzn = g.sum(rzn, red, par);
    const T beta = rzn / rz;
    rz = rzn;
    for (int c = g.rank(); c < n; c += step) p[c] = z[c] + beta * p[c];
    g.sync();
  }
  return it;
}

template <typename T>
struct GroupState3 {
  Level3<T> lev[kMaxLevels3];
  T *xv, *pv, *qv;
  double *x64, *r64;
  double eta[MAX_LAYERS_DEV], kc[MAX_LAYERS_DEV];
  int nl;
};

// Assemble, solve and reduce the QoI of one 3-D system with group g.
// Systems [0, n_samples) are fine; then n_coarse per sample with offset
// o = ox + 2 oy + 4 oz.
template <bool MIXED, typename G>
__device__ void solve_one3(const G& g, const SolveArgs& a, int64_t sys, unsigned char* base,
                           GroupState3<typename std::conditional<MIXED, float, double>::type>& gs,
                           typename std::conditional<MIXED, float, double>::type* red, double* red64, int& par,
                           int& m_prev, unsigned char* base64) {
  using T = typename std::conditional<MIXED, float, double>::type;
  int64_t sidx;
  int coarse = 0, ox = 0, oy = 0, oz = 0;
  if (sys < a.n_samples) {
    sidx = sys;
  } else {
    const int64_t t = sys - a.n_samples;
    sidx = t / a.n_coarse;
    const int o = (int)(t - sidx * a.n_coarse);
    coarse = 1;
    ox = o & 1;
    oy = (o >> 1) & 1;
    oz = o >> 2;
  }
  const int m = coarse ? a.m >> 1 : a.m;
  const int m2 = m * m, n = m2 * m;
  const uint64_t sample = (uint64_t)(a.first + sidx);
  if (m != m_prev) {  // level table of this system size (each block keeps its copy)
    g.sync();
    if (g.local_leader()) {
      size_t o = 0;
      const size_t n0 = (size_t)n;
      auto take = [&](size_t bytes) {
        unsigned char* p = base + o;
        o += align16_3(bytes);
        return p;
      };
      if (MIXED) {
        if (base64) {  // FP64 refinement vectors in global memory, the rest on chip
          gs.x64 = reinterpret_cast<double*>(base64);
          gs.r64 = reinterpret_cast<double*>(base64 + align16_3(n0 * 8));
        } else {
          gs.x64 = reinterpret_cast<double*>(take(n0 * 8));
          gs.r64 = reinterpret_cast<double*>(take(n0 * 8));
        }
      }
      int l = 0;
      for (int ml = m;; ml >>= 1, ++l) {
        const size_t nlv = (size_t)ml * ml * ml, nf = (size_t)ml * ml * (ml + 1);
        Level3<T>& L = gs.lev[l];
        L.m = ml;
        L.tx = reinterpret_cast<T*>(take(nf * sizeof(T)));
        L.ty = reinterpret_cast<T*>(take(nf * sizeof(T)));
        L.tz = reinterpret_cast<T*>(take(nf * sizeof(T)));
        L.diag = reinterpret_cast<T*>(take(nlv * sizeof(T)));
        L.invd = reinterpret_cast<T*>(take(nlv * sizeof(T)));
        L.e = reinterpret_cast<T*>(take(nlv * sizeof(T)));
        L.f = reinterpret_cast<T*>(take(nlv * sizeof(T)));
        if (l == 0) {
          gs.xv = reinterpret_cast<T*>(take(nlv * sizeof(T)));
          gs.pv = reinterpret_cast<T*>(take(nlv * sizeof(T)));
          gs.qv = reinterpret_cast<T*>(take(nlv * sizeof(T)));
        }
        if (ml == 1) break;
      }
      gs.nl = l + 1;
      if (!MIXED) {
        gs.x64 = reinterpret_cast<double*>(gs.xv);
        gs.r64 = reinterpret_cast<double*>(gs.lev[0].f);
      }
    }
    g.sync();
    m_prev = m;
  }
  const int nl = gs.nl;
  T* xv = gs.xv;
  T* pv = gs.pv;
  T* qv = gs.qv;
  double* x64 = gs.x64;
  double* r64 = gs.r64;
  const Level3<T>* lev = gs.lev;
  const Level3<T>& L0 = lev[0];

  // ---- layers and per-cell permeability (into r64 as scratch) ----
  if (a.ksrc != KSRC_ARRAY) {
    if (g.local_leader()) sample_layers(a, sample, gs.eta, gs.kc);
    g.sync();
  }
  const int n_if = a.geometry == 1 ? 0 : a.n_layers - 1;
  const int mf = a.m;
  // m and mf are powers of two: scaling by the reciprocal is exact
  const double inv_m = 1.0 / (double)m, inv_mf = 1.0 / (double)mf;
  for (int c = g.rank(); c < n; c += g.size()) {
    const int l = c / m2;
    const int rem = c - l * m2;
    const int j = rem / m, i = rem - j * m;
    double kk;
    if (a.ksrc == KSRC_ARRAY) {
      kk = a.k[sys * (int64_t)n + c];
    } else {
      const int jf = coarse ? 2 * j + oy : j;
      const int iff = coarse ? 2 * i + ox : i;
      const int lf = coarse ? 2 * l + oz : l;
      const bool own = coarse && !a.cgv_on_k;  // layer at the coarse centre
      const double yc = own ? ((double)j + 0.5) * inv_m : ((double)jf + 0.5) * inv_mf;
      const double xc = own ? ((double)i + 0.5) * inv_m : ((double)iff + 0.5) * inv_mf;
      const int t = layer_at_point(a.geometry, gs.eta, n_if, xc, yc);
      const int64_t gi = (((sidx * a.n_layers + t) * (int64_t)mf + lf) * mf + jf) * mf + iff;
      if (a.ksrc == KSRC_CONST) kk = gs.kc[t];
      else if (MIXED) kk = (double)expf(reinterpret_cast<const float*>(a.g)[gi]);
      else kk = exp(reinterpret_cast<const double*>(a.g)[gi]);
    }
    r64[c] = kk;
  }
  g.sync();
  // ---- faces (Eq. 3.3 in 3-D, harmonic averages; Dirichlet 2k; no-flow 0) ----
  {
    const int nf = m2 * (m + 1);
    for (int t = g.rank(); t < 3 * nf; t += g.size()) {
      const int axis = t / nf, u = t - axis * nf;
      T v = T(0);
      if (axis == 0) {
        const int lj = u / (m + 1), ip = u - lj * (m + 1);
        const int cb = lj * m;  // cell (0, j, l)
        if (ip == 0) v = T(2) * (T)r64[cb];
        else if (ip == m) v = T(2) * (T)r64[cb + m - 1];
        else {
          const T ka = (T)r64[cb + ip - 1], kb = (T)r64[cb + ip];
          v = T(2) * ka * kb / (ka + kb);
        }
        L0.tx[u] = v;
      } else if (axis == 1) {
        const int lj = u / m, i = u - lj * m;
        const int l = lj / (m + 1), jp = lj - l * (m + 1);
        if (jp > 0 && jp < m) {
          const T ka = (T)r64[(l * m + jp - 1) * m + i], kb = (T)r64[(l * m + jp) * m + i];
          v = T(2) * ka * kb / (ka + kb);
        } else if (a.problem == 1) {
          v = T(2) * (T)r64[(l * m + (jp == 0 ? 0 : m - 1)) * m + i];
        }
        L0.ty[u] = v;
      } else {
        const int lp = u / m2, ji = u - lp * m2;
        if (lp > 0 && lp < m) {
          const T ka = (T)r64[(lp - 1) * m2 + ji], kb = (T)r64[lp * m2 + ji];
          v = T(2) * ka * kb / (ka + kb);
        } else if (a.problem == 1) {
          v = T(2) * (T)r64[(lp == 0 ? 0 : m - 1) * m2 + ji];
        }
        L0.tz[u] = v;
      }
    }
    g.sync();
    build_diag3(g, L0);
  }
  for (int l = 1; l < nl; ++l) {
    build_coarse3(g, lev[l - 1], lev[l]);
    build_diag3(g, lev[l]);
  }
  // ---- solve ----
  const int nuc = a.mg_nu_coarse > 0 ? a.mg_nu_coarse : a.mg_nu;
  int status = 1, iters = 0;
  const double fmid = 1.0 / ((double)m * (double)m);  // Model Problem 1: f h^3 / h
  if (!MIXED) {
    T bb = T(0);
    for (int c = g.rank(); c < n; c += g.size()) {
      const int i = c % m;
      const T bv = a.problem == 1 ? (T)fmid : (i == 0 ? L0.tx[(c / m) * (m + 1)] : T(0));
      L0.f[c] = bv;
      bb += bv * bv;
    }
    bb = g.sum(bb, red, par);
    iters = pcg3(g, lev, nl, a.mg_gamma, a.mg_nu, nuc, xv, pv, qv, (T)(a.tol * a.tol) * bb, a.max_it, red, par,
                 status);
  } else {
    // FP64 refinement: r64 = b - A64 x64 with A64 = the FP32 faces in FP64.
    double bb = 0.0;
    for (int c = g.rank(); c < n; c += g.size()) {
      const int i = c % m;
      const double bv = a.problem == 1 ? fmid : (i == 0 ? (double)L0.tx[(c / m) * (m + 1)] : 0.0);
      x64[c] = 0.0;
      r64[c] = bv;
      bb += bv * bv;
    }
    bb = g.sum(bb, red64, par);
    double rr = bb;
    const double thr = a.tol * a.tol * bb;
    int sweeps = 0;
    while (true) {
      if (rr <= thr) {
        status = 0;
        break;
      }
      if (iters >= a.max_it || sweeps >= 40) {
        status = 1;
        break;
      }
      ++sweeps;
      const double inv = 1.0 / sqrt(rr);
      const double scl = sqrt(rr);
      T r32 = T(0);
      for (int c = g.rank(); c < n; c += g.size()) {
        const T v = (T)(r64[c] * inv);
        L0.f[c] = v;
        r32 += v * v;
      }
      r32 = g.sum(r32, red, par);
      int st_in = 1;
      const T thr_in = (T)(a.inner_tol * a.inner_tol) * r32;
      const int it = pcg3(g, lev, nl, a.mg_gamma, a.mg_nu, nuc, xv, pv, qv, thr_in, a.max_it - iters, red, par,
                          st_in);
      iters += it;
      for (int c = g.rank(); c < n; c += g.size()) x64[c] += scl * (double)xv[c];
      g.sync();
      rr = 0.0;
      for (int c = g.rank(); c < n; c += g.size()) {
        const int l = c / m2;
        const int rem = c - l * m2;
        const int j = rem / m, i = rem - j * m;
        const int rx = (l * m + j) * (m + 1) + i;
        const int ry = (l * (m + 1) + j) * m + i;
        const double tw = (double)L0.tx[rx], te = (double)L0.tx[rx + 1];
        const double ts = (double)L0.ty[ry], tn = (double)L0.ty[ry + m];
        const double tb = (double)L0.tz[c], tt = (double)L0.tz[c + m2];
        double ax = (((tw + te) + (ts + tn)) + (tb + tt)) * x64[c];
        if (i > 0) ax -= tw * x64[c - 1];
        if (i < m - 1) ax -= te * x64[c + 1];
        if (j > 0) ax -= ts * x64[c - m];
        if (j < m - 1) ax -= tn * x64[c + m];
        if (l > 0) ax -= tb * x64[c - m2];
        if (l < m - 1) ax -= tt * x64[c + m2];
        const double bv = a.problem == 1 ? fmid : (i == 0 ? tw : 0.0);
        const double rv = bv - ax;
        r64[c] = rv;
        rr += rv * rv;
      }
      rr = g.sum(rr, red64, par);
      if (it == 0 && st_in != 0) {
        status = 2;
        break;
      }
    }
  }
  // ---- QoI and outputs ----
  double qsum = 0.0;
  const double h = 1.0 / (double)m;
  if (a.problem == 1) {
    // M^(1): sum over cells of |cell & D*| / |D*| p, D* = [x0,x1] x [y0,y1] x [y0,y1]
    const double inv_vol = 1.0 / ((a.box[1] - a.box[0]) * (a.box[3] - a.box[2]) * (a.box[3] - a.box[2]));
    for (int c = g.rank(); c < n; c += g.size()) {
      const int l = c / m2;
      const int rem = c - l * m2;
      const int j = rem / m, i = rem - j * m;
      const double wx = fmin((i + 1) * h, a.box[1]) - fmax(i * h, a.box[0]);
      const double wy = fmin((j + 1) * h, a.box[3]) - fmax(j * h, a.box[2]);
      const double wz = fmin((l + 1) * h, a.box[3]) - fmax(l * h, a.box[2]);
      if (wx > 0.0 && wy > 0.0 && wz > 0.0) qsum += wx * wy * wz * inv_vol * x64[c];
    }
  } else {
    // M^(2): h times the flux sum over the faces x1 = 1
    for (int lj = g.rank(); lj < m2; lj += g.size())
      qsum += (double)L0.tx[lj * (m + 1) + m] * x64[lj * m + m - 1];
  }
  qsum = g.sum(qsum, red64, par);
  if (a.problem != 1) qsum *= h;
  if (g.rank() == 0) {
    a.q[sys] = status == 0 ? qsum : nan("");
    if (a.iters) a.iters[sys] = iters;
  }
  if (a.p_out && !coarse)
    for (int c = g.rank(); c < n; c += g.size()) a.p_out[sidx * (int64_t)n + c] = x64[c];
  g.sync();
}

constexpr int kWarpsPerBlock3 = 4;  // systems per block in warp mode

// MODE 0: one block per system; 1: one warp per system (kWarpsPerBlock3
// systems per block, no block barriers); 2: one thread-block cluster per
// system.
template <bool MIXED, int MODE>
__global__ void __launch_bounds__(MODE == 1 ? 32 * kWarpsPerBlock3 : kMaxThreads3, MODE == 1 ? 5 : 2)
    solve3_kernel(SolveArgs a) {
  using T = typename std::conditional<MIXED, float, double>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kGroups = MODE == 1 ? kWarpsPerBlock3 : 1;
  __shared__ GroupState3<T> gstates[kGroups];
  GroupState3<T>& gstate = gstates[0];
  __shared__ T red[MODE == 1 ? 1 : 132];
  __shared__ double red64[MODE == 1 ? 1 : 132];
  const int64_t n_all = a.n_samples * (int64_t)(1 + a.n_coarse);
  const int64_t sys0 = a.sys_begin, n_sys = a.sys_end > 0 ? a.sys_end : n_all;
  int par = 0, m_prev = -1;
  if (MODE == 2) {
    __shared__ double cl_part[2];
    cg::cluster_group cl = cg::this_cluster();
    const ClusterGroup g{cl.num_blocks(), cl.block_rank(), cl_part};
    const int64_t cid = blockIdx.x / g.nblk, ncl = gridDim.x / g.nblk;
    unsigned char* base = a.ws + (size_t)cid * a.ws_stride;
    for (int64_t sys = sys0 + cid; sys < n_sys; sys += ncl)
      solve_one3<MIXED>(g, a, sys, base, gstate, red, red64, par, m_prev, nullptr);
    cl.sync();  // no block leaves while others may still read its shared memory
    return;
  }
  const int gid = MODE == 1 ? (int)(threadIdx.x >> 5) : 0;
  const size_t slot = (size_t)blockIdx.x * kGroups + gid;
  unsigned char* base = a.use_smem ? smem_raw + (size_t)gid * a.ws_stride : a.ws + slot * a.ws_stride;
  unsigned char* base64 = a.ws64_stride ? a.ws64 + slot * a.ws64_stride : nullptr;
  const int64_t stride = (int64_t)gridDim.x * kGroups;
  for (int64_t sys = sys0 + (int64_t)blockIdx.x * kGroups + gid; sys < n_sys; sys += stride) {
    if (MODE == 1)
      solve_one3<MIXED>(WarpGroup(), a, sys, base, gstates[gid], red, red64, par, m_prev, base64);
    else
      solve_one3<MIXED>(BlockGroup(), a, sys, base, gstate, red, red64, par, m_prev, base64);
  }
}

const size_t kSmemCap3 = 110 * 1024;

template <bool MIXED, int MODE>
int plan_fill3(int m, int threads, int cluster, SolvePlan* P) {
  const size_t ws = ws3_layout(m, MIXED ? 1 : 0);
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  std::memset(P, 0, sizeof(*P));
  P->warp = MODE == 1;
  P->cluster = MODE == 2 ? cluster : 0;
  P->threads = MODE == 1 ? 32 * kWarpsPerBlock3 : threads;
  P->groups_per_block = MODE == 1 ? kWarpsPerBlock3 : 1;
  P->blocks_per_group = MODE == 2 ? cluster : 1;
  // prec 1: the FP64 refinement vectors stay in global memory when the rest
  // of the workspace fits on chip
  const size_t v64 = MIXED ? 2 * align16_3((size_t)m * m * m * 8) : 0;
  const size_t chip = ((ws - v64) + 255) & ~(size_t)255;
  P->use_smem = MODE != 2 && chip * P->groups_per_block <= kSmemCap3;
  P->ws_stride = P->use_smem ? chip : (ws + 255) & ~(size_t)255;
  P->ws64_stride = P->use_smem && v64 ? (v64 + 255) & ~(size_t)255 : 0;
  P->smem_bytes = P->use_smem ? P->ws_stride * P->groups_per_block : 0;
  P->stage_bytes = 0;
  P->gamma = 1;
  P->nu = 1;
  P->nu_coarse = 0;
  P->inner_tol = 1e-5;
  cudaFuncSetAttribute(solve3_kernel<MIXED, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap3);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve3_kernel<MIXED, MODE>, P->threads, P->smem_bytes) !=
      cudaSuccess)
    return -1;
  P->blocks_per_sm = nb < 1 ? 1 : nb;
  P->max_groups = nsm * P->blocks_per_sm * P->groups_per_block;
  if (MODE == 2) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cluster * nsm);
    cfg.blockDim = dim3(P->threads);
    cfg.dynamicSmemBytes = 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, solve3_kernel<MIXED, MODE>, &cfg) != cudaSuccess || ncl < 1) return -1;
    P->max_groups = ncl;
  }
  return 0;
}

int plan_fill3(int m, int prec, int mode, int threads, int cluster, SolvePlan* P) {
  if (prec) {
    if (mode == 1) return plan_fill3<true, 1>(m, threads, 0, P);
    return mode == 2 ? plan_fill3<true, 2>(m, threads, cluster, P) : plan_fill3<true, 0>(m, threads, 0, P);
  }
  if (mode == 1) return plan_fill3<false, 1>(m, threads, 0, P);
  return mode == 2 ? plan_fill3<false, 2>(m, threads, cluster, P) : plan_fill3<false, 0>(m, threads, 0, P);
}

// Threads of a block per system: about one per cell of a red-black half sweep.
int threads3(int m) {
  const int64_t half = (int64_t)m * m * m / 2;
  int t = 32;
  while (t < half && t < kMaxThreads3) t *= 2;
  return t;
}

}  // namespace

size_t solve3_ws_bytes(int m, int prec) { return ws3_layout(m, prec); }

// Default plan: one block per system (shared-memory workspace while it
// fits), a cluster of 4 blocks from m = 64 on.
int solve3_plan(int m, int prec, SolvePlan* P) {
  if (m >= 64) return plan_fill3(m, prec, 2, kMaxThreads3, 4, P);
  return plan_fill3(m, prec, 0, threads3(m), 0, P);
}

int solve3_plan_mode(int m, int prec, int mode, int threads, int cluster, SolvePlan* P) {
  return plan_fill3(m, prec, mode, mode == 2 ? kMaxThreads3 : threads, cluster, P);
}

int solve3_plan_candidates(int m, int prec, SolvePlan* out, int max_out) {
  int k = 0;
  auto add = [&](const SolvePlan& P) {
    if (k < max_out) out[k++] = P;
  };
  SolvePlan d;
  if (solve3_plan(m, prec, &d)) return 0;
  add(d);
  if (m <= 16) {  // one warp per system
    SolvePlan w;
    if (!plan_fill3(m, prec, 1, 0, 0, &w)) add(w);
  }
  for (int t : {64, 128, 256, 512}) {
    if (!d.cluster && t == d.threads) continue;
    if ((int64_t)t > (int64_t)m * m * m) continue;
    SolvePlan b;
    if (!plan_fill3(m, prec, 0, t, 0, &b)) add(b);
  }
  // global-workspace block plans also with one or two systems per SM (the
  // systems in flight then keep their working set in L2)
  const int k0 = k;
  for (int i = 0; i < k0; ++i)
    if (!out[i].use_smem && !out[i].cluster && out[i].blocks_per_sm > 1)
      for (int cap : {1, 2}) {
        if (cap >= out[i].blocks_per_sm) continue;
        SolvePlan c = out[i];
        c.cap_blocks_per_sm = cap;
        add(c);
      }
  if (m >= 16)
    for (int cl : {2, 4, 8}) {
      if (cl == d.cluster) continue;
      SolvePlan c;
      if (!plan_fill3(m, prec, 2, kMaxThreads3, cl, &c)) add(c);
    }
  return k;
}

int solve3_launch(const SolveArgs& a, int prec, const SolvePlan& P, int n_blocks, cudaStream_t st) {
  SolveArgs b = a;
  b.use_smem = P.use_smem;
  b.ws_stride = P.ws_stride;
  b.mg_gamma = P.gamma;
  b.mg_nu = P.nu;
  b.mg_nu_coarse = P.nu_coarse;
  b.inner_tol = P.inner_tol;
  b.ws64_stride = P.ws64_stride;
  // cudaLaunchKernelEx for every plan: its return value is this launch's status
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(n_blocks);
  cfg.blockDim = dim3(P.threads);
  cfg.dynamicSmemBytes = P.cluster ? 0 : P.smem_bytes;
  cfg.stream = st;
  if (P.cluster) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  cudaError_t e;
  if (P.cluster) e = prec ? cudaLaunchKernelEx(&cfg, solve3_kernel<true, 2>, b) : cudaLaunchKernelEx(&cfg, solve3_kernel<false, 2>, b);
  else if (P.warp) e = prec ? cudaLaunchKernelEx(&cfg, solve3_kernel<true, 1>, b) : cudaLaunchKernelEx(&cfg, solve3_kernel<false, 1>, b);
  else e = prec ? cudaLaunchKernelEx(&cfg, solve3_kernel<true, 0>, b) : cudaLaunchKernelEx(&cfg, solve3_kernel<false, 0>, b);
  last_launch_error() = e;
  return e == cudaSuccess ? 0 : -1;
}

}  // namespace mlmc

// One warp per 16 x 16 system with the finest grid held in registers
// (included by solve.cu after the generic solver; prec 1 only: FP32
// multigrid-preconditioned CG inside FP64 iterative refinement).
//
// The generic warp solver keeps every array of the system in shared memory
// and recomputes each cell's indices on every pass; at m = 16 it spends about
// 500 instructions per cell and CG iteration.  Here each lane owns eight
// cells of one grid row and keeps their values, faces, diagonal and inverse
// diagonal in registers; the four neighbours of a cell come from the lane's
// own registers or from a warp shuffle (rows j -/+ 1 are lanes -/+ 2, the two
// halves of a row are lanes 2j and 2j + 1).  The 8 x 8 and 4 x 4 levels of the
// multigrid hierarchy stay in shared memory and run the generic code.  The
// arithmetic is the generic solver's (Sec. 3.1 Eq. 3.3 with harmonic faces,
// the same multigrid cycle, CG, refinement and stopping test), so results
// agree with it to rounding order.
//
// Lane layout: lane L holds row j = L >> 1 and the columns 8h .. 8h + 7
// (h = L & 1).  Its red part (i + j even) is slot t = 0..3 at column
// i = 8h + 2t + (j & 1), its black part slot t at i = 8h + 2t + 1 - (j & 1).
// Then the vertical neighbours of a cell are slot t of the other colour in
// lanes L -/+ 2, and the horizontal ones slot t or t -/+ 1 of the other
// colour in the same lane (t - 1 of lane L - 1 across the row's middle).
#pragma once

namespace mlmc {

constexpr int kTinyM = 16;

template <typename T>
struct TinyVec {
  T r[4], b[4];  // red and black parts of the lane's eight cells
};

struct TinyLane {
  int lane, j, h, jp;
  __device__ __forceinline__ TinyLane() {
    lane = threadIdx.x & 31;
    j = lane >> 1;
    h = lane & 1;
    jp = j & 1;
  }
  __device__ __forceinline__ int i_red(int t) const { return 8 * h + 2 * t + jp; }
  __device__ __forceinline__ int i_black(int t) const { return 8 * h + 2 * t + 1 - jp; }
};

// Neighbour values W, E, S, N of the four cells of one colour, from the other
// colour's part X (zero outside the grid).  red = 1: the cells are red.
template <typename T>
__device__ __forceinline__ void tiny_nbrs(const T (&X)[4], const TinyLane& ln, bool red, T (&W)[4], T (&E)[4],
                                          T (&S)[4], T (&N)[4]) {
  const unsigned full = 0xffffffffu;
  const T from_left = __shfl_up_sync(full, X[3], 1);    // lane - 1's X[3]: column 8h - 1
  const T from_right = __shfl_down_sync(full, X[0], 1);  // lane + 1's X[0]: column 8h + 8
  const T xl0 = ln.h == 1 ? from_left : T(0);
  const T xr3 = ln.h == 0 ? from_right : T(0);
  // red cells take W = X[t] (odd rows) or X[t - 1] (even rows), E = X[t + 1]
  // or X[t]; black cells the other way round
  const bool same = red ? (ln.jp == 1) : (ln.jp == 0);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const T xl = t > 0 ? X[t - 1] : xl0;
    const T xr = t < 3 ? X[t + 1] : xr3;
    W[t] = same ? X[t] : xl;
    E[t] = same ? xr : X[t];
    const T s = __shfl_up_sync(full, X[t], 2);
    const T n = __shfl_down_sync(full, X[t], 2);
    S[t] = ln.j > 0 ? s : T(0);
    N[t] = ln.j < kTinyM - 1 ? n : T(0);
  }
}

// Faces, diagonal and inverse diagonal of the lane's cells of one colour.
struct TinyOp {
  float w[4], e[4], s[4], n[4], d[4], id[4];
};

// (A v) at the cells of one colour: diag v - tW vW - tE vE - tS vS - tN vN
// (the generic operator's order).
__device__ __forceinline__ void tiny_apply(const TinyOp& A, const float (&v)[4], const float (&W)[4],
                                           const float (&E)[4], const float (&S)[4], const float (&N)[4],
                                           float (&y)[4]) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    float s = A.d[t] * v[t];
    s -= A.w[t] * W[t];
    s -= A.e[t] * E[t];
    s -= A.s[t] * S[t];
    s -= A.n[t] * N[t];
    y[t] = s;
  }
}

// Red (red = true) or black Gauss-Seidel half sweep on the finest grid:
// e_c = (f_c + sum of the faces times the other colour's e) / diag_c.
__device__ __forceinline__ void tiny_half_sweep(const TinyOp& A, const float (&f)[4], float (&e_own)[4],
                                                const float (&e_oth)[4], const TinyLane& ln, bool red,
                                                bool zero_guess) {
  if (zero_guess) {
#pragma unroll
    for (int t = 0; t < 4; ++t) e_own[t] = f[t] * A.id[t];
    return;
  }
  float W[4], E[4], S[4], N[4];
  tiny_nbrs(e_oth, ln, red, W, E, S, N);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    float s = f[t];
    s += A.w[t] * W[t];
    s += A.e[t] * E[t];
    s += A.s[t] * S[t];
    s += A.n[t] * N[t];
    e_own[t] = s * A.id[t];
  }
}

// Per-system state of the tiny path in shared memory: the hierarchy below the
// finest grid (levels of side 8 and 4) in the generic layout, then the FP64
// refinement solution and residual of the finest grid, [slot][lane] (slots
// 0..3 red, 4..7 black), touched once per refinement sweep.
__host__ __device__ inline size_t tiny_lev_bytes() {
  size_t o = 0;
  auto take = [&](size_t bytes) { o += align16(bytes); };
  for (int ml = kTinyM / 2;; ml >>= 1) {
    const size_t nl = (size_t)ml * ml, nf = (size_t)ml * (ml + 1);
    take(nf * 4);
    take(nf * 4);
    for (int a = 0; a < 4; ++a) take(nl * 4);
    if (ml <= kCoarseSide) {
      take(nl * nl * 4);
      take((2 * nl + 1) * 4);
      break;
    }
  }
  return o;
}
__host__ __device__ inline size_t tiny_ws_bytes() { return tiny_lev_bytes() + 2 * 8 * 32 * sizeof(double); }

// One FP64 cell vector of the finest grid in shared memory, [slot][lane].
struct TinyVec64 {
  double* p;
  int lane;
  __device__ __forceinline__ double& r(int t) const { return p[t * 32 + lane]; }
  __device__ __forceinline__ double& b(int t) const { return p[(4 + t) * 32 + lane]; }
};

// Symmetric multigrid cycle z = B r with the finest level in registers:
// nu red-black sweep pairs, the residual of the red cells restricted to the
// 8 x 8 grid, gamma visits of the shared-memory hierarchy (the generic
// cycle), prolongation, nu black-red sweep pairs.
template <typename G>
__device__ __forceinline__ void tiny_precond(const G& g, const TinyOp& Ar, const TinyOp& Ab, const TinyLane& ln,
                                             const Level<float>* lev, int nl, int gamma, int nu, int nuc,
                                             const TinyVec<float>& r, TinyVec<float>& z) {
  for (int s = 0; s < nu; ++s) {
    tiny_half_sweep(Ar, r.r, z.r, z.b, ln, true, s == 0);
    tiny_half_sweep(Ab, r.b, z.b, z.r, ln, false, false);
  }
  // residual at the red cells (zero at the black ones after a black sweep);
  // coarse cell (I, J) = red slot t of rows 2J and 2J + 1, I = 4h + t
  {
    float W[4], E[4], S[4], N[4], az[4];
    tiny_nbrs(z.b, ln, true, W, E, S, N);
    tiny_apply(Ar, z.r, W, E, S, N, az);
    const Level<float>& C = lev[1];
    const RbIndex Rc(kTinyM / 2);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float res = r.r[t] - az[t];
      const float up = __shfl_down_sync(0xffffffffu, res, 2);  // row 2J + 1
      if (ln.jp == 0) C.f[Rc.at(4 * ln.h + t, ln.j >> 1)] = res + up;
    }
  }
  g.sync();
  const int nuc1 = nuc < 1 ? nu : nuc;
  const int visits = nl - 1 == 1 ? 1 : gamma;  // the next level is the coarsest: solved once
  for (int v = 0; v < visits; ++v) {
    if (gamma <= 1 && nuc1 <= 1 && v == 0)
      vcycle(g, lev + 1, nl - 1);
    else
      mg_cycle(g, lev + 1, nl - 1, gamma < 1 ? 1 : gamma, nuc1, nuc1, v == 0);
  }
  {
    const Level<float>& C = lev[1];
    const RbIndex Rc(kTinyM / 2);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float ec = C.e[Rc.at(4 * ln.h + t, ln.j >> 1)];
      z.r[t] += ec;
      z.b[t] += ec;
    }
  }
  g.sync();  // every lane has read the coarse correction before the next cycle writes it
  for (int s = 0; s < nu; ++s) {
    tiny_half_sweep(Ab, r.b, z.b, z.r, ln, false, false);
    tiny_half_sweep(Ar, r.r, z.r, z.b, ln, true, false);
  }
}

// q = A p on both colours; returns the lane's part of p.q.
__device__ __forceinline__ float tiny_matvec(const TinyOp& Ar, const TinyOp& Ab, const TinyLane& ln,
                                             const TinyVec<float>& p, TinyVec<float>& q) {
  float W[4], E[4], S[4], N[4];
  tiny_nbrs(p.b, ln, true, W, E, S, N);
  tiny_apply(Ar, p.r, W, E, S, N, q.r);
  tiny_nbrs(p.r, ln, false, W, E, S, N);
  tiny_apply(Ab, p.b, W, E, S, N, q.b);
  float pq = 0.f;
#pragma unroll
  for (int t = 0; t < 4; ++t) pq += p.r[t] * q.r[t];
#pragma unroll
  for (int t = 0; t < 4; ++t) pq += p.b[t] * q.b[t];
  return pq;
}

// FP64 residual r = b - A x of the cells of one colour, with the FP32 faces
// widened (the generic refinement residual's arithmetic); returns the sum of
// squares over those cells.
// Right-hand side of a cell: Model Problem 2 moves the Dirichlet value p = 1
// at x1 = 0 into b through the west face of column 0; Model Problem 1 has
// f / m^2 everywhere.
__device__ __forceinline__ double tiny_rhs(const SolveArgs& a, float west_face, int i) {
  return a.problem == 1 ? 1.0 / ((double)kTinyM * (double)kTinyM) : (i == 0 ? (double)west_face : 0.0);
}

__device__ __forceinline__ double tiny_residual64_colour(const SolveArgs& a, const TinyOp& A,
                                                         const double (&x_own)[4], const double (&x_oth)[4],
                                                         const TinyLane& ln, bool red, double (&r)[4]) {
  double W[4], E[4], S[4], N[4];
  tiny_nbrs(x_oth, ln, red, W, E, S, N);
  double s2 = 0.0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const double tw = A.w[t], te = A.e[t], ts = A.s[t], tn = A.n[t];
    double ax = ((tw + te) + (ts + tn)) * x_own[t];
    ax -= tw * W[t];
    ax -= te * E[t];
    ax -= ts * S[t];
    ax -= tn * N[t];
    r[t] = tiny_rhs(a, A.w[t], red ? ln.i_red(t) : ln.i_black(t)) - ax;
    s2 += r[t] * r[t];
  }
  return s2;
}

// k at cell (i, j) of a 16 x 16 system, as the generic assembly computes it;
// row_layer >= 0: the layer of every cell of row j (horizontal interfaces).
__device__ __forceinline__ double tiny_k_of_cell(const SolveArgs& a, const GroupState<float, float>& gs,
                                                 int64_t sys, int64_t sidx, bool coarse, int ox, int oy, int i,
                                                 int j, int row_layer) {
  const int m = kTinyM;
  if (a.ksrc == KSRC_ARRAY) return a.k[sys * (int64_t)(m * m) + j * m + i];
  const int jf = coarse ? 2 * j + oy : j;
  const int iff = coarse ? 2 * i + ox : i;
  int t = row_layer;
  if (t < 0) {
    const int n_if = a.geometry == 1 ? 0 : a.n_layers - 1;
    const double inv_m = 1.0 / (double)m, inv_mf = 1.0 / (double)a.m;
    const bool own = coarse && !a.cgv_on_k;
    const double yc = own ? ((double)j + 0.5) * inv_m : ((double)jf + 0.5) * inv_mf;
    const double xc = own ? ((double)i + 0.5) * inv_m : ((double)iff + 0.5) * inv_mf;
    t = layer_at_point(a.geometry, gs.eta, n_if, xc, yc);
  }
  if (a.ksrc == KSRC_CONST) return gs.kc[t];
  const float* gf = reinterpret_cast<const float*>(a.g);
  return (double)expf(gf[((sidx * a.n_layers + t) * (int64_t)a.m + jf) * a.m + iff]);
}

// Harmonic face average 2 ka kb / (ka + kb) in FP32, ka the west / south cell
// (the generic assembly's order, so both cells of a face get the same bits).
__device__ __forceinline__ float tiny_harm(float ka, float kb) { return 2.0f * ka * kb / (ka + kb); }

// Assemble, solve (prec 1) and reduce the QoI of one 16 x 16 system with one
// warp; m_prev is set to -kTinyM so that the generic path rebuilds its level
// table when the group next solves another size.
template <typename G>
__device__ void solve_one_tiny(const G& g, const SolveArgs& a, int64_t sys, unsigned char* base,
                               GroupState<float, float>& gs, int& m_prev) {
  using T = float;
  const int m = kTinyM, n = m * m;
  int64_t sidx;
  int coarse = 0, ox = 0, oy = 0;
  if (sys < a.n_samples) {
    sidx = sys;
  } else {
    const int64_t t = sys - a.n_samples;
    sidx = t / a.n_coarse;
    const int o = (int)(t - sidx * a.n_coarse);
    coarse = 1;
    ox = o & 1;
    oy = o >> 1;
  }
  const uint64_t sample = (uint64_t)(a.first + sidx);
  if (m_prev != -kTinyM) {  // level table of the shared-memory levels (8 x 8, 4 x 4)
    g.sync();
    if (g.local_leader()) {
      size_t o = 0;
      auto take = [&](size_t bytes) {
        unsigned char* p = base + o;
        o += align16(bytes);
        return p;
      };
      int l = 1;
      for (int ml = m / 2;; ml >>= 1, ++l) {
        const size_t nlv = (size_t)ml * ml, nf = (size_t)ml * (ml + 1);
        Level<T, T>& L = gs.lev[l];
        L.m = ml;
        L.tx = reinterpret_cast<T*>(take(nf * 4));
        L.ty = reinterpret_cast<T*>(take(nf * 4));
        L.diag = reinterpret_cast<T*>(take(nlv * 4));
        L.invd = reinterpret_cast<T*>(take(nlv * 4));
        L.e = reinterpret_cast<T*>(take(nlv * 4));
        L.f = reinterpret_cast<T*>(take(nlv * 4));
        L.cinv = L.cbuf = nullptr;
        L.stage = nullptr;
        L.stage_rows = 0;
        L.quads = 0;
        if (ml <= kCoarseSide) {
          L.cinv = reinterpret_cast<T*>(take(nlv * nlv * 4));
          L.cbuf = reinterpret_cast<T*>(take((2 * nlv + 1) * 4));
          break;
        }
      }
      gs.nl = l + 1;
      gs.lev[0].m = m;
    }
    g.sync();
    m_prev = -kTinyM;
  }
  const int nl = gs.nl;
  const Level<T>* lev = gs.lev;
  const TinyLane ln;
  // ---- layers, cell permeabilities (FP32, as the generic assembly rounds them) ----
  if (a.ksrc != KSRC_ARRAY) {
    if (g.local_leader()) sample_layers(a, sample, gs.eta, gs.kc);
    g.sync();
  }
  // horizontal interfaces: the layer depends on the row only (the same
  // centre comparison as the generic per-cell one, evaluated once per lane)
  int row_layer = -1;
  if (a.ksrc != KSRC_ARRAY && a.geometry != 1) {
    const bool own = coarse && !a.cgv_on_k;
    const double yc = own ? ((double)ln.j + 0.5) * (1.0 / (double)m)
                          : ((double)(coarse ? 2 * ln.j + oy : ln.j) + 0.5) * (1.0 / (double)a.m);
    row_layer = layer_at(gs.eta, a.n_layers - 1, yc);
  }
  TinyVec<float> k;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    k.r[t] = (float)tiny_k_of_cell(a, gs, sys, sidx, coarse, ox, oy, ln.i_red(t), ln.j, row_layer);
    k.b[t] = (float)tiny_k_of_cell(a, gs, sys, sidx, coarse, ox, oy, ln.i_black(t), ln.j, row_layer);
  }
  // ---- faces (Eq. 3.3: harmonic inside, 2k on Dirichlet faces, 0 on no-flow faces) ----
  TinyOp Ar, Ab;
  {
    float W[4], E[4], S[4], N[4];
    for (int col = 0; col < 2; ++col) {
      const bool red = col == 0;
      const float(&kc)[4] = red ? k.r : k.b;
      tiny_nbrs(red ? k.b : k.r, ln, red, W, E, S, N);
      TinyOp& A = red ? Ar : Ab;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int i = red ? ln.i_red(t) : ln.i_black(t);
        A.w[t] = i == 0 ? 2.0f * kc[t] : tiny_harm(W[t], kc[t]);
        A.e[t] = i == m - 1 ? 2.0f * kc[t] : tiny_harm(kc[t], E[t]);
        A.s[t] = ln.j == 0 ? (a.problem == 1 ? 2.0f * kc[t] : 0.0f) : tiny_harm(S[t], kc[t]);
        A.n[t] = ln.j == m - 1 ? (a.problem == 1 ? 2.0f * kc[t] : 0.0f) : tiny_harm(kc[t], N[t]);
        A.d[t] = (A.w[t] + A.e[t]) + (A.s[t] + A.n[t]);
        A.id[t] = 1.0f / A.d[t];
      }
    }
  }
  // ---- the 8 x 8 level's faces: means of the two fine faces forming each coarse face ----
  {
    const Level<T>& C = gs.lev[1];
    const int mc = m / 2;
    // tx: coarse face I' = 4h + t of coarse row J is fine face 2I' (the west
    // face of column 2I') of rows 2J, 2J + 1; I' = 8 is the east face of column 15
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float fw = ln.jp ? Ab.w[t] : Ar.w[t];  // column 8h + 2t is black in odd rows
      const float up = __shfl_down_sync(0xffffffffu, fw, 2);
      if (ln.jp == 0) C.tx[(ln.j >> 1) * (mc + 1) + 4 * ln.h + t] = 0.5f * (fw + up);
    }
    {
      const float fe = ln.jp ? Ar.e[3] : Ab.e[3];  // column 15: red in odd rows
      const float up = __shfl_down_sync(0xffffffffu, fe, 2);
      if (ln.jp == 0 && ln.h == 1) C.tx[(ln.j >> 1) * (mc + 1) + mc] = 0.5f * (fe + up);
    }
    // ty: coarse face J' of coarse column I = 4h + t is fine face 2J' of
    // columns 2I, 2I + 1 (south faces of row 2J'); J' = 8: north faces of row 15
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (ln.jp == 0) C.ty[(ln.j >> 1) * mc + 4 * ln.h + t] = 0.5f * (Ar.s[t] + Ab.s[t]);
      if (ln.j == m - 1) C.ty[mc * mc + 4 * ln.h + t] = 0.5f * (Ab.n[t] + Ar.n[t]);
    }
  }
  g.sync();
  build_diag<true>(g, gs.lev[1]);
  for (int l = 2; l < nl; ++l) {
    build_coarse(g, gs.lev[l - 1], gs.lev[l]);
    build_diag<true>(g, gs.lev[l]);
  }
  build_coarse_inverse(g, gs.lev[nl - 1]);
  // ---- FP64 refinement around FP32 PCG (restarted, or reliable updates) ----
  const TinyVec64 X64{reinterpret_cast<double*>(base + tiny_lev_bytes()), ln.lane};
  const TinyVec64 R64{X64.p + 8 * 32, ln.lane};
  double bb = 0.0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const double br = tiny_rhs(a, Ar.w[t], ln.i_red(t)), bk = tiny_rhs(a, Ab.w[t], ln.i_black(t));
    X64.r(t) = X64.b(t) = 0.0;
    R64.r(t) = br;
    R64.b(t) = bk;
    bb += br * br;
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) bb += R64.b(t) * R64.b(t);
  bb = warp_sum(bb);
  double rr = bb;
  const double thr = a.tol * a.tol * bb;
  auto residual64 = [&]() -> double {
    double xr[4], xk[4], rv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      xr[t] = X64.r(t);
      xk[t] = X64.b(t);
    }
    double s2 = tiny_residual64_colour(a, Ar, xr, xk, ln, true, rv);
#pragma unroll
    for (int t = 0; t < 4; ++t) R64.r(t) = rv[t];
    s2 += tiny_residual64_colour(a, Ab, xk, xr, ln, false, rv);
#pragma unroll
    for (int t = 0; t < 4; ++t) R64.b(t) = rv[t];
    return warp_sum(s2);
  };
  const int gamma = a.mg_gamma, nu = a.mg_nu < 1 ? 1 : a.mg_nu, nuc = a.mg_nu_coarse;
  TinyVec<float> x, r, p, q, z;
  int status = 1, iters = 0, sweeps = 0;
  // Each scheme calls the preconditioner from one place (at the top of its
  // iteration), which keeps the unrolled code small; the operations and their
  // order are the generic solver's.
  if (a.reliable) {
    // one FP32 CG on the correction with reliable updates (see the generic solver)
    if (rr <= thr) status = 0;
    double scl = sqrt(rr);
    float rr32 = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      r.r[t] = (float)(R64.r(t) / scl);
      r.b[t] = (float)(R64.b(t) / scl);
      x.r[t] = x.b[t] = 0.f;
      rr32 += r.r[t] * r.r[t] + r.b[t] * r.b[t];
    }
    rr32 = warp_sum(rr32);
    float rr_ref = rr32;
    const float d2 = (float)(a.inner_tol * a.inner_tol);
    float rz = 0.f;
    bool first = true;
    int since = 0;
    while (status != 0 && iters < a.max_it) {
      tiny_precond(g, Ar, Ab, ln, lev, nl, gamma, nu, nuc, r, z);
      float rzn = 0.f;
#pragma unroll
      for (int t = 0; t < 4; ++t) rzn += r.r[t] * z.r[t] + r.b[t] * z.b[t];
      rzn = warp_sum(rzn);
      const float beta = first ? 0.f : rzn / rz;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        p.r[t] = first ? z.r[t] : z.r[t] + beta * p.r[t];
        p.b[t] = first ? z.b[t] : z.b[t] + beta * p.b[t];
      }
      rz = rzn;
      first = false;
      ++iters;
      ++since;
      const float pq = warp_sum(tiny_matvec(Ar, Ab, ln, p, q));
      if (!(pq > 0.f) || !isfinite(pq) || !isfinite(rz)) {
        status = 2;
        break;
      }
      const float alpha = rz / pq;
      rr32 = 0.f;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        x.r[t] += alpha * p.r[t];
        x.b[t] += alpha * p.b[t];
        r.r[t] = r.r[t] - alpha * q.r[t];
        r.b[t] = r.b[t] - alpha * q.b[t];
        rr32 += r.r[t] * r.r[t] + r.b[t] * r.b[t];
      }
      rr32 = warp_sum(rr32);
      if ((double)rr32 * scl * scl <= thr || rr32 <= d2 * rr_ref || since >= 16) {  // reliable update
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          X64.r(t) += scl * (double)x.r[t];
          X64.b(t) += scl * (double)x.b[t];
        }
        rr = residual64();
        ++sweeps;
        if (rr <= thr) {
          status = 0;
          break;
        }
        const double scl_new = sqrt(rr);
        const float ratio = (float)(scl / scl_new);
        rr32 = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          r.r[t] = (float)(R64.r(t) / scl_new);
          r.b[t] = (float)(R64.b(t) / scl_new);
          x.r[t] = x.b[t] = 0.f;
          p.r[t] *= ratio;
          p.b[t] *= ratio;
          rr32 += r.r[t] * r.r[t] + r.b[t] * r.b[t];
        }
        rr32 = warp_sum(rr32);
        rz *= ratio * ratio;
        scl = scl_new;
        rr_ref = rr32;
        since = 0;
      }
    }
  } else {
    // restarted refinement: FP32 PCG solves to ||r|| <= inner_tol ||r0|| on the
    // scaled residual, each followed by x64 += scl x32 and the FP64 residual
    float thr_in = 0.f, rz = 0.f;
    double scl = 0.0;
    int it = 0;         // iterations of the current inner solve
    bool fresh = true;  // the next pass starts a refinement sweep
    bool small0 = false;  // the scaled residual already meets the inner tolerance
    while (true) {
      if (fresh) {
        if (rr <= thr) {
          status = 0;
          break;
        }
        if (iters >= a.max_it || sweeps >= 40) {
          status = 1;
          break;
        }
        ++sweeps;
        scl = sqrt(rr);
        const double inv = 1.0 / scl;
        float r32 = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          r.r[t] = (float)(R64.r(t) * inv);
          r.b[t] = (float)(R64.b(t) * inv);
          x.r[t] = x.b[t] = 0.f;
          r32 += r.r[t] * r.r[t] + r.b[t] * r.b[t];
        }
        r32 = warp_sum(r32);
        thr_in = (float)(a.inner_tol * a.inner_tol) * r32;
        small0 = r32 <= thr_in;
        it = 0;
        fresh = false;
      }
      int st_in = 1;  // 0 converged, 1 running / cap, 2 breakdown
      bool end_inner = false;
      if (it == 0 && small0) {
        st_in = 0;
        end_inner = true;
      } else if (it >= a.max_it - iters) {
        end_inner = true;  // cap (the generic pcg's loop condition)
      } else {
        tiny_precond(g, Ar, Ab, ln, lev, nl, gamma, nu, nuc, r, z);
        float rzn = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t) rzn += r.r[t] * z.r[t] + r.b[t] * z.b[t];
        rzn = warp_sum(rzn);
        const float beta = it == 0 ? 0.f : rzn / rz;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          p.r[t] = it == 0 ? z.r[t] : z.r[t] + beta * p.r[t];
          p.b[t] = it == 0 ? z.b[t] : z.b[t] + beta * p.b[t];
        }
        rz = rzn;
        ++it;
        const float pq = warp_sum(tiny_matvec(Ar, Ab, ln, p, q));
        if (!(pq > 0.f) || !isfinite(pq) || !isfinite(rz)) {
          st_in = 2;
          end_inner = true;
        } else {
          const float alpha = rz / pq;
          float rrs = 0.f;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            x.r[t] += alpha * p.r[t];
            x.b[t] += alpha * p.b[t];
            r.r[t] = r.r[t] - alpha * q.r[t];
            r.b[t] = r.b[t] - alpha * q.b[t];
            rrs += r.r[t] * r.r[t] + r.b[t] * r.b[t];
          }
          rrs = warp_sum(rrs);
          if (rrs <= thr_in) {
            st_in = 0;
            end_inner = true;
          }
        }
      }
      if (!end_inner) continue;
      // a breakdown counts its iteration only up to the failed step, as in pcg
      iters += it;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        X64.r(t) += scl * (double)x.r[t];
        X64.b(t) += scl * (double)x.b[t];
      }
      rr = residual64();
      if (it == 0 && st_in != 0) {  // inner solver made no progress
        status = 2;
        break;
      }
      fresh = true;
    }
  }
  // ---- QoI and outputs ----
  double qsum = 0.0;
  if (a.problem == 1) {
    const double hh = 1.0 / (double)m;
    const double inv_area = 1.0 / ((a.box[1] - a.box[0]) * (a.box[3] - a.box[2]));
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int i = t < 4 ? ln.i_red(t) : ln.i_black(t - 4);
      const double xv = t < 4 ? X64.r(t) : X64.b(t - 4);
      const double bx = fmin((i + 1) * hh, a.box[1]) - fmax(i * hh, a.box[0]);
      const double by = fmin((ln.j + 1) * hh, a.box[3]) - fmax(ln.j * hh, a.box[2]);
      if (bx > 0.0 && by > 0.0) qsum += bx * by * inv_area * xv;
    }
  } else if (ln.h == 1) {
    // outflow through x1 = 1: column 15 is red slot 3 in odd rows, black slot 3 in even rows
    qsum = ln.jp ? (double)Ar.e[3] * X64.r(3) : (double)Ab.e[3] * X64.b(3);
  }
  qsum = warp_sum(qsum);
  if (ln.lane == 0) {
    a.q[sys] = status == 0 ? qsum : nan("");
    if (a.iters) a.iters[sys] = iters;
  }
  if (a.p_out && !coarse) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      a.p_out[sidx * (int64_t)n + ln.j * m + ln.i_red(t)] = X64.r(t);
      a.p_out[sidx * (int64_t)n + ln.j * m + ln.i_black(t)] = X64.b(t);
    }
  }
  g.sync();
}

}  // namespace mlmc

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
// halves of a row are lanes 2j and 2j + 1).  The 8 x 8 level of the multigrid
// hierarchy is held the same way, two cells per lane (its operator in shared
// memory), and the 4 x 4 coarsest grid is solved with its dense inverse,
// built per system by Gauss-Jordan elimination in registers.  The arithmetic
// is the generic solver's (Sec. 3.1 Eq. 3.3 with harmonic faces, the same
// multigrid cycle, CG, refinement and stopping test; the coarsest inverse in
// natural instead of red-black cell order), so results agree with it to
// rounding order.
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

// Per-system state of the tiny path in shared memory: the 8 x 8 level's
// faces and inverse diagonal, [k][lane] (k = 0..4: west, east, south, north
// face and inverse diagonal of the lane's red cell; 5..9 its black cell), the
// dense inverse of the 4 x 4 grid's operator (16 x 16, natural cell order
// c = 4 J + I), then the FP64 refinement solution and residual of the finest
// grid, [slot][lane] (slots 0..3 red, 4..7 black), touched once per
// refinement sweep.
constexpr size_t kTinyOp8Bytes = 10 * 32 * sizeof(float);
constexpr size_t kTinyCinvBytes = 16 * 16 * sizeof(float);
__host__ __device__ inline size_t tiny_lev_bytes() { return kTinyOp8Bytes + kTinyCinvBytes; }
__host__ __device__ inline size_t tiny_ws_bytes() { return tiny_lev_bytes() + 2 * 8 * 32 * sizeof(double); }

// The lane's two cells of the 8 x 8 level: lane L holds row J = L >> 2 and
// columns 2q, 2q + 1 (q = L & 3); its red cell is column 2q + (J & 1), its
// black cell 2q + 1 - (J & 1).  Rows J -/+ 1 are lanes -/+ 4.
struct TinyC8 {
  int lane, J, q, jp;
  __device__ __forceinline__ TinyC8() {
    lane = threadIdx.x & 31;
    J = lane >> 2;
    q = lane & 3;
    jp = J & 1;
  }
};

// Neighbour values W, E, S, N of the lane's 8 x 8 cell of one colour, from
// the other colour's value x (zero outside the grid).
__device__ __forceinline__ void c8_nbrs(float x, const TinyC8& c, bool red, float& W, float& E, float& S,
                                        float& N) {
  const unsigned full = 0xffffffffu;
  const float from_left = __shfl_up_sync(full, x, 1);    // lane - 1's right cell: column 2q - 1
  const float from_right = __shfl_down_sync(full, x, 1);  // lane + 1's left cell: column 2q + 2
  const float s = __shfl_up_sync(full, x, 4);
  const float n = __shfl_down_sync(full, x, 4);
  // `right`: the cell is the lane's right one (column 2q + 1), its west
  // neighbour the lane's other cell
  const bool right = red ? (c.jp == 1) : (c.jp == 0);
  W = right ? x : (c.q > 0 ? from_left : 0.f);
  E = right ? (c.q < 3 ? from_right : 0.f) : x;
  S = c.J > 0 ? s : 0.f;
  N = c.J < 7 ? n : 0.f;
}

// Gauss-Seidel half sweep of one colour on the 8 x 8 level (op8: the faces
// and inverse diagonal, [k][lane]).
__device__ __forceinline__ void c8_half_sweep(const float* op8, const TinyC8& c, bool red, float f, float& e_own,
                                              float e_oth, bool zero_guess) {
  const int o = red ? 0 : 5;
  const float id = op8[(o + 4) * 32 + c.lane];
  if (zero_guess) {
    e_own = f * id;
    return;
  }
  float W, E, S, N;
  c8_nbrs(e_oth, c, red, W, E, S, N);
  float s = f;
  s += op8[o * 32 + c.lane] * W;
  s += op8[(o + 1) * 32 + c.lane] * E;
  s += op8[(o + 2) * 32 + c.lane] * S;
  s += op8[(o + 3) * 32 + c.lane] * N;
  e_own = s * id;
}

// One visit of the 8 x 8 level (Sec. 3.5 multigrid preconditioner, the
// generic cycle's steps on a two-level hierarchy): nuc red-black sweep pairs
// (from e = 0 when zero_start), the red cells' residual summed over each 2 x 2
// aggregate onto the 4 x 4 grid, its exact solve with the dense inverse,
// prolongation, nuc black-red sweep pairs.
__device__ __forceinline__ void c8_cycle(const float* op8, const float* cinv, const TinyC8& c, float fr, float fb,
                                         float& er, float& eb, int nuc, bool zero_start) {
  const unsigned full = 0xffffffffu;
  for (int s = 0; s < nuc; ++s) {
    c8_half_sweep(op8, c, true, fr, er, eb, zero_start && s == 0);
    c8_half_sweep(op8, c, false, fb, eb, er, false);
  }
  // residual at the red cell (zero at the black one after a black sweep):
  // f - (diag e - the faces times the neighbours), the generic order
  float W, E, S, N;
  c8_nbrs(eb, c, true, W, E, S, N);
  const float tw = op8[c.lane], te = op8[32 + c.lane], ts = op8[64 + c.lane], tn = op8[96 + c.lane];
  float ax = ((tw + te) + (ts + tn)) * er;
  ax -= tw * W;
  ax -= te * E;
  ax -= ts * S;
  ax -= tn * N;
  const float res = fr - ax;
  // coarse cell (I', J') = red cells (2I', 2J') [lane 8J' + I'] and
  // (2I' + 1, 2J' + 1) [lane 8J' + I' + 4]
  const float f4 = res + __shfl_down_sync(full, res, 4);
  // e4 = Cinv f4 at the lanes with even J (the others compute a value nobody uses)
  const int c4 = 4 * (c.J >> 1) + c.q;
  const float4* row = reinterpret_cast<const float4*>(cinv + c4 * 16);
  float e4 = 0.f;
#pragma unroll
  for (int k4 = 0; k4 < 4; ++k4) {
    const float4 w = row[k4];
    const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int cc = 4 * k4 + u;
      e4 += wv[u] * __shfl_sync(full, f4, 8 * (cc >> 2) + (cc & 3));
    }
  }
  const float ec = __shfl_sync(full, e4, 8 * (c.J >> 1) + c.q);
  er += ec;
  eb += ec;
  for (int s = 0; s < nuc; ++s) {
    c8_half_sweep(op8, c, false, fb, eb, er, false);
    c8_half_sweep(op8, c, true, fr, er, eb, false);
  }
}

// One FP64 cell vector of the finest grid in shared memory, [slot][lane].
struct TinyVec64 {
  double* p;
  int lane;
  __device__ __forceinline__ double& r(int t) const { return p[t * 32 + lane]; }
  __device__ __forceinline__ double& b(int t) const { return p[(4 + t) * 32 + lane]; }
};

// Symmetric multigrid cycle z = B r with the finest level in registers:
// nu red-black sweep pairs, the residual of the red cells restricted to the
// 8 x 8 grid, gamma visits of the 8 x 8 level (c8_cycle), prolongation, nu
// black-red sweep pairs.
__device__ __forceinline__ void tiny_precond(const TinyOp& Ar, const TinyOp& Ab, const TinyLane& ln,
                                             const TinyC8& c8, const float* op8, const float* cinv, int gamma,
                                             int nu, int nuc, const TinyVec<float>& r, TinyVec<float>& z) {
  const unsigned full = 0xffffffffu;
  for (int s = 0; s < nu; ++s) {
    tiny_half_sweep(Ar, r.r, z.r, z.b, ln, true, s == 0);
    tiny_half_sweep(Ab, r.b, z.b, z.r, ln, false, false);
  }
  // residual at the red cells (zero at the black ones after a black sweep);
  // coarse cell (I, J) = red slot t of rows 2J and 2J + 1, I = 4h + t, summed
  // in the lanes of row 2J
  float rs[4];
  {
    float W[4], E[4], S[4], N[4], az[4];
    tiny_nbrs(z.b, ln, true, W, E, S, N);
    tiny_apply(Ar, z.r, W, E, S, N, az);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float res = r.r[t] - az[t];
      rs[t] = res + __shfl_down_sync(full, res, 2);  // row 2J + 1
    }
  }
  // to the 8 x 8 layout: cell I = 2q + u of row J is slot t = 2 (q & 1) + u of lane 4J + (q >> 1)
  float fr, fb;
  {
    float v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) v[t] = __shfl_sync(full, rs[t], 4 * c8.J + (c8.q >> 1));
    const float u0 = (c8.q & 1) ? v[2] : v[0], u1 = (c8.q & 1) ? v[3] : v[1];
    fr = c8.jp ? u1 : u0;
    fb = c8.jp ? u0 : u1;
  }
  const int nuc1 = nuc < 1 ? nu : nuc;
  float er = 0.f, eb = 0.f;
  for (int v = 0; v < (gamma < 1 ? 1 : gamma); ++v) c8_cycle(op8, cinv, c8, fr, fb, er, eb, nuc1, v == 0);
  // prolongation: fine slot t of lane (j, h) takes coarse cell (4h + t, j >> 1),
  // cell u = t & 1 of 8 x 8 lane 4 (j >> 1) + 2h + (t >> 1), red there when u == (j >> 1) & 1
  {
    const int Jc = ln.j >> 1, s0 = 4 * Jc + 2 * ln.h;
    const float ar = __shfl_sync(full, er, s0), ab = __shfl_sync(full, eb, s0);
    const float br = __shfl_sync(full, er, s0 + 1), bb = __shfl_sync(full, eb, s0 + 1);
    const bool odd = Jc & 1;
    const float ec[4] = {odd ? ab : ar, odd ? ar : ab, odd ? bb : br, odd ? br : bb};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      z.r[t] += ec[t];
      z.b[t] += ec[t];
    }
  }
  for (int s = 0; s < nu; ++s) {
    tiny_half_sweep(Ab, r.b, z.b, z.r, ln, false, false);
    tiny_half_sweep(Ar, r.r, z.r, z.b, ln, true, false);
  }
}

// The 8 x 8 level's operator (faces: means of the two fine faces forming each
// coarse face; inverse diagonal) into op8, and the dense inverse of the 4 x 4
// grid's operator (faces from the 8 x 8 ones by the same rule) into cinv, by
// Gauss-Jordan elimination without pivoting (the operator is SPD) with lane L
// holding columns 8 (L & 1) .. + 7 of row L >> 1.
__device__ __forceinline__ void tiny_build_coarse(const TinyOp& Ar, const TinyOp& Ab, const TinyLane& ln,
                                                  const TinyC8& c8, float* op8, float* cinv) {
  const unsigned full = 0xffffffffu;
  // fine layout, lanes of even rows 2J: the coarse faces of cells (4h + t, J)
  float cw[4], ce[4], cs[4], cn[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    cw[t] = 0.5f * (Ar.w[t] + __shfl_down_sync(full, Ab.w[t], 2));
    ce[t] = 0.5f * (Ab.e[t] + __shfl_down_sync(full, Ar.e[t], 2));
    cs[t] = 0.5f * (Ar.s[t] + Ab.s[t]);
    cn[t] = 0.5f * (__shfl_down_sync(full, Ab.n[t], 2) + __shfl_down_sync(full, Ar.n[t], 2));
  }
  // 8 x 8 layout: faces of the lane's cells u = 0 (column 2q) and u = 1
  float w8[2], e8[2], s8[2], n8[2];
  {
    const int src = 4 * c8.J + (c8.q >> 1);
    const int t0 = 2 * (c8.q & 1);
    float v[4];
#define TINY_MOVE(X, Y)                                                   \
  for (int t = 0; t < 4; ++t) v[t] = __shfl_sync(full, X[t], src);        \
  Y[0] = t0 ? v[2] : v[0];                                                \
  Y[1] = t0 ? v[3] : v[1];
#pragma unroll
    TINY_MOVE(cw, w8)
#pragma unroll
    TINY_MOVE(ce, e8)
#pragma unroll
    TINY_MOVE(cs, s8)
#pragma unroll
    TINY_MOVE(cn, n8)
#undef TINY_MOVE
  }
#pragma unroll
  for (int col = 0; col < 2; ++col) {  // 0 red (u = jp), 1 black
    const int u = col == 0 ? c8.jp : 1 - c8.jp;
    const float w = u ? w8[1] : w8[0], e = u ? e8[1] : e8[0], s = u ? s8[1] : s8[0], n = u ? n8[1] : n8[0];
    float* o = op8 + col * 5 * 32 + c8.lane;
    o[0] = w;
    o[32] = e;
    o[64] = s;
    o[96] = n;
    o[128] = 1.0f / ((w + e) + (s + n));
  }
  // 4 x 4 faces at lanes 8J' + I' (rows 2J' and 2J' + 1 of the 8 x 8 level are lanes L and L + 4)
  const float w4 = 0.5f * (w8[0] + __shfl_down_sync(full, w8[0], 4));
  const float e4 = 0.5f * (e8[1] + __shfl_down_sync(full, e8[1], 4));
  const float s4 = 0.5f * (s8[0] + s8[1]);
  const float n4 = 0.5f * (__shfl_down_sync(full, n8[0], 4) + __shfl_down_sync(full, n8[1], 4));
  // row r = L >> 1 of the 4 x 4 operator, columns 8 hh .. 8 hh + 7
  const int r = ln.lane >> 1, hh = ln.lane & 1;
  const int src4 = 8 * (r >> 2) + (r & 3);
  const float rw = __shfl_sync(full, w4, src4), re = __shfl_sync(full, e4, src4);
  const float rsv = __shfl_sync(full, s4, src4), rn = __shfl_sync(full, n4, src4);
  float B[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int cc = 8 * hh + k;
    float v = 0.f;
    if (cc == r) v = (rw + re) + (rsv + rn);
    else if (cc == r - 1 && (r & 3) != 0) v = -rw;
    else if (cc == r + 1 && (r & 3) != 3) v = -re;
    else if (cc == r - 4) v = -rsv;
    else if (cc == r + 4) v = -rn;
    B[k] = v;
  }
  // Gauss-Jordan: at step k with pivot p = B[k][k], scaled pivot row B[k][j] / p and
  // column c_i = B[i][k]: B[k][k] <- 1/p, B[k][j] <- B[k][j] / p, B[i][k] <- -c_i / p,
  // B[i][j] <- B[i][j] - c_i (B[k][j] / p); after 16 steps B = A^-1
#pragma unroll
  for (int kk = 0; kk < 16; ++kk) {
    const float p = __shfl_sync(full, B[kk & 7], 2 * kk + (kk >> 3));
    const float ip = 1.0f / p;
    const float ci = __shfl_sync(full, B[kk & 7], (ln.lane & ~1) + (kk >> 3));
    float rj[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) rj[k] = __shfl_sync(full, B[k], 2 * kk + hh) * ip;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int jc = 8 * hh + k;
      float v;
      if (r == kk) v = jc == kk ? ip : rj[k];
      else if (jc == kk) v = -ci * ip;
      else v = fmaf(-ci, rj[k], B[k]);
      B[k] = v;
    }
  }
  float4* dst = reinterpret_cast<float4*>(cinv + r * 16 + 8 * hh);
  dst[0] = make_float4(B[0], B[1], B[2], B[3]);
  dst[1] = make_float4(B[4], B[5], B[6], B[7]);
  __syncwarp();
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
  if (m_prev != -kTinyM) {  // the workspace held another size's levels
    g.sync();
    m_prev = -kTinyM;
  }
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
  // ---- the 8 x 8 level's operator and the 4 x 4 grid's inverse ----
  const TinyC8 c8;
  float* op8 = reinterpret_cast<float*>(base);
  float* cinv = reinterpret_cast<float*>(base + kTinyOp8Bytes);
  tiny_build_coarse(Ar, Ab, ln, c8, op8, cinv);
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
      tiny_precond(Ar, Ab, ln, c8, op8, cinv, gamma, nu, nuc, r, z);
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
        tiny_precond(Ar, Ab, ln, c8, op8, cinv, gamma, nu, nuc, r, z);
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

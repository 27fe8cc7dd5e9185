// Fused assembly + multigrid-preconditioned CG + outflow QoI, one warp, one
// thread block or one thread-block cluster per linear system (many systems
// per launch, grid-stride over systems).
//
// System of one sample (Sec. 3.1 Eq. 3.3 with harmonic faces, Sec. 3.4 Model
// Problem 2): unknown p on m x m cells,
//   sum_faces T_f (p_c - p_nbr) = b_c,  T = 2 k_a k_b / (k_a + k_b) inside,
//   T = 2 k_c on the Dirichlet faces x1 = 0, 1 (p_nbr = 1 at x1 = 0, 0 at
//   x1 = 1, moved into b), T = 0 on the no-flow faces x2 = 0, 1.
// Solver (Sec. 3.5 uses CG preconditioned by one multigrid cycle, stopping at
// ||r|| / ||r0|| < tol, x0 = 0): the multigrid here is geometric and
// matrix-free: cell-centred 2x2 aggregation, coarse faces T_c = (T_a + T_b)/2
// over the two fine faces that make up a coarse face (the rediscretisation of
// a constant k), restriction = sum of the four fine residuals, prolongation =
// piecewise constant, red-black Gauss-Seidel smoothing (red-black before the
// coarse correction, black-red after it, so the cycle is symmetric), exact
// solve on the 4 x 4 grid (a dense inverse formed once per system; on an idle
// warp-wide grid the smaller levels cost as much as the 8 x 8 one).
//
// prec 0: CG and multigrid in FP64.
// prec 1: FP64 iterative refinement (solution, residual b - A x, stopping test
//         and QoI in FP64) around an FP32 CG with FP32 multigrid; the face
//         coefficients are rounded to FP32 once and the FP64 residual uses
//         exactly those values.
// prec 2: prec 1 with the multigrid preconditioner's face coefficients held
//         in BF16 on every level (the CG operator and the FP64 residual keep
//         the FP32 faces; each multigrid level's diagonal is the sum of its
//         own BF16 faces, so the preconditioner stays symmetric positive
//         definite).
// prec 3: FP64 faces, CG vectors, operator, dot products and stopping test;
//         only the multigrid preconditioner runs in FP32 (its faces rounded
//         from the FP64 ones, z = B (float) r widened to FP64).  The CG uses
//         the Polak-Ribiere beta (flexible CG), which tolerates a
//         preconditioner that is symmetric only to FP32 rounding.
// Outflow QoI M^(2) (Sec. 3.4): Q = sum_j T(m, j) p(m-1, j).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>

#include "../../include/mlmc.h"
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "groups.cuh"
#include "layers.cuh"

namespace cg = cooperative_groups;

namespace mlmc {

constexpr int kMaxLevels = 14;
// The coarsening stops at the 4 x 4 grid (or at the finest grid when m < 4),
// which is solved exactly with a dense inverse formed once per system.
constexpr int kCoarseSide = 4;

__host__ __device__ __forceinline__ size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// Workspace bytes of an m x m system, in the order solve_one() lays it out:
// prec 1, 2: FP64 x and r; prec 2: the CG operator's FP32 faces and diagonal;
// per level: faces tx, ty (solver type, BF16 with prec 2), diag, invd, e, f;
// after level 0 the CG vectors x, p, q.  Each array starts 16-byte aligned.
__host__ __device__ inline size_t ws_layout(int m, int prec) {
  const size_t ts = prec ? 4 : 8, fs = prec == 2 ? 2 : ts;
  size_t o = 0;
  const size_t n = (size_t)m * m, nf0 = (size_t)m * (m + 1);
  auto take = [&](size_t bytes) { o += align16(bytes); };
  if (prec)  // x64, r64 (prec 3 also p64, q64, z64)
    for (int v = 0; v < (prec == 3 ? 5 : 2); ++v) take(n * 8);
  if (prec >= 2) {  // the CG operator's own faces and diagonal (FP32, or FP64 with prec 3)
    const size_t os = prec == 3 ? 8 : 4;
    take(nf0 * os);
    take(nf0 * os);
    take(n * os);
  }
  for (int ml = m, l = 0;; ml >>= 1, ++l) {
    const size_t nl = (size_t)ml * ml, nf = (size_t)ml * (ml + 1);
    take(nf * fs);
    take(nf * fs);
    for (int a = 0; a < 4; ++a) take(nl * ts);
    if (l == 0 && prec != 3)
      for (int b = 0; b < 3; ++b) take(nl * ts);
    if (ml <= kCoarseSide) {  // coarsest grid: its dense inverse and a pivot buffer
      take(nl * nl * ts);
      take((2 * nl + 1) * ts);
      break;
    }
  }
  return o;
}

// Face coefficients are stored as F and used in the arithmetic type T.
template <typename T>
__device__ __forceinline__ T face_ld(T v) {
  return v;
}
__device__ __forceinline__ float face_ld(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename F, typename T>
__device__ __forceinline__ F face_st(T v) {
  return v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 face_st<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}

template <typename T, typename F = T>
struct Level {
  int m;
  F* tx;    // m rows x (m+1) faces
  F* ty;    // (m+1) face rows x m
  T* diag;  // sum of the four faces
  T* invd;  // 1 / diagonal (null for the CG operator of prec 2)
  T* e;     // correction (level 0: CG z)
  T* f;     // right-hand side (level 0: CG r)
  T* cinv;  // coarsest level only: dense inverse [m^2][m^2]
  T* cbuf;  // coarsest level only: pivot row, pivot column (2 m^2 + 1)
  unsigned char* stage;  // shared-memory staging of the half sweeps (null: direct loads)
  int stage_rows;        // rows per staged chunk
  int quads;             // FP32 half sweeps over quads of 16-byte accesses (global workspace,
                         // at least one quad per thread of the group)
};

// Cell arrays (solution, right-hand side, diagonal, CG vectors) are stored
// colour by colour: first the cells with i + j even ("red"), row by row with
// i/2 inside a row, then those with i + j odd ("black").  A red-black half
// sweep then reads and writes unit-stride runs of both colours.  Faces keep
// the natural layout (tx: m rows of m + 1, ty: m + 1 rows of m).  m is a
// power of two (m = 1: a single cell).
__device__ __forceinline__ int log2_pow2(int v) { return 31 - __clz(v); }  // v a power of two

struct RbIndex {
  int m, hm, lhm, half;  // side, m/2, log2(m/2), cells of colour 0
  __device__ __forceinline__ explicit RbIndex(int m_) {
    m = m_;
    hm = m_ >> 1;
    lhm = m_ >= 2 ? log2_pow2(hm) : 0;
    half = (m_ * m_ + 1) >> 1;
  }
  __device__ __forceinline__ int at(int i, int j) const { return ((i + j) & 1) * half + j * hm + (i >> 1); }
  __device__ __forceinline__ void cell(int c, int& i, int& j) const {
    const int col = c >= half ? 1 : 0;
    const int r = c - col * half;
    j = r >> lhm;
    i = ((r - (j << lhm)) << 1) + ((j + col) & 1);
  }
};

// (A v)_c = diag_c v_c - sum over the faces of T v_nbr (v_nbr = 0 outside:
// Dirichlet faces carry T but no neighbour, no-flow faces carry T = 0), for
// the cell (i, j) stored at c.  The four neighbours have the other colour:
// row j of that colour starts at ob, rows j -/+ 1 at ob -/+ m/2.
template <typename T, typename F>
__device__ __forceinline__ T apply_at(const Level<T, F>& L, const T* __restrict__ v, const RbIndex& R, int c, int i,
                                      int j) {
  const int m = L.m;
  const int ob = (((i + j) & 1) ^ 1) * R.half + j * R.hm;
  const int rf = j * (m + 1) + i;
  T s = L.diag[c] * v[c];
  if (i > 0) s -= face_ld(L.tx[rf]) * v[ob + ((i - 1) >> 1)];
  if (i < m - 1) s -= face_ld(L.tx[rf + 1]) * v[ob + ((i + 1) >> 1)];
  if (j > 0) s -= face_ld(L.ty[j * m + i]) * v[ob - R.hm + (i >> 1)];
  if (j < m - 1) s -= face_ld(L.ty[(j + 1) * m + i]) * v[ob + R.hm + (i >> 1)];
  return s;
}

// Cell loops below process G::kU cells per thread at a time, all loads of
// the batch before any store (the cells of one batch never read each other's
// outputs: same-colour cells of a red-black sweep, or distinct cells of a
// pointwise update).  Measured on GB300, batches of 2 or 4 raised register
// use enough to lower occupancy and ran slower in every plan (the cluster
// plan at m = 2048: 22 -> 66 ms per sample), so all plans use 1.

// Red (color 0) or black (color 1) Gauss-Seidel half sweep; `zero_guess`
// treats the other color as zero (first sweep of a cycle).
// ---- staged half sweeps ------------------------------------------------------
// In the cluster plans (workspace in global memory) a half sweep on a grid
// of side m >= kStageMin runs over chunks of `rows` grid rows: the chunk's right-hand side and
// inverse diagonal (own colour), the neighbour-colour rows j0 - 1 .. j0 + rows,
// and the faces of its rows are copied into shared memory with asynchronous
// 16-byte copies while the previous chunk is updated from shared memory (two
// buffers), so each thread keeps many loads in flight without holding
// registers for them.  The update is rb_sweep's, term for term.
constexpr int kStageMin = 128;

template <typename T>
struct StageVec {
  static constexpr int V = 16 / (int)sizeof(T);  // elements per 16-byte copy
};

// Element offsets of one chunk buffer (rows r at side m), each a multiple of
// 16 bytes: f, invd (r m/2 each), neighbour-colour rows ((r + 2) m/2), tx (the
// run of r (m + 1) faces widened to 16-byte boundaries), ty ((r + 1) m); size
// = the buffer's elements.
struct StageLayout {
  int f, d, e, x, y, size;
};
template <typename T>
__host__ __device__ inline StageLayout stage_layout(int m, int r) {
  const int V = StageVec<T>::V;
  const int hm = m / 2;
  auto up = [V](int n) { return (n + V - 1) / V * V; };
  StageLayout S;
  S.f = 0;
  S.d = S.f + up(r * hm);
  S.e = S.d + up(r * hm);
  S.x = S.e + up((r + 2) * hm);
  S.y = S.x + up(r * (m + 1) + 2 * V);
  S.size = S.y + up((r + 1) * m);
  return S;
}

// Rows per chunk: about one cell of the half sweep per thread of a block.
__host__ __device__ inline int stage_rows_for(int m, int threads) {
  const int r = threads / (m / 2);
  return r < 1 ? 1 : r;
}

// Shared-memory bytes of the two chunk buffers of a level of side ml.
template <typename T>
__host__ __device__ inline size_t stage_level_bytes(int ml, int threads) {
  return 2 * (size_t)stage_layout<T>(ml, stage_rows_for(ml, threads)).size * sizeof(T);
}

// A level is staged when ml >= kStageMin and its buffers fit in kStageCap;
// the launch reserves the largest of those (0: no level is staged).
constexpr size_t kStageCap = 96 * 1024;
template <typename T>
inline size_t stage_bytes_for(int m, int threads) {
  size_t best = 0;
  for (int ml = m; ml >= kStageMin; ml >>= 1) {
    const size_t bytes = stage_level_bytes<T>(ml, threads);
    if (bytes <= kStageCap && bytes > best) best = bytes;
  }
  return best;
}

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src_global) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src_global) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copy `count` elements (a multiple of 16 bytes; both ends 16-byte aligned).
template <typename T>
__device__ __forceinline__ void stage_copy(T* dst, const T* src, int count, int tid, int nt) {
  constexpr int V = StageVec<T>::V;
  for (int q = tid * V; q < count; q += nt * V) cp_async16(dst + q, src + q);
}

// Issue the copies of chunk q (rows q*rows ..) into chunk buffer s.
template <typename T>
__device__ __forceinline__ void stage_issue(const Level<T, T>& L, const StageLayout& S, T* s, int q, int rows,
                                            int hm, int own0, int oth0, bool zero_guess, int tid, int nt) {
  constexpr int V = StageVec<T>::V;
  const int m = L.m;
  const int j0 = q * rows;
  const int nr = min(rows, m - j0);
  stage_copy(s + S.f, L.f + own0 + j0 * hm, nr * hm, tid, nt);
  stage_copy(s + S.d, L.invd + own0 + j0 * hm, nr * hm, tid, nt);
  if (!zero_guess) {
    const int jlo = max(j0 - 1, 0), jhi = min(j0 + nr, m - 1);
    stage_copy(s + S.e, L.e + oth0 + jlo * hm, (jhi - jlo + 1) * hm, tid, nt);
    const int x0 = j0 * (m + 1), xa = x0 & ~(V - 1), xe = (j0 + nr) * (m + 1);
    stage_copy(s + S.x, L.tx + xa, (xe - xa + V - 1) & ~(V - 1), tid, nt);
    stage_copy(s + S.y, L.ty + j0 * m, (nr + 1) * m, tid, nt);
  }
  cp_async_commit();
}

template <typename T, typename G>
__device__ void rb_sweep_staged(const G& g, const Level<T, T>& L, int color, bool zero_guess) {
  constexpr int V = StageVec<T>::V;
  const int m = L.m;
  const RbIndex R(m);
  const int hm = R.hm;
  const int rows = L.stage_rows;
  const StageLayout S = stage_layout<T>(m, rows);
  const int of = S.f, od = S.d, oe = S.e, ox = S.x, oy = S.y, bsz = S.size;
  T* const buf = reinterpret_cast<T*>(L.stage);
  const int own0 = color * R.half, oth0 = (color ^ 1) * R.half;
  const int nchunk = (m + rows - 1) / rows;
  const int tid = g.lrank(), nt = g.lsize(), np = g.nblocks();
  int q = g.block_index(), t = 0;
  if (q < nchunk) stage_issue(L, S, buf, q, rows, hm, own0, oth0, zero_guess, tid, nt);
  for (; q < nchunk; q += np, ++t) {
    if (q + np < nchunk) {
      stage_issue(L, S, buf + ((t + 1) & 1) * bsz, q + np, rows, hm, own0, oth0, zero_guess, tid, nt);
      cp_async_wait<1>();  // this thread's copies of chunk q are done
    } else {
      cp_async_wait<0>();
    }
    g.lsync();  // and every thread's
    const T* s = buf + (t & 1) * bsz;
    const int j0 = q * rows, nr = min(rows, m - j0);
    const int jlo = max(j0 - 1, 0);
    const int x0 = j0 * (m + 1), xd = x0 - (x0 & ~(V - 1));
    T* const out = L.e + own0 + j0 * hm;
    for (int h = tid; h < nr * hm; h += nt) {
      const int jr = h >> R.lhm, k = h - (jr << R.lhm);
      const int j = j0 + jr;
      const int sh = (j + color) & 1;
      const int i = (k << 1) + sh;
      T v = s[of + h];
      if (!zero_guess) {
        const T* e = s + oe + (j - jlo) * hm + k;
        const T* tx = s + ox + xd + jr * (m + 1) + i;
        const T* ty = s + oy + jr * m + i;
        if (i > 0) v += tx[0] * e[sh - 1];
        if (i < m - 1) v += tx[1] * e[sh];
        if (j > 0) v += ty[0] * e[-hm];
        if (j < m - 1) v += ty[m] * e[hm];
      }
      out[h] = v * s[od + h];
    }
    g.lsync();  // buffer t & 1 is refilled two chunks later
  }
  g.sync();
}

// Four consecutive FP32 values of a cell or face array, one 16-byte access
// (the index a multiple of 4 from a 16-byte aligned array start).
struct F4 {
  float v[4];
};
__device__ __forceinline__ F4 ld4(const float* p) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  return F4{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ void st4(float* p, const F4& a) {
  *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}

// FP32 half sweep over quads of four consecutive cells of one colour in a
// row (m >= 8, so a colour row holds a multiple of four cells): the own
// colour's f, inverse diagonal and new e, the other colour's rows j - 1 and
// j + 1 at the same four indices, the other colour's row j (indices k0 - 1 ..
// k0 + 4) and the y-faces of rows j and j + 1 (columns 2 k0 .. 2 k0 + 7) move
// as 16-byte accesses; the x-faces (row stride m + 1, not aligned) as single
// values.  The arithmetic is rb_sweep's, term for term.
template <typename G>
__device__ __forceinline__ void rb_sweep_quads(const G& g, const Level<float, float>& L, int color, bool zero_guess) {
  const int m = L.m;
  const RbIndex R(m);
  const int hm = R.hm;
  const int nq = (m * hm) >> 2;
  const int own0 = color * R.half, oth0 = (color ^ 1) * R.half;
  for (int q = g.rank(); q < nq; q += g.size()) {
    const int h0 = q << 2;
    const int j = h0 >> R.lhm, k0 = h0 - (j << R.lhm);
    const int sh = (j + color) & 1;
    const int c0 = own0 + h0;
    F4 s = ld4(L.f + c0);
    const F4 id = ld4(L.invd + c0);
    if (!zero_guess) {
      const int ob = oth0 + j * hm + k0;
      const F4 mid = ld4(L.e + ob);
      float W[4], E[4];
      if (sh) {
        const float after = k0 + 4 < hm ? L.e[ob + 4] : 0.f;  // k0 + 4 (unused at the east boundary)
        W[0] = mid.v[0]; W[1] = mid.v[1]; W[2] = mid.v[2]; W[3] = mid.v[3];
        E[0] = mid.v[1]; E[1] = mid.v[2]; E[2] = mid.v[3]; E[3] = after;
      } else {
        const float before = k0 > 0 ? L.e[ob - 1] : 0.f;  // k0 - 1 (unused at the west boundary)
        W[0] = before; W[1] = mid.v[0]; W[2] = mid.v[1]; W[3] = mid.v[2];
        E[0] = mid.v[0]; E[1] = mid.v[1]; E[2] = mid.v[2]; E[3] = mid.v[3];
      }
      const int i0 = 2 * k0 + sh;
      const float* tx = L.tx + j * (m + 1) + i0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + 2 * u;
        if (i > 0) s.v[u] += tx[2 * u] * W[u];
        if (i < m - 1) s.v[u] += tx[2 * u + 1] * E[u];
      }
      if (j > 0) {
        const F4 es = ld4(L.e + ob - hm);
        const F4 ta = ld4(L.ty + j * m + 2 * k0), tb = ld4(L.ty + j * m + 2 * k0 + 4);
        const float ty[4] = {sh ? ta.v[1] : ta.v[0], sh ? ta.v[3] : ta.v[2], sh ? tb.v[1] : tb.v[0],
                             sh ? tb.v[3] : tb.v[2]};
#pragma unroll
        for (int u = 0; u < 4; ++u) s.v[u] += ty[u] * es.v[u];
      }
      if (j < m - 1) {
        const F4 en = ld4(L.e + ob + hm);
        const F4 ta = ld4(L.ty + (j + 1) * m + 2 * k0), tb = ld4(L.ty + (j + 1) * m + 2 * k0 + 4);
        const float ty[4] = {sh ? ta.v[1] : ta.v[0], sh ? ta.v[3] : ta.v[2], sh ? tb.v[1] : tb.v[0],
                             sh ? tb.v[3] : tb.v[2]};
#pragma unroll
        for (int u = 0; u < 4; ++u) s.v[u] += ty[u] * en.v[u];
      }
    }
    F4 out;
#pragma unroll
    for (int u = 0; u < 4; ++u) out.v[u] = s.v[u] * id.v[u];
    st4(L.e + c0, out);
  }
  g.sync();
}

// ---- FP32 CG passes over quads (streamed finest grids) ----
// The CG iteration's passes on 16-byte accesses, for the same grids as the
// quad half sweeps: q = A p over quads of one colour (apply_at's terms in its
// order, the neighbours as in rb_sweep_quads), and the pointwise updates over
// quads of the whole cell array (n = m^2 a multiple of 4).  Each returns the
// calling thread's part of its dot product.
template <typename G>
__device__ __forceinline__ float cg_matvec_quads(const G& g, const Level<float, float>& A,
                                                 const float* __restrict__ p, float* __restrict__ q) {
  const int m = A.m;
  const RbIndex R(m);
  const int hm = R.hm;
  const int nq = (m * hm) >> 2;  // quads of one colour
  float pq = 0.f;
  for (int t = g.rank(); t < 2 * nq; t += g.size()) {
    const int color = t >= nq ? 1 : 0;
    const int h0 = (t - color * nq) << 2;
    const int j = h0 >> R.lhm, k0 = h0 - (j << R.lhm);
    const int sh = (j + color) & 1;
    const int c0 = color * R.half + h0;
    const int ob = (color ^ 1) * R.half + j * hm + k0;
    const F4 v = ld4(p + c0), d = ld4(A.diag + c0), mid = ld4(p + ob);
    float W[4], E[4];
    if (sh) {
      const float after = k0 + 4 < hm ? p[ob + 4] : 0.f;
      W[0] = mid.v[0]; W[1] = mid.v[1]; W[2] = mid.v[2]; W[3] = mid.v[3];
      E[0] = mid.v[1]; E[1] = mid.v[2]; E[2] = mid.v[3]; E[3] = after;
    } else {
      const float before = k0 > 0 ? p[ob - 1] : 0.f;
      W[0] = before; W[1] = mid.v[0]; W[2] = mid.v[1]; W[3] = mid.v[2];
      E[0] = mid.v[0]; E[1] = mid.v[1]; E[2] = mid.v[2]; E[3] = mid.v[3];
    }
    F4 s;
#pragma unroll
    for (int u = 0; u < 4; ++u) s.v[u] = d.v[u] * v.v[u];
    const int i0 = 2 * k0 + sh;
    const float* tx = A.tx + j * (m + 1) + i0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + 2 * u;
      if (i > 0) s.v[u] -= tx[2 * u] * W[u];
      if (i < m - 1) s.v[u] -= tx[2 * u + 1] * E[u];
    }
    if (j > 0) {
      const F4 es = ld4(p + ob - hm);
      const F4 ta = ld4(A.ty + j * m + 2 * k0), tb = ld4(A.ty + j * m + 2 * k0 + 4);
      const float ty[4] = {sh ? ta.v[1] : ta.v[0], sh ? ta.v[3] : ta.v[2], sh ? tb.v[1] : tb.v[0],
                           sh ? tb.v[3] : tb.v[2]};
#pragma unroll
      for (int u = 0; u < 4; ++u) s.v[u] -= ty[u] * es.v[u];
    }
    if (j < m - 1) {
      const F4 en = ld4(p + ob + hm);
      const F4 ta = ld4(A.ty + (j + 1) * m + 2 * k0), tb = ld4(A.ty + (j + 1) * m + 2 * k0 + 4);
      const float ty[4] = {sh ? ta.v[1] : ta.v[0], sh ? ta.v[3] : ta.v[2], sh ? tb.v[1] : tb.v[0],
                           sh ? tb.v[3] : tb.v[2]};
#pragma unroll
      for (int u = 0; u < 4; ++u) s.v[u] -= ty[u] * en.v[u];
    }
    st4(q + c0, s);
#pragma unroll
    for (int u = 0; u < 4; ++u) pq += v.v[u] * s.v[u];
  }
  return pq;
}

// x += alpha p, r -= alpha q; returns the part of r.r
template <typename G>
__device__ __forceinline__ float cg_update_quads(const G& g, int n, float alpha, float* __restrict__ x,
                                                 const float* __restrict__ p, float* __restrict__ r,
                                                 const float* __restrict__ q) {
  float rr = 0.f;
  for (int t = g.rank(); t < (n >> 2); t += g.size()) {
    const int c = t << 2;
    F4 xv = ld4(x + c), rv = ld4(r + c);
    const F4 pv = ld4(p + c), qv = ld4(q + c);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      xv.v[u] += alpha * pv.v[u];
      rv.v[u] = rv.v[u] - alpha * qv.v[u];
      rr += rv.v[u] * rv.v[u];
    }
    st4(x + c, xv);
    st4(r + c, rv);
  }
  return rr;
}

// part of a.b
template <typename G>
__device__ __forceinline__ float cg_dot_quads(const G& g, int n, const float* __restrict__ a,
                                              const float* __restrict__ b) {
  float s = 0.f;
  for (int t = g.rank(); t < (n >> 2); t += g.size()) {
    const F4 av = ld4(a + 4 * t), bv = ld4(b + 4 * t);
#pragma unroll
    for (int u = 0; u < 4; ++u) s += av.v[u] * bv.v[u];
  }
  return s;
}

// p = z + beta p
template <typename G>
__device__ __forceinline__ void cg_xpay_quads(const G& g, int n, float beta, const float* __restrict__ z,
                                              float* __restrict__ p) {
  for (int t = g.rank(); t < (n >> 2); t += g.size()) {
    const F4 zv = ld4(z + 4 * t);
    F4 pv = ld4(p + 4 * t);
#pragma unroll
    for (int u = 0; u < 4; ++u) pv.v[u] = zv.v[u] + beta * pv.v[u];
    st4(p + 4 * t, pv);
  }
}

// ---- FP64 refinement passes over quads (the same grids) ----
// Four consecutive FP64 values, two 16-byte accesses.
struct D4 {
  double v[4];
};
__device__ __forceinline__ D4 ld4d(const double* p) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  return D4{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4d(double* p, const D4& a) {
  *reinterpret_cast<double2*>(p) = make_double2(a.v[0], a.v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(a.v[2], a.v[3]);
}

// r64 = b - A64 x64 with A64 = the FP32 faces widened (the refinement
// residual's terms in its order, the diagonal the FP64 sum of the four
// faces); returns the part of r64.r64.
template <typename G>
__device__ __forceinline__ double ref_residual_quads(const G& g, const Level<float, float>& A,
                                                     const double* __restrict__ x64, double* __restrict__ r64,
                                                     int problem, double fmid) {
  const int m = A.m;
  const RbIndex R(m);
  const int hm = R.hm;
  const int nq = (m * hm) >> 2;
  double s2 = 0.0;
  for (int t = g.rank(); t < 2 * nq; t += g.size()) {
    const int color = t >= nq ? 1 : 0;
    const int h0 = (t - color * nq) << 2;
    const int j = h0 >> R.lhm, k0 = h0 - (j << R.lhm);
    const int sh = (j + color) & 1;
    const int c0 = color * R.half + h0;
    const int ob = (color ^ 1) * R.half + j * hm + k0;
    const D4 xc = ld4d(x64 + c0), mid = ld4d(x64 + ob);
    double W[4], E[4];
    if (sh) {
      const double after = k0 + 4 < hm ? x64[ob + 4] : 0.0;
      W[0] = mid.v[0]; W[1] = mid.v[1]; W[2] = mid.v[2]; W[3] = mid.v[3];
      E[0] = mid.v[1]; E[1] = mid.v[2]; E[2] = mid.v[3]; E[3] = after;
    } else {
      const double before = k0 > 0 ? x64[ob - 1] : 0.0;
      W[0] = before; W[1] = mid.v[0]; W[2] = mid.v[1]; W[3] = mid.v[2];
      E[0] = mid.v[0]; E[1] = mid.v[1]; E[2] = mid.v[2]; E[3] = mid.v[3];
    }
    D4 S{{0.0, 0.0, 0.0, 0.0}}, N{{0.0, 0.0, 0.0, 0.0}};
    if (j > 0) S = ld4d(x64 + ob - hm);
    if (j < m - 1) N = ld4d(x64 + ob + hm);
    const F4 sa = ld4(A.ty + j * m + 2 * k0), sb = ld4(A.ty + j * m + 2 * k0 + 4);
    const F4 na = ld4(A.ty + (j + 1) * m + 2 * k0), nb = ld4(A.ty + (j + 1) * m + 2 * k0 + 4);
    const float tys[4] = {sh ? sa.v[1] : sa.v[0], sh ? sa.v[3] : sa.v[2], sh ? sb.v[1] : sb.v[0],
                          sh ? sb.v[3] : sb.v[2]};
    const float tyn[4] = {sh ? na.v[1] : na.v[0], sh ? na.v[3] : na.v[2], sh ? nb.v[1] : nb.v[0],
                          sh ? nb.v[3] : nb.v[2]};
    const int i0 = 2 * k0 + sh;
    const float* tx = A.tx + j * (m + 1) + i0;
    D4 out;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + 2 * u;
      const double tw = (double)tx[2 * u], te = (double)tx[2 * u + 1];
      const double ts = (double)tys[u], tn = (double)tyn[u];
      double ax = ((tw + te) + (ts + tn)) * xc.v[u];
      if (i > 0) ax -= tw * W[u];
      if (i < m - 1) ax -= te * E[u];
      if (j > 0) ax -= ts * S.v[u];
      if (j < m - 1) ax -= tn * N.v[u];
      const double bv = problem == 1 ? fmid : (i == 0 ? tw : 0.0);
      out.v[u] = bv - ax;
      s2 += out.v[u] * out.v[u];
    }
    st4d(r64 + c0, out);
  }
  return s2;
}

// x64 += scl xv
template <typename G>
__device__ __forceinline__ void ref_update_quads(const G& g, int n, double scl, double* __restrict__ x64,
                                                 const float* __restrict__ xv) {
  for (int t = g.rank(); t < (n >> 2); t += g.size()) {
    D4 x = ld4d(x64 + 4 * t);
    const F4 d = ld4(xv + 4 * t);
#pragma unroll
    for (int u = 0; u < 4; ++u) x.v[u] += scl * (double)d.v[u];
    st4d(x64 + 4 * t, x);
  }
}

// f = (float)(r64 inv), optionally xv = 0 and pv *= ratio; returns the part of f.f
template <typename G>
__device__ __forceinline__ float ref_rescale_quads(const G& g, int n, double inv, const double* __restrict__ r64,
                                                   float* __restrict__ f, float* __restrict__ xv,
                                                   float* __restrict__ pv, float ratio) {
  float s = 0.f;
  const F4 zero{{0.f, 0.f, 0.f, 0.f}};
  for (int t = g.rank(); t < (n >> 2); t += g.size()) {
    const D4 r = ld4d(r64 + 4 * t);
    F4 v;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      v.v[u] = (float)(r.v[u] * inv);
      s += v.v[u] * v.v[u];
    }
    st4(f + 4 * t, v);
    if (xv) st4(xv + 4 * t, zero);
    if (pv) {
      F4 pp = ld4(pv + 4 * t);
#pragma unroll
      for (int u = 0; u < 4; ++u) pp.v[u] *= ratio;
      st4(pv + 4 * t, pp);
    }
  }
  return s;
}

template <typename T, typename F, typename G>
__device__ __forceinline__ void rb_sweep(const G& g, const Level<T, F>& L, int color, bool zero_guess) {
  if constexpr (std::is_same<T, F>::value && G::kStaged) {
    if (L.stage) {
      rb_sweep_staged(g, L, color, zero_guess);
      return;
    }
  }
  if constexpr (std::is_same<T, float>::value && std::is_same<F, float>::value && G::kQuads) {
    if (L.quads) {
      rb_sweep_quads(g, L, color, zero_guess);
      return;
    }
  }
  const int m = L.m;
  const RbIndex R(m);
  const int nh = m * R.hm;  // cells of one colour
  const int own0 = color * R.half, oth0 = (color ^ 1) * R.half;
  const int step = g.size();
  int h0 = g.rank();
  for (; h0 < nh; h0 += G::kU * step) {
    T val[G::kU];
    int cc[G::kU];
#pragma unroll
    for (int u = 0; u < G::kU; ++u) {
      const int h = h0 + u * step;
      cc[u] = -1;
      if (h < nh) {
        const int j = h >> R.lhm;
        const int k = h - (j << R.lhm);
        const int sh = (j + color) & 1;  // i = 2k + sh; west neighbour at k - 1 + sh, east at k + sh
        const int i = (k << 1) + sh;
        const int c = own0 + h;
        T s = L.f[c];
        if (!zero_guess) {
          const int rf = j * (m + 1) + i;
          const int ob = oth0 + j * R.hm + k;
          if (i > 0) s += face_ld(L.tx[rf]) * L.e[ob - 1 + sh];
          if (i < m - 1) s += face_ld(L.tx[rf + 1]) * L.e[ob + sh];
          if (j > 0) s += face_ld(L.ty[j * m + i]) * L.e[ob - R.hm];
          if (j < m - 1) s += face_ld(L.ty[(j + 1) * m + i]) * L.e[ob + R.hm];
        }
        val[u] = s * L.invd[c];
        cc[u] = c;
      }
    }
#pragma unroll
    for (int u = 0; u < G::kU; ++u)
      if (cc[u] >= 0) L.e[cc[u]] = val[u];
  }
  g.sync();
}

// (A e) at a quad of four consecutive cells of colour `color` in row j
// (own-colour indices k0 .. k0 + 3): apply_at's terms in its order, with the
// neighbours read as in rb_sweep_quads.
template <typename G>
__device__ __forceinline__ F4 apply_quad(const Level<float, float>& L, const float* __restrict__ e, int color, int j,
                                         int k0) {
  const int m = L.m;
  const RbIndex R(m);
  const int hm = R.hm;
  const int sh = (j + color) & 1;
  const int c0 = color * R.half + j * hm + k0;
  const int ob = (color ^ 1) * R.half + j * hm + k0;
  const F4 v = ld4(e + c0), d = ld4(L.diag + c0), mid = ld4(e + ob);
  float W[4], E[4];
  if (sh) {
    const float after = k0 + 4 < hm ? e[ob + 4] : 0.f;
    W[0] = mid.v[0]; W[1] = mid.v[1]; W[2] = mid.v[2]; W[3] = mid.v[3];
    E[0] = mid.v[1]; E[1] = mid.v[2]; E[2] = mid.v[3]; E[3] = after;
  } else {
    const float before = k0 > 0 ? e[ob - 1] : 0.f;
    W[0] = before; W[1] = mid.v[0]; W[2] = mid.v[1]; W[3] = mid.v[2];
    E[0] = mid.v[0]; E[1] = mid.v[1]; E[2] = mid.v[2]; E[3] = mid.v[3];
  }
  F4 s;
#pragma unroll
  for (int u = 0; u < 4; ++u) s.v[u] = d.v[u] * v.v[u];
  const int i0 = 2 * k0 + sh;
  const float* tx = L.tx + j * (m + 1) + i0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + 2 * u;
    if (i > 0) s.v[u] -= tx[2 * u] * W[u];
    if (i < m - 1) s.v[u] -= tx[2 * u + 1] * E[u];
  }
  if (j > 0) {
    const F4 es = ld4(e + ob - hm);
    const F4 ta = ld4(L.ty + j * m + 2 * k0), tb = ld4(L.ty + j * m + 2 * k0 + 4);
    const float ty[4] = {sh ? ta.v[1] : ta.v[0], sh ? ta.v[3] : ta.v[2], sh ? tb.v[1] : tb.v[0],
                         sh ? tb.v[3] : tb.v[2]};
#pragma unroll
    for (int u = 0; u < 4; ++u) s.v[u] -= ty[u] * es.v[u];
  }
  if (j < m - 1) {
    const F4 en = ld4(e + ob + hm);
    const F4 ta = ld4(L.ty + (j + 1) * m + 2 * k0), tb = ld4(L.ty + (j + 1) * m + 2 * k0 + 4);
    const float ty[4] = {sh ? ta.v[1] : ta.v[0], sh ? ta.v[3] : ta.v[2], sh ? tb.v[1] : tb.v[0],
                         sh ? tb.v[3] : tb.v[2]};
#pragma unroll
    for (int u = 0; u < 4; ++u) s.v[u] -= ty[u] * en.v[u];
  }
  return s;
}

// restrict_residual over quads (FP32, the fine level m >= 8 streamed): four
// consecutive coarse cells I0 .. I0 + 3 of coarse row J take the red quads
// k = I0 .. I0 + 3 of fine rows 2J and 2J + 1; in the coarse colour-by-colour
// layout they are two pairs (columns I0, I0 + 2 of one colour and I0 + 1,
// I0 + 3 of the other), stored as 8-byte accesses.
template <typename G>
__device__ __forceinline__ void restrict_residual_quads(const G& g, const Level<float, float>& F,
                                                        const Level<float, float>& C) {
  const int mc = C.m, m = F.m;
  const RbIndex Rf(m), Rc(mc);
  const int qpr = mc >> 2;  // coarse quads per row
  const int nqc = mc * qpr;
  for (int t = g.rank(); t < nqc; t += g.size()) {
    const int J = t / qpr, I0 = (t - J * qpr) << 2;
    const F4 a0 = apply_quad<G>(F, F.e, 0, 2 * J, I0), a1 = apply_quad<G>(F, F.e, 0, 2 * J + 1, I0);
    const F4 f0 = ld4(F.f + 2 * J * Rf.hm + I0), f1 = ld4(F.f + (2 * J + 1) * Rf.hm + I0);
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = (f0.v[u] - a0.v[u]) + (f1.v[u] - a1.v[u]);
    const int ca = J & 1;  // colour of coarse columns I0, I0 + 2
    const int base_a = ca * Rc.half + J * Rc.hm + (I0 >> 1), base_b = (ca ^ 1) * Rc.half + J * Rc.hm + (I0 >> 1);
    *reinterpret_cast<float2*>(C.f + base_a) = make_float2(v[0], v[2]);
    *reinterpret_cast<float2*>(C.f + base_b) = make_float2(v[1], v[3]);
  }
  g.sync();
}

// prolong_add over quads: the fine quad k0 .. k0 + 3 of row j (either
// colour) takes coarse columns k0 .. k0 + 3 of coarse row j >> 1, two pairs
// of the coarse layout.
template <typename G>
__device__ __forceinline__ void prolong_add_quads(const G& g, const Level<float, float>& C,
                                                  const Level<float, float>& F) {
  const int m = F.m;
  const RbIndex Rf(m), Rc(C.m);
  const int nq = (m * Rf.hm) >> 2;  // quads of one colour
  for (int t = g.rank(); t < 2 * nq; t += g.size()) {
    const int color = t >= nq ? 1 : 0;
    const int h0 = (t - color * nq) << 2;
    const int j = h0 >> Rf.lhm, k0 = h0 - (j << Rf.lhm);
    const int J = j >> 1;
    const int ca = J & 1;
    const float2 pa = *reinterpret_cast<const float2*>(C.e + ca * Rc.half + J * Rc.hm + (k0 >> 1));
    const float2 pb = *reinterpret_cast<const float2*>(C.e + (ca ^ 1) * Rc.half + J * Rc.hm + (k0 >> 1));
    const int c0 = color * Rf.half + h0;
    F4 e = ld4(F.e + c0);
    e.v[0] += pa.x;
    e.v[1] += pb.x;
    e.v[2] += pa.y;
    e.v[3] += pb.y;
    st4(F.e + c0, e);
  }
  g.sync();
}

// Coarse f = sum of the fine residuals f - A e over each 2x2 aggregate.
// Called right after a black half sweep, which leaves the residual at the
// black cells zero, so only the two red cells (2I, 2J), (2I+1, 2J+1) of the
// aggregate contribute.
template <typename T, typename FT, typename G>
__device__ __forceinline__ void restrict_residual(const G& g, const Level<T, FT>& F, const Level<T, FT>& C) {
  if constexpr (std::is_same<T, float>::value && std::is_same<FT, float>::value && G::kQuads) {
    if (F.quads) {
      restrict_residual_quads(g, F, C);
      return;
    }
  }
  const int mc = C.m, m = F.m;
  const RbIndex Rf(m), Rc(mc);
  const int lmc = log2_pow2(mc);
  const int nc = mc * mc, step = g.size();
  for (int c0 = g.rank(); c0 < nc; c0 += G::kU * step) {
    T val[G::kU];
    int dst[G::kU];
#pragma unroll
    for (int u = 0; u < G::kU; ++u) {
      const int t = c0 + u * step;  // coarse cell (I, J) in natural order
      dst[u] = -1;
      if (t < nc) {
        const int J = t >> lmc, I = t - (J << lmc);
        const int i0 = 2 * I, j0 = 2 * J;
        const int f0 = J * m + I, f1 = f0 + Rf.hm;  // the red cells (2I, 2J) and (2I+1, 2J+1)
        const T r0 = F.f[f0] - apply_at(F, F.e, Rf, f0, i0, j0);
        const T r1 = F.f[f1] - apply_at(F, F.e, Rf, f1, i0 + 1, j0 + 1);
        val[u] = r0 + r1;
        dst[u] = Rc.at(I, J);
      }
    }
#pragma unroll
    for (int u = 0; u < G::kU; ++u)
      if (dst[u] >= 0) C.f[dst[u]] = val[u];
  }
  g.sync();
}

template <typename T, typename FT, typename G>
__device__ __forceinline__ void prolong_add(const G& g, const Level<T, FT>& C, const Level<T, FT>& F) {
  if constexpr (std::is_same<T, float>::value && std::is_same<FT, float>::value && G::kQuads) {
    if (F.quads) {
      prolong_add_quads(g, C, F);
      return;
    }
  }
  const int m = F.m, mc = C.m;
  const RbIndex Rf(m), Rc(mc);
  const int n = m * m, step = g.size();
  for (int c0 = g.rank(); c0 < n; c0 += G::kU * step) {
    T val[G::kU];
#pragma unroll
    for (int u = 0; u < G::kU; ++u) {
      const int c = c0 + u * step;
      if (c < n) {
        int i, j;
        Rf.cell(c, i, j);
        val[u] = F.e[c] + C.e[Rc.at(i >> 1, j >> 1)];
      }
    }
#pragma unroll
    for (int u = 0; u < G::kU; ++u)
      if (c0 + u * step < n) F.e[c0 + u * step] = val[u];
  }
  g.sync();
}

// Coarse faces: mean of the two fine faces forming each coarse face.
template <typename T, typename FT, typename G>
__device__ __forceinline__ void build_coarse(const G& g, const Level<T, FT>& F, const Level<T, FT>& C) {
  const int m = F.m, mc = C.m;
  const int nfx = mc * (mc + 1);
  for (int t = g.rank(); t < 2 * nfx; t += g.size()) {
    if (t < nfx) {
      const int J = t / (mc + 1), Ip = t - J * (mc + 1);
      C.tx[t] = face_st<FT>(T(0.5) * (face_ld(F.tx[(2 * J) * (m + 1) + 2 * Ip]) +
                                      face_ld(F.tx[(2 * J + 1) * (m + 1) + 2 * Ip])));
    } else {
      const int u = t - nfx;
      const int Jp = u / mc, I = u - Jp * mc;
      C.ty[u] = face_st<FT>(T(0.5) * (face_ld(F.ty[(2 * Jp) * m + 2 * I]) + face_ld(F.ty[(2 * Jp) * m + 2 * I + 1])));
    }
  }
  g.sync();
}

// Diagonal (sum of the four faces) and, with INV, its reciprocal.
template <bool INV, typename T, typename FT, typename G>
__device__ __forceinline__ void build_diag(const G& g, const Level<T, FT>& L) {
  const int m = L.m;
  const RbIndex R(m);
  for (int c = g.rank(); c < m * m; c += g.size()) {
    int i, j;
    R.cell(c, i, j);
    const int rf = j * (m + 1) + i;
    const T d = (face_ld(L.tx[rf]) + face_ld(L.tx[rf + 1])) +
                (face_ld(L.ty[j * m + i]) + face_ld(L.ty[(j + 1) * m + i]));
    L.diag[c] = d;
    if (INV) L.invd[c] = T(1) / d;
  }
  g.sync();
}

// Dense inverse of the coarsest grid's operator (n = m^2 <= 16 unknowns) by
// in-place Gauss-Jordan elimination without pivoting (the matrix is SPD, so
// every pivot, a Schur-complement diagonal, is positive): at step k with
// pivot p, row r_j = B[k][j] and column c_i = B[i][k],
//   B[k][k] <- 1/p, B[k][j] <- r_j / p, B[i][k] <- -c_i / p,
//   B[i][j] <- B[i][j] - c_i (r_j / p);  after n steps B = A^-1.
// The scaled pivot row is formed once per step, and the reciprocal of the
// next pivot by the one thread that writes it (into buf[2n]).
template <typename T, typename F, typename G>
__device__ void build_coarse_inverse(const G& g, const Level<T, F>& L) {
  const int m = L.m, n = m * m, nn = n * n;
  const RbIndex R(m);
  T* B = L.cinv;
  T* buf = L.cbuf;
  for (int idx = g.rank(); idx < nn; idx += g.size()) {
    const int r = idx / n, c = idx - r * n;  // cells in storage order
    int ir, jr, ic, jc;
    R.cell(r, ir, jr);
    R.cell(c, ic, jc);
    T v = T(0);
    if (r == c) v = L.diag[r];
    else if (jr == jc && (ir - ic == 1 || ic - ir == 1)) v = -face_ld(L.tx[jr * (m + 1) + (ir > ic ? ir : ic)]);
    else if (ir == ic && (jr - jc == 1 || jc - jr == 1)) v = -face_ld(L.ty[(jr > jc ? jr : jc) * m + ir]);
    B[idx] = v;
    if (idx == 0) buf[2 * n] = T(1) / v;
  }
  g.sync();
  for (int k = 0; k < n; ++k) {
    const T ip = buf[2 * n];
    for (int t = g.rank(); t < n; t += g.size()) {
      buf[t] = t == k ? ip : B[k * n + t] * ip;
      buf[n + t] = B[t * n + k];
    }
    g.sync();
    const int next = (k + 1) * (n + 1);  // B[k+1][k+1]
    for (int idx = g.rank(); idx < nn; idx += g.size()) {
      const int i = idx / n, j = idx - i * n;
      T v;
      if (i == k) v = buf[j];
      else if (j == k) v = -buf[n + i] * ip;
      else v = fma(-buf[n + i], buf[j], B[idx]);
      B[idx] = v;
      if (idx == next && k + 1 < n) buf[2 * n] = T(1) / v;
    }
    g.sync();
  }
}

// Exact solve on the coarsest grid: e = A^-1 f.
template <typename T, typename F, typename G>
__device__ __forceinline__ void coarse_solve(const G& g, const Level<T, F>& L) {
  const int n = L.m * L.m;
  for (int r = g.rank(); r < n; r += g.size()) {
    const T* row = L.cinv + r * n;
    T s = T(0);
    for (int c = 0; c < n; ++c) s += row[c] * L.f[c];
    L.e[r] = s;
  }
  g.sync();
}

// Symmetric multigrid cycle e_0 <- B f_0: on each level red-black then
// black-red Gauss-Seidel (nu sweep pairs on the finest level, nuc on the
// coarser ones) around the coarse correction, which itself is
// gamma cycles on the next level (gamma = 1: V-cycle, 2: W-cycle; one visit
// when the next level is the coarsest grid, solved exactly).  Written as a loop
// over an explicit per-level visit count (no recursion: the device stack
// stays fixed).  With adjoint pre- and post-smoothing the cycle is a
// symmetric positive definite preconditioner for any gamma.
// zero_start = false starts level 0 from its current e (a repeated visit).
template <typename T, typename F, typename G>
__device__ void mg_cycle(const G& g, const Level<T, F>* lev, int nl, int gamma, int nu, int nuc,
                         bool zero_start = true) {
  int done[kMaxLevels];   // visits of level l+1 finished in the current cycle on level l
  bool zero[kMaxLevels];  // level l starts from e_l = 0
  int l = 0;
  zero[0] = zero_start;
  while (true) {
    if (l < nl - 1) {  // descend: pre-smooth, restrict, enter the next level
      const int ns = l == 0 ? nu : nuc;
      for (int s = 0; s < ns; ++s) {
        rb_sweep(g, lev[l], 0, zero[l] && s == 0);
        rb_sweep(g, lev[l], 1, false);
      }
      restrict_residual(g, lev[l], lev[l + 1]);
      done[l] = 0;
      zero[l + 1] = true;
      ++l;
      continue;
    }
    coarse_solve(g, lev[l]);  // coarsest grid: exact
    // ascend until a level wants another visit of the level below it
    bool revisit = false;
    while (l > 0) {
      const int up = l - 1;
      const int visits = (up + 1 == nl - 1) ? 1 : gamma;
      if (++done[up] < visits) {
        zero[l] = false;  // visit level `l` again, from its current e
        revisit = true;
        break;
      }
      prolong_add(g, lev[l], lev[up]);
      const int ns = up == 0 ? nu : nuc;
      for (int s = 0; s < ns; ++s) {
        rb_sweep(g, lev[up], 1, false);
        rb_sweep(g, lev[up], 0, false);
      }
      l = up;
    }
    if (!revisit) return;
  }
}

// Symmetric V-cycle: level-0 e <- B f (the loop form of mg_cycle, gamma 1).
template <typename T, typename F, typename G>
__device__ void vcycle(const G& g, const Level<T, F>* lev, int nl) {
  for (int l = 0; l < nl - 1; ++l) {
    rb_sweep(g, lev[l], 0, true);
    rb_sweep(g, lev[l], 1, false);
    restrict_residual(g, lev[l], lev[l + 1]);
  }
  coarse_solve(g, lev[nl - 1]);  // coarsest grid: exact
  for (int l = nl - 2; l >= 0; --l) {
    prolong_add(g, lev[l + 1], lev[l]);
    rb_sweep(g, lev[l], 1, false);
    rb_sweep(g, lev[l], 0, false);
  }
}

template <typename T, typename F, typename G>
__device__ __forceinline__ void precond(const G& g, const Level<T, F>* lev, int nl, int gamma, int nu, int nuc) {
  if (nuc < 1) nuc = nu;
  if (gamma <= 1 && nu <= 1 && nuc <= 1)
    vcycle(g, lev, nl);
  else
    mg_cycle(g, lev, nl, gamma < 1 ? 1 : gamma, nu < 1 ? 1 : nu, nuc);
}

// CG on the operator A (faces and diagonal of the finest grid), multigrid
// preconditioner on lev (r = lev[0].f, z = lev[0].e): x = 0 on entry,
// r = rhs.  Stops when r.r <= thr; returns iterations, status 0 converged,
// 1 hit the cap, 2 breakdown (p.Ap <= 0 or not finite).
template <typename T, typename F, typename G>
__device__ int pcg(const G& g, const Level<T>& A, const Level<T, F>* lev, int nl, int gamma, int nu, int nuc,
                   T* __restrict__ x, T* __restrict__ p, T* __restrict__ q, T thr, int max_it, T* red, int& par,
                   int& status) {
  const Level<T, F>& L0 = lev[0];
  const int m = L0.m, n = m * m;
  T* __restrict__ r = L0.f;
  const T* __restrict__ z = L0.e;
  const int step = g.size();
  const RbIndex R(m);
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
  precond(g, lev, nl, gamma, nu, nuc);
  T rz = T(0);
  for (int c = g.rank(); c < n; c += step) {
    p[c] = z[c];
    rz += r[c] * z[c];
  }
  rz = g.sum(rz, red, par);
  int it = 0;
  // FP32 on a streamed finest grid: the passes on 16-byte quads
  bool vq = false;
  if constexpr (std::is_same<T, float>::value && G::kQuads) vq = L0.quads != 0;
  while (it < max_it) {
    ++it;
    T pq = T(0);
    if constexpr (std::is_same<T, float>::value && G::kQuads) {
      if (vq) pq = cg_matvec_quads(g, A, p, q);
    }
    if (!vq)
    for (int c0 = g.rank(); c0 < n; c0 += G::kU * step) {
      T val[G::kU];
#pragma unroll
      for (int u = 0; u < G::kU; ++u) {
        const int c = c0 + u * step;
        val[u] = T(0);
        if (c < n) {
          int i, j;
          R.cell(c, i, j);
          val[u] = apply_at(A, p, R, c, i, j);
          pq += p[c] * val[u];
        }
      }
#pragma unroll
      for (int u = 0; u < G::kU; ++u)
        if (c0 + u * step < n) q[c0 + u * step] = val[u];
    }
    pq = g.sum(pq, red, par);
    if (!(pq > T(0)) || !isfinite(pq) || !isfinite(rz)) {
      status = 2;
      break;
    }
    const T alpha = rz / pq;
    rr = T(0);
    if constexpr (std::is_same<T, float>::value && G::kQuads) {
      if (vq) rr = cg_update_quads(g, n, alpha, x, p, r, q);
    }
    if (!vq)
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
    precond(g, lev, nl, gamma, nu, nuc);
    T rzn = T(0);
    if constexpr (std::is_same<T, float>::value && G::kQuads) {
      if (vq) rzn = cg_dot_quads(g, n, r, z);
    }
    if (!vq)
      for (int c = g.rank(); c < n; c += step) rzn += r[c] * z[c];
    rzn = g.sum(rzn, red, par);
    const T beta = rzn / rz;
    rz = rzn;
    if constexpr (std::is_same<T, float>::value && G::kQuads) {
      if (vq) cg_xpay_quads(g, n, beta, z, p);
    }
    if (!vq)
      for (int c = g.rank(); c < n; c += step) p[c] = z[c] + beta * p[c];
    g.sync();
  }
  return it;
}

// prec 3: CG in FP64 on the FP64 operator A with the FP32 multigrid
// preconditioner on lev: z = (double) B (float) r.  r = rhs on entry, x = 0
// is set here.  beta = r_new.(z_new - z_old) / r_old.z_old (Polak-Ribiere,
// the flexible-CG form), so the preconditioner's FP32 rounding (a slightly
// varying, slightly unsymmetric B) does not stall the iteration.  Stops when
// r.r <= thr; status 0 converged, 1 cap, 2 breakdown.
template <typename G>
__device__ int pcg64_mg32(const G& g, const Level<double>& A, const Level<float>* lev, int nl, int gamma, int nu, int nuc,
                          double* __restrict__ x, double* __restrict__ r, double* __restrict__ p,
                          double* __restrict__ q, double* __restrict__ z, double thr, int max_it, double* red,
                          int& par, int& status) {
  const Level<float>& L0 = lev[0];
  const int m = A.m, n = m * m;
  const int step = g.size();
  const RbIndex R(m);
  double rr = 0.0;
  for (int c = g.rank(); c < n; c += step) {
    x[c] = 0.0;
    const double rv = r[c];
    L0.f[c] = (float)rv;
    rr += rv * rv;
  }
  rr = g.sum(rr, red, par);
  status = 1;
  if (rr <= thr) {
    status = 0;
    return 0;
  }
  g.sync();
  precond(g, lev, nl, gamma, nu, nuc);
  double rz = 0.0;
  for (int c = g.rank(); c < n; c += step) {
    const double zv = (double)L0.e[c];
    z[c] = zv;
    p[c] = zv;
    rz += r[c] * zv;
  }
  rz = g.sum(rz, red, par);
  int it = 0;
  while (it < max_it) {
    ++it;
    double pq = 0.0;
    for (int c = g.rank(); c < n; c += step) {
      int i, j;
      R.cell(c, i, j);
      const double v = apply_at(A, p, R, c, i, j);
      q[c] = v;
      pq += p[c] * v;
    }
    pq = g.sum(pq, red, par);
    if (!(pq > 0.0) || !isfinite(pq) || !(rz > 0.0) || !isfinite(rz)) {
      status = 2;
      break;
    }
    const double alpha = rz / pq;
    rr = 0.0;
    double rzo = 0.0;  // r_new . z_old
    for (int c = g.rank(); c < n; c += step) {
      x[c] += alpha * p[c];
      const double rv = r[c] - alpha * q[c];
      r[c] = rv;
      L0.f[c] = (float)rv;
      rr += rv * rv;
      rzo += rv * z[c];
    }
    rr = g.sum(rr, red, par);
    rzo = g.sum(rzo, red, par);
    if (rr <= thr) {
      status = 0;
      break;
    }
    precond(g, lev, nl, gamma, nu, nuc);
    double rzn = 0.0;
    for (int c = g.rank(); c < n; c += step) {
      const double zv = (double)L0.e[c];
      z[c] = zv;
      rzn += r[c] * zv;
    }
    rzn = g.sum(rzn, red, par);
    const double beta = (rzn - rzo) / rz;
    rz = rzn;
    for (int c = g.rank(); c < n; c += step) p[c] = z[c] + beta * p[c];
    g.sync();
  }
  return it;
}

constexpr int kMaxThreads = 512;
constexpr int kWarpsPerBlock = 4;  // systems per block in warp mode

// Per-system state shared by the threads of one group: the multigrid
// hierarchy and the CG operator (the finest level's arrays, or with prec 2
// separate FP32 faces and diagonal).
template <typename T, typename F>
struct GroupState {
  Level<T, F> lev[kMaxLevels];
  Level<T> op;
  Level<double> op64;  // prec 3: the FP64 CG operator
  T *xv, *pv, *qv;
  double *x64, *r64, *p64, *q64, *z64;
  double eta[MAX_LAYERS_DEV], kc[MAX_LAYERS_DEV];
  int nl;
};

// Launch shape for an m x m system: small grids get one warp per system
// (no block barriers), larger ones a block of about one thread per cell of
// the finest red-black half sweep, up to 512.
__host__ __device__ inline bool solve_warp_mode(int m) { return m <= 16; }
__host__ __device__ inline int solve_threads(int m) {
  return solve_warp_mode(m) ? 32 * kWarpsPerBlock : (m <= 64 ? 256 : 512);
}

// The CG operator: separate FP32 arrays with prec 2, else the finest level.
template <int PREC, typename T, typename F>
__device__ __forceinline__ const Level<T>& cg_operator(const GroupState<T, F>& gs) {
  if constexpr (PREC == 2)
    return gs.op;
  else
    return gs.lev[0];
}

template <int PREC>
struct SolverTypes {
  using T = typename std::conditional<PREC != 0, float, double>::type;       // arithmetic (multigrid)
  using F = typename std::conditional<PREC == 2, __nv_bfloat16, T>::type;  // multigrid faces
};

// Assemble, solve and reduce the QoI of one system with group g.
template <int PREC, typename G>
__device__ void solve_one(const G& g, const SolveArgs& a, int64_t sys, unsigned char* base,
                          GroupState<typename SolverTypes<PREC>::T, typename SolverTypes<PREC>::F>& gs,
                          typename SolverTypes<PREC>::T* red, double* red64, int& par, int& m_prev,
                          unsigned char* base64, unsigned char* stage) {
  using T = typename SolverTypes<PREC>::T;
  using F = typename SolverTypes<PREC>::F;
  using TF = typename std::conditional<PREC == 3, double, T>::type;  // face assembly
  constexpr bool REFINE = PREC == 1 || PREC == 2;                    // FP32 CG in FP64 refinement
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
  const int m = coarse ? a.m >> 1 : a.m;
  const int n = m * m;
  const uint64_t sample = (uint64_t)(a.first + sidx);
  if (m != m_prev) {  // level table of this system size (each block keeps its copy)
    g.sync();
    if (g.local_leader()) {
      // walk the layout of ws_layout() (same order, same alignment)
      size_t o = 0;
      const size_t n0 = (size_t)m * m;
      auto take = [&](size_t bytes) {
        unsigned char* p = base + o;
        o += align16(bytes);
        return p;
      };
      if (PREC != 0) {
        if (base64) {  // FP64 refinement vectors in global memory, the rest on chip
          gs.x64 = reinterpret_cast<double*>(base64);
          gs.r64 = reinterpret_cast<double*>(base64 + align16(n0 * 8));
        } else {
          gs.x64 = reinterpret_cast<double*>(take(n0 * 8));
          gs.r64 = reinterpret_cast<double*>(take(n0 * 8));
        }
      }
      if (PREC == 3) {
        const size_t nf0 = (size_t)m * (m + 1);
        gs.p64 = reinterpret_cast<double*>(take(n0 * 8));
        gs.q64 = reinterpret_cast<double*>(take(n0 * 8));
        gs.z64 = reinterpret_cast<double*>(take(n0 * 8));
        gs.op64.m = m;
        gs.op64.tx = reinterpret_cast<double*>(take(nf0 * 8));
        gs.op64.ty = reinterpret_cast<double*>(take(nf0 * 8));
        gs.op64.diag = reinterpret_cast<double*>(take(n0 * 8));
        gs.op64.invd = nullptr;
      }
      if (PREC == 2) {
        const size_t nf0 = (size_t)m * (m + 1);
        gs.op.tx = reinterpret_cast<T*>(take(nf0 * sizeof(T)));
        gs.op.ty = reinterpret_cast<T*>(take(nf0 * sizeof(T)));
        gs.op.diag = reinterpret_cast<T*>(take(n0 * sizeof(T)));
        gs.op.invd = nullptr;
      }
      int l = 0;
      for (int ml = m;; ml >>= 1, ++l) {
        const size_t nlv = (size_t)ml * ml, nf = (size_t)ml * (ml + 1);
        Level<T, F>& L = gs.lev[l];
        L.m = ml;
        L.tx = reinterpret_cast<F*>(take(nf * sizeof(F)));
        L.ty = reinterpret_cast<F*>(take(nf * sizeof(F)));
        L.diag = reinterpret_cast<T*>(take(nlv * sizeof(T)));
        L.invd = reinterpret_cast<T*>(take(nlv * sizeof(T)));
        L.e = reinterpret_cast<T*>(take(nlv * sizeof(T)));
        L.f = reinterpret_cast<T*>(take(nlv * sizeof(T)));
        if (l == 0 && PREC != 3) {
          gs.xv = reinterpret_cast<T*>(take(nlv * sizeof(T)));
          gs.pv = reinterpret_cast<T*>(take(nlv * sizeof(T)));
          gs.qv = reinterpret_cast<T*>(take(nlv * sizeof(T)));
        }
        L.cinv = L.cbuf = nullptr;
        L.stage = nullptr;
        L.stage_rows = 0;
        // measured on GB300: the quads pay where the level streams from global
        // memory and every thread gets one; on shared-memory levels, or with
        // idle threads, the single-cell loop is faster
        L.quads = !a.use_smem && ml >= 8 && ml * (ml / 2) / 4 >= g.size();
        if (std::is_same<T, F>::value && stage && ml >= kStageMin &&
            stage_level_bytes<T>(ml, (int)blockDim.x) <= a.stage_bytes) {
          L.stage = stage;
          L.stage_rows = stage_rows_for(ml, (int)blockDim.x);
        }
        if (ml <= kCoarseSide) {
          L.cinv = reinterpret_cast<T*>(take(nlv * nlv * sizeof(T)));
          L.cbuf = reinterpret_cast<T*>(take((2 * nlv + 1) * sizeof(T)));
          break;
        }
      }
      gs.nl = l + 1;
      gs.op.m = m;
      gs.op.e = gs.lev[0].e;
      gs.op.f = gs.lev[0].f;
      if (PREC == 0) {
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
  const Level<T, F>* lev = gs.lev;
  const Level<T, F>& L0 = lev[0];
  const Level<T>& A = cg_operator<PREC>(gs);
  const RbIndex R(m);  // cell-array layout (colour by colour)

  // ---- layers and per-cell permeability (into r64, or x with prec 1, 2, as scratch) ----
  if (a.ksrc != KSRC_ARRAY) {
    if (g.local_leader()) sample_layers(a, sample, gs.eta, gs.kc);
    g.sync();
  }
  const int n_if = a.geometry == 1 ? 0 : a.n_layers - 1;
  // m and a.m are powers of two: scaling by the reciprocal is exact, so the
  // centre (j + 1/2) / m is the same double as the quotient
  const double inv_m = 1.0 / (double)m, inv_mf = 1.0 / (double)a.m;
  // horizontal interfaces: the layer of each row, once per row (the same
  // centre and comparisons as per cell), in the finest level's e as scratch
  int* row_t = reinterpret_cast<int*>(L0.e);
  const bool by_row = a.ksrc != KSRC_ARRAY && a.geometry != 1;
  if (by_row) {
    const bool own = coarse && !a.cgv_on_k;
    for (int j = g.rank(); j < m; j += g.size()) {
      const int jf = coarse ? 2 * j + oy : j;
      const double yc = own ? ((double)j + 0.5) * inv_m : ((double)jf + 0.5) * inv_mf;
      row_t[j] = layer_at(gs.eta, n_if, yc);
    }
    g.sync();
  }
  // the cell permeabilities: FP32 for the FP32 operators (prec 1, 2; in the CG
  // x vector as scratch), else FP64 (in r64)
  float* k32 = reinterpret_cast<float*>(xv);
  for (int c = g.rank(); c < n; c += g.size()) {
    int i, j;
    R.cell(c, i, j);
    double kk;
    if (a.ksrc == KSRC_ARRAY) {
      kk = a.k[sys * (int64_t)n + j * m + i];  // natural layout in the caller's array
    } else {
      // fine cell of the value, and the centre that decides the layer
      const int jf = coarse ? 2 * j + oy : j;
      const int iff = coarse ? 2 * i + ox : i;
      const bool own = coarse && !a.cgv_on_k;  // layer at the coarse centre
      int t;
      if (by_row) {
        t = row_t[j];
      } else {
        const double yc = own ? ((double)j + 0.5) * inv_m : ((double)jf + 0.5) * inv_mf;
        const double xc = own ? ((double)i + 0.5) * inv_m : ((double)iff + 0.5) * inv_mf;
        t = layer_at_point(a.geometry, gs.eta, n_if, xc, yc);
      }
      if (a.ksrc == KSRC_CONST) {
        kk = gs.kc[t];
      } else if (REFINE) {
        const float* gf = reinterpret_cast<const float*>(a.g);
        kk = (double)expf(gf[((sidx * a.n_layers + t) * (int64_t)a.m + jf) * a.m + iff]);
      } else {
        const double* gd = reinterpret_cast<const double*>(a.g);
        kk = exp(gd[((sidx * a.n_layers + t) * (int64_t)a.m + jf) * a.m + iff]);
      }
    }
    if (REFINE) k32[c] = (float)kk;
    else r64[c] = kk;
  }
  g.sync();
  // ---- faces (Eq. 3.3, harmonic averages; Dirichlet 2k; no-flow 0) ----
  {
    auto kc = [&](int c) -> TF { return REFINE ? (TF)k32[c] : (TF)r64[c]; };
    const int nfx = m * (m + 1);
    for (int t = g.rank(); t < 2 * nfx; t += g.size()) {
      if (t < nfx) {
        const int j = t / (m + 1), ip = t - j * (m + 1);
        TF v;
        if (ip == 0) v = TF(2) * kc(R.at(0, j));
        else if (ip == m) v = TF(2) * kc(R.at(m - 1, j));
        else {
          const TF ka = kc(R.at(ip - 1, j)), kb = kc(R.at(ip, j));
          v = TF(2) * ka * kb / (ka + kb);
        }
        A.tx[t] = (T)v;
        if (PREC == 2) L0.tx[t] = face_st<F>((T)v);
        if (PREC == 3) gs.op64.tx[t] = (double)v;
      } else {
        const int u = t - nfx;
        const int jp = u / m, i = u - jp * m;
        TF v = TF(0);
        if (jp > 0 && jp < m) {
          const TF ka = kc(R.at(i, jp - 1)), kb = kc(R.at(i, jp));
          v = TF(2) * ka * kb / (ka + kb);
        } else if (a.problem == 1) {  // Dirichlet p = 0 half a cell away
          v = TF(2) * kc(R.at(i, jp == 0 ? 0 : m - 1));
        }
        A.ty[u] = (T)v;
        if (PREC == 2) L0.ty[u] = face_st<F>((T)v);
        if (PREC == 3) gs.op64.ty[u] = (double)v;
      }
    }
    g.sync();
    if (PREC == 2) build_diag<false>(g, A);
    if (PREC == 3) build_diag<false>(g, gs.op64);
    build_diag<true>(g, L0);
  }
  for (int l = 1; l < nl; ++l) {
    build_coarse(g, lev[l - 1], lev[l]);
    build_diag<true>(g, lev[l]);
  }
  build_coarse_inverse(g, lev[nl - 1]);
  // ---- solve ----
  int status = 1, iters = 0;
  if constexpr (PREC == 3) {
    const Level<double>& A64 = gs.op64;
    double bb = 0.0;
    const double fmid = 1.0 / ((double)m * (double)m);  // Model Problem 1: f / m^2
    for (int c = g.rank(); c < n; c += g.size()) {
      int i, j;
      R.cell(c, i, j);
      const double bv = a.problem == 1 ? fmid : (i == 0 ? A64.tx[j * (m + 1)] : 0.0);
      r64[c] = bv;
      bb += bv * bv;
    }
    bb = g.sum(bb, red64, par);
    iters = pcg64_mg32(g, A64, lev, nl, a.mg_gamma, a.mg_nu, a.mg_nu_coarse, x64, r64, gs.p64, gs.q64, gs.z64,
                       a.tol * a.tol * bb, a.max_it, red64, par, status);
  } else if (PREC == 0) {
    // r = b, bb = b.b; stop at r.r <= tol^2 b.b
    T bb = T(0);
    const T fmid = (T)(1.0 / ((double)m * (double)m));  // Model Problem 1: f / m^2
    for (int c = g.rank(); c < n; c += g.size()) {
      int i, j;
      R.cell(c, i, j);
      const T bv = a.problem == 1 ? fmid : (i == 0 ? A.tx[j * (m + 1)] : T(0));
      L0.f[c] = bv;
      bb += bv * bv;
    }
    bb = g.sum(bb, red, par);
    iters = pcg(g, A, lev, nl, a.mg_gamma, a.mg_nu, a.mg_nu_coarse, xv, pv, qv, (T)(a.tol * a.tol) * bb, a.max_it,
                red, par,
                status);
  } else {
    // FP64 refinement: r64 = b - A64 x64 with A64 = the FP32 faces in FP64.
    double bb = 0.0;
    const double fmid = 1.0 / ((double)m * (double)m);  // Model Problem 1: f / m^2
    for (int c = g.rank(); c < n; c += g.size()) {
      int i, j;
      R.cell(c, i, j);
      const double bv = a.problem == 1 ? fmid : (i == 0 ? (double)A.tx[j * (m + 1)] : 0.0);
      x64[c] = 0.0;
      r64[c] = bv;
      bb += bv * bv;
    }
    bb = g.sum(bb, red64, par);
    double rr = bb;
    const double thr = a.tol * a.tol * bb;
    // FP32 on a streamed finest grid: the passes on 16-byte quads
    bool vq = false;
    if constexpr (std::is_same<T, float>::value && G::kQuads) vq = L0.quads != 0;
    // r64 = b - A64 x64 and its squared norm
    auto residual64 = [&]() -> double {
      double s2 = 0.0;
      if constexpr (std::is_same<T, float>::value && G::kQuads) {
        if (vq) return g.sum(ref_residual_quads(g, A, x64, r64, a.problem, fmid), red64, par);
      }
      for (int c = g.rank(); c < n; c += g.size()) {
        int i, j;
        R.cell(c, i, j);
        const int rf = j * (m + 1) + i;
        const double tw = (double)A.tx[rf], te = (double)A.tx[rf + 1];
        const double ts = (double)A.ty[j * m + i], tn = (double)A.ty[(j + 1) * m + i];
        const int ob = (((i + j) & 1) ^ 1) * R.half + j * R.hm;  // row j of the other colour
        double ax = ((tw + te) + (ts + tn)) * x64[c];
        if (i > 0) ax -= tw * x64[ob + ((i - 1) >> 1)];
        if (i < m - 1) ax -= te * x64[ob + ((i + 1) >> 1)];
        if (j > 0) ax -= ts * x64[ob - R.hm + (i >> 1)];
        if (j < m - 1) ax -= tn * x64[ob + R.hm + (i >> 1)];
        const double bv = a.problem == 1 ? fmid : (i == 0 ? tw : 0.0);
        const double rv = bv - ax;
        r64[c] = rv;
        s2 += rv * rv;
      }
      return g.sum(s2, red64, par);
    };
    int sweeps = 0;
    if (a.reliable) {
      // FP32 CG with reliable updates (Sleijpen and van der Vorst, 1996): the
      // FP32 recursion runs on the correction, in units of the last true
      // residual norm; once its residual has fallen by inner_tol (or every 16
      // iterations) the correction is added to the FP64 solution, the true
      // residual is recomputed in FP64 and replaces the FP32 one, and the
      // search direction carries on (the Krylov recursion is not restarted,
      // unlike the refinement loop below).  Same FP64 stopping test.
      status = 1;
      if (rr <= thr) status = 0;
      double scl = sqrt(rr);
      T rr32 = T(0);
      // the scaled residual, by multiplication with the reciprocal (FP64 division
      // is a long instruction sequence at GB300's FP64 rate)
      const double inv0 = status == 0 ? 0.0 : 1.0 / scl;
      if constexpr (std::is_same<T, float>::value && G::kQuads) {
        if (vq) rr32 = ref_rescale_quads(g, n, inv0, r64, L0.f, xv, nullptr, 1.f);
      }
      if (!vq)
        for (int c = g.rank(); c < n; c += g.size()) {
          const T v = (T)(r64[c] * inv0);
          L0.f[c] = v;
          xv[c] = T(0);
          rr32 += v * v;
        }
      rr32 = g.sum(rr32, red, par);
      g.sync();
      T rr_ref = rr32;
      const T d2 = (T)(a.inner_tol * a.inner_tol);
      const int nuc = a.mg_nu_coarse;
      T rz = T(0);
      if (status != 0) {
        precond(g, lev, nl, a.mg_gamma, a.mg_nu, nuc);
        for (int c = g.rank(); c < n; c += g.size()) {
          pv[c] = L0.e[c];
          rz += L0.f[c] * L0.e[c];
        }
        rz = g.sum(rz, red, par);
      }
      int since = 0;
      while (status != 0 && iters < a.max_it) {
        ++iters;
        ++since;
        T pq = T(0);
        if constexpr (std::is_same<T, float>::value && G::kQuads) {
          if (vq) pq = cg_matvec_quads(g, A, pv, qv);
        }
        if (!vq)
          for (int c = g.rank(); c < n; c += g.size()) {
            int i, j;
            R.cell(c, i, j);
            const T v = apply_at(A, pv, R, c, i, j);
            qv[c] = v;
            pq += pv[c] * v;
          }
        pq = g.sum(pq, red, par);
        if (!(pq > T(0)) || !isfinite(pq) || !isfinite(rz)) {
          status = 2;
          break;
        }
        const T alpha = rz / pq;
        rr32 = T(0);
        if constexpr (std::is_same<T, float>::value && G::kQuads) {
          if (vq) rr32 = cg_update_quads(g, n, alpha, xv, pv, L0.f, qv);
        }
        if (!vq)
          for (int c = g.rank(); c < n; c += g.size()) {
            xv[c] += alpha * pv[c];
            const T rv = L0.f[c] - alpha * qv[c];
            L0.f[c] = rv;
            rr32 += rv * rv;
          }
        rr32 = g.sum(rr32, red, par);
        if ((double)rr32 * scl * scl <= thr || rr32 <= d2 * rr_ref || since >= 16) {  // reliable update
          if constexpr (std::is_same<T, float>::value && G::kQuads) {
            if (vq) ref_update_quads(g, n, scl, x64, xv);
          }
          if (!vq)
            for (int c = g.rank(); c < n; c += g.size()) x64[c] += scl * (double)xv[c];
          g.sync();
          rr = residual64();
          ++sweeps;
          if (rr <= thr) {
            status = 0;
            break;
          }
          const double scl_new = sqrt(rr);
          const T ratio = (T)(scl / scl_new);
          const double inv = 1.0 / scl_new;
          rr32 = T(0);
          if constexpr (std::is_same<T, float>::value && G::kQuads) {
            if (vq) rr32 = ref_rescale_quads(g, n, inv, r64, L0.f, xv, pv, ratio);
          }
          if (!vq)
            for (int c = g.rank(); c < n; c += g.size()) {
              const T v = (T)(r64[c] * inv);
              L0.f[c] = v;
              xv[c] = T(0);
              pv[c] *= ratio;
              rr32 += v * v;
            }
          rr32 = g.sum(rr32, red, par);
          g.sync();
          rz *= ratio * ratio;
          scl = scl_new;
          rr_ref = rr32;
          since = 0;
        }
        precond(g, lev, nl, a.mg_gamma, a.mg_nu, nuc);
        T rzn = T(0);
        if constexpr (std::is_same<T, float>::value && G::kQuads) {
          if (vq) rzn = cg_dot_quads(g, n, L0.f, L0.e);
        }
        if (!vq)
          for (int c = g.rank(); c < n; c += g.size()) rzn += L0.f[c] * L0.e[c];
        rzn = g.sum(rzn, red, par);
        const T beta = rzn / rz;
        rz = rzn;
        if constexpr (std::is_same<T, float>::value && G::kQuads) {
          if (vq) cg_xpay_quads(g, n, beta, L0.e, pv);
        }
        if (!vq)
          for (int c = g.rank(); c < n; c += g.size()) pv[c] = L0.e[c] + beta * pv[c];
        g.sync();
      }
    }
    while (!a.reliable) {
      if (rr <= thr) {
        status = 0;
        break;
      }
      if (iters >= a.max_it || sweeps >= 40) {
        status = 1;
        break;
      }
      ++sweeps;
      const double scl = sqrt(rr);
      const double inv = 1.0 / scl;
      T r32 = T(0);
      if constexpr (std::is_same<T, float>::value && G::kQuads) {
        if (vq) r32 = ref_rescale_quads(g, n, inv, r64, L0.f, nullptr, nullptr, 1.f);
      }
      if (!vq)
        for (int c = g.rank(); c < n; c += g.size()) {
          const T v = (T)(r64[c] * inv);
          L0.f[c] = v;
          r32 += v * v;
        }
      r32 = g.sum(r32, red, par);
      int st_in = 1;
      const T thr_in = (T)(a.inner_tol * a.inner_tol) * r32;
      const int it =
          pcg(g, A, lev, nl, a.mg_gamma, a.mg_nu, a.mg_nu_coarse, xv, pv, qv, thr_in, a.max_it - iters, red, par,
              st_in);
      iters += it;
      // x64 += scl * d, then r64 = b - A64 x64 (FP64)
      if constexpr (std::is_same<T, float>::value && G::kQuads) {
        if (vq) ref_update_quads(g, n, scl, x64, xv);
      }
      if (!vq)
        for (int c = g.rank(); c < n; c += g.size()) x64[c] += scl * (double)xv[c];
      g.sync();
      rr = residual64();
      if (it == 0 && st_in != 0) {  // inner solver made no progress
        status = 2;
        break;
      }
    }
  }
  // ---- QoI and outputs ----
  double qsum = 0.0;
  if (a.problem == 1) {
    // M^(1): sum over cells of |cell & D*| / |D*| p (p piecewise constant)
    const double h = 1.0 / (double)m;
    const double inv_area = 1.0 / ((a.box[1] - a.box[0]) * (a.box[3] - a.box[2]));
    for (int c = g.rank(); c < n; c += g.size()) {
      int i, j;
      R.cell(c, i, j);
      const double ox = fmin((i + 1) * h, a.box[1]) - fmax(i * h, a.box[0]);
      const double oy = fmin((j + 1) * h, a.box[3]) - fmax(j * h, a.box[2]);
      if (ox > 0.0 && oy > 0.0) qsum += ox * oy * inv_area * x64[c];
    }
  } else {
    // M^(2): outflow through x1 = 1
    for (int j = g.rank(); j < m; j += g.size()) {
      const double te = PREC == 3 ? gs.op64.tx[j * (m + 1) + m] : (double)A.tx[j * (m + 1) + m];
      qsum += te * x64[R.at(m - 1, j)];
    }
  }
  qsum = g.sum(qsum, red64, par);
  if (g.rank() == 0) {
    a.q[sys] = status == 0 ? qsum : nan("");
    if (a.iters) a.iters[sys] = iters;
  }
  if (a.p_out && !coarse)
    for (int c = g.rank(); c < n; c += g.size()) {  // natural layout in the caller's array
      int i, j;
      R.cell(c, i, j);
      a.p_out[sidx * (int64_t)n + j * m + i] = x64[c];
    }
  g.sync();
}

}  // namespace mlmc

#include "tiny.cuh"


namespace mlmc {

// MODE 0: one block per system; 1: one warp per system (kWarpsPerBlock
// systems per block); 2: one thread-block cluster per system; 3: one warp
// per system with 16 x 16 systems on the register-resident path (prec 1;
// other sizes of the launch take the generic warp path).
template <int PREC, int MODE>
__global__ void __launch_bounds__(MODE == 1 || MODE == 3 ? 32 * kWarpsPerBlock : kMaxThreads,
                                  MODE == 1 ? 5 : MODE == 3 ? 4 : 2)
    solve_kernel(SolveArgs a) {
  using T = typename SolverTypes<PREC>::T;
  using F = typename SolverTypes<PREC>::F;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kGroups = MODE == 1 || MODE == 3 ? kWarpsPerBlock : 1;
  __shared__ GroupState<T, F> gstate[kGroups];
  __shared__ T red[MODE == 1 || MODE == 3 ? 1 : 132];
  __shared__ double red64[MODE == 1 || MODE == 3 ? 1 : 132];
  const int64_t n_all = a.n_samples * (int64_t)(1 + a.n_coarse);
  const int64_t sys0 = a.sys_begin, n_sys = a.sys_end > 0 ? a.sys_end : n_all;
  int par = 0, m_prev = -1;
  if (MODE == 2) {
    __shared__ double cl_part[2];
    cg::cluster_group cl = cg::this_cluster();
    const ClusterGroup g{cl.num_blocks(), cl.block_rank(), cl_part};
    const int64_t cid = blockIdx.x / g.nblk, ncl = gridDim.x / g.nblk;
    unsigned char* base = a.ws + (size_t)cid * a.ws_stride;
    unsigned char* stage = a.stage_bytes ? smem_raw : nullptr;
    for (int64_t sys = sys0 + cid; sys < n_sys; sys += ncl)
      solve_one<PREC>(g, a, sys, base, gstate[0], red, red64, par, m_prev, nullptr, stage);
    cl.sync();  // no block leaves while others may still read its shared memory
    return;
  }
  const int gid = MODE == 1 || MODE == 3 ? (int)(threadIdx.x >> 5) : 0;
  const size_t slot = (size_t)blockIdx.x * kGroups + gid;
  unsigned char* base = a.use_smem ? smem_raw + (size_t)gid * a.ws_stride : a.ws + slot * a.ws_stride;
  unsigned char* base64 = a.ws64_stride ? a.ws64 + slot * a.ws64_stride : nullptr;
  const int64_t stride = (int64_t)gridDim.x * kGroups;
  for (int64_t sys = sys0 + (int64_t)blockIdx.x * kGroups + gid; sys < n_sys; sys += stride) {
    if constexpr (MODE == 3 && PREC == 1) {
      const int msys = sys < a.n_samples ? a.m : a.m >> 1;
      if (msys == kTinyM) {
        solve_one_tiny(WarpGroup(), a, sys, base, gstate[gid], m_prev);
        continue;
      }
    }
    if (MODE == 1 || MODE == 3)
      solve_one<PREC>(WarpGroup(), a, sys, base, gstate[gid], red, red64, par, m_prev, base64, nullptr);
    else
      solve_one<PREC>(BlockGroup(), a, sys, base, gstate[gid], red, red64, par, m_prev, base64, nullptr);
  }
}

// The same solver over the items of a SolveList: one persistent launch of a
// launch shape across the levels of an estimate round.  The systems form one
// work queue; each group (warp, block or cluster) takes the next system from
// the counter *L.next (a fetch-and-add: no group waits on another), so a group
// that drew long solves takes fewer of them and the launch ends when the
// queue is empty.  The caller lays the items out largest systems first, so the
// last systems handed out are the short ones.  A group copies its current
// item's arguments into shared memory when the item changes.
template <int PREC, int MODE>
__global__ void __launch_bounds__(MODE == 1 || MODE == 3 ? 32 * kWarpsPerBlock : kMaxThreads,
                                  MODE == 1 ? 5 : MODE == 3 ? 4 : 2)
    solve_list_kernel(const __grid_constant__ SolveList L) {
  using T = typename SolverTypes<PREC>::T;
  using F = typename SolverTypes<PREC>::F;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kGroups = MODE == 1 || MODE == 3 ? kWarpsPerBlock : 1;
  __shared__ GroupState<T, F> gstate[kGroups];
  __shared__ T red[MODE == 1 || MODE == 3 ? 1 : 132];
  __shared__ double red64[MODE == 1 || MODE == 3 ? 1 : 132];
  __shared__ __align__(16) SolveArgs args[kGroups];
  __shared__ long long wq[2];  // block and cluster groups: the taken work index (two slots, alternating)
  const int64_t total = L.start[L.n];
  const SolveArgs& a0 = L.a[0];  // the launch's workspace layout
  int par = 0, m_prev = -1;
  const int gid = MODE == 1 || MODE == 3 ? (int)(threadIdx.x >> 5) : 0;
  int cur = -1;  // item whose arguments args[gid] hold
  // the item of work index w and its system; refreshes the group's copy
  auto take = [&](const auto& g, int64_t w, int64_t& sys) -> const SolveArgs& {
    int k = 0;
    while (k + 1 < L.n && w >= L.start[k + 1]) ++k;
    if (k != cur) {
      g.lsync();  // nobody still reads the previous copy
      const unsigned* src = reinterpret_cast<const unsigned*>(&L.a[k]);
      unsigned* dst = reinterpret_cast<unsigned*>(&args[gid]);
      for (int t = g.lrank(); t < (int)(sizeof(SolveArgs) / 4); t += g.lsize()) dst[t] = src[t];
      g.lsync();
      cur = k;
    }
    sys = args[gid].sys_begin + (w - L.start[k]);
    return args[gid];
  };
  if (MODE == 2) {
    __shared__ double cl_part[2];
    cg::cluster_group cl = cg::this_cluster();
    const ClusterGroup g{cl.num_blocks(), cl.block_rank(), cl_part};
    const int64_t cid = blockIdx.x / g.nblk;
    unsigned char* base = a0.ws + (size_t)cid * a0.ws_stride;
    unsigned char* stage = a0.stage_bytes ? smem_raw : nullptr;
    for (int it = 0;; ++it) {
      // block 0 of the cluster takes the index; the others read it from its
      // shared memory after the cluster barrier (the slot it overwrites two
      // turns later was read before the barrier of the turn in between)
      if (g.brank == 0 && threadIdx.x == 0) wq[it & 1] = (long long)atomicAdd(L.next, 1ull);
      cl.sync();
      const int64_t w = *cl.map_shared_rank(&wq[it & 1], 0);
      if (w >= total) break;
      int64_t sys;
      const SolveArgs& a = take(g, w, sys);
      solve_one<PREC>(g, a, sys, base, gstate[0], red, red64, par, m_prev, nullptr, stage);
    }
    cl.sync();  // no block leaves while others may still read its shared memory
    return;
  }
  const size_t slot = (size_t)blockIdx.x * kGroups + gid;
  unsigned char* base = a0.use_smem ? smem_raw + (size_t)gid * a0.ws_stride : a0.ws + slot * a0.ws_stride;
  unsigned char* base64 = a0.ws64_stride ? a0.ws64 + slot * a0.ws64_stride : nullptr;
  for (int it = 0;; ++it) {
    int64_t sys;
    if (MODE == 1 || MODE == 3) {
      long long w = 0;
      if ((threadIdx.x & 31) == 0) w = (long long)atomicAdd(L.next, 1ull);
      w = __shfl_sync(0xffffffffu, w, 0);
      if (w >= total) break;
      const SolveArgs& a = take(WarpGroup(), w, sys);
      if constexpr (MODE == 3 && PREC == 1) {
        const int msys = sys < a.n_samples ? a.m : a.m >> 1;
        if (msys == kTinyM) {
          solve_one_tiny(WarpGroup(), a, sys, base, gstate[gid], m_prev);
          continue;
        }
      }
      solve_one<PREC>(WarpGroup(), a, sys, base, gstate[gid], red, red64, par, m_prev, base64, nullptr);
    } else {
      if (threadIdx.x == 0) wq[it & 1] = (long long)atomicAdd(L.next, 1ull);
      __syncthreads();
      const int64_t w = wq[it & 1];
      if (w >= total) break;
      const SolveArgs& a = take(BlockGroup(), w, sys);
      solve_one<PREC>(BlockGroup(), a, sys, base, gstate[gid], red, red64, par, m_prev, base64, nullptr);
    }
  }
}

size_t solve_ws_bytes(int m, int prec) { return ws_layout(m, prec); }

static const size_t kSmemCap = 110 * 1024;

template <int PREC, int MODE>
static int plan_fill(int m, int threads, int cluster, SolvePlan* P) {
  if (MODE == 3 && !(PREC == 1 && m == kTinyM)) return -1;  // the register path: m = 16, prec 1
  // MODE 3 solves its 16 x 16 systems with the register path (shared memory
  // for the coarser levels only) and any 8 x 8 coarse systems generically
  size_t ws = MODE == 3 ? std::max(tiny_ws_bytes(), solve_ws_bytes(m / 2, PREC)) : solve_ws_bytes(m, PREC);
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  P->warp = MODE == 1 ? 1 : MODE == 3 ? 2 : 0;
  P->cluster = MODE == 2 ? cluster : 0;
  P->threads = MODE == 1 || MODE == 3 ? 32 * kWarpsPerBlock : threads;
  P->groups_per_block = MODE == 1 || MODE == 3 ? kWarpsPerBlock : 1;
  P->blocks_per_group = MODE == 2 ? cluster : 1;
  // prec 1, 2: the FP64 solution and residual of the refinement (touched once
  // per refinement sweep) stay in global memory when the rest of the
  // workspace fits on chip, so more systems fit per SM
  const int m64 = MODE == 3 ? m / 2 : m;  // the register path keeps them in registers
  const size_t v64 = (PREC == 1 || PREC == 2) ? 2 * align16((size_t)m64 * m64 * 8) : 0;
  if (MODE == 3) ws += v64;  // chip = ws - v64 below
  const size_t chip = ((ws - v64) + 255) & ~(size_t)255;
  P->use_smem = MODE != 2 && chip * P->groups_per_block <= kSmemCap;
  if (MODE == 3 && !P->use_smem) return -1;
  P->ws_stride = P->use_smem ? chip : (ws + 255) & ~(size_t)255;
  P->ws64_stride = P->use_smem && v64 ? (v64 + 255) & ~(size_t)255 : 0;
  P->smem_bytes = P->use_smem ? P->ws_stride * P->groups_per_block : 0;
  // cluster plans (streamed workspace): shared memory stages the half sweeps
  // of the large levels.  Measured on GB300 the staging pays there (m = 512 /
  // 1024 / 2048: 8 / 11 / 18 % less time per sample) and costs 5-7 % in the
  // one-block-per-system plans at m = 128, 256, which stay on direct loads.
  P->stage_bytes = 0;
  if (MODE == 2 && !P->use_smem && PREC != 2) {
    using TS = typename SolverTypes<PREC>::T;
    P->stage_bytes = stage_bytes_for<TS>(m, P->threads);
    P->smem_bytes = P->stage_bytes;
  }
  P->cap_blocks_per_sm = 0;
  P->gamma = 1;
  P->nu = 1;
  P->nu_coarse = 0;
  P->inner_tol = 1e-5;
  P->reliable = 0;
  cudaFuncSetAttribute(solve_kernel<PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_kernel<PREC, MODE>, P->threads, P->smem_bytes) !=
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
    cfg.dynamicSmemBytes = P->smem_bytes;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, solve_kernel<PREC, MODE>, &cfg) != cudaSuccess || ncl < 1) return -1;
    P->max_groups = ncl;
  }
  return 0;
}

// mode: 0 block, 1 warp, 2 cluster of `cluster` blocks
template <int PREC>
static int plan_fill_mode(int m, int mode, int threads, int cluster, SolvePlan* P) {
  if (mode == 1) return plan_fill<PREC, 1>(m, threads, cluster, P);
  if (mode == 2) return plan_fill<PREC, 2>(m, threads, cluster, P);
  if (mode == 3) {
    if constexpr (PREC == 1) return plan_fill<1, 3>(m, threads, cluster, P);
    return -1;
  }
  return plan_fill<PREC, 0>(m, threads, cluster, P);
}

static int plan_fill(int m, int prec, int mode, int threads, int cluster, SolvePlan* P) {
  if (prec == 3) return plan_fill_mode<3>(m, mode, threads, cluster, P);
  if (prec == 2) return plan_fill_mode<2>(m, mode, threads, cluster, P);
  if (prec == 1) return plan_fill_mode<1>(m, mode, threads, cluster, P);
  return plan_fill_mode<0>(m, mode, threads, cluster, P);
}

// Default plan (measured on GB300 with the autotuner): a warp per system up
// to m = 16, a block up to m = 256, a cluster of 4 blocks at m = 512 and of 8
// above (the system's working set then sits in L2 instead of streaming).
int solve_plan(int m, int prec, SolvePlan* P) {
  if (m >= 512) return plan_fill(m, prec, 2, kMaxThreads, m >= 1024 ? 8 : 4, P);
  if (m == kTinyM && prec == 1 && plan_fill(m, prec, 3, 0, 0, P) == 0) return 0;
  return plan_fill(m, prec, solve_warp_mode(m) ? 1 : 0, solve_threads(m), 0, P);
}

int solve_plan_mode(int m, int prec, int mode, int threads, int cluster, SolvePlan* P) {
  return plan_fill(m, prec, mode, threads, cluster, P);
}

int solve_plan_candidates(int m, int prec, SolvePlan* out, int max_out) {
  int k = 0;
  auto add = [&](const SolvePlan& P) {
    if (k < max_out) out[k++] = P;
  };
  SolvePlan d;
  if (solve_plan(m, prec, &d)) return 0;
  add(d);
  if (d.cluster) {  // also the one-block plan
    SolvePlan b;
    if (!plan_fill(m, prec, 0, kMaxThreads, 0, &b)) add(b);
  }
  if (m <= 64 && d.warp != 1) {  // the generic warp plan
    SolvePlan w;
    if (!plan_fill(m, prec, 1, 0, 0, &w)) add(w);
  }
  for (int t : {64, 128, 256, 512}) {
    if (!d.warp && !d.cluster && t == d.threads) continue;
    if (d.cluster && t == kMaxThreads) continue;
    if (t > 2 * m * m) continue;  // more threads than cells
    SolvePlan b;
    if (!plan_fill(m, prec, 0, t, 0, &b)) add(b);
  }
  // global-workspace plans also with one system per SM (smaller working set)
  const int k0 = k;
  for (int i = 0; i < k0; ++i)
    if (!out[i].use_smem && out[i].blocks_per_sm > 1) {
      SolvePlan c = out[i];
      c.cap_blocks_per_sm = 1;
      add(c);
    }
  // large grids: one cluster of 2, 4 or 8 blocks per system
  if (m >= 128)
    for (int cl : {2, 4, 8}) {
      if (cl == d.cluster) continue;
      SolvePlan c;
      if (!plan_fill(m, prec, 2, kMaxThreads, cl, &c)) add(c);
    }
  return k;
}

// The plan's launch settings written into an item's arguments.
static void apply_plan(SolveArgs& b, const SolvePlan& P) {
  b.use_smem = P.use_smem;
  b.ws_stride = P.ws_stride;
  b.ws64_stride = P.ws64_stride;
  b.stage_bytes = P.stage_bytes;
  b.mg_gamma = P.gamma;
  b.mg_nu = P.nu;
  b.mg_nu_coarse = P.nu_coarse;
  b.inner_tol = P.inner_tol;
  b.reliable = P.reliable;
}

// Launch configuration of a plan.
struct LaunchCfg {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  int mode;
  LaunchCfg(const SolvePlan& P, int n_blocks, cudaStream_t st) {
    cfg = {};
    cfg.gridDim = dim3(n_blocks);  // cluster plans: a multiple of the cluster size
    cfg.blockDim = dim3(P.threads);
    cfg.dynamicSmemBytes = P.smem_bytes;
    cfg.stream = st;
    if (P.cluster) {
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = P.cluster;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
    }
    mode = P.cluster ? 2 : P.warp == 2 ? 3 : P.warp ? 1 : 0;
  }
};

void solve_apply_plan(SolveArgs& a, const SolvePlan& P) { apply_plan(a, P); }

int solve_launch(const SolveArgs& a, int prec, const SolvePlan& P, int n_blocks, cudaStream_t st) {
  SolveArgs b = a;
  apply_plan(b, P);
  // every plan goes through cudaLaunchKernelEx, whose return value is this
  // launch's own status (an error left pending by earlier work of the caller
  // is neither reported nor cleared here)
  LaunchCfg C(P, n_blocks, st);
  cudaLaunchConfig_t* cfg = &C.cfg;
  cudaError_t e = cudaErrorInvalidValue;
  if (C.mode == 3) {
    if (prec == 1) e = cudaLaunchKernelEx(cfg, solve_kernel<1, 3>, b);
    last_launch_error() = e;
    return e == cudaSuccess ? 0 : -1;
  }
  switch (prec * 3 + C.mode) {
    case 0: e = cudaLaunchKernelEx(cfg, solve_kernel<0, 0>, b); break;
    case 1: e = cudaLaunchKernelEx(cfg, solve_kernel<0, 1>, b); break;
    case 2: e = cudaLaunchKernelEx(cfg, solve_kernel<0, 2>, b); break;
    case 3: e = cudaLaunchKernelEx(cfg, solve_kernel<1, 0>, b); break;
    case 4: e = cudaLaunchKernelEx(cfg, solve_kernel<1, 1>, b); break;
    case 5: e = cudaLaunchKernelEx(cfg, solve_kernel<1, 2>, b); break;
    case 6: e = cudaLaunchKernelEx(cfg, solve_kernel<2, 0>, b); break;
    case 7: e = cudaLaunchKernelEx(cfg, solve_kernel<2, 1>, b); break;
    case 8: e = cudaLaunchKernelEx(cfg, solve_kernel<2, 2>, b); break;
    case 9: e = cudaLaunchKernelEx(cfg, solve_kernel<3, 0>, b); break;
    case 10: e = cudaLaunchKernelEx(cfg, solve_kernel<3, 1>, b); break;
    case 11: e = cudaLaunchKernelEx(cfg, solve_kernel<3, 2>, b); break;
    default: break;
  }
  last_launch_error() = e;
  return e == cudaSuccess ? 0 : -1;
}

// Let the list kernels take the plans' dynamic shared memory (outside any
// stream capture; once per process and device is enough, repeating is harmless).
int solve_list_prepare() {
  const int cap = (int)kSmemCap;
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    const cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (r != cudaSuccess) e = r;
  };
  set((const void*)solve_list_kernel<0, 0>);
  set((const void*)solve_list_kernel<0, 1>);
  set((const void*)solve_list_kernel<0, 2>);
  set((const void*)solve_list_kernel<1, 0>);
  set((const void*)solve_list_kernel<1, 1>);
  set((const void*)solve_list_kernel<1, 2>);
  set((const void*)solve_list_kernel<1, 3>);
  last_launch_error() = e;
  return e == cudaSuccess ? 0 : -1;
}

int solve_launch_list(const SolveList& L, int prec, const SolvePlan& P, int n_blocks, cudaStream_t st) {
  LaunchCfg C(P, n_blocks, st);
  cudaLaunchConfig_t* cfg = &C.cfg;
  cudaError_t e = cudaErrorInvalidValue;
  if (prec == 1) {
    switch (C.mode) {
      case 0: e = cudaLaunchKernelEx(cfg, solve_list_kernel<1, 0>, L); break;
      case 1: e = cudaLaunchKernelEx(cfg, solve_list_kernel<1, 1>, L); break;
      case 2: e = cudaLaunchKernelEx(cfg, solve_list_kernel<1, 2>, L); break;
      case 3: e = cudaLaunchKernelEx(cfg, solve_list_kernel<1, 3>, L); break;
      default: break;
    }
  } else if (prec == 0) {
    switch (C.mode) {
      case 0: e = cudaLaunchKernelEx(cfg, solve_list_kernel<0, 0>, L); break;
      case 1: e = cudaLaunchKernelEx(cfg, solve_list_kernel<0, 1>, L); break;
      case 2: e = cudaLaunchKernelEx(cfg, solve_list_kernel<0, 2>, L); break;
      default: break;
    }
  }
  last_launch_error() = e;
  return e == cudaSuccess ? 0 : -1;
}

// Blocks to launch for n_sys systems with plan P (at most max_groups_cap
// groups resident; 0 = no cap), and the groups that launch serves.
int64_t solve_groups(const SolvePlan& P, int64_t n_sys, int nsm, int64_t max_groups_cap, int64_t* n_blocks) {
  int64_t g = P.max_groups;
  if (P.cap_blocks_per_sm > 0) g = std::min<int64_t>(g, (int64_t)nsm * P.cap_blocks_per_sm * P.groups_per_block);
  if (max_groups_cap > 0) g = std::min<int64_t>(g, max_groups_cap);
  g = std::max<int64_t>(1, std::min<int64_t>(g, n_sys));
  // a capped launch that does not hold every system keeps whole blocks of
  // groups, so no group slot lies beyond the workspace of g groups (slots
  // past n_sys never run)
  if (g < n_sys && g > P.groups_per_block) g -= g % P.groups_per_block;
  *n_blocks = P.cluster ? g * P.cluster : (g + P.groups_per_block - 1) / P.groups_per_block;
  return g;
}

}  // namespace mlmc

namespace mlmc {

// Sorted interfaces of each sample (stage output for parity checks).
__global__ void interfaces_kernel(SolveArgs a, int64_t n, double* eta) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  double e[MAX_LAYERS_DEV], kc[MAX_LAYERS_DEV];
  SolveArgs b = a;
  b.ksrc = KSRC_FIELDS;  // interfaces only
  sample_layers(b, (uint64_t)(a.first + s), e, kc);
  const int ne = a.geometry == 1 ? 4 : a.n_layers - 1;
  for (int t = 0; t < ne; ++t) eta[s * ne + t] = e[t];
}

int interfaces_launch(const SolveArgs& a, int64_t n, double* eta, cudaStream_t st) {
  if (n <= 0 || (a.geometry != 1 && a.n_layers < 2)) return 0;
  interfaces_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(a, n, eta);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Ex. 1 fields: g_t = mu_t + sigma_t Z_t on every cell (stage output).
__global__ void const_fields_kernel(SolveArgs a, int64_t n, int64_t cells, double* g) {
  const int64_t s = blockIdx.x;
  if (s >= n) return;
  __shared__ double e[MAX_LAYERS_DEV], kc[MAX_LAYERS_DEV], gz[MAX_LAYERS_DEV];
  if (threadIdx.x == 0) {
    const uint64_t sample = (uint64_t)(a.first + s);
    SolveArgs b = a;
    b.ksrc = KSRC_FIELDS;
    sample_layers(b, sample, e, kc);
    for (int t = 0; t < a.n_layers; t += 4) {
      const Words4 w = philox4x64_10((uint64_t)(t >> 2), sample, (uint64_t)a.level, kStreamLayerZ,
                                     a.seed);
      double z[4];
      box_muller(uniform52(w.w0), uniform52(w.w1), z[0], z[1]);
      box_muller(uniform52(w.w2), uniform52(w.w3), z[2], z[3]);
      for (int u = 0; u < 4 && t + u < a.n_layers; ++u) gz[t + u] = a.mu[t + u] + a.sigma[t + u] * z[u];
    }
  }
  __syncthreads();
  const int64_t mm = cells;  // cells per layer: m^2 or m^3
  for (int64_t c = threadIdx.x; c < mm * a.n_layers; c += blockDim.x)
    g[s * mm * a.n_layers + c] = gz[c / mm];
}

int const_fields_launch(const SolveArgs& a, int64_t n, int64_t cells, double* g, cudaStream_t st) {
  if (n <= 0) return 0;
  const_fields_kernel<<<(unsigned)n, 256, 0, st>>>(a, n, cells, g);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace mlmc

// ---------------------------------------------------------------------------
// Solve entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc: a plug-in living inside a host
// application that has already reserved (nearly) all device memory for its
// own pool, or a latency-critical loop that cannot afford the device-wide
// synchronisation and unbounded latency of cudaMalloc / cudaFree.  For them,
// mlmc_solve_k_static() runs the same solver as mlmc_solve_k() but takes its
// per-block workspace from the fixed array below instead of a context.
// ---------------------------------------------------------------------------
namespace mlmc {

// Scratch of the static entry point: 32 MiB, in the module's global memory.
// Every GPU that loads this library holds it until the process exits.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};  // device address of g_static_scratch, per device
}  // namespace

}  // namespace mlmc

extern "C" int mlmc_solve_k_static(int device, int32_t m, int64_t n, const double* k, double* p,
                                   double* q, int32_t* iters, double tol, int32_t max_it,
                                   int32_t prec, void* cuda_stream) {
  using namespace mlmc;
  if (device < 0 || device >= kMaxDevices) return set_error(MLMC_ERR_ARG, "mlmc_solve_k_static: device index out of range");
  if (!k || !q || n < 0) return set_error(MLMC_ERR_ARG, "mlmc_solve_k_static: k and q are required, n >= 0");
  if (m < 1 || m > 4096 || (m & (m - 1))) return set_error(MLMC_ERR_ARG, "mlmc_solve_k_static: m must be a power of two, 1..4096");
  if (!(tol > 0) || max_it < 1 || prec < 0 || prec > 3)
    return set_error(MLMC_ERR_ARG, "mlmc_solve_k_static: tol > 0, max_it >= 1, prec 0..3");
  if (n == 0) return MLMC_OK;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return set_error(MLMC_ERR_NODEV, "mlmc_solve_k_static: no usable CUDA device");
  if (cudaSetDevice(device) != cudaSuccess) return set_error(MLMC_ERR_NODEV, "mlmc_solve_k_static: cannot select the device");
  int rc = MLMC_OK;
  do {
    // set-up, once per device, with that device current: the host-side name
    // g_static_scratch is only a stand-in; the kernel needs the device address
    void* base = nullptr;
    {
      std::lock_guard<std::mutex> lock(g_static_mu);
      if (!g_static_ptr[device]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) {
          rc = set_error(MLMC_ERR_CUDA, (std::string("mlmc_solve_k_static: cudaGetSymbolAddress: ") +
                                         cudaGetErrorString(e)).c_str());
          break;
        }
        g_static_ptr[device] = ptr;
      }
      base = g_static_ptr[device];
    }
    SolvePlan P;
    int nsm = 0;
    if (solve_plan(m, prec, &P) ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
      rc = set_error(MLMC_ERR_CUDA, "mlmc_solve_k_static: launch plan (occupancy query) failed");
      break;
    }
    SolveArgs a;
    memset(&a, 0, sizeof(a));
    a.n_samples = n;
    a.n_coarse = 0;
    a.m = m;
    a.ksrc = KSRC_ARRAY;
    a.n_layers = 1;
    a.k = k;
    a.tol = tol;
    a.max_it = max_it;
    a.inner_tol = 1e-5;
    a.q = q;
    a.iters = iters;
    a.p_out = p;
    int64_t cap = 0;
    if (!P.use_smem) {
      if (P.ws_stride > kStaticScratchBytes) {  // m above the static maximum (512)
        rc = set_error(MLMC_ERR_TOOBIG, "mlmc_solve_k_static: m above the maximum of 512 for the 32 MiB scratch array");
        break;
      }
      cap = (int64_t)(kStaticScratchBytes / P.ws_stride);
      a.ws = reinterpret_cast<unsigned char*>(base);
    } else if (P.ws64_stride) {  // the refinement's FP64 vectors
      cap = (int64_t)(kStaticScratchBytes / P.ws64_stride);
      a.ws64 = reinterpret_cast<unsigned char*>(base);
    }
    int64_t nb = 0;
    solve_groups(P, n, nsm, cap, &nb);
    if (solve_launch(a, prec, P, (int)nb, (cudaStream_t)cuda_stream))
      rc = set_error(MLMC_ERR_CUDA, (std::string("mlmc_solve_k_static: solve kernel launch: ") +
                                     cudaGetErrorString(last_launch_error())).c_str());
  } while (0);
  cudaSetDevice(prev);
  return rc;
}

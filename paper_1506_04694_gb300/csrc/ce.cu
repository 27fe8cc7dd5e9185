// Circulant-embedding sampler of the per-layer Gaussian fields (Sec. 2 Ex. 2,
// Eq. 2.3; circulant embedding as cited in Sec. 3.4), with a hand-written
// batched radix-2 FFT.
//
// A level with m x m cells embeds the cell-centre grid in an M x M torus,
// M = p m.  With s_q = sqrt(Lambda_q)/M (Lambda = unnormalised forward 2-D DFT
// of the torus covariance) and complex normals xi_q = z_re + i z_im,
//   y[b][a] = sum_{q2,q1} s[q2][q1] xi[q2][q1] exp(-2 pi i (a q1 + b q2)/M)
// gives two independent fields on the m x m grid: layer 2f <- Re y, layer
// 2f+1 <- Im y, for field pair f.  Only a < m and b < m are needed, so:
//   pass 1 (rows):    W[q2][a] = sum_q1 s xi exp(-2 pi i a q1/M),  a < m,
//                     normals generated on chip from Philox, never stored;
//   pass 2 (columns): y[b][a] = sum_q2 W[q2][a] exp(-2 pi i b q2/M), b < m,
//                     written as g_t = mu_t + Re/Im y.
// Each FFT of length M runs in shared memory: bit-reversed load, then log2 M
// radix-2 decimation-in-time stages.  M = 3 N (N a power of two, the cut-off
// embedding) splits the input by q mod 3 into three length-N sequences, each
// loaded bit-reversed and transformed as above, and one radix-3 stage
// combines them: X[k + jN] = F0[k] + W^(k+jN) F1[k] + W^(2(k+jN)) F2[k],
// W = exp(-2 pi i/M), j = 0, 1, 2 (only j = 0 when the outputs kept are
// fewer than N).
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace mlmc {

template <typename R>
struct Cplx {
  R x, y;
};

// Kernel launches queued by the samplers since the last ce_launches_take()
// (the host thread's own count, for the profiling counters).
static thread_local int g_ce_launches = 0;
int ce_launches_take() {
  const int n = g_ce_launches;
  g_ce_launches = 0;
  return n;
}

__device__ __forceinline__ unsigned brev_n(unsigned v, int logn) {
  return logn ? (__brev(v) >> (32 - logn)) : 0u;
}

// In-place DIT FFTs of `nrows` contiguous rows of length M (rows already in
// bit-reversed order) in shared memory; tw[k] = exp(-2 pi i k/M), k < M.
// Stages 0 and 1 run as one twiddle-free radix-4 pass; further pairs of full
// stages as radix-4 passes (the two radix-2 stages of half-spans h and 2h
// fused: three twiddles W^2p, W^p, W^3p of the 4h-point span, then a
// twiddle-free 4-point butterfly; 28 instead of 32 real operations per four
// points and one shared-memory pass instead of two).  Only the outputs
// k < nkeep of each row are needed (nkeep a power of two, 4 <= nkeep <= M):
// stages whose half-span hs is >= nkeep compute, in each group, the nkeep
// upper outputs u + w v only.
// tws: the twiddle table holds exp(-2 pi i k/(tws M)), k < tws M (tws = 3: the
// length-N sub-transforms of an M = 3N transform read every third entry).
template <typename R>
__device__ void block_fft_rows(Cplx<R>* s, int nrows, int M, int logM, const Cplx<R>* __restrict__ tw,
                               int nkeep, int tws = 1) {
  const int half = M >> 1;
  const int nb = nrows * half;
  // stages 0 and 1 together: their twiddles are 1 and -i (M >= 4)
  const int nq = nrows * (M >> 2);
  for (int t = threadIdx.x; t < nq; t += blockDim.x) {
    Cplx<R>* x = s + 4 * t;  // rows are contiguous and M is a multiple of 4
    const Cplx<R> x0 = x[0], x1 = x[1], x2 = x[2], x3 = x[3];
    const Cplx<R> a0{x0.x + x1.x, x0.y + x1.y}, a1{x0.x - x1.x, x0.y - x1.y};
    const Cplx<R> a2{x2.x + x3.x, x2.y + x3.y}, a3{x2.x - x3.x, x2.y - x3.y};
    x[0] = Cplx<R>{a0.x + a2.x, a0.y + a2.y};
    x[2] = Cplx<R>{a0.x - a2.x, a0.y - a2.y};
    x[1] = Cplx<R>{a1.x + a3.y, a1.y - a3.x};
    x[3] = Cplx<R>{a1.x - a3.y, a1.y + a3.x};
  }
  __syncthreads();
  int st = 2;
  for (; st + 1 < logM && (2 << st) < nkeep; st += 2) {  // radix-4: stages st, st + 1 (both full)
    const int h = 1 << st;
    const int ts4 = (M >> (st + 2)) * tws;  // twiddle index step M / (4 h)
    for (int t = threadIdx.x; t < nq; t += blockDim.x) {
      const int row = t / (M >> 2);
      const int b = t - row * (M >> 2);
      const int p = b & (h - 1);
      Cplx<R>* x = s + row * M + ((b >> st) << (st + 2)) + p;
      const Cplx<R> w1 = tw[2 * p * ts4], w2 = tw[p * ts4], w3 = tw[3 * p * ts4];
      const Cplx<R> a = x[0], v1 = x[h], v2 = x[2 * h], v3 = x[3 * h];
      const Cplx<R> b1{w1.x * v1.x - w1.y * v1.y, w1.x * v1.y + w1.y * v1.x};
      const Cplx<R> c1{w2.x * v2.x - w2.y * v2.y, w2.x * v2.y + w2.y * v2.x};
      const Cplx<R> d1{w3.x * v3.x - w3.y * v3.y, w3.x * v3.y + w3.y * v3.x};
      const Cplx<R> t0{a.x + b1.x, a.y + b1.y}, t1{a.x - b1.x, a.y - b1.y};
      const Cplx<R> t2{c1.x + d1.x, c1.y + d1.y}, t3{c1.x - d1.x, c1.y - d1.y};
      x[0] = Cplx<R>{t0.x + t2.x, t0.y + t2.y};
      x[2 * h] = Cplx<R>{t0.x - t2.x, t0.y - t2.y};
      x[h] = Cplx<R>{t1.x + t3.y, t1.y - t3.x};      // t1 - i t3
      x[3 * h] = Cplx<R>{t1.x - t3.y, t1.y + t3.x};  // t1 + i t3
    }
    __syncthreads();
  }
  for (; st < logM; ++st) {
    const int hs = 1 << st;
    const int tstride = (half >> st) * tws;  // twiddle index step M / (2 hs)
    if (hs >= nkeep) {  // pruned stage: upper outputs of the first nkeep positions
      const int ngrp = M >> (st + 1);
      const int np = nrows * ngrp * nkeep;
      for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int pos = t & (nkeep - 1);
        const int rg = t / nkeep;
        const int row = rg / ngrp, grp = rg - row * ngrp;
        Cplx<R>* base = s + row * M;
        const int i0 = (grp << (st + 1)) + pos;
        const Cplx<R> w = tw[pos * tstride];
        const Cplx<R> u = base[i0];
        const Cplx<R> v = base[i0 + hs];
        // u + w v as two fused multiply-add chains per component
        base[i0] = Cplx<R>{fma(w.x, v.x, fma(-w.y, v.y, u.x)), fma(w.x, v.y, fma(w.y, v.x, u.y))};
      }
      __syncthreads();
      continue;
    }
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
      const int row = t / half;
      const int b = t - row * half;
      const int grp = b >> st;
      const int pos = b & (hs - 1);
      Cplx<R>* base = s + row * M;
      const int i0 = (grp << (st + 1)) + pos;
      const int i1 = i0 + hs;
      const Cplx<R> w = tw[pos * tstride];
      const Cplx<R> u = base[i0];
      const Cplx<R> v = base[i1];
      const R tx = w.x * v.x - w.y * v.y;
      const R ty = w.x * v.y + w.y * v.x;
      base[i0] = Cplx<R>{u.x + tx, u.y + ty};
      base[i1] = Cplx<R>{u.x - tx, u.y - ty};
    }
    __syncthreads();
  }
}

// Position in shared memory of input q of a row of length M: bit reversal
// for a power of two (r3 = 0, logn = log2 M); for M = 3N (r3 = 1, logn =
// log2 N) the sub-sequence q mod 3 at offset (q mod 3) N, bit-reversed in q/3.
__device__ __forceinline__ int fft_pos(int q, int logn, int r3) {
  if (!r3) return (int)brev_n((unsigned)q, logn);
  const int d = q / 3, r = q - 3 * d;
  return (r << logn) + (int)brev_n((unsigned)d, logn);
}

// FFTs of `nrows` rows of length M = 3N in shared memory, inputs at fft_pos:
// the three length-N sub-transforms of each row (all N outputs), then the
// radix-3 stage.  nkeep <= N: outputs k < nkeep only, written in place of F0;
// nkeep == M: all outputs, X[k + jN] in place of F_j[k].  tw: M entries.
template <typename R>
__device__ void block_fft_rows3(Cplx<R>* s, int nrows, int N, int logN, const Cplx<R>* __restrict__ tw, int nkeep) {
  const int M = 3 * N;
  block_fft_rows(s, 3 * nrows, N, logN, tw, N, 3);
  const R c3 = R(0.8660254037844386467637);  // sin(2 pi / 3)
  const bool full = nkeep > N;
  const int nk = full ? N : nkeep;
  for (int t = threadIdx.x; t < nrows * nk; t += blockDim.x) {
    const int row = t / nk, k = t - row * nk;
    Cplx<R>* x = s + row * M + k;
    const Cplx<R> a = x[0], f1 = x[N], f2 = x[2 * N];
    const Cplx<R> w1 = tw[k], w2 = tw[2 * k];
    const Cplx<R> b{w1.x * f1.x - w1.y * f1.y, w1.x * f1.y + w1.y * f1.x};
    const Cplx<R> c{w2.x * f2.x - w2.y * f2.y, w2.x * f2.y + w2.y * f2.x};
    const Cplx<R> sm{b.x + c.x, b.y + c.y};
    x[0] = Cplx<R>{a.x + sm.x, a.y + sm.y};
    if (full) {
      // W^N = exp(-2 pi i/3): X[k+N] = a - sm/2 - i c3 (b - c), X[k+2N] = a - sm/2 + i c3 (b - c)
      const Cplx<R> h{a.x - R(0.5) * sm.x, a.y - R(0.5) * sm.y};
      const Cplx<R> d{c3 * (b.x - c.x), c3 * (b.y - c.y)};
      x[N] = Cplx<R>{h.x + d.y, h.y - d.x};
      x[2 * N] = Cplx<R>{h.x - d.y, h.y + d.x};
    }
  }
  __syncthreads();
}

// Row FFTs of either length kind (r3 = 0: M = 2^logn; r3 = 1: M = 3 2^logn).
template <typename R>
__device__ __forceinline__ void fft_rows_any(Cplx<R>* s, int nrows, int M, int logn, int r3,
                                             const Cplx<R>* __restrict__ tw, int nkeep) {
  if (r3)
    block_fft_rows3(s, nrows, M / 3, logn, tw, nkeep);
  else
    block_fft_rows(s, nrows, M, logn, tw, nkeep);
}

// ------------------------------------------------------------ set-up -------
template <typename R>
__global__ void twiddle_kernel(Cplx<R>* tw, int M) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < M) {
    double s, c;
    sincospi(-2.0 * (double)k / (double)M, &s, &c);
    tw[k] = Cplx<R>{(R)c, (R)s};
  }
}

// Torus covariance c[b][a] = sigma2 exp(-||(d_a h, d_b h)||_r / lam),
// d_a = min(a, M - a), h = 1/m (Eq. 2.3 at cell-centre offsets).
// cutoff (2-norm): the cut-off embedding's radial function instead: Eq. 2.3
// up to R0 = sqrt(2)(m - 1)/m (the largest centre distance), the C^1 cubic
// from (R0, value and slope of Eq. 2.3) to (R1 = M/(2m), 0 and slope 0),
// zero beyond R1.
__global__ void covariance_kernel(Cplx<double>* c, int m, int M, double sigma2, double lam,
                                  int norm_r, int cutoff) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)M * M) return;
  const int b = (int)(id / M), a = (int)(id - (int64_t)b * M);
  const double dx = (double)min(a, M - a) / (double)m;
  const double dy = (double)min(b, M - b) / (double)m;
  const double dist = norm_r == 1 ? fabs(dx) + fabs(dy) : sqrt(dx * dx + dy * dy);
  double v = sigma2 * exp(-dist / lam);
  if (cutoff) {
    const double R0 = sqrt(2.0) * (double)(m - 1) / (double)m, R1 = (double)M / (2.0 * (double)m);
    if (dist >= R1) {
      v = 0.0;
    } else if (dist > R0) {
      const double w = R1 - R0, t = (dist - R0) / w;
      const double c0 = sigma2 * exp(-R0 / lam), d0 = -c0 / lam * w;
      v = c0 * (2.0 * t * t * t - 3.0 * t * t + 1.0) + d0 * (t * t * t - 2.0 * t * t + t);
    }
  }
  c[id] = Cplx<double>{v, 0.0};
}

// Full in-place FFT of each row of a rows x M array (global), one row per block.
__global__ void fft_rows_full_kernel(Cplx<double>* data, int M, int logn, int r3, const Cplx<double>* tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<double>* s = reinterpret_cast<Cplx<double>*>(smem_raw);
  Cplx<double>* row = data + (int64_t)blockIdx.x * M;
  for (int t = threadIdx.x; t < M; t += blockDim.x) s[fft_pos(t, logn, r3)] = row[t];
  __syncthreads();
  fft_rows_any(s, 1, M, logn, r3, tw, M);
  for (int t = threadIdx.x; t < M; t += blockDim.x) row[t] = s[t];
}

__global__ void transpose_kernel(const Cplx<double>* in, Cplx<double>* out, int M) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)M * M) return;
  const int r = (int)(id / M), c = (int)(id - (int64_t)r * M);
  out[(int64_t)c * M + r] = in[id];
}

// Min and max of Re(data) over n entries, one block, fixed order.
__global__ void minmax_kernel(const Cplx<double>* data, int64_t n, double* out2) {
  __shared__ double smin[1024], smax[1024];
  double lo = 1e300, hi = -1e300;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    lo = fmin(lo, data[i].x);
    hi = fmax(hi, data[i].x);
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out2[0] = smin[0];
    out2[1] = smax[0];
  }
}

// s = sqrt(max(Lambda, 0)) / M in FP64 and FP32.
__global__ void scale_kernel(const Cplx<double>* lam, double* s64, float* s32, int M) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)M * M) return;
  const double v = sqrt(fmax(lam[id].x, 0.0)) / (double)M;
  s64[id] = v;
  s32[id] = (float)v;
}

// 3-D torus covariance c[c3][b][a] (Eq. 2.3 in d = 3, cell-centre offsets).
__global__ void covariance3_kernel(Cplx<double>* c, int m, int M, double sigma2, double lam, int norm_r) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t M2 = (int64_t)M * M;
  if (id >= M2 * M) return;
  const int c3 = (int)(id / M2);
  const int64_t r = id - (int64_t)c3 * M2;
  const int b = (int)(r / M), a = (int)(r - (int64_t)b * M);
  const double dx = (double)min(a, M - a) / (double)m;
  const double dy = (double)min(b, M - b) / (double)m;
  const double dz = (double)min(c3, M - c3) / (double)m;
  const double dist = norm_r == 1 ? (fabs(dx) + fabs(dy)) + fabs(dz) : sqrt(dx * dx + dy * dy + dz * dz);
  c[id] = Cplx<double>{sigma2 * exp(-dist / lam), 0.0};
}

// Full in-place FFT along one axis of an M^3 array: line `blockIdx.x` =
// (u, v) over the other two axes, elements base + k * stride.
__global__ void fft_line3_kernel(Cplx<double>* data, int M, int logM, const Cplx<double>* tw, int axis) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<double>* s = reinterpret_cast<Cplx<double>*>(smem_raw);
  const int64_t M2 = (int64_t)M * M;
  const int u = (int)(blockIdx.x / M), v = (int)(blockIdx.x - (int64_t)u * M);
  int64_t base, stride;
  if (axis == 0) {
    base = (int64_t)u * M2 + (int64_t)v * M;
    stride = 1;
  } else if (axis == 1) {
    base = (int64_t)u * M2 + v;
    stride = M;
  } else {
    base = (int64_t)u * M + v;
    stride = M2;
  }
  for (int t = threadIdx.x; t < M; t += blockDim.x) s[brev_n(t, logM)] = data[base + t * stride];
  __syncthreads();
  block_fft_rows(s, 1, M, logM, tw, M);
  for (int t = threadIdx.x; t < M; t += blockDim.x) data[base + t * stride] = s[t];
}

// s = sqrt(max(Lambda, 0) / M^3) in FP64 and FP32 (3-D scaling).
__global__ void scale3_kernel(const Cplx<double>* lam, double* s64, float* s32, int64_t n, double inv_n) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n) return;
  const double v = sqrt(fmax(lam[id].x, 0.0) * inv_n);
  s64[id] = v;
  s32[id] = (float)v;
}

// ------------------------------------------------------------ pass 1 -------
// Block (row block rb, sample s): rows r in [rb*R, rb*R + R) of the draw of
// field pair args.pair (2-D: r = q2 of the M x M draw; 3-D: r = q3 M + q2 of
// the M^3 draw; args.n_rows = M^(d-1) rows per sample), FFT along q1, keep
// a < m.  W layout: [sample][r][a] complex (one draw at a time).
template <typename R>
__global__ void ce_rows_kernel(CeRowsArgs args, const R* __restrict__ scale,
                               const Cplx<R>* __restrict__ tw, Cplx<R>* __restrict__ W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<R>* s = reinterpret_cast<Cplx<R>*>(smem_raw);
  const int M = args.M, logM = args.logM, r3 = args.r3, m = args.m, rows = args.rows_per_block;
  const int rb = blockIdx.x, f = args.pair;
  const int64_t sidx = blockIdx.z + args.z_offset;
  const uint64_t sample = (uint64_t)(args.first + sidx);
  const int q2_0 = rb * rows;
  const int halfM = M >> 1;
  const BmTables tb{args.bm_sc, args.bm_lg};
  // one Philox call per pair of consecutive q1 (two complex normals)
  const int ncalls = rows * halfM;
  for (int t = threadIdx.x; t < ncalls; t += blockDim.x) {
    const int r = t / halfM;
    const int q1 = (t - r * halfM) << 1;
    const int q2 = q2_0 + r;
    const uint64_t call = ((uint64_t)q2 * (uint64_t)M + (uint64_t)q1) >> 1;  // q = r M + q1
    const Words4 w = philox4x64_10(call, sample, (uint64_t)args.level, kStreamField0 + f, args.seed);
    R re0, im0, re1, im1;
    box_muller_tab(w.w0, w.w1, tb, re0, im0, scale[(int64_t)q2 * M + q1]);
    box_muller_tab(w.w2, w.w3, tb, re1, im1, scale[(int64_t)q2 * M + q1 + 1]);
    s[r * M + fft_pos(q1, logM, r3)] = Cplx<R>{re0, im0};
    s[r * M + fft_pos(q1 + 1, logM, r3)] = Cplx<R>{re1, im1};
  }
  __syncthreads();
  fft_rows_any(s, rows, M, logM, r3, tw, m >= 4 ? m : M);
  Cplx<R>* out = W + (sidx * (int64_t)args.n_rows + q2_0) * m;
  for (int t = threadIdx.x; t < rows * m; t += blockDim.x) {
    const int r = t / m, a = t - r * m;
    out[(int64_t)r * m + a] = s[r * M + a];
  }
}

// ------------------------------------------------------------ pass 2 -------
// Block (column block cb, sample s): columns a in [cb*C, cb*C + C) of the
// M x ncols array of the sample (2-D: ncols = m, the row-pass output; 3-D:
// ncols = m^2, the middle-pass output indexed [q3][b][a]), FFT along its M
// rows, keep the first m outputs; g layout [sample][layer][row][column]
// with m rows of ncols; Re goes to layer t_re, Im to layer t_im (if any).
template <typename R, typename G>
__global__ void ce_cols_kernel(CeColsArgs args, const Cplx<R>* __restrict__ tw,
                               const Cplx<R>* __restrict__ W, G* __restrict__ g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<R>* s = reinterpret_cast<Cplx<R>*>(smem_raw);
  const int M = args.M, logM = args.logM, r3 = args.r3, m = args.m, C = args.cols_per_block;
  const int64_t nc = args.ncols;
  const int cb = blockIdx.x;
  const int64_t sidx = blockIdx.z + args.z_offset;
  const int64_t a0 = (int64_t)cb * C;
  const Cplx<R>* in = W + (sidx * (int64_t)M) * nc + a0;
  for (int t = threadIdx.x; t < M * C; t += blockDim.x) {
    const int q2 = t / C, cc = t - q2 * C;
    s[cc * M + fft_pos(q2, logM, r3)] = in[(int64_t)q2 * nc + cc];
  }
  __syncthreads();
  fft_rows_any(s, C, M, logM, r3, tw, m >= 4 ? m : M);
  const bool has_im = args.t_im >= 0;
  G* g0 = g + (sidx * args.n_layers + args.t_re) * (int64_t)m * nc;
  G* g1 = g + (sidx * args.n_layers + (has_im ? args.t_im : args.t_re)) * (int64_t)m * nc;
  // FP32 fields add the mean in FP32 (an FP64 add and its two conversions
  // would run on the FP64 pipe, 1/64 of the FP32 rate on this GPU)
  const R mre = (R)args.mu_re, mim = (R)args.mu_im;
  for (int t = threadIdx.x; t < m * C; t += blockDim.x) {
    const int b = t / C, cc = t - b * C;
    const Cplx<R> v = s[cc * M + b];
    if constexpr (std::is_same<G, float>::value) {
      g0[(int64_t)b * nc + a0 + cc] = mre + v.x;
      if (has_im) g1[(int64_t)b * nc + a0 + cc] = mim + v.y;
    } else {
      g0[(int64_t)b * nc + a0 + cc] = (G)(args.mu_re + (double)v.x);
      if (has_im) g1[(int64_t)b * nc + a0 + cc] = (G)(args.mu_im + (double)v.y);
    }
  }
}

// ------------------------------------------------------ 3-D middle pass -----
// Block (column block cb, slab q3, sample s): columns a in [cb*C, cb*C + C)
// of the M x m slab q3 of the row-pass output W1[s][q3][q2][a], FFT along q2,
// keep b < m; output W2[s][q3][b][a] complex.
template <typename R>
__global__ void ce_mid_kernel(CeColsArgs args, const Cplx<R>* __restrict__ tw,
                              const Cplx<R>* __restrict__ W1, Cplx<R>* __restrict__ W2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<R>* s = reinterpret_cast<Cplx<R>*>(smem_raw);
  const int M = args.M, logM = args.logM, m = args.m, C = args.cols_per_block;
  const int a0 = blockIdx.x * C, q3 = blockIdx.y;
  const int64_t sidx = blockIdx.z + args.z_offset;
  const Cplx<R>* in = W1 + ((sidx * M + q3) * (int64_t)M) * m + a0;
  for (int t = threadIdx.x; t < M * C; t += blockDim.x) {
    const int q2 = t / C, cc = t - q2 * C;
    s[cc * M + brev_n(q2, logM)] = in[(int64_t)q2 * m + cc];
  }
  __syncthreads();
  block_fft_rows(s, C, M, logM, tw, m >= 4 ? m : M);
  Cplx<R>* out = W2 + ((sidx * M + q3) * (int64_t)m) * m + a0;
  for (int t = threadIdx.x; t < m * C; t += blockDim.x) {
    const int b = t / C, cc = t - b * C;
    out[(int64_t)b * m + cc] = s[cc * M + b];
  }
}

// ----------------------------------------------------------- host side ----
int ce_build_table(int m, int M, double sigma2, double lam, int norm_r, int cutoff, void* scratch,
                   double* s64, float* s32, double* minmax_dev, void* tw64, void* tw32,
                   cudaStream_t st) {
  const int r3 = M % 3 == 0 ? 1 : 0;
  const int logM = ilog2(r3 ? M / 3 : M);
  Cplx<double>* a = reinterpret_cast<Cplx<double>*>(scratch);
  Cplx<double>* b = a + (int64_t)M * M;
  const int64_t n = (int64_t)M * M;
  const int nt = 256;
  const unsigned nblk = (unsigned)((n + nt - 1) / nt);
  twiddle_kernel<double><<<(M + nt - 1) / nt, nt, 0, st>>>((Cplx<double>*)tw64, M);
  twiddle_kernel<float><<<(M + nt - 1) / nt, nt, 0, st>>>((Cplx<float>*)tw32, M);
  covariance_kernel<<<nblk, nt, 0, st>>>(a, m, M, sigma2, lam, norm_r, cutoff);
  const size_t sm = (size_t)M * sizeof(Cplx<double>);
  cudaFuncSetAttribute(fft_rows_full_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  fft_rows_full_kernel<<<M, 256, sm, st>>>(a, M, logM, r3, (const Cplx<double>*)tw64);
  transpose_kernel<<<nblk, nt, 0, st>>>(a, b, M);
  fft_rows_full_kernel<<<M, 256, sm, st>>>(b, M, logM, r3, (const Cplx<double>*)tw64);
  transpose_kernel<<<nblk, nt, 0, st>>>(b, a, M);
  minmax_kernel<<<1, 1024, 0, st>>>(a, n, minmax_dev);
  scale_kernel<<<nblk, nt, 0, st>>>(a, s64, s32, M);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int ce_build_table3(int m, int M, double sigma2, double lam, int norm_r, void* scratch, double* s64,
                    float* s32, double* minmax_dev, void* tw64, void* tw32, cudaStream_t st) {
  const int logM = ilog2(M);
  Cplx<double>* a = reinterpret_cast<Cplx<double>*>(scratch);
  const int64_t n = (int64_t)M * M * M;
  const int nt = 256;
  const unsigned nblk = (unsigned)((n + nt - 1) / nt);
  twiddle_kernel<double><<<(M + nt - 1) / nt, nt, 0, st>>>((Cplx<double>*)tw64, M);
  twiddle_kernel<float><<<(M + nt - 1) / nt, nt, 0, st>>>((Cplx<float>*)tw32, M);
  covariance3_kernel<<<nblk, nt, 0, st>>>(a, m, M, sigma2, lam, norm_r);
  const size_t sm = (size_t)M * sizeof(Cplx<double>);
  cudaFuncSetAttribute(fft_line3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  for (int axis = 0; axis < 3; ++axis)
    fft_line3_kernel<<<(unsigned)((int64_t)M * M), 256, sm, st>>>(a, M, logM, (const Cplx<double>*)tw64, axis);
  minmax_kernel<<<1, 1024, 0, st>>>(a, n, minmax_dev);
  scale3_kernel<<<nblk, nt, 0, st>>>(a, s64, s32, n, 1.0 / (double)n);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename R, typename G>
static int ce_sample3_impl(const CeLaunch& L, const R* scale, const void* tw, void* W, G* g, cudaStream_t st) {
  const size_t esz = sizeof(Cplx<R>);
  const int budget = (int)(65536 / sizeof(Cplx<double>)) * (int)(sizeof(Cplx<double>) / esz);
  const int M = L.M, m = L.m;
  const int per = std::max(1, std::min(budget / M, M));  // rows (pass 1) or columns per block
  const int rows = std::min(per, M);
  const int cmid = std::min(per, m);
  const int64_t ncol3 = (int64_t)m * m;
  const int c3 = (int)std::min<int64_t>(per, ncol3);
  Cplx<R>* W1 = reinterpret_cast<Cplx<R>*>(W);
  Cplx<R>* W2 = W1 + (int64_t)M * M * m * L.n_samples;
  CeRowsArgs ra;
  ra.bm_sc = L.bm_sc;
  ra.bm_lg = L.bm_lg;
  ra.M = M; ra.logM = ilog2(M); ra.r3 = 0; ra.m = m; ra.rows_per_block = rows; ra.pair = L.pair;
  ra.level = L.level; ra.seed = L.seed; ra.first = L.first; ra.n_rows = M * M;
  CeColsArgs ma;
  ma.M = M; ma.logM = ra.logM; ma.r3 = 0; ma.m = m; ma.cols_per_block = cmid; ma.n_layers = L.n_layers;
  ma.ncols = m;
  ma.t_re = L.t_re; ma.t_im = L.t_im; ma.mu_re = L.mu_re; ma.mu_im = L.mu_im;
  CeColsArgs ca = ma;
  ca.cols_per_block = c3;
  ca.ncols = ncol3;
  const size_t sm_r = (size_t)rows * M * esz, sm_m = (size_t)cmid * M * esz, sm_c = (size_t)c3 * M * esz;
  cudaFuncSetAttribute(ce_rows_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_r);
  cudaFuncSetAttribute(ce_mid_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_m);
  cudaFuncSetAttribute(ce_cols_kernel<R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_c);
  for (int64_t z0 = 0; z0 < L.n_samples; z0 += 65535) {
    const unsigned nz = (unsigned)((L.n_samples - z0) < 65535 ? (L.n_samples - z0) : 65535);
    ra.z_offset = ma.z_offset = ca.z_offset = z0;
    ce_rows_kernel<R><<<dim3((unsigned)(M * M / rows), 1u, nz), 256, sm_r, st>>>(ra, scale, (const Cplx<R>*)tw, W1);
    ce_mid_kernel<R><<<dim3((unsigned)(m / cmid), (unsigned)M, nz), 256, sm_m, st>>>(ma, (const Cplx<R>*)tw, W1, W2);
    ce_cols_kernel<R, G><<<dim3((unsigned)(ncol3 / c3), 1u, nz), 256, sm_c, st>>>(ca, (const Cplx<R>*)tw, W2, g);
    g_ce_launches += 3;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------- fused passes at M = 32 (FP32) -----
// The 16 x 16 grids of the standard embedding (M = 2m = 32): one block per
// sample does both passes.  The block draws the sample's 32 x 32 complex
// normals into shared memory (the same Philox calls and scaling as
// ce_rows_kernel), then each warp transforms whole rows with one point per
// lane: a 32-point decimation-in-frequency FFT whose butterflies exchange
// values between lanes by shuffles (stage of half-span h: the lane with bit
// h clear keeps u + v, the other (u - v) W^((lane mod h) 32 / (2h))), which
// leaves X[brev(lane)] in each lane; the even lanes hold the kept outputs a
// < 16 and store them transposed, and the columns go through the same FFT,
// the even lanes writing g[b][a] = mu + Re / Im for b < 16.  Same sums as the
// two-pass form up to rounding order.
constexpr int kFusedM = 32;


__device__ __forceinline__ void fft32_dif_warp(float& xr, float& xi, const float2 (&w)[5], int lane) {
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int h = 16 >> st;
    const float pr = __shfl_xor_sync(full, xr, h), pi = __shfl_xor_sync(full, xi, h);
    if ((lane & h) == 0) {
      xr = xr + pr;
      xi = xi + pi;
    } else {
      const float dr = pr - xr, di = pi - xi;  // (u - v), v = this lane's value
      xr = dr * w[st].x - di * w[st].y;
      xi = dr * w[st].y + di * w[st].x;
    }
  }
}

__global__ void __launch_bounds__(256) ce_fused32_kernel(CeRowsArgs args, CeColsArgs cargs,
                                                         const float* __restrict__ scale,
                                                         const Cplx<float>* __restrict__ tw,
                                                         float* __restrict__ g) {
  __shared__ Cplx<float> s[kFusedM * kFusedM];           // the draw, [q2][q1]
  __shared__ Cplx<float> wt[(kFusedM / 2) * kFusedM];    // row-pass output, [a][q2]
  constexpr int M = kFusedM, m = kFusedM / 2;
  const int64_t sidx = blockIdx.x + args.z_offset;
  const uint64_t sample = (uint64_t)(args.first + sidx);
  const BmTables tb{args.bm_sc, args.bm_lg};
  for (int c = threadIdx.x; c < M * M / 2; c += blockDim.x) {  // one Philox call per two points
    const int q = 2 * c, q2 = q / M, q1 = q - q2 * M;
    const Words4 w = philox4x64_10((uint64_t)c, sample, (uint64_t)args.level, kStreamField0 + args.pair, args.seed);
    float re0, im0, re1, im1;
    box_muller_tab(w.w0, w.w1, tb, re0, im0, scale[q]);
    box_muller_tab(w.w2, w.w3, tb, re1, im1, scale[q + 1]);
    s[q2 * M + q1] = Cplx<float>{re0, im0};
    s[q2 * M + q1 + 1] = Cplx<float>{re1, im1};
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  float2 w5[5];
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int h = 16 >> st;
    const Cplx<float> t = tw[(lane & (h - 1)) * (16 / h)];
    w5[st] = make_float2(t.x, t.y);
  }
  const int a_out = (int)(__brev((unsigned)lane) >> 27);  // this lane's output index
  __syncthreads();
  for (int q2 = warp; q2 < M; q2 += nwarp) {  // rows: W[q2][a], a < m
    Cplx<float> x = s[q2 * M + lane];
    fft32_dif_warp(x.x, x.y, w5, lane);
    if (a_out < m) wt[a_out * M + q2] = x;
  }
  __syncthreads();
  const bool has_im = cargs.t_im >= 0;
  float* g0 = g + (sidx * cargs.n_layers + cargs.t_re) * (int64_t)(m * m);
  float* g1 = g + (sidx * cargs.n_layers + (has_im ? cargs.t_im : cargs.t_re)) * (int64_t)(m * m);
  const float mre = (float)cargs.mu_re, mim = (float)cargs.mu_im;
  for (int a = warp; a < m; a += nwarp) {  // columns: y[b][a], b < m
    Cplx<float> x = wt[a * M + lane];
    fft32_dif_warp(x.x, x.y, w5, lane);
    if (a_out < m) {
      g0[a_out * m + a] = mre + x.x;
      if (has_im) g1[a_out * m + a] = mim + x.y;
    }
  }
}

template <typename R, typename G>
static int ce_sample_impl(const CeLaunch& L, const R* scale, const void* tw, void* W, G* g,
                          cudaStream_t st) {
  if (L.dim == 3) return ce_sample3_impl<R, G>(L, scale, tw, W, g, st);
  if constexpr (std::is_same<R, float>::value && std::is_same<G, float>::value) {
    if (L.M == kFusedM && L.m == kFusedM / 2) {  // both passes in one kernel, W unused
      CeRowsArgs ra{};
      ra.bm_sc = L.bm_sc;
      ra.bm_lg = L.bm_lg;
      ra.M = L.M; ra.logM = ilog2(L.M); ra.r3 = 0; ra.m = L.m; ra.rows_per_block = L.M;
      ra.pair = L.pair; ra.level = L.level; ra.seed = L.seed; ra.first = L.first; ra.n_rows = L.M;
      CeColsArgs ca{};
      ca.M = L.M; ca.logM = ra.logM; ca.r3 = 0; ca.m = L.m; ca.cols_per_block = L.m; ca.n_layers = L.n_layers;
      ca.ncols = L.m; ca.t_re = L.t_re; ca.t_im = L.t_im; ca.mu_re = L.mu_re; ca.mu_im = L.mu_im;
      for (int64_t z0 = 0; z0 < L.n_samples; z0 += (int64_t)1 << 30) {
        const int64_t nz = std::min<int64_t>(L.n_samples - z0, (int64_t)1 << 30);
        ra.z_offset = z0;
        ce_fused32_kernel<<<(unsigned)nz, 256, 0, st>>>(ra, ca, scale, (const Cplx<float>*)tw, g);
        g_ce_launches += 1;
      }
      return cudaGetLastError() == cudaSuccess ? 0 : -1;
    }
  }
  const size_t esz = sizeof(Cplx<R>);
  // rows / columns per block: at most 64 KB of FP64 (128 KB of FP32) per
  // block, a power of two so that it divides M (= 2^k or 3 2^k) and m
  const int budget = (int)(65536 / sizeof(Cplx<double>)) * (int)(sizeof(Cplx<double>) / esz);
  const int r3 = L.M % 3 == 0 ? 1 : 0;
  auto pow2_floor = [](int v) { int p = 1; while (2 * p <= v) p *= 2; return p; };
  int rows = pow2_floor(std::max(1, budget / L.M));
  while (L.M % rows) rows >>= 1;  // M = 3 2^k: at most 2^k rows per block
  int cols = pow2_floor(std::max(1, budget / L.M));
  if (cols > L.m) cols = L.m;
  CeRowsArgs ra;
  ra.bm_sc = L.bm_sc;
  ra.bm_lg = L.bm_lg;
  ra.M = L.M; ra.logM = ilog2(r3 ? L.M / 3 : L.M); ra.r3 = r3; ra.m = L.m; ra.rows_per_block = rows;
  ra.pair = L.pair; ra.level = L.level; ra.seed = L.seed; ra.first = L.first; ra.n_rows = L.M;
  CeColsArgs ca;
  ca.M = L.M; ca.logM = ra.logM; ca.r3 = r3; ca.m = L.m; ca.cols_per_block = cols; ca.n_layers = L.n_layers;
  ca.ncols = L.m;
  ca.t_re = L.t_re; ca.t_im = L.t_im; ca.mu_re = L.mu_re; ca.mu_im = L.mu_im;
  const size_t sm_r = (size_t)rows * L.M * esz;
  const size_t sm_c = (size_t)cols * L.M * esz;
  cudaFuncSetAttribute(ce_rows_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_r);
  cudaFuncSetAttribute(ce_cols_kernel<R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_c);
  // grid.z is limited to 65535: launch in slices of samples
  for (int64_t z0 = 0; z0 < L.n_samples; z0 += 65535) {
    const unsigned nz = (unsigned)((L.n_samples - z0) < 65535 ? (L.n_samples - z0) : 65535);
    ra.z_offset = z0;
    ca.z_offset = z0;
    dim3 gr((unsigned)(L.M / rows), 1u, nz);
    ce_rows_kernel<R><<<gr, 256, sm_r, st>>>(ra, scale, (const Cplx<R>*)tw, (Cplx<R>*)W);
    dim3 gc((unsigned)(L.m / cols), 1u, nz);
    ce_cols_kernel<R, G><<<gc, 256, sm_c, st>>>(ca, (const Cplx<R>*)tw, (const Cplx<R>*)W, g);
    g_ce_launches += 2;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int ce_sample_fp64(const CeLaunch& L, const double* scale, const void* tw, void* W, double* g,
                   cudaStream_t st) {
  return ce_sample_impl<double, double>(L, scale, tw, W, g, st);
}

int ce_sample_fp32(const CeLaunch& L, const float* scale, const void* tw, void* W, float* g,
                   cudaStream_t st) {
  return ce_sample_impl<float, float>(L, scale, tw, W, g, st);
}

__global__ void bm_tables_kernel(double2* sc, double* lg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kSinCosTab) {
    double sv, cv;
    sincospi(2.0 * (double)i / (double)kSinCosTab, &sv, &cv);
    sc[i] = make_double2(cv, sv);
  }
  if (i < kLogTab) {
    const double F = 0.5 + ((double)i + 0.5) / 2048.0;
    lg[3 * i] = F;
    lg[3 * i + 1] = -2.0 / F;
    lg[3 * i + 2] = -2.0 * log(F);
  }
  if (i < kLogExpTab) lg[3 * kLogTab + i] = -2.0 * log(ldexp(1.0, -i));  // 2 i ln 2
}

int bm_tables_build(double2* sc, double* lg, cudaStream_t st) {
  bm_tables_kernel<<<(kSinCosTab + 255) / 256, 256, 0, st>>>(sc, lg);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

size_t ce_w_bytes_per_sample(int m, int M, bool fp32, int dim) {
  const size_t e = fp32 ? sizeof(Cplx<float>) : sizeof(Cplx<double>);
  if (dim == 3) return ((size_t)M * M * m + (size_t)M * m * m) * e;  // W1 then W2
  return (size_t)M * m * e;
}

}  // namespace mlmc

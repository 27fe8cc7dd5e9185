// Per-sample gathering of system results and the level reduction (Eq. 3.6,
// Eq. 4.2): compensated FP64 sums of Q_f, Q_c, Y = Q_f - Q_c, the CGV
// average Q_cg = (1/4) sum of the four coarse Q's and Y_g = Q_f - Q_cg, and
// their squares, in a fixed order (deterministic for a given sample count).
#include "common.cuh"
#include "kernels.cuh"

namespace mlmc {

__global__ void gather_kernel(const double* q_sys, const int32_t* it_sys, int64_t n, int nc, int cgv,
                              int64_t cells_f, int64_t cells_c, double* qf, double* qc, double* qcg,
                              int32_t* iters, unsigned long long* it_acc) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  long long it = 0, itc = 0, itcc = 0;  // iterations; cells x iterations, fine and coarse
  if (s < n) {
    qf[s] = q_sys[s];
    it = it_sys[s];
    itc = (long long)it_sys[s] * cells_f;
    if (iters) iters[s] = it_sys[s];
    if (nc == 0) {
      qc[s] = 0.0;
      qcg[s] = cgv ? 0.0 : nan("");
    } else {
      const double* qq = q_sys + n + s * nc;
      qc[s] = qq[0];
      double acc = qq[0];
      for (int o = 0; o < nc; ++o) {
        it += it_sys[n + s * nc + o];
        itcc += (long long)it_sys[n + s * nc + o] * cells_c;
        if (o) acc += qq[o];
      }
      qcg[s] = nc >= 4 ? acc * (1.0 / nc) : nan("");
    }
  }
  it = warp_sum(it);
  itc = warp_sum(itc);
  itcc = warp_sum(itcc);
  if ((threadIdx.x & 31) == 0 && it) {
    atomicAdd(it_acc, (unsigned long long)it);
    atomicAdd(it_acc + 1, (unsigned long long)itc);
    if (itcc) atomicAdd(it_acc + 2, (unsigned long long)itcc);
  }
}

int gather_launch(const double* q_sys, const int32_t* it_sys, int64_t n, int n_coarse, int cgv,
                  int64_t cells_f, int64_t cells_c, double* qf, double* qc, double* qcg, int32_t* iters,
                  int64_t* it_acc, cudaStream_t st) {
  if (n <= 0) return 0;
  gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      q_sys, it_sys, n, n_coarse, cgv, cells_f, cells_c, qf, qc, qcg, iters, (unsigned long long*)it_acc);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

struct Neu {
  double s, c;
};

// Neumaier compensated addition.
__device__ __forceinline__ void neu_add(Neu& a, double x) {
  const double t = __dadd_rn(a.s, x);
  if (fabs(a.s) >= fabs(x))
    a.c = __dadd_rn(a.c, __dadd_rn(__dadd_rn(a.s, -t), x));
  else
    a.c = __dadd_rn(a.c, __dadd_rn(__dadd_rn(x, -t), a.s));
  a.s = t;
}

__device__ __forceinline__ void neu_merge(Neu& a, const Neu& b) {
  neu_add(a, b.s);
  a.c = __dadd_rn(a.c, b.c);
}

constexpr int kRedThreads = 512;
constexpr int kRedMaxBlocks = 256;

struct RedPartial {
  double s[10], c[10];
  long long n, n_failed;
};

// Phase 1: block b sums the samples of its contiguous range with Neumaier
// compensation, in a fixed order (threads strided, then a fixed tree).
__global__ void __launch_bounds__(kRedThreads) reduce_partial_kernel(const double* qf, const double* qc,
                                                                     const double* qcg, int64_t n, int cgv,
                                                                     RedPartial* part) {
  const int64_t lo = n * blockIdx.x / gridDim.x, hi = n * (blockIdx.x + 1) / gridDim.x;
  Neu acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = Neu{0.0, 0.0};
  long long nok = 0, nfail = 0;
  for (int64_t s = lo + threadIdx.x; s < hi; s += blockDim.x) {
    const double f = qf[s], c = qc[s];
    const double g = cgv ? qcg[s] : 0.0;
    if (!isfinite(f) || !isfinite(c) || !isfinite(g)) {
      ++nfail;
      continue;
    }
    ++nok;
    const double y = __dadd_rn(f, -c);
    neu_add(acc[0], f);
    neu_add(acc[1], __dmul_rn(f, f));
    neu_add(acc[2], c);
    neu_add(acc[3], __dmul_rn(c, c));
    neu_add(acc[4], y);
    neu_add(acc[5], __dmul_rn(y, y));
    if (cgv) {
      const double yg = __dadd_rn(f, -g);
      neu_add(acc[6], g);
      neu_add(acc[7], __dmul_rn(g, g));
      neu_add(acc[8], yg);
      neu_add(acc[9], __dmul_rn(yg, yg));
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      Neu b{__shfl_down_sync(0xffffffffu, acc[k].s, o), __shfl_down_sync(0xffffffffu, acc[k].c, o)};
      if (lane < o) neu_merge(acc[k], b);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    nok += __shfl_down_sync(0xffffffffu, nok, o);
    nfail += __shfl_down_sync(0xffffffffu, nfail, o);
  }
  __shared__ double ss[kRedThreads / 32][10], sc[kRedThreads / 32][10];
  __shared__ long long sn[kRedThreads / 32], sf[kRedThreads / 32];
  if (lane == 0) {
    for (int k = 0; k < 10; ++k) {
      ss[warp][k] = acc[k].s;
      sc[warp][k] = acc[k].c;
    }
    sn[warp] = nok;
    sf[warp] = nfail;
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    const int k = threadIdx.x;
    Neu t{0.0, 0.0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) neu_merge(t, Neu{ss[w][k], sc[w][k]});
    part[blockIdx.x].s[k] = t.s;
    part[blockIdx.x].c[k] = t.c;
  }
  if (threadIdx.x == 0) {
    long long tn = 0, tf = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tn += sn[w];
      tf += sf[w];
    }
    part[blockIdx.x].n = tn;
    part[blockIdx.x].n_failed = tf;
  }
}

// Phase 2: one thread per sum combines the partials in block order.
__global__ void reduce_final_kernel(const RedPartial* part, int nparts, const int64_t* it_acc,
                                    LevelSumsDev* out) {
  const int k = threadIdx.x;
  if (k < 10) {
    Neu t{0.0, 0.0};
    for (int b = 0; b < nparts; ++b) neu_merge(t, Neu{part[b].s[k], part[b].c[k]});
    out->s[k] = __dadd_rn(t.s, t.c);
  }
  if (k == 0) {
    long long tn = 0, tf = 0;
    for (int b = 0; b < nparts; ++b) {
      tn += part[b].n;
      tf += part[b].n_failed;
    }
    out->n = tn;
    out->n_failed = tf;
    out->iters = it_acc ? *it_acc : 0;
  }
}

size_t reduce_ws_bytes() { return sizeof(RedPartial) * kRedMaxBlocks; }

int reduce_launch(const double* qf, const double* qc, const double* qcg, int64_t n, int cgv,
                  const int64_t* it_acc, LevelSumsDev* out, void* ws, cudaStream_t st) {
  int64_t nb = (n + 8 * kRedThreads - 1) / (8 * kRedThreads);
  nb = nb < 1 ? 1 : (nb > kRedMaxBlocks ? kRedMaxBlocks : nb);
  RedPartial* part = reinterpret_cast<RedPartial*>(ws);
  reduce_partial_kernel<<<(unsigned)nb, kRedThreads, 0, st>>>(qf, qc, qcg, n, cgv, part);
  reduce_final_kernel<<<1, 32, 0, st>>>(part, (int)nb, it_acc, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

__global__ void philox_kernel(uint64_t seed, uint64_t level, uint64_t sample, uint64_t stream,
                              uint64_t first_call, int64_t n, uint64_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Words4 w = philox4x64_10(first_call + (uint64_t)i, sample, level, stream, seed);
  out[4 * i + 0] = w.w0;
  out[4 * i + 1] = w.w1;
  out[4 * i + 2] = w.w2;
  out[4 * i + 3] = w.w3;
}

int philox_launch(uint64_t seed, uint64_t level, uint64_t sample, uint64_t stream,
                  uint64_t first_call, int64_t n_calls, uint64_t* out, cudaStream_t st) {
  if (n_calls <= 0) return 0;
  philox_kernel<<<(unsigned)((n_calls + 255) / 256), 256, 0, st>>>(seed, level, sample, stream,
                                                                   first_call, n_calls, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// The four normals of each call, by the same Box-Muller routine the field
// kernels use (FP64 table-driven, or FP32 when fp32 != 0).
__global__ void normals_kernel(uint64_t seed, uint64_t level, uint64_t sample, uint64_t stream,
                               uint64_t first_call, int64_t n, BmTables tb, int fp32, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Words4 w = philox4x64_10(first_call + (uint64_t)i, sample, level, stream, seed);
  if (fp32) {
    float a, b, c, d;
    box_muller_tab(w.w0, w.w1, tb, a, b);
    box_muller_tab(w.w2, w.w3, tb, c, d);
    out[4 * i] = a, out[4 * i + 1] = b, out[4 * i + 2] = c, out[4 * i + 3] = d;
  } else {
    double a, b, c, d;
    box_muller_tab(w.w0, w.w1, tb, a, b);
    box_muller_tab(w.w2, w.w3, tb, c, d);
    out[4 * i] = a, out[4 * i + 1] = b, out[4 * i + 2] = c, out[4 * i + 3] = d;
  }
}

int normals_launch(uint64_t seed, uint64_t level, uint64_t sample, uint64_t stream, uint64_t first_call,
                   int64_t n_calls, const double2* sc, const double* lg, int fp32, double* out,
                   cudaStream_t st) {
  if (n_calls <= 0) return 0;
  normals_kernel<<<(unsigned)((n_calls + 255) / 256), 256, 0, st>>>(seed, level, sample, stream, first_call,
                                                                     n_calls, BmTables{sc, lg}, fp32, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

__global__ void f32_to_f64_kernel(const float* in, double* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}

int f32_to_f64_launch(const float* in, double* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return 0;
  f32_to_f64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace mlmc

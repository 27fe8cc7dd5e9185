// C ABI of the MLMC level-batch library: context, level batches, the adaptive
// estimator and stage outputs.  Declarations and contracts: include/mlmc.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mlmc.h"
#include "common.cuh"
#include "kernels.cuh"

using namespace mlmc;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& what) {
  g_last_error = what;
  return code;
}

#define CUDA_TRY(expr)                                                                    \
  do {                                                                                    \
    cudaError_t _e = (expr);                                                              \
    if (_e != cudaSuccess)                                                                \
      return fail(_e == cudaErrorMemoryAllocation ? MLMC_ERR_NOMEM : MLMC_ERR_CUDA,       \
                  std::string(#expr) + ": " + cudaGetErrorString(_e));                    \
  } while (0)

struct Buf {
  void* p = nullptr;
  size_t cap = 0;
  int ensure(size_t bytes) {
    if (bytes <= cap) return 0;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(MLMC_ERR_NOMEM, std::string("cudaMalloc(") + std::to_string(want) + "): " +
                                      cudaGetErrorString(e));
    }
    cap = want;
    return 0;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <typename T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

struct LevelTable {
  int m = 0, M = 0;
  double lam_min = 0, lam_max = 0;
  Buf s64, s32, tw64, tw32;
};

constexpr size_t kChunkBudget = size_t(2) << 30;  // bytes of per-sample buffers per chunk

}  // namespace

struct mlmc_ctx {
  int device = 0;
  cudaStream_t st = nullptr;
  mlmc_model model{};
  int nsm = 0;
  std::vector<LevelTable> lev;
  Buf W, g, ws, qsys, itsys, oqf, oqc, oqg, oit, sums, itacc, g64, bm;
  bool prof_on = false;
  mlmc_profile_stats prof{};
};

namespace {

int n_pairs(const mlmc_model& md) { return (md.n_layers + 1) / 2; }
int n_coarse(const mlmc_model& md, int level) { return level == 0 ? 0 : (md.cgv ? 4 : 1); }
bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int check_model(const mlmc_model& md) {
  if (md.n_layers < 1 || md.n_layers > MLMC_MAX_LAYERS) return fail(MLMC_ERR_ARG, "n_layers must be 1..8");
  if (md.k_kind != 0 && md.k_kind != 1) return fail(MLMC_ERR_ARG, "k_kind must be 0 or 1");
  if (md.norm_r != 1 && md.norm_r != 2) return fail(MLMC_ERR_ARG, "norm_r must be 1 or 2");
  if (!is_pow2(md.m0) || md.m0 < 2) return fail(MLMC_ERR_ARG, "m0 must be a power of two >= 2");
  if (md.L < 0 || md.L >= MLMC_MAX_LEVELS) return fail(MLMC_ERR_ARG, "L must be 0..11");
  if ((int64_t)md.m0 << md.L > 4096) return fail(MLMC_ERR_TOOBIG, "m0 * 2^L must be <= 4096");
  if (md.cgv < 0 || md.cgv > 2) return fail(MLMC_ERR_ARG, "cgv must be 0, 1 or 2");
  if (md.prec < 0 || md.prec > 1) return fail(MLMC_ERR_ARG, "prec must be 0 or 1");
  if (!(md.tol > 0) || md.max_it < 1) return fail(MLMC_ERR_ARG, "tol must be > 0 and max_it >= 1");
  if (!(md.if_hi >= md.if_lo)) return fail(MLMC_ERR_ARG, "if_hi must be >= if_lo");
  for (int t = 0; t < md.n_layers; ++t) {
    if (!(md.sigma2[t] >= 0)) return fail(MLMC_ERR_ARG, "sigma2 must be >= 0");
    if (md.k_kind == 1 && !(md.lam[t] > 0)) return fail(MLMC_ERR_ARG, "lam must be > 0");
  }
  if (md.k_kind == 1)
    for (int f = 0; 2 * f + 1 < md.n_layers; ++f)
      if (md.sigma2[2 * f] != md.sigma2[2 * f + 1] || md.lam[2 * f] != md.lam[2 * f + 1])
        return fail(MLMC_ERR_ARG, "layers 2f and 2f+1 must share sigma2 and lam");
  return 0;
}

SolveArgs base_args(const mlmc_ctx* c, int level, uint64_t seed, int64_t first) {
  const mlmc_model& md = c->model;
  SolveArgs a;
  std::memset(&a, 0, sizeof(a));
  a.m = md.m0 << level;
  a.level = level;
  a.seed = seed;
  a.first = first;
  a.n_layers = md.n_layers;
  a.if_lo = md.if_lo;
  a.if_hi = md.if_hi;
  for (int t = 0; t < MAX_LAYERS_DEV; ++t) {
    a.mu[t] = md.mu[t];
    a.sigma[t] = std::sqrt(md.sigma2[t]);
  }
  a.ksrc = md.k_kind == 0 ? KSRC_CONST : KSRC_FIELDS;
  a.cgv_on_k = md.cgv == 2;
  a.tol = md.tol;
  a.max_it = md.max_it;
  a.inner_tol = 1e-5;
  return a;
}

// Fields of chunk samples [first, first + n) of `level` into c->g.
int run_fields(mlmc_ctx* c, int level, int64_t first, int64_t n, uint64_t seed) {
  const mlmc_model& md = c->model;
  const LevelTable& T = c->lev[level];
  const bool f32 = md.prec != 0;
  CeLaunch L;
  L.bm_sc = c->bm.as<double2>();
  L.bm_lg = reinterpret_cast<const double*>(c->bm.as<double2>() + kSinCosTab);
  L.M = T.M;
  L.m = T.m;
  L.n_pairs = n_pairs(md);
  L.n_layers = md.n_layers;
  L.level = level;
  L.seed = seed;
  L.first = first;
  L.n_samples = n;
  for (int t = 0; t < MAX_LAYERS_DEV; ++t) L.mu[t] = md.mu[t];
  int r;
  if (int e = c->W.ensure(ce_w_bytes_per_sample(T.m, T.M, L.n_pairs, f32) * n)) return e;
  if (int e = c->g.ensure((size_t)n * md.n_layers * T.m * T.m * (f32 ? 4 : 8))) return e;
  if (f32)
    r = ce_sample_fp32(L, T.s32.as<float>(), T.tw32.p, c->W.p, c->g.as<float>(), c->st);
  else
    r = ce_sample_fp64(L, T.s64.as<double>(), T.tw64.p, c->W.p, c->g.as<double>(), c->st);
  if (r) return fail(MLMC_ERR_CUDA, std::string("field kernels: ") + cudaGetErrorString(cudaGetLastError()));
  return 0;
}

int64_t chunk_samples(const mlmc_ctx* c, int level) {
  const mlmc_model& md = c->model;
  const int m = md.m0 << level;
  const bool f32 = md.prec != 0;
  size_t per = (size_t)(1 + n_coarse(md, level)) * 12;
  if (md.k_kind == 1) {
    per += ce_w_bytes_per_sample(m, c->lev[level].M, n_pairs(md), f32);
    per += (size_t)md.n_layers * m * m * (f32 ? 4 : 8);
  }
  int64_t s = (int64_t)(kChunkBudget / per);
  return std::max<int64_t>(1, std::min<int64_t>(s, 1 << 18));
}

// Bytes of global solver workspace a context may hold (bounds the number of
// resident blocks for very large grids).
constexpr size_t kWsBudget = size_t(16) << 30;

// Solve the systems of one chunk; results into c->qsys / c->itsys.
int run_solves(mlmc_ctx* c, SolveArgs a, int64_t n_samples, int nc, int64_t max_rows) {
  const int prec = c->model.prec;
  a.n_samples = n_samples;
  a.n_coarse = nc;
  SolvePlan P;
  if (solve_plan(a.m, prec, &P)) return fail(MLMC_ERR_CUDA, "occupancy query failed");
  const int64_t n_sys = n_samples * (1 + nc);
  int64_t nb = std::min<int64_t>((n_sys + P.groups_per_block - 1) / P.groups_per_block,
                                 (int64_t)c->nsm * P.blocks_per_sm);
  if (!P.use_smem) {
    const size_t per_block = P.ws_stride * P.groups_per_block;
    nb = std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)(kWsBudget / per_block)));
    if (int e = c->ws.ensure(per_block * nb)) return e;
    a.ws = c->ws.as<unsigned char>();
  }
  if (int e = c->qsys.ensure((size_t)std::max<int64_t>(n_sys, max_rows) * 8)) return e;
  if (int e = c->itsys.ensure((size_t)std::max<int64_t>(n_sys, max_rows) * 4)) return e;
  a.q = c->qsys.as<double>();
  a.iters = c->itsys.as<int32_t>();
  if (solve_launch(a, prec, P, (int)nb, c->st))
    return fail(MLMC_ERR_CUDA, std::string("solve kernel: ") + cudaGetErrorString(cudaGetLastError()));
  return 0;
}

// CUDA-event timing of one stage on the context stream (profiling only).
struct StageTimer {
  mlmc_ctx* c;
  int stage;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  StageTimer(mlmc_ctx* c_, int stage_) : c(c_), stage(stage_) {
    if (!c->prof_on) return;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->st);
  }
  void stop(int launches) {
    if (!c->prof_on) return;
    cudaEventRecord(e1, c->st);
    c->prof.launches[stage] += launches;
    pending().push_back({stage, e0, e1});
    e0 = e1 = nullptr;
  }
  struct Pend {
    int stage;
    cudaEvent_t a, b;
  };
  static std::vector<Pend>& pending() {
    static thread_local std::vector<Pend> v;
    return v;
  }
  // after a stream synchronisation: fold the elapsed times into the counters
  static void collect(mlmc_ctx* c) {
    for (auto& p : pending()) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) c->prof.ms[p.stage] += ms;
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    pending().clear();
  }
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int level_batch_impl(mlmc_ctx* c, int level, int64_t first, int64_t n, uint64_t seed, double* qf,
                     double* qc, double* qcg, int32_t* iters, mlmc_level_sums* sums) {
  const mlmc_model& md = c->model;
  const int nc = n_coarse(md, level);
  const int64_t chunk = chunk_samples(c, level);
  if (int e = c->itacc.ensure(2 * sizeof(int64_t))) return e;
  if (int e = c->sums.ensure(256 + reduce_ws_bytes())) return e;  // sums at 0, partials at 256
  CUDA_TRY(cudaMemsetAsync(c->itacc.p, 0, 2 * sizeof(int64_t), c->st));
  const int m = md.m0 << level;
  const int M = c->lev[level].M;
  for (int64_t c0 = 0; c0 < n; c0 += chunk) {
    const int64_t cn = std::min<int64_t>(chunk, n - c0);
    SolveArgs a = base_args(c, level, seed, first + c0);
    if (md.k_kind == 1) {
      StageTimer t(c, 0);
      if (int e = run_fields(c, level, first + c0, cn, seed)) return e;
      t.stop(2 * (int)((cn + 65534) / 65535));
      a.g = c->g.p;
      if (c->prof_on) {
        c->prof.fft_row_points += (double)cn * n_pairs(md) * M * M;
        c->prof.fft_col_points += (double)cn * n_pairs(md) * M * m;
      }
    }
    {
      StageTimer t(c, 1);
      if (int e = run_solves(c, a, cn, nc, 0)) return e;
      t.stop(1);
    }
    StageTimer t(c, 2);
    if (gather_launch(c->qsys.as<double>(), c->itsys.as<int32_t>(), cn, nc, md.cgv, m, qf + c0,
                      qc + c0, qcg + c0, iters ? iters + c0 : nullptr, c->itacc.as<int64_t>(), c->st))
      return fail(MLMC_ERR_CUDA, "gather kernel");
    t.stop(1);
    if (c->prof_on) {
      c->prof.cells += (double)cn * ((double)m * m + nc * (double)(m / 2) * (m / 2));
      c->prof.samples += (double)cn;
    }
  }
  {
    StageTimer t(c, 2);
    if (reduce_launch(qf, qc, qcg, n, md.cgv != 0, c->itacc.as<int64_t>(), c->sums.as<LevelSumsDev>(),
                      c->sums.as<unsigned char>() + 256, c->st))
      return fail(MLMC_ERR_CUDA, "reduce kernel");
    t.stop(2);
  }
  LevelSumsDev h;
  int64_t itc[2];
  CUDA_TRY(cudaMemcpyAsync(&h, c->sums.p, sizeof(h), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(cudaMemcpyAsync(itc, c->itacc.p, sizeof(itc), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  if (c->prof_on) {
    StageTimer::collect(c);
    c->prof.cell_iters += (double)itc[1];
  }
  sums->n = h.n;
  sums->n_failed = h.n_failed;
  sums->iters_total = h.iters;
  double* dst[10] = {&sums->s_qf, &sums->s_qf2, &sums->s_qc, &sums->s_qc2, &sums->s_y,
                     &sums->s_y2, &sums->s_qcg, &sums->s_qcg2, &sums->s_yg, &sums->s_yg2};
  for (int k = 0; k < 10; ++k) *dst[k] = md.cgv || k < 6 ? h.s[k] : 0.0;
  return h.n_failed ? MLMC_SOME_FAILED : MLMC_OK;
}

int ensure_outputs(mlmc_ctx* c, int64_t n) {
  if (int e = c->oqf.ensure((size_t)n * 8)) return e;
  if (int e = c->oqc.ensure((size_t)n * 8)) return e;
  if (int e = c->oqg.ensure((size_t)n * 8)) return e;
  if (int e = c->oit.ensure((size_t)n * 4)) return e;
  return 0;
}

}  // namespace

extern "C" {

const char* mlmc_error_string(int code) {
  switch (code) {
    case MLMC_OK: return "success";
    case MLMC_SOME_FAILED: return "completed; some samples did not converge (Q = NaN, left out of the sums)";
    case MLMC_ERR_ARG: return "invalid argument";
    case MLMC_ERR_CUDA: return "CUDA runtime error";
    case MLMC_ERR_NOMEM: return "device allocation failed";
    case MLMC_ERR_EMBED: return "circulant embedding not non-negative up to padding 16";
    case MLMC_ERR_NODEV: return "no usable CUDA device";
    case MLMC_ERR_TOOBIG: return "size above the documented maximum";
    default: return "unknown error";
  }
}

const char* mlmc_last_error(void) { return g_last_error.c_str(); }

int mlmc_create(int device, const mlmc_model* model, void* cuda_stream, mlmc_ctx** out) {
  if (!out || !model) return fail(MLMC_ERR_ARG, "null argument");
  *out = nullptr;
  if (int e = check_model(*model)) return e;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(MLMC_ERR_NODEV, "no CUDA device");
  if (device < 0 || device >= ndev) return fail(MLMC_ERR_ARG, "device index out of range");
  CUDA_TRY(cudaSetDevice(device));
  mlmc_ctx* c = new mlmc_ctx();
  c->device = device;
  c->st = (cudaStream_t)cuda_stream;
  c->model = *model;
  cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device);
  c->lev.resize(model->L + 1);
  int err = 0;
  Buf scratch, mm;
  if ((err = c->bm.ensure(kSinCosTab * sizeof(double2) + 3 * kLogTab * sizeof(double))) == 0 &&
      bm_tables_build(c->bm.as<double2>(), reinterpret_cast<double*>(c->bm.as<double2>() + kSinCosTab),
                      c->st))
    err = fail(MLMC_ERR_CUDA, "Box-Muller table kernel");
  for (int l = 0; l <= model->L && !err; ++l) {
    LevelTable& T = c->lev[l];
    T.m = model->m0 << l;
    T.M = 0;
    if (model->k_kind != 1) continue;
    if ((err = mm.ensure(2 * sizeof(double)))) break;
    for (int p = 2; p <= 16; p *= 2) {
      const int M = p * T.m;
      if (M > 16384) {
        err = fail(MLMC_ERR_TOOBIG, "embedding size M above 16384");
        break;
      }
      if ((err = scratch.ensure((size_t)2 * M * M * 16))) break;
      if ((err = T.s64.ensure((size_t)M * M * 8)) || (err = T.s32.ensure((size_t)M * M * 4)) ||
          (err = T.tw64.ensure((size_t)M * 8)) || (err = T.tw32.ensure((size_t)M * 4)))
        break;
      if (ce_build_table(T.m, M, model->sigma2[0], model->lam[0], model->norm_r, scratch.p,
                         T.s64.as<double>(), T.s32.as<float>(), mm.as<double>(), T.tw64.p, T.tw32.p,
                         c->st)) {
        err = fail(MLMC_ERR_CUDA, "embedding set-up kernels");
        break;
      }
      double h[2];
      if (cudaMemcpyAsync(h, mm.p, sizeof(h), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
          cudaStreamSynchronize(c->st) != cudaSuccess) {
        err = fail(MLMC_ERR_CUDA, "embedding set-up copy");
        break;
      }
      T.lam_min = h[0];
      T.lam_max = h[1];
      if (h[0] >= -1e-13 * h[1]) {
        T.M = M;
        break;
      }
    }
    if (!err && T.M == 0) err = fail(MLMC_ERR_EMBED, "embedding negative at padding 16");
  }
  // layer pairs other than the first must have the same covariance as pair 0
  if (!err && model->k_kind == 1)
    for (int t = 1; t < model->n_layers; ++t)
      if (model->sigma2[t] != model->sigma2[0] || model->lam[t] != model->lam[0])
        err = fail(MLMC_ERR_ARG, "all layers must share sigma2 and lam (one embedding table per level)");
  scratch.release();
  mm.release();
  if (err) {
    mlmc_destroy(c);
    return err;
  }
  *out = c;
  return 0;
}

void mlmc_destroy(mlmc_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->st);
  for (auto& T : c->lev) {
    T.s64.release();
    T.s32.release();
    T.tw64.release();
    T.tw32.release();
  }
  for (Buf* b : {&c->W, &c->g, &c->ws, &c->qsys, &c->itsys, &c->oqf, &c->oqc, &c->oqg, &c->oit,
                 &c->sums, &c->itacc, &c->g64, &c->bm})
    b->release();
  delete c;
}

int mlmc_level_batch(mlmc_ctx* c, int level, int64_t first, int64_t n, uint64_t seed, double* qf,
                     double* qc, double* qc_cgv, int32_t* iters, mlmc_level_sums* sums) {
  if (!c || !sums) return fail(MLMC_ERR_ARG, "null context or sums");
  if (level < 0 || level > c->model.L) return fail(MLMC_ERR_ARG, "level out of range");
  if (n < 0 || first < 0) return fail(MLMC_ERR_ARG, "negative sample range");
  std::memset(sums, 0, sizeof(*sums));
  if (n == 0) return 0;
  const double t0 = now_s();
  CUDA_TRY(cudaSetDevice(c->device));
  if (!qf || !qc || !qc_cgv) {
    if (int e = ensure_outputs(c, n)) return e;
    if (!qf) qf = c->oqf.as<double>();
    if (!qc) qc = c->oqc.as<double>();
    if (!qc_cgv) qc_cgv = c->oqg.as<double>();
  }
  const int r = level_batch_impl(c, level, first, n, seed, qf, qc, qc_cgv, iters, sums);
  sums->seconds = now_s() - t0;
  return r;
}

int mlmc_level_batch_host(mlmc_ctx* c, int level, int64_t first, int64_t n, uint64_t seed, double* qf,
                          double* qc, double* qc_cgv, int32_t* iters, mlmc_level_sums* sums) {
  if (!c || !sums) return fail(MLMC_ERR_ARG, "null context or sums");
  if (n < 0 || first < 0) return fail(MLMC_ERR_ARG, "negative sample range");
  std::memset(sums, 0, sizeof(*sums));
  if (n == 0) return 0;
  const double t0 = now_s();
  CUDA_TRY(cudaSetDevice(c->device));
  if (int e = ensure_outputs(c, n)) return e;
  const int r = mlmc_level_batch(c, level, first, n, seed, c->oqf.as<double>(), c->oqc.as<double>(),
                                 c->oqg.as<double>(), iters ? c->oit.as<int32_t>() : nullptr, sums);
  if (r < 0) return r;
  if (qf) CUDA_TRY(cudaMemcpyAsync(qf, c->oqf.p, n * 8, cudaMemcpyDeviceToHost, c->st));
  if (qc) CUDA_TRY(cudaMemcpyAsync(qc, c->oqc.p, n * 8, cudaMemcpyDeviceToHost, c->st));
  if (qc_cgv) CUDA_TRY(cudaMemcpyAsync(qc_cgv, c->oqg.p, n * 8, cudaMemcpyDeviceToHost, c->st));
  if (iters) CUDA_TRY(cudaMemcpyAsync(iters, c->oit.p, n * 4, cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  sums->seconds = now_s() - t0;
  return r;
}

int mlmc_estimate(mlmc_ctx* c, double eps, uint64_t seed, int32_t n_pilot, int32_t cost_model,
                  mlmc_estimate_out* out) {
  if (!c || !out) return fail(MLMC_ERR_ARG, "null argument");
  if (!(eps > 0) || n_pilot < 2) return fail(MLMC_ERR_ARG, "eps must be > 0 and n_pilot >= 2");
  std::memset(out, 0, sizeof(*out));
  const double t0 = now_s();
  const mlmc_model& md = c->model;
  const int L = md.L;
  int rc_any = 0;
  std::vector<mlmc_level_sums> S(L + 1);
  std::vector<double> C(L + 1);
  for (int l = 0; l <= L; ++l) {
    int r = mlmc_level_batch(c, l, 0, n_pilot, seed, nullptr, nullptr, nullptr, nullptr, &S[l]);
    if (r < 0) return r;
    rc_any |= r;
    const double m2 = (double)(md.m0 << l) * (double)(md.m0 << l);
    C[l] = cost_model == 1 ? S[l].seconds / n_pilot : m2 * (1.0 + 0.25 * n_coarse(md, l));
  }
  auto stats = [&](int l, double* mean, double* var) {
    const bool g = md.cgv && l > 0;
    const double n = (double)S[l].n;
    const double s1 = g ? S[l].s_yg : S[l].s_y, s2 = g ? S[l].s_yg2 : S[l].s_y2;
    *mean = s1 / n;
    const double v = n > 1 ? (s2 - s1 * s1 / n) / (n - 1) : INFINITY;
    *var = v > 0 ? v : 0.0;
  };
  int rounds = 0;
  while (true) {
    std::vector<double> V(L + 1), mu(L + 1);
    for (int l = 0; l <= L; ++l) stats(l, &mu[l], &V[l]);
    double tot = 0;
    for (int l = 0; l <= L; ++l) tot += std::sqrt(V[l] * C[l]);
    bool any = false;
    std::vector<int64_t> todo(L + 1, 0);
    for (int l = 0; l <= L; ++l) {
      const double nopt = std::ceil(2.0 / (eps * eps) * std::sqrt(V[l] / C[l]) * tot);
      todo[l] = std::max<int64_t>(0, (int64_t)nopt - S[l].n);
      any |= todo[l] > 0;
    }
    if (!any || rounds >= 10) break;
    ++rounds;
    for (int l = 0; l <= L; ++l) {
      if (!todo[l]) continue;
      mlmc_level_sums add;
      const int64_t have = S[l].n + S[l].n_failed;
      int r = mlmc_level_batch(c, l, have, todo[l], seed, nullptr, nullptr, nullptr, nullptr, &add);
      if (r < 0) return r;
      rc_any |= r;
      S[l].n += add.n;
      S[l].n_failed += add.n_failed;
      S[l].iters_total += add.iters_total;
      S[l].seconds += add.seconds;
      double* a[10] = {&S[l].s_qf, &S[l].s_qf2, &S[l].s_qc, &S[l].s_qc2, &S[l].s_y,
                       &S[l].s_y2, &S[l].s_qcg, &S[l].s_qcg2, &S[l].s_yg, &S[l].s_yg2};
      const double* b[10] = {&add.s_qf, &add.s_qf2, &add.s_qc, &add.s_qc2, &add.s_y,
                             &add.s_y2, &add.s_qcg, &add.s_qcg2, &add.s_yg, &add.s_yg2};
      for (int k = 0; k < 10; ++k) *a[k] += *b[k];
    }
  }
  double qh = 0, vh = 0;
  for (int l = 0; l <= L; ++l) {
    double mean, var;
    stats(l, &mean, &var);
    out->N[l] = S[l].n;
    out->V[l] = var;
    out->mean[l] = mean;
    out->C[l] = C[l];
    out->sums[l] = S[l];
    qh += mean;
    vh += var / (double)S[l].n;
  }
  out->q_hat = qh;
  out->var_hat = vh;
  out->rounds = rounds;
  out->seconds = now_s() - t0;
  return rc_any ? MLMC_SOME_FAILED : MLMC_OK;
}

int mlmc_profile(mlmc_ctx* c, int enable) {
  if (!c) return fail(MLMC_ERR_ARG, "null context");
  if (enable) std::memset(&c->prof, 0, sizeof(c->prof));
  c->prof_on = enable != 0;
  return 0;
}

int mlmc_profile_read(mlmc_ctx* c, mlmc_profile_stats* out) {
  if (!c || !out) return fail(MLMC_ERR_ARG, "null argument");
  *out = c->prof;
  return 0;
}

int mlmc_ce_info(mlmc_ctx* c, int level, int32_t* M_out, double* lam_min, double* lam_max) {
  if (!c || level < 0 || level > c->model.L) return fail(MLMC_ERR_ARG, "bad context or level");
  if (M_out) *M_out = c->lev[level].M;
  if (lam_min) *lam_min = c->lev[level].lam_min;
  if (lam_max) *lam_max = c->lev[level].lam_max;
  return 0;
}

int mlmc_philox_words(uint64_t seed, uint64_t level, uint64_t sample, uint64_t stream,
                      uint64_t first_call, int64_t n_calls, uint64_t* out, void* cuda_stream) {
  if (n_calls < 0 || (n_calls > 0 && !out)) return fail(MLMC_ERR_ARG, "bad output");
  if (philox_launch(seed, level, sample, stream, first_call, n_calls, out, (cudaStream_t)cuda_stream))
    return fail(MLMC_ERR_CUDA, "philox kernel");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)cuda_stream));
  return 0;
}

int mlmc_normals(mlmc_ctx* c, uint64_t seed, uint64_t level, uint64_t sample, uint64_t stream,
                 uint64_t first_call, int64_t n_calls, double* out) {
  if (!c || n_calls < 0 || (n_calls > 0 && !out)) return fail(MLMC_ERR_ARG, "bad argument");
  CUDA_TRY(cudaSetDevice(c->device));
  if (normals_launch(seed, level, sample, stream, first_call, n_calls, c->bm.as<double2>(),
                     reinterpret_cast<const double*>(c->bm.as<double2>() + kSinCosTab), c->model.prec != 0,
                     out, c->st))
    return fail(MLMC_ERR_CUDA, "normals kernel");
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return 0;
}

int mlmc_sample_fields(mlmc_ctx* c, int level, int64_t first, int64_t n, uint64_t seed, double* g,
                       double* eta) {
  if (!c || !g || level < 0 || level > c->model.L || n < 0 || first < 0)
    return fail(MLMC_ERR_ARG, "bad argument");
  if (n == 0) return 0;
  CUDA_TRY(cudaSetDevice(c->device));
  const mlmc_model& md = c->model;
  const int m = md.m0 << level;
  SolveArgs a = base_args(c, level, seed, first);
  if (eta && interfaces_launch(a, n, eta, c->st)) return fail(MLMC_ERR_CUDA, "interfaces kernel");
  if (md.k_kind == 0) {
    if (const_fields_launch(a, n, g, c->st)) return fail(MLMC_ERR_CUDA, "fields kernel");
  } else {
    if (int e = run_fields(c, level, first, n, seed)) return e;
    const int64_t cnt = n * md.n_layers * (int64_t)m * m;
    if (md.prec)
      f32_to_f64_launch(c->g.as<float>(), g, cnt, c->st);
    else
      CUDA_TRY(cudaMemcpyAsync(g, c->g.p, cnt * 8, cudaMemcpyDeviceToDevice, c->st));
  }
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return 0;
}

int mlmc_solve_k(mlmc_ctx* c, int32_t m, int64_t n, const double* k, double* p, double* q,
                 int32_t* iters) {
  if (!c || !k || !q || n < 0) return fail(MLMC_ERR_ARG, "bad argument");
  if (!is_pow2(m) || m > 4096) return fail(MLMC_ERR_ARG, "m must be a power of two <= 4096");
  if (n == 0) return 0;
  CUDA_TRY(cudaSetDevice(c->device));
  SolveArgs a = base_args(c, 0, 0, 0);
  a.m = m;
  a.ksrc = KSRC_ARRAY;
  a.k = k;
  a.p_out = p;
  if (int e = run_solves(c, a, n, 0, n)) return e;
  CUDA_TRY(cudaMemcpyAsync(q, c->qsys.p, n * 8, cudaMemcpyDeviceToDevice, c->st));
  if (iters) CUDA_TRY(cudaMemcpyAsync(iters, c->itsys.p, n * 4, cudaMemcpyDeviceToDevice, c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return 0;
}

}  // extern "C"

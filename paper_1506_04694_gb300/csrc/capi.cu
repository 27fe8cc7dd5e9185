// C ABI of the MLMC level-batch library: context, level batches, the adaptive
// estimator and stage outputs.  Declarations and contracts: include/mlmc.h.
#include <algorithm>
#include <atomic>
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

// Bumped on every device (re)allocation: a kept CUDA graph is only valid
// while no buffer it points into has moved.
std::atomic<long long> g_alloc_generation{0};

struct Buf {
  void* p = nullptr;
  size_t cap = 0;
  int ensure(size_t bytes) {
    if (bytes <= cap) return 0;
    ++g_alloc_generation;
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

// Embedding table of one complex draw (pair) on one level.
struct PairTable {
  int M = 0;
  double lam_min = 0, lam_max = 0;
  Buf s64, s32, tw64, tw32;
};

struct LevelTable {
  int m = 0;
  std::vector<PairTable> pair;  // one per embedding draw
};

constexpr size_t kChunkBudget = size_t(2) << 30;  // bytes of per-sample buffers per chunk

// Work buffers of a chain of chunk launches: the embedding intermediate W,
// the fields g, the solver workspace ws and the per-system outputs.
struct WorkBufs {
  Buf W, g, ws, qsys, itsys;
  void release() {
    for (Buf* b : {&W, &g, &ws, &qsys, &itsys}) b->release();
  }
};

}  // namespace

namespace mlmc {
cudaError_t& last_launch_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}
int set_error(int code, const char* what) { return fail(code, what); }
}  // namespace mlmc

// A pair of events bracketing one stage (profiling).
struct StagePend {
  int stage, launches;
  cudaEvent_t a, b;
  int cls;  // >= 0: also the time of this profiled work-queue launch shape
};

// Device results of one enqueued level range, copied to pinned host memory.
struct HostLevel {
  LevelSumsDev s;
  int64_t itc[3];  // iterations; cells x iterations of the fine and of the coarse systems
};

struct mlmc_ctx {
  int device = 0;
  cudaStream_t st = nullptr;
  mlmc_model model{};

  int nsm = 0;
  std::vector<LevelTable> lev;
  // layers onto embedding draws: layer t is part part_of[t] (0 Re, 1 Im) of
  // draw pair_of[t]; draw f has covariance (pair_sigma2[f], pair_lam[f])
  int n_draws = 0;
  int pair_of[MLMC_MAX_LAYERS], part_of[MLMC_MAX_LAYERS];
  double pair_sigma2[MLMC_MAX_LAYERS], pair_lam[MLMC_MAX_LAYERS];
  Buf oqf, oqc, oqg, oit, sums, itacc, g64, bm;
  // work buffers and stream of the chain being queued: `misc` on the context
  // stream for single-level calls and set-up, a level's own set on its own
  // stream when the levels of a round run side by side
  WorkBufs misc;
  WorkBufs* wb = &misc;
  cudaStream_t wst = nullptr;
  cudaStream_t lst[MLMC_MAX_LEVELS] = {};
  cudaEvent_t lev_done[MLMC_MAX_LEVELS] = {};
  cudaEvent_t fork = nullptr;
  bool prof_on = false;
  mlmc_profile_stats prof{};
  // per-level slots of the multilevel batch (outputs, sums, iteration counters)
  struct Slot {
    Buf qf, qc, qg, it, sums, itacc;
    WorkBufs wb;
  } slot[MLMC_MAX_LEVELS];
  HostLevel* host = nullptr;  // pinned, MLMC_MAX_LEVELS + 1 entries (last: single-level calls)
  // launch plans chosen by mlmc_autotune() or set by hand, per level: for the
  // fine systems (or all of them), and for the coarse systems in a launch of
  // their own
  SolvePlan tuned[MLMC_MAX_LEVELS];
  bool tuned_ok[MLMC_MAX_LEVELS] = {};
  SolvePlan tuned_c[MLMC_MAX_LEVELS];
  bool tuned_c_ok[MLMC_MAX_LEVELS] = {};
  // estimator state: of the last estimate (for mlmc_checkpoint) and a loaded
  // one that the next estimate continues from (mlmc_resume)
  struct EstState {
    bool valid = false;
    double eps = 0;
    uint64_t seed = 0;
    int cost_model = 0, rounds = 0;
    std::vector<mlmc_level_sums> S;
    std::vector<double> C;
  } last_est, resume_est;
  // last captured multilevel graph and the arguments it was captured with
  cudaGraphExec_t gexec = nullptr;
  std::vector<int64_t> gkey;
  // work-queue schedule of the multilevel batch (mlmc_set_schedule): the
  // solves of all levels in one launch per launch shape ("class"), each on a
  // class stream of its own with its own workspace and work counter
  static constexpr int kClasses = 2 * MLMC_MAX_LEVELS;
  int sched = 1;
  // per-sample GPU cost of each level measured by mlmc_calibrate_costs (seconds)
  double cal_C[MLMC_MAX_LEVELS] = {};
  bool cal_ok = false;
  cudaStream_t cst[kClasses] = {};
  cudaEvent_t class_done[kClasses] = {}, fields_done[MLMC_MAX_LEVELS] = {};
  Buf sched_cnt, sched_ws[kClasses];
};

namespace {
// Queue the next chunk launches with these buffers on this stream (restored
// on scope exit).
struct UseBufs {
  mlmc_ctx* c;
  WorkBufs* wb0;
  cudaStream_t st0;
  UseBufs(mlmc_ctx* c_, WorkBufs* wb, cudaStream_t st) : c(c_), wb0(c_->wb), st0(c_->wst) {
    c->wb = wb;
    c->wst = st;
  }
  ~UseBufs() {
    c->wb = wb0;
    c->wst = st0;
  }
};
}  // namespace

namespace {

// Greedy pairing (same rule as the model documentation): layers in order,
// each joins an earlier draw of equal (sigma2, lam) whose Im part is free.
void pair_layers(mlmc_ctx* c) {
  const mlmc_model& md = c->model;
  int open_im[MLMC_MAX_LAYERS];
  int n_open = 0;
  c->n_draws = 0;
  for (int t = 0; t < md.n_layers; ++t) {
    int hit = -1;
    for (int k = 0; k < n_open; ++k) {
      const int f = open_im[k];
      if (c->pair_sigma2[f] == md.sigma2[t] && c->pair_lam[f] == md.lam[t]) {
        hit = k;
        break;
      }
    }
    if (hit >= 0) {
      c->pair_of[t] = open_im[hit];
      c->part_of[t] = 1;
      open_im[hit] = open_im[--n_open];
      // keep the remaining open draws in creation order
      for (int a = 0; a + 1 < n_open; ++a)
        for (int b = a + 1; b < n_open; ++b)
          if (open_im[b] < open_im[a]) std::swap(open_im[a], open_im[b]);
    } else {
      const int f = c->n_draws++;
      c->pair_sigma2[f] = md.sigma2[t];
      c->pair_lam[f] = md.lam[t];
      c->pair_of[t] = f;
      c->part_of[t] = 0;
      open_im[n_open++] = f;
    }
  }
}

int max_M(const mlmc_ctx* c, int level) {
  int M = 0;
  for (const auto& T : c->lev[level].pair) M = std::max(M, T.M);
  return M;
}
int dim_of(const mlmc_model& md) { return md.dim == 3 ? 3 : 2; }
// Cells of an m^d grid.
int64_t cells_of(const mlmc_model& md, int m) { return dim_of(md) == 3 ? (int64_t)m * m * m : (int64_t)m * m; }
int n_coarse(const mlmc_model& md, int level) { return level == 0 ? 0 : (md.cgv ? (dim_of(md) == 3 ? 8 : 4) : 1); }
// Solver plan / launch of the model's dimension.
int plan_of(const mlmc_model& md, int m, SolvePlan* P) {
  return dim_of(md) == 3 ? solve3_plan(m, md.prec, P) : solve_plan(m, md.prec, P);
}
bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int check_model(const mlmc_model& md) {
  if (md.n_layers < 1 || md.n_layers > MLMC_MAX_LAYERS) return fail(MLMC_ERR_ARG, "n_layers must be 1..8");
  if (md.k_kind != 0 && md.k_kind != 1) return fail(MLMC_ERR_ARG, "k_kind must be 0 or 1");
  if (md.norm_r != 1 && md.norm_r != 2) return fail(MLMC_ERR_ARG, "norm_r must be 1 or 2");
  if (!is_pow2(md.m0) || md.m0 < 2) return fail(MLMC_ERR_ARG, "m0 must be a power of two >= 2");
  if (md.L < 0 || md.L >= MLMC_MAX_LEVELS) return fail(MLMC_ERR_ARG, "L must be 0..11");
  if ((int64_t)md.m0 << md.L > 4096) return fail(MLMC_ERR_TOOBIG, "m0 * 2^L must be <= 4096");
  if (md.cgv < 0 || md.cgv > 2) return fail(MLMC_ERR_ARG, "cgv must be 0, 1 or 2");
  if (md.prec < 0 || md.prec > 3) return fail(MLMC_ERR_ARG, "prec must be 0, 1, 2 or 3");
  if (!(md.tol > 0) || md.max_it < 1) return fail(MLMC_ERR_ARG, "tol must be > 0 and max_it >= 1");
  if (!(md.if_hi >= md.if_lo)) return fail(MLMC_ERR_ARG, "if_hi must be >= if_lo");
  for (int t = 0; t < md.n_layers; ++t) {
    if (!(md.sigma2[t] >= 0)) return fail(MLMC_ERR_ARG, "sigma2 must be >= 0");
    if (md.k_kind == 1 && !(md.lam[t] > 0)) return fail(MLMC_ERR_ARG, "lam must be > 0");
  }
  if (md.problem != 0 && md.problem != 1 && md.problem != 2) return fail(MLMC_ERR_ARG, "problem must be 0, 1 or 2");
  if (md.problem == 1) {
    const double* b = md.qoi_box;
    const bool zero = b[0] == 0 && b[1] == 0 && b[2] == 0 && b[3] == 0;
    if (!zero && !(b[0] >= 0 && b[1] <= 1 && b[0] < b[1] && b[2] >= 0 && b[3] <= 1 && b[2] < b[3]))
      return fail(MLMC_ERR_ARG, "qoi_box must be x0 < x1, y0 < y1 inside [0, 1]");
  }
  if (md.geometry != 0 && md.geometry != 1) return fail(MLMC_ERR_ARG, "geometry must be 0 or 1");
  if (md.dim != 0 && md.dim != 2 && md.dim != 3) return fail(MLMC_ERR_ARG, "dim must be 0, 2 or 3");
  if (md.embed != 0 && md.embed != 1) return fail(MLMC_ERR_ARG, "embed must be 0 or 1");
  if (md.dim == 3) {
    if ((int64_t)md.m0 << md.L > 128) return fail(MLMC_ERR_TOOBIG, "3-D: m0 * 2^L must be <= 128");
    if (md.prec != 0 && md.prec != 1) return fail(MLMC_ERR_ARG, "3-D: prec must be 0 or 1");
  }
  if (md.geometry == 1) {
    if (md.n_layers != 3) return fail(MLMC_ERR_ARG, "geometry 1 has three layers");
    bool zero = true;
    for (int t = 0; t < 4; ++t) zero = zero && md.line_lo[t] == 0 && md.line_hi[t] == 0;
    for (int t = 0; t < 4 && !zero; ++t)
      if (!(md.line_lo[t] <= md.line_hi[t] && md.line_lo[t] >= 0 && md.line_hi[t] <= 1))
        return fail(MLMC_ERR_ARG, "line_lo[t] <= line_hi[t] inside [0, 1]");
  }
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
  a.geometry = md.geometry;
  a.if_lo = md.if_lo;
  a.if_hi = md.if_hi;
  {
    bool zero = true;
    for (int t = 0; t < 4; ++t) zero = zero && md.line_lo[t] == 0 && md.line_hi[t] == 0;
    const double lo[4] = {0.8, 0.6, 0.2, 0.4}, hi[4] = {0.9, 0.7, 0.3, 0.5};
    for (int t = 0; t < 4; ++t) {
      a.line_lo[t] = zero ? lo[t] : md.line_lo[t];
      a.line_hi[t] = zero ? hi[t] : md.line_hi[t];
    }
  }
  for (int t = 0; t < MAX_LAYERS_DEV; ++t) {
    a.mu[t] = md.mu[t];
    a.sigma[t] = std::sqrt(md.sigma2[t]);
  }
  a.ksrc = md.k_kind == 0 ? KSRC_CONST : KSRC_FIELDS;
  a.cgv_on_k = md.cgv == 2;
  a.tol = md.tol;
  a.max_it = md.max_it;
  a.problem = md.problem == 1 ? 1 : 2;
  const bool zero_box = md.qoi_box[0] == 0 && md.qoi_box[1] == 0 && md.qoi_box[2] == 0 && md.qoi_box[3] == 0;
  const double dflt[4] = {7.0 / 16, 9.0 / 16, 7.0 / 16, 9.0 / 16};
  for (int k = 0; k < 4; ++k) a.box[k] = zero_box ? dflt[k] : md.qoi_box[k];
  a.inner_tol = 1e-5;
  return a;
}

// prec 1 and 2 sample the fields in FP32; prec 0 and 3 in FP64.
static bool fields_f32(const mlmc_model& md) { return md.prec == 1 || md.prec == 2; }

// Fields of chunk samples [first, first + n) of `level` into the selected work
// buffers (c->wb), or into g_out when given.
int run_fields(mlmc_ctx* c, int level, int64_t first, int64_t n, uint64_t seed, void* g_out = nullptr,
               int* launches = nullptr) {
  const mlmc_model& md = c->model;
  const LevelTable& LT = c->lev[level];
  const bool f32 = fields_f32(md);
  WorkBufs& B = *c->wb;
  if (int e = B.W.ensure(ce_w_bytes_per_sample(LT.m, max_M(c, level), f32, dim_of(md)) * n)) return e;
  if (!g_out) {
    if (int e = B.g.ensure((size_t)n * md.n_layers * cells_of(md, LT.m) * (f32 ? 4 : 8))) return e;
    g_out = B.g.p;
  }
  for (int f = 0; f < c->n_draws; ++f) {  // one draw at a time, W reused
    const PairTable& T = LT.pair[f];
    CeLaunch L;
    L.bm_sc = c->bm.as<double2>();
    L.bm_lg = reinterpret_cast<const double*>(c->bm.as<double2>() + kSinCosTab);
    L.M = T.M;
    L.m = LT.m;
    L.dim = dim_of(md);
    L.pair = f;
    L.n_layers = md.n_layers;
    L.level = level;
    L.seed = seed;
    L.first = first;
    L.n_samples = n;
    L.t_re = L.t_im = -1;
    for (int t = 0; t < md.n_layers; ++t)
      if (c->pair_of[t] == f) (c->part_of[t] == 0 ? L.t_re : L.t_im) = t;
    L.mu_re = md.mu[L.t_re];
    L.mu_im = L.t_im >= 0 ? md.mu[L.t_im] : 0.0;
    int r;
    if (f32)
      r = ce_sample_fp32(L, T.s32.as<float>(), T.tw32.p, B.W.p, static_cast<float*>(g_out), c->wst);
    else
      r = ce_sample_fp64(L, T.s64.as<double>(), T.tw64.p, B.W.p, static_cast<double*>(g_out), c->wst);
    if (r) return fail(MLMC_ERR_CUDA, std::string("field kernels: ") + cudaGetErrorString(cudaGetLastError()));
  }
  const int nl = ce_launches_take();
  if (launches) *launches += nl;
  return 0;
}

int64_t chunk_samples(const mlmc_ctx* c, int level) {
  const mlmc_model& md = c->model;
  const int m = md.m0 << level;
  const bool f32 = fields_f32(md);
  size_t per = (size_t)(1 + n_coarse(md, level)) * 12;
  if (md.k_kind == 1) {
    per += ce_w_bytes_per_sample(m, max_M(c, level), f32, dim_of(md));
    per += (size_t)md.n_layers * cells_of(md, m) * (f32 ? 4 : 8);
  }
  int64_t s = (int64_t)(kChunkBudget / per);
  return std::max<int64_t>(1, std::min<int64_t>(s, 1 << 18));
}

// Bytes of global solver workspace a context may hold (bounds the number of
// resident blocks for very large grids).
constexpr size_t kWsBudget = size_t(16) << 30;

// Workspace bytes and blocks of one solver launch over n_sys systems.
struct LaunchSize {
  size_t ws;
  int64_t blocks;
};
LaunchSize launch_size(const mlmc_ctx* c, const SolvePlan& P, int64_t n_sys) {
  const int64_t cap = P.use_smem ? 0 : (int64_t)(kWsBudget / P.ws_stride);
  int64_t nb = 0;
  const int64_t groups = solve_groups(P, n_sys, c->nsm, cap, &nb);
  const size_t ws = !P.use_smem ? P.ws_stride * groups : P.ws64_stride * groups;
  return {ws, nb};
}

// Solve the systems of one chunk; results into the selected work buffers
// (qsys, itsys).  With a plan for the coarse systems (plan_c) the fine and the
// coarse systems run as two launches, each with its own plan, one after the
// other on the stream (sharing the workspace); which = 1 / 2 queues only the
// fine / only the coarse launch (autotuning).
int run_solves(mlmc_ctx* c, SolveArgs a, int64_t n_samples, int nc, int64_t max_rows,
               const SolvePlan* plan = nullptr, const SolvePlan* plan_c = nullptr, int which = 0) {
  const int prec = c->model.prec;
  a.n_samples = n_samples;
  a.n_coarse = nc;
  SolvePlan P;
  if (plan) P = *plan;
  else if (plan_of(c->model, a.m, &P)) return fail(MLMC_ERR_CUDA, "occupancy query failed");
  const int64_t n_sys = n_samples * (1 + nc);
  const bool split = plan_c && nc > 0;
  struct Part {
    const SolvePlan* P;
    int64_t b, e;
  } parts[2];
  int np = 0;
  if (!split) {
    parts[np++] = {&P, 0, n_sys};
  } else {
    if (which != 2) parts[np++] = {&P, 0, n_samples};
    if (which != 1) parts[np++] = {plan_c, n_samples, n_sys};
  }
  WorkBufs& B = *c->wb;
  size_t ws = 0;
  for (int k = 0; k < np; ++k) ws = std::max(ws, launch_size(c, *parts[k].P, parts[k].e - parts[k].b).ws);
  if (ws)
    if (int e = B.ws.ensure(ws)) return e;
  if (int e = B.qsys.ensure((size_t)std::max<int64_t>(n_sys, max_rows) * 8)) return e;
  if (int e = B.itsys.ensure((size_t)std::max<int64_t>(n_sys, max_rows) * 4)) return e;
  a.q = B.qsys.as<double>();
  a.iters = B.itsys.as<int32_t>();
  for (int k = 0; k < np; ++k) {
    const SolvePlan& Q = *parts[k].P;
    SolveArgs b = a;
    b.sys_begin = parts[k].b;
    b.sys_end = parts[k].e;
    b.ws = nullptr;
    b.ws64 = nullptr;
    if (!Q.use_smem) b.ws = B.ws.as<unsigned char>();
    else if (Q.ws64_stride) b.ws64 = B.ws.as<unsigned char>();
    const int64_t nb = launch_size(c, Q, parts[k].e - parts[k].b).blocks;
    const int lr = dim_of(c->model) == 3 ? solve3_launch(b, prec, Q, (int)nb, c->wst)
                                         : solve_launch(b, prec, Q, (int)nb, c->wst);
    if (lr) return fail(MLMC_ERR_CUDA, std::string("solve kernel launch: ") + cudaGetErrorString(last_launch_error()));
  }
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
    cudaEventRecord(e0, c->wst);
  }
  void stop(int launches, int cls = -1) {
    if (!c->prof_on) return;
    cudaEventRecord(e1, c->wst);
    pending().push_back({stage, launches, e0, e1, cls});
    e0 = e1 = nullptr;
  }
  static std::vector<StagePend>& pending() {
    static thread_local std::vector<StagePend> v;
    return v;
  }
  // after a stream synchronisation: fold elapsed times and launch counts into
  // the counters
  static void collect(mlmc_ctx* c) {
    for (auto& p : pending()) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        c->prof.ms[p.stage] += ms;
        if (p.cls >= 0) c->prof.class_ms[p.cls] += ms;
      }
      c->prof.launches[p.stage] += p.launches;
      if (p.cls >= 0) c->prof.class_launches[p.cls] += p.launches;
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    pending().clear();
  }
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Profiling counters of the field passes of n samples of `level`:
// transformed points, FFT flops and the algorithmic bytes.
void count_fields(mlmc_ctx* c, int level, int64_t n) {
  if (!c->prof_on) return;
  const mlmc_model& md = c->model;
  const int m = md.m0 << level;
  double sumM2 = 0, sumM = 0, fftf = 0, fftb = 0;  // transformed points, FFT flops and bytes per sample
  const bool d3 = dim_of(md) == 3;
  const double sc = fields_f32(md) ? 8.0 : 16.0;     // bytes of a complex intermediate value
  for (const auto& T : c->lev[level].pair) {
    const double Md = T.M;
    sumM2 += d3 ? Md * Md * Md : Md * Md;              // points of the row pass
    sumM += d3 ? Md * Md + Md * m : Md;                // (3-D: middle and last passes) / m
    fftf += 5.0 * std::log2(Md) * (d3 ? Md * Md * Md + Md * Md * m + Md * m * m : Md * Md + Md * m);
    // intermediates written once and read once (2-D: M x m; 3-D: M^2 m and M m^2)
    fftb += 2.0 * sc * (d3 ? Md * Md * m + Md * m * m : Md * m);
  }
  fftb += (double)md.n_layers * (double)cells_of(md, m) * (fields_f32(md) ? 4.0 : 8.0);  // fields written
  c->prof.fft_row_points += (double)n * sumM2;
  c->prof.fft_col_points += (double)n * sumM * m;
  c->prof.fft_flops += (double)n * fftf;
  c->prof.fft_bytes += (double)n * fftb;
}

// Queue samples first .. first+n-1 of `level` on the context stream: fields,
// solves and gathers chunk by chunk, then the level reduction into sums_dev
// (256 bytes of sums + the reduction partials) and an asynchronous copy of
// the sums and iteration counters into *host.  No host synchronisation.
int enqueue_level(mlmc_ctx* c, int level, int64_t first, int64_t n, uint64_t seed, double* qf, double* qc,
                  double* qcg, int32_t* iters, unsigned char* sums_dev, int64_t* itacc, HostLevel* host) {
  const mlmc_model& md = c->model;
  const int nc = n_coarse(md, level);
  const int64_t chunk = chunk_samples(c, level);
  const SolvePlan* plan = c->tuned_ok[level] ? &c->tuned[level] : nullptr;
  const SolvePlan* plan_c = c->tuned_c_ok[level] ? &c->tuned_c[level] : nullptr;
  CUDA_TRY(cudaMemsetAsync(itacc, 0, 3 * sizeof(int64_t), c->wst));
  const int m = md.m0 << level;
  for (int64_t c0 = 0; c0 < n; c0 += chunk) {
    const int64_t cn = std::min<int64_t>(chunk, n - c0);
    SolveArgs a = base_args(c, level, seed, first + c0);
    if (md.k_kind == 1) {
      StageTimer t(c, 0);
      int nlaunch = 0;
      if (int e = run_fields(c, level, first + c0, cn, seed, nullptr, &nlaunch)) return e;
      t.stop(nlaunch);
      a.g = c->wb->g.p;
      count_fields(c, level, cn);
    }
    if (plan_c && nc > 0) {  // the fine and the coarse systems, each timed as a stage of its own
      {
        StageTimer t(c, 1);
        if (int e = run_solves(c, a, cn, nc, 0, plan, plan_c, 1)) return e;
        t.stop(1);
      }
      StageTimer t(c, 3);
      if (int e = run_solves(c, a, cn, nc, 0, plan, plan_c, 2)) return e;
      t.stop(1);
    } else {
      StageTimer t(c, 1);
      if (int e = run_solves(c, a, cn, nc, 0, plan)) return e;
      t.stop(1);
    }
    StageTimer t(c, 2);
    if (gather_launch(c->wb->qsys.as<double>(), c->wb->itsys.as<int32_t>(), cn, nc, md.cgv, cells_of(md, m),
                      cells_of(md, m / 2), qf + c0,
                      qc + c0, qcg + c0, iters ? iters + c0 : nullptr, itacc, c->wst))
      return fail(MLMC_ERR_CUDA, "gather kernel");
    t.stop(1);
    if (c->prof_on) {
      c->prof.cells += (double)cn * ((double)cells_of(md, m) + nc * (double)cells_of(md, m / 2));
      c->prof.samples += (double)cn;
    }
  }
  {
    StageTimer t(c, 2);
    if (reduce_launch(qf, qc, qcg, n, md.cgv != 0, itacc, reinterpret_cast<LevelSumsDev*>(sums_dev),
                      sums_dev + 256, c->wst))
      return fail(MLMC_ERR_CUDA, "reduce kernel");
    t.stop(2);
  }
  CUDA_TRY(cudaMemcpyAsync(&host->s, sums_dev, sizeof(LevelSumsDev), cudaMemcpyDeviceToHost, c->wst));
  CUDA_TRY(cudaMemcpyAsync(host->itc, itacc, sizeof(host->itc), cudaMemcpyDeviceToHost, c->wst));
  return 0;
}

// Algorithmic flops per cell and CG iteration (FMA = 2): operator apply 9,
// p.q 2, x, r, r.r 6, r.z 2, p update 2; on the finest grid of the cycle a
// zero-guess red half sweep 0.5, black 4.5, every further sweep pair 9, the
// red-cell residual restriction 5.25, prolongation 1 and 9 per post-sweep
// pair; coarser grids (nuc sweep pairs) add 1/3 (V) or 1 (W) of that.  The
// flexible CG of prec 3 adds the dot product r_new.z_old (2).
// 3-D: operator apply 13, CG vectors 12; on the finest grid of the cycle the
// zero-guess red half sweep 0.5, black 6.5, every further sweep pair 13, the
// red-cell restriction 7.4, prolongation 1 and 13 per post-sweep pair;
// coarser grids add 1/7 (V) or 1/3 (W) of that.
double flops_per_cell_iter3(int gamma, int nu, int nuc) {
  const double fine = 2.4 + 26.0 * nu, coarse = 2.4 + 26.0 * (nuc > 0 ? nuc : nu);
  return 25.0 + fine + coarse * (gamma >= 2 ? 1.0 / 3.0 : 1.0 / 7.0);
}

double flops_per_cell_iter(int prec, int gamma, int nu, int nuc) {
  const double fine = 2.25 + 18.0 * nu, coarse = 2.25 + 18.0 * (nuc > 0 ? nuc : nu);
  return (prec == 3 ? 23.0 : 21.0) + fine + coarse * (gamma >= 2 ? 1.0 : 1.0 / 3.0);
}

// Algorithmic bytes per cell and CG iteration: every pass of the iteration
// reads each operand array once and writes each result once (no reuse
// between passes), with s = bytes of a cell value and fs of a face (about
// two faces per cell in 2-D, three in 3-D).  CG: operator apply (p, diag,
// faces read, q written), x and r updates (4 reads, 2 writes), r.z (2
// reads), p update (2 reads, 1 write): 14 s + 2 fs.  Multigrid, per cell of
// a level: zero-guess red half sweep 1.5 s (f, invd, e of one colour), black
// half sweep 2 s + 2 fs (plus the other colour's e and every face once),
// each further half sweep the same, red-cell restriction 2.25 s + 2 fs,
// prolongation 2.25 s: 6 s + 4 fs + (2 nu - 1)(4 s + 4 fs); coarser levels
// add 1/3 (V) or 1 (W) of that with their own sweep count.  3-D: CG 14 s +
// 3 fs; a level 5.75 s + 6 fs + (2 nu - 1)(4 s + 6 fs), coarser 1/7 (V) or
// 1/3 (W).  prec 1, 2, 3: the cycle in FP32 (prec 2: BF16 faces); the CG in
// FP32 for prec 1, 2, in FP64 for prec 0, 3.
double bytes_per_cell_iter(int prec, int dim, int gamma, int nu, int nuc) {
  const double s_cg = (prec == 1 || prec == 2) ? 4.0 : 8.0, fs_cg = s_cg;
  const double s_mg = prec == 0 ? 8.0 : 4.0, fs_mg = prec == 0 ? 8.0 : prec == 2 ? 2.0 : 4.0;
  const int nc = nuc > 0 ? nuc : nu;
  if (dim == 3) {
    auto lev = [&](int n) { return 5.75 * s_mg + 6.0 * fs_mg + (2.0 * n - 1.0) * (4.0 * s_mg + 6.0 * fs_mg); };
    return 14.0 * s_cg + 3.0 * fs_cg + lev(nu) + lev(nc) * (gamma >= 2 ? 1.0 / 3.0 : 1.0 / 7.0);
  }
  auto lev = [&](int n) { return 6.0 * s_mg + 4.0 * fs_mg + (2.0 * n - 1.0) * (4.0 * s_mg + 4.0 * fs_mg); };
  return 14.0 * s_cg + 2.0 * fs_cg + lev(nu) + lev(nc) * (gamma >= 2 ? 1.0 : 1.0 / 3.0);
}

// After the stream reached the copies of enqueue_level(): fill the sums.
int finish_level(mlmc_ctx* c, int level, const HostLevel& h, mlmc_level_sums* sums) {
  const mlmc_model& md = c->model;
  if (c->prof_on) {
    c->prof.cell_iters += (double)(h.itc[1] + h.itc[2]);
    SolvePlan P;
    if (c->tuned_ok[level]) P = c->tuned[level];
    else if (plan_of(md, md.m0 << level, &P)) P.gamma = P.nu = 1;
    const SolvePlan& Pc = c->tuned_c_ok[level] ? c->tuned_c[level] : P;  // the coarse systems' plan
    for (int part = 0; part < 2; ++part) {
      const SolvePlan& Q = part ? Pc : P;
      const double ci = (double)h.itc[1 + part];
      const double fl = ci * (dim_of(md) == 3 ? flops_per_cell_iter3(Q.gamma, Q.nu, Q.nu_coarse)
                                              : flops_per_cell_iter(md.prec, Q.gamma, Q.nu, Q.nu_coarse));
      const double by = ci * bytes_per_cell_iter(md.prec, dim_of(md), Q.gamma, Q.nu, Q.nu_coarse);
      c->prof.solve_flops += fl;
      c->prof.solve_bytes += by;
      if (part == 1) {
        c->prof.cell_iters_c += ci;
        c->prof.solve_flops_c += fl;
        c->prof.solve_bytes_c += by;
      }
    }
  }
  sums->n = h.s.n;
  sums->n_failed = h.s.n_failed;
  sums->iters_total = h.s.iters;
  double* dst[10] = {&sums->s_qf, &sums->s_qf2, &sums->s_qc, &sums->s_qc2, &sums->s_y,
                     &sums->s_y2, &sums->s_qcg, &sums->s_qcg2, &sums->s_yg, &sums->s_yg2};
  for (int k = 0; k < 10; ++k) *dst[k] = md.cgv || k < 6 ? h.s.s[k] : 0.0;
  return h.s.n_failed ? MLMC_SOME_FAILED : MLMC_OK;
}

int level_batch_impl(mlmc_ctx* c, int level, int64_t first, int64_t n, uint64_t seed, double* qf,
                     double* qc, double* qcg, int32_t* iters, mlmc_level_sums* sums) {
  if (int e = c->itacc.ensure(3 * sizeof(int64_t))) return e;
  if (int e = c->sums.ensure(256 + reduce_ws_bytes())) return e;  // sums at 0, partials at 256
  HostLevel* h = c->host + MLMC_MAX_LEVELS;
  if (int e = enqueue_level(c, level, first, n, seed, qf, qc, qcg, iters, c->sums.as<unsigned char>(),
                            c->itacc.as<int64_t>(), h))
    return e;
  CUDA_TRY(cudaStreamSynchronize(c->st));
  if (c->prof_on) StageTimer::collect(c);
  return finish_level(c, level, *h, sums);
}

// Allocate, outside any stream capture, every buffer a range of n samples of
// `level` will touch.
int prepare_level(mlmc_ctx* c, int level, int64_t n, bool want_iters = false) {
  const mlmc_model& md = c->model;
  const int m = md.m0 << level;
  const bool f32 = fields_f32(md);
  const int nc = n_coarse(md, level);
  const int64_t cn = std::min<int64_t>(n, chunk_samples(c, level));
  WorkBufs& B = c->slot[level].wb;
  if (md.k_kind == 1) {
    if (int e = B.W.ensure(ce_w_bytes_per_sample(m, max_M(c, level), f32, dim_of(md)) * cn)) return e;
    if (int e = B.g.ensure((size_t)cn * md.n_layers * cells_of(md, m) * (f32 ? 4 : 8))) return e;
  }
  SolvePlan P;
  if (c->tuned_ok[level]) P = c->tuned[level];
  else if (plan_of(md, m, &P)) return fail(MLMC_ERR_CUDA, "occupancy query failed");
  const int64_t n_sys = cn * (1 + nc);
  size_t ws = 0;
  if (c->tuned_c_ok[level] && nc > 0)
    ws = std::max(launch_size(c, P, cn).ws, launch_size(c, c->tuned_c[level], cn * nc).ws);
  else
    ws = launch_size(c, P, n_sys).ws;
  if (ws)
    if (int e = B.ws.ensure(ws)) return e;
  if (int e = B.qsys.ensure((size_t)n_sys * 8)) return e;
  if (int e = B.itsys.ensure((size_t)n_sys * 4)) return e;
  auto& S = c->slot[level];
  if (int e = S.qf.ensure((size_t)n * 8)) return e;
  if (int e = S.qc.ensure((size_t)n * 8)) return e;
  if (int e = S.qg.ensure((size_t)n * 8)) return e;
  if (want_iters)
    if (int e = S.it.ensure((size_t)n * 4)) return e;
  if (int e = S.sums.ensure(256 + reduce_ws_bytes())) return e;
  if (int e = S.itacc.ensure(3 * sizeof(int64_t))) return e;
  return 0;
}

// ---- work-queue schedule: one solver launch per launch shape across levels ----

// One range of a level's systems with the plan that solves it.
struct SchedPart {
  int level;
  int64_t b, e;  // systems [b, e) of the level
  int msys;      // cells per side of the range's first system
  SolvePlan P;
};

// The parts that share a launch shape, largest systems first, and the plan
// their launch takes (workspace strides of the largest part).
struct SchedClass {
  SolvePlan P;
  std::vector<SchedPart> parts;
  int64_t n_sys = 0;
};

// Plans that launch the same kernel with the same block, cluster, shared
// memory and residency can share a launch.
bool same_shape(const SolvePlan& a, const SolvePlan& b) {
  return a.warp == b.warp && a.cluster == b.cluster && a.threads == b.threads && a.use_smem == b.use_smem &&
         a.groups_per_block == b.groups_per_block && a.smem_bytes == b.smem_bytes &&
         a.cap_blocks_per_sm == b.cap_blocks_per_sm;
}

// The classes of a multilevel batch of n[l] samples per level.
int sched_classes(const mlmc_ctx* c, int n_levels, const int64_t* n, std::vector<SchedClass>& out) {
  const mlmc_model& md = c->model;
  out.clear();
  for (int l = 0; l < n_levels; ++l) {
    if (n[l] <= 0) continue;
    const int m = md.m0 << l, nc = n_coarse(md, l);
    SolvePlan P;
    if (c->tuned_ok[l]) P = c->tuned[l];
    else if (plan_of(md, m, &P)) return fail(MLMC_ERR_CUDA, "occupancy query failed");
    SchedPart parts[2];
    int np = 0;
    if (c->tuned_c_ok[l] && nc > 0) {
      parts[np++] = {l, 0, n[l], m, P};
      parts[np++] = {l, n[l], n[l] * (1 + nc), m / 2, c->tuned_c[l]};
    } else {
      parts[np++] = {l, 0, n[l] * (1 + nc), m, P};
    }
    for (int k = 0; k < np; ++k) {
      SchedClass* C = nullptr;
      for (auto& x : out)
        if (same_shape(x.P, parts[k].P)) C = &x;
      if (!C) {
        if ((int)out.size() == mlmc_ctx::kClasses) return fail(MLMC_ERR_ARG, "too many launch shapes");
        out.emplace_back();
        C = &out.back();
        C->P = parts[k].P;
      }
      C->parts.push_back(parts[k]);
      C->n_sys += parts[k].e - parts[k].b;
      C->P.ws_stride = std::max(C->P.ws_stride, parts[k].P.ws_stride);
      C->P.ws64_stride = std::max(C->P.ws64_stride, parts[k].P.ws64_stride);
      C->P.stage_bytes = std::max(C->P.stage_bytes, parts[k].P.stage_bytes);
    }
  }
  for (auto& C : out)
    std::stable_sort(C.parts.begin(), C.parts.end(),
                     [](const SchedPart& x, const SchedPart& y) { return x.msys > y.msys; });
  return 0;
}

constexpr size_t kSchedBudget = size_t(24) << 30;  // bytes of whole-level fields and outputs

// Whether this multilevel batch takes the work-queue schedule: 2-D, FP64 or
// FP32-multigrid precision, and the fields of every level's whole range
// within kSchedBudget.
bool sched_usable(const mlmc_ctx* c, int n_levels, const int64_t* n) {
  const mlmc_model& md = c->model;
  if (!c->sched || dim_of(md) == 3 || (md.prec != 0 && md.prec != 1)) return false;
  double bytes = 0;
  for (int l = 0; l < n_levels; ++l) {
    if (n[l] <= 0) continue;
    const int m = md.m0 << l;
    bytes += (double)n[l] * (1 + n_coarse(md, l)) * 12.0;
    if (md.k_kind == 1) bytes += (double)n[l] * md.n_layers * cells_of(md, m) * (fields_f32(md) ? 4.0 : 8.0);
  }
  return bytes <= (double)kSchedBudget;
}

// Allocate, outside any stream capture, what the work-queue schedule of this
// batch touches: per level one chunk of embedding intermediates, the fields
// and the per-system outputs of the whole range, the level's results; per
// class a workspace and a work counter, a stream and an event.
int prepare_sched(mlmc_ctx* c, int n_levels, const int64_t* n, const std::vector<SchedClass>& cls,
                  bool want_iters) {
  const mlmc_model& md = c->model;
  const bool f32 = fields_f32(md);
  for (int l = 0; l < n_levels; ++l) {
    if (n[l] <= 0) continue;
    const int m = md.m0 << l;
    const int64_t n_sys = n[l] * (1 + n_coarse(md, l));
    auto& S = c->slot[l];
    WorkBufs& B = S.wb;
    if (md.k_kind == 1) {
      const int64_t cn = std::min<int64_t>(n[l], chunk_samples(c, l));
      if (int e = B.W.ensure(ce_w_bytes_per_sample(m, max_M(c, l), f32, dim_of(md)) * cn)) return e;
      if (int e = B.g.ensure((size_t)n[l] * md.n_layers * cells_of(md, m) * (f32 ? 4 : 8))) return e;
    }
    if (int e = B.qsys.ensure((size_t)n_sys * 8)) return e;
    if (int e = B.itsys.ensure((size_t)n_sys * 4)) return e;
    if (int e = S.qf.ensure((size_t)n[l] * 8)) return e;
    if (int e = S.qc.ensure((size_t)n[l] * 8)) return e;
    if (int e = S.qg.ensure((size_t)n[l] * 8)) return e;
    if (want_iters)
      if (int e = S.it.ensure((size_t)n[l] * 4)) return e;
    if (int e = S.sums.ensure(256 + reduce_ws_bytes())) return e;
    if (int e = S.itacc.ensure(3 * sizeof(int64_t))) return e;
    if (!c->fields_done[l] && cudaEventCreateWithFlags(&c->fields_done[l], cudaEventDisableTiming) != cudaSuccess)
      return fail(MLMC_ERR_CUDA, "event");
  }
  if (int e = c->sched_cnt.ensure(mlmc_ctx::kClasses * sizeof(unsigned long long))) return e;
  if (solve_list_prepare())
    return fail(MLMC_ERR_CUDA, std::string("list kernel attributes: ") + cudaGetErrorString(last_launch_error()));
  for (size_t k = 0; k < cls.size(); ++k) {
    const size_t ws = launch_size(c, cls[k].P, cls[k].n_sys).ws;
    if (ws)
      if (int e = c->sched_ws[k].ensure(ws)) return e;
    if (!c->cst[k] && cudaStreamCreateWithFlags(&c->cst[k], cudaStreamNonBlocking) != cudaSuccess)
      return fail(MLMC_ERR_CUDA, "class stream");
    if (!c->class_done[k] && cudaEventCreateWithFlags(&c->class_done[k], cudaEventDisableTiming) != cudaSuccess)
      return fail(MLMC_ERR_CUDA, "event");
  }
  return 0;
}

// Queue a multilevel batch in the work-queue schedule: (A) each level's
// fields, chunk by chunk, on its level stream; (B) per class, after the
// fields of its levels, one persistent solver launch over all its parts
// (further launches only past kMaxSolveItems parts); (C) per level, after
// its classes, the gather, the level reduction and the copy of its sums to
// host memory, joined into the context stream.  With `serial` the three
// phases run in this order on the context stream.
int enqueue_sched(mlmc_ctx* c, int n_levels, const int64_t* first, const int64_t* n, uint64_t seed,
                  const std::vector<SchedClass>& cls, int* prof_cls, bool serial, bool want_iters) {
  const mlmc_model& md = c->model;
  const bool f32 = fields_f32(md);
  // serial: everything in order on the context stream (events and waits then
  // order nothing): with stage profiling on (each launch's event time its
  // own) and under graph capture (measured on GB300: a graph of the side-by-side
  // form ran the headline estimate in 636 ms, the same launches as one chain
  // in 615 ms, direct side-by-side launches in 610 ms)
  if (cudaEventRecord(c->fork, c->st) != cudaSuccess) return fail(MLMC_ERR_CUDA, "fork event");
  for (int l = 0; l < n_levels; ++l) {
    if (n[l] <= 0) continue;
    auto& S = c->slot[l];
    const cudaStream_t ls = serial ? c->st : c->lst[l];
    if (cudaStreamWaitEvent(ls, c->fork, 0) != cudaSuccess) return fail(MLMC_ERR_CUDA, "fork wait");
    UseBufs use(c, &S.wb, ls);
    CUDA_TRY(cudaMemsetAsync(S.itacc.p, 0, 3 * sizeof(int64_t), ls));
    if (md.k_kind == 1) {
      const int m = md.m0 << l;
      const size_t gps = (size_t)md.n_layers * cells_of(md, m) * (f32 ? 4 : 8);
      const int64_t chunk = chunk_samples(c, l);
      for (int64_t c0 = 0; c0 < n[l]; c0 += chunk) {
        const int64_t cn = std::min<int64_t>(chunk, n[l] - c0);
        StageTimer t(c, 0);
        int nlaunch = 0;
        if (int e = run_fields(c, l, first[l] + c0, cn, seed, S.wb.g.as<unsigned char>() + (size_t)c0 * gps,
                               &nlaunch))
          return e;
        t.stop(nlaunch);
        count_fields(c, l, cn);
      }
    }
    CUDA_TRY(cudaEventRecord(c->fields_done[l], ls));
  }
  unsigned long long* cnt = c->sched_cnt.as<unsigned long long>();
  for (size_t k = 0; k < cls.size(); ++k) {
    const SchedClass& C = cls[k];
    const cudaStream_t cs = serial ? c->st : c->cst[k];
    UseBufs use(c, c->wb, cs);
    bool waited[MLMC_MAX_LEVELS] = {};
    for (const auto& p : C.parts)
      if (!waited[p.level]) {
        CUDA_TRY(cudaStreamWaitEvent(cs, c->fields_done[p.level], 0));
        waited[p.level] = true;
      }
    for (size_t p0 = 0; p0 < C.parts.size(); p0 += kMaxSolveItems) {
      SolveList L;
      std::memset(&L, 0, sizeof(L));
      L.next = cnt + k;
      int64_t total = 0;
      for (size_t i = p0; i < C.parts.size() && L.n < kMaxSolveItems; ++i) {
        const SchedPart& q = C.parts[i];
        const auto& S = c->slot[q.level];
        SolveArgs a = base_args(c, q.level, seed, first[q.level]);
        a.n_samples = n[q.level];
        a.n_coarse = n_coarse(md, q.level);
        if (md.k_kind == 1) a.g = S.wb.g.p;
        a.q = S.wb.qsys.as<double>();
        a.iters = S.wb.itsys.as<int32_t>();
        a.sys_begin = q.b;
        a.sys_end = q.e;
        solve_apply_plan(a, q.P);
        a.ws_stride = C.P.ws_stride;
        a.ws64_stride = C.P.ws64_stride;
        a.ws = !C.P.use_smem ? c->sched_ws[k].as<unsigned char>() : nullptr;
        a.ws64 = C.P.use_smem && C.P.ws64_stride ? c->sched_ws[k].as<unsigned char>() : nullptr;
        L.start[L.n] = total;
        L.a[L.n++] = a;
        total += q.e - q.b;
      }
      L.start[L.n] = total;
      CUDA_TRY(cudaMemsetAsync(cnt + k, 0, sizeof(unsigned long long), cs));
      const int64_t nb = launch_size(c, C.P, total).blocks;
      StageTimer t(c, 1);
      if (solve_launch_list(L, md.prec, C.P, (int)nb, cs))
        return fail(MLMC_ERR_CUDA, std::string("solve list launch: ") + cudaGetErrorString(last_launch_error()));
      t.stop(1, prof_cls ? prof_cls[k] : -1);
    }
    CUDA_TRY(cudaEventRecord(c->class_done[k], cs));
  }
  for (int l = 0; l < n_levels; ++l) {
    if (n[l] <= 0) continue;
    auto& S = c->slot[l];
    const cudaStream_t ls = serial ? c->st : c->lst[l];
    UseBufs use(c, &S.wb, ls);
    for (size_t k = 0; k < cls.size(); ++k) {
      bool has = false;
      for (const auto& p : cls[k].parts) has = has || p.level == l;
      if (has) CUDA_TRY(cudaStreamWaitEvent(ls, c->class_done[k], 0));
    }
    const int m = md.m0 << l;
    const int nc = n_coarse(md, l);
    double* qf = S.qf.as<double>();
    double* qc = S.qc.as<double>();
    double* qg = S.qg.as<double>();
    int64_t* itacc = S.itacc.as<int64_t>();
    StageTimer t(c, 2);
    if (gather_launch(S.wb.qsys.as<double>(), S.wb.itsys.as<int32_t>(), n[l], nc, md.cgv, cells_of(md, m),
                      cells_of(md, m / 2), qf, qc, qg, want_iters ? S.it.as<int32_t>() : nullptr, itacc, ls))
      return fail(MLMC_ERR_CUDA, "gather kernel");
    unsigned char* sums_dev = S.sums.as<unsigned char>();
    if (reduce_launch(qf, qc, qg, n[l], md.cgv != 0, itacc, reinterpret_cast<LevelSumsDev*>(sums_dev),
                      sums_dev + 256, ls))
      return fail(MLMC_ERR_CUDA, "reduce kernel");
    t.stop(3);
    if (c->prof_on) {
      c->prof.cells += (double)n[l] * ((double)cells_of(md, m) + nc * (double)cells_of(md, m / 2));
      c->prof.samples += (double)n[l];
    }
    CUDA_TRY(cudaMemcpyAsync(&c->host[l].s, sums_dev, sizeof(LevelSumsDev), cudaMemcpyDeviceToHost, ls));
    CUDA_TRY(cudaMemcpyAsync(c->host[l].itc, itacc, sizeof(c->host[l].itc), cudaMemcpyDeviceToHost, ls));
    CUDA_TRY(cudaEventRecord(c->lev_done[l], ls));
    CUDA_TRY(cudaStreamWaitEvent(c->st, c->lev_done[l], 0));
  }
  return 0;
}

// All levels' ranges queued back to back with one host synchronisation;
// with use_graph the queue is captured once into a CUDA graph (kept for the
// next call with the same arguments) and launched as one graph.
int multilevel_impl(mlmc_ctx* c, int n_levels, const int64_t* first, const int64_t* n, uint64_t seed,
                    bool use_graph, mlmc_level_sums* sums, bool want_iters = false) {
  std::vector<SchedClass> cls;
  const bool sched = sched_usable(c, n_levels, n);
  if (sched) {
    if (int e = sched_classes(c, n_levels, n, cls)) return e;
    if (int e = prepare_sched(c, n_levels, n, cls, want_iters)) return e;
  } else {
    for (int l = 0; l < n_levels; ++l)
      if (n[l] > 0)
        if (int e = prepare_level(c, l, n[l], want_iters)) return e;
  }
  // the levels run side by side, each on its own stream with its own work
  // buffers, forked from and joined back into the context stream; with
  // stage profiling on they run one after another on the context stream, so
  // that every stage's CUDA-event time is its own
  const bool side_by_side = !c->prof_on;
  // stage timing needs events between the launches, so profiling runs ungraphed
  const bool graph = use_graph && c->st != nullptr && !c->prof_on;
  // profiled work-queue launches: their launch shape's slot in the counters
  int prof_cls[mlmc_ctx::kClasses];
  for (size_t k = 0; k < cls.size(); ++k) {
    prof_cls[k] = -1;
    if (!c->prof_on) continue;
    const SolvePlan& P = cls[k].P;
    const int mode = P.cluster ? 2 : P.warp == 2 ? 3 : P.warp ? 1 : 0;
    mlmc_profile_stats& S = c->prof;
    for (int j = 0; j < S.n_classes; ++j)
      if (S.class_mode[j] == mode && S.class_threads[j] == P.threads && S.class_cluster[j] == P.cluster &&
          S.class_smem[j] == P.use_smem)
        prof_cls[k] = j;
    if (prof_cls[k] < 0 && S.n_classes < MLMC_PROFILE_CLASSES) {
      const int j = S.n_classes++;
      S.class_mode[j] = mode;
      S.class_threads[j] = P.threads;
      S.class_cluster[j] = P.cluster;
      S.class_smem[j] = P.use_smem;
      prof_cls[k] = j;
    }
  }
  auto enqueue_all = [&]() -> int {
    if (sched) return enqueue_sched(c, n_levels, first, n, seed, cls, prof_cls, c->prof_on || graph, want_iters);
    if (side_by_side && cudaEventRecord(c->fork, c->st) != cudaSuccess) return fail(MLMC_ERR_CUDA, "fork event");
    for (int l = 0; l < n_levels; ++l) {
      if (n[l] <= 0) continue;
      auto& S = c->slot[l];
      const cudaStream_t ls = side_by_side ? c->lst[l] : c->st;
      if (side_by_side && cudaStreamWaitEvent(ls, c->fork, 0) != cudaSuccess) return fail(MLMC_ERR_CUDA, "fork wait");
      {
        UseBufs use(c, &S.wb, ls);
        if (int e = enqueue_level(c, l, first[l], n[l], seed, S.qf.as<double>(), S.qc.as<double>(),
                                  S.qg.as<double>(), want_iters ? S.it.as<int32_t>() : nullptr,
                                  S.sums.as<unsigned char>(), S.itacc.as<int64_t>(), c->host + l))
          return e;
      }
      if (side_by_side && (cudaEventRecord(c->lev_done[l], ls) != cudaSuccess ||
                           cudaStreamWaitEvent(c->st, c->lev_done[l], 0) != cudaSuccess))
        return fail(MLMC_ERR_CUDA, "join event");
    }
    return 0;
  };
  if (graph) {
    std::vector<int64_t> key = {(int64_t)n_levels, (int64_t)seed, (int64_t)g_alloc_generation.load(),
                                (int64_t)sched, (int64_t)want_iters};
    for (int l = 0; l < n_levels; ++l) {
      key.push_back(c->tuned_ok[l] ? ((int64_t)c->tuned[l].nu << 28) + ((int64_t)c->tuned[l].gamma << 24) +
                                         ((int64_t)c->tuned[l].threads << 16) +
                                         (c->tuned[l].cluster << 8) + (c->tuned[l].warp << 4) +
                                         c->tuned[l].cap_blocks_per_sm
                                   : -1);
      int64_t tol_bits = 0;
      if (c->tuned_ok[l]) std::memcpy(&tol_bits, &c->tuned[l].inner_tol, sizeof tol_bits);
      key.push_back(tol_bits);
      key.push_back(c->tuned_ok[l] ? c->tuned[l].nu_coarse : -1);
      key.push_back(c->tuned_ok[l] ? c->tuned[l].reliable : -1);
      if (c->tuned_c_ok[l]) {
        const SolvePlan& Q = c->tuned_c[l];
        key.push_back(((int64_t)Q.nu << 28) + ((int64_t)Q.gamma << 24) + ((int64_t)Q.threads << 16) +
                      (Q.cluster << 8) + (Q.warp << 4) + Q.cap_blocks_per_sm);
        int64_t tb = 0;
        std::memcpy(&tb, &Q.inner_tol, sizeof tb);
        key.push_back(tb);
        key.push_back(((int64_t)Q.nu_coarse << 8) + Q.reliable);
      } else {
        key.push_back(-2);
      }
    }
    for (int l = 0; l < n_levels; ++l) {
      key.push_back(first[l]);
      key.push_back(n[l]);
    }
    if (!c->gexec || key != c->gkey) {
      if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
      }
      CUDA_TRY(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeRelaxed));
      const int e = enqueue_all();
      cudaGraph_t gr = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(c->st, &gr);
      if (e) {
        if (gr) cudaGraphDestroy(gr);
        return e;
      }
      if (ce != cudaSuccess) return fail(MLMC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
      const cudaError_t ie = cudaGraphInstantiate(&c->gexec, gr, 0);
      cudaGraphDestroy(gr);
      if (ie != cudaSuccess) {
        c->gexec = nullptr;
        return fail(MLMC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
      }
      c->gkey = key;
    }
    CUDA_TRY(cudaGraphLaunch(c->gexec, c->st));
    CUDA_TRY(cudaStreamSynchronize(c->st));
  } else {
    if (int e = enqueue_all()) return e;
    CUDA_TRY(cudaStreamSynchronize(c->st));
    if (c->prof_on) StageTimer::collect(c);
  }
  if (sched && c->prof_on)  // the work of each profiled work-queue launch shape
    for (size_t k = 0; k < cls.size(); ++k) {
      const int j = prof_cls[k];
      if (j < 0) continue;
      for (const SchedPart& q : cls[k].parts) {
        const HostLevel& h = c->host[q.level];
        const double ci = (double)(q.b == 0 ? h.itc[1] : 0) + (double)(q.e > n[q.level] ? h.itc[2] : 0);
        c->prof.class_levels[j] |= 1 << q.level;
        c->prof.class_cell_iters[j] += ci;
        c->prof.class_flops[j] += ci * flops_per_cell_iter(c->model.prec, q.P.gamma, q.P.nu, q.P.nu_coarse);
        c->prof.class_bytes[j] += ci * bytes_per_cell_iter(c->model.prec, 2, q.P.gamma, q.P.nu, q.P.nu_coarse);
      }
    }
  int rc = MLMC_OK;
  for (int l = 0; l < n_levels; ++l) {
    std::memset(&sums[l], 0, sizeof(sums[l]));
    if (n[l] > 0) rc |= finish_level(c, l, c->host[l], &sums[l]);
  }
  return rc;
}

void add_sums(mlmc_level_sums& S, const mlmc_level_sums& add) {
  S.n += add.n;
  S.n_failed += add.n_failed;
  S.iters_total += add.iters_total;
  S.seconds += add.seconds;
  double* a[10] = {&S.s_qf, &S.s_qf2, &S.s_qc, &S.s_qc2, &S.s_y, &S.s_y2, &S.s_qcg, &S.s_qcg2, &S.s_yg, &S.s_yg2};
  const double* b[10] = {&add.s_qf, &add.s_qf2, &add.s_qc, &add.s_qc2, &add.s_y,
                         &add.s_y2, &add.s_qcg, &add.s_qcg2, &add.s_yg, &add.s_yg2};
  for (int k = 0; k < 10; ++k) *a[k] += *b[k];
}

// The model block of a checkpoint: every field of mlmc_model that changes a
// sample's Q (or which samples fail), doubles at 17 significant digits.
void write_model_block(FILE* f, const mlmc_model& md) {
  std::fprintf(f, "model %d %d %d %d %d %d %d %d %d %d %d %d\n", md.n_layers, md.k_kind, md.norm_r, md.m0, md.L,
               md.cgv, md.prec, md.max_it, md.problem, md.geometry, dim_of(md), md.embed);
  std::fprintf(f, "model_if %.17g %.17g\nmodel_tol %.17g\n", md.if_lo, md.if_hi, md.tol);
  auto arr = [&](const char* key, const double* v, int n) {
    std::fprintf(f, "%s", key);
    for (int k = 0; k < n; ++k) std::fprintf(f, " %.17g", v[k]);
    std::fprintf(f, "\n");
  };
  arr("model_mu", md.mu, MLMC_MAX_LAYERS);
  arr("model_sigma2", md.sigma2, MLMC_MAX_LAYERS);
  arr("model_lam", md.lam, MLMC_MAX_LAYERS);
  arr("model_qoi_box", md.qoi_box, 4);
  arr("model_line_lo", md.line_lo, 4);
  arr("model_line_hi", md.line_hi, 4);
}

bool read_model_block(FILE* f, mlmc_model* md) {
  if (std::fscanf(f, "model %d %d %d %d %d %d %d %d %d %d %d %d\n", &md->n_layers, &md->k_kind, &md->norm_r, &md->m0,
                  &md->L, &md->cgv, &md->prec, &md->max_it, &md->problem, &md->geometry, &md->dim, &md->embed) != 12)
    return false;
  if (std::fscanf(f, "model_if %lg %lg\nmodel_tol %lg\n", &md->if_lo, &md->if_hi, &md->tol) != 3) return false;
  auto arr = [&](const char* key, double* v, int n) {
    char name[32] = {};
    if (std::fscanf(f, "%31s", name) != 1 || std::strcmp(name, key) != 0) return false;
    for (int k = 0; k < n; ++k)
      if (std::fscanf(f, " %lg", &v[k]) != 1) return false;
    return std::fscanf(f, "\n") == 0;
  };
  return arr("model_mu", md->mu, MLMC_MAX_LAYERS) && arr("model_sigma2", md->sigma2, MLMC_MAX_LAYERS) &&
         arr("model_lam", md->lam, MLMC_MAX_LAYERS) && arr("model_qoi_box", md->qoi_box, 4) &&
         arr("model_line_lo", md->line_lo, 4) && arr("model_line_hi", md->line_hi, 4);
}

// The first field in which two models differ where the difference changes a
// sample's Q or its failure (per-layer entries only below n_layers, the
// interface range only with horizontal layers, the correlation lengths only
// for log-normal fields, the box only for Model Problem 1, the line ranges
// only for the sloped geometry); nullptr when they agree.
const char* model_difference(const mlmc_model& a, const mlmc_model& b) {
  if (a.n_layers != b.n_layers) return "n_layers";
  if (a.k_kind != b.k_kind) return "k_kind";
  if (a.m0 != b.m0) return "m0";
  if (a.L != b.L) return "L";
  if (a.cgv != b.cgv) return "cgv";
  if (a.prec != b.prec) return "prec";
  if (a.max_it != b.max_it) return "max_it";
  if (a.tol != b.tol) return "tol";
  if ((a.problem == 1) != (b.problem == 1)) return "problem";
  if (a.geometry != b.geometry) return "geometry";
  if (dim_of(a) != dim_of(b)) return "dim";
  for (int t = 0; t < a.n_layers; ++t) {
    if (a.mu[t] != b.mu[t]) return "mu";
    if (a.sigma2[t] != b.sigma2[t]) return "sigma2";
    if (a.k_kind == 1 && a.lam[t] != b.lam[t]) return "lam";
  }
  if (a.k_kind == 1 && a.norm_r != b.norm_r) return "norm_r";
  if (a.k_kind == 1 && a.embed != b.embed) return "embed";
  if (a.geometry == 0 && a.n_layers > 1 && (a.if_lo != b.if_lo || a.if_hi != b.if_hi)) return "if_lo/if_hi";
  if (a.problem == 1)
    for (int k = 0; k < 4; ++k)
      if (a.qoi_box[k] != b.qoi_box[k]) return "qoi_box";
  if (a.geometry == 1)
    for (int k = 0; k < 4; ++k)
      if (a.line_lo[k] != b.line_lo[k] || a.line_hi[k] != b.line_hi[k]) return "line_lo/line_hi";
  return nullptr;
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
  c->wst = c->st;
  c->model = *model;
  cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device);
  c->lev.resize(model->L + 1);
  int err = 0;
  Buf scratch, mm;
  if (cudaMallocHost(&c->host, sizeof(HostLevel) * (MLMC_MAX_LEVELS + 1)) != cudaSuccess) {
    c->host = nullptr;
    delete c;
    return fail(MLMC_ERR_NOMEM, "pinned host buffer");
  }
  if ((err = c->bm.ensure(kSinCosTab * sizeof(double2) + kBmLgDoubles * sizeof(double))) == 0 &&
      bm_tables_build(c->bm.as<double2>(), reinterpret_cast<double*>(c->bm.as<double2>() + kSinCosTab),
                      c->st))
    err = fail(MLMC_ERR_CUDA, "Box-Muller table kernel");
  if (!err && cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess)
    err = fail(MLMC_ERR_CUDA, "event");
  for (int l = 0; l <= model->L && !err; ++l)
    if (cudaStreamCreateWithFlags(&c->lst[l], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->lev_done[l], cudaEventDisableTiming) != cudaSuccess)
      err = fail(MLMC_ERR_CUDA, "level stream");
  pair_layers(c);
  for (int l = 0; l <= model->L && !err; ++l) {
    LevelTable& LT = c->lev[l];
    LT.m = model->m0 << l;
    if (model->k_kind != 1) continue;
    LT.pair.resize(c->n_draws);
    if ((err = mm.ensure(2 * sizeof(double)))) break;
    for (int f = 0; f < c->n_draws && !err; ++f) {
      PairTable& T = LT.pair[f];
      T.M = 0;
      const bool d3 = dim_of(*model) == 3;
      // padding candidates in order: M = 2m, the cut-off embedding at 3m (2-D,
      // 2-norm, m >= 8, unless embed = 1), then 4m, 8m, 16m
      const int cand_p[5] = {2, 3, 4, 8, 16};
      for (int ci = 0; ci < 5; ++ci) {
        const int p = cand_p[ci];
        const bool cut = p == 3;
        if (cut && (d3 || model->norm_r != 2 || LT.m < 8 || model->embed != 0)) continue;
        const int M = p * LT.m;
        if (M > (d3 ? 256 : 16384)) {
          err = fail(MLMC_ERR_TOOBIG, d3 ? "3-D embedding size M above 256" : "embedding size M above 16384");
          break;
        }
        const size_t npts = d3 ? (size_t)M * M * M : (size_t)M * M;
        if ((err = scratch.ensure((d3 ? 1 : 2) * npts * 16))) break;
        if ((err = T.s64.ensure(npts * 8)) || (err = T.s32.ensure(npts * 4)) ||
            (err = T.tw64.ensure((size_t)M * 16)) || (err = T.tw32.ensure((size_t)M * 8)))
          break;
        const int br = d3 ? ce_build_table3(LT.m, M, c->pair_sigma2[f], c->pair_lam[f], model->norm_r, scratch.p,
                                            T.s64.as<double>(), T.s32.as<float>(), mm.as<double>(), T.tw64.p,
                                            T.tw32.p, c->st)
                          : ce_build_table(LT.m, M, c->pair_sigma2[f], c->pair_lam[f], model->norm_r, cut ? 1 : 0,
                                           scratch.p,
                                           T.s64.as<double>(), T.s32.as<float>(), mm.as<double>(), T.tw64.p,
                                           T.tw32.p, c->st);
        if (br) {
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
  }
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
  for (auto& LT : c->lev)
    for (auto& T : LT.pair) {
      T.s64.release();
      T.s32.release();
      T.tw64.release();
      T.tw32.release();
    }
  for (Buf* b : {&c->oqf, &c->oqc, &c->oqg, &c->oit, &c->sums, &c->itacc, &c->g64, &c->bm}) b->release();
  c->misc.release();
  for (auto& S : c->slot) {
    for (Buf* b : {&S.qf, &S.qc, &S.qg, &S.it, &S.sums, &S.itacc}) b->release();
    S.wb.release();
  }
  for (int l = 0; l < MLMC_MAX_LEVELS; ++l) {
    if (c->lst[l]) cudaStreamDestroy(c->lst[l]);
    if (c->lev_done[l]) cudaEventDestroy(c->lev_done[l]);
  }
  for (int k = 0; k < mlmc_ctx::kClasses; ++k) {
    if (c->cst[k]) cudaStreamDestroy(c->cst[k]);
    if (c->class_done[k]) cudaEventDestroy(c->class_done[k]);
    c->sched_ws[k].release();
  }
  for (int l = 0; l < MLMC_MAX_LEVELS; ++l)
    if (c->fields_done[l]) cudaEventDestroy(c->fields_done[l]);
  c->sched_cnt.release();
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->host) cudaFreeHost(c->host);
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

int mlmc_estimate_ex(mlmc_ctx* c, double eps, uint64_t seed, int32_t n_pilot, int32_t cost_model,
                     int32_t max_rounds, mlmc_estimate_out* out) {
  if (!c || !out) return fail(MLMC_ERR_ARG, "null argument");
  if (!(eps > 0) || n_pilot < 2 || max_rounds < 0) return fail(MLMC_ERR_ARG, "eps > 0, n_pilot >= 2, max_rounds >= 0");
  if (cost_model < 0 || cost_model > 2) return fail(MLMC_ERR_ARG, "cost_model must be 0, 1 or 2");
  std::memset(out, 0, sizeof(*out));
  CUDA_TRY(cudaSetDevice(c->device));
  const double t0 = now_s();
  const mlmc_model& md = c->model;
  const int L = md.L;
  const int NL = L + 1;
  int rc_any = 0;
  std::vector<mlmc_level_sums> S(NL);
  std::vector<double> C(NL);
  std::vector<int64_t> first(NL, 0), cnt(NL, n_pilot);
  int rounds = 0;
  if (c->resume_est.valid) {
    // continue a checkpointed estimate: its sums stand in for the pilot and the
    // rounds already done
    if (c->resume_est.seed != seed || (int)c->resume_est.S.size() != NL)
      return fail(MLMC_ERR_ARG, "resumed state has another seed or level count");
    S = c->resume_est.S;
    C = c->resume_est.C;
    rounds = c->resume_est.rounds;
    c->resume_est.valid = false;
  } else if (cost_model == 2) {
    if (!c->cal_ok) return fail(MLMC_ERR_ARG, "cost_model 2 needs mlmc_calibrate_costs first");
    int r = multilevel_impl(c, NL, first.data(), cnt.data(), seed, true, S.data());
    if (r < 0) return r;
    rc_any |= r;
    for (int l = 0; l < NL; ++l) C[l] = c->cal_C[l];
  } else if (cost_model == 1) {
    // measured cost: the pilot runs level by level so that each is timed
    for (int l = 0; l < NL; ++l) {
      int r = mlmc_level_batch(c, l, 0, n_pilot, seed, nullptr, nullptr, nullptr, nullptr, &S[l]);
      if (r < 0) return r;
      rc_any |= r;
      C[l] = S[l].seconds / n_pilot;
    }
  } else {
    int r = multilevel_impl(c, NL, first.data(), cnt.data(), seed, true, S.data());
    if (r < 0) return r;
    rc_any |= r;
    for (int l = 0; l < NL; ++l) {
      const double md_cells = (double)cells_of(md, md.m0 << l);
      C[l] = md_cells * (1.0 + n_coarse(md, l) / (dim_of(md) == 3 ? 8.0 : 4.0));
    }
  }
  auto stats = [&](int l, double* mean, double* var) {
    const bool g = md.cgv && l > 0;
    const double n = (double)S[l].n;
    const double s1 = g ? S[l].s_yg : S[l].s_y, s2 = g ? S[l].s_yg2 : S[l].s_y2;
    *mean = s1 / n;
    const double v = n > 1 ? (s2 - s1 * s1 / n) / (n - 1) : INFINITY;
    *var = v > 0 ? v : 0.0;
  };
  while (true) {
    std::vector<double> V(NL), mu(NL);
    for (int l = 0; l < NL; ++l) stats(l, &mu[l], &V[l]);
    double tot = 0;
    for (int l = 0; l < NL; ++l) tot += std::sqrt(V[l] * C[l]);
    bool any = false;
    for (int l = 0; l < NL; ++l) {
      const double nopt = std::ceil(2.0 / (eps * eps) * std::sqrt(V[l] / C[l]) * tot);
      cnt[l] = std::max<int64_t>(0, (int64_t)nopt - S[l].n);
      first[l] = S[l].n + S[l].n_failed;
      any |= cnt[l] > 0;
    }
    if (!any || rounds >= max_rounds) break;
    ++rounds;
    std::vector<mlmc_level_sums> add(NL);
    int r = multilevel_impl(c, NL, first.data(), cnt.data(), seed, true, add.data());
    if (r < 0) return r;
    rc_any |= r;
    for (int l = 0; l < NL; ++l)
      if (cnt[l] > 0) add_sums(S[l], add[l]);
  }
  double qh = 0, vh = 0;
  for (int l = 0; l < NL; ++l) {
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
  // weak-error rate and bias of the finest level (reported, not controlled)
  out->alpha = out->bias = std::nan("");
  out->bias_flag = 0;
  if (NL >= 2) {
    double sl = 0, sy = 0, sll = 0, sly = 0;
    int k = 0;
    for (int l = 1; l < NL; ++l)
      if (out->mean[l] != 0.0) {
        const double y = std::log2(std::fabs(out->mean[l]));
        sl += l;
        sy += y;
        sll += (double)l * l;
        sly += l * y;
        ++k;
      }
    double alpha = 1.0;
    if (k >= 2) alpha = -(k * sly - sl * sy) / (k * sll - sl * sl);
    alpha = std::max(alpha, 0.5);
    out->alpha = alpha;
    out->bias = std::fabs(out->mean[NL - 1]) / (std::exp2(alpha) - 1.0);
    out->bias_flag = out->bias > eps / std::sqrt(2.0) ? 1 : 0;
  }
  out->seconds = now_s() - t0;
  auto& st = c->last_est;
  st.valid = true;
  st.eps = eps;
  st.seed = seed;
  st.cost_model = cost_model;
  st.rounds = rounds;
  st.S = S;
  st.C = C;
  return rc_any ? MLMC_SOME_FAILED : MLMC_OK;
}

int mlmc_estimate(mlmc_ctx* c, double eps, uint64_t seed, int32_t n_pilot, int32_t cost_model,
                  mlmc_estimate_out* out) {
  return mlmc_estimate_ex(c, eps, seed, n_pilot, cost_model, 10, out);
}

// Text format, one "key value..." per line; doubles with 17 significant
// digits so that a resumed estimate is bit-identical to an uninterrupted one,
// and so that the model fields read back exactly.
int mlmc_checkpoint(mlmc_ctx* c, const char* path) {
  if (!c || !path) return fail(MLMC_ERR_ARG, "null argument");
  const auto& st = c->last_est;
  if (!st.valid) return fail(MLMC_ERR_ARG, "no estimate to checkpoint");
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(MLMC_ERR_ARG, std::string("cannot write ") + path);
  std::fprintf(f, "mlmc_checkpoint 2\n");
  write_model_block(f, c->model);
  std::fprintf(f, "seed %llu\neps %.17g\ncost_model %d\nrounds %d\nlevels %d\n", (unsigned long long)st.seed,
               st.eps, st.cost_model, st.rounds, (int)st.S.size());
  for (size_t l = 0; l < st.S.size(); ++l) {
    const auto& x = st.S[l];
    std::fprintf(f, "level %zu %lld %lld %lld %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g\n",
                 l, (long long)x.n, (long long)x.n_failed, (long long)x.iters_total, x.s_qf, x.s_qf2, x.s_qc, x.s_qc2,
                 x.s_y, x.s_y2, x.s_qcg, x.s_qcg2, x.s_yg, x.s_yg2, x.seconds, st.C[l]);
  }
  const bool ok = std::fclose(f) == 0;
  return ok ? 0 : fail(MLMC_ERR_ARG, std::string("error writing ") + path);
}

int mlmc_checkpoint_check(const mlmc_model* model, const char* path) {
  if (!model || !path) return fail(MLMC_ERR_ARG, "null argument");
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(MLMC_ERR_ARG, std::string("cannot read ") + path);
  int ver = 0;
  int r = std::fscanf(f, "mlmc_checkpoint %d\n", &ver) == 1 && ver == 2 ? 0
          : fail(MLMC_ERR_ARG, std::string("not a version-2 checkpoint: ") + path);
  mlmc_model other{};
  if (!r) r = read_model_block(f, &other) ? 0 : fail(MLMC_ERR_ARG, std::string("unreadable model block: ") + path);
  std::fclose(f);
  if (r) return r;
  const char* diff = model_difference(*model, other);
  if (diff) return fail(MLMC_ERR_ARG, std::string("checkpoint of another model (") + diff + " differs): " + path);
  return 0;
}

int mlmc_resume(mlmc_ctx* c, const char* path) {
  if (!c || !path) return fail(MLMC_ERR_ARG, "null argument");
  if (int e = mlmc_checkpoint_check(&c->model, path)) return e;
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(MLMC_ERR_ARG, std::string("cannot read ") + path);
  mlmc_ctx::EstState st;
  int ver = 0, nl = 0;
  unsigned long long seed = 0;
  mlmc_model skip{};
  bool ok = std::fscanf(f, "mlmc_checkpoint %d\n", &ver) == 1 && read_model_block(f, &skip) &&
            std::fscanf(f, "seed %llu\neps %lg\ncost_model %d\nrounds %d\nlevels %d\n", &seed, &st.eps,
                        &st.cost_model, &st.rounds, &nl) == 5 &&
            nl == c->model.L + 1;
  for (int l = 0; ok && l < nl; ++l) {
    mlmc_level_sums x{};
    long long a, b, cc;
    size_t ll;
    double cost;
    ok = std::fscanf(f, "level %zu %lld %lld %lld %lg %lg %lg %lg %lg %lg %lg %lg %lg %lg %lg %lg\n", &ll, &a, &b,
                     &cc, &x.s_qf, &x.s_qf2, &x.s_qc, &x.s_qc2, &x.s_y, &x.s_y2, &x.s_qcg, &x.s_qcg2, &x.s_yg,
                     &x.s_yg2, &x.seconds, &cost) == 16 &&
         ll == (size_t)l;
    x.n = a;
    x.n_failed = b;
    x.iters_total = cc;
    st.S.push_back(x);
    st.C.push_back(cost);
  }
  std::fclose(f);
  if (!ok) return fail(MLMC_ERR_ARG, std::string("unreadable estimator state: ") + path);
  st.seed = seed;
  st.valid = true;
  c->resume_est = st;
  return 0;
}

int mlmc_multilevel_batch(mlmc_ctx* c, int32_t n_levels, const int64_t* first, const int64_t* n, uint64_t seed,
                          int32_t use_graph, mlmc_level_sums* sums) {
  if (!c || !first || !n || !sums) return fail(MLMC_ERR_ARG, "null argument");
  if (n_levels < 1 || n_levels > c->model.L + 1) return fail(MLMC_ERR_ARG, "n_levels out of range");
  for (int l = 0; l < n_levels; ++l)
    if (n[l] < 0 || first[l] < 0) return fail(MLMC_ERR_ARG, "negative sample range");
  CUDA_TRY(cudaSetDevice(c->device));
  const double t0 = now_s();
  const int r = multilevel_impl(c, n_levels, first, n, seed, use_graph != 0, sums);
  const double dt = now_s() - t0;
  for (int l = 0; l < n_levels; ++l) sums[l].seconds = dt;
  return r;
}

int mlmc_multilevel_batch_host(mlmc_ctx* c, int32_t n_levels, const int64_t* first, const int64_t* n,
                               uint64_t seed, int32_t use_graph, double* const* qf, double* const* qc,
                               double* const* qc_cgv, int32_t* const* iters, mlmc_level_sums* sums) {
  if (!c || !first || !n || !sums) return fail(MLMC_ERR_ARG, "null argument");
  if (n_levels < 1 || n_levels > c->model.L + 1) return fail(MLMC_ERR_ARG, "n_levels out of range");
  for (int l = 0; l < n_levels; ++l)
    if (n[l] < 0 || first[l] < 0) return fail(MLMC_ERR_ARG, "negative sample range");
  CUDA_TRY(cudaSetDevice(c->device));
  bool want_iters = false;
  for (int l = 0; l < n_levels && iters; ++l) want_iters = want_iters || (iters[l] && n[l] > 0);
  const double t0 = now_s();
  const int r = multilevel_impl(c, n_levels, first, n, seed, use_graph != 0, sums, want_iters);
  if (r < 0) return r;
  for (int l = 0; l < n_levels; ++l) {
    if (n[l] <= 0) continue;
    const auto& S = c->slot[l];
    const size_t nb = (size_t)n[l];
    if (qf && qf[l]) CUDA_TRY(cudaMemcpyAsync(qf[l], S.qf.p, nb * 8, cudaMemcpyDeviceToHost, c->st));
    if (qc && qc[l]) CUDA_TRY(cudaMemcpyAsync(qc[l], S.qc.p, nb * 8, cudaMemcpyDeviceToHost, c->st));
    if (qc_cgv && qc_cgv[l]) CUDA_TRY(cudaMemcpyAsync(qc_cgv[l], S.qg.p, nb * 8, cudaMemcpyDeviceToHost, c->st));
    if (iters && iters[l]) CUDA_TRY(cudaMemcpyAsync(iters[l], S.it.p, nb * 4, cudaMemcpyDeviceToHost, c->st));
  }
  CUDA_TRY(cudaStreamSynchronize(c->st));
  const double dt = now_s() - t0;
  for (int l = 0; l < n_levels; ++l) sums[l].seconds = dt;
  return r;
}

// Candidate launch plans of each level timed on a probe batch; the fastest
// is kept for the level's solves.
int mlmc_autotune(mlmc_ctx* c, uint64_t seed, mlmc_tune_report* rep) {
  if (!c) return fail(MLMC_ERR_ARG, "null context");
  CUDA_TRY(cudaSetDevice(c->device));
  const mlmc_model& md = c->model;
  if (rep) std::memset(rep, 0, sizeof(*rep));
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  int err = 0;
  for (int l = 0; l <= md.L && !err; ++l) {
    c->tuned_ok[l] = false;
    c->tuned_c_ok[l] = false;
    const int m = md.m0 << l;
    const int nc = n_coarse(md, l);
    // probe: enough systems to fill the GPU, few enough to stay short
    int64_t n = std::max<int64_t>(4, std::min<int64_t>(65536, ((int64_t)1 << 24) / cells_of(md, m)));
    n = std::min<int64_t>(n, chunk_samples(c, l));
    if ((err = prepare_level(c, l, n))) break;
    SolveArgs a = base_args(c, l, seed, (int64_t)1 << 40);
    if (md.k_kind == 1) {
      if ((err = run_fields(c, l, a.first, n, seed))) break;
      a.g = c->wb->g.p;
    }
    // which = 0: all systems in one launch (level 0); 1: the fine systems;
    // 2: the coarse systems (their own launch and plan); fine_plan is the
    // fine launch's plan while the coarse one is tuned
    SolvePlan fine_plan{};
    auto tune = [&](int which, int msz, SolvePlan* best_out, float* def_out, float* best_ms_out,
                    int* nk_out) -> int {
      SolvePlan cand[28];
      int nk = dim_of(md) == 3 ? solve3_plan_candidates(msz, md.prec, cand, 16)
                               : solve_plan_candidates(msz, md.prec, cand, 16);
      float best = 1e30f, def_ms = 0.f;
      int best_k = -1;
      auto time_plan = [&](const SolvePlan& P) -> float {
        float ms = 1e30f;
        for (int rep_i = 0; rep_i < 2 && !err; ++rep_i) {
          cudaEventRecord(e0, c->st);
          if (which == 0) err = run_solves(c, a, n, nc, 0, &P);
          else if (which == 1) err = run_solves(c, a, n, nc, 0, &P, &P, 1);
          else err = run_solves(c, a, n, nc, 0, &fine_plan, &P, 2);
          cudaEventRecord(e1, c->st);
          if (cudaEventSynchronize(e1) != cudaSuccess) err = fail(MLMC_ERR_CUDA, "autotune timing");
          float t = 0.f;
          cudaEventElapsedTime(&t, e0, e1);
          ms = t;
          if (rep_i == 0 && t > 3.f * best) break;  // clearly slower: one run is enough
        }
        return ms;
      };
      auto consider = [&](const SolvePlan& P) {
        cand[nk] = P;
        const float ms = time_plan(cand[nk]);
        if (ms < best) {
          best = ms;
          best_k = nk;
        }
        ++nk;
      };
      for (int k = 0; k < nk && !err; ++k) {
        const float ms = time_plan(cand[k]);
        if (k == 0) def_ms = ms;
        if (ms < best) {
          best = ms;
          best_k = k;
        }
      }
      if (!err && best_k >= 0) {  // the fastest plan once more with W-cycles, and with two sweep pairs
        const SolvePlan base = cand[best_k];
        for (int v = 0; v < 2 && !err; ++v) {
          SolvePlan q = base;
          if (v == 0) q.gamma = 2;
          else q.nu = 2;
          consider(q);
        }
      }
      if (!err && best_k >= 0) {  // stronger smoothing on the finest grid only: (nu, nuc) = (2, 1), (3, 1)
        const SolvePlan base = cand[best_k];
        for (int nu : {2, 3}) {
          if (err) break;
          SolvePlan q = base;
          q.nu = nu;
          q.nu_coarse = 1;
          consider(q);
        }
      }
      if (!err && best_k >= 0 && (md.prec == 1 || md.prec == 2)) {  // mixed: looser or tighter FP32 inner solves
        const SolvePlan base = cand[best_k];
        for (double it : {1e-4, 1e-6}) {
          if (err) break;
          SolvePlan q = base;
          q.inner_tol = it;
          consider(q);
        }
        // one FP32 CG with reliable updates instead of restarted refinement (2-D)
        for (double it : {1e-2, 1e-3}) {
          if (err || dim_of(md) == 3) break;
          SolvePlan q = base;
          q.reliable = 1;
          q.inner_tol = it;
          consider(q);
        }
      }
      if (err) return err;
      if (best_k < 0) return fail(MLMC_ERR_CUDA, "autotune: no launch plan ran");
      *best_out = cand[best_k];
      *def_out = def_ms;
      *best_ms_out = best;
      *nk_out = nk;
      return 0;
    };
    SolvePlan best{}, best_c{};
    float def_ms = 0.f, best_ms = 0.f, def_c = 0.f, best_c_ms = 0.f;
    int nk = 0, nk_c = 0;
    bool split = false;
    if (nc == 0) {
      if ((err = tune(0, m, &best, &def_ms, &best_ms, &nk))) break;
    } else {
      if ((err = tune(1, m, &best, &def_ms, &best_ms, &nk))) break;
      fine_plan = best;
      if ((err = tune(2, m / 2, &best_c, &def_c, &best_c_ms, &nk_c))) break;
      // two launches run one after the other: keep them only if they beat one
      // launch of all the level's systems on the fine systems' plan
      float one = 1e30f;
      for (int rep_i = 0; rep_i < 2 && !err; ++rep_i) {
        cudaEventRecord(e0, c->st);
        err = run_solves(c, a, n, nc, 0, &best);
        cudaEventRecord(e1, c->st);
        if (cudaEventSynchronize(e1) != cudaSuccess) err = fail(MLMC_ERR_CUDA, "autotune timing");
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        one = std::min(one, t);
      }
      if (err) break;
      split = best_ms + best_c_ms < one;
      if (!split) {
        best_ms = one;
        best_c_ms = 0.f;
      }
    }
    c->tuned[l] = best;
    c->tuned_ok[l] = true;
    if (split) {
      c->tuned_c[l] = best_c;
      c->tuned_c_ok[l] = true;
    }
    if (rep) {
      rep->threads[l] = best.threads;
      rep->warp[l] = best.warp;
      rep->cap_blocks_per_sm[l] = best.cap_blocks_per_sm;
      rep->cluster[l] = best.cluster;
      rep->gamma[l] = best.gamma;
      rep->nu[l] = best.nu;
      rep->nu_coarse[l] = best.nu_coarse > 0 ? best.nu_coarse : best.nu;
      rep->inner_tol[l] = best.inner_tol;
      rep->reliable[l] = best.reliable;
      rep->candidates[l] = nk + nk_c;
      rep->smem[l] = best.use_smem;
      rep->ms_default[l] = (def_ms + def_c) / n;
      rep->ms_best[l] = (best_ms + best_c_ms) / n;
      if (split) {
        rep->c_threads[l] = best_c.threads;
        rep->c_warp[l] = best_c.warp;
        rep->c_cluster[l] = best_c.cluster;
        rep->c_cap_blocks_per_sm[l] = best_c.cap_blocks_per_sm;
        rep->c_gamma[l] = best_c.gamma;
        rep->c_nu[l] = best_c.nu;
        rep->c_nu_coarse[l] = best_c.nu_coarse > 0 ? best_c.nu_coarse : best_c.nu;
        rep->c_inner_tol[l] = best_c.inner_tol;
        rep->c_reliable[l] = best_c.reliable;
        rep->c_smem[l] = best_c.use_smem;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return err;
}

// Plan fields of a tune report from the context's current plans.
static void report_plans(const mlmc_ctx* c, mlmc_tune_report* rep) {
  std::memset(rep, 0, sizeof(*rep));
  const mlmc_model& md = c->model;
  for (int l = 0; l <= md.L; ++l) {
    SolvePlan P;
    if (c->tuned_ok[l]) P = c->tuned[l];
    else if (plan_of(md, md.m0 << l, &P)) continue;
    rep->threads[l] = P.threads;
    rep->warp[l] = P.warp;
    rep->cap_blocks_per_sm[l] = P.cap_blocks_per_sm;
    rep->cluster[l] = P.cluster;
    rep->gamma[l] = P.gamma;
    rep->nu[l] = P.nu;
    rep->nu_coarse[l] = P.nu_coarse > 0 ? P.nu_coarse : P.nu;
    rep->inner_tol[l] = P.inner_tol;
    rep->reliable[l] = P.reliable;
    rep->smem[l] = P.use_smem;
    if (c->tuned_c_ok[l]) {
      const SolvePlan& Q = c->tuned_c[l];
      rep->c_threads[l] = Q.threads;
      rep->c_warp[l] = Q.warp;
      rep->c_cluster[l] = Q.cluster;
      rep->c_cap_blocks_per_sm[l] = Q.cap_blocks_per_sm;
      rep->c_gamma[l] = Q.gamma;
      rep->c_nu[l] = Q.nu;
      rep->c_nu_coarse[l] = Q.nu_coarse > 0 ? Q.nu_coarse : Q.nu;
      rep->c_inner_tol[l] = Q.inner_tol;
      rep->c_reliable[l] = Q.reliable;
      rep->c_smem[l] = Q.use_smem;
    }
  }
}

int mlmc_autotune_schedule(mlmc_ctx* c, double eps, uint64_t seed, int32_t n_pilot, int32_t cost_model,
                           int32_t reps, double* ms, mlmc_tune_report* rep) {
  if (!c) return fail(MLMC_ERR_ARG, "null context");
  if (!(eps > 0) || n_pilot < 2 || reps < 1 || cost_model < 0 || cost_model > 2)
    return fail(MLMC_ERR_ARG, "eps > 0, n_pilot >= 2, reps >= 1, cost_model 0, 1 or 2");
  CUDA_TRY(cudaSetDevice(c->device));
  const mlmc_model& md = c->model;
  if (ms) ms[0] = ms[1] = 0.0;
  if (!c->sched || dim_of(md) == 3 || (md.prec != 0 && md.prec != 1)) {
    if (rep) report_plans(c, rep);
    return 0;
  }
  for (int l = 0; l <= md.L; ++l)  // explicit plans for every level, to vary
    if (!c->tuned_ok[l]) {
      if (plan_of(md, md.m0 << l, &c->tuned[l])) return fail(MLMC_ERR_CUDA, "occupancy query failed");
      c->tuned_ok[l] = true;
    }
  const auto saved_last = c->last_est, saved_resume = c->resume_est;
  c->resume_est.valid = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  int err = 0;
  auto time_estimate = [&](double* out) -> int {
    mlmc_estimate_out o;
    int e = mlmc_estimate(c, eps, seed, n_pilot, cost_model, &o);  // untimed: captures the round graphs
    if (e < 0) return e;
    double best = 1e300;
    for (int r = 0; r < reps; ++r) {
      if (cudaEventRecord(e0, c->st) != cudaSuccess) return fail(MLMC_ERR_CUDA, "event");
      e = mlmc_estimate(c, eps, seed, n_pilot, cost_model, &o);
      if (e < 0) return e;
      if (cudaEventRecord(e1, c->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
        return fail(MLMC_ERR_CUDA, "event");
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      best = std::min(best, (double)t);
    }
    *out = best;
    return 0;
  };
  double best = 0.0;
  err = time_estimate(&best);
  if (ms) ms[0] = best;
  for (int l = md.L; l >= 0 && !err; --l) {
    const int m = md.m0 << l;
    const int nc = n_coarse(md, l);
    for (int part = 0; part < 2 && !err; ++part) {
      if (part == 1 && nc == 0) break;
      const int msz = part == 0 ? m : m / 2;
      if (msz < 256) continue;
      const bool split = c->tuned_c_ok[l];
      const SolvePlan cur = part == 0 ? c->tuned[l] : (split ? c->tuned_c[l] : c->tuned[l]);
      // candidate shapes (mode, cluster)
      int shapes[2][2], ns = 0;
      if (part == 1 && !split) {  // the coarse systems share the fine launch: try a launch of their own
        shapes[ns][0] = 0, shapes[ns][1] = 0, ++ns;
        shapes[ns][0] = 2, shapes[ns][1] = 4, ++ns;
      } else if (cur.cluster) {
        shapes[ns][0] = 0, shapes[ns][1] = 0, ++ns;
        shapes[ns][0] = 2, shapes[ns][1] = cur.cluster == 4 ? 8 : 4, ++ns;
      } else {
        shapes[ns][0] = 2, shapes[ns][1] = 4, ++ns;
      }
      for (int k = 0; k < ns && !err; ++k) {
        SolvePlan P;
        const int mode = shapes[k][0], cl = shapes[k][1];
        if (solve_plan_mode(msz, md.prec, mode, 512, cl, &P)) continue;
        if (part == 1 && split == false && mode == 0 && !cur.cluster && cur.threads == 512 && !cur.warp)
          continue;  // the shared launch already is a block of 512
        P.gamma = cur.gamma;
        P.nu = cur.nu;
        P.nu_coarse = cur.nu_coarse;
        P.reliable = cur.reliable;
        P.inner_tol = cur.inner_tol;
        P.cap_blocks_per_sm = 0;
        const SolvePlan keep = part == 0 ? c->tuned[l] : c->tuned_c[l];
        const bool keep_ok = part == 0 ? true : c->tuned_c_ok[l];
        if (part == 0) c->tuned[l] = P;
        else {
          c->tuned_c[l] = P;
          c->tuned_c_ok[l] = true;
        }
        double t = 0.0;
        if ((err = time_estimate(&t))) break;
        if (t < 0.995 * best) {
          best = t;
        } else if (part == 0) {
          c->tuned[l] = keep;
        } else {
          c->tuned_c[l] = keep;
          c->tuned_c_ok[l] = keep_ok;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->last_est = saved_last;
  c->resume_est = saved_resume;
  if (err) return err;
  if (ms) ms[1] = best;
  if (rep) report_plans(c, rep);
  return 0;
}

int mlmc_calibrate_costs(mlmc_ctx* c, uint64_t seed, double* C_out) {
  if (!c) return fail(MLMC_ERR_ARG, "null context");
  CUDA_TRY(cudaSetDevice(c->device));
  const mlmc_model& md = c->model;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  int err = 0;
  for (int l = 0; l <= md.L && !err; ++l) {
    // enough samples to fill the GPU at every level (2^26 cells, 64 .. 65536
    // samples), from sample index 2^40 on so that no sample of real use is
    // consumed; one untimed batch (allocations, caches), then the faster of two
    const int64_t n = std::max<int64_t>(64, std::min<int64_t>(65536, ((int64_t)1 << 26) / cells_of(md, md.m0 << l)));
    mlmc_level_sums s;
    double best = 1e300;
    for (int r = 0; r < 3 && !err; ++r) {
      if (r > 0 && cudaEventRecord(e0, c->st) != cudaSuccess) err = fail(MLMC_ERR_CUDA, "event");
      if (!err) {
        const int rc = mlmc_level_batch(c, l, (int64_t)1 << 40, n, seed, nullptr, nullptr, nullptr, nullptr, &s);
        if (rc < 0) err = rc;
      }
      if (!err && r > 0) {
        if (cudaEventRecord(e1, c->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
          err = fail(MLMC_ERR_CUDA, "event");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, (double)ms);
      }
    }
    if (!err) c->cal_C[l] = best * 1e-3 / (double)n;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err) return err;
  c->cal_ok = true;
  if (C_out)
    for (int l = 0; l <= md.L; ++l) C_out[l] = c->cal_C[l];
  return 0;
}

int mlmc_set_costs(mlmc_ctx* c, const double* C) {
  if (!c || !C) return fail(MLMC_ERR_ARG, "null argument");
  for (int l = 0; l <= c->model.L; ++l)
    if (!(C[l] > 0) || !std::isfinite(C[l])) return fail(MLMC_ERR_ARG, "costs must be positive and finite");
  for (int l = 0; l <= c->model.L; ++l) c->cal_C[l] = C[l];
  c->cal_ok = true;
  return 0;
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

int mlmc_set_launch(mlmc_ctx* c, int level, int32_t mode, int32_t threads, int32_t cluster, int32_t gamma,
                    int32_t nu) {
  if (!c || level < 0 || level > c->model.L) return fail(MLMC_ERR_ARG, "bad context or level");
  CUDA_TRY(cudaSetDevice(c->device));
  if (mode < 0) {
    c->tuned_ok[level] = false;
    c->tuned_c_ok[level] = false;
    return 0;
  }
  if (mode > 3 || (mode == 0 && (threads < 32 || threads > 512 || threads % 32)) ||
      (mode == 2 && (cluster < 2 || cluster > 8 || (cluster & (cluster - 1)))))
    return fail(MLMC_ERR_ARG, "mode 0: threads 32..512 (multiple of 32); mode 2: cluster 2, 4 or 8");
  if (mode == 3 && ((c->model.m0 << level) != 16 || c->model.prec != 1 || dim_of(c->model) == 3))
    return fail(MLMC_ERR_ARG, "mode 3 (register path) needs m = 16, prec 1, 2-D");
  SolvePlan P;
  if (gamma < 1 || gamma > 2) return fail(MLMC_ERR_ARG, "gamma must be 1 (V-cycle) or 2 (W-cycle)");
  if (nu < 1 || nu > 4) return fail(MLMC_ERR_ARG, "nu must be 1..4");
  const int lm = c->model.m0 << level;
  const int mr = dim_of(c->model) == 3 ? solve3_plan_mode(lm, c->model.prec, mode, mode == 0 ? threads : 512, cluster, &P)
                                       : solve_plan_mode(lm, c->model.prec, mode, mode == 0 ? threads : 512, cluster, &P);
  if (mr)
    return fail(MLMC_ERR_CUDA, "launch plan query failed");
  P.gamma = gamma;
  P.nu = nu;
  c->tuned[level] = P;
  c->tuned_ok[level] = true;
  c->tuned_c_ok[level] = false;  // one launch for all the level's systems
  return 0;
}

int mlmc_set_launch_coarse(mlmc_ctx* c, int level, int32_t mode, int32_t threads, int32_t cluster, int32_t gamma,
                           int32_t nu) {
  if (!c || level < 1 || level > c->model.L) return fail(MLMC_ERR_ARG, "bad context or level (>= 1)");
  CUDA_TRY(cudaSetDevice(c->device));
  if (mode < 0) {
    c->tuned_c_ok[level] = false;
    return 0;
  }
  if (mode > 3 || (mode == 0 && (threads < 32 || threads > 512 || threads % 32)) ||
      (mode == 2 && (cluster < 2 || cluster > 8 || (cluster & (cluster - 1)))))
    return fail(MLMC_ERR_ARG, "mode 0: threads 32..512 (multiple of 32); mode 2: cluster 2, 4 or 8");
  const int mc = (c->model.m0 << level) / 2;
  if (mode == 3 && (mc != 16 || c->model.prec != 1 || dim_of(c->model) == 3))
    return fail(MLMC_ERR_ARG, "mode 3 (register path) needs coarse m = 16, prec 1, 2-D");
  if (gamma < 1 || gamma > 2) return fail(MLMC_ERR_ARG, "gamma must be 1 (V-cycle) or 2 (W-cycle)");
  if (nu < 1 || nu > 4) return fail(MLMC_ERR_ARG, "nu must be 1..4");
  SolvePlan P;
  const int mr = dim_of(c->model) == 3 ? solve3_plan_mode(mc, c->model.prec, mode, mode == 0 ? threads : 512, cluster, &P)
                                       : solve_plan_mode(mc, c->model.prec, mode, mode == 0 ? threads : 512, cluster, &P);
  if (mr) return fail(MLMC_ERR_CUDA, "launch plan query failed");
  P.gamma = gamma;
  P.nu = nu;
  if (!c->tuned_ok[level]) {  // the fine systems keep the default plan
    SolvePlan F;
    if (plan_of(c->model, c->model.m0 << level, &F)) return fail(MLMC_ERR_CUDA, "launch plan query failed");
    c->tuned[level] = F;
    c->tuned_ok[level] = true;
  }
  c->tuned_c[level] = P;
  c->tuned_c_ok[level] = true;
  return 0;
}

int mlmc_set_schedule(mlmc_ctx* c, int32_t schedule) {
  if (!c) return fail(MLMC_ERR_ARG, "null context");
  if (schedule != 0 && schedule != 1) return fail(MLMC_ERR_ARG, "schedule must be 0 or 1");
  c->sched = schedule;
  return 0;
}

int mlmc_set_launch_ex(mlmc_ctx* c, int level, int32_t part, int32_t mode, int32_t threads, int32_t cluster,
                       int32_t gamma, int32_t nu, int32_t nu_coarse, int32_t cap_blocks_per_sm, int32_t reliable,
                       double inner_tol) {
  if (!c || level < 0 || level > c->model.L) return fail(MLMC_ERR_ARG, "bad context or level");
  if (part != 0 && part != 1) return fail(MLMC_ERR_ARG, "part must be 0 (fine) or 1 (coarse)");
  if (part == 1 && (level < 1 || n_coarse(c->model, level) == 0))
    return fail(MLMC_ERR_ARG, "part 1 needs a level >= 1 with coarse systems");
  if (mode < 0 || mode > 3 || (mode == 0 && (threads < 32 || threads > 512 || threads % 32)) ||
      (mode == 2 && (cluster < 2 || cluster > 8 || (cluster & (cluster - 1)))))
    return fail(MLMC_ERR_ARG, "mode 0..3; mode 0: threads 32..512 (multiple of 32); mode 2: cluster 2, 4 or 8");
  const int msz = part == 0 ? c->model.m0 << level : (c->model.m0 << level) / 2;
  if (mode == 3 && (msz != 16 || c->model.prec != 1 || dim_of(c->model) == 3))
    return fail(MLMC_ERR_ARG, "mode 3 (register path) needs systems of side 16, prec 1, 2-D");
  if (gamma < 1 || gamma > 2) return fail(MLMC_ERR_ARG, "gamma must be 1 (V-cycle) or 2 (W-cycle)");
  if (nu < 1 || nu > 4 || nu_coarse < 0 || nu_coarse > 4) return fail(MLMC_ERR_ARG, "nu 1..4, nu_coarse 0..4");
  if (cap_blocks_per_sm < 0) return fail(MLMC_ERR_ARG, "cap_blocks_per_sm >= 0");
  if ((reliable != 0 && reliable != 1) || !(inner_tol > 0 && inner_tol <= 0.5))
    return fail(MLMC_ERR_ARG, "reliable must be 0 or 1 and inner_tol in (0, 0.5]");
  if (reliable && dim_of(c->model) == 3) return fail(MLMC_ERR_ARG, "reliable updates are 2-D only");
  CUDA_TRY(cudaSetDevice(c->device));
  SolvePlan P;
  const int t = mode == 0 ? threads : 512;
  const int mr = dim_of(c->model) == 3 ? solve3_plan_mode(msz, c->model.prec, mode, t, cluster, &P)
                                       : solve_plan_mode(msz, c->model.prec, mode, t, cluster, &P);
  if (mr) return fail(MLMC_ERR_CUDA, "launch plan query failed");
  P.gamma = gamma;
  P.nu = nu;
  P.nu_coarse = nu_coarse;
  P.cap_blocks_per_sm = cap_blocks_per_sm;
  P.reliable = reliable;
  P.inner_tol = inner_tol;
  if (part == 0) {
    c->tuned[level] = P;
    c->tuned_ok[level] = true;
  } else {
    if (!c->tuned_ok[level]) {  // the fine systems keep the default plan
      SolvePlan F;
      if (plan_of(c->model, c->model.m0 << level, &F)) return fail(MLMC_ERR_CUDA, "launch plan query failed");
      c->tuned[level] = F;
      c->tuned_ok[level] = true;
    }
    c->tuned_c[level] = P;
    c->tuned_c_ok[level] = true;
  }
  return 0;
}

int mlmc_set_solver(mlmc_ctx* c, int level, int32_t reliable, double inner_tol) {
  if (!c || level < 0 || level > c->model.L) return fail(MLMC_ERR_ARG, "bad context or level");
  if ((reliable != 0 && reliable != 1) || !(inner_tol > 0 && inner_tol <= 0.5))
    return fail(MLMC_ERR_ARG, "reliable must be 0 or 1 and inner_tol in (0, 0.5]");
  if (reliable && dim_of(c->model) == 3) return fail(MLMC_ERR_ARG, "reliable updates are 2-D only");
  CUDA_TRY(cudaSetDevice(c->device));
  if (!c->tuned_ok[level]) {
    SolvePlan P;
    if (plan_of(c->model, c->model.m0 << level, &P)) return fail(MLMC_ERR_CUDA, "launch plan query failed");
    c->tuned[level] = P;
    c->tuned_ok[level] = true;
  }
  c->tuned[level].reliable = reliable;
  c->tuned[level].inner_tol = inner_tol;
  if (c->tuned_c_ok[level]) {
    c->tuned_c[level].reliable = reliable;
    c->tuned_c[level].inner_tol = inner_tol;
  }
  return 0;
}

int mlmc_ce_info(mlmc_ctx* c, int level, int32_t* M_out, double* lam_min, double* lam_max) {
  if (!c || level < 0 || level > c->model.L) return fail(MLMC_ERR_ARG, "bad context or level");
  const bool any = !c->lev[level].pair.empty();
  if (M_out) *M_out = any ? c->lev[level].pair[0].M : 0;
  if (lam_min) *lam_min = any ? c->lev[level].pair[0].lam_min : 0.0;
  if (lam_max) *lam_max = any ? c->lev[level].pair[0].lam_max : 0.0;
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
                     reinterpret_cast<const double*>(c->bm.as<double2>() + kSinCosTab), fields_f32(c->model),
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
    if (const_fields_launch(a, n, cells_of(md, m), g, c->st)) return fail(MLMC_ERR_CUDA, "fields kernel");
  } else {
    if (int e = run_fields(c, level, first, n, seed)) return e;
    const int64_t cnt = n * md.n_layers * cells_of(md, m);
    if (fields_f32(md))
      f32_to_f64_launch(c->wb->g.as<float>(), g, cnt, c->st);
    else
      CUDA_TRY(cudaMemcpyAsync(g, c->wb->g.p, cnt * 8, cudaMemcpyDeviceToDevice, c->st));
  }
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return 0;
}

int mlmc_solve_k(mlmc_ctx* c, int32_t m, int64_t n, const double* k, double* p, double* q,
                 int32_t* iters) {
  if (!c || !k || !q || n < 0) return fail(MLMC_ERR_ARG, "bad argument");
  if (!is_pow2(m) || m > (dim_of(c->model) == 3 ? 128 : 4096))
    return fail(MLMC_ERR_ARG, "m must be a power of two <= 4096 (2-D) or 128 (3-D)");
  if (n == 0) return 0;
  CUDA_TRY(cudaSetDevice(c->device));
  SolveArgs a = base_args(c, 0, 0, 0);
  a.m = m;
  a.ksrc = KSRC_ARRAY;
  a.k = k;
  a.p_out = p;
  if (int e = run_solves(c, a, n, 0, n)) return e;
  CUDA_TRY(cudaMemcpyAsync(q, c->wb->qsys.p, n * 8, cudaMemcpyDeviceToDevice, c->st));
  if (iters) CUDA_TRY(cudaMemcpyAsync(iters, c->wb->itsys.p, n * 4, cudaMemcpyDeviceToDevice, c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return 0;
}

}  // extern "C"

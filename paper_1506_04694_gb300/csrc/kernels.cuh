// Launch descriptors and host entry points of the kernels (internal header).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace mlmc {

constexpr int MAX_LAYERS_DEV = 8;

// ------------------------------------------------------------------- CE ---
struct CeRowsArgs {
  const double2* bm_sc;  // Box-Muller tables (common.cuh, BmTables)
  const double* bm_lg;
  int M, logM, m, rows_per_block, pair, level;
  int r3;            // 1: M = 3 2^logM (cut-off embedding), 0: M = 2^logM
  int n_rows;        // rows of M points per sample: M (2-D) or M^2 (3-D)
  uint64_t seed;
  int64_t first;     // sample index of chunk entry 0
  int64_t z_offset;  // chunk entry of blockIdx.z == 0
};

struct CeColsArgs {
  int M, logM, m, cols_per_block, n_layers;
  int r3;          // as in CeRowsArgs
  int64_t ncols;   // columns of the M-row input: m (2-D), m (3-D middle pass) or m^2 (3-D last pass)
  int t_re, t_im;  // layers fed by Re and Im of this draw (t_im < 0: none)
  double mu_re, mu_im;
  int64_t z_offset;
};

// One complex embedding draw (pair) for a chunk of samples.
struct CeLaunch {
  const double2* bm_sc;
  const double* bm_lg;
  int M, m, pair, n_layers, level;
  int dim;  // 2 or 3
  int t_re, t_im;
  double mu_re, mu_im;
  uint64_t seed;
  int64_t first, n_samples;
};

// M = 2^k, or M = 3 2^k with the cut-off embedding (cutoff = 1, 2-norm).
int ce_build_table(int m, int M, double sigma2, double lam, int norm_r, int cutoff, void* scratch,
                   double* s64, float* s32, double* minmax_dev, void* tw64, void* tw32,
                   cudaStream_t st);
int ce_build_table3(int m, int M, double sigma2, double lam, int norm_r, void* scratch, double* s64,
                    float* s32, double* minmax_dev, void* tw64, void* tw32, cudaStream_t st);
int ce_sample_fp64(const CeLaunch& L, const double* scale, const void* tw, void* W, double* g,
                   cudaStream_t st);
int ce_sample_fp32(const CeLaunch& L, const float* scale, const void* tw, void* W, float* g,
                   cudaStream_t st);
// Kernel launches the samplers queued on this host thread since the last call (and reset).
int ce_launches_take();
size_t ce_w_bytes_per_sample(int m, int M, bool fp32, int dim);
// Box-Muller tables: sc 1024 double2, lg 3*128 doubles.
int bm_tables_build(double2* sc, double* lg, cudaStream_t st);

// ---------------------------------------------------------------- solve ---
// Where the permeability of a system comes from.
enum KSource : int {
  KSRC_FIELDS = 0,   // g fields of the chunk + layer map from the interfaces
  KSRC_CONST = 1,    // Ex. 1: per-layer constants exp(mu + sigma Z) + layer map
  KSRC_ARRAY = 2,    // a caller-given k array per system (fine systems only)
};

struct SolveArgs {
  // systems: fine systems [0, n_samples), then n_coarse per sample; a launch
  // solves systems [sys_begin, sys_end) (sys_end 0: all of them)
  int64_t n_samples;
  int64_t sys_begin, sys_end;
  int n_coarse;        // 0, 1 (plain, offset (0,0)) or 4 (CGV offsets)
  int m;               // fine cells per side
  int ksrc;
  int cgv_on_k;        // coarse k = strided fine k (CGV mode 2)
  int level;
  uint64_t seed;
  int64_t first;       // sample index of chunk entry 0
  int n_layers;
  int geometry;        // 0 horizontal interfaces; 1 sloped lines (four ends)
  double if_lo, if_hi;
  double line_lo[4], line_hi[4];
  double mu[MAX_LAYERS_DEV];
  double sigma[MAX_LAYERS_DEV];
  const void* g;       // fields [sample][layer][j][i] (double or float by precision)
  const double* k;     // KSRC_ARRAY: [system][j][i]
  double tol;
  int max_it;
  int problem;         // 2: outflow (Model Problem 2); 1: local average, f = 1, Dirichlet 0 (Model Problem 1)
  double box[4];       // problem 1: x0, x1, y0, y1 of D*
  double inner_tol;    // mixed: relative tolerance of each FP32 inner solve (reliable: the update trigger)
  int reliable;        // mixed: FP32 CG with reliable updates instead of restarted refinement
  int mg_gamma;        // multigrid cycle: 1 V, 2 W (set from the launch plan)
  int mg_nu;           // red-black sweep pairs before and after the coarse correction
  int mg_nu_coarse;    // the same on the coarser levels (0: mg_nu)
  // workspace
  int use_smem;
  size_t ws_stride;    // bytes per block slot (global workspace)
  unsigned char* ws;   // global workspace base (n_blocks * ws_stride)
  size_t ws64_stride;  // > 0: bytes per group of FP64 refinement vectors in global memory at ws64
  unsigned char* ws64;
  size_t stage_bytes;  // > 0: dynamic shared memory per block for the staged half sweeps
  // outputs per system
  double* q;           // outflow Q (NaN when not converged)
  int32_t* iters;      // CG iterations
  double* p_out;       // optional pressure of fine systems [sample][j][i]
};

// Launch shape of the solver for one system size (solve.cu).
struct SolvePlan {
  int warp;              // one warp per system
  int cluster;           // > 0: one thread-block cluster of this many blocks per system
  int blocks_per_group;  // blocks per system (cluster size, else 1)
  int max_groups;        // systems that can be resident at once on the GPU
  int threads;           // threads per block
  int groups_per_block;  // systems solved side by side in one block
  int blocks_per_sm;     // occupancy
  int use_smem;          // workspace in shared memory (else global, ws_stride per group)
  size_t ws_stride;      // bytes of workspace per group
  size_t ws64_stride;    // > 0 (prec 1, 2 on chip): global bytes per group of the FP64 refinement vectors
  size_t smem_bytes;     // dynamic shared memory per block
  size_t stage_bytes;    // of which the staging buffers of the streamed half sweeps (0: none)
  int cap_blocks_per_sm; // > 0: launch at most this many blocks per SM (L2 residency)
  int gamma;             // multigrid cycle index: 1 V-cycle, 2 W-cycle
  int nu;                // smoothing: red-black sweep pairs before and after the coarse correction
  int nu_coarse;         // the same on the coarser levels (0: nu)
  double inner_tol;      // mixed precision: relative tolerance of each FP32 inner solve
  int reliable;          // mixed precision: reliable updates (inner_tol = residual drop between updates)
};

// The work of one solver launch: items (ranges of systems, each with its own
// arguments: level, fields, outputs, multigrid and refinement settings) laid
// end to end.  Work index w < start[n] is system a[k].sys_begin + (w -
// start[k]) of the item k with start[k] <= w < start[k + 1]; the groups take
// work indices from the counter *next (zero at launch).  All items of a
// launch share its launch shape and workspace (ws, ws_stride, ws64,
// ws64_stride, use_smem and stage_bytes of item 0, sized for the largest
// item).  Passed by value as the kernel parameter (about 5.4 KB).
constexpr int kMaxSolveItems = 12;
struct SolveList {
  int n;
  unsigned long long* next;
  int64_t start[kMaxSolveItems + 1];
  SolveArgs a[kMaxSolveItems];
};

size_t solve_ws_bytes(int m, int prec);
int solve_plan(int m, int prec, SolvePlan* plan);
// An explicit plan: mode 0 block of `threads`, 1 warp, 2 cluster of `cluster` blocks.
int solve_plan_mode(int m, int prec, int mode, int threads, int cluster, SolvePlan* plan);
// Launch plans worth timing for one system size (the default first); returns the count.
int solve_plan_candidates(int m, int prec, SolvePlan* out, int max_out);
// Groups (systems in flight) and blocks of a launch for n_sys systems;
// max_groups_cap > 0 bounds the groups (workspace budget).  The global
// workspace (plan.use_smem == 0) must hold groups * ws_stride bytes.
int64_t solve_groups(const SolvePlan& plan, int64_t n_sys, int nsm, int64_t max_groups_cap, int64_t* n_blocks);
int solve_launch(const SolveArgs& a, int prec, const SolvePlan& plan, int n_blocks, cudaStream_t st);
// Write a plan's launch settings (workspace layout, multigrid and refinement
// settings) into an item's arguments.
void solve_apply_plan(SolveArgs& a, const SolvePlan& plan);
// One launch over the items of L with plan's shape (2-D, prec 0 or 1; the
// caller has applied each item's own plan settings); -1 for other precisions.
int solve_launch_list(const SolveList& L, int prec, const SolvePlan& plan, int n_blocks, cudaStream_t st);
// Shared-memory limits of the list kernels (call before the first list launch, outside stream capture).
int solve_list_prepare();
// The same for the 3-D seven-point systems (solve3.cu; prec 0 or 1; modes 0 block, 2 cluster).
size_t solve3_ws_bytes(int m, int prec);
int solve3_plan(int m, int prec, SolvePlan* plan);
int solve3_plan_mode(int m, int prec, int mode, int threads, int cluster, SolvePlan* plan);
int solve3_plan_candidates(int m, int prec, SolvePlan* out, int max_out);
int solve3_launch(const SolveArgs& a, int prec, const SolvePlan& plan, int n_blocks, cudaStream_t st);

// --------------------------------------------------------------- reduce ---
struct LevelSumsDev {
  double s[10];  // qf, qf2, qc, qc2, y, y2, qcg, qcg2, yg, yg2
  long long n, n_failed, iters;
};

// Gather system Q's of a chunk into the per-sample outputs.
// it_acc[0] += iterations of all systems, it_acc[1] += cells x iterations of
// the fine systems, it_acc[2] += the same of the coarse systems.
// cells_f / cells_c: cells of a fine / coarse system; Q_cgv is the mean of the
// n_coarse (4 or 8) coarse Q's, summed left to right.
int gather_launch(const double* q_sys, const int32_t* it_sys, int64_t n_samples, int n_coarse,
                  int cgv, int64_t cells_f, int64_t cells_c, double* qf, double* qc, double* qcg,
                  int32_t* iters, int64_t* it_acc, cudaStream_t st);
// Level sums in two launches (per-block partials, then a fixed-order
// combine); ws must hold reduce_ws_bytes().
size_t reduce_ws_bytes();
int reduce_launch(const double* qf, const double* qc, const double* qcg, int64_t n, int cgv,
                  const int64_t* it_acc, LevelSumsDev* out, void* ws, cudaStream_t st);
int philox_launch(uint64_t seed, uint64_t level, uint64_t sample, uint64_t stream,
                  uint64_t first_call, int64_t n_calls, uint64_t* out, cudaStream_t st);
int interfaces_launch(const SolveArgs& a, int64_t n, double* eta, cudaStream_t st);
int const_fields_launch(const SolveArgs& a, int64_t n, int64_t cells, double* g, cudaStream_t st);
int normals_launch(uint64_t seed, uint64_t level, uint64_t sample, uint64_t stream, uint64_t first_call,
                   int64_t n_calls, const double2* sc, const double* lg, int fp32, double* out,
                   cudaStream_t st);
int f32_to_f64_launch(const float* in, double* out, int64_t n, cudaStream_t st);

// Status of the last solver launch made by this host thread (solve_launch,
// solve3_launch), so that a caller can report the launch's own error.
cudaError_t& last_launch_error();
// Record `what` as this thread's mlmc_last_error() text; returns `code`.
int set_error(int code, const char* what);

}  // namespace mlmc

/*
 * mlmc.h -- C ABI of the GB300 MLMC level-batch library (libmlmc.so).
 *
 * The library computes, on one GPU, the per-level sample batch of the
 * multilevel Monte Carlo method of Park & Teckentrup (arXiv 1506.04694) for
 * steady Darcy flow in randomly layered media, Model Problem 2 of Sec. 3.4:
 *   -div(k grad p) = 0 on (0,1)^2, p = 1 at x1 = 0, p = 0 at x1 = 1,
 *   no flow at x2 = 0 and x2 = 1, quantity of interest Q = outflow at x1 = 1.
 * Each sample draws a layered permeability (Sec. 2, Ex. 1 piecewise constant
 * or Ex. 2 piecewise log-normal with the exponential covariance of Eq. 2.3,
 * sampled by circulant embedding), assembles the cell-centred five-point
 * finite-volume system of Eq. 3.3 with harmonic face averages, solves it,
 * and reduces Q into the level sums of the estimators of Eq. 3.6 (plain) and
 * Eq. 4.2 (Coarse Grid Variates, coarse samples from Eq. 4.1).
 *
 * Conventions shared by every entry point:
 *  - Return value: 0 = success; MLMC_SOME_FAILED (+1) = completed but some
 *    samples did not converge (their Q is NaN and they are left out of the
 *    sums); a negative value is an error, described by mlmc_error_string().
 *  - "device pointer" arguments must point to memory of the context's GPU;
 *    they are owned by the caller.  "host pointer" arguments are owned by the
 *    caller too.  The context owns every internal workspace and table.
 *  - All GPU work is issued on the stream given to mlmc_create(); a call
 *    returns after its host-visible results are complete (except
 *    mlmc_solve_k_static, which only queues its work).
 *  - A context is used by one host thread at a time; different contexts
 *    are independent.
 *  - There is no CPU fallback: without a usable GPU, mlmc_create() fails.
 *  - Grid layout: level l has m = m0 * 2^l cells per side; cell (i, j),
 *    0-based, has centre ((i + 1/2)/m, (j + 1/2)/m); per-sample arrays are
 *    stored row-major as [j][i] (x1, the flow direction, fastest).
 *  - Random numbers: sample i of level l with seed s is a pure function of
 *    (s, l, i), drawn from Philox4x64-10 (Salmon et al. 2011) with key (s, 0)
 *    and counter (call index, i, l, stream); see mlmc_philox_words().
 */
#ifndef MLMC_H
#define MLMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLMC_MAX_LAYERS 8

#if defined(__GNUC__)
#define MLMC_API __attribute__((visibility("default")))
#else
#define MLMC_API
#endif

/* Error codes. */
#define MLMC_OK 0
#define MLMC_SOME_FAILED 1
#define MLMC_ERR_ARG (-1)       /* invalid argument */
#define MLMC_ERR_CUDA (-2)      /* a CUDA runtime call failed */
#define MLMC_ERR_NOMEM (-3)     /* device allocation failed */
#define MLMC_ERR_EMBED (-4)     /* circulant embedding not non-negative up to padding 16 */
#define MLMC_ERR_NODEV (-5)     /* no usable CUDA device */
#define MLMC_ERR_TOOBIG (-6)    /* size above a documented maximum */

/* Model and solver parameters (Sec. 2 Ex. 1 / Ex. 2, Sec. 3.4, Sec. 3.5, Sec. 4.1). */
typedef struct mlmc_model {
  int32_t n_layers;            /* 1..8 horizontal layers; layer 0 is the bottom one */
  int32_t k_kind;              /* 0: k_t = exp(mu_t + sqrt(sigma2_t) Z_t), Z_t ~ N(0,1) (Ex. 1)
                                  1: k_t = exp(g_t), g_t Gaussian field, mean mu_t, covariance
                                     sigma2_t exp(-||x - y||_r / lam_t) (Ex. 2, Eq. 2.3) */
  double if_lo, if_hi;         /* the n_layers-1 interface heights are U(if_lo, if_hi) draws,
                                  sorted ascending; a row whose centre lies at or above
                                  interface t is above it */
  double mu[MLMC_MAX_LAYERS], sigma2[MLMC_MAX_LAYERS], lam[MLMC_MAX_LAYERS];
                               /* k_kind 1: layers are taken in order and paired greedily
                                  with an earlier layer of equal (sigma2, lam) whose complex
                                  draw has its imaginary part free; each draw f (Philox
                                  stream 2 + f) has its own embedding table per level */
  int32_t norm_r;              /* 1 or 2: the l_r norm of Eq. 2.3 */
  int32_t m0, L;               /* coarsest cells per side (power of two, 2..4096); finest level */
  int32_t cgv;                 /* 0: plain coupling, coarse sample = fine fields at the even
                                     cells (offset (0,0)) composed on the coarse layer map;
                                  1: Coarse Grid Variates, Eq. 4.1 / 4.2, the four offsets
                                     (0,0), (1,0), (0,1), (1,1) of the per-layer fields (3-D:
                                     the eight offsets, ox fastest);
                                  2: Coarse Grid Variates on the composed k */
  int32_t prec;                /* 0: FP64 throughout;
                                  1: FP32 multigrid-preconditioned CG inside FP64 iterative
                                     refinement (FP64 residual, solution, QoI and sums),
                                     FP32 circulant-embedding FFT;
                                  2: as 1, with the multigrid preconditioner's face
                                     coefficients stored in BF16 on every level (the CG
                                     operator and the FP64 residual keep FP32 faces);
                                  3: FP64 fields, faces, CG (flexible, Polak-Ribiere beta),
                                     stopping test and QoI, with an FP32 multigrid
                                     preconditioner (faces rounded to FP32) */
  double tol;                  /* stop when ||b - A x||_2 < tol ||b||_2 (Sec. 3.5 uses 1e-10) */
  int32_t max_it;              /* cap on CG iterations per solve (sum over refinement sweeps) */
  int32_t problem;             /* 0 or 2: Model Problem 2 of Sec. 3.4 (p = 1 / 0 at x1 = 0 / 1, no
                                     flow elsewhere, Q = outflow at x1 = 1);
                                  1: Model Problem 1 of Sec. 3.4 (f = 1, p = 0 on the whole
                                     boundary, Q = mean of p over the box qoi_box) */
  double qoi_box[4];           /* problem 1: D* = [x0, x1] x [y0, y1] inside (0,1)^2; all zero
                                  selects [7/16, 9/16]^2 around x* = (1/2, 1/2) */
  int32_t geometry;            /* 0: horizontal interfaces (if_lo, if_hi above);
                                  1: the three layers of Sec. 3.4 cut by the lines
                                     (0, y1)-(1, y2) (upper) and (0, y3)-(1, y4) (lower),
                                     y_t ~ U(line_lo[t], line_hi[t]); needs n_layers = 3; a cell
                                     belongs to the layer counted by the lines at or below its
                                     centre */
  double line_lo[4], line_hi[4];  /* geometry 1; all zero selects the paper's ranges
                                  (0.8, 0.9), (0.6, 0.7), (0.2, 0.3), (0.4, 0.5) */
  int32_t dim;                 /* 0 or 2: the unit square; 3: the unit cube of Sec. 3.4, the layers
                                  extruded along x3 (a cell's layer depends on (x1, x2) only),
                                  m^3 cells with the seven-point system (face coefficients as in
                                  2-D, Q = h * outflow face sum), 3-D embedding draws, CGV over
                                  the 8 offsets (ox, oy, oz) in the order ox fastest; needs
                                  m0 * 2^L <= 128, prec 0 or 1; problem 1 takes D* = [x0, x1] x
                                  [y0, y1] x [y0, y1] */
  int32_t embed;               /* circulant embedding of k_kind 1 (Sec. 3.4 cites the method):
                                  0: padding M = 2m, else (2-D, 2-norm, m >= 8) the cut-off
                                     embedding at M = 3m, else 4m, 8m, 16m; the cut-off one
                                     keeps the covariance of Eq. 2.3 up to the largest
                                     distance between cell centres, sqrt(2)(m - 1)/m, then
                                     tapers it to zero at M/(2m) with a C^1 cubic, so it
                                     samples the same fields law on a smaller torus;
                                  1: periodic embeddings with M = 2m, 4m, 8m, 16m only */
} mlmc_model;

/* Level sums over a range of samples (Eq. 3.6 and Eq. 4.2): Q_f is Q_l of the
 * sample, Q_c the plain coarse Q_{l-1} (0 at level 0), Y = Q_f - Q_c;
 * Q_cg = the mean of the 2^d CGV coarse Q's (four in 2-D, eight in 3-D,
 * summed in offset order), Y_g = Q_f - Q_cg (zero when
 * cgv == 0).  Sums are FP64 with Neumaier compensation in a fixed order. */
typedef struct mlmc_level_sums {
  int64_t n;                   /* samples summed (converged ones) */
  int64_t n_failed;            /* samples whose solve did not converge */
  int64_t iters_total;         /* CG iterations over all solves of the range */
  double s_qf, s_qf2, s_qc, s_qc2, s_y, s_y2;
  double s_qcg, s_qcg2, s_yg, s_yg2;
  double seconds;              /* wall time of the call */
} mlmc_level_sums;

#define MLMC_MAX_LEVELS 12

/* Result of mlmc_estimate(). */
typedef struct mlmc_estimate_out {
  double q_hat;                        /* MLMC estimate of E[Q_L] (Eq. 3.6 / Eq. 4.2) */
  double var_hat;                      /* sum_l V_l / N_l, held <= eps^2 / 2 */
  int64_t N[MLMC_MAX_LEVELS];          /* samples per level */
  double V[MLMC_MAX_LEVELS];           /* unbiased sample variance of the level correction */
  double mean[MLMC_MAX_LEVELS];        /* sample mean of the level correction */
  double C[MLMC_MAX_LEVELS];           /* cost per sample used in the sample-size rule */
  mlmc_level_sums sums[MLMC_MAX_LEVELS];
  int32_t rounds;                      /* top-up rounds after the pilot */
  double seconds;                      /* wall time */
  /* Bias of the finest level, reported only (L is fixed by the model; the
   * sample-size rule controls the sampling error alone, Eq. 3.7): the weak
   * rate alpha is the least-squares slope of -log2 |mean_l| over the levels
   * l >= 1 with a nonzero mean (at least two of them; else alpha = 1, the
   * rate Sec. 3.4 observes for the outflow), floored at 0.5, and
   * bias = |mean_L| / (2^alpha - 1).  NaN when L = 0. */
  double alpha;
  double bias;
  int32_t bias_flag;                   /* 1: bias > eps / sqrt(2), the bias half of the MSE budget */
} mlmc_estimate_out;

typedef struct mlmc_ctx mlmc_ctx;

/* Create a context on CUDA device `device` for `model`, issuing work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  Builds
 * the circulant-embedding tables of every level (the first embedding in the
 * order of model.embed whose eigenvalues are all >= -1e-13 max; the
 * remaining negative ones are set to 0).
 * Errors: MLMC_ERR_ARG (bad model), MLMC_ERR_NODEV, MLMC_ERR_EMBED, MLMC_ERR_NOMEM,
 * MLMC_ERR_CUDA.  On error *out is NULL. */
MLMC_API int mlmc_create(int device, const mlmc_model* model, void* cuda_stream, mlmc_ctx** out);

/* Release the context and all its device memory.  NULL is allowed. */
MLMC_API void mlmc_destroy(mlmc_ctx* ctx);

/* Samples first .. first+n-1 of level `level` (Eq. 3.6 / Eq. 4.2).
 * qf, qc, qc_cgv: device pointers to n doubles each, or NULL; receive Q_l,
 *   the plain coarse Q_{l-1} (0 at level 0) and the CGV coarse average (NaN
 *   when cgv == 0).  Failed samples hold NaN.
 * iters: device pointer to n int32 (CG iterations of the fine solve) or NULL.
 * sums: host pointer, required; receives the level sums of the range.
 * Returns MLMC_OK, MLMC_SOME_FAILED or a negative error. */
MLMC_API int mlmc_level_batch(mlmc_ctx* ctx, int level, int64_t first, int64_t n, uint64_t seed,
                     double* qf, double* qc, double* qc_cgv, int32_t* iters,
                     mlmc_level_sums* sums);

/* Same as mlmc_level_batch() but qf, qc, qc_cgv, iters are HOST pointers (or
 * NULL); the library copies results back before returning. */
MLMC_API int mlmc_level_batch_host(mlmc_ctx* ctx, int level, int64_t first, int64_t n, uint64_t seed,
                          double* qf, double* qc, double* qc_cgv, int32_t* iters,
                          mlmc_level_sums* sums);

/* Adaptive MLMC estimate with sampling error sum_l V_l/N_l <= eps^2/2 (the
 * even split of Eq. 3.7): n_pilot samples per level, then repeated top-ups
 * to N_l = ceil(2 eps^-2 sqrt(V_l/C_l) sum_k sqrt(V_k C_k)) until no level
 * needs more (at most 10 rounds).  cost_model 0: C_l = m_l^d (1 + n_coarse/2^d)
 * with n_coarse = 0 at level 0, 1 plain, 2^d CGV (deterministic); 1: C_l =
 * measured seconds per sample of the pilot (64-sample batches: latency more
 * than throughput); 2: C_l = the per-sample GPU time of each level measured
 * by mlmc_calibrate_costs() or set by mlmc_set_costs() (deterministic while
 * those costs are kept).  out: host pointer, required.  Errors: MLMC_ERR_ARG
 * (eps <= 0, n_pilot < 2, cost_model not 0..2, cost_model 2 without costs). */
MLMC_API int mlmc_estimate(mlmc_ctx* ctx, double eps, uint64_t seed, int32_t n_pilot,
                  int32_t cost_model, mlmc_estimate_out* out);

/* Measure the cost C_l of one sample of each level for the estimator's
 * sample sizes (Eq. 3.7's N_l depend on the costs; cost_model 2 of
 * mlmc_estimate): the per-sample GPU time (CUDA events on the context stream:
 * fields, fine and coarse solves, reductions) of a batch of each level alone,
 * large enough to fill the GPU (2^26 cells, 64 to 65536 samples, from sample
 * index 2^40 on, so that no sample of real use is consumed), the faster of
 * two after one untimed batch, with the context's current launch plans (run
 * it after tuning).  The context keeps the costs; C (host array of L+1, or
 * NULL) receives them in seconds.  Errors: those of mlmc_level_batch(). */
MLMC_API int mlmc_calibrate_costs(mlmc_ctx* ctx, uint64_t seed, double* C);

/* Set the per-sample costs of cost_model 2 by hand (C: host array of L+1
 * positive values, seconds or any common unit), e.g. those an earlier
 * mlmc_calibrate_costs() returned, so that estimates in another process use
 * the same sample-size rule.  Errors: MLMC_ERR_ARG. */
MLMC_API int mlmc_set_costs(mlmc_ctx* ctx, const double* C);

/* mlmc_estimate() with a cap on the number of top-up rounds (0 = pilot only);
 * mlmc_estimate() is this call with max_rounds = 10.  After a call the
 * context keeps the estimator state (per-level sums, costs, rounds, seed,
 * eps) for mlmc_checkpoint(); after mlmc_resume() the next call with the same
 * seed starts from the loaded state instead of a pilot (the Philox streams
 * make the result identical to an uninterrupted run). */
MLMC_API int mlmc_estimate_ex(mlmc_ctx* ctx, double eps, uint64_t seed, int32_t n_pilot, int32_t cost_model,
                              int32_t max_rounds, mlmc_estimate_out* out);

/* Write the estimator state of the last mlmc_estimate / _ex call to a text
 * file (host path).  Format (version 2), one key per line: "mlmc_checkpoint
 * 2"; "model" n_layers k_kind norm_r m0 L cgv prec max_it problem geometry
 * dim embed; "model_if" if_lo if_hi; "model_tol" tol; "model_mu", "model_sigma2",
 * "model_lam" (8 values each), "model_qoi_box", "model_line_lo",
 * "model_line_hi" (4 each); then seed, eps, cost_model, rounds, levels and
 * one "level" line of counts, sums and cost per level.  Doubles carry 17
 * significant digits, so they read back exactly.
 * Errors: MLMC_ERR_ARG (no estimate yet, unwritable). */
MLMC_API int mlmc_checkpoint(mlmc_ctx* ctx, const char* path);

/* Check, on the host alone (no context or GPU needed), that the checkpoint
 * at `path` was written for `model`: every field that changes a sample's Q
 * or its failure must be equal (per-layer mu, sigma2 and, for log-normal
 * fields, lam, norm_r and embed below n_layers; the interface range with horizontal
 * layers; the box with Model Problem 1; the line ranges with the sloped
 * geometry; n_layers, k_kind, m0, L, cgv, prec, tol, max_it, problem,
 * geometry and dim always).  Merging level sums of another model into an
 * estimate would bias the telescoping sum of Eq. 3.6 without any error, so
 * mlmc_resume() runs this check first.  Returns 0 or MLMC_ERR_ARG, with the
 * first differing field named in mlmc_last_error(). */
MLMC_API int mlmc_checkpoint_check(const mlmc_model* model, const char* path);

/* Load a state written by mlmc_checkpoint() for the same model (checked by
 * mlmc_checkpoint_check()); the next estimate continues from it.
 * Errors: MLMC_ERR_ARG (unreadable, other model). */
MLMC_API int mlmc_resume(mlmc_ctx* ctx, const char* path);

/* Levels 0 .. n_levels-1 in one call: samples first[l] .. first[l]+n[l]-1 of
 * each level l (n[l] may be 0), the levels side by side on streams of their
 * own (forked from and joined back into the context stream; one after
 * another on the context stream while profiling is on), each with work
 * buffers of its own that the context keeps between calls, with a single
 * host synchronisation at the end; sums[l] (host array of
 * n_levels) receives the level sums of Eq. 3.6 / Eq. 4.2 as in
 * mlmc_level_batch().  use_graph != 0 captures the whole queue into one CUDA
 * graph (kept and relaunched while the arguments repeat); it needs a context
 * created on a non-default stream and is skipped while profiling is on (stage
 * timing puts events between the launches).  Under the work-queue schedule a
 * captured batch queues its phases as one chain on the context stream (the
 * graph of that chain ran faster than a graph of the side-by-side form).
 * Per-sample values are not returned (use mlmc_level_batch for those).
 * mlmc_estimate() runs its pilot and every top-up round through this call.
 * With the work-queue schedule (mlmc_set_schedule, the default) a 2-D batch
 * in precision 0 or 1 runs its solves as one persistent launch per launch
 * shape across all levels instead of one per level (no effect on results).
 */
MLMC_API int mlmc_multilevel_batch(mlmc_ctx* ctx, int32_t n_levels, const int64_t* first, const int64_t* n,
                                   uint64_t seed, int32_t use_graph, mlmc_level_sums* sums);

/* mlmc_multilevel_batch() with the per-sample results of every level copied
 * to host memory before returning (the multilevel form of
 * mlmc_level_batch_host(): the levels of a round run together, in the same
 * schedule and graph).  qf, qc, qc_cgv, iters: host arrays of n_levels
 * pointers (or NULL), each entry a host array of n[l] values (or NULL: not
 * copied); the values are those of mlmc_level_batch() (Q_f, Q_c, the CGV
 * average of Eq. 4.1, CG iterations).  Ownership stays with the caller.
 * Errors: as mlmc_multilevel_batch(). */
MLMC_API int mlmc_multilevel_batch_host(mlmc_ctx* ctx, int32_t n_levels, const int64_t* first, const int64_t* n,
                                        uint64_t seed, int32_t use_graph, double* const* qf, double* const* qc,
                                        double* const* qc_cgv, int32_t* const* iters, mlmc_level_sums* sums);

/* Result of mlmc_autotune(), per level. */
typedef struct mlmc_tune_report {
  int32_t threads[MLMC_MAX_LEVELS];            /* threads per block chosen */
  int32_t warp[MLMC_MAX_LEVELS];               /* 1: one warp per system; 2: the same with the
                                                  finest grid in registers (m = 16, prec 1) */
  int32_t cap_blocks_per_sm[MLMC_MAX_LEVELS];  /* 0: occupancy limit */
  int32_t cluster[MLMC_MAX_LEVELS];            /* > 0: blocks of the cluster that solves one system */
  int32_t gamma[MLMC_MAX_LEVELS];              /* multigrid cycle: 1 V, 2 W */
  int32_t nu[MLMC_MAX_LEVELS];                 /* red-black sweep pairs per smoothing, finest grid */
  int32_t nu_coarse[MLMC_MAX_LEVELS];          /* the same on the coarser grids */
  double inner_tol[MLMC_MAX_LEVELS];           /* prec 1, 2: relative tolerance of the FP32 inner solves */
  int32_t reliable[MLMC_MAX_LEVELS];           /* prec 1, 2: 1 = reliable updates (mlmc_set_solver) */
  int32_t candidates[MLMC_MAX_LEVELS];         /* plans timed */
  double ms_default[MLMC_MAX_LEVELS];          /* ms per sample, default plan */
  double ms_best[MLMC_MAX_LEVELS];             /* ms per sample, chosen plan */
  int32_t smem[MLMC_MAX_LEVELS];               /* 1: the chosen plan keeps a system's workspace in
                                                  shared memory (else global memory, streamed) */
  /* levels >= 1: the plan of the coarse systems (side m/2), tuned on them alone
     and run as a launch of its own after the fine systems' launch when the two
     launches beat one launch of all systems (c_threads = 0: one launch); the
     fields above are the fine systems' plan */
  int32_t c_threads[MLMC_MAX_LEVELS], c_warp[MLMC_MAX_LEVELS], c_cluster[MLMC_MAX_LEVELS];
  int32_t c_cap_blocks_per_sm[MLMC_MAX_LEVELS], c_gamma[MLMC_MAX_LEVELS], c_nu[MLMC_MAX_LEVELS];
  int32_t c_nu_coarse[MLMC_MAX_LEVELS];
  double c_inner_tol[MLMC_MAX_LEVELS];
  int32_t c_reliable[MLMC_MAX_LEVELS], c_smem[MLMC_MAX_LEVELS];
} mlmc_tune_report;

/* Times the candidate launch plans of the solver, for each level separately
 * for its fine systems and (levels >= 1) its coarse systems, which then run as
 * two launches with their own plans if that beats one launch of all systems
 * on the fine plan (candidates: one warp, one block of
 * 64/128/256/512 threads, or, for m >= 128, one thread-block cluster of 2, 4
 * or 8 blocks per system; all resident blocks or one per SM; for the
 * fastest of those, W-cycles, two smoothing sweep pairs on every grid, two
 * or three on the finest grid with one on the coarser ones, and with prec 1
 * or 2 an FP32 inner tolerance of 1e-4, 1e-5 or 1e-6, and reliable updates
 * after a residual drop of 1e-2 or 1e-3) on a probe batch of
 * each level (samples from index 2^40 on, so no sample of real use is
 * consumed) and keeps the fastest for that level's solves.  A plan changes
 * the path of the iteration (cycle, smoothing, inner tolerance, summation
 * order of the dot products), never the stopping test, so results agree to
 * the solver tolerance.  rep: host pointer or NULL. */
MLMC_API int mlmc_autotune(mlmc_ctx* ctx, uint64_t seed, mlmc_tune_report* rep);

/* Launch shapes for the work-queue schedule (no paper counterpart: a
 * throughput setting of this implementation).  mlmc_autotune() times each
 * level alone, where a level with few large systems pays for the tail of its
 * launch; in the work-queue schedule the systems of all levels that share a
 * launch shape fill each other's tails.  This pass, run after
 * mlmc_autotune() (or on the default plans), re-times whole adaptive
 * estimates (mlmc_estimate(ctx, eps, seed, n_pilot, cost_model), cost_model
 * 0, 1 or 2: one untimed, then the fastest of `reps` timed with CUDA events on the context
 * stream) while it changes the launch shape of each part with systems of
 * side >= 256 (the fine systems of a level, and its coarse systems as a
 * launch of their own), finest level first: a cluster plan tries one block
 * of 512 threads and the other cluster size (4 or 8), a block plan a cluster
 * of 4; each part keeps its cycle, smoothing and mixed-precision settings, and
 * a change stays only if the estimate gets faster by more than 0.5 %.
 * Only for 2-D contexts in precision 0 or 1 with schedule 1 (otherwise it
 * does nothing).  The estimates' state is not kept (the last estimate and a
 * pending resume are restored).  ms: host array of 2 or NULL, receives the
 * estimate's time before and after.  rep: host pointer or NULL, receives the
 * final plans (plan fields only).  Errors: MLMC_ERR_ARG, and those of
 * mlmc_estimate(). */
MLMC_API int mlmc_autotune_schedule(mlmc_ctx* ctx, double eps, uint64_t seed, int32_t n_pilot,
                                    int32_t cost_model, int32_t reps, double* ms, mlmc_tune_report* rep);

/* Fix the solver's launch plan of one level by hand (overrides
 * mlmc_autotune; all the level's systems in one launch): mode 0 = one block of `threads` (32..512, multiple of 32)
 * per system, 1 = one warp per system, 2 = one thread-block cluster of
 * `cluster` (2, 4, 8) blocks of 512 threads per system, 3 = one warp per
 * system with the finest grid in registers (m = 16, prec 1, 2-D; the
 * default there); gamma 1 = V-cycle,
 * 2 = W-cycle preconditioner; nu = 1..4 red-black sweep pairs before and
 * after each coarse correction; mode < 0 restores the built-in default
 * (V-cycle, nu = 1).  Errors: MLMC_ERR_ARG. */
MLMC_API int mlmc_set_launch(mlmc_ctx* ctx, int level, int32_t mode, int32_t threads, int32_t cluster,
                             int32_t gamma, int32_t nu);

/* Fix the launch plan of the coarse systems (side m/2) of level `level` >= 1
 * by hand: they then run as a launch of their own after the fine systems'
 * (whose plan mlmc_set_launch() or the default sets); arguments as in
 * mlmc_set_launch(), for the coarse size (mode 3 needs m/2 = 16, prec 1);
 * mode < 0 returns to one launch for all the level's systems.
 * Errors: MLMC_ERR_ARG. */
MLMC_API int mlmc_set_launch_coarse(mlmc_ctx* ctx, int level, int32_t mode, int32_t threads, int32_t cluster,
                                    int32_t gamma, int32_t nu);

/* Schedule of mlmc_multilevel_batch() (and so of mlmc_estimate()).
 * schedule 1 (the default): the work-queue schedule.  The fields of every
 * level's whole range are sampled first (each level on its own stream); then
 * the level ranges, split into fine and coarse systems where a level has a
 * coarse plan of its own, are grouped by launch shape (kernel, block,
 * cluster, shared memory, residency), and each group runs as ONE persistent
 * solver launch over all its systems, largest systems first, whose thread
 * groups take the next system from an atomic work counter (a group that drew
 * long solves takes fewer; no group waits on another).  Each system keeps its
 * own level's multigrid and refinement settings.  Then each level's gather
 * and reduction.  It applies to 2-D contexts in precision 0 or 1 while stage
 * profiling is off and the fields and per-system outputs of all levels'
 * ranges fit in 24 GB; otherwise the batch takes schedule 0.
 * schedule 0: one launch chain per level (fields, solves, gather chunk by
 * chunk), the levels side by side on their streams.
 * The two schedules give bit-identical results.  Errors: MLMC_ERR_ARG. */
MLMC_API int mlmc_set_schedule(mlmc_ctx* ctx, int32_t schedule);

/* A complete launch plan set by hand, as mlmc_autotune() or
 * mlmc_autotune_schedule() report it (so that a tuning result can be
 * replayed in another process): part 0 = the fine systems of `level` (or all
 * of them while the level has no coarse plan), part 1 = its coarse systems
 * (level >= 1) as a launch of their own.  mode, threads, cluster, gamma, nu
 * as in mlmc_set_launch() (mode 3 needs systems of side 16 and prec 1; no
 * mode < 0 here); nu_coarse 0..4 (0: nu) the sweep pairs on the coarser
 * grids; cap_blocks_per_sm >= 0 (0: the occupancy limit); reliable 0 / 1 and
 * inner_tol in (0, 0.5] as in mlmc_set_solver() (used with prec 1, 2).
 * Errors: MLMC_ERR_ARG. */
MLMC_API int mlmc_set_launch_ex(mlmc_ctx* ctx, int level, int32_t part, int32_t mode, int32_t threads,
                                int32_t cluster, int32_t gamma, int32_t nu, int32_t nu_coarse,
                                int32_t cap_blocks_per_sm, int32_t reliable, double inner_tol);

/* Mixed precision (prec 1, 2) of one level's solver, on top of its launch
 * plan (the autotuned or set one, else the default): reliable = 0 runs FP32
 * multigrid-preconditioned CG solves to the relative tolerance inner_tol
 * inside FP64 iterative refinement (each refinement sweep restarts the CG);
 * reliable = 1 runs one FP32 CG with reliable updates (Sleijpen and van der
 * Vorst, 1996): whenever its residual has fallen by inner_tol since the last
 * update, or after 16 iterations, the correction is added to the FP64
 * solution and the FP64 residual b - A x replaces the FP32 one, and the CG
 * carries on with its search direction.  Both stop on the same FP64 test
 * ||b - A x|| < tol ||b||.  inner_tol in (0, 0.5]; reliable = 1 needs a 2-D
 * context.  Errors: MLMC_ERR_ARG. */
MLMC_API int mlmc_set_solver(mlmc_ctx* ctx, int level, int32_t reliable, double inner_tol);

/* Padding of level `level` for the first embedding draw (pair 0): *M_out = M,
 * and the smallest / largest raw embedding eigenvalue before clipping (host
 * pointers, any may be NULL). */
MLMC_API int mlmc_ce_info(mlmc_ctx* ctx, int level, int32_t* M_out, double* lam_min, double* lam_max);

/* Raw Philox4x64-10 words for calls first_call .. first_call+n_calls-1 of one
 * (seed, level, sample, stream): out is a device pointer to 4*n_calls uint64,
 * call-major.  Stream 0 holds interface uniforms, 1 the Ex. 1 layer normals,
 * 2+f the complex normals of circulant-embedding field pair f. */
MLMC_API int mlmc_philox_words(uint64_t seed, uint64_t level, uint64_t sample, uint64_t stream,
                      uint64_t first_call, int64_t n_calls, uint64_t* out, void* cuda_stream);

/* Stage output for parity checks: the four standard normals of each Philox
 * call first_call .. first_call+n_calls-1 of one (seed, level, sample,
 * stream), in the order BM(u0,u1).re, BM(u0,u1).im, BM(u2,u3).re,
 * BM(u2,u3).im, where BM(ua, ub) = sqrt(-2 ln ua) (cos 2 pi ub, sin 2 pi ub)
 * (Box-Muller; the normals of Ex. 1 and of the circulant-embedding draw),
 * computed by the routine the field kernels of the context's precision use.
 * out: device pointer to 4*n_calls doubles. */
MLMC_API int mlmc_normals(mlmc_ctx* ctx, uint64_t seed, uint64_t level, uint64_t sample, uint64_t stream,
                          uint64_t first_call, int64_t n_calls, double* out);

/* Stage output for parity checks: the per-layer fields g_t of the fine grid of
 * samples first .. first+n-1 of `level` (Ex. 1 constants or Ex. 2 fields),
 * g: device pointer to n * n_layers * m * m doubles ([sample][t][j][i]; 3-D
 *   contexts n * n_layers * m^3, [sample][t][l][j][i]);
 * eta: device pointer to n * n_ends doubles or NULL: the sorted interfaces
 *   (geometry 0, n_ends = n_layers - 1) or the line ends y1..y4 (geometry 1,
 *   n_ends = 4). */
MLMC_API int mlmc_sample_fields(mlmc_ctx* ctx, int level, int64_t first, int64_t n, uint64_t seed,
                       double* g, double* eta);

/* Solve n independent systems of size m x m (m a power of two, 1..4096)
 * for given cell permeabilities, with the context's solver settings; a 3-D
 * context (dim 3) solves m x m x m systems (m <= 128), k and p [s][l][j][i].
 * k: device pointer to n*m*m (3-D: n*m*m*m) doubles ([s][j][i]), all > 0.
 * p: device pointer to n*m*m (3-D: n*m*m*m) doubles (pressure) or NULL.
 * q: device pointer to n doubles (outflow Q; NaN if not converged), required.
 * iters: device pointer to n int32 or NULL. */
MLMC_API int mlmc_solve_k(mlmc_ctx* ctx, int32_t m, int64_t n, const double* k, double* p, double* q,
                 int32_t* iters);

/* Same solve as mlmc_solve_k(), for callers that cannot allocate device
 * memory: a plug-in inside a host application that has already reserved
 * (nearly) all GPU memory for its own pool, or a latency-critical loop that
 * cannot afford the device-wide synchronisation of cudaMalloc / cudaFree.
 * The paper has no counterpart; this is a deployment variant of the solver.
 * It needs no context and calls no allocating routine: the per-block solver
 * workspace lives in a fixed 32 MiB array in the library's device memory,
 * which every GPU that loads the library holds until the process exits.
 *   device: CUDA device to run on (made current for the call, then restored).
 *   m, n, k, p, q, iters: as in mlmc_solve_k() (k, p, q, iters device
 *     pointers; p and iters may be NULL).
 *   tol, max_it, prec: solver settings as in mlmc_model.
 *   cuda_stream: cudaStream_t to queue the work on; the call returns after
 *     queuing it (results are ready when the stream reaches this point).
 * The first call on a device looks up the array's device address (one
 * cudaGetSymbolAddress per device); make that first call before any stream
 * capture.  Only systems with m <= 32 and prec 0 or 3 run in shared memory
 * alone; every other call keeps workspace in the array (with prec 1 or 2 and
 * m <= 32, the FP64 refinement vectors; above m = 32, the whole workspace of
 * each system in flight), so m > 512 returns MLMC_ERR_TOOBIG.  The array
 * bounds the systems in flight: at m = 256 it holds 5 to 8 of them, at
 * m = 512 one or two (the rest wait their turn), so large batches run with
 * less parallelism than mlmc_solve_k().
 * Every call shares the one array and the solver initialises everything it
 * reads, so nothing carries over between calls; calls that overlap on the
 * GPU (other streams, other threads) race on the array and must be ordered
 * by the caller.  On an error the text of mlmc_last_error() describes it.
 * Errors: MLMC_ERR_ARG, MLMC_ERR_NODEV, MLMC_ERR_TOOBIG, MLMC_ERR_CUDA. */
MLMC_API int mlmc_solve_k_static(int device, int32_t m, int64_t n, const double* k, double* p,
                                 double* q, int32_t* iters, double tol, int32_t max_it,
                                 int32_t prec, void* cuda_stream);

/* Per-stage device timing of a context, collected with CUDA events on the
 * context's stream while enabled (used by the benchmark for the roofline). */
#define MLMC_PROFILE_CLASSES 8

typedef struct mlmc_profile_stats {
  int64_t launches[4];     /* kernel launches: 0 field kernels (both FFT passes),
                              1 fused assembly + solve + QoI (all systems, or the fine ones when
                              the coarse systems have a plan of their own), 2 gather + level
                              reduction, 3 the coarse systems' solve launches */
  double ms[4];            /* summed event time of each stage */
  double cell_iters;       /* sum over all solves of (cells x CG iterations) */
  double cells;            /* sum over all solves of cells */
  double fft_row_points;   /* sum of M*M complex points transformed by the row pass */
  double fft_col_points;   /* sum of m*M complex points transformed by the column pass */
  double samples;          /* samples processed */
  double solve_flops;      /* algorithmic flops of the CG iterations: per cell-iteration 21 for CG
                              (23 with prec 3) plus (2.25 + 18 nu) per finest cell for the
                              multigrid cycle, times 4/3 (V-cycle) or 2 (W-cycle) for the coarser
                              grids; the cycle runs in FP32 with prec 1, 2, 3 */
  double fft_flops;        /* 5 log2(M) flops per complex point of every length-M transform of the
                              row and column passes (the radix-2 count), summed over levels */
  double solve_bytes;      /* algorithmic bytes of the CG iterations: cells x iterations x the bytes
                              one iteration moves when every pass reads its operands and writes its
                              results once (CG vectors, faces and diagonal, every multigrid level;
                              no reuse between passes) */
  double fft_bytes;        /* algorithmic bytes of the field passes: every complex intermediate
                              written once and read once, the fields written once */
  double cell_iters_c;     /* the part of cell_iters, solve_flops, solve_bytes due to the */
  double solve_flops_c;    /* coarse systems (stage 3 when they run as a launch of their own) */
  double solve_bytes_c;
  /* The work-queue launches of profiled multilevel batches (mlmc_set_schedule
   * 1; their time is also in ms[1]), summed per launch shape, at most
   * MLMC_PROFILE_CLASSES shapes (further ones are counted in ms[1] only). */
  int32_t n_classes;
  int32_t class_mode[MLMC_PROFILE_CLASSES];      /* 0 block, 1 warp, 2 cluster, 3 register path */
  int32_t class_threads[MLMC_PROFILE_CLASSES];   /* threads per block */
  int32_t class_cluster[MLMC_PROFILE_CLASSES];   /* blocks per cluster (0: none) */
  int32_t class_smem[MLMC_PROFILE_CLASSES];      /* 1: workspace in shared memory */
  int32_t class_levels[MLMC_PROFILE_CLASSES];    /* bit l: held systems of level l */
  int32_t class_launches[MLMC_PROFILE_CLASSES];
  double class_ms[MLMC_PROFILE_CLASSES];         /* summed event time of the launches */
  double class_cell_iters[MLMC_PROFILE_CLASSES]; /* cells x CG iterations of their systems */
  double class_flops[MLMC_PROFILE_CLASSES];      /* algorithmic flops, as solve_flops */
  double class_bytes[MLMC_PROFILE_CLASSES];      /* algorithmic bytes, as solve_bytes */
} mlmc_profile_stats;

/* enable != 0: reset the counters and start collecting; 0: stop. */
MLMC_API int mlmc_profile(mlmc_ctx* ctx, int enable);

/* Copy the counters collected so far (host pointer, required). */
MLMC_API int mlmc_profile_read(mlmc_ctx* ctx, mlmc_profile_stats* out);

/* Arithmetic peak of the GPU, measured (no paper counterpart: the roofline
 * denominator of the ALU-bound kernels, whose bound the paper's CPU setting
 * never needed).  Runs one kernel of independent fused multiply-add chains
 * (FP64 if fp64 != 0, else FP32) on every SM of `device` for `iters` rounds
 * of 32 FMAs per thread, timed with CUDA events after one warm-up launch, on
 * a stream of its own; *tflops (host pointer, required) receives 2 flops per
 * FMA / event time, *ms (host pointer or NULL) the event time.  Allocates
 * one value of device memory for the duration of the call.
 * Errors: MLMC_ERR_ARG, MLMC_ERR_NODEV, MLMC_ERR_NOMEM, MLMC_ERR_CUDA. */
MLMC_API int mlmc_fma_peak(int device, int fp64, int32_t iters, double* tflops, double* ms);

/* Human-readable text of an error code (static storage). */
MLMC_API const char* mlmc_error_string(int code);

/* Description of the last error on this thread (static storage). */
MLMC_API const char* mlmc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MLMC_H */

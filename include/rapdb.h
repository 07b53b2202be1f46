/*
 * rapdb.h -- C ABI of the GB300 (sm_103a) rAPDB solver for convex QCQPs.
 *
 * Problem (Sec. 2.1, eq. (QCQP), with the simple set X a box and no linear
 * equalities):
 *
 *     min_x  0.5 x'Q_0 x + c_0'x
 *     s.t.   g_i(x) = 0.5 x'Q_i x + c_i'x + d_i <= 0,   i = 1..m,
 *            lb <= x <= ub,
 *
 * with every Q_i symmetric positive semidefinite (the caller asserts this).
 * The paper writes q_i for c_i and r_i for d_i.  The solver is rAPDB:
 * APDB-yx (Sec. 3.2, eq. (apdb-yx-y) and its test function) or APDB-xy
 * (Algorithm 1 with eq. (backtracking)), monotone or non-monotone step sizes
 * (Remark on non-monotone step sizes, eq. (nonmonotone-tau)), restarted at a
 * fixed frequency (Algorithm 2; restart from the last iterate as in Sec. 5.1)
 * or adaptively on the smoothed gap (eq. (ada_restart)), with Euclidean
 * Bregman distances and the dual ball not imposed (Sec. 5.1).
 *
 * Conventions shared by every entry point:
 *   - Pointers marked "device" are CUDA device addresses (from cudaMalloc or
 *     torch); "host" pointers are ordinary host memory.  All arrays are
 *     dense, row-major, float32 unless stated.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call is ordered on that stream; calls that return
 *     results to the host (rapdb_solve, rapdb_kkt_residual, ...) synchronise
 *     the stream before returning.
 *   - Return value: RAPDB_OK or an error status; no exception or abort ever
 *     crosses the ABI.  rapdb_last_error(ctx) gives a one-line description of
 *     the last failure on that context (rapdb_last_error(NULL) for failures
 *     that happened before a context existed).
 *   - A context is not thread safe: one host thread at a time per context.
 */
#ifndef RAPDB_H
#define RAPDB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RAPDB_OK = 0,
  RAPDB_ERR_INVALID = 1,    /* bad argument: size, pointer, parameter, NaN input   */
  RAPDB_ERR_CUDA = 2,       /* a CUDA runtime call failed                          */
  RAPDB_ERR_NOMEM = 3,      /* device allocation failed                            */
  RAPDB_ERR_BACKTRACK = 4,  /* max_trials step-size reductions without acceptance  */
  RAPDB_ERR_MAXITER = 5,    /* max_iter iterations without reaching tol            */
  RAPDB_ERR_TIMEOUT = 6,    /* time_limit_s exceeded (checked on the device)       */
  RAPDB_ERR_NUMERIC = 7     /* NaN / Inf met in a reduction                        */
} rapdb_status;

typedef enum { RAPDB_YX = 0, RAPDB_XY = 1 } rapdb_variant;
/* Storage of the Q_i in the coupling pass.  F32: the caller's float32 Q is
 * read directly.  BF16: round-to-nearest-even copy.  FP8: E4M3 codes of the
 * symmetrically Jacobi-scaled matrix, Q~ = S C S with S = diag(s),
 * s_j = sqrt(Q_jj)/16, C = e4m3(256 * Q_jk / sqrt(Q_jj Q_kk)). */
typedef enum { RAPDB_F32 = 0, RAPDB_BF16 = 1, RAPDB_FP8 = 2 } rapdb_storage;

/* Dual set Y.  RAPDB_DUAL_NONNEG: y >= 0, the multipliers of the QCQP
 * 0.5x'Q_ix + c_i'x + d_i <= 0.  RAPDB_DUAL_SIMPLEX: y on the simplex
 * {y >= 0, sum y = dual_radius}, which turns the problem into
 * min_x f(x) + dual_radius * max_i g_i(x), the min-max form of the paper's
 * kernel-learning experiment (Sec. 5.2, eq. min-max-KML); the dual start y0
 * must lie on the simplex. */
typedef enum { RAPDB_DUAL_NONNEG = 0, RAPDB_DUAL_SIMPLEX = 1 } rapdb_dual_set;
typedef enum { RAPDB_Q0_DENSE = 0, RAPDB_Q0_DIAG = 1, RAPDB_Q0_ZERO = 2 } rapdb_q0_kind;
typedef enum { RAPDB_RESTART_NONE = 0, RAPDB_RESTART_FIXED = 1, RAPDB_RESTART_GAP = 2 } rapdb_restart;

/* Solver parameters.  rapdb_default_params() fills the paper's experiment
 * settings (Sec. 5.1): eta = 0.7; yx: c_alpha = 0.4, delta = 0.5; xy:
 * c_alpha = 0.25, c_beta = 0.3, delta = 0.4; xi = 0.04, q = 1/2; first gap
 * evaluation at k = 50 (yx) / 100 (xy). */
typedef struct {
  int32_t variant;            /* rapdb_variant                                        */
  int32_t c_nm;               /* 0 monotone, 1 non-monotone step rule                 */
  int32_t backtracking;       /* 0: fixed step tau_bar, every trial accepted          */
  int32_t restart;            /* rapdb_restart                                        */
  double mu;                  /* strong convexity modulus used by gamma_{k+1}         */
  double c_alpha, c_beta, delta, eta;
  double tau_bar;             /* first trial step of every run (of the first run only  */
                              /*    with restart_warm_tau)                            */
  double gamma0;              /* sigma = gamma * tau                                  */
  int32_t restart_period;     /* fixed restart: iterations per run (Algorithm 2's K^) */
  int32_t restart_from_average; /* 1: restart from the weighted average (Algorithm 2)   */
  double xi, q;               /* smoothed gap parameters (eq. (ada_restart))           */
  int32_t gap_first, gap_every; /* gap schedule: first evaluation, then period          */
  int32_t storage;            /* rapdb_storage                                        */
  int32_t refine;             /* 1: compensated (double-float) float32 products: from */
                              /*    the start with F32 storage; BF16/FP8 storage      */
                              /*    switches to them when a precision check (restart  */
                              /*    boundaries, every restart_period/4 iterations)    */
                              /*    finds a stall, the stored problem solved, or the  */
                              /*    true residual above twice the stored level's.     */
                              /*    BF16/FP8 storage with pack_sym starts instead at  */
                              /*    the quantised-increment level: the trial products */
                              /*    are U^k + Q~ d, the increment Q~ d read from the  */
                              /*    packed BF16/FP8 tiles and U^k a compensated       */
                              /*    float32 product re-formed (anchored) by the       */
                              /*    precision check every 64 accepted iterations (and */
                              /*    whenever the level's own residual reaches tol);   */
                              /*    it switches to the float32 tiles when four checks */
                              /*    in a row find no true residual below the lowest   */
                              /*    one so far while the level's own residual misses  */
                              /*    the true one by more than half of it              */
  double stall_ratio;         /* stall: the true rel KKT fell by less than this factor */
                              /*    since the previous precision check               */
  int32_t max_iter, max_trials, kkt_every;
  int32_t use_graph;          /* 1: loop bodies captured in a CUDA graph of 32 bodies */
                              /*    (two launches kept in flight); 0: host launches    */
                              /*    the kernels of 16 bodies at a time                */
  double tol;                 /* stop when rel KKT <= tol (checked every kkt_every)  */
  double time_limit_s;        /* <= 0: none                                           */
  int32_t rows_per_block;     /* coupling pass tile height; 0 = autotune at create   */
  int32_t gap_inner_max;      /* inner iterations of the smoothed-gap box QP          */
  int32_t pass_variant;       /* tile variant when rows_per_block > 0 (0..9, see     */
                              /* rapdb_get_tile); ignored when autotuning           */
  int32_t dual_set;           /* rapdb_dual_set: y >= 0 (the QCQP's multipliers) or  */
                              /* y on the simplex {y >= 0, sum y = dual_radius} (the */
                              /* min-max kernel-learning problem, Sec. 5.2)         */
  double dual_radius;         /* the simplex's sum (> 0), used with RAPDB_DUAL_SIMPLEX */
  int32_t restart_warm_tau;   /* 1: a restart starts from the last accepted tau       */
                              /*    instead of tau_bar (0, the paper's reset)          */
  int32_t pack_sym;           /* 1: symmetric block packing.  The context keeps the   */
                              /*    upper block triangle of every float32 Q_i in      */
                              /*    128 x 128 tiles (about half of Q's bytes, on top  */
                              /*    of Q), and the incremental trial passes and the   */
                              /*    smoothed gap's passes read each tile once for its */
                              /*    rows and, transposed, for its columns: half the   */
                              /*    bytes of a row-streaming pass.  BF16/FP8 storage  */
                              /*    also keeps its codes in the same tiles (a half /  */
                              /*    a quarter of the float32 tiles' bytes), read by   */
                              /*    the trials of the quantised-increment level on    */
                              /*    the tcgen05 tensor cores (the right-hand side     */
                              /*    split into exact pieces of the codes' type; the   */
                              /*    products meet the float32 error bound of the      */
                              /*    stored matrices).                                 */
                              /*    Needs refine = 1, exactly symmetric Q_i (checked  */
                              /*    at create: RAPDB_ERR_INVALID) and a single-       */
                              /*    instance context; rows_per_block and              */
                              /*    pass_variant are ignored (the other passes use    */
                              /*    64-row items of tile variant 1, 8 for FP8).       */
                              /*    Results are                                       */
                              /*    reproducible run to run; they differ from an      */
                              /*    unpacked context's in rounding only.              */
} rapdb_params;

typedef struct {
  int32_t iters;              /* accepted iterations                                  */
  int32_t trials;             /* test evaluations = coupling passes in the loop      */
  int32_t restarts;
  int32_t precision_switches;
  int32_t passes;             /* all coupling passes (trials + setup + gap + KKT32)  */
  int32_t status;             /* rapdb_status of the solve                           */
  double rel_kkt, r_stat, r_feas;
  double obj;                 /* 0.5 x'Q_0 x + c_0'x at the returned x              */
  double seconds;             /* device time of the solve (CUDA events)             */
  int64_t launches;           /* kernels this call launched (device loop + set-up)  */
  int32_t switch_iter;        /* iteration of the first precision switch (-1: none) */
  int32_t reserved_;
} rapdb_info;

typedef struct rapdb_ctx rapdb_ctx;

/* Fill *p with the paper's settings for `variant` (rapdb_variant), fixed
 * restart every 200 iterations, tol 1e-6, max_iter 50000, max_trials 60,
 * tau_bar = gamma0 = 1, F32 storage. */
void rapdb_default_params(rapdb_params *p, int32_t variant);

/* Create a single-instance context.
 *   n  > 0 variables, 0 <= m <= 6400 constraints (m = 0: box-constrained QP, which
 *   needs q0_kind = DENSE so that one matrix is streamed).
 *   q0_kind: DENSE -> Q holds (m+1) matrices, Q_0 first; DIAG -> Q holds the
 *            m constraint matrices and q0diag (device, n) the diagonal of Q_0;
 *            ZERO -> Q holds the m constraint matrices, Q_0 = 0.
 *   Q     device, (M, n, n) float32, M = m+1 (DENSE) or m; symmetric.
 *   c     device, (m+1, n): row 0 = c_0, row i = c_i.
 *   d     device, (m,): the constants d_i (may be NULL when m = 0).
 *   lb,ub device, (n,), lb <= ub.
 *   lb,ub may be infinite (lb = -inf, ub = +inf) but not NaN.
 * Ownership: with F32 storage, n % 4 == 0 and Q 16-byte aligned the context
 * BORROWS Q (no copy): it must stay alive and unchanged until rapdb_destroy.
 * Otherwise the context owns a padded copy (F32 rows padded to a multiple of 4,
 * BF16 to 8, FP8 to 16 elements).  With refine = 1 the float32 Q is borrowed
 * as well.  c, d, lb, ub, q0diag are copied.  Errors: RAPDB_ERR_INVALID for
 * sizes, NULL pointers, lb > ub, a negative diagonal entry of some Q_i or a
 * NaN in the data; RAPDB_ERR_NOMEM / RAPDB_ERR_CUDA otherwise. */
rapdb_status rapdb_create(rapdb_ctx **out, int64_t n, int64_t m, int32_t q0_kind,
                          const float *Q, const float *q0diag, const float *c,
                          const float *d, const float *lb, const float *ub,
                          const rapdb_params *p, void *stream);

/* rapdb_create with a block of linear equalities A_eq x = b_eq (the equality
 * block of the paper's problem class, eq. NCP; for instance the constraint
 * b'x = 0 of the kernel-learning problem, Sec. 5.2).
 *   p_eq  >= 0 equalities (p_eq = 0 is rapdb_create).
 *   A_eq  device, (p_eq, n) float32 row-major; b_eq device, (p_eq,) float32
 *         (both copied).
 * Each equality a_k'x - b_k is handled as constraint m + k (k = 1..p_eq)
 * with no quadratic term (nothing extra is streamed) and a free multiplier:
 * the dual vector y of rapdb_solve, rapdb_resume and rapdb_kkt_residual then
 * has m + p_eq entries, the equality multipliers last (any real start), and
 * the (m+1, n) arrays of rapdb_coupling_pass have m + p_eq + 1 rows.  Its
 * KKT component is |a_k'x - b_k|.  Errors as for rapdb_create, plus
 * RAPDB_ERR_INVALID for p_eq < 0, m + p_eq > 6400, NULL A_eq / b_eq with
 * p_eq > 0 or a NaN in them. */
rapdb_status rapdb_create_eq(rapdb_ctx **out, int64_t n, int64_t m, int32_t q0_kind,
                             const float *Q, const float *q0diag, const float *c,
                             const float *d, const float *lb, const float *ub,
                             int64_t p_eq, const float *A_eq, const float *b_eq,
                             const rapdb_params *p, void *stream);

/* Optional parts of a problem beyond those of rapdb_create (zero-initialise
 * and set what is used).
 *   p_eq, A_eq, b_eq: linear equalities A_eq x = b_eq with free multipliers,
 *     as for rapdb_create_eq.
 *   x_hyp_a, x_hyp_beta: the primal set becomes X = {lb <= x <= ub,
 *     x_hyp_a'x = x_hyp_beta} (x_hyp_a: device, n floats, copied; NULL keeps
 *     the box).  The paper's kernel-learning problem (Sec. 5.2, eq.
 *     min-max-KML) minimises over {x >= 0, b'x = 0}: lb = 0, ub = +inf (the
 *     box may be unbounded on either side), a = b, beta = 0.  Every trial
 *     point and every step of the smoothed gap's x-subproblem is projected
 *     onto X: x = clamp(v - nu a, lb, ub) with the scalar nu for which
 *     a'x = beta (found on one CTA in double-float arithmetic, to 1e-13 of
 *     sum |a_j x_j| + |beta|), and the KKT residual's r_stat is
 *     dist(0, grad_x L + N_X(x)), N_X(x) = {t a + N_box(x)}, minimised over t.
 *     x0 must lie in X (|a'x0 - beta| <= 1e-6 (1 + sum |a_j x0_j| + |beta|)).
 *     Single-instance contexts only. */
typedef struct {
  int64_t p_eq;
  const float *A_eq;
  const float *b_eq;
  const float *x_hyp_a;
  double x_hyp_beta;
} rapdb_extras;

/* rapdb_create with the optional parts in *ex (may be NULL: rapdb_create).
 * Errors as for rapdb_create_eq, plus RAPDB_ERR_INVALID for a NaN, an
 * infinite or an all-zero x_hyp_a. */
rapdb_status rapdb_create_ex(rapdb_ctx **out, int64_t n, int64_t m, int32_t q0_kind, const float *Q,
                             const float *q0diag, const float *c, const float *d, const float *lb,
                             const float *ub, const rapdb_extras *ex, const rapdb_params *p, void *stream);

/* Run rAPDB from (x, y) (device, n and m floats -- m + p_eq with equalities;
 * overwritten with the final iterate).  x must lie in the box; y in the dual
 * set: y >= 0, or on the simplex with RAPDB_DUAL_SIMPLEX, equality
 * multipliers free (RAPDB_ERR_INVALID otherwise).  The whole loop -- trial
 * steps, coupling passes, FP64 backtracking tests, step-size updates,
 * restarts, precision checks and the KKT stop test -- runs on the device; the
 * host waits once per graph launch (32 loop bodies) and at the end, then fills
 * *info (host, may be NULL).  Returns info->status. */
rapdb_status rapdb_solve(rapdb_ctx *ctx, float *x, float *y, rapdb_info *info);

/* The float64 iterate of the last rapdb_solve / rapdb_resume: x (device, n
 * doubles) and y (device, m doubles; may be NULL).  rapdb_solve returns x
 * and y rounded to float32; near a 1e-7 residual that rounding alone can
 * move the residual, so callers that need the solver's own point read it
 * here.  Synchronises the context's stream. */
rapdb_status rapdb_get_solution_f64(rapdb_ctx *ctx, double *x, double *y);

/* Relative KKT residual at (x, y) (device): one coupling pass with the most
 * precise products the context has (compensated float32 products when it
 * was created with refine = 1, else the float32 Q, else the stored copy),
 * then
 *   r_stat_j = dist(0, grad_x L(x,y)_j + N_[lb,ub](x_j)),
 *   ||r_feas|| = dist(g(x), N_Y(y)) over the inequality constraints, plus
 *                the equality residuals: with Y the orthant (RAPDB_DUAL_NONNEG)
 *                its components are |g_i(x)| if y_i > 0 else max(g_i(x), 0);
 *                with Y the simplex {y >= 0, sum y = dual_radius}
 *                (RAPDB_DUAL_SIMPLEX), N_Y(y) = {t 1 - nu : nu >= 0, nu_i = 0
 *                where y_i > 0}, so the components are g_i(x) - t if y_i > 0
 *                else max(g_i(x) - t, 0) with the scalar t that minimises
 *                their norm; every linear equality a_k'x = b_k of
 *                rapdb_create_eq adds the component |a_k'x - b_k|,
 *   rel = max(||r_stat|| / (1 + max(||Q_0x+c_0||, ||sum_i y_i(Q_ix+c_i)||)),
 *             ||r_feas|| / (1 + max(||d||, ||(g_i(x) - d_i)_i||))),
 * (with equalities, d holds -b_k and g_i(x) - d_i holds a_k'x for them),
 * the residual r(x, v, lambda) of the metric subregularity theorem (Sec. 4)
 * with the normalisation stated above.  Outputs are host doubles (any may be
 * NULL). */
rapdb_status rapdb_kkt_residual(rapdb_ctx *ctx, const float *x, const float *y,
                                double *rel_kkt, double *r_stat, double *r_feas);

/* One fused coupling pass on the stored Q (the hot operator, exposed for tests
 * and for timing): for every constraint index i = 0..m
 *     U[i] = Q_i x,  W[i] = Q_i v           (device, (m+1, n) float32 each)
 * plus the per-matrix float64 dot products
 *     dots[5*i + 0] = x'U[i], dots[5*i+1] = v'W[i], dots[5*i+2] = v'Uold[i],
 *     dots[5*i + 3] = c_i'x,  dots[5*i+4] = c_i'v
 * (device, 5*(m+1) doubles; Uold is the (m+1, n) device array `uold`, which
 * may be NULL, giving zeros).  x, v: device, n floats.  Asynchronous on the
 * context's stream. */
rapdb_status rapdb_coupling_pass(rapdb_ctx *ctx, const float *x, const float *v,
                                 const float *uold, float *U, float *W, double *dots);

/* The packed incremental pass of a pack_sym context (the form of its trial
 * passes, with zero low parts), for every STORED matrix Q_i in order (i = 0..m
 * when Q_0 is dense, i = 1..m otherwise; M matrices):
 *     W[s] = Q_i v,   U[s] = Uold[s] + W[s]   (rounded once from double-float)
 * where, in a BF16 / FP8 context, Q_i is the stored (quantised) matrix read
 * from its packed tiles (the quantised-increment level's trials) and, with
 * FP8, the right-hand side enters as s .* v and the rows are scaled by s
 * computed from the upper block triangle (each off-diagonal tile read once
 * for its rows and, transposed, for its columns) and, when dots is not NULL,
 *     dots[5*s + 0] = x'U[s], dots[5*s+1] = v'W[s], dots[5*s+2] = v'Uold[s],
 *     dots[5*s + 3] = c_i'x,  dots[5*s+4] = c_i'v
 * (float64; the same fixed-order sums the solver forms).  x, v: device, n
 * floats; uold, U, W: device, (M, n) float32 row-major; dots: device, 5*M
 * doubles.  The context's solver state is not changed.  Runs on the
 * context's stream and returns when it has finished.  RAPDB_ERR_INVALID
 * without pack_sym or on NULL arguments. */
rapdb_status rapdb_packed_pass(rapdb_ctx *ctx, const float *x, const float *v, const float *uold,
                               float *U, float *W, double *dots);

/* Time the context's coupling-pass kernel: `reps` back-to-back launches on
 * the context's stream, on the current solver iterate (x^k, and d of the
 * last trial as the second right-hand side), bracketed by two CUDA events on
 * that stream.  level: -1 = the precision the last solve ended at, 0 = the
 * stored Q, 1 = the float32 Q of a BF16/FP8 context, 2 = float32 Q with
 * compensated (double-float) products (contexts created with refine = 1),
 * 3 = the incremental form of level 2 that the solver's trial passes use
 * (U = U^k + Q d: one float32 right-hand side added to the double-float
 * products at x^k), 4 = level 3 through the packed upper block triangle
 * (contexts created with pack_sym = 1; the form their trials use: the tile
 * kernel, then the row-block kernel), 5 = the tile kernel of level 4 alone,
 * 6 = the tensor-core tile kernel over the packed BF16 / FP8 tiles of a
 * quantised pack_sym context (the quantised-increment level's trials; the
 * right-hand side's pieces are formed once, before the timed launches),
 * 7 = level 6 with the pieces formed in every pass and the row-block kernel;
 * -1 in a context whose last solve ended at the quantised-increment level
 * times level 7.
 * *ms_per_pass (host) receives the average duration of one launch,
 * *bytes_per_pass (host) the algorithmic bytes of one pass: the Q entries
 * read, M * n * n * (4 | 2 | 1) (+ M * n * 4 scale bytes for FP8); at
 * levels 4 and 5 the packed tiles, M * T(T+1)/2 * 128 * 128 * 4 with
 * T = ceil(n / 128); at levels 6 and 7 M * T(T+1)/2 * 128 * 128 * (2 | 1)
 * (+ M * n * 4 scale bytes for FP8).  Outputs go to context scratch; the
 * solver state is not changed.  RAPDB_ERR_INVALID
 * when the level does not exist in this context. */
rapdb_status rapdb_time_pass(rapdb_ctx *ctx, int32_t reps, int32_t level, double *ms_per_pass,
                             int64_t *bytes_per_pass);

/* Record the first `capacity` iterations of the next rapdb_solve calls:
 * tau_k (device doubles), test evaluations of iteration k (device int32),
 * and, when non-NULL, the iterates x^{k+1} (x_log: device, capacity x n
 * floats), y^{k+1} (y_log: capacity x m floats) and the relative KKT
 * residual measured at iterate k (kkt_log: capacity doubles; entries of
 * iterations where it was not evaluated are left untouched) and, with the
 * adaptive restart, the smoothed gap G_xi of each evaluation in order
 * (gap_log: capacity doubles); obj_log and infeas_log (capacity doubles
 * each, optional) receive f(x^{k+1}) and mean_i max(g_i(x^{k+1}), 0) of each
 * accepted iteration k, the two terms of the paper's termination measure for
 * random QCQPs (Sec. 5.1).  capacity = 0 switches logging off.  The buffers
 * are borrowed.  Single-instance contexts only (RAPDB_ERR_INVALID on a
 * batched context). */
rapdb_status rapdb_set_log(rapdb_ctx *ctx, int32_t capacity, double *tau_log,
                           int32_t *trials_log, float *x_log, float *y_log,
                           double *kkt_log, double *gap_log, double *obj_log,
                           double *infeas_log);

/* Batched contexts: B independent problems with their own n_b, m_b, solved
 * together in one device loop with per-instance step sizes, restart counters
 * and convergence flags.  Q_dense[b], c[b], d[b], lb[b], ub[b] are host arrays
 * of B device pointers with the layout of rapdb_create (Q_0 dense).  Data are
 * copied into one packed arena owned by the context (F32 storage only).
 * Tiles: with rows_per_block = 0 the context autotunes at create.  The
 * instances are grouped by size class (ceil(log2 n)); the largest instance of
 * each class times every tile variant and rows per block (32, 64, 128) on the
 * pass its trials run; one variant serves the whole batch (the one with the
 * least time summed over the classes, weighted by their counts) and each class
 * takes its fastest rows per block (rapdb_get_instance_tile reports them).
 * With rows_per_block > 0 every instance takes that tile and pass_variant. */
rapdb_status rapdb_create_batched(rapdb_ctx **out, int32_t B, const int64_t *n,
                                  const int64_t *m, const float *const *Q,
                                  const float *const *c, const float *const *d,
                                  const float *const *lb, const float *const *ub,
                                  const rapdb_params *p, void *stream);

/* Solve every instance: x[b], y[b] (host arrays of device pointers) hold the
 * start points and receive the results; info (host, B entries, may be NULL).
 * Returns RAPDB_OK when every instance reached tol, else the first failing
 * instance's status. */
rapdb_status rapdb_solve_batched(rapdb_ctx *ctx, float *const *x, float *const *y,
                                 rapdb_info *info);

/* Checkpoint / resume of the solver state (iterates, caches, step sizes,
 * counters) at the end of a rapdb_solve.  get: *len receives the size; buf
 * (host) may be NULL to query it.  set: restores a state taken from a context
 * built on the same data and parameters; the next rapdb_solve continues from
 * it (its x, y arguments are then outputs only). */
rapdb_status rapdb_get_state(rapdb_ctx *ctx, void *buf, size_t *len);
rapdb_status rapdb_set_state(rapdb_ctx *ctx, const void *buf, size_t len);

/* Continue the device loop from the context's current state (after a solve
 * that stopped on max_iter or time_limit_s, or after rapdb_set_state, which
 * may come from a context created with a larger max_iter).  x, y (device, n
 * and m floats) receive the final iterate; info as for rapdb_solve.  Because
 * every reduction runs in a fixed order, a solve split by a checkpoint ends
 * bit for bit where the uninterrupted solve ends, provided both contexts use
 * the same coupling-pass tile (fix rows_per_block and pass_variant: tiles
 * with different rows per warp add the products in different orders). */
rapdb_status rapdb_resume(rapdb_ctx *ctx, float *x, float *y, rapdb_info *info);

/* Coupling-pass tile of the context: rows per CTA, CTAs per pass, rows each
 * warp streams together, and 16-byte chunks in flight per row (any output
 * may be NULL).  With rows_per_block = 0 in the parameters, rapdb_create
 * times every supported tile on the context's own data (CUDA events on its
 * stream) and keeps the fastest; the choice is remembered for the process,
 * per device and problem shape (n, stored matrices, storage, refinement,
 * row stride, Q_0 kind), and later contexts of that shape reuse it without
 * timing. */
rapdb_status rapdb_get_tile(const rapdb_ctx *ctx, int32_t *rows_per_block, int32_t *ctas,
                            int32_t *rows_per_warp, int32_t *chunks_in_flight);

/* The coupling pass of rapdb_coupling_pass for callers that cannot allocate
 * device memory (no context; the paper has no counterpart to this call).
 * Creating a context calls cudaMalloc; callers working inside another
 * framework's memory pool or a fixed, pre-planned memory budget, real-time
 * loops that must not enter the allocator, and code recording a CUDA graph
 * cannot do that.  This call allocates nothing: its only scratch, the
 * per-block float64 partial dots, lives in a fixed array of 131072 doubles
 * (1 MiB) that the library reserves on every GPU that loads it, until the
 * process exits.
 *   Q     device, (m+1, n, n) float32, Q_0 first, symmetric, 16-byte aligned
 *   c     device, (m+1, n);  x, v: device, n floats, 16-byte aligned
 *   uold  device, (m+1, n) or NULL (then the third dot is zero)
 *   U, W  device outputs, (m+1, n): U[i] = Q_i x, W[i] = Q_i v
 *   dots  device output, (m+1, 5) doubles as in rapdb_coupling_pass
 * Limits: n % 4 == 0 and (m+1) * 5 * ceil(n/32) <= 131072 (e.g. n = 4096 with
 * m up to 203); otherwise RAPDB_ERR_INVALID and nothing runs.  The call is
 * asynchronous on `stream` (a cudaStream_t, NULL = default stream).  Each
 * call looks up the scratch array's device address for the current device
 * (so a call after cudaDeviceReset, or under another context, finds the
 * array where that context holds it); the first call on a device also loads
 * the library's device code there, so make that first call before any
 * stream capture.
 * Every call on a device shares the one scratch array, so calls whose work
 * overlaps on the GPU (different streams without ordering, or several host
 * threads) race and give wrong results: order them on one stream.  Each call
 * overwrites every scratch slot it reads, so no clearing is needed. */
rapdb_status rapdb_coupling_pass_noalloc(int64_t n, int64_t m, const float *Q, const float *c,
                                         const float *x, const float *v, const float *uold,
                                         float *U, float *W, double *dots, void *stream);

/* Self-test of the bounded wait that guards every bulk-copy stage of the
 * coupling pass (the paper has no counterpart: it is failure detection).  One
 * warp waits on an mbarrier phase with the pass's own wait routine under a
 * limit of limit_us microseconds (1 .. 2,000,000).  complete = 1: a real
 * 16-byte bulk copy completes the phase; the wait returns, *gave_up = 0 and
 * *copied_sum = 10 (the sum of the four copied floats).  complete = 0: the
 * barrier expects 16 bytes that no copy delivers; the wait gives up at the
 * limit, *gave_up = 1 and *copied_sum = -1.  *waited_ms is the device time
 * the wait took.  No copy is ever left in flight, so the device stays usable
 * either way.  Runs synchronously on the current device (default stream);
 * allocates and frees one small device buffer.  Outputs may be NULL.
 * Returns RAPDB_ERR_INVALID for a bad limit or flag, RAPDB_ERR_CUDA if a
 * CUDA call fails. */
rapdb_status rapdb_wait_selftest(int32_t complete, int64_t limit_us, int32_t *gave_up, double *waited_ms,
                                 float *copied_sum);

/* The tile of instance `instance` of a context (0 for a single-instance
 * context): its rows per block and the context's tile variant (0..9, as
 * rapdb_params.pass_variant).  RAPDB_ERR_INVALID for a bad instance. */
rapdb_status rapdb_get_instance_tile(const rapdb_ctx *ctx, int32_t instance, int32_t *rows_per_block,
                                     int32_t *variant);

const char *rapdb_last_error(const rapdb_ctx *ctx);
void rapdb_destroy(rapdb_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* RAPDB_H */

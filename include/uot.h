/*
 * uot.h -- C ABI of the GB300 (sm_103a) generalized Sinkhorn scaling library.
 *
 * Method: Chizat, Peyre, Schmitzer, Vialard, "Scaling algorithms for unbalanced
 * optimal transport problems" (arXiv:1607.05816).
 *
 * Discrete problem (Sec. 4.2, eq. primal_discr, weighted by the reference
 * measures): points x_1..x_n with reference probability weights dx, points
 * y_1..y_m with weights dy, densities p (w.r.t. dx) and q (w.r.t. dy), cost C,
 * Gibbs kernel K = exp(-C/eps) (eq. GibbsKernel), marginal penalties
 * F1(s) = sum_i dx_i D_phi1(s_i | p_i), F2(s) = sum_j dy_j D_phi2(s_j | q_j)
 * (eq. UOT, eq. divergencefunctions):
 *
 *   min_R  F1(R dy) + F2(R^T dx) + eps sum_ij dx_i dy_j KL(R_ij | K_ij).
 *
 * The solver runs the scaling iterations (S) of Sec. 3.3,
 *   a <- proxdiv_F1(K (b.dy)),  b <- proxdiv_F2(K^T (a.dx)),
 * in the log domain of Sec. 4.3 (Algorithm 2 with every update absorbed), and
 * returns the dual potentials U = eps log a, V = eps log b.  The optimal plan
 * is R_ij = exp((U_i + V_j - C_ij)/eps) (Theorem 3.2).
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller unless the
 *    comment says "host".  The library keeps no pointer after it returns.
 *  - Floating-point arrays have the element type selected by `precision`:
 *    UOT_F64 -> double, UOT_F32 and UOT_MIXED -> float.  (UOT_F32 runs the
 *    per-entry kernel arithmetic in FP32 and keeps every per-point quantity
 *    -- potentials, log densities, log weights, intermediate log-sums -- as
 *    a float-float pair (hi + lo, about 48 significant bits) built from
 *    error-free FP32 transformations, so the FP64 pipe stays idle; outputs
 *    are rounded to float unless uot_opts.out_f64 asks for double.)
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  Entry points that return host values (uot_solve's result,
 *    uot_objective) synchronise that stream before returning.
 *  - Temporary device memory is taken from the CUDA stream-ordered allocator
 *    (cudaMallocAsync) and released before return.
 *  - Calls may run at the same time from several host threads on different
 *    streams (a serving loop solving independent problems side by side): a
 *    call keeps its state in its own scratch and on its own stream, the last
 *    error is per thread, CUDA-graph capture uses the thread-local mode, and
 *    per-kernel launch limits are only ever raised.  The results do not depend
 *    on what else runs.  Exceptions: uot_gibbs_log_noalloc (one shared
 *    array), the profiling pair below, and the first use of a grid shape by
 *    the tile tuner (its timings, not its results, see the other streams).
 *    The per-kernel launch settings are kept for the life of the process:
 *    after a cudaDeviceReset the library must not be called again.
 *  - Errors are returned as uot_status, never thrown.  Arguments are checked on
 *    the host before any launch; UOT_EINVAL leaves outputs untouched.
 *  - There is no CPU fallback: if no sm_103a device is present every entry
 *    point returns UOT_ECUDA.
 */
#ifndef UOT_H
#define UOT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  UOT_OK = 0,
  UOT_NOT_CONVERGED = 1, /* iteration cap reached before `tol`; outputs hold the last iterate */
  UOT_EINVAL = -1,       /* invalid argument (checked on the host, nothing launched) */
  UOT_ENOMEM = -2,       /* device allocation failed */
  UOT_NUMERICAL = -3,    /* NaN appeared in the potentials */
  UOT_TIMEOUT = -4,      /* a bounded device-side wait expired */
  UOT_ECUDA = -5,        /* CUDA runtime error (no device, launch failure, ...) */
  UOT_EUNSUPPORTED = -6  /* valid request outside what this library implements */
} uot_status;

/* Marginal penalties (Sec. 2.1 examples; Table 1 rows). */
typedef enum {
  UOT_DIV_EQ = 0, /* iota_{=}(s|p): s = p exactly (balanced OT) */
  UOT_DIV_KL = 1, /* lambda KL(s|p),  lambda > 0 */
  UOT_DIV_TV = 2, /* lambda TV(s|p),  lambda > 0 */
  UOT_DIV_RG = 3  /* RG[alpha,beta](s|p): alpha p <= s <= beta p, 0 <= alpha <= beta <= +inf */
} uot_div_kind;

typedef struct {
  int kind;      /* uot_div_kind */
  double lambda; /* KL, TV weight */
  double alpha;  /* RG lower ratio (>= 0) */
  double beta;   /* RG upper ratio (may be +INFINITY) */
} uot_div;

/* Where the points live and how the cost is given. */
typedef enum {
  UOT_GEOM_DENSE = 0,  /* explicit cost matrix C[n*m], row-major */
  UOT_GEOM_GRID = 1,   /* Cartesian grids, cost |x - y|^2, applied axis by axis (Sec. 4.4) */
  UOT_GEOM_POINTS = 2  /* point clouds x[n*d], y[m*d], cost |x - y|^2 computed on the fly */
} uot_geom_kind;

#define UOT_MAX_DIM 3

typedef struct {
  int kind; /* uot_geom_kind */
  int n, m; /* number of points on each side; for grids the product of the shape */
  /* UOT_GEOM_DENSE */
  const void* C; /* [n*m] row-major; C_ij >= 0 need not hold; +INFINITY means K_ij = 0 (not for
                    uot_objective or plain_scaling, which need finite costs); no NaN or -inf */
  /* UOT_GEOM_GRID: potentials and densities are row-major arrays of the grid's shape.
     Size limits (UOT_EUNSUPPORTED, with a message, before any launch): every axis
     has at most 3000 points, and every separable pass covers at most 65535 lines.
     Passes run from the last axis to the first, so the pass along axis a covers the
     input side's axes before a and the output side's axes after a.  1-D and 2-D
     grids always fit; a 3-D grid with the same shape on both sides fits when each
     product of two axes is at most 65535 (2 x 255 x 257 does, 2 x 256 x 256 does
     not). */
  int ndim;                        /* 1..UOT_MAX_DIM */
  int shape_x[UOT_MAX_DIM];        /* grid of X: shape_x[0] x ... x shape_x[ndim-1] */
  int shape_y[UOT_MAX_DIM];        /* grid of Y */
  const void* axes_x[UOT_MAX_DIM]; /* 1-D coordinates of each axis of X, length shape_x[k] */
  const void* axes_y[UOT_MAX_DIM];
  /* UOT_GEOM_POINTS */
  const void* x; /* [n*d] row-major */
  const void* y; /* [m*d] row-major */
  int d;         /* 1..8 */
} uot_geom;

/*
 * UOT_MIXED: as UOT_F32 (float arrays, float-float per-point state), but on
 * grids the separable passes run on the tensor cores (tcgen05, BF16 operands,
 * FP32 accumulation) in a block-stabilised form that needs about a tenth of
 * the exponentials; results carry the BF16 operand rounding (relative error of
 * the kernel sums ~2^-8).  Grid axes whose 32-point blocks are too wide for
 * that form at the given eps, and non-grid geometries, use the FP32 kernels.
 * In uot_solve / uot_solve_many with tol > 0 the tensor-core passes run through
 * the eps-scaling stages and at the final eps until the marginal violation
 * falls to uot_opts.mixed_switch (or stops improving: the BF16 floor); the
 * remaining iterations use the FP32 passes, to tol.  With uot_opts.verify the
 * stop is then confirmed in FP64: BF16, then FP32, then FP64 for the check.
 */
typedef enum { UOT_F64 = 0, UOT_F32 = 1, UOT_MIXED = 2 } uot_precision;

typedef struct {
  int precision;       /* uot_precision */
  double eps;          /* final entropic regularisation eps > 0 */
  double eps_start;    /* eps-scaling start (Sec. 4.4); <= eps disables eps-scaling */
  int eps_stages;      /* number of divisions of eps (the paper uses 10) */
  int iters_per_stage; /* iterations before each division (the paper uses 100) */
  int max_iter;        /* iterations at the final eps (cap) */
  double tol;          /* stop when the marginal violation <= tol; 0 runs max_iter */
  int check_every;     /* iterations between violation checks (>= 1) */
  int plain_scaling;   /* 1: Algorithm 1 (non-log scalings a, b on a stored kernel
                          K = exp(-C/eps)); dense geometry and UOT_F64 only.
                          0: log domain (Algorithm 2 with every update absorbed) */
  int launch_mode;     /* 0: one launch per Gibbs pass (consecutive passes overlap through
                          programmatic dependent launch), convergence tested by the host every
                          check_every iterations;
                          1: FP32 grid problems (batch 1) run as one persistent cooperative
                          launch, eps stages and convergence test on the device, grid barriers
                          between passes (measured slower at 256 x 256: 23.7k vs 39.5k it/s);
                          with plain_scaling (Algorithm 1), each eps runs as one launch of one
                          thread-block cluster (16 CTAs, else 8) holding K and K^T in shared
                          memory, convergence tested on the device: the same iterates as 0,
                          used where 8 (ceil(n/CL) m + ceil(m/CL) n + 2(n + m)) bytes fit in
                          200 KB, else as 0; other problems ignore it;
                          2: as 0, but once a block of check_every iterations at the final eps
                          repeats the same launches (shifts from the previous iteration), it
                          is captured once as a CUDA graph and replayed block by block (log
                          domain, all geometries, uot_solve_many and uot_barycenter too;
                          per-pass launches where capture fails);
                          3: FP32 2-D grids (batch 1): two kernels per iteration, each fusing two
                          passes on one grid line (the U-update's last pass with the V-update's
                          first, contracting axis 0 first, and the V-update's last pass with the
                          next U-update's first), replayed as CUDA-graph blocks like 2; other
                          problems run as 2 */
  const void* U0;      /* optional warm start [n] (NULL: U = 0); -inf allowed (zero scaling),
                          NaN or +inf rejected with UOT_EINVAL (uot_solve, uot_solve_many) */
  const void* V0;      /* optional warm start [m] (NULL: V = 0, i.e. b = 1 as in Algorithm 1) */
  int out_f64;         /* 1: U and V are written as double whatever the precision (UOT_F32 and
                          UOT_MIXED: the float-float state, about 48 significant bits, rounded
                          to FP64 instead of FP32); 0: the precision's type.  uot_solve,
                          uot_solve_many and uot_solve_batch */
  int verify;          /* 1 (log domain, UOT_F32 / UOT_MIXED, tol > 0): a stop signalled by the
                          FP32 check is confirmed by evaluating the marginal violation of the
                          current potentials in FP64 (FP64 Gibbs operator on FP64 copies of
                          the geometry and of the state).  If the FP64 value is above tol
                          the FP32 iteration continues with a proportionally lower internal
                          threshold; once the FP32 check stops decreasing (its rounding
                          floor), the remaining iterations run in FP64 from the current
                          state, checked every iteration, until the FP64 violation is
                          <= tol.  marg_err is then the FP64 value.  Launch mode 1 runs as
                          0, launch mode 3 as 2.  0: the FP32 check decides. */
  double mixed_switch; /* UOT_MIXED with tol > 0: violation at which the tensor-core (BF16)
                          passes hand over to the FP32 passes; 0 means 1e-3 */
  int translate;       /* 1 (uot_solve, uot_solve_many; log domain; UOT_DIV_KL on both sides,
                          else UOT_EUNSUPPORTED): after the V-update of every checked iteration
                          (every check_every iterations at the final eps, the FP64 finish of
                          opts.verify included) and of iterations check_every, 2 check_every,
                          ... of each eps-scaling stage, U += c and V -= c per problem with
                          c = lam1 lam2 / (lam1 + lam2) (log A - log B), A = sum_i dx_i p_i
                          e^{-U_i/lam1}, B = sum_j dy_j q_j e^{-V_j/lam2}: the exact maximum of
                          the dual (Theorem 3.2) along that direction, which leaves the plan
                          unchanged.  Not in the paper (the translation step of Sejourne,
                          Vialard, Peyre 2022): the scaling iteration damps this direction
                          only by (lam / (lam + eps))^2 per iteration, so for lam >> eps it
                          removes the slowest mode, and it bounds how far FP32 rounding can
                          push the state along it.  Same fixed point; different iterates.
                          Launch mode 1 runs as 0, launch mode 3 as 2.  0: Algorithm 2 as
                          printed. */
} uot_opts;

typedef struct {
  int iters;        /* iterations run at the final eps */
  int total_iters;  /* including the eps-scaling stages */
  double marg_err;  /* last measured marginal violation (see uot_solve) */
  double ms;        /* device time of the whole solve (CUDA events) */
  int status;       /* uot_status of the solve */
  int verifications;    /* FP64 confirmations run (opts.verify) */
  int polish_iters;     /* iterations run in FP64 after the FP32 floor (opts.verify) */
  double marg_err_fp32; /* last FP32-evaluated violation (NaN if none) */
  int mixed_iters;      /* UOT_MIXED: iterations (stages included) run with the tensor-core passes */
  int precise_iters;    /* opts.verify on grids and point clouds (d <= 3): FP32 iterations run with
                           the passes that form their exponents in float-float, after the plain
                           FP32 check stalled */
} uot_result;

/* Version string of the library build. */
const char* uot_version(void);

/* Message of the last failed call on this thread: a CUDA error string or the
   reason for a refusal ("" if none).  The solver, Gibbs, plan, objective,
   barycenter, mass, WF, colour-transfer and self-test entry points reset it
   when they start, so it describes the latest of those calls. */
const char* uot_last_error(void);

/*
 * Instrumentation (not part of the method).
 * uot_launch_count: number of kernels this library has launched in this
 * process (host-side counter, incremented at every launch).
 * uot_profile_begin / uot_profile_end: while enabled, each launch of a Gibbs
 * operator kernel is bracketed by a pair of CUDA events recorded on the stream
 * it is launched on; uot_profile_end synchronises those events and returns the
 * summed kernel time (ms) and the number of launches of one family:
 *   family 0: separable grid passes (log-sum-exp tiles, tensor-core passes),
 *   family 1: row kernels (dense / points), family 2: separable grid passes run
 *   by the block-stabilised kernel of uniform axes.
 * Not thread-safe across concurrent solves.
 */
long long uot_launch_count(void);
void uot_profile_begin(void);
uot_status uot_profile_end(int family, double* total_ms, long long* launches);

/*
 * Tile-shape tuner of the FP32 separable grid pass (a schedule choice, not
 * part of the method: every shape computes the same sums of Sec. 4.4 up to
 * FP32 rounding order).  A tile is (warps splitting the contraction index,
 * outputs per lane); the first time a pass shape (lines, inputs, outputs,
 * batch) is met on a device, every tile is timed on scratch inputs of that
 * shape with CUDA events (this synchronises the stream once and allocates
 * stream-ordered scratch); the fastest is kept for the process lifetime,
 * except that the first tile stays unless another is more than 5% faster.
 * No tuning happens inside a stream capture or in uot_gibbs_log_noalloc: the
 * first tile is used there until the shape has been tuned elsewhere.
 *
 * uot_set_autotune(mode): 1 (default) = tune on first use; 0 = always the
 *   first tile (results then do not depend on timing).  Returns the previous mode.
 * uot_force_grid_tile(idx): use tile idx (0 .. uot_grid_tile_count()-1) for
 *   every FP32 grid pass; idx = -1 returns to the tuned choice.  UOT_EINVAL if
 *   idx is out of range.
 * uot_autotune_table(buf, len): writes the tuned shapes, the chosen tile and
 *   every tile's measured time per launch as text (one line per pass shape,
 *   NUL-terminated, truncated to len-1 bytes); returns the full text length.
 * Process-wide settings, guarded by a mutex.
 */
int uot_set_autotune(int mode);
uot_status uot_force_grid_tile(int idx);
int uot_grid_tile_count(void);
int uot_autotune_table(char* buf, int len);

/*
 * CTA size of uot_solve_batch (a schedule choice; results differ only in FP32
 * summation order).  8 or 16 warps per CTA are compiled; with the tuner on,
 * the first call for a batch shape (d, largest n, largest m) times both on a
 * sample of the batch (every (nprob/S)-th problem of the size-ordered queue,
 * S = 2 x SM count, six iterations) and keeps the 8-warp CTA unless the other
 * is more than 3% faster; uot_autotune_table lists the choice.
 * uot_force_batch_warps(w): w = 8 or 16 forces that size, 0 returns to the
 * tuned one; UOT_EINVAL otherwise.
 */
uot_status uot_force_batch_warps(int warps);

/*
 * uot_probe_pipes -- throughput probes (instrumentation): out (host) receives
 * the sustained rates of the pipes the kernels are bound by, in operations per
 * clock per SM measured with in-kernel clock64() over dependent-chain loops
 * with 64 resident warps per SM:
 *   out[0]: FP32 FMA lane operations, out[1]: MUFU ex2.approx.f32, out[2]: FP64
 *   FMA lane operations, out[3]: FP64 exponentials exp() (the function the FP64
 *   Gibbs passes evaluate per kernel term).  out holds 4 doubles.
 * A few milliseconds of work; synchronises `stream`.
 */
uot_status uot_probe_pipes(double* out, void* stream);

/*
 * uot_force_precise_passes -- on = 1: every FP32 Gibbs pass on a grid or on
 * point clouds of dimension <= 3 (uot_solve, uot_solve_many, uot_gibbs_log,
 * ...) runs the pass that forms its exponents t_j - k |x_i - y_j|^2 - m_i in
 * float-float (the coordinate differences by exact TwoSum, the staged input
 * values, the squared distance, its product with k = log2(e)/eps and the
 * running maximum), rounding only the final small difference to FP32 for the
 * exponential.  The usual passes form these exponents in FP32, which costs
 * ulp(|t_j|) per term when values and costs are large (lambda >> eps): their
 * rounding floor on the marginal violation can then lie above 1e-6.  Solves
 * with opts.verify switch to the precise pass by themselves when their FP32
 * check stalls (uot_result.precise_iters); this switch forces it everywhere
 * (tests, measurements).  on = 0 restores the default.  Returns the previous
 * setting.  Process-wide, not tied to a stream.
 */
int uot_force_precise_passes(int on);

/*
 * uot_fuse_short_passes(on): FP32 separable grids run two consecutive passes
 * whose four axis sizes are all at most 64 (the 32-point axes of a 64x32x32
 * colour grid, the axes of 64x64 images) as one launch per plane of the two
 * axes, the intermediate kept in shared memory (1), or as two launches (0, the
 * default: on the 64x32x32 colour transfer the fused form takes 61 ms against
 * 45 ms, since one CTA per plane leaves most SMs idle).  The results are the same bit for bit as two passes on the
 * short-line kernel; a tile forced by uot_force_grid_tile other than that
 * kernel turns the fusion off.  The setting is process-wide.  Returns the
 * previous setting.
 */
int uot_fuse_short_passes(int on);

/*
 * uot_selftest_bounded_wait -- failure-detection self-test (instrumentation).
 * Runs the bounded device-side wait that guards every wait of a kernel on
 * other CTAs (the persistent solve's grid barrier) on a flag that nothing
 * sets: after `seconds` (0 < seconds <= 10) of the GPU's global timer the
 * wait gives up, sets its status flag and the kernel returns, so the call
 * returns UOT_TIMEOUT with the CUDA context intact.  Returns UOT_OK only if
 * the flag were set, UOT_EINVAL for seconds out of range.  Synchronises
 * `stream`.
 */
uot_status uot_selftest_bounded_wait(double seconds, void* stream);

/*
 * uot_solve -- scaling iterations for entropic unbalanced OT (eq. S, Sec. 3.3;
 * Algorithm 2 of Sec. 4.3 in log form; eps-scaling of Sec. 4.4).
 *
 *  g           geometry (dense cost, grid or point clouds)
 *  p, dx       [n] density of mu w.r.t. dx (p >= 0) and reference weights (dx > 0)
 *  q, dy       [m] density of nu w.r.t. dy and reference weights
 *  F1, F2      host structs, marginal penalties on the X and Y marginals
 *  o           host struct, options
 *  U, V        [n], [m] outputs: dual potentials eps log a, eps log b;
 *              -inf where the scaling is 0 (zero density, Prop. 5.1)
 *  res         host struct, may be NULL
 *
 * One iteration: S = eps log K(b.dy); U = prox_F1(S); T = eps log K^T(a.dx);
 * V = prox_F2(T), with the Table 1 rows in log form (U_bar = eps log p - S):
 *   EQ: U = U_bar;  KL: U = lambda/(lambda+eps) U_bar;  TV: U = clamp(U_bar, -lambda, lambda);
 *   RG: U = min(eps log beta + U_bar, max(eps log alpha + U_bar, 0)).
 * Marginal violation (the stopping criterion, which the paper leaves open):
 *   sum_i dx_i |r1_i - t_i| / sum_i dx_i t_i, r1 = a.K(b.dy) the first marginal
 *   of the current plan and t = prox^KL_{F1/eps}(K(b.dy)) its target.  It is
 *   measured inside the a-update of the iteration after the checked one, so
 *   the returned iterate is one iteration past the checked state.
 * Returns UOT_OK (tol reached), UOT_NOT_CONVERGED (cap hit; tol > 0 only),
 * UOT_NUMERICAL, UOT_EINVAL, UOT_ENOMEM, UOT_ECUDA.
 */
uot_status uot_solve(const uot_geom* g, const void* p, const void* dx, const void* q,
                     const void* dy, const uot_div* F1, const uot_div* F2, const uot_opts* o,
                     void* U, void* V, uot_result* res, void* stream);

/*
 * uot_solve_many -- the iteration of uot_solve (eq. S in the log form of
 * Sec. 4.3, Table 1 rows) for `batch` independent problems that share the
 * geometry, the reference weights dx, dy, eps and the penalties F1, F2 but not
 * the densities: p and U are [batch][n], q and V are [batch][m] (row-major).  For
 * grids every Gibbs-operator pass treats all problems in one launch.  Options
 * as in uot_solve (plain_scaling unsupported); the iteration runs until every
 * problem's marginal violation is <= tol, and res->marg_err is the largest.
 */
uot_status uot_solve_many(const uot_geom* g, int batch, const void* p, const void* dx,
                          const void* q, const void* dy, const uot_div* F1, const uot_div* F2,
                          const uot_opts* o, void* U, void* V, uot_result* res, void* stream);

/*
 * uot_solve_mass -- scaling iterations with a third divergence on the total
 * mass of the plan (Algorithm 4, Sec. 4.5), in the log domain of Sec. 4.3
 * with eps-scaling (Sec. 4.4):
 *
 *   min_R  F1(R dy) + F2(R^T dx) + F3(sum_ij dx_i dy_j R_ij) + eps KL(R | K),
 *
 * F3(s) = D_phi3(s | m0) for a scalar s, any Table 1 row (EQ fixes the total
 * mass to m0).  The plan is R_ij = exp((U_i + V_j + Z - C_ij)/eps): a scalar
 * z = e^{Z/eps} multiplies the two scalings.
 *
 * One iteration: S = eps log K(b.dy); then, except in the very first
 * iteration (z = 1), the z-update of Algorithm 4 with the current a and the
 * new b: M = sum_i dx_i exp((U_i + S_i)/eps), Z = the Table 1 row of F3 at
 * log-mass eps log M with p = m0; U = prox_F1(S + Z); T = eps log K^T(a.dx);
 * V = prox_F2(T + Z).  The marginal violation is that of uot_solve with
 * S + Z in place of S, or the mass violation |exp((Z_old - Z)/eps) - 1| of
 * the z-update if larger (with a saturated F1 the a-side can be stationary
 * while z still moves).
 *
 *  m0          target mass of F3, 0 < m0 < inf
 *  Z           host double, output: eps log z of the last iteration
 *  other arguments as for uot_solve (plain_scaling unsupported: UOT_EUNSUPPORTED;
 *  launch modes 1 and 3 run as 2).  The iteration starts from z = 1.
 * Returns as uot_solve; UOT_NUMERICAL also when Z is NaN.
 */
uot_status uot_solve_mass(const uot_geom* g, const void* p, const void* dx, const void* q,
                          const void* dy, const uot_div* F1, const uot_div* F2, const uot_div* F3,
                          double m0, const uot_opts* o, void* U, void* V, double* Z, uot_result* res,
                          void* stream);

/*
 * uot_gibbs_log -- the log-domain Gibbs operator alone (Sec. 4.2, 4.3):
 *   transpose = 0: out_i = eps log sum_j exp((W_j - C_ij)/eps) w_j   (out [n], W,w [m])
 *   transpose = 1: out_j = eps log sum_i exp((W_i - C_ij)/eps) w_i   (out [m], W,w [n])
 * i.e. eps log K(e^{W/eps} . w).  W may hold -inf (zero scaling).
 * UOT_MIXED synchronises `stream` and returns UOT_TIMEOUT if a bounded wait of
 * the tensor-core pass expired.
 */
uot_status uot_gibbs_log(const uot_geom* g, const void* W, const void* w, double eps,
                         int transpose, int precision, void* out, void* stream);

/*
 * uot_gibbs_log_noalloc -- uot_gibbs_log (the log-domain Gibbs operator of
 * Sec. 4.3, passes one axis at a time on grids as in Sec. 4.4) without any
 * device allocation.
 *
 * The allocation-free form has no counterpart in the paper.  It serves callers
 * that cannot call cudaMalloc or cudaMallocAsync: code running under a foreign
 * allocator that owns all device memory (a framework's pool or a pre-reserved
 * arena, where a second allocator would fight it for memory), and real-time
 * or latency-critical loops in which an allocation may block, synchronise or
 * fail.  Arguments, layout and result are those of uot_gibbs_log; the caller
 * still provides W, w and out.  Temporary buffers come from one fixed device
 * array of UOT_NOALLOC_SCRATCH_BYTES bytes inside the library, which every GPU
 * that loads the library holds until the process exits.
 *  - Grid and point-cloud geometries, UOT_F64 and UOT_F32 (UOT_EUNSUPPORTED for
 *    dense costs and for UOT_MIXED, whose set-up reads the grid axes back to
 *    the host and synchronises the stream).
 *  - Scratch needed, each buffer rounded up to 256 bytes, with nin, nout the
 *    input and output sizes:
 *      grids:  8 (2 nin + nout), plus 16 prod_k max(shape_x[k], shape_y[k]) when
 *              ndim > 1, plus 256 for UOT_F32;
 *      points: 8 (2 nin + nout) + 8 max(n, m) + 512, plus for UOT_F32 with d <= 3
 *              8 x the chunk partials, max(c(m, n) n, c(n, m) m), where c(nin, nout)
 *              >= ceil(nin / 1024) is the number of input chunks of a pass.
 *    A square 2-D grid needs about 40 bytes per point: up to 323 x 323 fits
 *    (256 x 256 does, 512 x 512 does not).  A larger problem is rejected with
 *    UOT_EINVAL and a message in uot_last_error(), before anything is launched.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current, checks the result, and
 *    keeps it for the life of the process; make that first call before any
 *    stream capture on the device.  The kept address belongs to the CUDA
 *    context of that first call: do not use this entry point after
 *    cudaDeviceReset.
 *  - All calls share the array and it keeps the last call's contents (every
 *    buffer is written before it is read, so nothing needs clearing): calls
 *    whose work overlaps on the GPU (different streams, or several host
 *    threads) race and corrupt each other's results.  Serialise them.
 *  - No cudaMalloc, cudaMallocAsync, cudaFree or allocating library routine is
 *    called, and the grid tile tuner (which allocates) is held off.
 */
#define UOT_NOALLOC_SCRATCH_BYTES (4u << 20)
uot_status uot_gibbs_log_noalloc(const uot_geom* g, const void* W, const void* w, double eps,
                                 int transpose, int precision, void* out, void* stream);

/*
 * uot_apply_plan -- apply the plan R_ij = exp((U_i + V_j - C_ij)/eps) to
 * nonnegative functions (Sec. 4.2 projections; barycentric projection, Sec. 5.1):
 *   transpose = 0: out[i*ncols + c] = sum_j R_ij dy_j f[j*ncols + c]   (f [m*ncols])
 *   transpose = 1: out[j*ncols + c] = sum_i R_ij dx_i f[i*ncols + c]   (f [n*ncols])
 * f = NULL means f = 1, which gives the marginals r1 = R dy, r2 = R^T dx.
 * f must be >= 0 (UOT_EINVAL is not detected on the device; negative entries
 * give NaN).  1 <= ncols <= 64.
 */
uot_status uot_apply_plan(const uot_geom* g, const void* U, const void* V, double eps,
                          const void* dx, const void* dy, const void* f, int ncols,
                          int transpose, int precision, void* out, void* stream);

/*
 * uot_objective -- primal, dual and gap at potentials (U, V) (Theorem 3.2):
 *   primal = F1(r1) + F2(r2) + eps sum_ij dx_i dy_j (R_ij log(R_ij/K_ij) - R_ij + K_ij)
 *   dual   = -F1*(-U) - F2*(-V) - eps sum_ij dx_i dy_j (R_ij - K_ij)
 *   gap    = primal - dual = sum over both sides of F(r) + F*(-U) + <U, r>_dx,
 * with r1 = R dy, r2 = R^T dx.  out (host) receives {primal, dual, gap, marg_err}
 * in FP64 (reductions in FP64).  EQ and RG penalties are +inf off their
 * constraint sets, so primal/gap are +inf unless the marginal is feasible to
 * the relative tolerance 1e-9.
 */
uot_status uot_objective(const uot_geom* g, const void* p, const void* dx, const void* q,
                         const void* dy, const uot_div* F1, const uot_div* F2, double eps,
                         const void* U, const void* V, int precision, double* out, void* stream);

/* One problem of a batch for uot_solve_batch. */
typedef struct {
  int n, m;      /* points on each side, 1..3072 */
  uot_div F1;    /* penalty on the first marginal */
  uot_div F2;    /* penalty on the second marginal */
} uot_batch_problem;

/*
 * uot_solve_batch -- many independent unbalanced OT problems between point
 * clouds (cost |x - y|^2, computed on the fly) solved in one persistent launch.
 * Each problem runs the iteration of uot_solve (eq. S, Sec. 3.3; log form of
 * Sec. 4.3; eps-scaling of Sec. 4.4) to its own tolerance; problems of uneven
 * sizes are taken from a device work queue, largest first.
 *  nprob       number of problems >= 1
 *  probs       host [nprob] sizes and penalties
 *  d           dimension of the points, 1..3
 *  x, dx, p    packed X sides: problem k occupies points [Xk, Xk + n_k) with
 *              Xk = n_0 + ... + n_{k-1}; x is [sum n][d] row-major, dx and p [sum n]
 *  y, dy, q    packed Y sides likewise
 *  o           options: precision must be UOT_F32; eps, eps_start, eps_stages,
 *              iters_per_stage, max_iter, tol, check_every as in uot_solve;
 *              translate (every problem KL / KL, else UOT_EUNSUPPORTED) and
 *              out_f64 as in uot_solve; plain_scaling, verify, U0 and V0 must
 *              be 0/NULL
 *  U, V        [sum n], [sum m] outputs (float, or double with out_f64: the
 *              float-float state rounded to FP64), packed like the inputs
 *  iters       host [nprob] iterations at the final eps per problem, or NULL
 *  errs        host [nprob] last measured marginal violation per problem, or NULL
 * Returns UOT_OK if every problem reached tol (or tol == 0), UOT_NOT_CONVERGED
 * if some hit the cap.  Synchronises `stream`.
 */
uot_status uot_solve_batch(int nprob, const uot_batch_problem* probs, int d, const void* x,
                           const void* p, const void* dx, const void* y, const void* q,
                           const void* dy, const uot_opts* o, void* U, void* V, int* iters,
                           double* errs, uot_result* res, void* stream);

/* Barycenter divergence for uot_barycenter (Table 2 rows). */
typedef enum { UOT_BARY_KL = 1, UOT_BARY_EQ = 0, UOT_BARY_TV = 2, UOT_BARY_RG = 3 } uot_bary_kind;

/*
 * uot_barycenter -- unbalanced barycenter of K measures (Sec. 5.2) by the
 * scaling iterations with K couplings sharing the kernel exp(-c/eps)
 * (c_k = alpha_k c with the weighted entropy of Sec. 5.2).
 *   F1 acts per measure (eq. proxcomponentbary): proxdiv with p_k;
 *   F2(s) = min_h lambda sum_k alpha_k D(s_k | h) (eq. Fbary), h from Table 2
 *   (UOT_BARY_KL: power mean; UOT_BARY_EQ: geometric mean; UOT_BARY_TV: the
 *   root of (iii)), then V_k = prox for lambda D(.|h) (Table 1 with p -> h).
 *   UOT_BARY_RG needs its range: use uot_barycenter_div (UOT_EINVAL here).
 *  Kmeas       number of measures K >= 1
 *  alpha       host [K] weights alpha_k > 0
 *  P           [K*n] densities of the measures w.r.t. dx
 *  F1          host, penalty of each coupling's first marginal (EQ in the
 *              paper's experiments; KL/TV/RG accepted, see the weighting reading)
 *  lambda      barycenter weight lambda > 0 (ignored for UOT_BARY_EQ)
 *  logh        [m] output eps log h of the barycenter density h (w.r.t. dy)
 *  U, V        [K*n], [K*m] outputs
 * tol/check_every are honoured with the violation of the first coupling's F1
 * side summed over k.
 */
uot_status uot_barycenter(const uot_geom* g, int Kmeas, const double* alpha, const void* P,
                          const void* dx, const void* dy, const uot_div* F1, double lambda,
                          int bary_kind, const uot_opts* o, void* logh, void* U, void* V,
                          uot_result* res, void* stream);

/*
 * uot_barycenter_div -- uot_barycenter with the barycenter divergence given as
 * a uot_div Fh (Table 2, with Table 1 for the V_k updates, p -> h):
 *   UOT_DIV_EQ        (i)   geometric mean;
 *   UOT_DIV_KL lambda (ii)  power mean;
 *   UOT_DIV_TV lambda (iii) h = 0 if the weight of the measures with s_k = 0 is at
 *                           least half of the total, else eps log h = W solves
 *                           A0 + sum_{s_k > 0} alpha_k clamp((W - eps log s_k)/lambda, -1, 1) = 0;
 *   UOT_DIV_RG [alpha, beta] (iv), 0 < alpha <= beta < inf: h = 0 if some s_k = 0,
 *                           else W solves sum_k alpha_k [beta min(W - eps log s_k + eps log beta, 0)
 *                           + alpha max(W - eps log s_k + eps log alpha, 0)] = 0.
 * (iii) and (iv) are continuous, non-decreasing and piecewise linear in W; the
 * root is located exactly from the values at the 2K breakpoints, and where the
 * function vanishes on an interval its midpoint is taken (every point of it
 * minimises the per-point prox problem; the V_k do not depend on the choice).
 * TV and RG take K <= 1024.  Other arguments as for uot_barycenter.
 */
uot_status uot_barycenter_div(const uot_geom* g, int Kmeas, const double* alpha, const void* P,
                              const void* dx, const void* dy, const uot_div* F1, const uot_div* Fh,
                              const uot_opts* o, void* logh, void* U, void* V, uot_result* res,
                              void* stream);

/*
 * uot_wf_cost -- dense cost matrix of the Wasserstein-Fisher-Rao distance
 * (eq. logcost, Definition WF of Sec. 2):
 *   C[i*m + j] = -log cos^2((pi/2) |x_i - y_j| / cut)   for |x_i - y_j| < cut,
 *              = +INFINITY                               otherwise (K_ij = 0),
 * i.e. the distance rescaled so that the cut locus lies at distance `cut`
 * (cut = pi/2: the plain Euclidean distance).  x [n*d], y [m*d] row-major,
 * 1 <= d <= 8, C [n*m] in the precision's type (UOT_F64 or UOT_F32; computed
 * in FP64 either way).  Use it as a UOT_GEOM_DENSE geometry.
 */
uot_status uot_wf_cost(const void* x, int n, const void* y, int m, int d, double cut, int precision,
                       void* C, void* stream);

/*
 * uot_wf_flow -- WF gradient flow with growth (Sec. 2 "Gradient flows",
 * eq. grad-flow; Sec. 5.3, the tumor example and its extension to several
 * species): `nsteps` minimizing-movement steps of
 *   G(mu^1..mu^S) = -alpha sum_k mu^k(X) + iota_{<=1}(sum_k d mu^k/dx)
 * for S = nspecies measures on the same points (X = Y, dy = dx, g->n == g->m),
 * with the geometry's cost (uot_wf_cost for WF).  Each step solves
 *   min over couplings R^k:  sum_k [lam KL(R^k dy | p^k) + lam KL(R^k^T dx | mu^k)
 *                            + eps KL(R^k | K)] + 2 tau G(mu^1..mu^S)
 * by the scaling iteration in log form started from U = V = 0 (b = 1):
 *   U^k = lam/(lam+eps) (eps log p^k - S^k)                     (F1 = lam KL(.|p^k))
 *   V^k = min(-lam log c, -lam Ttot/(lam+eps)),  Ttot = eps log sum_k e^{T^k/eps}
 * with c = 1 - 2 tau alpha/lam (lam = 1 is the paper's WF; with lam = 1, S = 1
 * this is the paper's printed proxdiv for the tumor example, and for S = 2
 * its 1/beta form).  The step ends with the next densities
 *   p^k <- r2^k / max(c, sum_k r2^k),  r2^k = e^{(V^k + T^k)/eps},
 * the minimisers of F2's inner infimum at the couplings' second marginals
 * (for one species min(r2/c, 1)).
 *  nspecies    S >= 1
 *  P0          [S*n] initial densities w.r.t. dx (>= 0)
 *  dx          [n] reference weights (> 0)
 *  tau, alpha  time step > 0 and growth rate >= 0 with 2 tau alpha < lambda
 *  lambda      KL weight lam > 0
 *  o           precision UOT_F64 or UOT_F32 (UOT_MIXED: UOT_EUNSUPPORTED); eps, and the
 *              eps-scaling fields, apply within every step; max_iter = iterations per step
 *              at eps (the paper stops each step after a fixed count); tol must be 0;
 *              U0, V0 must be NULL; launch_mode 2 replays the whole step as one CUDA graph
 *  P           [nsteps*S*n] output: the densities after each step
 *  U, V        [S*n] outputs: the last step's potentials
 *  res         iters = max_iter, total_iters = all iterations, marg_err = NaN (not measured)
 * The paper's runs use eps = 1e-7 and 1e-8 on 3000 points: only UOT_F64 resolves the
 * marginals there (FP32 carries exponent errors of |U|/eps x 6e-8).
 */
uot_status uot_wf_flow(const uot_geom* g, int nspecies, const void* P0, const void* dx, double tau,
                       double alpha, double lambda, const uot_opts* o, int nsteps, void* P, void* U,
                       void* V, uot_result* res, void* stream);

/*
 * Colour transfer (Sec. 5.1): colours are points of [0, 1]^d (the paper uses
 * CIE-Lab rescaled to [0, 1]^3 and 64 x 32 x 32 bins), an image's colour
 * histogram is the pushforward of its pixel measure, the plan between two
 * histograms gives a map by barycentric projection, and the new image is
 * T o g_X.  Binning: bin k of axis a covers [k/n_a, (k+1)/n_a), decided on the
 * FP32 product x * n_a; points outside the cube go to the nearest bin (NaN to
 * bin 0); bins are numbered row-major, like the potentials of a grid.
 *
 * uot_histogram: p [prod shape] (precision's type) = fraction of the npts points
 *   pts [npts*d] (float, row-major) in each bin, i.e. the density w.r.t. the
 *   reference measure with unit mass per bin (the paper's dx = 1).  1 <= d <= 8,
 *   shape host [d], 1 <= npts < 2^32.
 * uot_barycentric_map: T [n*dim] (precision's type, UOT_F64 or UOT_F32) with
 *   T_i = sum_j R_ij dy_j y_j / sum_j R_ij dy_j, R_ij = exp((U_i + V_j - C_ij)/eps)
 *   the plan, y_j the points of Y (grid points or the cloud); dim = g->ndim or g->d.
 *   Rows of zero plan mass keep their own point x_i.  Grid and point geometries
 *   (UOT_EUNSUPPORTED for dense costs).
 * uot_apply_bin_map: out [npts*d] (float) = T[bin(pts_k)] for every point,
 *   T [prod shape * d] in the precision's type.
 */
uot_status uot_histogram(const float* pts, long long npts, int d, const int* shape, int precision, void* p,
                         void* stream);
uot_status uot_barycentric_map(const uot_geom* g, const void* U, const void* V, double eps, const void* dx,
                               const void* dy, int precision, void* T, void* stream);
uot_status uot_apply_bin_map(const float* pts, long long npts, int d, const int* shape, const void* T,
                             int precision, float* out, void* stream);

/*
 * Learned warm start (not in the paper).  A small dilated convolutional
 * network maps (log p, log q, log eps, log lambda) on a grid to initial
 * potentials (U0, V0) that replace b = 1 of Algorithm 1; the plain iteration
 * decides the result.  These are its training and inference
 * kernels; all arrays are FP32 device arrays, activations [N][C][H][W],
 * weights [Cout][Cin][3][3], biases [Cout].
 *
 * uot_conv2d_forward: y = act(b + conv3x3_dilated(x, w)), zero padding;
 *   leaky = 1: act(v) = v (v >= 0), 0.1 v (v < 0); leaky = 0: identity.
 * uot_conv2d_backward: given dy = dLoss/dy of the layer's output y (the
 *   post-activation values stored by the forward pass), writes dx (if not
 *   NULL), dw and db (both overwritten).
 * uot_adam_step: one Adam update of n parameters (step counts from 1).
 * uot_mse_grad: grad = 2 (pred - target)/n and *loss_dev = mean (pred - target)^2
 *   (loss_dev is a device double).
 * uot_scale_instances: x[n][...] *= scale[n] for n < N, per_instance values
 *   each (the network works with potentials divided by lambda).
 * uot_warmstart_features: out [N][4][H][W] = (max(log p, -30), max(log q, -30),
 *   log eps, log lambda) / 4, from p, q [N][H][W] and per-instance log_eps,
 *   log_lam [N].
 */
uot_status uot_conv2d_forward(const float* x, const float* w, const float* b, float* y, int N,
                              int Cin, int Cout, int H, int W, int dilation, int leaky, void* stream);
uot_status uot_conv2d_backward(const float* x, const float* w, const float* y, const float* dy,
                               float* dx, float* dw, float* db, int N, int Cin, int Cout, int H,
                               int W, int dilation, int leaky, void* stream);
uot_status uot_adam_step(float* param, const float* grad, float* m, float* v, long long n,
                         float lr, float beta1, float beta2, float eps, int step, void* stream);
uot_status uot_mse_grad(const float* pred, const float* target, float* grad, long long n,
                        double* loss_dev, void* stream);
uot_status uot_scale_instances(float* x, const float* scale, int N, long long per_instance,
                               void* stream);
uot_status uot_warmstart_features(const float* p, const float* q, const float* log_eps,
                                  const float* log_lam, float* out, int N, int H, int W,
                                  void* stream);

/*
 * Learned warm start on the tensor cores (not in the paper): BF16 3x3 dilated
 * convolutions with zero padding on images of width 64, as implicit GEMMs on
 * tcgen05 with FP32 accumulation in tensor memory, every operand tile loaded
 * by TMA.  BF16 tensors are passed as void pointers.  Activations are NHWC
 * with a channel stride; weights are K-major rows [rows][9 taps][channels].
 * All calls are asynchronous on `stream`; UOT_EUNSUPPORTED if the driver's
 * tensor-map encoder is unavailable; `err` (device int, may be NULL) is set
 * to 1 if a bounded wait inside a kernel expired (its outputs are then not
 * written).
 *
 * uot_conv_tc_forward: y[p][co] = epi(sum_{tap, c} wk[co][tap][c] x[p + dil s(tap)][c]),
 *   s(tap) = (tap/3 - 1, tap%3 - 1) in (y, x), x out of the image = 0.
 *   x [N][H][W][ldx] (ldx multiple of 8, <= cin_pad; channels ldx..cin_pad-1
 *   read as 0), wk [bn][9][cin_pad] (bn = 16, 64 or 128; rows >= nout are 0),
 *   W = 64, H even, cin_pad a multiple of 64, 1 <= nout <= bn.
 *   mode 0: + bias[co]; 1: + bias then leaky ReLU (slope 0.1); 2: multiplied by
 *   the leaky-ReLU derivative at ref[p][co] (ref [P][ldref], BF16): with the
 *   weights of uot_conv_weights_bf16's wb this is the data gradient of a
 *   layer.  Outputs: y [P][ldy] BF16 (ldy multiple of 16; channels nout..ldy-1
 *   written 0) and/or yf [P][nout] FP32.
 * uot_conv_tc_wgrad: dw[co][ci][kh][kw] (FP32, the layer's shape) =
 *   sum_p dy[p][co] x[p + dil s(3 kh + kw)][ci], from dyT [cout_rows][N][H][W]
 *   (uot_nhwc_transpose of dy) and xT [3][cin_pad][N][H][W]
 *   (uot_nhwc_shift_transpose of x); Cout <= 128, cin_pad 64 or 128; part is
 *   FP32 scratch of splits x 9 x 128 x cin_pad partial sums.
 * uot_nhwc_shift_transpose: xT[d][c][n][y][x] = x[n][y][x + (d-1) dil][c] (0 off the
 *   image), d = 0, 1, 2; x [N][H][W][C], W <= 64.
 * uot_nhwc_transpose: yT[c][p] = y[p][c], y [P][C].
 * uot_bias_grad_bf16: db[c] = sum_p dy[p][c], dy [P][ld].
 * uot_conv_weights_bf16: from FP32 w [Cout][Cin][3][3]: wf [cout_pad][9][cin_pad] =
 *   w[co][ci][tap] and (if wb) wb [cin_rows][9][cout_kpad] = w[co][ci][8 - tap]
 *   (the data-gradient weights), zero padding, BF16.
 * uot_warmstart_features_nhwc: out [N][H][W][64] BF16 = (max(log p, -30),
 *   max(log q, -30), log eps, log lambda) / 4, zeros in channels 4..63.
 * uot_mse_grad_nhwc: for pred [P][2] FP32 (P = N HW) and targets U, V [N][HW]
 *   scaled by scale[n]: grad [P][16] BF16 = 2 (pred - target) / (2P) in
 *   channels 0, 1 (0 beyond), *loss_dev += the mean squared difference.
 * uot_pred_to_potentials: U0[p] = pred[p][0] scale[n], V0[p] = pred[p][1] scale[n].
 */
uot_status uot_conv_tc_forward(const void* x, int ldx, const void* wk, int bn, int N, int H, int W, int cin_pad,
                               int nout, int dil, int mode, const float* bias, const void* ref, int ldref, void* y,
                               int ldy, float* yf, int* err, void* stream);
uot_status uot_conv_tc_wgrad(const void* dyT, int cout_rows, const void* xT, int cin_pad, int N, int H, int W,
                             int dil, int Cout, int Cin, float* part, int splits, float* dw, int* err, void* stream);
uot_status uot_nhwc_shift_transpose(const void* x, int N, int H, int W, int C, int dil, void* xT, void* stream);
uot_status uot_nhwc_transpose(const void* y, long long P, int C, void* yT, void* stream);
uot_status uot_bias_grad_bf16(const void* dy, long long P, int ld, int C, float* db, void* stream);
uot_status uot_conv_weights_bf16(const float* w, int Cout, int Cin, int cout_pad, int cin_pad, int cin_rows,
                                 int cout_kpad, void* wf, void* wb, void* stream);
uot_status uot_warmstart_features_nhwc(const float* p, const float* q, const float* log_eps, const float* log_lam,
                                       void* out, int N, int H, int W, void* stream);
uot_status uot_mse_grad_nhwc(const float* pred, const float* U, const float* V, const float* scale, int N, int HW,
                             void* grad, double* loss_dev, void* stream);
uot_status uot_pred_to_potentials(const float* pred, const float* scale, int N, int HW, float* U0, float* V0,
                                  void* stream);

#ifdef __cplusplus
}
#endif

#endif /* UOT_H */

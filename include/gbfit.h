/*
 * gbfit.h -- C ABI of the GB300 trust-region-reflective curve-fit library.
 *
 * The library fits h(x; p) to observations (x_i, y_i) with per-point
 * uncertainties sigma_i by minimising f(p) = 1/2 sum_i ((h(x_i;p) - y_i)/sigma_i)^2
 * (paper Section 2, Eqs. residual and msqe; Appendix C, Eq. explicit) with the
 * trust-region method of Algorithms 1-3, Coleman-Li reflective bounds, and the
 * scaled subproblem solved through the n x n factorisation of J^T J
 * (Appendix B).  Everything after argument checking runs on one GPU: model,
 * residual and Jacobian rows are formed in registers and reduced to J^T J,
 * J^T r and the cost without writing J to memory; the n x n step, ratio,
 * radius update and termination run on the device; every iteration of a
 * call runs inside one persistent (cooperative) kernel launch, so a fit
 * makes no host round trip per iteration.
 *
 * Conventions shared by every entry point
 *   - Return value: GBFIT_OK (0) or a negative GBFIT_E_* code; the message of
 *     the last error on the calling thread is gbfit_last_error().
 *   - Data arrays (xdata, ydata, sigma, offsets' data) may be device pointers
 *     (preferred; read in place, never written or freed) or host pointers
 *     (detected with cudaPointerGetAttributes; copied to the device inside the
 *     call, pinned host memory copies fastest).
 *   - Parameter-sized arrays (p0, lb, ub, x_scale) and all outputs are HOST
 *     pointers owned by the caller.
 *   - cuda_stream is a cudaStream_t (NULL = legacy default stream).  The call
 *     enqueues its work on that stream and returns after the results have
 *     been copied back (one stream synchronisation per call).
 *   - Calls on one device are serialised by an internal lock (the device
 *     workspace and the cached launch are shared).
 *   - Fit non-convergence is not an error: it is reported in fit_status.
 */
#ifndef GBFIT_H
#define GBFIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBFIT_VERSION 1

/* ---- return codes ---- */
#define GBFIT_OK                 0
#define GBFIT_E_INVALID_ARG     -1  /* bad id/layout/dtype, m < n, lb >= ub, non-finite p0, sigma <= 0 or non-finite data */
#define GBFIT_E_INFEASIBLE_X0   -2  /* p0 not strictly inside (lb, ub) */
#define GBFIT_E_OOM             -3  /* device or pinned allocation failed */
#define GBFIT_E_BUDGET          -4  /* serving: request larger than the HBM budget */
#define GBFIT_E_CUDA            -5  /* a CUDA runtime call failed (message has the CUDA error) */
#define GBFIT_E_TIMEOUT         -6  /* a bounded device wait gave up */
#define GBFIT_E_UNSUPPORTED     -7  /* valid request this build does not implement */
#define GBFIT_E_CANCELLED       -8  /* serving: the request was cancelled (gbfit_server_cancel) */

/* ---- fit_status (per fit; mirrors the termination tests) ---- */
#define GBFIT_FIT_NUMERICAL     -1  /* non-finite cost or Jacobian at p0, or a bounded wait for
                                       streamed data gave up (the sums are incomplete) */
#define GBFIT_FIT_MAX_NFEV       0  /* nfev reached max_nfev */
#define GBFIT_FIT_GTOL           1  /* ||v * g||_inf < gtol */
#define GBFIT_FIT_FTOL           2  /* accepted step with f - f_new < ftol * f */
#define GBFIT_FIT_XTOL           3  /* step with ||w|| < xtol * (xtol + ||x||); mixed precision, FP32
                                       passes: also a rejected trial whose predicted reduction is
                                       below ftol * f (a stall in the FP32 rounding noise) */
#define GBFIT_FIT_FTOL_XTOL      4  /* both on the same step */
#define GBFIT_FIT_INVALID_DATA  -2  /* sigma <= 0 or non-finite x/y/sigma found on the device */

/* ---- built-in models (model_id) ---- */
#define GBFIT_MODEL_GAUSS1D  0  /* A exp(-(x-mu)^2/(2 s^2)) + c;          p = (A, mu, s, c)           */
#define GBFIT_MODEL_DEXP     1  /* a1 exp(-x/t1) + a2 exp(-x/t2) + c;     p = (a1, t1, a2, t2, c)     */
#define GBFIT_MODEL_GAUSS2D  2  /* rotated elliptical 2D Gaussian + c;     p = (A, x0, y0, sx, sy, theta, c);
                                   u = (X-x0)cos th + (Y-y0)sin th, v = -(X-x0)sin th + (Y-y0)cos th,
                                   h = A exp(-u^2/(2 sx^2) - v^2/(2 sy^2)) + c                          */
#define GBFIT_MODEL_POLY2    3  /* p0 + p1 x + p2 x^2 (linear test model); p = (p0, p1, p2)           */
#define GBFIT_NUM_MODELS     4
#define GBFIT_MAX_PARAMS     8

/* ---- x layouts ---- */
#define GBFIT_X_VEC   0  /* xdata: [m] (1D models)                                            */
#define GBFIT_X_SOA2  1  /* xdata: [2][m], X row then Y row (2D models)                       */
#define GBFIT_X_GRID  2  /* xdata unused: point i is pixel X = i % W, Y = i / W, W*H == m      */

/* ---- data dtypes ---- */
#define GBFIT_F32 0
#define GBFIT_F64 1

/* ---- precision modes ---- */
#define GBFIT_PREC_FP64   0  /* plain: model, Jacobian, reductions and solve in FP64           */
#define GBFIT_PREC_MIXED  1  /* model and Jacobian rows in FP32 (actual reduction in the
                                cancellation-free difference form), tile sums promoted to
                                FP64; combine, n x n solve, ratio and tests in FP64            */

/* ---- robust losses (the paper's Section 5 names "various loss functions"
 * without stating them; the library's reading): the cost becomes
 * f = 1/2 C^2 sum rho(z_i), z_i = (r_i / C)^2 with C = f_scale, and the method
 * runs on rows rescaled to the loss's gradient and Gauss-Newton Hessian
 * (J_i * sqrt(s_i), r_i * rho'(z_i) / sqrt(s_i), s_i = rho' + 2 z rho'').
 * pcov then comes from the rescaled Jacobian and the robust cost. ---- */
#define GBFIT_LOSS_LINEAR   0  /* rho = z                                  */
#define GBFIT_LOSS_SOFT_L1  1  /* rho = 2 (sqrt(1 + z) - 1)                */
#define GBFIT_LOSS_HUBER    2  /* rho = z (z <= 1), 2 sqrt(z) - 1 beyond   */
#define GBFIT_LOSS_CAUCHY   3  /* rho = ln(1 + z)                          */
#define GBFIT_LOSS_ARCTAN   4  /* rho = arctan(z)                          */

typedef struct gbfit_options {
    double ftol, xtol, gtol;   /* termination tolerances (defaults 1e-8)                         */
    int max_nfev;              /* <= 0: 100 * n                                                  */
    int x_scale_jac;           /* 1: D from running Jacobian column norms; 0: D = 1/x_scale      */
    const double* x_scale;     /* host [n] or NULL (all ones); ignored when x_scale_jac          */
    int absolute_sigma;        /* 1: pcov not rescaled by 2 cost / (m - n)                       */
    int precision;             /* GBFIT_PREC_*                                                   */
    int tile_points;           /* points per reduction tile; 0 = library choice                  */
    int group_tiles;           /* tiles per first-level combine group; 0 = library choice        */
    int loss;                  /* GBFIT_LOSS_* (default linear)                                  */
    int reserved[1];
    double f_scale;            /* robust loss scale C > 0; 0 reads as 1                          */
    /* Precision guard of GBFIT_PREC_MIXED (linear loss, no full covariance):
     * a fit continues with FP64 evaluation passes from its current point when
     * the equilibrated condition number of its Gram exceeds guard_cond, or
     * when it meets a tolerance while its estimated FP32 rounding floor in
     * popt (relative, |dp| / max(|p|, 1)) exceeds guard_floor; max_nfev
     * bounds all evaluations together.  <= 0: the defaults below; +inf: off
     * (every pass FP32, the fastest and least accurate form). */
    double guard_cond;
    double guard_floor;
    /* Limit, in seconds, of the loop kernel's grid-wide waits (round barrier,
     * owner wait, idle wait of queue mode); past it the launch aborts and the
     * call returns GBFIT_E_TIMEOUT with the context still usable.  <= 0: the
     * default, 10 s.  Small values exist for testing that path: a launch
     * whose waits are shorter than one trust-region step times out. */
    double wait_limit_s;
} gbfit_options;

#define GBFIT_GUARD_COND_DEFAULT 1.0e3
#define GBFIT_GUARD_FLOOR_DEFAULT 1.0e-7

/* Test entry point: y[i] = 1/x[i] by the trust-region step's FP64 reciprocal
 * (Newton-Raphson from the FP32 reciprocal; the paper has no counterpart: it
 * is an implementation detail of the on-device step, exposed so that its
 * accuracy can be checked against 1.0 / x).  x, y: device arrays of n
 * doubles; synchronous on cuda_stream. */
int gbfit_check_rcp64(const double* x, double* y, int64_t n, void* cuda_stream);

/* Library version (GBFIT_VERSION). */
int gbfit_version(void);

/* Message of the last failing call on this thread ("" if none).  Owned by the library. */
const char* gbfit_last_error(void);

/* Fill *opt with defaults (tolerances 1e-8, mixed precision, D = I). */
int gbfit_default_options(gbfit_options* opt);

/* Registry query: number of parameters and coordinate dimensions of model_id
 * (built-in or user-defined). */
int gbfit_model_info(int model_id, int* n_params, int* x_dims);

/* ---- user-defined models (the paper's user-written fit function, whose
 * Jacobian JAX forms by automatic differentiation: Section 2, Eq. jacobian).
 *
 * source: CUDA C++ text that defines, at namespace scope,
 *     template <class T, class S> __device__ T NAME(const T* p, S x, S x2);
 * returning h(x; p) for the n parameters p[0..n) at coordinate x (x2: second
 * coordinate of a 2D model, 0 for 1D).  T is a number type of the library
 * (forward-mode dual numbers: FP64 value and partials for the plain path;
 * for the mixed path FP32 value at p, the difference h(p') - h(p) propagated
 * without cancellation, and FP32 partials at p'); S is float or double.  The
 * body may use + - * / between T values and plain numbers, and exp, log,
 * sqrt, pow(T, number), sin, cos, tanh, atan, square.  Smooth models only.
 * func_name: NAME (NULL: "model").  n_params: 1..GBFIT_MAX_PARAMS.  x_dims:
 * 1 (layout GBFIT_X_VEC) or 2 (GBFIT_X_SOA2 / GBFIT_X_GRID).
 *
 * The source is compiled once, here, with NVRTC (loaded from the CUDA
 * toolkit at run time) into the library's persistent loop kernels for both
 * precisions; the code is loaded on the device at the model's first fit.
 * Returns the new id (>= GBFIT_USER_MODEL_BASE) in *model_id, usable with
 * gbfit_curve_fit, gbfit_curve_fit_batch and gbfit_evaluate (the serving,
 * tuning and allocation-free entry points take built-in models only).
 * Errors: GBFIT_E_INVALID_ARG (bad arguments, or the source does not compile:
 * the start of the compiler log is in gbfit_last_error(), all of it in
 * gbfit_model_log), GBFIT_E_UNSUPPORTED (NVRTC not found), GBFIT_E_OOM
 * (more than GBFIT_MAX_USER_MODELS models).  Thread-safe. ---- */
#define GBFIT_USER_MODEL_BASE 100
#define GBFIT_MAX_USER_MODELS 64
int gbfit_model_register(const char* source, const char* func_name, int n_params, int x_dims, int* model_id);

/* Compiler log of the last gbfit_model_register call on any thread
 * (NUL-terminated, truncated to cap bytes); *len = full length. */
int gbfit_model_log(char* buf, size_t cap, size_t* len);

/*
 * One fit (paper Section 2, Algorithm 1; the SciPy-style problem statement the
 * paper's drop-in claim refers to).
 *   model_id   GBFIT_MODEL_*
 *   xdata      coordinates in x_layout (NULL for GBFIT_X_GRID), dtype
 *   m          number of points (>= n)
 *   x_layout   GBFIT_X_*; grid_wh = host int64[2] {W, H} for GBFIT_X_GRID, else NULL
 *   ydata      [m] observations, dtype
 *   sigma      [m] per-point standard deviations (> 0, Appendix C Eq. svector) or NULL (= 1)
 *   dtype      GBFIT_F32 | GBFIT_F64 (applies to xdata, ydata, sigma)
 *   p0         host [n] start, strictly inside (lb, ub)
 *   lb, ub     host [n] bounds (+-INFINITY for none) or NULL (unbounded)
 *   opt        options or NULL (defaults)
 * Outputs (host): popt [n]; pcov [n*n] row-major or NULL; cost = f(popt);
 *   nfev (function evaluations, including the one at p0); fit_status GBFIT_FIT_*.
 * Errors: GBFIT_E_INVALID_ARG, GBFIT_E_INFEASIBLE_X0, GBFIT_E_OOM, GBFIT_E_CUDA.
 */
int gbfit_curve_fit(int model_id,
                    const void* xdata, int64_t m, int x_layout, const int64_t* grid_wh,
                    const void* ydata, const void* sigma, int dtype,
                    const double* p0, const double* lb, const double* ub,
                    const gbfit_options* opt,
                    double* popt, double* pcov, double* cost, int* nfev, int* fit_status,
                    void* cuda_stream);

/*
 * Many independent fits of one model over concatenated data (paper Appendix A's
 * fixed-size padding replaced by segment offsets: no point of one fit touches
 * another).  All fits iterate together in one launch: each round evaluates
 * every running fit once, and a fit that has finished takes no further work.
 * A fit's reduction shape comes from the tile table (gbfit_tune_shape) and
 * depends only on its own m, so its result is bit-identical alone (with the
 * same shape) and in any batch.
 *   nfits      number of fits (>= 1)
 *   offsets    host int64 [nfits + 1], offsets[0] = 0, strictly increasing by >= n
 *   xdata      [total] (GBFIT_X_VEC) or [2][total] (GBFIT_X_SOA2)
 *   ydata, sigma  [total] (sigma may be NULL)
 *   p0         host [nfits * n];  lb, ub host [nfits * n] or NULL
 * Outputs (host, per fit): popt [nfits*n], pcov [nfits*n*n] or NULL, cost [nfits],
 *   nfev [nfits], fit_status [nfits].
 */
int gbfit_curve_fit_batch(int model_id, int nfits, const int64_t* offsets,
                          const void* xdata, int x_layout,
                          const void* ydata, const void* sigma, int dtype,
                          const double* p0, const double* lb, const double* ub,
                          const gbfit_options* opt,
                          double* popt, double* pcov, double* cost, int* nfev, int* fit_status,
                          void* cuda_stream);

/*
 * Tiling of batched and served fits (no paper counterpart: the paper's JAX
 * kernels are shaped per problem by its compiler).  A fit's evaluation pass
 * is cut into reduction tiles of tile_points points (one CTA reduces one
 * tile to a row of partial sums); rows are combined in groups of
 * group_tiles, then across groups.  The best shape depends on the model, the
 * precision mode and m.  The library keeps one table indexed
 * [model_id][precision][floor(log2 m)] (the last bucket also takes larger m);
 * gbfit_curve_fit_batch and the server read it for every fit whose options
 * leave tile_points / group_tiles at 0, so a fit's shape depends only on its
 * own m and the installed table.  Single fits (gbfit_curve_fit) instead
 * spread m over every SM.  Defaults: mixed 32768 points, FP64 4096 points,
 * groups of 32 (a fit smaller than its tile is one tile).
 */
#define GBFIT_TUNE_BUCKETS 32
typedef struct gbfit_tune_table {
    int32_t tile_points[GBFIT_NUM_MODELS][2][GBFIT_TUNE_BUCKETS];   /* [model][precision][log2 m] */
    int32_t group_tiles[GBFIT_NUM_MODELS][2][GBFIT_TUNE_BUCKETS];
} gbfit_tune_table;

/* Copy out the installed table. */
int gbfit_tune_get(gbfit_tune_table* out);

/* Install a table (host memory, copied).  Each tile_points must be a multiple
 * of 256 in [256, 2^24], each group_tiles in [1, 1024]; otherwise
 * GBFIT_E_INVALID_ARG and the installed table is unchanged.  Servers created
 * earlier keep admitting with the table installed when they admit. */
int gbfit_tune_set(const gbfit_tune_table* in);

/* The shape a batched or served fit of m points gets from the installed table. */
int gbfit_tune_shape(int model_id, int precision, int64_t m, int* tile_points, int* group_tiles);

/*
 * Autotuner: for every bucket b whose middle size m_b = 1.5 * 2^b lies in
 * [2^10, m_max], times batched fits of model_id with m_b points each (as many
 * fits as fill points_per_run points, at most 4096; points_per_run <= 0
 * means 2^25) for candidate shapes: tile_points 2^10 .. 2^18 (and one tile
 * per fit), group_tiles 8, 32, 128.  Every fit runs exactly 4 evaluations on
 * synthetic calibration data drawn on the device (FP32 for the mixed mode,
 * FP64 for the plain one), timed with CUDA events.  Each bucket gets, among
 * the shapes within 3 % of its fastest, the one with the most tiles per fit
 * (the shortest passes for the largest fits of a mixed batch); buckets below
 * 2^10 take bucket 10's, buckets above m_max keep their entries.  out (optional) receives the resulting table.
 * Allocates and frees device memory for the calibration data; takes about
 * a second per bucket.  Errors: GBFIT_E_INVALID_ARG, GBFIT_E_OOM, GBFIT_E_CUDA.
 */
int gbfit_autotune(int model_id, int precision, int64_t m_max, int64_t points_per_run,
                   gbfit_tune_table* out, void* cuda_stream);

/*
 * One fit with a full covariance matrix of the observations (Appendix C,
 * Eq. covariance; SciPy's 2D sigma).  C = L L^T is factored once on the
 * device (FP64 Cholesky, then X = L^-1 by forward substitution) and the
 * method runs on L^-1 r and L^-1 J (Eqs. slsq1, slsq2): every evaluation is
 * two rounds of the loop kernel, the points into a buffer, then rows of
 * X [h - y, J] reduced like points (the row-parallel product takes the place
 * of the paper's per-iteration triangular solves).
 *   cov   [m][m] FP64, host or device, symmetric positive definite (only the
 *         lower triangle is read); m <= GBFIT_COV_MAX_M
 *   other arguments as gbfit_curve_fit (no sigma; linear loss only).
 * Device memory: about 3 m^2 * 8 bytes (C / L, X in FP64, X in FP32 for the
 * mixed path), kept between calls.  Staging costs O(m^3) FP64 work (tens of
 * ms at m = 4096) and one synchronisation.
 * Errors: as gbfit_curve_fit, plus GBFIT_E_INVALID_ARG when C is not
 * positive definite, GBFIT_E_UNSUPPORTED for a robust loss.
 */
#define GBFIT_COV_MAX_M 8192
int gbfit_curve_fit_cov(int model_id, const void* xdata, int64_t m, int x_layout, const int64_t* grid_wh,
                        const void* ydata, const double* cov, int dtype, const double* p0, const double* lb,
                        const double* ub, const gbfit_options* opt, double* popt, double* pcov, double* cost,
                        int* nfev, int* fit_status, void* cuda_stream);

/* gbfit_evaluate with a full covariance matrix: B, g and cost of the
 * whitened problem at p (out as gbfit_evaluate). */
int gbfit_evaluate_cov(int model_id, const void* xdata, int64_t m, int x_layout, const int64_t* grid_wh,
                       const void* ydata, const double* cov, int dtype, const double* p, int precision,
                       double* out, void* cuda_stream);

/*
 * Evaluate the fused reduction once at parameters p (no iteration): the
 * packed upper triangle of B = J^T J (n(n+1)/2), g = J^T r (n) and cost
 * f = r^T r / 2, all FP64, for the given precision mode (paper Eqs. msqe,
 * gradient, hessian).  Output is a host array out[n(n+1)/2 + n + 1].
 */
int gbfit_evaluate(int model_id,
                   const void* xdata, int64_t m, int x_layout, const int64_t* grid_wh,
                   const void* ydata, const void* sigma, int dtype,
                   const double* p, int precision, int tile_points,
                   double* out, void* cuda_stream);

/*
 * Solve one scaled trust-region subproblem on the device (paper Algorithm 1's
 * step with Algorithm 2; Appendix B): given the symmetric n x n B (host,
 * row-major), g [n], radius Delta and the previous LM parameter alpha0,
 * returns p [n] minimising g.p + p^T B p / 2 within ||p|| <= Delta (to
 * Algorithm 2's accuracy), the LM parameter alpha and the eigenvalues lam [n]
 * (ascending order not guaranteed).  Runs the same device code as the fit.
 */
int gbfit_tr_subproblem(int n, const double* B, const double* g, double Delta, double alpha0,
                        double* p, double* alpha, double* lam, void* cuda_stream);

/*
 * Serving: continuous batching of independent fit requests (many models and
 * sizes) on one GPU.  The server owns a device pool of hbm_budget_bytes for
 * request data and up to max_slots fit records that stay on the device while
 * a fit runs.  Each gbfit_server_step: (1) retires fits that finished,
 * releasing their memory and slot; (2) admits queued requests in arrival
 * order while a slot is free and their data fits in the pool (copying it in);
 * (3) runs `rounds_per_step` trust-region iterations for every admitted fit
 * in shared launches (one evaluation kernel per iteration for all fits).
 * A fit's reduction tiling depends only on its own m (through the tile
 * table, gbfit_tune_shape), so its result is the same, bit for bit, whatever
 * else is being served.
 */
typedef struct gbfit_server gbfit_server;

typedef struct gbfit_server_config {
    size_t hbm_budget_bytes;   /* device pool for request data (x, y, sigma) and tile scratch */
    int max_slots;             /* fits resident at once (default 4096)                         */
    int precision;             /* GBFIT_PREC_*                                                 */
    int rounds_per_step;       /* iterations per step (default 4)                              */
    int reserved[4];
    double guard_cond;         /* precision guard of mixed served fits, as in gbfit_options    */
    double guard_floor;
} gbfit_server_config;

typedef struct gbfit_request {
    int model_id, x_layout, dtype, has_bounds;
    int64_t m, grid_w, grid_h;           /* grid_w, grid_h for GBFIT_X_GRID                     */
    const void* xdata;                   /* host or device; copied into the pool on admission   */
    const void* ydata;
    const void* sigma;                   /* may be NULL                                        */
    double p0[GBFIT_MAX_PARAMS], lb[GBFIT_MAX_PARAMS], ub[GBFIT_MAX_PARAMS];
    double ftol, xtol, gtol;
    int max_nfev;
    uint64_t tag;                        /* returned with the result                            */
    int loss;                            /* GBFIT_LOSS_* (0 = linear)                           */
    double f_scale;                      /* robust loss scale; 0 reads as 1                     */
} gbfit_request;

typedef struct gbfit_result_rec {
    uint64_t ticket, tag;
    int status;                          /* GBFIT_OK or a GBFIT_E_* code for this request       */
    int fit_status, nfev, n_params;
    double cost;
    double popt[GBFIT_MAX_PARAMS];
    double t_submit, t_admit, t_done;    /* seconds, host steady clock                          */
} gbfit_result_rec;

/* Create a server on the current device (allocates the pool once). */
int gbfit_server_create(const gbfit_server_config* cfg, gbfit_server** out);

/* Queue a request (its data pointers must stay valid until it is admitted).
 * GBFIT_E_BUDGET if its data can never fit in the pool. */
int gbfit_server_submit(gbfit_server* s, const gbfit_request* req, uint64_t* ticket);

/* Retire, admit, and run one step of iterations; *n_active = fits resident
 * after the step, *n_queued = requests still waiting.  Blocking. */
int gbfit_server_step(gbfit_server* s, int* n_active, int* n_queued);

/* Cancel a queued or resident request (between steps: nothing of it is in
 * flight then).  Its record is queued for gbfit_server_poll with status
 * GBFIT_E_CANCELLED, popt and cost of its current point (p0 if it never ran)
 * and the evaluations done; its pool, tile and slot are freed.
 * GBFIT_E_INVALID_ARG if the ticket is neither queued nor resident. */
int gbfit_server_cancel(gbfit_server* s, uint64_t ticket);

/* Snapshot of a resident fit's state between steps (checkpoint): the
 * trust-region state kept on the device (point, trial point, radius, Gram,
 * scaling, eigen cache, pass constants, counters).  Resubmitting the same
 * request with it (gbfit_server_submit_resume) continues the fit where it
 * was; with the same data and tile table the result is bitwise the one of an
 * uninterrupted fit. */
#define GBFIT_SNAPSHOT_MAGIC 0x67626673u
#define GBFIT_SNAPSHOT_STATE_BYTES 2048
typedef struct gbfit_fit_snapshot {
    uint32_t magic;                     /* GBFIT_SNAPSHOT_MAGIC                          */
    uint32_t state_bytes;               /* bytes of state[] in use                       */
    int32_t model_id, precision;
    int64_t m;
    int64_t reserved;                   /* (state[] starts on a 16-byte boundary)        */
    unsigned char state[GBFIT_SNAPSHOT_STATE_BYTES];
} gbfit_fit_snapshot;

/* GBFIT_E_INVALID_ARG unless the ticket is resident (admitted, not finished). */
int gbfit_server_snapshot(gbfit_server* s, uint64_t ticket, gbfit_fit_snapshot* out);

/* Queue a request that resumes from a snapshot of the same model, size and
 * server precision (refused otherwise); its p0 is ignored. */
int gbfit_server_submit_resume(gbfit_server* s, const gbfit_request* req, const gbfit_fit_snapshot* snap,
                               uint64_t* ticket);

/* Copy up to max finished results (oldest first) into out; *count = copied. */
int gbfit_server_poll(gbfit_server* s, gbfit_result_rec* out, int max, int* count);

/* Free the server and its pool. */
int gbfit_server_destroy(gbfit_server* s);

/*
 * gbfit_evaluate without any device or pinned-host allocation (the paper has
 * no counterpart).  It serves callers that may not allocate memory when they
 * call: applications whose memory manager owns all device memory (a pool
 * sized at start-up, where a cudaMalloc beside it fails or fragments it), and
 * loops that cannot take the implicit device-wide synchronisation of
 * cudaMalloc / cudaFree.  Same arguments and output as gbfit_evaluate, with
 * these differences:
 *   - xdata, ydata and sigma must be device pointers (no staging copy);
 *   - the pass's scratch (tile and group partial sums, arrival counters, the
 *     one-fit job record) lives in a fixed file-scope device array of about
 *     1 MB that every GPU loading the library keeps until the process exits;
 *     at most 2048 reduction tiles fit: m <= 134,217,728 points with
 *     tile_points = 0 (the default tile is made coarser, up to 65536 points,
 *     where it would need more tiles), m <= 2048 * tile_points otherwise;
 *     larger requests fail with GBFIT_E_INVALID_ARG, before any CUDA call,
 *     with a message giving the limit;
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture;
 *   - the call is synchronous: it enqueues an upload of the job record, two
 *     kernels and the result copy on cuda_stream, then waits on that stream
 *     (also on its error paths, once anything is enqueued) before it returns;
 *   - every call reuses the same array, which keeps the last call's
 *     contents (each call re-initialises what must start at zero); calls
 *     whose work overlapped on the GPU would race on it, which the host lock
 *     and the wait at the end of each call prevent for calls made through
 *     this entry point.
 */
int gbfit_evaluate_noalloc(int model_id,
                           const void* xdata, int64_t m, int x_layout, const int64_t* grid_wh,
                           const void* ydata, const void* sigma, int dtype,
                           const double* p, int precision, int tile_points,
                           double* out, void* cuda_stream);

/*
 * Runtime counters and per-launch timing (the per-operation timing the paper
 * reports in Section 4 / Fig. 3, taken here with CUDA events).
 * Counters are process-wide and accumulate over calls until reset.
 */
typedef struct gbfit_stats {
    int64_t calls;            /* gbfit_curve_fit / _batch / _evaluate calls            */
    int64_t fits;             /* fits completed                                        */
    int64_t kernel_launches;  /* kernels the library launched                           */
    int64_t graph_rounds;     /* rounds of the persistent loop kernel (one evaluation of
                                 every running fit each)                              */
    int64_t passes;           /* data passes = sum over fits of nfev                   */
    double point_passes;      /* sum over fits of m * nfev                             */
    double eval_ms;           /* profiling on: summed CUDA-event time of loop-kernel launches */
    int64_t eval_launches;    /* profiling on: loop-kernel launches timed              */
    double phase_cycles[32];  /* summed over fits and iterations (SM cycles unless noted):
                                 0 own tile, 1 combine, 2 accept/terminate logic,
                                 3 n x n eigen-decomposition, 4 combine: store, fence and
                                 arrival, 5 step (solve, Algorithm 2, bounded selection),
                                 6 pass constants, 7 final pcov, 8-9 combine: group,
                                 final, 10-13 eigen: warm start, FP32 Jacobi,
                                 re-orthonormalisation, refinement, 14 FP32 Jacobi sweeps
                                 (count), 15 refinement passes (count), 16 Gauss-Newton
                                 fast path, 17 fast-path steps (count), 18 eigen
                                 decompositions (count), 19 Algorithm 2 iterations
                                 (count), 20 bounded non-full steps (count), 21 item start to
                                 tile start, 22 tile loop (of 0), 23 waits for streamed
                                 chunks inside the tile loop (of 22); owner mode (ns of the
                                 global timer, per round of the fit's owner CTA): 24 round
                                 (barrier exit to barrier arrival), 25 owner's wait for the
                                 group sums, 26 barrier (arrival to exit), 27 launch start
                                 to the first round (once per fit); 28 evaluations in FP64
                                 by a mixed fit (count), 29-30 precision-guard escalations
                                 and FP64 finishes (count), 31 wide trials evaluated in the
                                 direct form (count) */
    double host_ms;           /* host wall time inside the run of fits (job set-up, launch,
                                 wait for the device, result copy)                    */
    double loop_busy_ms;      /* loop kernel, summed over CTAs: time in rounds' work    */
    double loop_wait_ms;      /* loop kernel, summed over CTAs: time at round barriers  */
    int64_t loop_ctas;        /* CTAs summed over loop-kernel launches (busy / ctas = the
                                 average CTA's time in work per launch)               */
} gbfit_stats;

/* Zero the counters. */
int gbfit_stats_reset(void);

/* Copy the counters into *out. */
int gbfit_stats_get(gbfit_stats* out);

/*
 * on = 1: each launch of the loop kernel (one per fit or batch call) is
 * bracketed by CUDA events on the call's stream and its time added to
 * gbfit_stats.eval_ms (one extra host synchronisation per call).  A short
 * hold kernel (60 us) is queued ahead of the start event, so that the host
 * has submitted the launch by the time the event fires: the events time the
 * kernel, not the host's submission.
 * on = 0 (default): no events, no hold.  Results are identical.
 */
int gbfit_set_profiling(int on);

#ifdef __cplusplus
}
#endif
#endif /* GBFIT_H */

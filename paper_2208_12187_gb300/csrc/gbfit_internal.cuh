// Internal device/host data structures of libgbfit (not part of the C ABI).
#pragma once
#include "rtc_compat.cuh"

namespace gbfit {

constexpr int NMAX = 8;                          // max parameters (rotated 2D Gaussian has 7)
constexpr int NTMAX = NMAX * (NMAX + 1) / 2;     // packed upper triangle size
constexpr int KMAX = NTMAX + NMAX + 3;           // accumulator slots per evaluation
constexpr int EVAL_THREADS = 256;                // threads per reduction CTA
constexpr int GROUP_TILES = 32;                  // tiles per first-level combine group
constexpr int PF = 32;                           // float pass constants (mixed)
constexpr int PD = 16;                           // double pass constants (plain)

enum Prec { PREC_FP64 = 0, PREC_MIXED = 1 };
enum Layout { X_VEC = 0, X_SOA2 = 1, X_GRID = 2 };
enum DType { F32 = 0, F64 = 1 };
enum WKind { W_NONE = 0, W_ARRAY = 1, W_SIGMA = 2 };
enum RunState { RS_RUNNING = 0, RS_DONE = 1 };
// PH_REINIT: the fit's current point is evaluated again in FP64 (precision
// guard of the mixed path); the fit then continues with FP64 passes.
// PH_WIDE: a trial of the mixed path whose predicted reduction is at least
// WIDE_PRED_FRAC of f, evaluated in the direct form (no difference); its
// actual reduction is f - f' of the two FP32-evaluated costs.
enum Phase { PH_INIT = 0, PH_TRIAL = 1, PH_REINIT = 2, PH_WIDE = 3 };
constexpr double WIDE_PRED_FRAC = 1e-2;
enum Loss { LOSS_LINEAR = 0, LOSS_SOFT_L1, LOSS_HUBER, LOSS_CAUCHY, LOSS_ARCTAN };
// pass-constant slots holding the robust loss's C^2 and 1/C^2
constexpr int PF_C2 = PF - 1, PF_IC2 = PF - 2, PD_C2 = PD - 1, PD_IC2 = PD - 2;

// Accumulator slot layout for a model with n parameters (NT = n(n+1)/2):
//   [0, NT)        packed upper triangle of J'^T J' at the evaluated point
//   [NT, NT+n)     J'^T r'
//   NT+n           sum r'^2                        (= 2 f at the evaluated point)
//   NT+n+1         sum dr (2 r + dr)   mixed only  (= 2 (f' - f), cancellation-free); at a fit's
//                                                  first evaluation (dr = 0) it carries sum (w h)^2
//                                                  instead (scale of the FP32 rounding of r, for the
//                                                  precision guard)
__host__ __device__ constexpr int n_tri(int n) { return n * (n + 1) / 2; }
__host__ __device__ constexpr int n_acc(int n, int prec) { return n_tri(n) + n + (prec == PREC_MIXED ? 2 : 1); }

// Immutable description of one fit (uploaded once).
struct FitDesc {
    int model, n, layout, dtype;
    int prec, wkind, bounded, jac_scale;
    int64_t m;
    int64_t grid_w;
    const void* x;         // VEC: [m]; SOA2: X row at x, Y row at x2
    const void* x2;
    const void* y;
    const void* w;         // staged weights (plain) or sigma (mixed) or null
    int tile_points, n_tiles, n_groups, max_nfev;
    int64_t tile_base;     // first row of this fit in the tile-partial buffer
    int64_t group_base;    // first row in the group-partial buffer / group counters
    double lb[NMAX], ub[NMAX], xscale[NMAX];
    double ftol, xtol, gtol;
    int absolute_sigma, group_tiles;
    int loss, pad2;
    double f_scale;        // robust loss scale C (1 for the linear loss)
    // full covariance (Appendix C): rounds alternate between evaluating the
    // points into hbuf and reducing rows of X hbuf, X = L^-1 (C = L L^T)
    int cov;
    int eval_only;         // one evaluation at p (gbfit_evaluate): no trust-region work, no pcov
    unsigned long long wait_ns;   // limit of the loop kernel's grid-wide waits (the launch takes the smallest)
    // precision guard of the mixed path (off: +inf): a fit whose equilibrated
    // Gram condition number exceeds guard_cond continues with FP64 passes
    // from its current point; a fit that meets a tolerance while its
    // estimated FP32 rounding floor in popt exceeds guard_floor finishes with
    // FP64 passes
    double guard_cond, guard_floor;
    const void* xinv;      // X, [m][m] column-major (X_ij at xinv[j m + i]), lower triangle, zeros above;
                           // FP32 for the mixed path, FP64 for the plain path
    void* hbuf;            // [columns][m]: mixed h - y, dh, J_0..J_n-1 (FP32); plain h' - y, J (FP64)
};
constexpr int COV_ROWS = 32;                     // points / rows per work item of a covariance fit

// Mutable per-fit state, kept on the device across iterations.
struct alignas(16) FitState {
    // --- read by the evaluation pass ---
    int run;               // RunState
    int phase;             // Phase of the pending evaluation
    int bad_data;          // set by the INIT pass when sigma <= 0 or non-finite data
    int cov_stage;         // covariance fits: 0 = the next round evaluates points, 1 = it reduces rows
    float pf[PF];          // mixed-precision pass constants (base x -> trial xt)
    double pd[PD];         // plain pass constants (trial xt)
    // --- TRF state ---
    int fit_status, nfev, njev, factor_valid;
    int last_kind, alg2_iters, jacobi_sweeps, has_basis;
    int eval64;            // mixed path: 1 once the fit evaluates in FP64 (precision guard)
    int n_eval64;          // evaluations done in FP64 by a mixed fit
    int guard_why;         // why the guard moved the fit to FP64 (GUARD_* in trf_step.cuh; 0: it did not)
    int pad_g;
    double f, Delta, alpha;
    double x[NMAX], xt[NMAX], g[NMAX];
    double B[NTMAX];       // packed Gram at x
    double scale_inv[NMAX];
    double V[NMAX * NMAX]; // eigenvectors (columns) of the scaled model matrix at x
    double lam[NMAX];
    double predicted, step_norm, s_norm, xtol_thr;
    double s_h[NMAX];      // scaled step of the pending trial
    double floor_x;        // mixed path: estimated FP32 rounding floor of popt at x (relative)
    double serel_x;        // mixed path: largest standard error relative to its parameter at x
    double wh2;            // mixed path: sum (w h)^2 at p0 (from the first evaluation)
    // --- (the step reads everything above from a shared-memory copy) ---
    unsigned long long trace[32];  // SM cycles / ns / counts per phase (TracePhase), summed over iterations
};

struct WorkItem { int fit; int tile; };

constexpr int SM_IDS = 1024;                     // bound on %nsmid for the per-SM CTA counters

struct FitResult;

// Everything one launch of the iteration graph works on.  It lives at the
// start of the job buffer in device memory (kernels receive its address), so
// the cached graph stays valid while per-call sizes and scratch change.
struct Engine {
    FitResult* results;    // [fits]
    int* out;              // result header: [0] running, [1] rounds, [2] abort; u64 words 2-3: loop busy / wait ns
    FitDesc* desc;
    FitState* state;
    WorkItem* items;
    int* n_items;
    double* tile_part_d;   // [tiles][KMAX] tile sums (FP64; mixed tiles are summed in FP32 and
                           // widened by their own CTA, so that the combine only adds)
    double* group_part;    // [groups][KMAX]
    int* group_cnt;        // [groups]
    int* fit_cnt;          // [fits]
    int* running;          // number of running fits
    int* rounds;           // graph bodies executed since launch
    int* max_rounds;       // cap on graph bodies (guarantees the WHILE loop ends)
    int* nfits_dev;        // number of fits of the current launch
    int* sm_cnt;           // [SM_IDS + 1] CTAs per SM of the loop kernel, then the round's next
                           // dynamic work item (all zero between launches)
    int sc[8];             // the scalars the pointers above refer to
    int owner_mode;        // 1: fit f's final combine and step run in the CTA of rank f (launches of few
                           // fits: that SM keeps the step's code and state warm); 0: in the last arriver
    int queue_mode;        // 1: no lock-step rounds: a fit's tiles are claimed from its own counter
                           // and re-armed by its step (batches of many fits); 0: rounds
    unsigned* fit_bits;    // queue mode: bit f set while fit f has unclaimed tiles ([ceil(fits / 32)])
    int* next_tile;        // queue mode: per fit, the next tile to claim in its current evaluation
    unsigned long long wait_ns;   // limit of the grid-wide waits (round barrier, owner wait, queue idle wait)
};

}  // namespace gbfit

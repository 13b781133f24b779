// On-device trust-region step for one fit, run by one warp (lanes 0..31).
//
// Everything here is FP64.  On GB300 an FP64 warp instruction occupies its
// SM sub-partition for ~64 cycles whether 1 or 32 lanes are active, so every
// n-vector or n x n operation is spread over the lanes of the warp:
//   vectors   lane i < n holds element i (lanes >= n hold 0);
//   matrices  n <= 8, row-major 8 x 8 in shared memory, 32 lanes x 2 elements.
// Steps, with the passage each follows:
//   combine   fixed-order FP64 sums of tile partials        Eqs. msqe, gradient, hessian
//   scaling   D, Coleman-Li v, dv, C                        Eq. hat (R7, R9)
//   factor    cyclic Jacobi eigen of B_hat = D B D + C     Appendix B (B_hat = V S^2 V^T)
//   step      p_t = -B_hat^+ g_hat, else Algorithm 2        Algorithm 1, Eqs. phi, alphaupdate (R1-R4, R10)
//   bounds    truncated / reflected / gradient candidates    R9
//   ratio     gamma = actual / predicted                    Eq. accuracy
//   update    Algorithm 3 and termination                   R5, R8
//   pcov      V S^-2 V^T of the unscaled Gram                R13
// The R-numbered readings are the interpretations of the paper's silent or
// garbled passages that both this code and the oracle implement:
//   R1 Alg. 2 loops while |phi| > 0.1 Delta, at most 10 passes; R2 the step
//   carries Eq. lm's minus sign; R3 u0 = ||g||/Delta, l0 = -phi(0)/phi'(0) at
//   full rank else 0, alpha0 = previous alpha safeguarded to
//   max(0.001u, sqrt(lu)); R4 trial alpha, then l/u update from alpha_q, then
//   the trial kept only inside the updated bracket; R5 Alg. 3 as printed,
//   non-finite trial cost or non-positive prediction rejects; R6 Delta0 =
//   ||D x0|| (1 if 0); R7 D = 1/x_scale or running Jacobian column norms;
//   R8 gtol on ||v g||_inf before a trial, ftol on accepted steps, xtol on
//   every trial, max_nfev = 100 n; R9 Coleman-Li reflective bounds; R10
//   lambda <= 8 n eps lambda_max counts as zero; R13 pcov scaled by
//   2f/(m-n) unless absolute_sigma.
#pragma once
#include "gbfit_internal.cuh"
#include "models.cuh"

namespace gbfit {

constexpr unsigned FULL = 0xffffffffu;
constexpr double EPS64 = 2.220446049250313e-16;

enum FitStatusCode {
    FS_INVALID_DATA = -2, FS_NUMERICAL = -1, FS_MAX_NFEV = 0, FS_GTOL = 1,
    FS_FTOL = 2, FS_XTOL = 3, FS_FTOL_XTOL = 4, FS_RUNNING = 99
};

struct FitResult {
    double popt[NMAX];
    double pcov[NMAX * NMAX];
    double tot[KMAX];      // sums of the last evaluation (Gram, gradient, cost)
    double trace[32];      // per phase (see TracePhase), summed over iterations
    double cost;
    int nfev, njev, fit_status, rounds;
};

// Phases timed (clock64, SM cycles) inside the step, summed per fit.
enum TracePhase { TR_TILE = 0, TR_COMBINE, TR_LOGIC, TR_EIGEN, TR_C_FENCE, TR_STEP, TR_PREP, TR_FINISH,
                  TR_C_GROUP, TR_C_FINAL, TR_E_WARM, TR_E_J32, TR_E_NS, TR_E_RR, TR_E_SWEEPS, TR_E_REFINES,
                  TR_GN, TR_N_GN, TR_N_EIG, TR_N_ALG2IT, TR_N_BOUNDED, TR_PRE_TILE, TR_TILE_LOOP, TR_RING_WAIT,
                  TR_ROUND_NS, TR_OWNER_WAIT_NS, TR_BARRIER_NS, TR_START_NS, TR_N_EVAL64, TR_N_ESC, TR_N_FIN,
                  TR_N_WIDE };

// Shared-memory workspace of the warp that runs one fit's step.
struct TrfSmem {
    FitState stc;     // copy of the fit's state up to its trace (read-only view for the step)
    double tot[KMAX];
    double B[64];     // Gram at x, full symmetric 8x8
    double A[64];     // Jacobi work matrix
    double Ah[64];    // scaled model matrix D B D + diag(C)
    double V[64];
    double W[64];     // scratch matrix
    double V0[64];    // scratch matrix (starting basis)
    double H[64];     // partial products of mm8
    double vec[16][8];
    double sd[12];
    double pds[PD];
    float Af[64];     // FP32 Jacobi work matrix
    float Af2[64];
    float Rf[64];     // FP32 accumulated rotations
    float Rf2[64];
    float Lf[64];     // FP32 inverse of the equilibrated matrix (fast path)
    float csf[8];
    float pfs[PF];
    MixedParams mp;
    int si[12];
    int pairs[8];
};
// named rows of TrfSmem::vec
enum { VX = 0, VXT, VG, VLB, VUB, VSX, VV, VDV, VD, VGH, VC, VLAM, VGV, VSTR, VSH, VTMP };

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// 1/x to about one ulp by Newton-Raphson iteration for the reciprocal
// (y <- y + y (1 - x y), each step squaring the relative error) from the
// correctly rounded FP32 reciprocal (relative error <= 2^-24): two steps reach
// FP64 rounding (2^-96 before the final rounding).  An FP64 division costs
// ~10 FP64 instructions on GB300, this ~6.  Outside FP32's comfortable range
// (|x| <= 1e-36 or >= 1e36, non-finite) it falls back to the division.
// Checked against 1.0 / x by gbfit_check_rcp64 (within 1 ulp).
__device__ __forceinline__ double rcp64(double x) {
    float xf = float(x);
    float ax = fabsf(xf);
    if (!(ax > 1e-36f && ax < 1e36f)) return 1.0 / x;
    double y = double(__frcp_rn(xf));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// sum over lanes 0..7 (lanes 8..31 form their own groups); result in every lane of the group
__device__ __forceinline__ double gsum8(double v) {
    v += __shfl_xor_sync(FULL, v, 4);
    v += __shfl_xor_sync(FULL, v, 2);
    v += __shfl_xor_sync(FULL, v, 1);
    return __shfl_sync(FULL, v, 0);
}
__device__ __forceinline__ double gmax8(double v) {
    v = fmax(v, __shfl_xor_sync(FULL, v, 4));
    v = fmax(v, __shfl_xor_sync(FULL, v, 2));
    v = fmax(v, __shfl_xor_sync(FULL, v, 1));
    return __shfl_sync(FULL, v, 0);
}
__device__ __forceinline__ double gmin8(double v) {
    v = fmin(v, __shfl_xor_sync(FULL, v, 4));
    v = fmin(v, __shfl_xor_sync(FULL, v, 2));
    v = fmin(v, __shfl_xor_sync(FULL, v, 1));
    return __shfl_sync(FULL, v, 0);
}
// element i of an smem vector as a lane value (0 beyond n)
__device__ __forceinline__ double ld(const double* v, int n) { int l = lane_id(); return l < n ? v[l & 7] : 0.0; }
__device__ __forceinline__ void vstore(double* v, int n, double x) { int l = lane_id(); if (l < n) v[l] = x; __syncwarp(); }
__device__ __forceinline__ double dot8(const double* a, const double* b, int n) {
    int l = lane_id();
    return gsum8(l < n ? a[l & 7] * b[l & 7] : 0.0);
}

// y = M s for 8x8 row-major M in smem; 32 lanes: lane -> (row l>>2, cols (l&3), (l&3)+4).
// Returns y_i in lane i (< n), 0 elsewhere.
__device__ __forceinline__ double matvec8(const double* M, const double* s, int n) {
    int l = lane_id();
    int i = l >> 2, j = l & 3;
    double acc = 0.0;
    if (i < n) {
        if (j < n) acc = M[i * 8 + j] * s[j];
        if (j + 4 < n) acc = fma(M[i * 8 + j + 4], s[j + 4], acc);
    }
    acc += __shfl_xor_sync(FULL, acc, 1);
    acc += __shfl_xor_sync(FULL, acc, 2);
    double r = __shfl_sync(FULL, acc, (l & 7) << 2);
    return l < n ? r : 0.0;
}

// Cyclic Jacobi eigen-decomposition of the symmetric n x n matrix A (smem,
// 8x8 row-major), accumulating rotations into V (columns = eigenvectors).
// Parallel round-robin ordering: every round rotates floor(n'/2) disjoint
// pairs at once.  Stops when a sweep rotates nothing (|a_pq| <= eps
// sqrt(a_pp a_qq)) or after max_sweeps.  Returns the sweeps used.
__device__ inline int jacobi_eig(int n, double* A, double* V, double* cs, int* pairs, int max_sweeps) {
    int l = lane_id();
    int np = n + (n & 1);
    int npairs = np / 2;
    int sweeps = 0;
    for (; sweeps < max_sweeps; ++sweeps) {
        int rotated = 0;
        for (int r = 0; r < np - 1; ++r) {
            if (l < npairs) {
                auto pos = [&](int i) { return i == 0 ? 0 : ((i - 1 + r) % (np - 1)) + 1; };
                int p = pos(l), q = pos(np - 1 - l);
                if (p > q) { int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0;
                int act = 0;
                if (q < n) {
                    double app = A[p * 8 + p], aqq = A[q * 8 + q], apq = A[p * 8 + q];
                    if (apq != 0.0 && apq * apq > EPS64 * EPS64 * fabs(app * aqq)) {
                        double th = (aqq - app) / (2.0 * apq);
                        double t;
                        if (fabs(th) > 1e150) t = 0.5 / th;
                        else t = copysign(1.0, th) / (fabs(th) + sqrt(fma(th, th, 1.0)));
                        c = rsqrt(fma(t, t, 1.0));
                        s = t * c;
                        act = 1;
                    }
                }
                pairs[l] = act ? (p | (q << 8)) : -1;
                cs[2 * l] = c;
                cs[2 * l + 1] = s;
                rotated |= act;
            }
            rotated = __any_sync(FULL, rotated);
            __syncwarp();
            // rows: lane -> (pair k = l>>3, column j = l&7)
            {
                int k = l >> 3, j = l & 7;
                int pq = k < npairs ? pairs[k] : -1;
                if (pq >= 0 && j < n) {
                    int p = pq & 255, q = pq >> 8;
                    double c = cs[2 * k], s = cs[2 * k + 1];
                    double a = A[p * 8 + j], b = A[q * 8 + j];
                    A[p * 8 + j] = c * a - s * b;
                    A[q * 8 + j] = fma(s, a, c * b);
                }
            }
            __syncwarp();
            // columns of A and V: lane -> (pair k = l>>3, row i = l&7)
            {
                int k = l >> 3, i = l & 7;
                int pq = k < npairs ? pairs[k] : -1;
                if (pq >= 0 && i < n) {
                    int p = pq & 255, q = pq >> 8;
                    double c = cs[2 * k], s = cs[2 * k + 1];
                    double a = A[i * 8 + p], b = A[i * 8 + q];
                    A[i * 8 + p] = c * a - s * b;
                    A[i * 8 + q] = fma(s, a, c * b);
                    double va = V[i * 8 + p], vb = V[i * 8 + q];
                    V[i * 8 + p] = c * va - s * vb;
                    V[i * 8 + q] = fma(s, va, c * vb);
                }
            }
            __syncwarp();
            if (l < npairs && pairs[l] >= 0) {
                int p = pairs[l] & 255, q = pairs[l] >> 8;
                A[p * 8 + q] = 0.0;
                A[q * 8 + p] = 0.0;
            }
            __syncwarp();
        }
        if (!rotated) break;
    }
    return sweeps;
}

// S = V0^T M V0 into A (all 8x8 smem); 32 lanes x 2 outputs, n-term sums.
__device__ inline void congruence(int n, const double* M, const double* V0, double* W, double* A) {
    int l = lane_id();
    for (int e = l; e < 64; e += 32) {          // W = M V0
        int i = e >> 3, j = e & 7;
        double acc = 0.0;
        if (i < n && j < n)
            for (int k = 0; k < n; ++k) acc = fma(M[i * 8 + k], V0[k * 8 + j], acc);
        W[e] = acc;
    }
    __syncwarp();
    for (int e = l; e < 64; e += 32) {          // A = V0^T W
        int i = e >> 3, j = e & 7;
        double acc = 0.0;
        if (i < n && j < n)
            for (int k = 0; k < n; ++k) acc = fma(V0[k * 8 + i], W[k * 8 + j], acc);
        A[e] = acc;
    }
    __syncwarp();
    for (int e = l; e < 64; e += 32) {          // exact symmetry
        int i = e >> 3, j = e & 7;
        if (i < j) { double s = 0.5 * (A[i * 8 + j] + A[j * 8 + i]); A[i * 8 + j] = s; A[j * 8 + i] = s; }
    }
    __syncwarp();
}

// phi(alpha) and phi'(alpha) (Eq. phi) from eigenvalues lam and gV = V^T g_hat (lane values).
__device__ __forceinline__ void phi_dphi(double lam, double gv, double alpha, double Delta, double& phi, double& dphi) {
    double qa = 0.0, qb = 0.0;
    if (gv != 0.0) {
        double r = rcp64(lam + alpha);
        qa = gv * r;
        qb = qa * qa * r;
    }
    double pn = sqrt(gsum8(qa * qa));
    phi = pn - Delta;
    dphi = -gsum8(qb) * rcp64(pn);
}

// Algorithm 2 (readings R1, R3, R4). lam, gv: lane values.
__device__ inline double lm_parameter(double lam, double gv, double gh_norm, double Delta, double alpha0,
                               bool full_rank, int* iters) {
    double u = gh_norm * rcp64(Delta);
    double lo = 0.0;
    if (full_rank) {
        double phi0, dphi0;
        phi_dphi(lam, gv, 0.0, Delta, phi0, dphi0);
        lo = -phi0 * rcp64(dphi0);
    }
    double alpha = alpha0;
    if (!(lo <= alpha && alpha <= u)) alpha = fmax(0.001 * u, sqrt(lo * u));
    int it = 0;
    for (; it < 10; ++it) {
        double phi, dphi;
        phi_dphi(lam, gv, alpha, Delta, phi, dphi);
        if (fabs(phi) <= 0.1 * Delta) break;
        double ratio = phi * rcp64(dphi);
        double at = alpha - ((phi + Delta) * rcp64(Delta)) * ratio;
        lo = fmax(lo, alpha - ratio);
        if (phi < 0.0) u = alpha;
        alpha = (lo <= at && at <= u) ? at : fmax(0.001 * u, sqrt(lo * u));
    }
    *iters = it;
    return alpha;
}

// q(s) = g_hat.s + s^T Ah s / 2 for an smem vector s.
__device__ __forceinline__ double quad_value(const double* Ah, const double* gh, const double* s, int n) {
    double As = matvec8(Ah, s, n);
    int l = lane_id();
    double sl = l < n ? s[l] : 0.0;
    double gl = l < n ? gh[l] : 0.0;
    return gsum8(gl * sl + 0.5 * sl * As);
}

// Largest t >= 0 with lb <= x + t s <= ub (lane values); hits = lanes that bind.
__device__ __forceinline__ double step_to_bound(double x, double s, double lb, double ub, bool& hit) {
    double t = INFINITY;
    if (s > 0.0) t = (ub - x) * rcp64(s);
    else if (s < 0.0) t = (lb - x) * rcp64(s);
    double tmin = gmin8(lane_id() < 8 ? t : INFINITY);
    hit = (t == tmin) && isfinite(t);
    return fmax(tmin, 0.0);
}

// Positive root of ||s0 + t r|| = Delta (lane values).
__device__ __forceinline__ double tr_intersect(double s0, double r, double Delta) {
    double a = gsum8(r * r), b = 2.0 * gsum8(s0 * r), c = gsum8(s0 * s0) - Delta * Delta;
    double disc = sqrt(fmax(b * b - 4.0 * a * c, 0.0));
    return b <= 0.0 ? (-b + disc) * rcp64(2.0 * a) : (2.0 * c) * rcp64(-b - disc);
}

// min over [t_lo, t_hi] of t -> q(s0 + t r); s0, r smem vectors, tmp scratch vector.
__device__ inline double minimize_on_segment(const double* Ah, const double* gh, const double* s0, const double* r,
                                      double* tmp, int n, double t_lo, double t_hi, double& best_t) {
    int l = lane_id();
    double Ar = matvec8(Ah, r, n);
    double As0 = matvec8(Ah, s0, n);
    double rl = l < n ? r[l] : 0.0, s0l = l < n ? s0[l] : 0.0, gl = l < n ? gh[l] : 0.0;
    double curv = gsum8(rl * Ar);
    double slope = gsum8(gl * rl + s0l * Ar);
    double q0 = gsum8(gl * s0l + 0.5 * s0l * As0);
    double cand[3] = {t_lo, t_hi, t_lo};
    int nc = 2;
    if (curv > 0.0) {
        double ts = -slope * rcp64(curv);
        if (t_lo < ts && ts < t_hi) { cand[2] = ts; nc = 3; }
    }
    // q(s0 + t r) = q0 + t slope + t^2 curv / 2 (exact for the quadratic model)
    double bv = INFINITY;
    best_t = t_lo;
    for (int c = 0; c < nc; ++c) {
        double t = cand[c];
        double v = q0 + t * slope + 0.5 * t * t * curv;
        if (v < bv) { bv = v; best_t = t; }
    }
    (void)tmp;
    return bv;
}

}  // namespace gbfit

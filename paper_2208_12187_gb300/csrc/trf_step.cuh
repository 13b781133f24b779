// The trust-region step of one fit, run by the CTA that completed the fit's
// evaluation (all EVAL_THREADS threads call it; warp 0 carries the scalar and
// n-vector logic, warps 0-3 share the FP64 8x8 matrix products).
//
// GB300 FP64 issues at ~1/64 of FP32 and one FP64 warp instruction occupies
// its SM sub-partition for ~64 cycles whatever the active lanes, so:
//   * n x n products are spread over 4 warps (one per sub-partition);
//   * the eigen-decomposition runs its many sequential Jacobi rotations in
//     FP32, then an FP64 refinement made of matrix products only restores
//     FP64 accuracy (Newton-Schulz re-orthonormalisation, Rayleigh-Ritz
//     V^T A V, and a first/second-order perturbation update); every
//     quantity the algorithm decides on is FP64;
//   * divisions use an FP32 reciprocal refined by two FP64 Newton steps;
//   * norms needed by the next iteration are formed once, at step time.
#pragma once
#include "gbfit_internal.cuh"
#include "models.cuh"
#include "trf_device.cuh"

namespace gbfit {

// Trace counters are bumped with reductions that return nothing (RED), so
// that the step never waits on an L2 round trip for its own bookkeeping.
__device__ __forceinline__ void trace_bump(unsigned long long* trace, int phase, unsigned long long v) {
    atomicAdd(trace + phase, v);
}

__device__ __forceinline__ void trace_add(FitState* st, int phase, long long& t) {
    long long now = clock64();
    if (threadIdx.x == 0) trace_bump(st->trace, phase, (unsigned long long)(now - t));
    t = now;
}

__device__ __forceinline__ void trace_add_arr(unsigned long long* trace, int phase, long long& t) {
    long long now = clock64();
    if (threadIdx.x == 0) trace_bump(trace, phase, (unsigned long long)(now - t));
    t = now;
}

// C = op(A) B on n x n blocks of 8x8 row-major smem matrices (C must not
// alias A or B).  Warps 0-3 (one per SM sub-partition) each take half of
// the k range of 32 outputs; the halves meet through shared memory.  Every
// thread of the CTA must call (two __syncthreads).
__device__ __forceinline__ void mm8(int n, const double* A, bool tA, const double* B, double* C,
                                    double* half) {
    int t = threadIdx.x;
    if (t < 128) {
        int e = t & 63, h = t >> 6;
        int i = e >> 3, j = e & 7;
        double acc = 0.0;
        int k0 = h * 4, k1 = min(n, k0 + 4);
        if (i < n && j < n)
            for (int k = k0; k < k1; ++k) acc = fma(tA ? A[k * 8 + i] : A[i * 8 + k], B[k * 8 + j], acc);
        if (h) half[e] = acc;
        __syncthreads();
        if (!h) C[e] = acc + half[e];
    } else {
        __syncthreads();
    }
    __syncthreads();
}

// Partner of each index in round r of the parallel round-robin ordering on
// np = 2, 4, 6, 8 indices (an index paired with itself rests that round);
// 3 bits per index so that every lane reads the same word.
static __constant__ unsigned c_partner_packed[4][7] = {
    {0xfac681u, 0xfac688u, 0xfac688u, 0xfac688u, 0xfac688u, 0xfac688u, 0xfac688u},
    {0xfac053u, 0xfac4c1u, 0xfac21au, 0xfac688u, 0xfac688u, 0xfac688u, 0xfac688u},
    {0xf814e5u, 0xf93941u, 0xfa521au, 0xf8a12bu, 0xf98a54u, 0xfac688u, 0xfac688u},
    {0x053977u, 0x4e5dc1u, 0x97721au, 0xdca12bu, 0x298bbcu, 0x706e55u, 0xa394e6u},
};

// FP32 cyclic Jacobi, one fused pass per round (warp 0 only).  The lane
// numbered like the smaller index of each pair forms that pair's rotation
// (branch-free); every lane then takes the rotations its elements need by
// shuffle and updates two elements of A' = J^T A J and of R' = R J into the
// second buffer (one __syncwarp per round).  Relative stopping test
// |a_pq| <= 2.5e-7 sqrt(a_pp a_qq).  A, A2, R, R2: float 8x8 smem; on return
// *Ares / *Rres point at the results.
__device__ inline int jacobi32(int n, float* A, float* A2, float* R, float* R2, int max_sweeps,
                        float** Ares, float** Rres) {
    const int l = threadIdx.x & 31;
    const int np = n + (n & 1);
    const float tol2 = 2.5e-7f * 2.5e-7f;
    const int i0 = l >> 3, i1 = i0 + 4, j = l & 7;
    int sweeps = 0;
    for (; sweeps < max_sweeps; ++sweeps) {
        bool any = false;
        for (int r = 0; r < np - 1; ++r) {
            const unsigned word = c_partner_packed[np / 2 - 1][r];
            // owner lane l (< 8) rotates the pair (l, partner) when l < partner < n
            float c = 1.0f, s = 0.0f;
            {
                int x = l & 7, y = (word >> (3 * x)) & 7;
                bool own = l < 8 && x < y && y < n;
                float app = A[x * 8 + x], aqq = A[y * 8 + y], apq = A[x * 8 + y];
                bool act = own && (apq * apq > tol2 * fabsf(app * aqq)) && apq != 0.0f;
                float th = __fdividef(aqq - app, 2.0f * (act ? apq : 1.0f));
                float h = fmaf(th, th, 1.0f);
                float t = copysignf(__fdividef(1.0f, fabsf(th) + h * rsqrtf(h)), th);
                t = (h < 1e36f) ? t : __fdividef(0.5f, th);
                float cc = rsqrtf(fmaf(t, t, 1.0f));
                float ss = t * cc;
                float nf = fmaf(-0.5f, fmaf(cc, cc, ss * ss), 1.5f);   // c^2 + s^2 -> 1
                c = act ? cc * nf : 1.0f;
                s = act ? ss * nf : 0.0f;
                any |= act;
            }
            int pj = (word >> (3 * j)) & 7, p0 = (word >> (3 * i0)) & 7, p1 = (word >> (3 * i1)) & 7;
            // rotation of index x: owner lane min(x, partner); coefficient on the partner is -s for the smaller index
            float cj = __shfl_sync(FULL, c, min(j, pj)), sj = __shfl_sync(FULL, s, min(j, pj));
            float c0 = __shfl_sync(FULL, c, min(i0, p0)), s0 = __shfl_sync(FULL, s, min(i0, p0));
            float c1 = __shfl_sync(FULL, c, min(i1, p1)), s1 = __shfl_sync(FULL, s, min(i1, p1));
            bool aj = sj != 0.0f;
            sj = (j < pj) ? -sj : sj;
            s0 = (i0 < p0) ? -s0 : s0;
            s1 = (i1 < p1) ? -s1 : s1;
            float x0 = c0 * (cj * A[i0 * 8 + j] + sj * A[i0 * 8 + pj]) + s0 * (cj * A[p0 * 8 + j] + sj * A[p0 * 8 + pj]);
            float x1 = c1 * (cj * A[i1 * 8 + j] + sj * A[i1 * 8 + pj]) + s1 * (cj * A[p1 * 8 + j] + sj * A[p1 * 8 + pj]);
            if (aj && p0 == j) x0 = 0.0f;      // the rotated pair's off-diagonal
            if (aj && p1 == j) x1 = 0.0f;
            A2[i0 * 8 + j] = x0;
            A2[i1 * 8 + j] = x1;
            R2[i0 * 8 + j] = cj * R[i0 * 8 + j] + sj * R[i0 * 8 + pj];
            R2[i1 * 8 + j] = cj * R[i1 * 8 + j] + sj * R[i1 * 8 + pj];
            __syncwarp();
            float* tA = A; A = A2; A2 = tA;
            float* tR = R; R = R2; R2 = tR;
        }
        if (!__any_sync(FULL, any)) break;
    }
    *Ares = A;
    *Rres = R;
    return sweeps;
}

// ---- Gauss-Newton fast path: FP32 inverse, FP64 iterative refinement.
// M = sc * Ah (sc = 1 / max diagonal).  Mi <- M^-1 in FP32 by Gauss-Jordan
// elimination without pivoting, in place (float 8x8 smem; rows and columns
// >= n stay those of the identity).  The pivots are those of M's LDL^T
// factorisation, so M is positive definite exactly when all are positive;
// returns false otherwise.  min_diag: smallest diagonal entry of M.  One
// warp; each lane owns two entries, n rank-one steps.
__device__ inline bool inv32(int n, const double* Ah, float* Mi, float& sc, float& min_diag) {
    const int l = threadIdx.x & 31;
    double dmax = gmax8((l < n) ? Ah[l * 8 + l] : 0.0);
    if (!(dmax > 0.0)) return false;
    sc = float(rcp64(dmax));
    // the 8x8 matrix in registers: lane l holds rows i0 = l/8 and i1 = 4 + l/8
    // of column j = l%8; the pivot row and column come in by shuffles
    const int j = l & 7, i0 = l >> 3, i1 = i0 + 4;
    float a0 = (i0 < n && j < n) ? float(Ah[l]) * sc : (i0 == j ? 1.0f : 0.0f);
    float a1 = (i1 < n && j < n) ? float(Ah[l + 32]) * sc : (i1 == j ? 1.0f : 0.0f);
    float dg = fminf((i0 == j && j < n) ? a0 : INFINITY, (i1 == j && j < n) ? a1 : INFINITY);
    for (int o = 16; o; o >>= 1) dg = fminf(dg, __shfl_xor_sync(FULL, dg, o));
    min_diag = fminf(1.0f, dg);
    bool ok = true;
    for (int k = 0; k < n; ++k) {
        const float rowk = (k < 4) ? a0 : a1;                 // the register that holds row k
        const int kb = (k & 3) << 3;
        const float piv = __shfl_sync(FULL, rowk, kb + k);
        const float akj = __shfl_sync(FULL, rowk, kb + j);
        const float ai0 = __shfl_sync(FULL, a0, (l & ~7) + k);
        const float ai1 = __shfl_sync(FULL, a1, (l & ~7) + k);
        ok = ok && piv > 0.0f;
        const float r = __frcp_rn(piv > 0.0f ? piv : 1.0f);
        a0 = (i0 == k) ? ((j == k) ? r : akj * r) : ((j == k) ? -ai0 * r : fmaf(-ai0 * r, akj, a0));
        a1 = (i1 == k) ? ((j == k) ? r : akj * r) : ((j == k) ? -ai1 * r : fmaf(-ai1 * r, akj, a1));
    }
    Mi[l] = a0;
    Mi[l + 32] = a1;
    __syncwarp();
    return ok;
}

// y = Mi v in FP32 (lane values; lane j holds v_j, lane i receives y_i).
__device__ __forceinline__ float apply32(int n, const float* Mi, float v) {
    const int l = threadIdx.x & 31;
    const int i = l >> 2, j = l & 3;
    float v0 = __shfl_sync(FULL, v, j), v1 = __shfl_sync(FULL, v, j + 4);
    float acc = fmaf(Mi[i * 8 + j], v0, Mi[i * 8 + j + 4] * v1);
    acc += __shfl_xor_sync(FULL, acc, 1);
    acc += __shfl_xor_sync(FULL, acc, 2);
    float r = __shfl_sync(FULL, acc, (l & 7) << 2);
    return l < n ? r : 0.0f;
}

// Ah p = rhs to FP64 accuracy: FP32 solve with M^-1 (M = sc Ah, so
// p = M^-1 (sc rhs)), then two rounds of FP64 residual + FP32 correction.
// d1, d2: norms of the two corrections (FP32); their ratio estimates
// eps32 * cond of the equilibrated matrix.  tmp: an 8-double smem vector
// of the calling warp.
__device__ inline double solve_refined(int n, const double* Ah, const float* Mi, float sc, double rhs, double* tmp,
                                float& d1, float& d2) {
    const int l = threadIdx.x & 31;
    double p = double(apply32(n, Mi, float(rhs) * sc));
    float dn[2];
    for (int it = 0; it < 2; ++it) {
        if (l < 8) tmp[l] = (l < n) ? p : 0.0;
        __syncwarp();
        double r = rhs - matvec8(Ah, tmp, n);
        float dz = apply32(n, Mi, float(r) * sc);
        p += double(dz);
        float q = dz * dz;
        for (int o = 4; o; o >>= 1) q += __shfl_xor_sync(FULL, q, o);
        dn[it] = sqrtf(__shfl_sync(FULL, q, 0));
    }
    d1 = dn[0];
    d2 = dn[1];
    return (l < n) ? p : 0.0;
}

// The refined solve is trusted (as an FP64-accurate solve with a
// non-singular matrix) when the refinement contracts (ratio ~ eps32 cond of
// the equilibrated matrix) and min_diag / cond stays far above the rank
// cutoff 8 n eps64 of the pseudo-inverse (lambda_max <= n after
// equilibration), so that the pseudo-inverse would drop nothing.
__device__ __forceinline__ bool refined_ok(float d1, float d2, float min_diag) {
    float cond = fmaxf(1.0f, __fdividef(d2, fmaxf(d1, 1e-37f) * 6e-8f));
    return (d2 <= 1e-3f * d1 || d2 == 0.0f) && __fdividef(min_diag, cond) > 1e-11f;
}

// FP64-accurate eigen-decomposition Ah = V diag(lam) V^T (Appendix B: Ah =
// B_hat, lam = Sigma^2).  Vwarm (global, may be null): a previous basis to
// start from.  All CTA threads call; results in S.V and S.vec[VLAM].
// Returns the FP32 Jacobi sweeps.
__device__ inline int eig_fast(int n, const double* Ah, const double* Vwarm, TrfSmem& S,
                        unsigned long long* trace = nullptr) {
    const int t = threadIdx.x, warp = t >> 5, l = t & 31;
    const bool warm = Vwarm != nullptr;
    long long tc = clock64();
    // 1. starting matrix in the warm basis
    if (t < 64) {
        int i = t >> 3, j = t & 7;
        S.V0[t] = warm ? Vwarm[t] : ((i == j && i < n) ? 1.0 : 0.0);
    }
    __syncthreads();
    if (warm) {
        mm8(n, Ah, false, S.V0, S.W, S.H);          // W = Ah V0
        mm8(n, S.V0, true, S.W, S.A, S.H);          // A = V0^T Ah V0
    } else {
        if (t < 64) S.A[t] = Ah[t];
        __syncthreads();
    }
    if (trace) trace_add_arr(trace, TR_E_WARM, tc);
    // 2. FP32 Jacobi on A / max diag
    int sweeps = 0;
    if (warp == 0) {
        double dg = (l < n) ? fabs(S.A[l * 8 + l]) : 0.0;
        double dmax = gmax8(dg);
        float sc = dmax > 0.0 ? float(rcp64(dmax)) : 1.0f;
        for (int e = l; e < 64; e += 32) {
            int i = e >> 3, j = e & 7;
            bool in = i < n && j < n;
            S.Af[e] = in ? float(S.A[e]) * sc : 0.0f;
            S.Rf[e] = (i == j) ? 1.0f : 0.0f;
        }
        __syncwarp();
        float *Ares, *Rres;
        sweeps = jacobi32(n, S.Af, S.Af2, S.Rf, S.Rf2, 20, &Ares, &Rres);
        if (Rres != S.Rf)
            for (int e = l; e < 64; e += 32) S.Rf[e] = Rres[e];
        if (trace && t == 0) trace_bump(trace, TR_E_SWEEPS, sweeps);
    }
    __syncthreads();
    if (trace) trace_add_arr(trace, TR_E_J32, tc);
    // 3. V = V0 R (or R)
    if (t < 64) S.W[t] = double(S.Rf[t]);
    __syncthreads();
    if (warm) mm8(n, S.V0, false, S.W, S.V, S.H);
    else { if (t < 64) S.V[t] = S.W[t]; __syncthreads(); }
    // 4. Newton-Schulz: V <- V (3 I - V^T V) / 2
    mm8(n, S.V, true, S.V, S.A, S.H);               // G = V^T V
    if (t < 64) { int i = t >> 3, j = t & 7; S.W[t] = (i == j ? 1.5 : 0.0) - 0.5 * S.A[t]; }
    __syncthreads();
    mm8(n, S.V, false, S.W, S.V0, S.H);             // V0 <- V T
    if (trace) trace_add_arr(trace, TR_E_NS, tc);
    // 5-6. Rayleigh-Ritz A1 = V^T Ah V and perturbation update
    //    X_rc = A1_rc / (A1_cc - A1_rr), V <- V (I + X),
    //    lam_c = A1_cc + sum_r A1_rc^2 / (A1_cc - A1_rr);
    //    repeated once more when the first correction was not already tiny.
    for (int pass = 0; pass < 2; ++pass) {
        mm8(n, Ah, false, S.V0, S.W, S.H);
        mm8(n, S.V0, true, S.W, S.A, S.H);
        if (t < 64) {
            int r = t >> 3, c = t & 7;
            double x = 0.0;
            if (r < n && c < n && r != c) {
                double a = S.A[t];
                double gap = S.A[c * 8 + c] - S.A[r * 8 + r];
                float gf = float(gap), af = float(a);
                if (fabsf(gf) > 1e3f * fabsf(af) && fabsf(gf) > 1e-30f) x = double(af * __frcp_rn(gf));
            }
            S.W[t] = x;
        }
        __syncthreads();
        if (warp == 0) {
            double lam = 0.0;
            if (l < n) {
                lam = S.A[l * 8 + l];
                for (int r = 0; r < n; ++r)
                    if (r != l) lam = fma(S.A[r * 8 + l], S.W[r * 8 + l], lam);
            }
            if (l < 8) S.vec[VLAM][l] = lam;
            // largest correction decides whether a second pass is needed
            float xm = 0.0f;
            for (int e = l; e < 64; e += 32) xm = fmaxf(xm, fabsf(float(S.W[e])));
            for (int o = 16; o; o >>= 1) xm = fmaxf(xm, __shfl_xor_sync(FULL, xm, o));
            if (l == 0) S.si[7] = (xm > 1e-9f) ? 1 : 0;
        }
        __syncthreads();
        mm8(n, S.V0, false, S.W, S.A, S.H);             // A = V X
        if (t < 64) S.V0[t] += S.A[t];
        __syncthreads();
        if (trace && t == 0) trace_bump(trace, TR_E_REFINES, 1);
        if (!S.si[7]) break;
    }
    if (t < 64) S.V[t] = S.V0[t];
    __syncthreads();
    if (trace) trace_add_arr(trace, TR_E_RR, tc);
    return sweeps;
}

// Coleman-Li scaling at the current x, g (lane values; lanes >= n: v = dv = 0).
// st: the fit's state (the step passes its shared-memory copy).
__device__ __forceinline__ void cl_scaling_xg(const FitDesc& d, const FitState* st, int n, double x, double g,
                                              double& v, double& dv, double& sx) {
    int l = threadIdx.x & 31;
    v = 0.0; dv = 0.0; sx = 1.0;
    if (l < n) {
        double lb = d.lb[l], ub = d.ub[l];
        v = 1.0;
        if (d.bounded) {
            if (g < 0.0 && ub < INFINITY) { v = ub - x; dv = -1.0; }
            else if (g > 0.0 && lb > -INFINITY) { v = x - lb; dv = 1.0; }
        }
        sx = d.jac_scale ? rcp64(st->scale_inv[l]) : d.xscale[l];
    }
}
__device__ __forceinline__ void cl_scaling(const FitDesc& d, const FitState* st, const TrfSmem& S, int n,
                                           double& v, double& dv, double& sx) {
    int l = threadIdx.x & 31;
    double x = (l < n) ? S.vec[VX][l] : 0.0, g = (l < n) ? S.vec[VG][l] : 0.0;
    cl_scaling_xg(d, st, n, x, g, v, dv, sx);
}

// Pass constants for evaluating xt relative to x (warp 0).
// e64: the fit evaluates in FP64 although the kernel is the mixed one (guard).
template <int PREC, class MS>
__device__ void prep_pass(const FitDesc& d, FitState* st, TrfSmem& S, bool e64 = false) {
    int l = threadIdx.x & 31;
    int n = d.n;
    if (PREC == PREC_MIXED && !e64) {
        if (l < n) {
            double x = S.vec[VX][l], xt = S.vec[VXT][l];
            float xf = float(x);
            S.mp.x[l] = xf;
            S.mp.xlo[l] = float(x - double(xf));
            S.mp.xt[l] = float(xt);
            S.mp.dx[l] = float(xt - x);
        }
        __syncwarp();
        S.pfs[l] = 0.0f;
        __syncwarp();
        MS::dispatch(d.model, [&](auto m) { prep_mixed_model<decltype(m)>(S.mp, S.pfs, S.Af); });
        if (l == 0) {
            const float C = float(d.f_scale);
            S.pfs[PF_C2] = C * C;
            S.pfs[PF_IC2] = 1.0f / (C * C);
        }
        __syncwarp();
        st->pf[l] = S.pfs[l];
    } else {
        if (l == 0) {
            for (int k = 0; k < PD; ++k) S.pds[k] = 0.0;
            MS::dispatch(d.model, [&](auto m) { decltype(m)::prep_plain(S.vec[VXT], S.pds); });
        }
        if (l == 0) {
            S.pds[PD_C2] = d.f_scale * d.f_scale;
            S.pds[PD_IC2] = 1.0 / (d.f_scale * d.f_scale);
        }
        __syncwarp();
        if (l < PD) st->pd[l] = S.pds[l];
    }
    __syncwarp();
}

// Scalar slots of TrfSmem::sd / si shared between the phases.
enum { SD_F = 0, SD_DELTA, SD_ALPHA, SD_GNORM, SD_SC, SD_MIND, SD_PT2, SD_COND, SD_FLOOR, SD_SEREL };
enum { SI_STATUS = 0, SI_NFEV, SI_NJEV, SI_FACTOR, SI_GN, SI_REJECTED, SI_PCOV, SI_SPEC, SI_ESC };

// ---- precision guard of the mixed path.  FP32 evaluation has two limits:
// the Gram is formed from FP32 products and sums, so its error relative to
// the equilibrated matrix is ~1e-7..1e-6 and the step's error grows with the
// equilibrated condition number; and the residuals carry FP32 rounding
// (absolute ~C_H eps32 |w h| per point), which moves the fixed point of the
// iteration.  guard_estimates measures both at the point just evaluated:
//   cond  = ||M||_inf ||M^-1||_inf, M = S B S with S = diag(B)^-1/2 (M^-1 from
//           the FP32 Gauss-Jordan inverse; +inf when M is not positive
//           definite in FP32);
//   floor = max_j C_H eps32 rms(w h) sqrt((B^-1)_jj) / max(|p_j|, 1): the
//           rounding-induced shift of popt (relative, as the tolerances are
//           stated) — random per-point errors e_i move the fixed point by
//           B^-1 J^T e, whose covariance is (C_H eps32 rms(w h))^2 B^-1.
//   serel = max_j se_j / |p_j| with se_j^2 = 2f/(m-n) (B^-1)_jj: a fit whose
//           parameters are this poorly determined has a flat cost valley in
//           which an FP32 iteration stops measurably above the FP64 minimum
//           (cost excess 1e-9..1e-8 relative at serel ~0.1), so it too
//           finishes in FP64 beyond GUARD_SE_REL.
// C_H = 16 covers the exponential models' argument rounding (|q| eps32 per
// exp for exponents up to ~10), measured against FP64 fixed points.
constexpr double GUARD_C_H = 16.0;
constexpr double GUARD_SE_REL = 0.05;
// A stall by rejections (a stop on xtol alone) finishes in FP64 when the floor
// estimate exceeds this fraction of guard_floor (ten times stricter than a
// stop on ftol: the stalled point is anywhere within the noise ball, not at
// the FP32 fixed point).
constexpr double GUARD_STALL_FRAC = 0.1;
constexpr double EPS32 = 5.960464477539063e-08;

// Termination scale of a mixed fit the guard moved to FP64 passes after FP32
// iterations (a finish, or an escalation past the first evaluation): its
// tolerances are tightened 100x, since its FP64 iterations start where FP32
// rounding left it and the requested tolerances could stop it there.  A fit
// escalated at its first evaluation runs the plain FP64 iteration from p0
// with the requested tolerances.
enum { GUARD_NONE = 0, GUARD_ESC_INIT = 1, GUARD_FINISH = 2, GUARD_ESC_MID = 3 };
__device__ __forceinline__ double guard_tol_scale(const FitState* cst) {
    return (cst->eval64 && (cst->guard_why == GUARD_FINISH || cst->guard_why == GUARD_ESC_MID)) ? 1e-2 : 1.0;
}

// One warp, FP32 throughout (estimates need a digit or two; FP64 divisions
// and square roots would make this the longest warp of the step's first
// phase).  tot: packed sums of the evaluation at xt; wh2: sum (w h)^2 at p0;
// m: points.  Writes S.sd[SD_COND], S.sd[SD_FLOOR] and
// S.sd[SD_SEREL].  The matrix lives in registers as in inv32: lane l holds
// rows i0 = l/8 and i1 = 4 + l/8 of column j = l%8.
__device__ inline void guard_estimates(int n, int64_t m, const double* tot, double wh2, const double* xt,
                                       TrfSmem& S) {
    const int l = threadIdx.x & 31;
    const int NT = n_tri(n);
    // S_l = 1/sqrt(B_ll) in lane l
    float sdl = 0.0f;
    bool pos = true;
    if (l < n) {
        const float bll = float(tot[l * n - l * (l - 1) / 2]);
        pos = bll > 1e-30f && bll < 1e30f;
        sdl = pos ? rsqrtf(bll) : 0.0f;
    }
    pos = __all_sync(FULL, pos);
    const int j = l & 7, i0 = l >> 3, i1 = i0 + 4;
    const float sj = __shfl_sync(FULL, sdl, j), s0 = __shfl_sync(FULL, sdl, i0), s1 = __shfl_sync(FULL, sdl, i1);
    auto entry = [&](int i, float si) -> float {          // M = S B S, unit diagonal, identity outside n
        if (i == j) return 1.0f;
        if (i >= n || j >= n) return 0.0f;
        const int a = min(i, j), c = max(i, j);
        return float(tot[a * n - a * (a - 1) / 2 + (c - a)]) * si * sj;
    };
    float a0 = entry(i0, s0), a1 = entry(i1, s1);
    auto rowmax = [&](float v0, float v1) -> float {      // max over rows of the row sums of |.|
        float r0 = fabsf(v0), r1 = fabsf(v1);
        for (int o = 1; o < 8; o <<= 1) { r0 += __shfl_xor_sync(FULL, r0, o); r1 += __shfl_xor_sync(FULL, r1, o); }
        float r = fmaxf(r0, r1);
        for (int o = 8; o < 32; o <<= 1) r = fmaxf(r, __shfl_xor_sync(FULL, r, o));
        return r;
    };
    const float rm = rowmax(i0 < n ? a0 : 0.0f, i1 < n ? a1 : 0.0f);
    // Gauss-Jordan inverse without pivoting (pivots of the LDL^T factors: all
    // positive exactly when M is positive definite)
    bool ok = pos;
    for (int k = 0; k < n; ++k) {
        const float rowk = (k < 4) ? a0 : a1;
        const int kb = (k & 3) << 3;
        const float piv = __shfl_sync(FULL, rowk, kb + k);
        const float akj = __shfl_sync(FULL, rowk, kb + j);
        const float ai0 = __shfl_sync(FULL, a0, (l & ~7) + k);
        const float ai1 = __shfl_sync(FULL, a1, (l & ~7) + k);
        ok = ok && piv > 0.0f;
        const float r = __frcp_rn(piv > 0.0f ? piv : 1.0f);
        a0 = (i0 == k) ? ((j == k) ? r : akj * r) : ((j == k) ? -ai0 * r : fmaf(-ai0 * r, akj, a0));
        a1 = (i1 == k) ? ((j == k) ? r : akj * r) : ((j == k) ? -ai1 * r : fmaf(-ai1 * r, akj, a1));
    }
    ok = __all_sync(FULL, ok);
    const float ri = rowmax(i0 < n ? a0 : 0.0f, i1 < n ? a1 : 0.0f);
    // (M^-1)_ll to lane l: row l < 4 is a0 of lane 9 l, row l >= 4 is a1 of lane 8 (l - 4) + l
    const float d0 = __shfl_sync(FULL, a0, (l & 3) * 9), d1 = __shfl_sync(FULL, a1, (l & 3) * 8 + 4 + (l & 3));
    const float dinv = (l < 4) ? d0 : d1;
    // rounding floor and relative standard errors: (B^-1)_ll = S_l^2 (M^-1)_ll
    const float rms = sqrtf(fmaxf(float(wh2), 0.0f) / float(m));
    const float s2 = (m > n) ? float(tot[NT + n]) / float(m - n) : INFINITY;     // 2f / (m - n)
    float fl = 0.0f, se = 0.0f;
    if (l < n) {
        const float binv = (dinv > 0.0f) ? dinv * sdl * sdl : INFINITY;
        const float ax = fabsf(float(xt[l]));
        fl = float(GUARD_C_H * EPS32) * rms * sqrtf(binv) / fmaxf(ax, 1.0f);
        se = sqrtf(s2 * binv) / ax;
    }
    for (int o = 16; o; o >>= 1) {
        fl = fmaxf(fl, __shfl_xor_sync(FULL, fl, o));
        se = fmaxf(se, __shfl_xor_sync(FULL, se, o));
    }
    if (l == 0) {
        S.sd[SD_COND] = ok ? double(rm) * double(ri) : INFINITY;
        S.sd[SD_FLOOR] = ok ? double(fl) : INFINITY;
        S.sd[SD_SEREL] = ok ? double(se) : INFINITY;
    }
    __syncwarp();
}

// Phase 2 on one warp: D, D g and the Coleman-Li diagonal C, then the scaled
// model matrix Ah = D B D + diag(C), from the scaling (v, dv, sx), the
// gradient g (lane values) and the full Gram Bf.
__device__ __forceinline__ void scaled_model(const FitDesc& d, int n, double v, double dv, double sx, double g,
                                             const double* Bf, TrfSmem& S) {
    const int l = threadIdx.x & 31;
    double dl = (l < n) ? (d.bounded ? sqrt(v) : 1.0) * sx : 0.0;
    if (l < 8) {
        S.vec[VD][l] = dl;
        S.vec[VGH][l] = dl * g;
        S.vec[VC][l] = (l < n && d.bounded) ? g * dv * sx * sx : 0.0;
    }
    __syncwarp();
    for (int e = l; e < 64; e += 32) {
        int i = e >> 3, j = e & 7;
        double a = 0.0;
        if (i < n && j < n) a = fma(S.vec[VD][i] * S.vec[VD][j], Bf[e], (i == j) ? S.vec[VC][i] : 0.0);
        S.Ah[e] = a;
    }
    __syncwarp();
}

// Gauss-Newton fast path on one warp: when Ah is safely full rank, the
// FP64-accurate solution of Ah pt = -D g into VSTR and its squared norm in
// pt2 (+inf when Ah is not positive definite).  Returns whether the solve is
// trusted (refined_ok).
__device__ __forceinline__ bool gn_try(int n, TrfSmem& S, double& pt2) {
    const int l = threadIdx.x & 31;
    float sc = 1.0f, mind = 0.0f;
    bool ok = inv32(n, S.Ah, S.Lf, sc, mind);
    ok = __all_sync(FULL, ok);
    pt2 = INFINITY;
    if (ok) {
        double gh = (l < n) ? S.vec[VGH][l] : 0.0;
        float d1, d2;
        double pt = solve_refined(n, S.Ah, S.Lf, sc, -gh, S.vec[VTMP], d1, d2);
        ok = refined_ok(d1, d2, mind);
        pt2 = gsum8(pt * pt);
        if (l < 8) S.vec[VSTR][l] = pt;
    }
    return ok;
}

// Result record with pcov (R13) from an FP64-accurate eigen-decomposition of
// the unscaled Gram at the solution.  All CTA threads call.
__device__ inline void write_result(const FitDesc& d, FitState* st, FitResult* res, int status, TrfSmem& S) {
    const int n = d.n, t = threadIdx.x;
    if (t < n) res->popt[t] = st->x[t];
    for (int k = t; k < KMAX; k += EVAL_THREADS) res->tot[k] = S.tot[k];
    if (t == 0) { res->cost = st->f; res->nfev = st->nfev; res->njev = st->njev; res->fit_status = status; }
    if (d.eval_only) {                   // gbfit_evaluate wants the sums only
        __syncthreads();
        return;
    }
    bool ok = (status >= 0) && d.m > n;
    if (!ok) {
        if (t < 64) res->pcov[t] = INFINITY;
        __syncthreads();
        return;
    }
    __syncthreads();
    // Well-conditioned Gram: its inverse, one refined solve per column, one
    // column per warp (equal to the pseudo-inverse when nothing is cut).
    if (t < 32) {
        float sc = 1.0f, mind = 0.0f;
        bool ok = __all_sync(FULL, inv32(n, S.B, S.Lf, sc, mind));
        if (t == 0) { S.si[SI_PCOV] = ok ? 1 : 0; S.sd[SD_SC] = sc; S.sd[SD_MIND] = mind; }
    }
    __syncthreads();
    if (S.si[SI_PCOV]) {
        const int w = t >> 5, l = t & 31;
        if (w < n) {
            float d1, d2;
            double col = solve_refined(n, S.B, S.Lf, float(S.sd[SD_SC]), (l == w) ? 1.0 : 0.0, S.W + 8 * w, d1, d2);
            if (l < n) S.H[l * 8 + w] = col;
            if (l == 0 && !refined_ok(d1, d2, float(S.sd[SD_MIND]))) S.si[SI_PCOV] = 0;
        }
        __syncthreads();
        if (S.si[SI_PCOV]) {
            double scale = d.absolute_sigma ? 1.0 : 2.0 * st->f / double(d.m - n);
            if (t < 64) {
                int i = t >> 3, j = t & 7;
                if (i < n && j < n) res->pcov[i * n + j] = 0.5 * (S.H[i * 8 + j] + S.H[j * 8 + i]) * scale;
            }
            __syncthreads();
            return;
        }
    }
    eig_fast(n, S.B, nullptr, S);
    if (t < 32) {
        int l = t;
        double lam = (l < n) ? S.vec[VLAM][l] : 0.0;
        double lmax = gmax8(l < n ? lam : -INFINITY);
        double inv = (l < n && lmax > 0.0 && lam > lmax * (8.0 * n * EPS64)) ? rcp64(lam) : 0.0;
        if (l < 8) S.vec[VTMP][l] = inv;
    }
    __syncthreads();
    double scale = d.absolute_sigma ? 1.0 : 2.0 * st->f / double(d.m - n);
    if (t < 64) {
        int i = t >> 3, j = t & 7;
        if (i < n && j < n) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc = fma(S.V[i * 8 + k] * S.vec[VTMP][k], S.V[j * 8 + k], acc);
            res->pcov[i * n + j] = acc * scale;
        }
    }
    __syncthreads();
}

// Copy the fit's state (up to its trace counters) into S.stc with all
// threads of the CTA; L2 loads, since other CTAs wrote it in earlier rounds.
// Issued before the final combine so that the loads overlap it; the
// combine's closing barrier publishes the copy.
#ifdef __CUDACC_RTC__
constexpr int STATE_WORDS = GBFIT_STATE_WORDS;   // given by the host compiler's layout of FitState
#else
constexpr int STATE_WORDS = (int)(offsetof(FitState, trace) / sizeof(uint4));
static_assert(offsetof(FitState, trace) % sizeof(uint4) == 0, "FitState prefix must be whole 16-byte words");
#endif
__device__ __forceinline__ void prefetch_state(const FitState* st, TrfSmem& S) {
    const uint4* src = reinterpret_cast<const uint4*>(st);
    uint4* dst = reinterpret_cast<uint4*>(&S.stc);
    for (int k = threadIdx.x; k < STATE_WORDS; k += blockDim.x) dst[k] = __ldcg(src + k);
}


// One trust-region iteration for one fit.  S.tot holds the combined sums of
// the evaluation at st->xt that just finished; S.stc the state as it was
// before this step (prefetch_state).  State is read from S.stc and written
// to st (and to S.stc where a later phase of the same step reads it).
template <int PREC, class MS>
__device__ void trf_step(const FitDesc& d, FitState* st, FitResult* res, TrfSmem& S, int* running) {
    const FitState* cst = &S.stc;
    const int n = d.n;
    const int t = threadIdx.x, warp = t >> 5, l = t & 31;
    const int NT = n_tri(n);
    long long tclk = clock64();
    // the evaluation just finished ran in FP64 although this is the mixed kernel (guard)
    const bool e64 = PREC == PREC_MIXED && cst->eval64;
    const bool guard_on = PREC == PREC_MIXED && !e64 && (d.guard_cond < INFINITY || d.guard_floor < INFINITY);
    if (e64 && t == 0) trace_bump(st->trace, TR_N_EVAL64, 1);
    // data flags raised by the pass's tiles (bit 0: invalid data at the first
    // evaluation, bit 1: a bounded bulk-copy wait gave up), read from L2: the
    // prefetched state copy can predate other CTAs' flags
    const int bad = __ldcg(&st->bad_data);

    // ================= evaluation only (gbfit_evaluate): the sums at p are the result
    if (d.eval_only) {
        if (t < n) res->popt[t] = cst->x[t];
        for (int k = t; k < KMAX; k += EVAL_THREADS) res->tot[k] = S.tot[k];
        if (t == 0) {
            const int status = (bad & 1) ? FS_INVALID_DATA : (bad & 2) ? FS_NUMERICAL : FS_MAX_NFEV;
            res->cost = 0.5 * S.tot[NT + n]; res->nfev = 1; res->njev = 1; res->fit_status = status;
            st->f = res->cost; st->nfev = 1; st->njev = 1;
            st->run = RS_DONE; st->fit_status = status;
            atomicSub(running, 1);
        }
        __syncthreads();
        if (t < 32) res->trace[t] = double(__ldcg(st->trace + t));
        return;
    }

    // ================= phase 1 (warp 0): accept / reject, termination tests
    if (warp == 0) {
        if (l < n) {
            S.vec[VX][l] = cst->x[l];
            S.vec[VXT][l] = cst->xt[l];
            S.vec[VG][l] = cst->g[l];
        }
        const bool init = cst->phase == PH_INIT;
        const bool reinit = cst->phase == PH_REINIT;
        const bool mixed_pass = PREC == PREC_MIXED && !cst->eval64;
        const double f2n = S.tot[NT + n];
        int status = FS_RUNNING;
        double f = cst->f, Delta = cst->Delta, alpha = cst->alpha;
        int nfev = cst->nfev, njev = cst->njev, factor_valid = cst->factor_valid;
        bool take = false, rejected = false;
        if (init || reinit) {
            // init: the first evaluation (at p0); reinit: the current point
            // evaluated again in FP64 (precision guard), radius and alpha kept
            take = true;
            f = 0.5 * f2n;
            nfev += 1; njev += 1;                 // (both 0 before a fit's first evaluation)
            if (reinit) factor_valid = 0;
            bool fin = (l >= NT + n + 1 || isfinite(S.tot[l])) && (l + 32 >= NT + n + 1 || isfinite(S.tot[l + 32]));
            fin = __all_sync(FULL, fin);
            if (init && (bad & 1)) status = FS_INVALID_DATA;
            else if (!fin || (bad & 2)) status = FS_NUMERICAL;
        } else {
            nfev += 1;
            double f_new = 0.5 * f2n;
            // mixed FP32 pass: the cancellation-free sum, except after a wide trial (direct form)
            double actual = (mixed_pass && cst->phase != PH_WIDE) ? -0.5 * S.tot[NT + n + 1] : f - f_new;
            double pred = cst->predicted;
            double gamma = (isfinite(f_new) && isfinite(actual) && pred > 0.0) ? actual * rcp64(pred) : -INFINITY;
            bool accepted;
            double Dn;
            if (gamma > 0.75) { accepted = true; Dn = 2.0 * Delta; }
            else if (gamma >= 0.25 && gamma <= 0.75) { accepted = true; Dn = Delta; }
            else { accepted = false; Dn = 0.25 * cst->s_norm; }
            rejected = !accepted;
            // a fit the guard moved to FP64 after an FP32 stretch stops on
            // tolerances 100x tighter, so that it ends at the FP64 fixed
            // point rather than where FP32 left it (see guard_tol_scale)
            const double tsc = guard_tol_scale(cst);
            bool ftol_ok = accepted && actual < tsc * d.ftol * f;
            bool xtol_ok = cst->step_norm < tsc * cst->xtol_thr;
            if (accepted) { take = true; f = f_new; njev += 1; factor_valid = 0; }
            Delta = Dn;
            if (ftol_ok && xtol_ok) status = FS_FTOL_XTOL;
            else if (ftol_ok) status = FS_FTOL;
            else if (xtol_ok) status = FS_XTOL;
            // FP32 passes: a rejected trial whose predicted reduction is below
            // ftol f ends the fit as a stall (status xtol, as the shrinking
            // radius would after a few more rejected passes): any later
            // accepted step would reduce f by less still, and in FP32 such a
            // step follows the rounding noise of the gradient (the guard's
            // stall rule then decides on an FP64 finish)
            else if (rejected && mixed_pass && pred < d.ftol * f) status = FS_XTOL;
            if (bad & 2) status = FS_NUMERICAL;
        }
        // the Gram at the (new) current point, unpacked from its packed upper triangle
        {
            const double* srcB = take ? S.tot : cst->B;
            for (int e = l; e < 64; e += 32) {
                int i = e >> 3, j = e & 7;
                double b = 0.0;
                if (i < n && j < n) { int a = min(i, j), c = max(i, j); b = srcB[a * n - a * (a - 1) / 2 + (c - a)]; }
                S.B[e] = b;
            }
        }
        if (take) {
            if (l < n) { S.vec[VX][l] = S.vec[VXT][l]; S.vec[VG][l] = S.tot[NT + l]; }
            __syncwarp();
            if (d.jac_scale && status == FS_RUNNING && l < n) {
                double c = sqrt(S.B[l * 8 + l]);
                if (!init) c = fmax(c, cst->scale_inv[l]);
                c = (c == 0.0) ? 1.0 : c;
                S.stc.scale_inv[l] = c;
                st->scale_inv[l] = c;
            }
            __syncwarp();
        }
        double gnorm = 0.0;
        if (status == FS_RUNNING) {
            double v, dv, sx;
            cl_scaling(d, cst, S, n, v, dv, sx);
            if (l < 8) { S.vec[VV][l] = v; S.vec[VDV][l] = dv; S.vec[VSX][l] = sx; }   // for phase 2
            // the radius of R6 at the first evaluation, and again when a fit that
            // met a tolerance resumes in FP64 (its last radius was sized for FP32 steps)
            if (init || (reinit && cst->guard_why == GUARD_FINISH)) {
                double xl = (l < n) ? S.vec[VX][l] : 0.0;
                double dd = (l < n) ? (d.bounded ? sqrt(v) : 1.0) * sx : 1.0;
                double q = (l < n) ? xl * rcp64(dd) : 0.0;
                Delta = sqrt(gsum8(q * q));
                if (Delta == 0.0) Delta = 1.0;
                alpha = 0.0;
                factor_valid = 0;
            }
            double g = (l < n) ? S.vec[VG][l] : 0.0;
            gnorm = gmax8(fabs(v * g));
            if (gnorm < guard_tol_scale(cst) * d.gtol) status = FS_GTOL;
            else if (nfev >= d.max_nfev) status = FS_MAX_NFEV;
        }
        if (l == 0) {
            S.sd[SD_F] = f; S.sd[SD_DELTA] = Delta; S.sd[SD_ALPHA] = alpha; S.sd[SD_GNORM] = gnorm;
            S.si[SI_STATUS] = status; S.si[SI_NFEV] = nfev; S.si[SI_NJEV] = njev; S.si[SI_FACTOR] = factor_valid;
            S.si[SI_REJECTED] = rejected ? 1 : 0;
            st->factor_valid = factor_valid;   // the eigen cache describes the current B only
        }
    } else if (warp == 1) {
        // ---- speculation (warp 1, on another sub-partition, while warp 0
        // decides): phase 2 and the Gauss-Newton fast path at the trial point
        // as if the trial is accepted (the common case), with the same
        // arithmetic as the path after the decision.  Used when it is.
        int spec = 0;
        if (!d.jac_scale && !d.eval_only) {
            const double x = (l < n) ? cst->xt[l] : 0.0, g = (l < n) ? S.tot[NT + l] : 0.0;
            for (int e = l; e < 64; e += 32) {
                int i = e >> 3, j = e & 7;
                double b = 0.0;
                if (i < n && j < n) { int a = min(i, j), c = max(i, j); b = S.tot[a * n - a * (a - 1) / 2 + (c - a)]; }
                S.W[e] = b;
            }
            __syncwarp();
            double v, dv, sx;
            cl_scaling_xg(d, cst, n, x, g, v, dv, sx);
            scaled_model(d, n, v, dv, sx, g, S.W, S);
            double pt2;
            const bool ok = gn_try(n, S, pt2);
            spec = 1 | (ok ? 2 : 0);
            if (l == 0) S.sd[SD_PT2] = pt2;
        }
        if (l == 0) S.si[SI_SPEC] = spec;
    } else if (warp == 2) {
        // precision guard estimates at the point just evaluated (used when it is taken)
        // sum (w h)^2: this evaluation's when it is the first (slot NT+n+1), else the one kept
        if (guard_on && !d.eval_only)
            guard_estimates(n, d.m, S.tot, cst->phase == PH_INIT ? S.tot[NT + n + 1] : cst->wh2, cst->xt, S);
    }
    __syncthreads();
    trace_add(st, TR_LOGIC, tclk);

    // ================= precision guard (mixed path).  FP64 passes from here
    // on when the Gram at the new point is too ill-conditioned for FP32 steps
    // (cond > guard_cond), or when a tolerance is met while the estimated
    // FP32 floor of popt at the current point exceeds guard_floor.  The next
    // evaluation is then the current point, in FP64 (the full first
    // evaluation again when the fit is still at p0).
    if (guard_on) {
        if (t == 0) {
            const int stt = S.si[SI_STATUS];
            const bool take = !S.si[SI_REJECTED];
            const double floor_x = take ? S.sd[SD_FLOOR] : cst->floor_x;
            const double serel_x = take ? S.sd[SD_SEREL] : cst->serel_x;
            int esc = 0;
            if (stt == FS_RUNNING && take && d.guard_cond < INFINITY && !(S.sd[SD_COND] <= d.guard_cond))
                esc = (cst->phase == PH_INIT) ? GUARD_ESC_INIT : GUARD_ESC_MID;
            // a finish: the floor estimate is above guard_floor, a parameter's
            // standard error is above GUARD_SE_REL of it, or the FP32
            // iteration stopped on xtol alone with a floor estimate above
            // GUARD_STALL_FRAC of guard_floor.  (A stop on xtol alone is a
            // stall by rejections: the gradient has sunk into its FP32
            // rounding noise, so the point lies anywhere within about the
            // floor of the FP32 fixed point; a stop on ftol and xtol together
            // ends on an accepted step, like ftol.)
            else if (stt >= FS_GTOL && stt <= FS_FTOL_XTOL && d.guard_floor < INFINITY &&
                     (!(floor_x <= d.guard_floor) || !(serel_x <= GUARD_SE_REL) ||
                      (stt == FS_XTOL && !(floor_x <= GUARD_STALL_FRAC * d.guard_floor))))
                esc = GUARD_FINISH;
            S.si[SI_ESC] = esc;
            if (take) { st->floor_x = S.sd[SD_FLOOR]; st->serel_x = S.sd[SD_SEREL]; }
            if (cst->phase == PH_INIT) st->wh2 = S.tot[NT + n + 1];
        }
        __syncthreads();
        if (S.si[SI_ESC]) {
            const bool was_init = cst->phase == PH_INIT;
            if (t < n) { st->x[t] = S.vec[VX][t]; st->xt[t] = S.vec[VX][t]; st->g[t] = S.vec[VG][t]; }
            if (t < 8) S.vec[VXT][t] = S.vec[VX][t];
            if (t == 0) {
                st->f = S.sd[SD_F]; st->Delta = S.sd[SD_DELTA]; st->alpha = S.sd[SD_ALPHA];
                st->nfev = S.si[SI_NFEV]; st->njev = S.si[SI_NJEV]; st->factor_valid = 0;
                st->eval64 = 1; st->guard_why = S.si[SI_ESC];
                st->phase = was_init ? PH_INIT : PH_REINIT;
                st->cov_stage = 0;
                trace_bump(st->trace, S.si[SI_ESC] == GUARD_FINISH ? TR_N_FIN : TR_N_ESC, 1);
                S.si[SI_STATUS] = FS_RUNNING;     // the fit goes on (queue mode re-arms its tiles)
            }
            __syncthreads();
            if (warp == 0) prep_pass<PREC, MS>(d, st, S, true);
            trace_add(st, TR_PREP, tclk);
            return;
        }
    }

    const int status = S.si[SI_STATUS];
    if (status != FS_RUNNING) {
        if (t == 0) { st->f = S.sd[SD_F]; st->nfev = S.si[SI_NFEV]; st->njev = S.si[SI_NJEV]; st->Delta = S.sd[SD_DELTA]; }
        if (t < n) st->x[t] = S.vec[VX][t];
        __syncthreads();
        write_result(d, st, res, status, S);
        trace_add(st, TR_FINISH, tclk);
        if (t == 0) { st->run = RS_DONE; st->fit_status = status; atomicSub(running, 1); }
        __syncthreads();
        if (t < 32) res->trace[t] = double(__ldcg(st->trace + t));
        return;
    }

    // ================= phase 2: scaled model matrix Ah = D B D + diag(C), and
    // the Gauss-Newton fast path: when B_hat is safely full rank (no
    // eigenvalue near the rank cutoff) and the trial step lies in the region,
    // the step needs no eigen-decomposition.
    // Guard: the refinement must contract (ratio ~ eps32 cond of the
    // equilibrated matrix), and lambda_min >= min_diag / cond must stay far
    // above the rank cutoff lambda_max 8 n eps64 (lambda_max <= n here), so
    // that the pseudo-inverse of the eigen path would drop nothing.
    // After a rejected trial B_hat and g_hat are unchanged and Delta has
    // shrunk below the rejected step (Algorithm 3), so the Gauss-Newton step
    // (inside the old region or not) cannot be inside the new one: skip it.
    // An accepted trial takes warp 1's speculative results as they are.
    const bool spec_used = (S.si[SI_SPEC] & 1) && !S.si[SI_REJECTED];
    if (!spec_used) {
        if (warp == 0) {
            const double v = (l < 8) ? S.vec[VV][l] : 0.0, dv = (l < 8) ? S.vec[VDV][l] : 0.0;
            const double sx = (l < 8) ? S.vec[VSX][l] : 1.0;
            const double g = (l < n) ? S.vec[VG][l] : 0.0;
            scaled_model(d, n, v, dv, sx, g, S.B, S);
            if (!S.si[SI_REJECTED]) {
                double pt2;
                const bool ok = gn_try(n, S, pt2);
                const double Delta = S.sd[SD_DELTA];
                const bool inside = ok && pt2 <= Delta * Delta;
                if (l == 0) {
                    S.si[SI_GN] = inside ? 1 : 0;
                    if (inside) trace_bump(st->trace, TR_N_GN, 1);
                }
            } else if (l == 0) {
                S.si[SI_GN] = 0;
            }
        }
    } else if (warp == 0 && l == 0) {
        const double Delta = S.sd[SD_DELTA];
        const bool inside = (S.si[SI_SPEC] & 2) && S.sd[SD_PT2] <= Delta * Delta;
        S.si[SI_GN] = inside ? 1 : 0;
        if (inside) trace_bump(st->trace, TR_N_GN, 1);
    }
    __syncthreads();
    trace_add(st, TR_GN, tclk);

    // ================= factorisation (all threads), reused after a rejection
    if (S.si[SI_GN]) {
        // not needed
    } else if (!S.si[SI_FACTOR]) {
        int sw = eig_fast(n, S.Ah, cst->has_basis ? cst->V : nullptr, S, st->trace);
        if (t < 64) st->V[t] = S.V[t];
        if (t < 8) st->lam[t] = S.vec[VLAM][t];
        if (t == 0) { st->has_basis = 1; st->factor_valid = 1; st->jacobi_sweeps = sw; trace_bump(st->trace, TR_N_EIG, 1); }
    } else {
        if (t < 64) S.V[t] = cst->V[t];
        if (t < 8) S.vec[VLAM][t] = cst->lam[t];
    }
    __syncthreads();
    trace_add(st, TR_EIGEN, tclk);

    // ================= phase 3 (warp 0): step
    if (warp == 0) {
        double Delta = S.sd[SD_DELTA], alpha = S.sd[SD_ALPHA], gnorm = S.sd[SD_GNORM];
        double gh = (l < n) ? S.vec[VGH][l] : 0.0;
        double dl = (l < n) ? S.vec[VD][l] : 0.0;
        const bool gn = S.si[SI_GN] != 0;
        double theta = fmax(0.995, 1.0 - gnorm);
        int a2it = 0;
        if (gn) alpha = 0.0;
        else {
        // gV = V^T g_hat
        double gV;
        {
            int i = l >> 2, j = l & 3;
            double acc = 0.0;
            if (i < n) {
                if (j < n) acc = S.V[j * 8 + i] * S.vec[VGH][j];
                if (j + 4 < n) acc = fma(S.V[(j + 4) * 8 + i], S.vec[VGH][j + 4], acc);
            }
            acc += __shfl_xor_sync(FULL, acc, 1);
            acc += __shfl_xor_sync(FULL, acc, 2);
            gV = __shfl_sync(FULL, acc, (l & 7) << 2);
            if (l >= n) gV = 0.0;
        }
        double lam = (l < n) ? S.vec[VLAM][l] : 0.0;
        double lmax = gmax8(l < n ? lam : -INFINITY);
        bool keep = (l < n) && lmax > 0.0 && lam > lmax * (8.0 * n * EPS64);
        if (!keep) { gV = 0.0; lam = 0.0; }
        bool full_rank = __all_sync(FULL, keep || l >= n);
        // Algorithm 1: Gauss-Newton trial step, else Algorithm 2
        double comp = (gV != 0.0) ? gV * rcp64(lam) : 0.0;
        double ptn2 = gsum8(comp * comp);
        if (ptn2 <= Delta * Delta) {
            alpha = 0.0;
        } else {
            double ghn = sqrt(gsum8(gh * gh));
            alpha = lm_parameter(lam, gV, ghn, Delta, alpha, full_rank, &a2it);
            comp = (gV != 0.0) ? gV * rcp64(lam + alpha) : 0.0;
        }
        vstore(S.vec[VTMP], n, comp);
        double s_tr0 = -matvec8(S.V, S.vec[VTMP], n);
        vstore(S.vec[VSTR], n, s_tr0);
        }
        const double s_tr = (l < n) ? S.vec[VSTR][l] : 0.0;
        double sh = s_tr, qval;
        int kind = 0;
        if (d.bounded) {
            double x = (l < n) ? S.vec[VX][l] : 0.0;
            double lbl = (l < n) ? d.lb[l] : -INFINITY, ubl = (l < n) ? d.ub[l] : INFINITY;
            double sfull = dl * s_tr;
            bool inside = __all_sync(FULL, l >= n || (x + sfull >= lbl && x + sfull <= ubl));
            qval = quad_value(S.Ah, S.vec[VGH], S.vec[VSTR], n);
            if (!inside) {
                bool hit;
                double tau = step_to_bound(x, (l < n) ? sfull : 0.0, lbl, ubl, hit);
                double sA = theta * tau * s_tr;                         // A: truncated
                vstore(S.vec[VTMP], n, sA);
                double best = quad_value(S.Ah, S.vec[VGH], S.vec[VTMP], n);
                sh = sA; kind = 1;
                double sb = tau * s_tr;                                 // B: reflected
                double rh = hit ? -s_tr : s_tr;
                double xb = x + dl * sb;
                bool hit2;
                double t_box = step_to_bound(xb, (l < n) ? dl * rh : 0.0, lbl, ubl, hit2);
                double t_tr = tr_intersect(l < n ? sb : 0.0, l < n ? rh : 0.0, Delta);
                double t_max = fmin(t_box, t_tr);
                if (t_max > 0.0) {
                    double t_lo = (1.0 - theta) * t_max;
                    double t_hi = (t_box <= t_tr) ? theta * t_box : t_tr;
                    if (t_lo <= t_hi) {
                        vstore(S.vec[VTMP], n, sb);
                        vstore(S.vec[VSH], n, rh);
                        double tB;
                        double vB = minimize_on_segment(S.Ah, S.vec[VGH], S.vec[VTMP], S.vec[VSH], nullptr, n, t_lo, t_hi, tB);
                        if (vB < best) { best = vB; sh = sb + tB * rh; kind = 2; }
                    }
                }
                double ag = -gh;                                        // C: scaled anti-gradient
                double agn = sqrt(gsum8(ag * ag));
                if (agn > 0.0) {
                    double t_tr2 = Delta * rcp64(agn);
                    bool hit3;
                    double t_box2 = step_to_bound(x, (l < n) ? dl * ag : 0.0, lbl, ubl, hit3);
                    double t_hi = (t_box2 < t_tr2) ? theta * t_box2 : t_tr2;
                    vstore(S.vec[VTMP], n, 0.0);
                    vstore(S.vec[VSH], n, ag);
                    double tC;
                    double vC = minimize_on_segment(S.Ah, S.vec[VGH], S.vec[VTMP], S.vec[VSH], nullptr, n, 0.0, t_hi, tC);
                    if (vC < best) { best = vC; sh = tC * ag; kind = 3; }
                }
                qval = best;
            }
        } else {
            qval = quad_value(S.Ah, S.vec[VGH], S.vec[VSTR], n);
        }
        if (l >= n) sh = 0.0;
        double step = dl * sh;
        double x = (l < n) ? S.vec[VX][l] : 0.0;
        double xt = x + step;
        if (d.bounded && l < n) {
            if (xt <= d.lb[l]) xt = nextafter(d.lb[l], (double)INFINITY);
            if (xt >= d.ub[l]) xt = nextafter(d.ub[l], -(double)INFINITY);
        }
        if (l < 8) S.vec[VXT][l] = (l < n) ? xt : 0.0;
        // ||s_h||, ||w||, ||x|| for the next iteration's radius and xtol tests
        // the three sums in one butterfly: lanes 0-7 ||s_h||^2, 8-15 ||w||^2,
        // 16-23 ||x||^2 (each group in gsum8's order)
        double nv;
        {
            const double ww_l = __shfl_sync(FULL, step * step, l & 7), xx_l = __shfl_sync(FULL, x * x, l & 7);
            nv = (l < 8) ? sh * sh : (l < 16) ? ww_l : (l < 24) ? xx_l : 0.0;
            nv += __shfl_xor_sync(FULL, nv, 4);
            nv += __shfl_xor_sync(FULL, nv, 2);
            nv += __shfl_xor_sync(FULL, nv, 1);
        }
        nv = sqrt(nv);
        double s_norm = __shfl_sync(FULL, nv, 0), w_norm = __shfl_sync(FULL, nv, 8), x_norm = __shfl_sync(FULL, nv, 16);
        if (l < n) { st->x[l] = x; st->xt[l] = xt; st->g[l] = S.vec[VG][l]; st->s_h[l] = sh; }
        for (int k = l; k < NT; k += 32) {
            int a = 0, r = k;
            while (r >= n - a) { r -= n - a; ++a; }
            st->B[k] = S.B[a * 8 + a + r];
        }
        // a trial whose predicted reduction is a large fraction of f is evaluated
        // in the direct form (packed models, linear loss, mixed FP32 passes)
        int packed = 0;
        MS::dispatch(d.model, [&](auto m) { packed = decltype(m)::PACK; });
        const bool wide = PREC == PREC_MIXED && !e64 && packed != 0 && d.loss == LOSS_LINEAR && !d.cov &&
                          -qval >= WIDE_PRED_FRAC * S.sd[SD_F];
        if (l == 0) {
            st->f = S.sd[SD_F]; st->Delta = Delta; st->alpha = alpha; st->nfev = S.si[SI_NFEV];
            st->njev = S.si[SI_NJEV]; st->predicted = -qval;
            st->step_norm = w_norm; st->s_norm = s_norm; st->xtol_thr = d.xtol * (d.xtol + x_norm);
            st->phase = wide ? PH_WIDE : PH_TRIAL; st->last_kind = kind; st->alg2_iters = a2it;
            st->cov_stage = 0;
            trace_bump(st->trace, TR_N_ALG2IT, a2it);
            trace_bump(st->trace, TR_N_BOUNDED, kind != 0);
            trace_bump(st->trace, TR_N_WIDE, wide ? 1 : 0);
        }
        __syncwarp();
    }
    trace_add(st, TR_STEP, tclk);
    if (warp == 0) prep_pass<PREC, MS>(d, st, S, e64);
    trace_add(st, TR_PREP, tclk);
}

}  // namespace gbfit

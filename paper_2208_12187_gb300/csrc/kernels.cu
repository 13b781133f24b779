// Device kernels of libgbfit.
//
//   eval_round_kernel<PREC>  one trust-region iteration for every running fit:
//       each CTA takes (fit, tile) work items, evaluates model, residual and
//       Jacobian row per point in registers, reduces J^T J, J^T r and cost
//       sums over its tile (never writing J), and writes one tile partial.
//       The last CTA of a group of tiles combines the group (FP64, fixed
//       order); the last group of a fit combines the fit and runs the
//       trust-region step for it (trf_step), which prepares the next
//       evaluation point.  No CTA waits for another: the hand-off is an
//       atomic arrival counter (last arriver continues).
//   round_end_kernel  sets the CUDA-graph WHILE condition (any fit running
//       and under the round cap).
//   stage_weights_kernel  w = 1/sigma in FP64 for the plain path.
//   tr_subproblem_kernel  one subproblem solve (test entry point).
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>
#include "gbfit_internal.cuh"
#include "models.cuh"
#include "trf_device.cuh"

namespace gbfit {

// ------------------------------------------------------------------ warp/block reduction
// Reduce-scatter across the warp: after 5 halvings lane l holds the warp sum
// of ceil(K/32) slots.  Costs about K shuffles instead of 5 K.
template <int K, typename T>
struct WarpRS {
    static constexpr int H1 = (K + 1) / 2, H2 = (H1 + 1) / 2, H3 = (H2 + 1) / 2, H4 = (H3 + 1) / 2,
                         H5 = (H4 + 1) / 2;
    template <int C, int H>
    __device__ __forceinline__ static void level(T (&v)[K], int lane, int off) {
        bool up = lane & off;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            T a = v[i];
            T b = (i + H < C) ? v[i + H] : T(0);
            T send = up ? a : b;
            T keep = up ? b : a;
            v[i] = keep + __shfl_xor_sync(FULL, send, off);
        }
    }
    // original slot held in v[i] by `lane` after all levels, or -1 for padding:
    // unwind the halvings, checking the index against each level's count.
    __device__ __forceinline__ static int slot(int lane, int i) {
        int k = i + ((lane & 1) ? H5 : 0);
        if (k >= H4) return -1;
        k += (lane & 2) ? H4 : 0;
        if (k >= H3) return -1;
        k += (lane & 4) ? H3 : 0;
        if (k >= H2) return -1;
        k += (lane & 8) ? H2 : 0;
        if (k >= H1) return -1;
        k += (lane & 16) ? H1 : 0;
        return k < K ? k : -1;
    }
    __device__ __forceinline__ static void run(T (&v)[K], int lane) {
        level<K, H1>(v, lane, 16);
        level<H1, H2>(v, lane, 8);
        level<H2, H3>(v, lane, 4);
        level<H3, H4>(v, lane, 2);
        level<H4, H5>(v, lane, 1);
    }
};

// Block sum of acc[K] over EVAL_THREADS threads; thread k < K gets slot k in out.
template <int K, typename T>
__device__ __forceinline__ void block_reduce(T (&acc)[K], T* red /*[8][K]*/, T& out) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpRS<K, T>::run(acc, lane);
#pragma unroll
    for (int i = 0; i < WarpRS<K, T>::H5; ++i) {
        int s = WarpRS<K, T>::slot(lane, i);
        if (s >= 0) red[warp * K + s] = acc[i];
    }
    __syncthreads();
    if (threadIdx.x < K) {
        T sum = red[threadIdx.x];
#pragma unroll
        for (int w = 1; w < EVAL_THREADS / 32; ++w) sum += red[w * K + threadIdx.x];
        out = sum;
    }
}

// ------------------------------------------------------------------ point loops
template <typename T> __device__ __forceinline__ T ldg_t(const void* p, int64_t i) { return __ldg((const T*)p + i); }

struct PointCoord {
    // incremental pixel coordinates for the implicit grid
    int64_t X, Y, W;
    __device__ void init(int64_t i, int64_t w) { W = w; Y = i / w; X = i - Y * w; }
    __device__ void advance(int64_t step) {
        X += step;
        if (X >= W) { if (W >= EVAL_THREADS) { X -= W; Y += 1; } else { Y += X / W; X = X % W; } }
    }
};

template <class M, int PREC, typename DT, int LAYOUT, int WK>
__device__ __forceinline__ void tile_points(const FitDesc& d, const float* pf, const double* pd,
                                            int64_t i0, int64_t i1, bool check,
                                            typename std::conditional<PREC == PREC_MIXED, float, double>::type
                                                (&acc)[n_acc(M::N, PREC)],
                                            int& bad) {
    using AT = typename std::conditional<PREC == PREC_MIXED, float, double>::type;
    constexpr int N = M::N;
    constexpr int NT = n_tri(N);
    constexpr int K = n_acc(N, PREC);
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = AT(0);
    float pfl[PF];
    double pdl[PD];
    if (PREC == PREC_MIXED) {
#pragma unroll
        for (int k = 0; k < PF; ++k) pfl[k] = pf[k];
    } else {
#pragma unroll
        for (int k = 0; k < PD; ++k) pdl[k] = pd[k];
    }
    PointCoord pc;
    int64_t i = i0 + threadIdx.x;
    if (LAYOUT == X_GRID) pc.init(i, d.grid_w);
    for (; i < i1; i += EVAL_THREADS) {
        AT X, Y = AT(0);
        if (LAYOUT == X_GRID) {
            X = AT(pc.X); Y = AT(pc.Y);
            pc.advance(EVAL_THREADS);
        } else {
            X = AT(ldg_t<DT>(d.x, i));
            if (LAYOUT == X_SOA2) Y = AT(ldg_t<DT>(d.x2, i));
        }
        AT yv = AT(ldg_t<DT>(d.y, i));
        AT w = AT(1);
        if (WK == W_ARRAY) w = AT(ldg_t<double>(d.w, i));   // staged FP64 weights
        if (WK == W_SIGMA) {
            AT s = AT(ldg_t<DT>(d.w, i));
            if (check && !(s > AT(0) && isfinite(s))) bad = 1;
            if (PREC == PREC_MIXED) w = __frcp_rn(float(s)); else w = AT(1) / s;
        }
        if (check) {
            if (!isfinite(X) || !isfinite(Y) || !isfinite(yv)) bad = 1;
            if (WK == W_ARRAY && !(w > AT(0) && isfinite(w))) bad = 1;
        }
        AT Jw[N];
        if constexpr (PREC == PREC_MIXED) {
            float hb, dh, J[N];
            M::eval_mixed(pfl, X, Y, hb, dh, J);
            float r = w * (hb - yv);
            float dr = w * dh;
            float rn = r + dr;
#pragma unroll
            for (int a = 0; a < N; ++a) Jw[a] = w * J[a];
            int idx = 0;
#pragma unroll
            for (int a = 0; a < N; ++a)
#pragma unroll
                for (int b = a; b < N; ++b) { acc[idx] = fmaf(Jw[a], Jw[b], acc[idx]); ++idx; }
#pragma unroll
            for (int a = 0; a < N; ++a) acc[NT + a] = fmaf(Jw[a], rn, acc[NT + a]);
            acc[NT + N] = fmaf(rn, rn, acc[NT + N]);
            acc[NT + N + 1] = fmaf(dr, fmaf(2.0f, r, dr), acc[NT + N + 1]);
            acc[NT + N + 2] = fmaf(r, r, acc[NT + N + 2]);
        } else {
            double h, J[N];
            M::eval_plain(pdl, X, Y, h, J);
            double r = w * (h - yv);
#pragma unroll
            for (int a = 0; a < N; ++a) Jw[a] = w * J[a];
            int idx = 0;
#pragma unroll
            for (int a = 0; a < N; ++a)
#pragma unroll
                for (int b = a; b < N; ++b) { acc[idx] = fma(Jw[a], Jw[b], acc[idx]); ++idx; }
#pragma unroll
            for (int a = 0; a < N; ++a) acc[NT + a] = fma(Jw[a], r, acc[NT + a]);
            acc[NT + N] = fma(r, r, acc[NT + N]);
        }
    }
}

// ------------------------------------------------------------------ shared memory of the round kernel
struct RoundSmem {
    FitDesc desc;
    float pf[PF];
    double pd[PD];
    int flag[4];
    union {
        float redf[8 * KMAX];
        double redd[8 * KMAX];
        double comb[EVAL_THREADS];
    };
    TrfSmem trf;
};

// Sum rows [0, nrows) of a [rows][KMAX] array into out[0..K) in a fixed order
// using all threads: thread t handles slot t % K over rows = part (mod P).
template <typename T>
__device__ void combine_rows(const T* rows, int nrows, int K, double* scratch, double* out) {
    int P = EVAL_THREADS / K;
    int t = threadIdx.x;
    int k = t % K, part = t / K;
    double s = 0.0;
    if (part < P)
        for (int r = part; r < nrows; r += P) s += double(__ldcg(rows + (int64_t)r * KMAX + k));   // L2: written by other CTAs
    scratch[t] = s;
    __syncthreads();
    if (t < K) {
        double tot = 0.0;
        for (int p = 0; p < P; ++p) tot += scratch[p * K + t];
        out[t] = tot;
    }
    __syncthreads();
}

// ------------------------------------------------------------------ the trust-region step
__device__ void write_result(const FitDesc& d, FitState* st, FitResult* res, int status, TrfSmem& S);

// Load scaling quantities (lane values) for the current x and g.
__device__ __forceinline__ void scaling(const FitDesc& d, const FitState* st, TrfSmem& S, int n,
                                        double& v, double& dv, double& sx) {
    int l = lane_id();
    double x = ld(S.vec[VX], n), g = ld(S.vec[VG], n);
    v = 1.0; dv = 0.0; sx = 0.0;
    if (l < n) {
        double lb = d.lb[l], ub = d.ub[l];
        if (g < 0.0 && isfinite(ub)) { v = ub - x; dv = -1.0; }
        else if (g > 0.0 && isfinite(lb)) { v = x - lb; dv = 1.0; }
        sx = d.jac_scale ? 1.0 / st->scale_inv[l] : d.xscale[l];
    } else {
        v = 0.0;
    }
}

__device__ void jac_scale_update(FitState* st, const TrfSmem& S, int n, bool first) {
    int l = lane_id();
    if (l < n) {
        double c = sqrt(S.B[l * 8 + l]);
        if (!first) c = fmax(c, st->scale_inv[l]);
        if (c == 0.0) c = 1.0;
        st->scale_inv[l] = c;
    }
    __syncwarp();
}

// Prepare the pass constants for evaluating xt relative to x.
template <int PREC>
__device__ void prep_pass(const FitDesc& d, FitState* st, TrfSmem& S) {
    int l = lane_id();
    int n = d.n;
    if (PREC == PREC_MIXED) {
        __shared__ MixedParams P;
        if (l < n) {
            double x = S.vec[VX][l], xt = S.vec[VXT][l];
            float xf = float(x);
            P.x[l] = xf;
            P.xlo[l] = float(x - double(xf));
            P.xt[l] = float(xt);
            P.dx[l] = float(xt - x);
        }
        __syncwarp();
        if (l == 0) {
            float pf[PF];
            for (int k = 0; k < PF; ++k) pf[k] = 0.0f;
            switch (d.model) {
                case 0: MGauss1D::prep_mixed(P, pf); break;
                case 1: MDexp::prep_mixed(P, pf); break;
                case 2: MGauss2D::prep_mixed(P, pf); break;
                case 3: MPoly2::prep_mixed(P, pf); break;
            }
            for (int k = 0; k < PF; ++k) st->pf[k] = pf[k];
        }
    } else {
        if (l == 0) {
            double pd[PD];
            for (int k = 0; k < PD; ++k) pd[k] = 0.0;
            switch (d.model) {
                case 0: MGauss1D::prep_plain(S.vec[VXT], pd); break;
                case 1: MDexp::prep_plain(S.vec[VXT], pd); break;
                case 2: MGauss2D::prep_plain(S.vec[VXT], pd); break;
                case 3: MPoly2::prep_plain(S.vec[VXT], pd); break;
            }
            for (int k = 0; k < PD; ++k) st->pd[k] = pd[k];
        }
    }
    __syncwarp();
}

// One trust-region iteration for one fit (warp 0 of the finishing CTA).
// S.tot holds the combined sums of the evaluation that just finished.
template <int PREC>
__device__ void trf_step(const FitDesc& d, FitState* st, FitResult* res, TrfSmem& S, int* running) {
    const int n = d.n;
    const int l = lane_id();
    const int NT = n_tri(n);
    // ---- load state
    if (l < n) {
        S.vec[VX][l] = st->x[l];
        S.vec[VXT][l] = st->xt[l];
        S.vec[VG][l] = st->g[l];
    }
    for (int e = l; e < 64; e += 32) {
        int i = e >> 3, j = e & 7;
        double b = 0.0;
        if (i < n && j < n) { int a = min(i, j), c = max(i, j); b = st->B[a * n - a * (a - 1) / 2 + (c - a)]; }
        S.B[e] = b;
    }
    __syncwarp();
    const double f2n = S.tot[NT + n];
    int status = FS_RUNNING;
    double f = st->f, Delta = st->Delta, alpha = st->alpha;
    int nfev = st->nfev, njev = st->njev, factor_valid = st->factor_valid;

    auto take_new_eval = [&]() {
        // x <- xt, g, B <- the evaluation just combined
        if (l < n) { S.vec[VX][l] = S.vec[VXT][l]; S.vec[VG][l] = S.tot[NT + l]; }
        for (int e = l; e < 64; e += 32) {
            int i = e >> 3, j = e & 7;
            double b = 0.0;
            if (i < n && j < n) { int a = min(i, j), c = max(i, j); b = S.tot[a * n - a * (a - 1) / 2 + (c - a)]; }
            S.B[e] = b;
        }
        __syncwarp();
    };

    if (st->phase == PH_INIT) {
        take_new_eval();
        f = 0.5 * f2n;
        nfev = 1; njev = 1;
        bool finite_all = isfinite(f);
        for (int k = 0; k < NT + n; ++k) finite_all = finite_all && isfinite(S.tot[k]);
        if (st->bad_data) status = FS_INVALID_DATA;
        else if (!finite_all) status = FS_NUMERICAL;
        if (status == FS_RUNNING) {
            if (d.jac_scale) jac_scale_update(st, S, n, true);
            double v, dv, sx;
            scaling(d, st, S, n, v, dv, sx);
            double xl = ld(S.vec[VX], n);
            double q = (l < n) ? xl / (sqrt(v) * sx) : 0.0;
            Delta = sqrt(gsum8(q * q));
            if (Delta == 0.0) Delta = 1.0;
            alpha = 0.0;
            factor_valid = 0;
        }
    } else {
        nfev += 1;
        double f_new = 0.5 * f2n;
        double actual = (PREC == PREC_MIXED) ? -0.5 * S.tot[NT + n + 1] : f - f_new;
        double pred = st->predicted;
        double gamma = (isfinite(f_new) && isfinite(actual) && pred > 0.0) ? actual / pred : -INFINITY;
        double snorm = sqrt(gsum8(l < n ? st->s_h[l] * st->s_h[l] : 0.0));
        bool accepted;
        double Dn;
        if (gamma > 0.75) { accepted = true; Dn = 2.0 * Delta; }
        else if (gamma >= 0.25 && gamma <= 0.75) { accepted = true; Dn = Delta; }
        else { accepted = false; Dn = 0.25 * snorm; }
        double xnorm = sqrt(dot8(S.vec[VX], S.vec[VX], n));
        bool ftol_ok = accepted && actual < d.ftol * f;
        bool xtol_ok = st->step_norm < d.xtol * (d.xtol + xnorm);
        if (accepted) {
            take_new_eval();
            f = f_new;
            njev += 1;
            if (d.jac_scale) jac_scale_update(st, S, n, false);
            factor_valid = 0;
        }
        Delta = Dn;
        if (ftol_ok && xtol_ok) status = FS_FTOL_XTOL;
        else if (ftol_ok) status = FS_FTOL;
        else if (xtol_ok) status = FS_XTOL;
    }

    double v = 1.0, dv = 0.0, sx = 1.0, gnorm = 0.0;
    if (status == FS_RUNNING) {
        scaling(d, st, S, n, v, dv, sx);
        double g = ld(S.vec[VG], n);
        gnorm = gmax8(l < n ? fabs(v * g) : 0.0);
        if (gnorm < d.gtol) status = FS_GTOL;
        else if (nfev >= d.max_nfev) status = FS_MAX_NFEV;
    }
    if (status != FS_RUNNING) {
        st->f = f; st->nfev = nfev; st->njev = njev; st->Delta = Delta;
        if (l < n) st->x[l] = S.vec[VX][l];
        __syncwarp();
        write_result(d, st, res, status, S);
        if (l == 0) { st->run = RS_DONE; st->fit_status = status; atomicSub(running, 1); }
        return;
    }

    // ---- scaled problem: d = sqrt(v) sx, g_hat = d g, C = g dv sx^2, Ah = D B D + diag(C)
    double g = ld(S.vec[VG], n);
    double dl = (l < n) ? sqrt(v) * sx : 0.0;
    double gh = dl * g;
    double Cl = (l < n && d.bounded) ? g * dv * sx * sx : 0.0;
    vstore(S.vec[VD], n, dl);
    vstore(S.vec[VGH], n, gh);
    vstore(S.vec[VC], n, Cl);
    for (int e = l; e < 64; e += 32) {
        int i = e >> 3, j = e & 7;
        double a = 0.0;
        if (i < n && j < n) a = S.vec[VD][i] * S.B[e] * S.vec[VD][j] + (i == j ? S.vec[VC][i] : 0.0);
        S.Ah[e] = a;
    }
    __syncwarp();
    if (!factor_valid) {
        // warm start: rotate the new matrix into the previous eigenbasis, where
        // it is nearly diagonal once the fit settles (fewer sweeps).
        bool warm = st->has_basis != 0;
        for (int e = l; e < 64; e += 32) {
            int i = e >> 3, j = e & 7;
            S.V[e] = warm ? st->V[e] : ((i == j && i < n) ? 1.0 : 0.0);
        }
        __syncwarp();
        if (warm) congruence(n, S.Ah, S.V, S.W, S.A);
        else for (int e = l; e < 64; e += 32) S.A[e] = S.Ah[e];
        __syncwarp();
        int sw = jacobi_eig(n, S.A, S.V, S.cs, S.pairs, 30);
        if (l == 0) st->jacobi_sweeps = sw;
        double lam = (l < n) ? S.A[l * 8 + l] : 0.0;
        vstore(S.vec[VLAM], n, lam);
        for (int e = l; e < 64; e += 32) st->V[e] = S.V[e];
        if (l < n) st->lam[l] = lam;
        if (l == 0) st->has_basis = 1;
        factor_valid = 1;
    } else {
        for (int e = l; e < 64; e += 32) S.V[e] = st->V[e];
        if (l < n) S.vec[VLAM][l] = st->lam[l];
        __syncwarp();
    }
    // gV = V^T g_hat; rank cutoff (R10)
    double lam = ld(S.vec[VLAM], n);
    double gV;
    {
        int i = l >> 2, j = l & 3;    // lane -> (column i of V, rows j, j+4)
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
    double lmax = gmax8(l < n ? lam : -INFINITY);
    bool keep = (l < n) && lmax > 0.0 && lam > lmax * (8.0 * n * EPS64);
    if (!keep) { gV = 0.0; lam = 0.0; }
    bool full_rank = __all_sync(FULL, keep || l >= n);
    double theta = fmax(0.995, 1.0 - gnorm);

    // ---- Algorithm 1: trial Gauss-Newton step, else Algorithm 2
    double comp = (gV != 0.0) ? gV / lam : 0.0;           // p_t in the eigenbasis (negated)
    double ptn = sqrt(gsum8(comp * comp));
    int a2it = 0;
    if (ptn <= Delta) {
        alpha = 0.0;
    } else {
        double ghn = sqrt(gsum8(gh * gh));
        alpha = lm_parameter(lam, gV, ghn, Delta, alpha, full_rank, &a2it);
        comp = (gV != 0.0) ? gV / (lam + alpha) : 0.0;
    }
    // s_tr = -V comp
    vstore(S.vec[VTMP], n, comp);
    double s_tr = -matvec8(S.V, S.vec[VTMP], n);
    vstore(S.vec[VSTR], n, s_tr);

    // ---- bounded step selection (R9)
    double sh = s_tr;
    double qval;
    int kind = 0;
    if (d.bounded) {
        double x = ld(S.vec[VX], n);
        double lbl = (l < n) ? d.lb[l] : -INFINITY, ubl = (l < n) ? d.ub[l] : INFINITY;
        double sfull = dl * s_tr;
        bool inside = __all_sync(FULL, l >= n || (x + sfull >= lbl && x + sfull <= ubl));
        qval = quad_value(S.Ah, S.vec[VGH], S.vec[VSTR], n);
        if (!inside) {
            bool hit;
            double tau = step_to_bound(x, (l < n) ? sfull : 0.0, lbl, ubl, hit);
            // A: truncated
            double sA = theta * tau * s_tr;
            vstore(S.vec[VTMP], n, sA);
            double best = quad_value(S.Ah, S.vec[VGH], S.vec[VTMP], n);
            sh = sA; kind = 1;
            // B: reflected
            double sb = tau * s_tr;
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
            // C: scaled anti-gradient
            double ag = -gh;
            double agn = sqrt(gsum8(ag * ag));
            if (agn > 0.0) {
                double t_tr2 = Delta / agn;
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
    // ---- trial point
    double step = dl * sh;
    double x = ld(S.vec[VX], n);
    double xt = x + step;
    if (d.bounded && l < n) {
        if (xt <= d.lb[l]) xt = nextafter(d.lb[l], INFINITY);
        if (xt >= d.ub[l]) xt = nextafter(d.ub[l], -INFINITY);
    }
    vstore(S.vec[VXT], n, xt);
    double step_norm = sqrt(gsum8(step * step));
    // ---- store
    if (l < n) {
        st->x[l] = x; st->xt[l] = xt; st->g[l] = S.vec[VG][l]; st->s_h[l] = sh;
    }
    for (int k = l; k < NT; k += 32) {
        int a = 0, r = k;
        while (r >= n - a) { r -= n - a; ++a; }
        st->B[k] = S.B[a * 8 + a + r];
    }
    if (l == 0) {
        st->f = f; st->Delta = Delta; st->alpha = alpha; st->nfev = nfev; st->njev = njev;
        st->factor_valid = factor_valid; st->predicted = -qval; st->step_norm = step_norm;
        st->phase = PH_TRIAL; st->last_kind = kind; st->alg2_iters = a2it;
    }
    __syncwarp();
    prep_pass<PREC>(d, st, S);
}

// pcov (R13) and the result record.
__device__ void write_result(const FitDesc& d, FitState* st, FitResult* res, int status, TrfSmem& S) {
    int n = d.n, l = lane_id();
    if (l < n) res->popt[l] = st->x[l];
    for (int k = l; k < KMAX; k += 32) res->tot[k] = S.tot[k];
    if (l == 0) {
        res->cost = st->f; res->nfev = st->nfev; res->njev = st->njev; res->fit_status = status;
    }
    bool ok = (status >= 0) && d.m > n;
    if (!ok) {
        for (int e = l; e < 64; e += 32) res->pcov[e] = INFINITY;
        __syncwarp();
        return;
    }
    for (int e = l; e < 64; e += 32) {
        int i = e >> 3, j = e & 7;
        S.A[e] = S.B[e];
        S.V[e] = (i == j && i < n) ? 1.0 : 0.0;
    }
    __syncwarp();
    jacobi_eig(n, S.A, S.V, S.cs, S.pairs, 30);
    double lam = (l < n) ? S.A[l * 8 + l] : 0.0;
    double lmax = gmax8(l < n ? lam : -INFINITY);
    double inv = (l < n && lmax > 0.0 && lam > lmax * (8.0 * n * EPS64)) ? 1.0 / lam : 0.0;
    if (l < 8) S.vec[VTMP][l] = inv;
    __syncwarp();
    double scale = d.absolute_sigma ? 1.0 : 2.0 * st->f / double(d.m - n);
    for (int e = l; e < 64; e += 32) {
        int i = e >> 3, j = e & 7;
        double acc = 0.0;
        if (i < n && j < n)
            for (int k = 0; k < n; ++k) acc = fma(S.V[i * 8 + k] * S.vec[VTMP][k], S.V[j * 8 + k], acc);
        if (i < n && j < n) res->pcov[i * n + j] = acc * scale;
    }
    __syncwarp();
}

// ------------------------------------------------------------------ the round kernel
template <class M, int PREC>
__device__ void eval_tile_dispatch(const RoundSmem& sm, int64_t i0, int64_t i1, bool check, int& bad,
                                   typename std::conditional<PREC == PREC_MIXED, float, double>::type
                                       (&acc)[n_acc(M::N, PREC)]) {
    const FitDesc& d = sm.desc;
    bool f64 = d.dtype == F64;
#define GB_CASE(LAY, WKV)                                                                         \
    if (f64) tile_points<M, PREC, double, LAY, WKV>(d, sm.pf, sm.pd, i0, i1, check, acc, bad);    \
    else tile_points<M, PREC, float, LAY, WKV>(d, sm.pf, sm.pd, i0, i1, check, acc, bad);
    int wk = d.wkind;
    if (M::N == 7) {
        if (d.layout == X_GRID) {
            if (wk == W_NONE) { GB_CASE(X_GRID, W_NONE) } else if (wk == W_ARRAY) { GB_CASE(X_GRID, W_ARRAY) } else { GB_CASE(X_GRID, W_SIGMA) }
        } else {
            if (wk == W_NONE) { GB_CASE(X_SOA2, W_NONE) } else if (wk == W_ARRAY) { GB_CASE(X_SOA2, W_ARRAY) } else { GB_CASE(X_SOA2, W_SIGMA) }
        }
    } else {
        if (wk == W_NONE) { GB_CASE(X_VEC, W_NONE) } else if (wk == W_ARRAY) { GB_CASE(X_VEC, W_ARRAY) } else { GB_CASE(X_VEC, W_SIGMA) }
    }
#undef GB_CASE
}

template <class M, int PREC>
__device__ void process_item(RoundSmem& sm, const Engine& E, FitResult* results, int fit, int tile) {
    using AT = typename std::conditional<PREC == PREC_MIXED, float, double>::type;
    constexpr int N = M::N;
    constexpr int K = n_acc(N, PREC);
    const FitDesc& d = sm.desc;
    FitState* stp = E.state + fit;
    int64_t i0 = (int64_t)tile * d.tile_points;
    int64_t i1 = i0 + d.tile_points;
    if (i1 > d.m) i1 = d.m;
    bool check = sm.flag[1] == PH_INIT;
    int bad = 0;
    AT acc[K];
    eval_tile_dispatch<M, PREC>(sm, i0, i1, check, bad, acc);
    if (check) {
        int any = __syncthreads_or(bad);
        if (any && threadIdx.x == 0) atomicOr(&stp->bad_data, 1);
    }
    AT* red = (PREC == PREC_MIXED) ? (AT*)sm.redf : (AT*)sm.redd;
    AT tsum;
    block_reduce<K, AT>(acc, red, tsum);
    int64_t row = d.tile_base + tile;
    if (threadIdx.x < K) {
        if (PREC == PREC_MIXED) E.tile_part[row * KMAX + threadIdx.x] = float(tsum);
        else E.tile_part_d[row * KMAX + threadIdx.x] = double(tsum);
    }
    // ---- last arriver of the group combines the group
    __threadfence();
    __syncthreads();
    int group = tile / GROUP_TILES;
    int g0 = group * GROUP_TILES;
    int gsize = min(GROUP_TILES, d.n_tiles - g0);
    if (threadIdx.x == 0) {
        int old = atomicAdd(&E.group_cnt[d.group_base + group], 1);
        sm.flag[2] = (old == gsize - 1);
    }
    __syncthreads();
    if (!sm.flag[2]) return;
    __threadfence();
    double* gout = E.group_part + (d.group_base + group) * KMAX;
    if (PREC == PREC_MIXED)
        combine_rows<float>(E.tile_part + (d.tile_base + g0) * KMAX, gsize, K, sm.comb, sm.trf.tot);
    else
        combine_rows<double>(E.tile_part_d + (d.tile_base + g0) * KMAX, gsize, K, sm.comb, sm.trf.tot);
    if (threadIdx.x < K) gout[threadIdx.x] = sm.trf.tot[threadIdx.x];
    if (threadIdx.x == 0) E.group_cnt[d.group_base + group] = 0;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        int old = atomicAdd(&E.fit_cnt[fit], 1);
        sm.flag[3] = (old == d.n_groups - 1);
    }
    __syncthreads();
    if (!sm.flag[3]) return;
    __threadfence();
    combine_rows<double>(E.group_part + d.group_base * KMAX, d.n_groups, K, sm.comb, sm.trf.tot);
    if (threadIdx.x == 0) E.fit_cnt[fit] = 0;
    __syncthreads();
    if (threadIdx.x < 32) trf_step<PREC>(d, stp, results + fit, sm.trf, E.running);
    __syncthreads();
}

template <int PREC>
__global__ void __launch_bounds__(EVAL_THREADS) eval_round_kernel(Engine E, FitResult* results) {
    __shared__ RoundSmem sm;
    int n_items = *E.n_items;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        WorkItem wi = E.items[it];
        FitState* stp = E.state + wi.fit;
        if (threadIdx.x == 0) { sm.flag[0] = stp->run; sm.flag[1] = stp->phase; }
        __syncthreads();
        if (sm.flag[0] != RS_RUNNING) { __syncthreads(); continue; }
        // stage desc and pass constants
        {
            const int* src = (const int*)(E.desc + wi.fit);
            int* dst = (int*)&sm.desc;
            for (int k = threadIdx.x; k < (int)(sizeof(FitDesc) / 4); k += EVAL_THREADS) dst[k] = src[k];
            if (PREC == PREC_MIXED) { if (threadIdx.x < PF) sm.pf[threadIdx.x] = stp->pf[threadIdx.x]; }
            else { if (threadIdx.x < PD) sm.pd[threadIdx.x] = stp->pd[threadIdx.x]; }
        }
        __syncthreads();
        switch (sm.desc.model) {
            case 0: process_item<MGauss1D, PREC>(sm, E, results, wi.fit, wi.tile); break;
            case 1: process_item<MDexp, PREC>(sm, E, results, wi.fit, wi.tile); break;
            case 2: process_item<MGauss2D, PREC>(sm, E, results, wi.fit, wi.tile); break;
            case 3: process_item<MPoly2, PREC>(sm, E, results, wi.fit, wi.tile); break;
        }
        __syncthreads();
    }
}

// Pass constants for the first evaluation (at p0): base = trial = p0.
template <int PREC>
__global__ void init_fits_kernel(Engine E) {
    __shared__ TrfSmem S;
    int nf = E.nfits_dev ? *E.nfits_dev : 0;
    for (int f = blockIdx.x; f < nf; f += gridDim.x) {
        const FitDesc& d = E.desc[f];
        FitState* st = E.state + f;
        int l = threadIdx.x;
        if (l < 8) { S.vec[VX][l] = (l < d.n) ? st->x[l] : 0.0; S.vec[VXT][l] = S.vec[VX][l]; }
        __syncwarp();
        prep_pass<PREC>(d, st, S);
        __syncwarp();
    }
}

__global__ void round_end_kernel(Engine E, cudaGraphConditionalHandle h) {
    int r = ++(*E.rounds);
    unsigned keep = (*E.running > 0 && r < *E.max_rounds) ? 1u : 0u;
    cudaGraphSetConditional(h, keep);
}

// w = 1/sigma (FP64) for the plain path.
template <typename DT>
__global__ void stage_weights_kernel(const DT* sigma, double* w, int64_t m) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        double s = double(sigma[i]);
        w[i] = (s > 0.0 && isfinite(s)) ? 1.0 / s : NAN;
    }
}

// One scaled subproblem: eigen-decompose B, then Algorithm 1's step with Algorithm 2.
__global__ void tr_subproblem_kernel(int n, const double* B, const double* g, double Delta, double alpha0,
                                     double* p_out, double* alpha_out, double* lam_out) {
    __shared__ TrfSmem S;
    int l = threadIdx.x;
    for (int e = l; e < 64; e += 32) {
        int i = e >> 3, j = e & 7;
        double b = (i < n && j < n) ? B[i * n + j] : 0.0;
        S.A[e] = b;
        S.Ah[e] = b;
        S.V[e] = (i == j && i < n) ? 1.0 : 0.0;
    }
    __syncwarp();
    jacobi_eig(n, S.A, S.V, S.cs, S.pairs, 30);
    double lam = (l < n) ? S.A[l * 8 + l] : 0.0;
    double gl = (l < n) ? g[l] : 0.0;
    vstore(S.vec[VGH], n, gl);
    int i = l >> 2, j = l & 3;
    double acc = 0.0;
    if (i < n) {
        if (j < n) acc = S.V[j * 8 + i] * S.vec[VGH][j];
        if (j + 4 < n) acc = fma(S.V[(j + 4) * 8 + i], S.vec[VGH][j + 4], acc);
    }
    acc += __shfl_xor_sync(FULL, acc, 1);
    acc += __shfl_xor_sync(FULL, acc, 2);
    double gV = __shfl_sync(FULL, acc, (l & 7) << 2);
    if (l >= n) gV = 0.0;
    double lmax = gmax8(l < n ? lam : -INFINITY);
    bool keep = (l < n) && lmax > 0.0 && lam > lmax * (8.0 * n * EPS64);
    if (!keep) { gV = 0.0; }
    double lam_c = keep ? lam : 0.0;
    bool full_rank = __all_sync(FULL, keep || l >= n);
    double comp = (gV != 0.0) ? gV / lam_c : 0.0;
    double ptn = sqrt(gsum8(comp * comp));
    double alpha = 0.0;
    int it = 0;
    if (ptn > Delta) {
        double ghn = sqrt(gsum8(gl * gl));
        alpha = lm_parameter(lam_c, gV, ghn, Delta, alpha0, full_rank, &it);
        comp = (gV != 0.0) ? gV / (lam_c + alpha) : 0.0;
    }
    vstore(S.vec[VTMP], n, comp);
    double p = -matvec8(S.V, S.vec[VTMP], n);
    if (l < n) { p_out[l] = p; lam_out[l] = lam; }
    if (l == 0) *alpha_out = alpha;
}

// ------------------------------------------------------------------ host-side handles
void* kernel_eval_round(int prec) {
    return prec == PREC_MIXED ? (void*)eval_round_kernel<PREC_MIXED> : (void*)eval_round_kernel<PREC_FP64>;
}
void* kernel_init_fits(int prec) {
    return prec == PREC_MIXED ? (void*)init_fits_kernel<PREC_MIXED> : (void*)init_fits_kernel<PREC_FP64>;
}
void* kernel_round_end() { return (void*)round_end_kernel; }
int eval_blocks_per_sm(int prec) {
    int b = 0;
    if (prec == PREC_MIXED) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, eval_round_kernel<PREC_MIXED>, EVAL_THREADS, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, eval_round_kernel<PREC_FP64>, EVAL_THREADS, 0);
    return b;
}
cudaError_t launch_stage_weights(bool f64, const void* sigma, double* w, int64_t m, int blocks, cudaStream_t s) {
    if (f64) stage_weights_kernel<double><<<blocks, 256, 0, s>>>((const double*)sigma, w, m);
    else stage_weights_kernel<float><<<blocks, 256, 0, s>>>((const float*)sigma, w, m);
    return cudaGetLastError();
}
cudaError_t launch_tr_subproblem(int n, const double* B, const double* g, double Delta, double alpha0,
                                 double* p_out, double* alpha_out, double* lam_out, cudaStream_t s) {
    tr_subproblem_kernel<<<1, 32, 0, s>>>(n, B, g, Delta, alpha0, p_out, alpha_out, lam_out);
    return cudaGetLastError();
}

}  // namespace gbfit

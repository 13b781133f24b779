// Model registry: h(x; p) and analytic partials dh/dp for each built-in model.
//
// The paper forms the Jacobian (Section 2, Eq. jacobian) by automatic
// differentiation; this library ships a fixed registry of models with their
// partials written out, the explicit-Jacobian alternative Appendix C allows.
//
// Two evaluation forms per model:
//   plain  (FP64): value and partials at the trial point p'.
//   mixed  (FP32): value at the base point p, the difference
//                  dh = h(p') - h(p) in a cancellation-free form (no
//                  subtraction of two O(h) numbers), and the partials at p'.
//                  The actual reduction of Eq. accuracy is then accumulated as
//                  sum dr (2 r + dr), which keeps full relative accuracy when
//                  f(p) - f(p') is many orders below f (near convergence).
//   direct (FP32, packed models): value and partials at p' alone.  It serves
//                  evaluations that need no difference: a fit's first one
//                  (p' = p; the same bits as the mixed form's) and trial
//                  points whose predicted reduction is a large fraction of
//                  f, where f - f' from two FP32-evaluated costs resolves the
//                  ratio of Eq. accuracy well enough.
// Pass constants are prepared once per pass from FP64 parameters:
//   plain: pd[] (doubles) from p'.
//   mixed: pf[] (floats) from float images of p, p' and of the FP64
//          differences p' - p; location parameters also carry a lo word
//          (p = hi + lo) so that x - x0 keeps ~46 bits of x0.
#pragma once
#include "gbfit_internal.cuh"

namespace gbfit {

// E' = exp(-q_new) and dE = E' - E without cancellation, where E = exp(-q)
// and dq = q_new - q is formed without cancellation by the caller.
// |dq| <= 1/8: dE = E expm1(-dq), expm1 by its Taylor series through z^6
// (truncation below 1e-9 relative).  |dq| > 1/8: the plain difference,
// where |dE| >= 11% of max(E, E'), so it keeps ~5e-6 relative accuracy
// (those are large steps, far from the region where the actual reduction
// must be resolved below FP32 rounding of the cost).
__device__ __forceinline__ void exp_shift(float E, float q_new, float dq, float& En, float& dE) {
    En = __expf(-q_new);
    float z = -dq;
    float p = fmaf(z, 1.0f / 720.0f, 1.0f / 120.0f);
    p = fmaf(z, p, 1.0f / 24.0f);
    p = fmaf(z, p, 1.0f / 6.0f);
    p = fmaf(z, p, 0.5f);
    p = fmaf(z, p, 1.0f);
    float dEs = E * (p * z);
    dE = fabsf(z) <= 0.125f ? dEs : En - E;
}

// ---- packed FP32 (sm_100 family: one FFMA2 / FMUL2 / FADD2 instruction
// does the operation for two points).  Every packed helper below is one
// instruction except the exponentials (one MUFU ex2 per lane element).
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(bc(-1.0f), b, a); }   // exact a - b
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// exp(-q) elementwise (2^(-q log2 e))
__device__ __forceinline__ float2 expn2(float2 q) {
    float2 t = mul2(q, bc(-1.4426950408889634f));
    return make_float2(ex2_approx(t.x), ex2_approx(t.y));
}

// exp_shift for two points: E' = exp(-q_new), dE = E' - E (series in dq for
// |dq| <= 1/8, written in dq so that no negation is needed).
__device__ __forceinline__ void exp_shift2(float2 E, float2 q_new, float2 dq, float2& En, float2& dE) {
    En = expn2(q_new);
    // expm1(-u) = u (-1 + u (1/2 + u (-1/6 + u (1/24 + u (-1/120 + u / 720)))))
    float2 p = fma2(dq, bc(1.0f / 720.0f), bc(-1.0f / 120.0f));
    p = fma2(dq, p, bc(1.0f / 24.0f));
    p = fma2(dq, p, bc(-1.0f / 6.0f));
    p = fma2(dq, p, bc(0.5f));
    p = fma2(dq, p, bc(-1.0f));
    float2 dEs = mul2(E, mul2(p, dq));
    dE.x = fabsf(dq.x) <= 0.125f ? dEs.x : En.x - E.x;
    dE.y = fabsf(dq.y) <= 0.125f ? dEs.y : En.y - E.y;
}

// ---- robust losses (Section 5 names loss functions without stating them;
// reading R14): rho(z), rho'(z), rho''(z) with z = (r / C)^2, and the change
// rho(z + dz) - rho(z) written without cancellation (dz is formed from the
// residual change as in the cancellation-free actual reduction).
template <typename T>
__device__ __forceinline__ void loss_rho(int loss, T z, T& rho, T& r1, T& r2) {
    switch (loss) {
        case LOSS_SOFT_L1: {
            T t = T(1) + z, st = sqrt(t), it = T(1) / st;
            rho = T(2) * z / (st + T(1)); r1 = it; r2 = T(-0.5) * it / t;
            break;
        }
        case LOSS_HUBER:
            if (z <= T(1)) { rho = z; r1 = T(1); r2 = T(0); }
            else { T sz = sqrt(z); rho = T(2) * sz - T(1); r1 = T(1) / sz; r2 = T(-0.5) * r1 / z; }
            break;
        case LOSS_CAUCHY: {
            T it = T(1) / (T(1) + z);
            rho = log1p(z); r1 = it; r2 = -it * it;
            break;
        }
        case LOSS_ARCTAN: {
            T it = T(1) / (T(1) + z * z);
            rho = atan(z); r1 = it; r2 = T(-2) * z * it * it;
            break;
        }
        default: rho = z; r1 = T(1); r2 = T(0); break;
    }
}

template <typename T>
__device__ __forceinline__ T loss_drho(int loss, T z, T dz) {
    const T zn = z + dz;
    switch (loss) {
        case LOSS_SOFT_L1: return T(2) * dz / (sqrt(T(1) + zn) + sqrt(T(1) + z));
        case LOSS_HUBER:
            if (z <= T(1) && zn <= T(1)) return dz;
            if (z > T(1) && zn > T(1)) return T(2) * dz / (sqrt(zn) + sqrt(z));
            return (zn <= T(1) ? zn : T(2) * sqrt(zn) - T(1)) - (z <= T(1) ? z : T(2) * sqrt(z) - T(1));
        case LOSS_CAUCHY: return log1p(dz / (T(1) + z));
        case LOSS_ARCTAN: return atan(dz / (T(1) + z * zn));
        default: return dz;
    }
}

// Float images of the FP64 parameters handed to the mixed prep.
struct MixedParams {
    float x[NMAX];    // base p (rounded)
    float xlo[NMAX];  // p - double(x) (rounded)
    float xt[NMAX];   // trial p' (rounded)
    float dx[NMAX];   // p' - p (FP64 difference, rounded)
};

// ------------------------------------------------------------------ gauss1d
// h = A exp(-(x-mu)^2/(2 s^2)) + c,  p = (A, mu, s, c)
struct MGauss1D {
    static constexpr int N = 4;
    static constexpr int DIM = 1;               // coordinate dimensions
    static constexpr bool WARP_PREP = false;
    __device__ static void prep_plain(const double* p, double* pd) {
        double s = p[2];
        double is2 = 1.0 / (s * s);
        pd[0] = p[0]; pd[1] = p[1]; pd[2] = 0.5 * is2; pd[3] = p[3];
        pd[4] = p[0] * is2; pd[5] = p[0] * is2 / s;
    }
    __device__ static void eval_plain(const double* pd, double X, double, double& h, double* J) {
        double d = X - pd[1];
        double E = exp(-pd[2] * d * d);
        h = fma(pd[0], E, pd[3]);
        J[0] = E; J[1] = pd[4] * E * d; J[2] = pd[5] * E * d * d; J[3] = 1.0;
    }
    __device__ static void prep_mixed(const MixedParams& P, float* pf) {
        float s = P.x[2], st = P.xt[2], ds = P.dx[2];
        float k = 0.5f / (s * s), kt = 0.5f / (st * st);
        pf[0] = P.x[0]; pf[1] = P.x[1]; pf[2] = P.xlo[1]; pf[3] = k; pf[4] = P.x[3];
        pf[5] = P.dx[1];                                   // dmu
        pf[6] = -ds * (st + s) * k * kt * 2.0f;            // k' - k = -(s'-s)(s'+s)/(2 s^2 s'^2)
        pf[7] = kt; pf[8] = P.xt[0]; pf[9] = P.dx[0]; pf[10] = P.dx[3];
        pf[11] = P.xt[0] * 2.0f * kt;                      // A'/s'^2
        pf[12] = P.xt[0] * 2.0f * kt / st;                 // A'/s'^3
        pf[13] = P.xt[3];                                  // c'
    }
    __device__ static void eval_mixed(const float* pf, float X, float, float& hb, float& dh, float* J) {
        float d = (X - pf[1]) - pf[2];
        float q = pf[3] * d * d;
        float E = __expf(-q);
        hb = fmaf(pf[0], E, pf[4]);
        float dn = d - pf[5];
        float dq = fmaf(pf[7] * (-pf[5]), dn + d, pf[6] * d * d);
        float En, dE;
        exp_shift(E, pf[7] * dn * dn, dq, En, dE);
        dh = fmaf(pf[0], dE, fmaf(pf[9], En, pf[10]));
        J[0] = En; J[1] = pf[11] * En * dn; J[2] = pf[12] * En * dn * dn; J[3] = 1.0f;
    }
    // the same for two points at once (packed FP32); PACK 1: packed
    // accumulators too (few slots), 2: scalar accumulators (many slots)
    static constexpr int PACK = 1;
    __device__ static void eval_mixed2(const float* pf, float2 X, float2, float2& hb, float2& dh, float2* J) {
        float2 d = sub2(sub2(X, bc(pf[1])), bc(pf[2]));
        float2 dd = mul2(d, d);
        float2 E = expn2(mul2(bc(pf[3]), dd));
        hb = fma2(bc(pf[0]), E, bc(pf[4]));
        float2 dn = sub2(d, bc(pf[5]));
        float2 dq = fma2(bc(pf[7] * (-pf[5])), add2(dn, d), mul2(bc(pf[6]), dd));
        float2 En, dE;
        exp_shift2(E, mul2(bc(pf[7]), mul2(dn, dn)), dq, En, dE);
        dh = fma2(bc(pf[0]), dE, fma2(bc(pf[9]), En, bc(pf[10])));
        float2 t = mul2(En, dn);
        J[0] = En; J[1] = mul2(bc(pf[11]), t); J[2] = mul2(bc(pf[12]), mul2(t, dn)); J[3] = bc(1.0f);
    }
    // value and partials at the trial point alone (direct form, no
    // difference): the same operations as the trial side of eval_mixed2, so
    // that at a first evaluation (trial = base) both forms give the same bits
    __device__ static void eval_direct2(const float* pf, float2 X, float2, float2& h, float2* J) {
        float2 dn = sub2(sub2(sub2(X, bc(pf[1])), bc(pf[2])), bc(pf[5]));
        float2 En = expn2(mul2(bc(pf[7]), mul2(dn, dn)));
        h = fma2(bc(pf[8]), En, bc(pf[13]));
        float2 t = mul2(En, dn);
        J[0] = En; J[1] = mul2(bc(pf[11]), t); J[2] = mul2(bc(pf[12]), mul2(t, dn)); J[3] = bc(1.0f);
    }
};

// ------------------------------------------------------------------ dexp
// h = a1 exp(-x/t1) + a2 exp(-x/t2) + c,  p = (a1, t1, a2, t2, c)
struct MDexp {
    static constexpr int N = 5;
    static constexpr int DIM = 1;               // coordinate dimensions
    static constexpr bool WARP_PREP = false;
    __device__ static void prep_plain(const double* p, double* pd) {
        double k1 = 1.0 / p[1], k2 = 1.0 / p[3];
        pd[0] = p[0]; pd[1] = k1; pd[2] = p[2]; pd[3] = k2; pd[4] = p[4];
        pd[5] = p[0] * k1 * k1; pd[6] = p[2] * k2 * k2;
    }
    __device__ static void eval_plain(const double* pd, double X, double, double& h, double* J) {
        double e1 = exp(-X * pd[1]), e2 = exp(-X * pd[3]);
        h = pd[0] * e1 + pd[2] * e2 + pd[4];
        J[0] = e1; J[1] = pd[5] * X * e1; J[2] = e2; J[3] = pd[6] * X * e2; J[4] = 1.0;
    }
    __device__ static void prep_mixed(const MixedParams& P, float* pf) {
        float t1 = P.x[1], t2 = P.x[3], t1n = P.xt[1], t2n = P.xt[3];
        float k1 = 1.0f / t1, k2 = 1.0f / t2, k1n = 1.0f / t1n, k2n = 1.0f / t2n;
        pf[0] = P.x[0]; pf[1] = k1; pf[2] = P.x[2]; pf[3] = k2; pf[4] = P.x[4];
        pf[5] = -P.dx[1] * k1 * k1n;                        // 1/t1' - 1/t1
        pf[6] = -P.dx[3] * k2 * k2n;
        pf[7] = P.xt[0]; pf[8] = P.xt[2];
        pf[9] = P.dx[0]; pf[10] = P.dx[2]; pf[11] = P.dx[4];
        pf[12] = P.xt[0] * k1n * k1n; pf[13] = P.xt[2] * k2n * k2n;
        pf[14] = k1n; pf[15] = k2n;
        pf[16] = P.xt[4];                                   // c'
    }
    __device__ static void eval_mixed(const float* pf, float X, float, float& hb, float& dh, float* J) {
        float q1 = X * pf[1], q2 = X * pf[3];
        float e1 = __expf(-q1), e2 = __expf(-q2);
        hb = fmaf(pf[0], e1, fmaf(pf[2], e2, pf[4]));
        float e1n, de1, e2n, de2;
        exp_shift(e1, X * pf[14], X * pf[5], e1n, de1);
        exp_shift(e2, X * pf[15], X * pf[6], e2n, de2);
        dh = fmaf(pf[0], de1, fmaf(pf[9], e1n, fmaf(pf[2], de2, fmaf(pf[10], e2n, pf[11]))));
        J[0] = e1n; J[1] = pf[12] * X * e1n; J[2] = e2n; J[3] = pf[13] * X * e2n; J[4] = 1.0f;
    }
    static constexpr int PACK = 1;
    __device__ static void eval_mixed2(const float* pf, float2 X, float2, float2& hb, float2& dh, float2* J) {
        float2 e1 = expn2(mul2(X, bc(pf[1]))), e2 = expn2(mul2(X, bc(pf[3])));
        hb = fma2(bc(pf[0]), e1, fma2(bc(pf[2]), e2, bc(pf[4])));
        float2 e1n, de1, e2n, de2;
        exp_shift2(e1, mul2(X, bc(pf[14])), mul2(X, bc(pf[5])), e1n, de1);
        exp_shift2(e2, mul2(X, bc(pf[15])), mul2(X, bc(pf[6])), e2n, de2);
        dh = fma2(bc(pf[0]), de1, fma2(bc(pf[9]), e1n, fma2(bc(pf[2]), de2, fma2(bc(pf[10]), e2n, bc(pf[11])))));
        J[0] = e1n; J[1] = mul2(bc(pf[12]), mul2(X, e1n)); J[2] = e2n; J[3] = mul2(bc(pf[13]), mul2(X, e2n));
        J[4] = bc(1.0f);
    }
    // direct form at the trial point (the trial side of eval_mixed2)
    __device__ static void eval_direct2(const float* pf, float2 X, float2, float2& h, float2* J) {
        float2 e1n = expn2(mul2(X, bc(pf[14]))), e2n = expn2(mul2(X, bc(pf[15])));
        h = fma2(bc(pf[7]), e1n, fma2(bc(pf[8]), e2n, bc(pf[16])));
        J[0] = e1n; J[1] = mul2(bc(pf[12]), mul2(X, e1n)); J[2] = e2n; J[3] = mul2(bc(pf[13]), mul2(X, e2n));
        J[4] = bc(1.0f);
    }
};

// ------------------------------------------------------------------ gauss2d
// u =  (X-x0) cos th + (Y-y0) sin th,  v = -(X-x0) sin th + (Y-y0) cos th
// h = A exp(-u^2/(2 sx^2) - v^2/(2 sy^2)) + c,  p = (A, x0, y0, sx, sy, th, c)
struct MGauss2D {
    static constexpr int N = 7;
    static constexpr int DIM = 2;               // coordinate dimensions
    static constexpr bool WARP_PREP = true;
    static constexpr int PACK = 2;
    __device__ static void prep_plain(const double* p, double* pd) {
        double s, c;
        sincos(p[5], &s, &c);
        double ka = 0.5 / (p[3] * p[3]), kb = 0.5 / (p[4] * p[4]);
        pd[0] = p[0]; pd[1] = p[1]; pd[2] = p[2]; pd[3] = c; pd[4] = s;
        pd[5] = ka; pd[6] = kb; pd[7] = p[6];
        pd[8] = 2.0 * ka / p[3]; pd[9] = 2.0 * kb / p[4];
    }
    __device__ static void eval_plain(const double* pd, double X, double Y, double& h, double* J) {
        double dx = X - pd[1], dy = Y - pd[2];
        double u = dx * pd[3] + dy * pd[4];
        double v = -dx * pd[4] + dy * pd[3];
        double E = exp(-(pd[5] * u * u + pd[6] * v * v));
        double Q = pd[0] * E;
        h = Q + pd[7];
        double au = 2.0 * pd[5] * u, bv = 2.0 * pd[6] * v;
        J[0] = E;
        J[1] = Q * (au * pd[3] - bv * pd[4]);
        J[2] = Q * (au * pd[4] + bv * pd[3]);
        J[3] = Q * pd[8] * u * u;
        J[4] = Q * pd[9] * v * v;
        J[5] = Q * 2.0 * u * v * (pd[6] - pd[5]);
        J[6] = 1.0;
    }
    __device__ static void prep_mixed(const MixedParams& P, float* pf) {
        float th = P.x[5], tht = P.xt[5], dth = P.dx[5];
        float s, c, st, ct;
        sincosf(th, &s, &c);
        sincosf(tht, &st, &ct);
        float mid = th + 0.5f * dth;
        float sh = sinf(0.5f * dth);
        float dc = -2.0f * sinf(mid) * sh;                  // cos th' - cos th
        float ds = 2.0f * cosf(mid) * sh;                   // sin th' - sin th
        float sx = P.x[3], sy = P.x[4], sxt = P.xt[3], syt = P.xt[4];
        float ka = 0.5f / (sx * sx), kb = 0.5f / (sy * sy);
        float kat = 0.5f / (sxt * sxt), kbt = 0.5f / (syt * syt);
        float dx0 = P.dx[1], dy0 = P.dx[2];
        pf[0] = P.x[0]; pf[1] = P.x[1]; pf[2] = P.xlo[1]; pf[3] = P.x[2]; pf[4] = P.xlo[2];
        pf[5] = c; pf[6] = s; pf[7] = ka; pf[8] = kb; pf[9] = P.x[6];
        pf[10] = dc; pf[11] = ds;
        pf[12] = -dx0 * ct - dy0 * st;                      // ku
        pf[13] = dx0 * st - dy0 * ct;                       // kv
        pf[14] = kat; pf[15] = kbt;
        pf[16] = -P.dx[3] * (sxt + sx) * 2.0f * ka * kat;   // ka' - ka
        pf[17] = -P.dx[4] * (syt + sy) * 2.0f * kb * kbt;   // kb' - kb
        pf[18] = P.xt[0]; pf[19] = P.dx[0]; pf[20] = P.dx[6];
        pf[21] = ct; pf[22] = st;
        pf[23] = 2.0f * kat / sxt; pf[24] = 2.0f * kbt / syt;
        pf[25] = P.xt[6];                                   // c'
    }
    // prep_mixed on a whole warp: the four angles' sin/cos and the four
    // widths' 1/(2 w^2) (and 2 k / w) in lanes 0-3 at once, the rest on
    // lane 0.  tmp: 16 floats of shared memory.
    __device__ static void prep_mixed_warp(const MixedParams& P, float* pf, float* tmp) {
        const int l = threadIdx.x & 31;
        const int q = l & 3;
        const float th = P.x[5], dth = P.dx[5];
        float ang = q == 0 ? th : q == 1 ? P.xt[5] : q == 2 ? 0.5f * dth : th + 0.5f * dth;
        float sn, cs;
        sincosf(ang, &sn, &cs);
        float w = q == 0 ? P.x[3] : q == 1 ? P.x[4] : q == 2 ? P.xt[3] : P.xt[4];
        float kk = 0.5f / (w * w);
        float rk = 2.0f * kk / w;
        if (l < 4) { tmp[l] = sn; tmp[4 + l] = cs; tmp[8 + l] = kk; tmp[12 + l] = rk; }
        __syncwarp();
        if (l == 0) {
            float s = tmp[0], c = tmp[4], st = tmp[1], ct = tmp[5], sh = tmp[2];
            float dc = -2.0f * tmp[3] * sh, ds = 2.0f * tmp[7] * sh;
            float sx = P.x[3], sy = P.x[4], sxt = P.xt[3], syt = P.xt[4];
            float ka = tmp[8], kb = tmp[9], kat = tmp[10], kbt = tmp[11];
            float dx0 = P.dx[1], dy0 = P.dx[2];
            pf[0] = P.x[0]; pf[1] = P.x[1]; pf[2] = P.xlo[1]; pf[3] = P.x[2]; pf[4] = P.xlo[2];
            pf[5] = c; pf[6] = s; pf[7] = ka; pf[8] = kb; pf[9] = P.x[6];
            pf[10] = dc; pf[11] = ds;
            pf[12] = -dx0 * ct - dy0 * st;
            pf[13] = dx0 * st - dy0 * ct;
            pf[14] = kat; pf[15] = kbt;
            pf[16] = -P.dx[3] * (sxt + sx) * 2.0f * ka * kat;
            pf[17] = -P.dx[4] * (syt + sy) * 2.0f * kb * kbt;
            pf[18] = P.xt[0]; pf[19] = P.dx[0]; pf[20] = P.dx[6];
            pf[21] = ct; pf[22] = st;
            pf[23] = tmp[14]; pf[24] = tmp[15];
            pf[25] = P.xt[6];
        }
        __syncwarp();
    }
    __device__ static void eval_mixed(const float* pf, float X, float Y, float& hb, float& dh, float* J) {
        float dx = (X - pf[1]) - pf[2];
        float dy = (Y - pf[3]) - pf[4];
        float u = fmaf(dx, pf[5], dy * pf[6]);
        float v = fmaf(dy, pf[5], -dx * pf[6]);
        float q = fmaf(pf[7] * u, u, pf[8] * v * v);
        float E = __expf(-q);
        hb = fmaf(pf[0], E, pf[9]);
        float du = fmaf(dx, pf[10], fmaf(dy, pf[11], pf[12]));
        float dv = fmaf(dy, pf[10], fmaf(-dx, pf[11], pf[13]));
        float un = u + du, vn = v + dv;
        float dq = fmaf(pf[14] * du, un + u, fmaf(pf[16] * u, u, fmaf(pf[15] * dv, vn + v, pf[17] * v * v)));
        float qn = fmaf(pf[14] * un, un, pf[15] * vn * vn);
        float En, dE;
        exp_shift(E, qn, dq, En, dE);
        dh = fmaf(pf[0], dE, fmaf(pf[19], En, pf[20]));
        float Q = pf[18] * En;
        float au = 2.0f * pf[14] * un, bv = 2.0f * pf[15] * vn;
        J[0] = En;
        J[1] = Q * fmaf(au, pf[21], -bv * pf[22]);
        J[2] = Q * fmaf(au, pf[22], bv * pf[21]);
        J[3] = Q * pf[23] * un * un;
        J[4] = Q * pf[24] * vn * vn;
        J[5] = Q * 2.0f * un * vn * (pf[15] - pf[14]);
        J[6] = 1.0f;
    }
    __device__ static void eval_mixed2(const float* pf, float2 X, float2 Y, float2& hb, float2& dh, float2* J) {
        float2 dx = sub2(sub2(X, bc(pf[1])), bc(pf[2]));
        float2 dy = sub2(sub2(Y, bc(pf[3])), bc(pf[4]));
        float2 u = fma2(dx, bc(pf[5]), mul2(dy, bc(pf[6])));
        float2 v = fma2(dy, bc(pf[5]), mul2(dx, bc(-pf[6])));
        float2 q = fma2(mul2(bc(pf[7]), u), u, mul2(mul2(bc(pf[8]), v), v));
        float2 E = expn2(q);
        hb = fma2(bc(pf[0]), E, bc(pf[9]));
        float2 du = fma2(dx, bc(pf[10]), fma2(dy, bc(pf[11]), bc(pf[12])));
        float2 dv = fma2(dy, bc(pf[10]), fma2(dx, bc(-pf[11]), bc(pf[13])));
        float2 un = add2(u, du), vn = add2(v, dv);
        float2 dq = fma2(mul2(bc(pf[14]), du), add2(un, u),
                         fma2(mul2(bc(pf[16]), u), u, fma2(mul2(bc(pf[15]), dv), add2(vn, v), mul2(mul2(bc(pf[17]), v), v))));
        float2 qn = fma2(mul2(bc(pf[14]), un), un, mul2(mul2(bc(pf[15]), vn), vn));
        float2 En, dE;
        exp_shift2(E, qn, dq, En, dE);
        dh = fma2(bc(pf[0]), dE, fma2(bc(pf[19]), En, bc(pf[20])));
        float2 Q = mul2(bc(pf[18]), En);
        float2 au = mul2(bc(2.0f * pf[14]), un), bv = mul2(bc(2.0f * pf[15]), vn);
        J[0] = En;
        J[1] = mul2(Q, fma2(au, bc(pf[21]), mul2(bv, bc(-pf[22]))));
        J[2] = mul2(Q, fma2(au, bc(pf[22]), mul2(bv, bc(pf[21]))));
        J[3] = mul2(mul2(mul2(Q, bc(pf[23])), un), un);
        J[4] = mul2(mul2(mul2(Q, bc(pf[24])), vn), vn);
        J[5] = mul2(mul2(mul2(Q, bc(2.0f * (pf[15] - pf[14]))), un), vn);
        J[6] = bc(1.0f);
    }
    // direct form at the trial point: u' = (X - x0') cos th' + (Y - y0') sin th'
    // and v' from the base offsets and the shifts ku, kv (at a first
    // evaluation ku = kv = 0 and th' = th: the bits of eval_mixed2's u, v)
    __device__ static void eval_direct2(const float* pf, float2 X, float2 Y, float2& h, float2* J) {
        float2 dx = sub2(sub2(X, bc(pf[1])), bc(pf[2]));
        float2 dy = sub2(sub2(Y, bc(pf[3])), bc(pf[4]));
        float2 un = fma2(dx, bc(pf[21]), fma2(dy, bc(pf[22]), bc(pf[12])));
        float2 vn = fma2(dy, bc(pf[21]), fma2(dx, bc(-pf[22]), bc(pf[13])));
        float2 qn = fma2(mul2(bc(pf[14]), un), un, mul2(mul2(bc(pf[15]), vn), vn));
        float2 En = expn2(qn);
        h = fma2(bc(pf[18]), En, bc(pf[25]));
        float2 Q = mul2(bc(pf[18]), En);
        float2 au = mul2(bc(2.0f * pf[14]), un), bv = mul2(bc(2.0f * pf[15]), vn);
        J[0] = En;
        J[1] = mul2(Q, fma2(au, bc(pf[21]), mul2(bv, bc(-pf[22]))));
        J[2] = mul2(Q, fma2(au, bc(pf[22]), mul2(bv, bc(pf[21]))));
        J[3] = mul2(mul2(mul2(Q, bc(pf[23])), un), un);
        J[4] = mul2(mul2(mul2(Q, bc(pf[24])), vn), vn);
        J[5] = mul2(mul2(mul2(Q, bc(2.0f * (pf[15] - pf[14]))), un), vn);
        J[6] = bc(1.0f);
    }
};

// ------------------------------------------------------------------ poly2
// h = p0 + p1 x + p2 x^2  (linear in p)
struct MPoly2 {
    static constexpr int N = 3;
    static constexpr int DIM = 1;               // coordinate dimensions
    static constexpr bool WARP_PREP = false;
    static constexpr int PACK = 0;
    __device__ static void eval_mixed2(const float*, float2, float2, float2&, float2&, float2*) {}
    __device__ static void eval_direct2(const float*, float2, float2, float2&, float2*) {}
    __device__ static void prep_plain(const double* p, double* pd) { pd[0] = p[0]; pd[1] = p[1]; pd[2] = p[2]; }
    __device__ static void eval_plain(const double* pd, double X, double, double& h, double* J) {
        h = fma(fma(pd[2], X, pd[1]), X, pd[0]);
        J[0] = 1.0; J[1] = X; J[2] = X * X;
    }
    __device__ static void prep_mixed(const MixedParams& P, float* pf) {
        pf[0] = P.x[0]; pf[1] = P.x[1]; pf[2] = P.x[2];
        pf[3] = P.dx[0]; pf[4] = P.dx[1]; pf[5] = P.dx[2];
    }
    __device__ static void eval_mixed(const float* pf, float X, float, float& hb, float& dh, float* J) {
        hb = fmaf(fmaf(pf[2], X, pf[1]), X, pf[0]);
        dh = fmaf(fmaf(pf[5], X, pf[4]), X, pf[3]);
        J[0] = 1.0f; J[1] = X; J[2] = X * X;
    }
};

__host__ __device__ inline int model_nparams(int model) {
    switch (model) {
        case 0: return MGauss1D::N;
        case 1: return MDexp::N;
        case 2: return MGauss2D::N;
        case 3: return MPoly2::N;
    }
    return 0;
}
__host__ __device__ inline int model_xdims(int model) { return model == 2 ? 2 : 1; }

// Mixed pass constants of model M, called by a whole warp (models with a
// warp-parallel prep use all lanes, the others lane 0).  tmp: 16 floats.
template <class M>
__device__ __forceinline__ void prep_mixed_model(const MixedParams& P, float* pf, float* tmp) {
    if constexpr (M::WARP_PREP) M::prep_mixed_warp(P, pf, tmp);
    else if ((threadIdx.x & 31) == 0) M::prep_mixed(P, pf);
}

// A model set: the kernels are instantiated once per set and reach a fit's
// model through dispatch(id, f), which calls f with a value of the model's
// type.  The built-in registry is one set; a user-defined model compiled at
// run time is a set of one.
struct BuiltinModels {
    template <class F>
    __device__ __forceinline__ static void dispatch(int model, F&& f) {
        switch (model) {
            case 0: f(MGauss1D{}); break;
            case 1: f(MDexp{}); break;
            case 2: f(MGauss2D{}); break;
            case 3: f(MPoly2{}); break;
        }
    }
};

}  // namespace gbfit

// User-defined models: the fit function h(x; p) supplied as source code and
// compiled at run time (NVRTC) into the same round kernels as the built-in
// registry.
//
// The paper lets the user write h in JAX and forms the Jacobian by automatic
// differentiation (Section 2, Eq. jacobian; Section 3 on autodiff).  Here the
// user writes h once as a template over the number type, and the kernels
// evaluate it with forward-mode dual numbers:
//
//   plain (FP64)  DualD<N>: value and the n partials at the trial point p'.
//   mixed (FP32)  DiffF<N>: value at the base point p, the difference
//                 h(p') - h(p) propagated through every operation without
//                 subtracting two nearly equal numbers (the mixed evaluation
//                 form of the built-in models, made generic), and the n
//                 partials at p'.
//
// Rules of the difference propagation, for intermediate a with base value a,
// difference da (a' = a + da):
//   a +- b:  da +- db
//   a * b:   a db + da b'                (= a' b' - a b exactly)
//   a / b:   (da b - a db) / (b b')
//   exp a:   exp(a) expm1(da)
//   log a:   log1p(da / a)
//   sqrt a:  da / (sqrt a + sqrt a')
//   a^k:     a^k expm1(k log1p(da / a))  (a > 0)
//   sin a:   2 cos(a + da/2) sin(da/2);  cos a: -2 sin(a + da/2) sin(da/2)
//   tanh a:  sinh(da) / (cosh a cosh a')
//   atan a:  atan(da / (1 + a a'))
// Each keeps the difference to a few FP32 roundings of itself, however small
// it is against the values.  The base point itself is p rounded to FP32 plus
// a first-order correction lo carried alongside (each parameter's rounding
// error p - float(p), propagated with the partials), so that the residual at
// p is not off by the parameters' rounding (which, near convergence, exceeds
// the steps themselves).
//
// The user source must define, at namespace scope,
//     template <class T, class S> __device__ T model(const T* p, S x, S x2);
// with p the n parameters, x the coordinate (x2 the second coordinate of a
// 2D model, 0 for 1D) as a plain number of type S (float or double).  It may
// use + - * / with T and plain numbers, and exp, log, sqrt, pow(T, number),
// sin, cos, tanh, atan, square.  Smooth models only: a branch on a parameter
// would take different sides at p and p'.
#pragma once
#include "models.cuh"

namespace gbfit {
namespace ad {

template <bool B, class T = void> struct enable_if {};
template <class T> struct enable_if<true, T> { using type = T; };
template <class S> struct is_plain { static constexpr bool value = false; };
template <> struct is_plain<int> { static constexpr bool value = true; };
template <> struct is_plain<long long> { static constexpr bool value = true; };
template <> struct is_plain<unsigned> { static constexpr bool value = true; };
template <> struct is_plain<float> { static constexpr bool value = true; };
template <> struct is_plain<double> { static constexpr bool value = true; };
#define GBFIT_IF_PLAIN(S, R) typename enable_if<is_plain<S>::value, R>::type

// ------------------------------------------------------------------ FP64 dual number
template <int N>
struct DualD {
    double v;
    double g[N];
};
template <int N>
__device__ __forceinline__ DualD<N> scaled(const DualD<N>& a, double v, double k) {
    DualD<N> r;
    r.v = v;
#pragma unroll
    for (int j = 0; j < N; ++j) r.g[j] = k * a.g[j];
    return r;
}
template <int N>
__device__ __forceinline__ DualD<N> operator+(const DualD<N>& a, const DualD<N>& b) {
    DualD<N> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int j = 0; j < N; ++j) r.g[j] = a.g[j] + b.g[j];
    return r;
}
template <int N>
__device__ __forceinline__ DualD<N> operator-(const DualD<N>& a, const DualD<N>& b) {
    DualD<N> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int j = 0; j < N; ++j) r.g[j] = a.g[j] - b.g[j];
    return r;
}
template <int N>
__device__ __forceinline__ DualD<N> operator-(const DualD<N>& a) { return scaled(a, -a.v, -1.0); }
template <int N>
__device__ __forceinline__ DualD<N> operator*(const DualD<N>& a, const DualD<N>& b) {
    DualD<N> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int j = 0; j < N; ++j) r.g[j] = fma(a.v, b.g[j], b.v * a.g[j]);
    return r;
}
template <int N>
__device__ __forceinline__ DualD<N> operator/(const DualD<N>& a, const DualD<N>& b) {
    DualD<N> r;
    const double ib = 1.0 / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int j = 0; j < N; ++j) r.g[j] = (a.g[j] - r.v * b.g[j]) * ib;
    return r;
}
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DualD<N>) operator+(const DualD<N>& a, S s) { DualD<N> r = a; r.v += double(s); return r; }
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DualD<N>) operator+(S s, const DualD<N>& a) { return a + s; }
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DualD<N>) operator-(const DualD<N>& a, S s) { DualD<N> r = a; r.v -= double(s); return r; }
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DualD<N>) operator-(S s, const DualD<N>& a) { return scaled(a, double(s) - a.v, -1.0); }
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DualD<N>) operator*(const DualD<N>& a, S s) { return scaled(a, a.v * double(s), double(s)); }
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DualD<N>) operator*(S s, const DualD<N>& a) { return a * s; }
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DualD<N>) operator/(const DualD<N>& a, S s) {
    const double is = 1.0 / double(s);
    return scaled(a, a.v * is, is);
}
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DualD<N>) operator/(S s, const DualD<N>& a) {
    const double q = double(s) / a.v;
    return scaled(a, q, -q / a.v);
}
template <int N>
__device__ __forceinline__ DualD<N> exp(const DualD<N>& a) { const double e = ::exp(a.v); return scaled(a, e, e); }
template <int N>
__device__ __forceinline__ DualD<N> log(const DualD<N>& a) { return scaled(a, ::log(a.v), 1.0 / a.v); }
template <int N>
__device__ __forceinline__ DualD<N> sqrt(const DualD<N>& a) { const double s = ::sqrt(a.v); return scaled(a, s, 0.5 / s); }
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DualD<N>) pow(const DualD<N>& a, S k) {
    const double kk = double(k), v = ::pow(a.v, kk);
    return scaled(a, v, kk * ::pow(a.v, kk - 1.0));
}
template <int N>
__device__ __forceinline__ DualD<N> sin(const DualD<N>& a) { return scaled(a, ::sin(a.v), ::cos(a.v)); }
template <int N>
__device__ __forceinline__ DualD<N> cos(const DualD<N>& a) { return scaled(a, ::cos(a.v), -::sin(a.v)); }
template <int N>
__device__ __forceinline__ DualD<N> tanh(const DualD<N>& a) { const double t = ::tanh(a.v); return scaled(a, t, 1.0 - t * t); }
template <int N>
__device__ __forceinline__ DualD<N> atan(const DualD<N>& a) { return scaled(a, ::atan(a.v), 1.0 / (1.0 + a.v * a.v)); }
template <int N>
__device__ __forceinline__ DualD<N> square(const DualD<N>& a) { return scaled(a, a.v * a.v, 2.0 * a.v); }

// ------------------------------------------------------------------ FP32 difference-dual number
template <int N>
struct DiffF {
    float v;      // value at the FP32-rounded base point
    float lo;     // first-order correction for the parameters' rounding: value at p = v + lo
    float d;      // value at p' minus value at p
    float g[N];   // partials at p'
};
template <int N>
__device__ __forceinline__ DiffF<N> chain(const DiffF<N>& a, float v, float d, float k) {
    DiffF<N> r;
    r.v = v;
    r.lo = k * a.lo;
    r.d = d;
#pragma unroll
    for (int j = 0; j < N; ++j) r.g[j] = k * a.g[j];
    return r;
}
template <int N>
__device__ __forceinline__ DiffF<N> operator+(const DiffF<N>& a, const DiffF<N>& b) {
    DiffF<N> r;
    r.v = a.v + b.v;
    r.lo = a.lo + b.lo;
    r.d = a.d + b.d;
#pragma unroll
    for (int j = 0; j < N; ++j) r.g[j] = a.g[j] + b.g[j];
    return r;
}
template <int N>
__device__ __forceinline__ DiffF<N> operator-(const DiffF<N>& a, const DiffF<N>& b) {
    DiffF<N> r;
    r.v = a.v - b.v;
    r.lo = a.lo - b.lo;
    r.d = a.d - b.d;
#pragma unroll
    for (int j = 0; j < N; ++j) r.g[j] = a.g[j] - b.g[j];
    return r;
}
template <int N>
__device__ __forceinline__ DiffF<N> operator-(const DiffF<N>& a) { return chain(a, -a.v, -a.d, -1.0f); }
template <int N>
__device__ __forceinline__ DiffF<N> operator*(const DiffF<N>& a, const DiffF<N>& b) {
    DiffF<N> r;
    const float at = a.v + a.d, bt = b.v + b.d;
    r.v = a.v * b.v;
    r.lo = fmaf(at, b.lo, bt * a.lo);
    r.d = fmaf(a.v, b.d, a.d * bt);
#pragma unroll
    for (int j = 0; j < N; ++j) r.g[j] = fmaf(at, b.g[j], bt * a.g[j]);
    return r;
}
template <int N>
__device__ __forceinline__ DiffF<N> operator/(const DiffF<N>& a, const DiffF<N>& b) {
    DiffF<N> r;
    const float bt = b.v + b.d, ibt = 1.0f / bt;
    r.v = a.v / b.v;
    r.d = fmaf(a.d, b.v, -a.v * b.d) / (b.v * bt);
    const float qt = (a.v + a.d) * ibt;
    r.lo = fmaf(-qt, b.lo, a.lo) * ibt;
#pragma unroll
    for (int j = 0; j < N; ++j) r.g[j] = fmaf(-qt, b.g[j], a.g[j]) * ibt;
    return r;
}
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DiffF<N>) operator+(const DiffF<N>& a, S s) { DiffF<N> r = a; r.v += float(s); return r; }
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DiffF<N>) operator+(S s, const DiffF<N>& a) { return a + s; }
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DiffF<N>) operator-(const DiffF<N>& a, S s) { DiffF<N> r = a; r.v -= float(s); return r; }
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DiffF<N>) operator-(S s, const DiffF<N>& a) { return chain(a, float(s) - a.v, -a.d, -1.0f); }
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DiffF<N>) operator*(const DiffF<N>& a, S s) {
    const float k = float(s);
    return chain(a, a.v * k, a.d * k, k);
}
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DiffF<N>) operator*(S s, const DiffF<N>& a) { return a * s; }
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DiffF<N>) operator/(const DiffF<N>& a, S s) {
    const float k = float(s);
    return chain(a, a.v / k, a.d / k, 1.0f / k);
}
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DiffF<N>) operator/(S s, const DiffF<N>& a) {
    const float k = float(s), at = a.v + a.d, qt = k / at;
    return chain(a, k / a.v, -k * a.d / (a.v * at), -qt / at);
}
template <int N>
__device__ __forceinline__ DiffF<N> exp(const DiffF<N>& a) {
    const float e = expf(a.v), de = e * expm1f(a.d);
    return chain(a, e, de, e + de);
}
template <int N>
__device__ __forceinline__ DiffF<N> log(const DiffF<N>& a) {
    return chain(a, logf(a.v), log1pf(a.d / a.v), 1.0f / (a.v + a.d));
}
template <int N>
__device__ __forceinline__ DiffF<N> sqrt(const DiffF<N>& a) {
    const float s = sqrtf(a.v), st = sqrtf(a.v + a.d);
    return chain(a, s, a.d / (s + st), 0.5f / st);
}
template <int N, class S>
__device__ __forceinline__ GBFIT_IF_PLAIN(S, DiffF<N>) pow(const DiffF<N>& a, S k) {
    const float kk = float(k), v = powf(a.v, kk);
    const float dv = v * expm1f(kk * log1pf(a.d / a.v));
    return chain(a, v, dv, kk * (v + dv) / (a.v + a.d));
}
template <int N>
__device__ __forceinline__ DiffF<N> sin(const DiffF<N>& a) {
    const float h = 0.5f * a.d;
    return chain(a, sinf(a.v), 2.0f * cosf(a.v + h) * sinf(h), cosf(a.v + a.d));
}
template <int N>
__device__ __forceinline__ DiffF<N> cos(const DiffF<N>& a) {
    const float h = 0.5f * a.d;
    return chain(a, cosf(a.v), -2.0f * sinf(a.v + h) * sinf(h), -sinf(a.v + a.d));
}
template <int N>
__device__ __forceinline__ DiffF<N> tanh(const DiffF<N>& a) {
    const float at = a.v + a.d, t = tanhf(a.v), tt = tanhf(at);
    // sinh(da) / (cosh a cosh a') while the cosh stay finite, else the plain difference
    const float d = (fabsf(a.v) < 40.0f && fabsf(at) < 40.0f) ? sinhf(a.d) / (coshf(a.v) * coshf(at)) : tt - t;
    return chain(a, t, d, 1.0f - tt * tt);
}
template <int N>
__device__ __forceinline__ DiffF<N> atan(const DiffF<N>& a) {
    const float at = a.v + a.d, den = fmaf(a.v, at, 1.0f), t = atanf(a.v);
    // atan(a') - atan(a) = atan(da / (1 + a a')) while 1 + a a' > 0
    const float d = den > 0.0f ? atanf(a.d / den) : atanf(at) - t;
    return chain(a, t, d, 1.0f / fmaf(at, at, 1.0f));
}
template <int N>
__device__ __forceinline__ DiffF<N> square(const DiffF<N>& a) { return a * a; }
#undef GBFIT_IF_PLAIN

}  // namespace ad

// The kernels' model interface for a user definition Def, which supplies
// N, DIM (1 or 2) and template <class T, class S> static T h(const T* p, S x, S x2).
// Pass constants: plain pd[0..n) = p'; mixed pf[0..n) = float(p),
// pf[8..8+n) = p' - p (FP64 difference, rounded), pf[16..16+n) = p - float(p).
template <class Def>
struct MUser {
    static constexpr int N = Def::N;
    static constexpr int DIM = Def::DIM;
    static constexpr int PACK = 0;
    static constexpr bool WARP_PREP = false;
    static_assert(N >= 1 && N <= NMAX, "a user model has 1 to 8 parameters");
    __device__ static void prep_plain(const double* p, double* pd) {
        for (int k = 0; k < N; ++k) pd[k] = p[k];
    }
    __device__ static void eval_plain(const double* pd, double X, double Y, double& h, double* J) {
        ad::DualD<N> P[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            P[j].v = pd[j];
#pragma unroll
            for (int k = 0; k < N; ++k) P[j].g[k] = (j == k) ? 1.0 : 0.0;
        }
        const ad::DualD<N> r = Def::template h<ad::DualD<N>, double>(P, X, Y);
        h = r.v;
#pragma unroll
        for (int j = 0; j < N; ++j) J[j] = r.g[j];
    }
    __device__ static void prep_mixed(const MixedParams& P, float* pf) {
        for (int k = 0; k < N; ++k) { pf[k] = P.x[k]; pf[8 + k] = P.dx[k]; pf[16 + k] = P.xlo[k]; }
    }
    __device__ static void eval_mixed(const float* pf, float X, float Y, float& hb, float& dh, float* J) {
        ad::DiffF<N> P[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            P[j].v = pf[j];
            P[j].lo = pf[16 + j];
            P[j].d = pf[8 + j];
#pragma unroll
            for (int k = 0; k < N; ++k) P[j].g[k] = (j == k) ? 1.0f : 0.0f;
        }
        const ad::DiffF<N> r = Def::template h<ad::DiffF<N>, float>(P, X, Y);
        hb = r.v + r.lo;
        dh = r.d;
#pragma unroll
        for (int j = 0; j < N; ++j) J[j] = r.g[j];
    }
    __device__ static void eval_mixed2(const float*, float2, float2, float2&, float2&, float2*) {}
    __device__ static void eval_direct2(const float*, float2, float2, float2&, float2*) {}
};

// A model set of one user model: every fit of a launch is that model.
template <class M>
struct SingleModel {
    template <class F>
    __device__ __forceinline__ static void dispatch(int, F&& f) { f(M{}); }
};

}  // namespace gbfit

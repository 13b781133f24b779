#pragma once
// Per-precision device machinery of libgbfit (included by kernels_mixed.cu
// and kernels_fp64.cu, one instantiation each, compiled in parallel).
//
//   eval_round_kernel<PREC, MS>  one trust-region iteration for every running fit:
//       each CTA takes (fit, tile) work items, evaluates model, residual and
//       Jacobian row per point in registers, reduces J^T J, J^T r and cost
//       sums over its tile (never writing J), and writes one tile partial.
//       The last CTA of a group of tiles combines the group (FP64, fixed
//       order); the last group of a fit combines the fit and runs the
//       trust-region step for it (trf_step), which prepares the next
//       evaluation point.  No CTA waits for another: the hand-off is an
//       atomic arrival counter (last arriver continues).
//   fit_loop_kernel<PREC, MS>  the same rounds in one cooperative launch,
//       separated by a grid-wide barrier (bounded waits), until no fit runs
//       or the round cap is reached.
//   init_fits_kernel / init_slots_kernel  pass constants at p0.
#include "gbfit_internal.cuh"
#include "sync_device.cuh"
#include "models.cuh"
#include "trf_device.cuh"
#include "trf_step.cuh"

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
    // incremental pixel coordinates for the implicit grid (W, H < 2^31)
    int X, Y, W;
    __device__ void init(int64_t i, int64_t w) { W = (int)w; Y = (int)(i / w); X = (int)(i - (int64_t)Y * w); }
    __device__ void advance(int step) {
        X += step;
        if (X >= W) { if (W >= step) { X -= W; Y += 1; } else { Y += X / W; X = X % W; } }
    }
};

template <int PREC> struct AccT { using T = double; };
template <> struct AccT<PREC_MIXED> { using T = float; };

// One point: model value, residual and Jacobian row in registers, added to
// the Gram / gradient / cost accumulators (slot layout in gbfit_internal.cuh).
// ROB: a robust loss (R14): the rows are rescaled by sqrt(s) and rho'/sqrt(s)
// and the cost slots take C^2 rho and C^2 (rho(z') - rho(z)).
template <class M, int PREC, int WK, bool ROB = false>
__device__ __forceinline__ void accum_point(const float* pfl, const double* pdl, typename AccT<PREC>::T X,
                                            typename AccT<PREC>::T Y, typename AccT<PREC>::T yv,
                                            typename AccT<PREC>::T sv, bool check,
                                            typename AccT<PREC>::T (&acc)[n_acc(M::N, PREC)], int& bad,
                                            int loss = LOSS_LINEAR) {
    using AT = typename AccT<PREC>::T;
    constexpr int N = M::N;
    constexpr int NT = n_tri(N);
    AT w = AT(1);
    if (WK == W_ARRAY) w = sv;
    if (WK == W_SIGMA) {
        if (check && !(sv > AT(0) && isfinite(sv))) bad = 1;
        if (PREC == PREC_MIXED) w = __fdividef(1.0f, float(sv)); else w = AT(1) / sv;
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
        float cn = 0.0f, dc = 0.0f, rt = rn, js = w;
        if constexpr (ROB) {
            const float C2 = pfl[PF_C2], iC2 = pfl[PF_IC2];
            const float zn = rn * rn * iC2;
            float rho, r1, r2;
            loss_rho<float>(loss, zn, rho, r1, r2);
            const float rs = sqrtf(fmaxf(fmaf(2.0f * zn, r2, r1), 2.220446e-16f));
            js = w * rs;
            rt = r1 * rn / rs;
            cn = C2 * rho;
            dc = C2 * loss_drho<float>(loss, r * r * iC2, dr * fmaf(2.0f, r, dr) * iC2);
        }
#pragma unroll
        for (int a = 0; a < N; ++a) Jw[a] = js * J[a];
        int idx = 0;
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = a; b < N; ++b) { acc[idx] = fmaf(Jw[a], Jw[b], acc[idx]); ++idx; }
#pragma unroll
        for (int a = 0; a < N; ++a) acc[NT + a] = fmaf(Jw[a], rt, acc[NT + a]);
        if constexpr (ROB) {
            acc[NT + N] += cn;
            acc[NT + N + 1] += dc;
        } else {
            acc[NT + N] = fmaf(rn, rn, acc[NT + N]);
            // sum dr (2 r + dr); at the first evaluation (check, dr = 0): sum (w h)^2
            const float wh = w * hb;
            acc[NT + N + 1] = check ? fmaf(wh, wh, acc[NT + N + 1]) : fmaf(dr, fmaf(2.0f, r, dr), acc[NT + N + 1]);
        }
    } else {
        double h, J[N];
        M::eval_plain(pdl, X, Y, h, J);
        double r = w * (h - yv);
        double js = w, rt = r, cn = 0.0;
        if constexpr (ROB) {
            const double z = r * r * pdl[PD_IC2];
            double rho, r1, r2;
            loss_rho<double>(loss, z, rho, r1, r2);
            const double rs = sqrt(fmax(fma(2.0 * z, r2, r1), 2.220446049250313e-16));
            js = w * rs;
            rt = r1 * r / rs;
            cn = pdl[PD_C2] * rho;
        }
#pragma unroll
        for (int a = 0; a < N; ++a) Jw[a] = js * J[a];
        int idx = 0;
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = a; b < N; ++b) { acc[idx] = fma(Jw[a], Jw[b], acc[idx]); ++idx; }
#pragma unroll
        for (int a = 0; a < N; ++a) acc[NT + a] = fma(Jw[a], rt, acc[NT + a]);
        if constexpr (ROB) acc[NT + N] += cn;
        else acc[NT + N] = fma(r, r, acc[NT + N]);
    }
}

// Two points at once with packed FP32 (mixed precision): model, residual
// and weights packed; accumulators packed (ACC = float2, two partial sums
// per slot) or scalar (ACC = float, both points added to one sum).
// DIR: the direct form (value and partials at the trial point alone, no
// difference): slot NT+N+1 takes sum (w h)^2 at a first evaluation (check)
// and nothing otherwise (the step then forms f - f' itself).
// Data checks (check: a first evaluation) ride on two running values: chk
// = sum v * 0 over the checked values v (0 while every v is finite, NaN from
// the first non-finite one on) and smin = min sigma; the caller tests them
// once after its loop.  XY: the coordinates come from memory (not the grid).
template <class M, int WK, typename ACC, bool DIR = false, bool XY = true>
__device__ __forceinline__ void accum_point2(const float* pfl, float2 X, float2 Y, float2 yv, float2 sv, bool check,
                                             ACC (&acc)[n_acc(M::N, PREC_MIXED)], float2& chk, float& smin) {
    constexpr int N = M::N;
    constexpr int NT = n_tri(N);
    float2 w = bc(1.0f);
    if (check) {
        chk = fma2(yv, bc(0.0f), chk);
        if (XY) chk = fma2(X, bc(0.0f), chk);
        if (XY && M::DIM == 2) chk = fma2(Y, bc(0.0f), chk);
        if (WK == W_SIGMA) {
            chk = fma2(sv, bc(0.0f), chk);
            smin = fminf(smin, fminf(sv.x, sv.y));
        }
    }
    if (WK == W_SIGMA) w = make_float2(__fdividef(1.0f, sv.x), __fdividef(1.0f, sv.y));
    float2 hb, dh, J[N];
    if constexpr (DIR) {
        M::eval_direct2(pfl, X, Y, hb, J);
        dh = bc(0.0f);
    } else {
        M::eval_mixed2(pfl, X, Y, hb, dh, J);
    }
    float2 r = sub2(hb, yv), dr = dh, wh = hb;
    if (WK == W_SIGMA) {
        r = mul2(w, r);
        if (!DIR) dr = mul2(w, dr);
        wh = mul2(w, hb);
#pragma unroll
        for (int a = 0; a < N; ++a) J[a] = mul2(w, J[a]);
    }
    const float2 rn = DIR ? r : add2(r, dr);
    const float2 dc = DIR ? bc(0.0f) : mul2(dr, fma2(bc(2.0f), r, dr));
    if constexpr (std::is_same<ACC, float2>::value) {
        int idx = 0;
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = a; b < N; ++b) { acc[idx] = fma2(J[a], J[b], acc[idx]); ++idx; }
#pragma unroll
        for (int a = 0; a < N; ++a) acc[NT + a] = fma2(J[a], rn, acc[NT + a]);
        acc[NT + N] = fma2(rn, rn, acc[NT + N]);
        if (!DIR || check) acc[NT + N + 1] = check ? fma2(wh, wh, acc[NT + N + 1]) : add2(dc, acc[NT + N + 1]);
    } else {
        int idx = 0;
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = a; b < N; ++b) {
                acc[idx] = fmaf(J[a].y, J[b].y, fmaf(J[a].x, J[b].x, acc[idx]));
                ++idx;
            }
#pragma unroll
        for (int a = 0; a < N; ++a) acc[NT + a] = fmaf(J[a].y, rn.y, fmaf(J[a].x, rn.x, acc[NT + a]));
        acc[NT + N] = fmaf(rn.y, rn.y, fmaf(rn.x, rn.x, acc[NT + N]));
        if (!DIR || check)
            acc[NT + N + 1] = check ? fmaf(wh.y, wh.y, fmaf(wh.x, wh.x, acc[NT + N + 1])) : acc[NT + N + 1] + (dc.x + dc.y);
    }
}

// Points [i0, i1) with register loads (software-pipelined one point ahead).
template <class M, int PREC, typename DT, int LAYOUT, int WK, bool ROB = false>
__device__ __forceinline__ void tile_points(const FitDesc& d, const float* pfl, const double* pdl,
                                            int64_t i0, int64_t i1, bool check,
                                            typename AccT<PREC>::T (&acc)[n_acc(M::N, PREC)], int& bad) {
    using AT = typename AccT<PREC>::T;
    PointCoord pc;
    int64_t i = i0 + threadIdx.x;
    if (LAYOUT == X_GRID) pc.init(i, d.grid_w);
    AT nX = AT(0), nY = AT(0), ny = AT(0), ns = AT(1);
    auto load = [&](int64_t j, AT& X, AT& Y, AT& yv, AT& sv) {
        if (LAYOUT == X_GRID) {
            X = AT(pc.X); Y = AT(pc.Y);
            pc.advance(EVAL_THREADS);
        } else {
            X = AT(ldg_t<DT>(d.x, j));
            if (LAYOUT == X_SOA2) Y = AT(ldg_t<DT>(d.x2, j));
        }
        yv = AT(ldg_t<DT>(d.y, j));
        if (WK == W_ARRAY) sv = AT(ldg_t<double>(d.w, j));      // staged FP64 weights
        if (WK == W_SIGMA) sv = AT(ldg_t<DT>(d.w, j));
    };
    if (i < i1) load(i, nX, nY, ny, ns);
    for (; i < i1; i += EVAL_THREADS) {
        AT X = nX, Y = nY, yv = ny, sv = ns;
        if (i + EVAL_THREADS < i1) load(i + EVAL_THREADS, nX, nY, ny, ns);
        accum_point<M, PREC, WK, ROB>(pfl, pdl, X, Y, yv, sv, check, acc, bad, d.loss);
    }
}

// ---- bulk-copy ring (mixed precision, FP32 data): each CTA streams its
// tile through NST shared-memory stages of CH points per array with
// cp.async.bulk, completion tracked by one mbarrier per stage, so that
// about NST-1 chunks (tens of KB per SM) are in flight while the threads
// compute from shared memory.
constexpr int NST = 4;
constexpr int STAGE_FLOATS = 4096;                   // 16 KB per stage, shared by the streamed arrays
constexpr size_t RING_BYTES = size_t(NST) * STAGE_FLOATS * sizeof(float);
// Arrays a layout streams (x, x2, y, sigma as present) and the chunk (points
// per stage) that fills a stage with them: 4096 / 2048 / 1024 points.
template <int LAYOUT, int WK>
struct RingShape {
    static constexpr int NA = (LAYOUT == X_GRID ? 0 : LAYOUT == X_SOA2 ? 2 : 1) + 1 + (WK == W_SIGMA ? 1 : 0);
    static constexpr int CH = NA <= 1 ? 4096 : NA == 2 ? 2048 : 1024;
    static constexpr int SX = 0, SX2 = 1;                                   // slots (when present)
    static constexpr int SY = LAYOUT == X_GRID ? 0 : LAYOUT == X_SOA2 ? 2 : 1;
    static constexpr int SS = SY + 1;
    // the implicit grid tracks each thread's pixel by advancing 2 x EVAL_THREADS
    // points per step: a chunk must be a whole number of such steps
    static_assert(LAYOUT != X_GRID || CH % (2 * EVAL_THREADS) == 0, "grid chunks must be multiples of 512 points");
};
constexpr long long MBAR_SPIN_LIMIT = 1ll << 22;     // bounded waits (error flag past the limit)

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded both in polls and in time (global timer, checked every 256 polls):
// a chunk that never lands gives up within about MBAR_WAIT_NS.
constexpr unsigned long long MBAR_WAIT_NS = 1000ull * 1000 * 1000;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long it = 1; it < MBAR_SPIN_LIMIT; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 0 && global_ns() - t0 > MBAR_WAIT_NS) break;
    }
    return false;
}

// Arrival on a combine counter: one gpu-scope acq_rel atomic by one thread
// after a CTA barrier releases the CTA's partial-sum stores (cumulativity
// through the barrier) and, for the last arriver, acquires everyone else's.
__device__ __forceinline__ int arrive_acq_rel(int* ctr) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(ctr) : "memory");
    return old;
}

__device__ __forceinline__ unsigned atom_add_acq_rel_cta_shared(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_addr(p)), "r"(v)
                 : "memory");
    return old;
}

struct RingState {
    unsigned long long* bar;     // [NST] full barriers (bulk-copy completion)
    unsigned* rel;               // [NST] per-stage release counters (one acq_rel add per warp per consumed chunk;
                                 // the warp that completes a multiple of the warp count refills the stage)
    float* buf;                  // [NST][STAGE_FLOATS]
    unsigned seq;                // chunks consumed by this CTA so far (same in all threads)
    int* fail;                   // shared flag: a bounded wait gave up
    long long wait_cycles;       // thread 0: cycles spent waiting for chunks of the current tile
};

template <class M, int LAYOUT, int WK, bool DIR = false>
__device__ void tile_points_ring(const FitDesc& d, const float* pfl, int64_t i0, int64_t i1, bool check,
                                 float (&acc)[n_acc(M::N, PREC_MIXED)], int& bad, RingState& R) {
    using RS = RingShape<LAYOUT, WK>;
    constexpr int CH = RS::CH;
    const int t = threadIdx.x;
    // streamed arrays in slot order
    const float* src[4] = {nullptr, nullptr, nullptr, nullptr};
    if (LAYOUT != X_GRID) src[RS::SX] = (const float*)d.x;
    if (LAYOUT == X_SOA2) src[RS::SX2] = (const float*)d.x2;
    src[RS::SY] = (const float*)d.y;
    if (WK == W_SIGMA) src[RS::SS] = (const float*)d.w;
    // head up to 16-byte alignment of y; every streamed array must share it
    int64_t h = (int64_t)(((16 - (reinterpret_cast<uintptr_t>(src[RS::SY] + i0) & 15)) & 15) / 4);
    bool aligned = true;
#pragma unroll
    for (int a = 0; a < RS::NA; ++a)
        if (reinterpret_cast<uintptr_t>(src[a] + i0 + h) & 15) aligned = false;
    int64_t a0 = i0 + h;
    if (!aligned || a0 + 4 > i1) { tile_points<M, PREC_MIXED, float, LAYOUT, WK>(d, pfl, nullptr, i0, i1, check, acc, bad); return; }
    // whole 16-byte words go through the ring (a short last chunk allowed),
    // at most 3 trailing points through plain loads
    const int64_t nring = ((i1 - a0) / 4) * 4;
    const int nch = (int)((nring + CH - 1) / CH);
    const int64_t a1 = a0 + nring;
    auto count = [&](int c) { return (int)min((int64_t)CH, nring - (int64_t)c * CH); };
    // issue chunk c into its stage (free: at a tile's start every earlier
    // chunk is consumed; later, the caller is the last warp to release it)
    auto issue = [&](int c) {
        unsigned g = R.seq + c;
        int s = g % NST;
        unsigned long long* bar = R.bar + s;
        const unsigned nb = (unsigned)count(c) * sizeof(float);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, nb * RS::NA);
#pragma unroll
        for (int a = 0; a < RS::NA; ++a)
            bulk_load(R.buf + s * STAGE_FLOATS + a * CH, src[a] + a0 + (int64_t)c * CH, nb, bar);
    };
    if (t == 0)
        for (int c = 0; c < nch && c < NST; ++c) issue(c);
    // head points with plain loads while the first chunks stream in
    tile_points<M, PREC_MIXED, float, LAYOUT, WK>(d, pfl, nullptr, i0, a0, check, acc, bad);
    PointCoord pc;
    if (LAYOUT == X_GRID) pc.init(a0 + (M::PACK == 2 ? 2 * t : t), d.grid_w);
    // two points per thread step: 1D models on explicit x (packed sums),
    // the 2D model on the grid or explicit coordinates (scalar sums)
    constexpr bool PK = M::PACK == 1 && LAYOUT == X_VEC;
    constexpr bool PK2 = M::PACK == 2 && LAYOUT != X_VEC;
    constexpr int K = n_acc(M::N, PREC_MIXED);
    float2 acc2[PK ? K : 1];         // (the head's sums move in, so that acc[] is dead in the loop)
#pragma unroll
    for (int k = 0; k < (PK ? K : 1); ++k) acc2[k] = make_float2(PK ? acc[k] : 0.0f, 0.0f);
    float2 chk = bc(0.0f);           // data checks of the packed loops (accum_point2)
    float smin = INFINITY;
    for (int c = 0; c < nch; ++c) {
        unsigned g = R.seq + c;
        int s = g % NST;
        long long tw = (t == 0) ? clock64() : 0;
        if (!mbar_wait(R.bar + s, (g / NST) & 1)) *R.fail = 1;
        if (t == 0) R.wait_cycles += clock64() - tw;
        if (*R.fail) break;
        const float* B = R.buf + s * STAGE_FLOATS;
        const int cnt = count(c);
        if constexpr (PK) {
#pragma unroll 2
            for (int k = 2 * t; k < cnt; k += 2 * EVAL_THREADS) {
                float2 X = *reinterpret_cast<const float2*>(B + RS::SX * CH + k);
                float2 yv = *reinterpret_cast<const float2*>(B + RS::SY * CH + k);
                float2 sv = (WK == W_SIGMA) ? *reinterpret_cast<const float2*>(B + RS::SS * CH + k) : bc(1.0f);
                accum_point2<M, WK, float2, DIR>(pfl, X, bc(0.0f), yv, sv, check, acc2, chk, smin);
            }
        } else if constexpr (PK2) {
            for (int k = 2 * t; k < cnt; k += 2 * EVAL_THREADS) {
                float2 X, Y;
                if (LAYOUT == X_GRID) {
                    // pixels k, k + 1 of the chunk: (X, Y) and its right neighbour (next row at the edge)
                    X.x = float(pc.X);
                    Y.x = float(pc.Y);
                    bool wrap = pc.X + 1 >= pc.W;
                    X.y = wrap ? 0.0f : float(pc.X + 1);
                    Y.y = wrap ? float(pc.Y + 1) : float(pc.Y);
                    pc.advance(2 * EVAL_THREADS);
                } else {
                    X = *reinterpret_cast<const float2*>(B + RS::SX * CH + k);
                    Y = *reinterpret_cast<const float2*>(B + RS::SX2 * CH + k);
                }
                float2 yv = *reinterpret_cast<const float2*>(B + RS::SY * CH + k);
                float2 sv = (WK == W_SIGMA) ? *reinterpret_cast<const float2*>(B + RS::SS * CH + k) : bc(1.0f);
                accum_point2<M, WK, float, DIR, LAYOUT != X_GRID>(pfl, X, Y, yv, sv, check, acc, chk, smin);
            }
        } else
#pragma unroll 2
        for (int k = t; k < cnt; k += EVAL_THREADS) {
            float X = 0.0f, Y = 0.0f;
            if (LAYOUT == X_GRID) {
                X = float(pc.X);
                Y = float(pc.Y);
                pc.advance(EVAL_THREADS);
            } else {
                X = B[RS::SX * CH + k];
                if (LAYOUT == X_SOA2) Y = B[RS::SX2 * CH + k];
            }
            float yv = B[RS::SY * CH + k];
            float sv = (WK == W_SIGMA) ? B[RS::SS * CH + k] : 1.0f;
            accum_point<M, PREC_MIXED, WK>(pfl, nullptr, X, Y, yv, sv, check, acc, bad);
        }
        __syncwarp();
        if ((t & 31) == 0) {
            // this warp is done with the stage; the last of the CTA's warps
            // to release it refills it with the chunk NST ahead (no warp waits)
            const unsigned old = atom_add_acq_rel_cta_shared(R.rel + s, 1u);
            if ((old + 1) % (EVAL_THREADS / 32) == 0 && c + NST < nch) issue(c + NST);
        }
    }
    __syncthreads();
    if (*R.fail) {
        // give copies still in flight a bounded chance to land before leaving
        for (int c = 0; c < nch; ++c) { unsigned g = R.seq + c; mbar_wait(R.bar + (g % NST), (g / NST) & 1); }
        if (t < NST) R.rel[t] = 0;      // warps that left early did not release their stages
        __syncthreads();
    }
    R.seq += nch;
    if (check && !(chk.x == 0.0f && chk.y == 0.0f && smin > 0.0f)) bad = 1;
    if constexpr (PK) {
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = acc2[k].x + acc2[k].y;
    }
    // tail with plain loads
    tile_points<M, PREC_MIXED, float, LAYOUT, WK>(d, pfl, nullptr, a1, i1, check, acc, bad);
}

// ------------------------------------------------------------------ shared memory of the round kernel
struct RoundSmem {
    Engine eng;                        // the launch's engine record (kept out of registers)
    unsigned long long mbar[NST];
    unsigned ring_rel[NST];
    int ring_fail;
    FitDesc desc;
    long long t_mark, t_fence, t_group, t_loop;
    float pf[PF];
    double pd[PD];
    int flag[4];
    int cov_stage;                     // covariance fits: the item's round (FitState::cov_stage)
    int eval64;                        // mixed path: the item's fit evaluates in FP64 (precision guard)
    int ctl;
    int desc_fit;                      // fit whose descriptor is in desc (-1: none yet)
    union {
        float redf[8 * KMAX];
        double redd[8 * KMAX];
        double comb[EVAL_THREADS];
    };
    TrfSmem trf;
};

// Sum rows [0, nrows) of a [rows][KMAX] array into out[0..K) in a fixed order
// using all threads: thread t handles slot t % K over rows = part (mod P).
// Loads go out in batches of 8 rows per thread before any add, so that one
// L2 round trip covers a batch (rows were written by other CTAs: __ldcg).
template <typename T>
__device__ void combine_rows(const T* rows, int nrows, int K, double* scratch, double* out) {
    constexpr int BATCH = 8;
    int P = EVAL_THREADS / K;
    int t = threadIdx.x;
    int k = t % K, part = t / K;
    double s = 0.0;
    if (part < P)
        for (int r0 = part; r0 < nrows; r0 += BATCH * P) {
            T v[BATCH];
#pragma unroll
            for (int u = 0; u < BATCH; ++u) {
                int r = r0 + u * P;
                v[u] = r < nrows ? __ldcg(rows + (int64_t)r * KMAX + k) : T(0);
            }
#pragma unroll
            for (int u = 0; u < BATCH; ++u) s += double(v[u]);
        }
    scratch[t] = s;
    __syncthreads();
    if (t < K) {
        double tot = 0.0;
        for (int p = 0; p < P; ++p) tot += scratch[p * K + t];
        out[t] = tot;
    }
    __syncthreads();
}

// ------------------------------------------------------------------ the round kernel
template <class M, int PREC>
__device__ void eval_tile_dispatch(const RoundSmem& sm, int64_t i0, int64_t i1, bool check, int& bad,
                                   typename AccT<PREC>::T (&acc)[n_acc(M::N, PREC)], RingState& R) {
    using AT = typename AccT<PREC>::T;
    const FitDesc& d = sm.desc;
#pragma unroll
    for (int k = 0; k < n_acc(M::N, PREC); ++k) acc[k] = AT(0);
    float pfl[PF];
    double pdl[PD];
    if (PREC == PREC_MIXED) {
#pragma unroll
        for (int k = 0; k < PF; ++k) pfl[k] = sm.pf[k];
    } else {
#pragma unroll
        for (int k = 0; k < PD; ++k) pdl[k] = sm.pd[k];
    }
    const bool f64 = d.dtype == F64;
    int wk = d.wkind;
    if (d.loss != LOSS_LINEAR) {
        // robust losses (R14): plain loads, one point per thread step
#define RB_CASE(LAY, WKV)                                                                              \
        if (f64) tile_points<M, PREC, double, LAY, WKV, true>(d, pfl, pdl, i0, i1, check, acc, bad);   \
        else tile_points<M, PREC, float, LAY, WKV, true>(d, pfl, pdl, i0, i1, check, acc, bad);
        if (M::DIM == 2) {
            if (d.layout == X_GRID) {
                if (wk == W_NONE) { RB_CASE(X_GRID, W_NONE) } else if (wk == W_ARRAY) { RB_CASE(X_GRID, W_ARRAY) } else { RB_CASE(X_GRID, W_SIGMA) }
            } else {
                if (wk == W_NONE) { RB_CASE(X_SOA2, W_NONE) } else if (wk == W_ARRAY) { RB_CASE(X_SOA2, W_ARRAY) } else { RB_CASE(X_SOA2, W_SIGMA) }
            }
        } else {
            if (wk == W_NONE) { RB_CASE(X_VEC, W_NONE) } else if (wk == W_ARRAY) { RB_CASE(X_VEC, W_ARRAY) } else { RB_CASE(X_VEC, W_SIGMA) }
        }
#undef RB_CASE
        return;
    }
    // mixed precision on FP32 data streams through the bulk-copy ring; packed
    // models evaluate a first evaluation and a wide trial in the direct form
    const bool dir = M::PACK != 0 && sm.flag[1] != PH_TRIAL;
#define GB_CASE(LAY, WKV)                                                                              \
    if constexpr (PREC == PREC_MIXED && WKV != W_ARRAY) {                                              \
        if (f64) tile_points<M, PREC, double, LAY, WKV>(d, pfl, pdl, i0, i1, check, acc, bad);         \
        else if constexpr (M::PACK != 0) {                                                             \
            if (dir) tile_points_ring<M, LAY, WKV, true>(d, pfl, i0, i1, check, acc, bad, R);          \
            else tile_points_ring<M, LAY, WKV, false>(d, pfl, i0, i1, check, acc, bad, R);             \
        } else tile_points_ring<M, LAY, WKV>(d, pfl, i0, i1, check, acc, bad, R);                      \
    } else {                                                                                           \
        if (f64) tile_points<M, PREC, double, LAY, WKV>(d, pfl, pdl, i0, i1, check, acc, bad);         \
        else tile_points<M, PREC, float, LAY, WKV>(d, pfl, pdl, i0, i1, check, acc, bad);              \
    }
    if (M::DIM == 2) {
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

// ---- full covariance (Appendix C, Eqs. covariance, slsq1, slsq2).  With
// C = L L^T the method runs on L^-1 r and L^-1 J.  A covariance fit
// alternates two rounds per evaluation: the points of each item into hbuf,
// then rows of Z = X hbuf (X = L^-1, precomputed), each row reduced like a
// point.  The row-parallel product replaces the paper's per-iteration
// triangular solves, whose rows depend on one another.
constexpr int COV_SMEM_BYTES = 20480;            // shared scratch of the row reduction

template <class M, int PREC, typename DT, int LAYOUT>
__device__ void cov_eval_points(const FitDesc& d, const float* pfl, const double* pdl, int64_t i0, int64_t i1,
                                bool check, int& bad) {
    const int64_t m = d.m;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += EVAL_THREADS) {
        double X, Y = 0.0;
        if (LAYOUT == X_GRID) {
            X = double(i % d.grid_w);
            Y = double(i / d.grid_w);
        } else {
            X = double(ldg_t<DT>(d.x, i));
            if (LAYOUT == X_SOA2) Y = double(ldg_t<DT>(d.x2, i));
        }
        const double yv = double(ldg_t<DT>(d.y, i));
        if (check && !(isfinite(X) && isfinite(Y) && isfinite(yv))) bad = 1;
        if constexpr (PREC == PREC_MIXED) {
            float hb, dh, J[M::N];
            M::eval_mixed(pfl, float(X), float(Y), hb, dh, J);
            float* H = (float*)d.hbuf;
            H[i] = hb - float(yv);
            H[m + i] = dh;
#pragma unroll
            for (int a = 0; a < M::N; ++a) H[(2 + a) * m + i] = J[a];
        } else {
            double h, J[M::N];
            M::eval_plain(pdl, X, Y, h, J);
            double* H = (double*)d.hbuf;
            H[i] = h - yv;
#pragma unroll
            for (int a = 0; a < M::N; ++a) H[(1 + a) * m + i] = J[a];
        }
    }
}

template <class M, int PREC>
__device__ void cov_eval_dispatch(const FitDesc& d, const float* pfl, const double* pdl, int64_t i0, int64_t i1,
                                  bool check, int& bad) {
    const bool f64 = d.dtype == F64;
    if (M::DIM == 2) {
        if (d.layout == X_GRID) {
            if (f64) cov_eval_points<M, PREC, double, X_GRID>(d, pfl, pdl, i0, i1, check, bad);
            else cov_eval_points<M, PREC, float, X_GRID>(d, pfl, pdl, i0, i1, check, bad);
        } else {
            if (f64) cov_eval_points<M, PREC, double, X_SOA2>(d, pfl, pdl, i0, i1, check, bad);
            else cov_eval_points<M, PREC, float, X_SOA2>(d, pfl, pdl, i0, i1, check, bad);
        }
    } else {
        if (f64) cov_eval_points<M, PREC, double, X_VEC>(d, pfl, pdl, i0, i1, check, bad);
        else cov_eval_points<M, PREC, float, X_VEC>(d, pfl, pdl, i0, i1, check, bad);
    }
}

// Rows [32 tile, 32 tile + 32) of Z = X H into the accumulators: lane =
// row, the warps split the column index j (chunks of H staged in shared
// memory, X read coalesced down its columns), partial rows summed over the
// warps in a fixed order, then warp 0 adds each row as one point.
template <int N, int PREC>
__device__ void cov_rows(const FitDesc& d, int tile, void* scratch, typename AccT<PREC>::T (&acc)[n_acc(N, PREC)]) {
    using HT = typename AccT<PREC>::T;
    constexpr int NC = (PREC == PREC_MIXED) ? N + 2 : N + 1;
    constexpr int CJ = COV_SMEM_BYTES / (NC * (int)sizeof(HT)) / 32 * 32;
    constexpr int NW = EVAL_THREADS / 32;
    static_assert(NW * NC * 32 * sizeof(HT) <= COV_SMEM_BYTES, "row partials must fit the scratch");
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t m = d.m;
    const int64_t i = (int64_t)tile * COV_ROWS + lane;
    const bool row_ok = i < m;
    const int64_t jend = min(m, (int64_t)(tile + 1) * COV_ROWS);
    const HT* Xc = (const HT*)d.xinv;
    const HT* Hg = (const HT*)d.hbuf;
    HT* Hs = (HT*)scratch;                          // [NC][CJ]
    HT z[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) z[c] = HT(0);
    for (int64_t j0 = 0; j0 < jend; j0 += CJ) {
        const int cj = (int)min((int64_t)CJ, jend - j0);
        __syncthreads();                            // the previous chunk is consumed
        for (int k = t; k < NC * cj; k += EVAL_THREADS) {
            const int c = k / cj, jj = k - c * cj;
            Hs[c * CJ + jj] = __ldcg(Hg + (int64_t)c * m + j0 + jj);   // written by other CTAs last round
        }
        __syncthreads();
        for (int jj = warp; jj < cj; jj += NW) {
            const HT x = row_ok ? Xc[(j0 + jj) * m + i] : HT(0);
#pragma unroll
            for (int c = 0; c < NC; ++c) z[c] = fma(x, Hs[c * CJ + jj], z[c]);
        }
    }
    __syncthreads();
    HT* red = (HT*)scratch;                         // [NW][NC][32]
#pragma unroll
    for (int c = 0; c < NC; ++c) red[(warp * NC + c) * 32 + lane] = z[c];
    __syncthreads();
    if (warp == 0 && row_ok) {
        HT s[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            HT v = HT(0);
            for (int w = 0; w < NW; ++w) v += red[(w * NC + c) * 32 + lane];
            s[c] = v;
        }
        constexpr int NT = n_tri(N);
        constexpr int J0 = (PREC == PREC_MIXED) ? 2 : 1;
        const HT r = s[0];
        const HT rn = (PREC == PREC_MIXED) ? r + s[1] : r;
        int idx = 0;
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = a; b < N; ++b) { acc[idx] = fma(s[J0 + a], s[J0 + b], acc[idx]); ++idx; }
#pragma unroll
        for (int a = 0; a < N; ++a) acc[NT + a] = fma(s[J0 + a], rn, acc[NT + a]);
        acc[NT + N] = fma(rn, rn, acc[NT + N]);
        if constexpr (PREC == PREC_MIXED) acc[NT + N + 1] += s[1] * (HT(2) * r + s[1]);
    }
    __syncthreads();                                // the scratch is free again
}

// FP64 evaluation of points [i0, i1) inside the mixed-precision kernel (a fit
// that the precision guard moved to FP64 passes), block-reduced: thread
// k < n_acc(N, FP64) returns slot k of the tile sum.
template <class M>
__device__ __forceinline__ double tile_sum_fp64(RoundSmem& sm, int64_t i0, int64_t i1, bool check, int* bad_out) {
    constexpr int K = n_acc(M::N, PREC_FP64);
    double acc[K];
    int bad = 0;
    RingState R{};                     // the FP64 point loops take no bulk-copy ring
    eval_tile_dispatch<M, PREC_FP64>(sm, i0, i1, check, bad, acc, R);
    *bad_out = bad;
    double tsum = 0.0;
    block_reduce<K, double>(acc, sm.redd, tsum);
    return tsum;
}

// Tile part of a work item: evaluate the tile's points, reduce them and
// store the tile's partial sums.  Returns the number of sum slots, or 0 when
// the item has nothing more to do (the evaluation round of a covariance fit).
template <class M, int PREC>
__device__ __forceinline__ int item_tile(RoundSmem& sm, const Engine& E, int fit, int tile, RingState& R) {
    using AT = typename AccT<PREC>::T;
    constexpr int N = M::N;
    constexpr int K = n_acc(N, PREC);
    const FitDesc& d = sm.desc;
    FitState* stp = E.state + fit;
    int64_t i0 = (int64_t)tile * d.tile_points;
    int64_t i1 = i0 + d.tile_points;
    if (i1 > d.m) i1 = d.m;
    bool check = sm.flag[1] == PH_INIT;
    R.wait_cycles = 0;
    int bad = 0;
    AT acc[K];
    if (d.cov) {
        if (sm.cov_stage == 0) {
            // evaluation round: the item's points into hbuf; the last item of
            // the fit to finish opens the row round (the grid barrier
            // publishes hbuf and the stage)
            cov_eval_dispatch<M, PREC>(d, sm.pf, sm.pd, i0, i1, check, bad);
            if (check) {
                int any = __syncthreads_or(bad);
                if (any && threadIdx.x == 0) atomicOr(&stp->bad_data, 1);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int old = arrive_acq_rel(&E.fit_cnt[fit]);
                if (old == d.n_tiles - 1) {
                    E.fit_cnt[fit] = 0;
                    stp->cov_stage = 1;
                }
            }
            return 0;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = AT(0);
        cov_rows<N, PREC>(d, tile, R.buf, acc);
        check = false;
    } else {
        eval_tile_dispatch<M, PREC>(sm, i0, i1, check, bad, acc, R);
    }
    if (threadIdx.x == 0) sm.t_loop = clock64();
    if (sm.ring_fail && threadIdx.x == 0) atomicOr(&stp->bad_data, 2);   // a bounded wait gave up
    if (check) {
        int any = __syncthreads_or(bad);
        if (any && threadIdx.x == 0) atomicOr(&stp->bad_data, 1);
    }
    AT* red = (PREC == PREC_MIXED) ? (AT*)sm.redf : (AT*)sm.redd;
    AT tsum;
    block_reduce<K, AT>(acc, red, tsum);
    if (threadIdx.x == 0) sm.t_mark = clock64();
    const int64_t row = d.tile_base + tile;
    if (threadIdx.x < K) E.tile_part_d[row * KMAX + threadIdx.x] = double(tsum);
    return K;
}

// The same for a fit the guard moved to FP64 passes (mixed kernel only).  Not
// inlined: its FP64 registers stay out of the streaming FP32 path's
// allocation, and it is called where little else is live.
template <class M>
__device__ __noinline__ int item_tile_e64(RoundSmem& sm, const Engine& E, int fit, int tile) {
    constexpr int K = n_acc(M::N, PREC_FP64);
    const FitDesc& d = sm.desc;
    FitState* stp = E.state + fit;
    const int64_t i0 = (int64_t)tile * d.tile_points;
    const int64_t i1 = min(i0 + (int64_t)d.tile_points, d.m);
    const bool check = sm.flag[1] == PH_INIT;
    int bad = 0;
    const double tsum = tile_sum_fp64<M>(sm, i0, i1, check, &bad);
    if (threadIdx.x == 0) sm.t_loop = clock64();
    if (check) {
        int any = __syncthreads_or(bad);
        if (any && threadIdx.x == 0) atomicOr(&stp->bad_data, 1);
    }
    if (threadIdx.x == 0) sm.t_mark = clock64();
    const int64_t row = d.tile_base + tile;
    if (threadIdx.x < K) E.tile_part_d[row * KMAX + threadIdx.x] = tsum;
    return K;
}

// One work item: its tile, then (by the last arriver) the group and fit
// combines and the fit's trust-region step.
template <class M, int PREC, class MS>
__device__ void process_item(RoundSmem& sm, const Engine& E, int fit, int tile, RingState& R, long long t_item) {
    const long long t_tile = clock64();
    int Kuse;
    if (PREC == PREC_MIXED && sm.eval64 && !sm.desc.cov) {
        Kuse = item_tile_e64<M>(sm, E, fit, tile);
        R.wait_cycles = 0;
    } else {
        Kuse = item_tile<M, PREC>(sm, E, fit, tile, R);
    }
    if (Kuse == 0) return;
    const FitDesc& d = sm.desc;
    FitState* stp = E.state + fit;
    // ---- last arriver of the group combines the group
    __syncthreads();
    int group = tile / d.group_tiles;
    int g0 = group * d.group_tiles;
    int gsize = min(d.group_tiles, d.n_tiles - g0);
    if (threadIdx.x == 0) {
        int old = arrive_acq_rel(&E.group_cnt[d.group_base + group]);
        sm.flag[2] = (old == gsize - 1);
    }
    __syncthreads();
    if (!sm.flag[2]) return;
    if (d.n_groups == 1 && !E.owner_mode) prefetch_state(stp, sm.trf);      // this CTA runs the step
    if (threadIdx.x == 0) sm.t_fence = clock64();
    double* gout = E.group_part + (d.group_base + group) * KMAX;
    combine_rows<double>(E.tile_part_d + (d.tile_base + g0) * KMAX, gsize, Kuse, sm.comb, sm.trf.tot);
    if (threadIdx.x == 0) {
        E.group_cnt[d.group_base + group] = 0;
        sm.t_group = clock64();
    }
    if (E.owner_mode) {
        // the fit's owner CTA (owner_steps) combines the group sums and steps
        if (threadIdx.x < Kuse) gout[threadIdx.x] = sm.trf.tot[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) {
            int old = arrive_acq_rel(&E.fit_cnt[fit]);
            if (old == d.n_groups - 1) {
                trace_bump(stp->trace, TR_COMBINE, (unsigned long long)(sm.t_group - sm.t_mark));
                trace_bump(stp->trace, TR_C_FENCE, (unsigned long long)(sm.t_fence - sm.t_mark));
                trace_bump(stp->trace, TR_C_GROUP, (unsigned long long)(sm.t_group - sm.t_fence));
                trace_bump(stp->trace, TR_TILE, (unsigned long long)(sm.t_mark - t_tile));
                trace_bump(stp->trace, TR_PRE_TILE, (unsigned long long)(t_tile - t_item));
                trace_bump(stp->trace, TR_TILE_LOOP, (unsigned long long)(sm.t_loop - t_tile));
                trace_bump(stp->trace, TR_RING_WAIT, (unsigned long long)R.wait_cycles);
            }
        }
        return;
    }
    if (d.n_groups > 1) {
        // second level: the last group of the fit combines the group sums
        if (threadIdx.x < Kuse) gout[threadIdx.x] = sm.trf.tot[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) {
            int old = arrive_acq_rel(&E.fit_cnt[fit]);
            sm.flag[3] = (old == d.n_groups - 1);
        }
        __syncthreads();
        if (!sm.flag[3]) return;
        prefetch_state(stp, sm.trf);
        combine_rows<double>(E.group_part + d.group_base * KMAX, d.n_groups, Kuse, sm.comb, sm.trf.tot);
    }
    if (threadIdx.x == 0) {
        E.fit_cnt[fit] = 0;
        long long now = clock64();
        trace_bump(stp->trace, TR_COMBINE, (unsigned long long)(now - sm.t_mark));
        trace_bump(stp->trace, TR_C_FENCE, (unsigned long long)(sm.t_fence - sm.t_mark));
        trace_bump(stp->trace, TR_C_GROUP, (unsigned long long)(sm.t_group - sm.t_fence));
        trace_bump(stp->trace, TR_C_FINAL, (unsigned long long)(now - sm.t_group));
        trace_bump(stp->trace, TR_TILE, (unsigned long long)(sm.t_mark - t_tile));
        trace_bump(stp->trace, TR_PRE_TILE, (unsigned long long)(t_tile - t_item));
        trace_bump(stp->trace, TR_TILE_LOOP, (unsigned long long)(sm.t_loop - t_tile));
        trace_bump(stp->trace, TR_RING_WAIT, (unsigned long long)R.wait_cycles);
    }
    __syncthreads();
    trf_step<PREC, MS>(d, stp, E.results + fit, sm.trf, E.running);
    __syncthreads();
    if (E.queue_mode && threadIdx.x == 0 && sm.trf.si[SI_STATUS] == FS_RUNNING) {
        // queue mode: the next evaluation's tiles become claimable (the CTA
        // barrier above orders the new state before these releases)
        unsigned old;
        asm volatile("atom.release.gpu.global.exch.b32 %0, [%1], 0;" : "=r"(old) : "l"(E.next_tile + fit) : "memory");
        asm volatile("atom.release.gpu.global.or.b32 %0, [%1], %2;"
                     : "=r"(old) : "l"(E.fit_bits + (fit >> 5)), "r"(1u << (fit & 31)) : "memory");
    }
}

// Copy the engine record into shared memory (round_setup's barrier publishes it).
__device__ __forceinline__ void stage_engine(RoundSmem& sm, const Engine* Ep) {
    const int* src = (const int*)Ep;
    int* dst = (int*)&sm.eng;
    for (int k = threadIdx.x; k < (int)(sizeof(Engine) / 4); k += blockDim.x) dst[k] = src[k];
}

// Ring barriers and flags at the start of a round kernel.
template <int PREC>
__device__ __forceinline__ void round_setup(RoundSmem& sm, float* ring_buf, RingState& R) {
    R.bar = sm.mbar;
    R.rel = sm.ring_rel;
    R.buf = ring_buf;
    R.seq = 0;
    R.fail = &sm.ring_fail;
    if (threadIdx.x == 0) sm.desc_fit = -1;
    if (PREC == PREC_MIXED) {
        if (threadIdx.x == 0) {
            for (int s = 0; s < NST; ++s) {
                mbar_init(&sm.mbar[s], 1);
                sm.ring_rel[s] = 0;
            }
            sm.ring_fail = 0;
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    } else if (threadIdx.x == 0) {
        sm.ring_fail = 0;
    }
    __syncthreads();
}

// One round: this CTA's share of the work items.  The first item of every
// CTA is `first` (items 0 .. grid-1 one per CTA); after that either
// grid-stride (static) or the next unclaimed item from the round's counter
// (dynamic: CTAs that finish early take more, so no CTA ends a round far
// behind the others).  Which CTA processes an item does not change any sum.
template <int PREC, class MS>
__device__ __forceinline__ void run_items(RoundSmem& sm, const Engine& E, RingState& R, int first,
                                          int* next_item) {
    int n_items = *E.n_items;
    for (int it = first; it < n_items;) {
        long long t_item = clock64();
        WorkItem wi = E.items[it];
        FitState* stp = E.state + wi.fit;
        // one round trip for the item's state words, pass constants and (when
        // this CTA's previous item was another fit) descriptor; state from
        // L2, since other CTAs rewrite it between rounds
        if (threadIdx.x == 0) {
            sm.flag[0] = __ldcg(&stp->run);
            sm.flag[1] = __ldcg(&stp->phase);
            sm.cov_stage = __ldcg(&stp->cov_stage);
            sm.eval64 = __ldcg(&stp->eval64);
        }
        // mixed path: both sets of pass constants (the FP64 ones serve a fit the guard moved to FP64)
        if (PREC == PREC_MIXED) {
            if (threadIdx.x < PF) sm.pf[threadIdx.x] = __ldcg(stp->pf + threadIdx.x);
            else if (threadIdx.x < PF + PD) sm.pd[threadIdx.x - PF] = __ldcg(stp->pd + threadIdx.x - PF);
        } else if (threadIdx.x < PD) {
            sm.pd[threadIdx.x] = __ldcg(stp->pd + threadIdx.x);
        }
        if (wi.fit != sm.desc_fit) {
            const int* src = (const int*)(E.desc + wi.fit);
            int* dst = (int*)&sm.desc;
            for (int k = threadIdx.x; k < (int)(sizeof(FitDesc) / 4); k += EVAL_THREADS) dst[k] = src[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) sm.desc_fit = wi.fit;
        if (sm.flag[0] != RS_RUNNING) {
            __syncthreads();
            if (next_item) {
                if (threadIdx.x == 0) sm.flag[0] = (int)gridDim.x + atomicAdd(next_item, 1);
                __syncthreads();
                it = sm.flag[0];
                __syncthreads();
            } else {
                it += gridDim.x;
            }
            continue;
        }
        MS::dispatch(sm.desc.model,
                     [&](auto m) { process_item<decltype(m), PREC, MS>(sm, E, wi.fit, wi.tile, R, t_item); });
        if (next_item) {
            if (threadIdx.x == 0) sm.flag[0] = (int)gridDim.x + atomicAdd(next_item, 1);
            __syncthreads();
            it = sm.flag[0];
        } else {
            it += gridDim.x;
        }
        __syncthreads();
    }
}

template <int PREC, class MS>
__global__ void __launch_bounds__(EVAL_THREADS, 2) eval_round_kernel(const Engine* __restrict__ Ep) {
    __shared__ RoundSmem sm;
    extern __shared__ __align__(128) float ring_buf[];
    stage_engine(sm, Ep);
    RingState R;
    round_setup<PREC>(sm, ring_buf, R);
    run_items<PREC, MS>(sm, sm.eng, R, blockIdx.x, nullptr);
}

// ---- grid-wide round barrier of the persistent loop.  The loop kernel is
// launched cooperatively (every CTA resident), so a CTA that waits here
// waits only for CTAs that are running.  Waits are bounded in time; past
// the bound the CTA raises the abort bit and every CTA leaves the loop.
constexpr unsigned long long ROUND_WAIT_LIMIT_NS = 10ull * 1000 * 1000 * 1000;   // default of Engine::wait_ns
__device__ __forceinline__ unsigned long long wait_limit(const Engine& E) {
    return E.wait_ns ? E.wait_ns : ROUND_WAIT_LIMIT_NS;
}
enum { CTL_STOP = 1, CTL_ABORT = 2 };

// All CTAs arrive; the last one closes the round (rounds, running, stop
// decision; count_round false for the set-up barrier) and opens the next.
// Returns the control word (CTL_*) for every thread of every CTA.
__device__ inline int grid_round_end(Engine* Ed, const Engine& E, int* ctl_smem, bool count_round) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* cnt = (unsigned*)&Ed->sc[5];
        unsigned* gen = (unsigned*)&Ed->sc[6];      // (generation << 2) | control word of the round closed last
        volatile int* ctl = &Ed->sc[7];             // abort requests raised during the round
        const unsigned g = ld_acquire_u32(gen);
        unsigned old;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(cnt) : "memory");
        int c;
        if (old == gridDim.x - 1) {
            // the loads the decision needs go out together, then one release
            const int pend = *ctl;
            int r = 0, run = 0, cap = 0;
            if (count_round) {
                r = *(volatile int*)E.rounds;
                run = *(volatile int*)E.running;
                cap = *(volatile int*)E.max_rounds;
            }
            *(volatile unsigned*)cnt = 0;
            c = pend & CTL_ABORT;
            if (count_round) {
                E.sm_cnt[SM_IDS] = 0;                 // next round's dynamic items start over
                r += 1;
                *(volatile int*)E.rounds = r;
                E.out[0] = run;
                E.out[1] = r;
                if (run <= 0 || r >= cap) c |= CTL_STOP;
            }
            st_release_u32(gen, (((g >> 2) + 1u) << 2) | (unsigned)c);
        } else {
            const unsigned long long t0 = global_ns();
            unsigned v;
            bool timed_out = false;
            while ((v = ld_acquire_u32(gen)) == g) {
                __nanosleep(128);
                if (global_ns() - t0 > wait_limit(E)) {
                    atomicOr((int*)ctl, CTL_ABORT);
                    timed_out = true;
                    break;
                }
            }
            c = timed_out ? CTL_ABORT : (int)(v & 3u);   // the control word travels with the release
        }
        if (c & CTL_ABORT) atomicOr(E.out + 2, 1);
        *ctl_smem = c;
    }
    __syncthreads();
    return *ctl_smem;
}

// Owner mode: after its items, the CTA of rank f waits (bounded) until every
// group of fit f has published its sum, then combines the group sums in
// index order and runs the fit's trust-region step.  The step then runs on
// the same SM every round, with its code in that SM's instruction caches.
template <class M, int PREC, class MS>
__device__ void owner_combine_step(RoundSmem& sm, const Engine& E, int fit) {
    const FitDesc& d = sm.desc;
    // slots of the evaluation just finished (the prefetched state says which precision ran it)
    const int K = (PREC == PREC_MIXED && sm.trf.stc.eval64 && !d.cov) ? n_acc(M::N, PREC_FP64) : n_acc(M::N, PREC);
    FitState* stp = E.state + fit;
    long long t0 = clock64();
    combine_rows<double>(E.group_part + d.group_base * KMAX, d.n_groups, K, sm.comb, sm.trf.tot);
    if (threadIdx.x == 0) {
        unsigned long long dt = (unsigned long long)(clock64() - t0);
        trace_bump(stp->trace, TR_COMBINE, dt);
        trace_bump(stp->trace, TR_C_FINAL, dt);
    }
    __syncthreads();
    trf_step<PREC, MS>(d, stp, E.results + fit, sm.trf, E.running);
    __syncthreads();
}

template <int PREC, class MS>
__device__ void owner_steps(RoundSmem& sm, const Engine& E, Engine* Ed, int rank) {
    const int nf = *E.nfits_dev;
    for (int f = rank; f < nf; f += gridDim.x) {
        FitState* stp = E.state + f;
        if (threadIdx.x == 0) sm.flag[0] = __ldcg(&stp->run);
        if (f != sm.desc_fit) {
            const int* src = (const int*)(E.desc + f);
            int* dst = (int*)&sm.desc;
            for (int k = threadIdx.x; k < (int)(sizeof(FitDesc) / 4); k += EVAL_THREADS) dst[k] = src[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) sm.desc_fit = f;
        if (sm.flag[0] != RS_RUNNING) {
            __syncthreads();
            continue;
        }
        prefetch_state(stp, sm.trf);                       // overlaps the wait
        if (threadIdx.x == 0) {
            const unsigned want = (unsigned)sm.desc.n_groups;
            const unsigned* cnt = reinterpret_cast<const unsigned*>(E.fit_cnt + f);
            const unsigned long long g0 = global_ns();
            int ok = 1;
            while (ld_acquire_u32(cnt) != want) {
                if (global_ns() - g0 > wait_limit(E)) { ok = 0; break; }
            }
            if (ok) E.fit_cnt[f] = 0;
            else atomicOr(&Ed->sc[7], CTL_ABORT);
            sm.flag[3] = ok;
            trace_bump(stp->trace, TR_OWNER_WAIT_NS, global_ns() - g0);
        }
        __syncthreads();
        if (!sm.flag[3]) continue;
        MS::dispatch(sm.desc.model, [&](auto m) { owner_combine_step<decltype(m), PREC, MS>(sm, E, f); });
    }
}

// ---- queue mode (launches of many fits): no lock-step rounds.  Fit f's
// tiles of its current evaluation are claimed from next_tile[f]; bit f of
// fit_bits says it may still have some.  The claimer of the last tile clears
// the bit; the fit's step re-arms both for the next evaluation after writing
// the new state (process_item).  So a fit's next pass starts as soon as its
// step ends, and no CTA waits for the slowest fit of a round.  A CTA with
// nothing to claim backs off and looks again; it leaves when no fit runs, on
// the abort bit, or after a bounded idle wait (raising the abort bit).
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Warp 0: one look over the bitmap for a claimable tile (fit, tile), or fit = -1.
__device__ __forceinline__ void queue_claim(const Engine& E, int nf, int rank, int& fit, int& tile) {
    const int l = threadIdx.x & 31;
    const int nw = (nf + 31) / 32;
    fit = -1;
    tile = -1;
    for (int base = 0; base < nw && fit < 0; base += 32) {
        const int w = (rank + base + l) % nw;
        const unsigned bits = (base + l < nw) ? __ldcg(E.fit_bits + w) : 0u;
        unsigned any = __ballot_sync(FULL, bits != 0u);
        while (any && fit < 0) {
            const int src = __ffs(any) - 1;
            any &= any - 1;
            const unsigned b = __shfl_sync(FULL, bits, src);
            const int ws = __shfl_sync(FULL, w, src);
            int f = -1, t = -1;
            if (l == 0) {
                // one set bit of the word, from a rank-dependent position
                const int rot = rank & 31;
                const unsigned r = __funnelshift_r(b, b, rot);
                const int bit = ((__ffs(r) - 1) + rot) & 31;
                const int cand = ws * 32 + bit;
                if (cand < nf) {
                    const int nt = __ldg(&E.desc[cand].n_tiles);
                    const unsigned c = atom_add_acq_rel(reinterpret_cast<unsigned*>(E.next_tile + cand), 1u);
                    if ((int)c < nt) {
                        f = cand;
                        t = (int)c;
                        if ((int)c == nt - 1) atomicAnd(E.fit_bits + ws, ~(1u << bit));   // the epoch is claimed
                    }
                }
            }
            fit = __shfl_sync(FULL, f, 0);
            tile = __shfl_sync(FULL, t, 0);
        }
    }
}

template <int PREC, class MS>
__device__ void queue_loop(RoundSmem& sm, const Engine& E, Engine* Ed, RingState& R, int rank,
                           unsigned long long* acct) {
    const int nf = *E.nfits_dev;
    volatile int* ctl = &Ed->sc[7];
    unsigned long long busy = 0, idle = 0;
    while (true) {
        const unsigned long long t0 = global_ns();
        if (threadIdx.x < 32) {
            int fit = -1, tile = -1, stop = 0;
            unsigned back = 32;
            while (true) {
                queue_claim(E, nf, rank, fit, tile);
                if (fit >= 0) break;
                int st = 0;
                if (threadIdx.x == 0)
                    st = (ld_acquire_u32(reinterpret_cast<const unsigned*>(E.running)) == 0u || (*ctl & CTL_ABORT)) ? 1 : 0;
                stop = __shfl_sync(FULL, st, 0);
                if (stop) break;
                if (global_ns() - t0 > wait_limit(E)) {
                    if (threadIdx.x == 0) atomicOr((int*)ctl, CTL_ABORT);
                    stop = 1;
                    break;
                }
                __nanosleep(back);
                back = back < 512 ? back * 2 : 512;
            }
            if (threadIdx.x == 0) { sm.flag[0] = fit; sm.flag[1] = tile; sm.flag[2] = stop; }
        }
        __syncthreads();
        const int fit = sm.flag[0], tile = sm.flag[1], stop = sm.flag[2];
        __syncthreads();
        const unsigned long long t1 = global_ns();
        idle += t1 - t0;
        if (stop) break;
        // the item's state words, pass constants and descriptor (L2: other CTAs wrote them)
        FitState* stp = E.state + fit;
        if (threadIdx.x == 0) {
            sm.flag[0] = __ldcg(&stp->run);
            sm.flag[1] = __ldcg(&stp->phase);
            sm.cov_stage = __ldcg(&stp->cov_stage);
            sm.eval64 = __ldcg(&stp->eval64);
        }
        // mixed path: both sets of pass constants (the FP64 ones serve a fit the guard moved to FP64)
        if (PREC == PREC_MIXED) {
            if (threadIdx.x < PF) sm.pf[threadIdx.x] = __ldcg(stp->pf + threadIdx.x);
            else if (threadIdx.x < PF + PD) sm.pd[threadIdx.x - PF] = __ldcg(stp->pd + threadIdx.x - PF);
        } else if (threadIdx.x < PD) {
            sm.pd[threadIdx.x] = __ldcg(stp->pd + threadIdx.x);
        }
        if (fit != sm.desc_fit) {
            const int* src = (const int*)(E.desc + fit);
            int* dst = (int*)&sm.desc;
            for (int k = threadIdx.x; k < (int)(sizeof(FitDesc) / 4); k += EVAL_THREADS) dst[k] = src[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) sm.desc_fit = fit;
        MS::dispatch(sm.desc.model,
                     [&](auto m) { process_item<decltype(m), PREC, MS>(sm, E, fit, tile, R, (long long)clock64()); });
        __syncthreads();
        busy += global_ns() - t1;
    }
    if (threadIdx.x == 0) {
        atomicAdd(acct, busy);
        atomicAdd(acct + 1, idle);
        const int c = *ctl;
        if (c & CTL_ABORT) atomicOr(E.out + 2, 1);
        E.out[0] = *(volatile int*)E.running;   // 0 unless aborted
        E.out[1] = 1;
    }
}

// Persistent form of the iteration: pass constants at p0 (do_init), then
// rounds of run_items separated by the grid barrier until no fit runs or the
// round cap is reached.  One cooperative launch replaces a graph of
// per-round kernels.
template <int PREC, class MS>
__global__ void __launch_bounds__(EVAL_THREADS, 2) fit_loop_kernel(const Engine* __restrict__ Ep, int do_init) {
    __shared__ RoundSmem sm;
    extern __shared__ __align__(128) float ring_buf[];
    const unsigned long long t_launch = global_ns();
    stage_engine(sm, Ep);
    const Engine& E = sm.eng;
    Engine* Ed = const_cast<Engine*>(Ep);
    RingState R;
    round_setup<PREC>(sm, ring_buf, R);
    // This CTA's rank among all CTAs ordered by (slot on its SM, SM id), so
    // that work items 0, 1, 2, ... land on distinct SMs before any SM gets a
    // second one (a fit with fewer tiles than SMs gets one SM per tile).
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        sm.flag[0] = (int)smid;
        sm.flag[1] = atomicAdd(E.sm_cnt + (smid < SM_IDS ? smid : SM_IDS - 1), 1);
    }
    if (do_init) {
        // pass constants at p0 (strided by block index: needs no rank), published by the rank barrier
        int nf = *E.nfits_dev;
        for (int f = blockIdx.x; f < nf; f += gridDim.x) {
            if (threadIdx.x < 32) {
                const FitDesc& d = E.desc[f];
                FitState* st = E.state + f;
                int l = threadIdx.x;
                if (l < 8) { sm.trf.vec[VX][l] = (l < d.n) ? st->x[l] : 0.0; sm.trf.vec[VXT][l] = sm.trf.vec[VX][l]; }
                __syncwarp();
                prep_pass<PREC, MS>(d, st, sm.trf);
            }
            __syncthreads();
        }
    }
    if (grid_round_end(Ed, E, &sm.ctl, false)) return;
    int first;
    {
        const int smid = sm.flag[0], slot = sm.flag[1];
        unsigned nsm;
        asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsm));
        nsm = nsm < SM_IDS ? nsm : SM_IDS;
        int part = 0;
        for (int k = threadIdx.x; k < (int)nsm; k += blockDim.x) {
            int c = __ldcg(E.sm_cnt + k);
            part += min(c, slot) + ((k < smid && c > slot) ? 1 : 0);
        }
        for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
        __syncthreads();                                  // flag[0..1] read by every thread
        if (threadIdx.x == 0) sm.flag[2] = 0;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) atomicAdd(&sm.flag[2], part);
        __syncthreads();
        first = sm.flag[2];
    }
    // time accounting of the loop (result header, 64-bit words 2..3):
    // per-CTA time in rounds' work and time waiting at the barrier
    unsigned long long* acct = reinterpret_cast<unsigned long long*>(E.out) + 2;
    if (E.queue_mode) {
        queue_loop<PREC, MS>(sm, E, Ed, R, first, acct);
        if (first == 0)
            for (int k = threadIdx.x; k <= SM_IDS; k += blockDim.x) E.sm_cnt[k] = 0;
        return;
    }
    // owner mode: the owner CTA of a fit also times its rounds (global timer)
    unsigned long long* otrace = (E.owner_mode && first < *E.nfits_dev) ? E.state[first].trace : nullptr;
    if (otrace && threadIdx.x == 0) trace_bump(otrace, TR_START_NS, global_ns() - t_launch);
    while (true) {
        unsigned long long t0 = global_ns();
        run_items<PREC, MS>(sm, E, R, first, E.sm_cnt + SM_IDS);
        if (E.owner_mode) owner_steps<PREC, MS>(sm, E, Ed, first);
        unsigned long long t1 = global_ns();
        int c = grid_round_end(Ed, E, &sm.ctl, true);
        if (threadIdx.x == 0) {
            const unsigned long long t2 = global_ns();
            atomicAdd(acct, t1 - t0);
            atomicAdd(acct + 1, t2 - t1);
            if (otrace) {
                trace_bump(otrace, TR_ROUND_NS, t1 - t0);
                trace_bump(otrace, TR_BARRIER_NS, t2 - t1);
            }
        }
        if (c) break;
    }
    // every CTA has read the counters (before the first round): rank 0 clears them for the next launch
    if (first == 0)
        for (int k = threadIdx.x; k <= SM_IDS; k += blockDim.x) E.sm_cnt[k] = 0;
}

// Pass constants for the first evaluation (at p0): base = trial = p0.
template <int PREC, class MS>
__global__ void init_fits_kernel(const Engine* __restrict__ Ep) {
    __shared__ TrfSmem S;
    const Engine E = *Ep;
    int nf = E.nfits_dev ? *E.nfits_dev : 0;
    for (int f = blockIdx.x; f < nf; f += gridDim.x) {
        const FitDesc& d = E.desc[f];
        FitState* st = E.state + f;
        int l = threadIdx.x;
        if (l < 8) { S.vec[VX][l] = (l < d.n) ? st->x[l] : 0.0; S.vec[VXT][l] = S.vec[VX][l]; }
        __syncwarp();
        prep_pass<PREC, MS>(d, st, S);
        __syncwarp();
    }
}

// Pass constants at p0 for the listed fits only (serving: newly admitted
// fits join while others are mid-fit).
template <int PREC, class MS>
__global__ void init_slots_kernel(const Engine* __restrict__ Ep, const int* __restrict__ slots, int count) {
    __shared__ TrfSmem S;
    const Engine E = *Ep;
    for (int k = blockIdx.x; k < count; k += gridDim.x) {
        int f = slots[k];
        const FitDesc& d = E.desc[f];
        FitState* st = E.state + f;
        int l = threadIdx.x;
        if (l < 8) { S.vec[VX][l] = (l < d.n) ? st->x[l] : 0.0; S.vec[VXT][l] = S.vec[VX][l]; }
        __syncwarp();
        prep_pass<PREC, MS>(d, st, S);
        __syncwarp();
    }
}

}  // namespace gbfit

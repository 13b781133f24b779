// Host side of libgbfit: argument checking, device workspace and the
// extern "C" entry points declared in gbfit.h.
//
// One fit or a batch of fits runs as ONE cooperative launch of the
// persistent loop kernel (fit_loop_kernel): pass constants at p0, then
// rounds (one TRF iteration of every running fit each) separated by a
// grid-wide barrier, until no fit runs or the round cap is reached.  One
// host-to-device copy of the job image before it, one device-to-host copy of
// the per-fit results after it.  On GB300 a kernel boundary plus a graph
// WHILE trip cost several microseconds per iteration; the barrier costs
// about one.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gbfit.h"
#include "kernels.cuh"
#include "models.cuh"
#include "user_models.h"
#include <map>
#include <utility>

using namespace gbfit;

namespace {

constexpr int TILE_MIN = 2048, TILE_MAX = 65536, TILE_SPLIT = 304;   // TILE_SPLIT: grid when none is known
constexpr size_t OWNER_MAX_FITS = 8;            // launches of at most this many fits use owner mode
constexpr bool QUEUE_MODE = true;               // larger launches run without lock-step rounds

thread_local std::string g_err;

std::mutex g_stats_mu;
gbfit_stats g_stats = {};
int g_profiling = 0;
// profiling: the stream is held this long before a timed launch's start event
// (longer than the host's submission of the launch that follows it)
constexpr unsigned long long PROFILE_HOLD_NS = 60000;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

}  // namespace

namespace gbfit {

// NVTX ranges around each call and its phases (staging, the loop launch, the
// result copy; the server's retire / admit / launch), for timelines in
// Nsight tools; free when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
int set_error(int code, const char* msg) {
    g_err = msg;
    return code;
}
}  // namespace gbfit

namespace {

#define CUDA_TRY(x)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (x);                                                                \
        if (e_ != cudaSuccess) return fail(GBFIT_E_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
int grow_dev(T*& p, size_t& cap, size_t need, bool& changed) {
    if (need <= cap && p) return GBFIT_OK;
    size_t n = need > 16 ? need + need / 2 : 16;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc((void**)&p, n * sizeof(T));
    if (e != cudaSuccess) { p = nullptr; return fail(GBFIT_E_OOM, "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e)); }
    cap = n;
    changed = true;
    return GBFIT_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte layout of one call's job buffer: what the host uploads ([0, res_hdr))
// and what it reads back ([res_hdr, end)) are each one contiguous copy.
struct JobLayout {
    size_t eng, desc, state, items, gcnt, fcnt, smcnt, bits, ntc, res_hdr, res, end;
    JobLayout(size_t nf, size_t ntiles, size_t ngroups) {
        size_t o = 0;
        eng = o;     o += align256(sizeof(Engine));
        desc = o;    o += align256(nf * sizeof(FitDesc));
        state = o;   o += align256(nf * sizeof(FitState));
        items = o;   o += align256(ntiles * sizeof(WorkItem));
        gcnt = o;    o += align256(ngroups * sizeof(int));
        fcnt = o;    o += align256(nf * sizeof(int));
        smcnt = o;   o += align256((SM_IDS + 1) * sizeof(int));
        bits = o;    o += align256((nf + 31) / 32 * sizeof(unsigned));
        ntc = o;     o += align256(nf * sizeof(int));
        res_hdr = o; o += 256;
        res = o;     o += align256(nf * sizeof(FitResult));
        end = o;
    }
};

struct Ctx {
    int device = -1, sms = 0, grid_p[2] = {0, 0};
    std::mutex mu;
    char* job = nullptr; size_t cap_job = 0;   // Engine header + per-fit records
    double* tile_part_d = nullptr; size_t cap_tpd = 0;
    double* group_part = nullptr; size_t cap_gp = 0;
    double* wbuf = nullptr; size_t cap_w = 0;
    char* databuf = nullptr; size_t cap_data = 0;
    double* small = nullptr;      // subproblem scratch
    // full covariance: C -> L in place, 1 / L_kk, X = L^-1 (FP64 and FP32),
    // the per-point columns of the evaluation round, barrier words + flag
    double* cov_a = nullptr; size_t cap_cov_a = 0;
    double* cov_rd = nullptr; size_t cap_cov_rd = 0;
    double* cov_x = nullptr; size_t cap_cov_x = 0;
    float* cov_xf = nullptr; size_t cap_cov_xf = 0;
    double* cov_h = nullptr; size_t cap_cov_h = 0;
    int* cov_sync = nullptr; size_t cap_cov_sync = 0;
    // pinned host staging
    char* hbuf = nullptr; size_t hcap = 0;
    // one-node graphs holding the cooperative loop launch, per precision (a
    // graph launch costs the host less than a direct cooperative launch);
    // bound to the job buffer's address
    std::map<std::pair<int, int>, cudaGraphExec_t> loop_exec;   // (kernel set, precision)
    void drop_graphs() {
        for (auto& kv : loop_exec) cudaGraphExecDestroy(kv.second);
        loop_exec.clear();
    }

    Engine* eng_dev() const { return (Engine*)job; }
    Engine engine(const JobLayout& L) const {
        Engine E;
        memset(&E, 0, sizeof E);
        Engine* ed = eng_dev();
        E.results = (FitResult*)(job + L.res);
        E.out = (int*)(job + L.res_hdr);
        E.desc = (FitDesc*)(job + L.desc);
        E.state = (FitState*)(job + L.state);
        E.items = (WorkItem*)(job + L.items);
        E.group_cnt = (int*)(job + L.gcnt);
        E.fit_cnt = (int*)(job + L.fcnt);
        E.sm_cnt = (int*)(job + L.smcnt);
        E.fit_bits = (unsigned*)(job + L.bits);
        E.next_tile = (int*)(job + L.ntc);
        E.tile_part_d = tile_part_d; E.group_part = group_part;
        E.n_items = &ed->sc[0]; E.running = &ed->sc[1]; E.rounds = &ed->sc[2];
        E.max_rounds = &ed->sc[3]; E.nfits_dev = &ed->sc[4];
        return E;
    }
    int pinned(size_t need) {
        if (need <= hcap) return GBFIT_OK;
        if (hbuf) cudaFreeHost(hbuf);
        hbuf = nullptr; hcap = 0;
        size_t n = need + need / 2 + 4096;
        cudaError_t e = cudaMallocHost((void**)&hbuf, n);
        if (e != cudaSuccess) return fail(GBFIT_E_OOM, "cudaMallocHost(%zu): %s", n, cudaGetErrorString(e));
        hcap = n;
        return GBFIT_OK;
    }
};

std::mutex g_ctx_mu;
Ctx* g_ctx[64] = {};

int get_ctx(Ctx** out) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(GBFIT_E_CUDA, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> g(g_ctx_mu);
    if (!g_ctx[dev]) {
        Ctx* c = new Ctx();
        c->device = dev;
        cudaDeviceProp prop;
        cudaError_t e = cudaGetDeviceProperties(&prop, dev);
        if (e != cudaSuccess) { delete c; return fail(GBFIT_E_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e)); }
        c->sms = prop.multiProcessorCount;
        int b0 = eval_blocks_per_sm(PREC_FP64), b1 = eval_blocks_per_sm(PREC_MIXED);
        c->grid_p[PREC_FP64] = c->sms * (b0 < 1 ? 1 : b0);
        c->grid_p[PREC_MIXED] = c->sms * (b1 < 1 ? 1 : b1);
        e = cudaMalloc((void**)&c->small, 256 * sizeof(double));
        if (e != cudaSuccess) { delete c; return fail(GBFIT_E_OOM, "cudaMalloc: %s", cudaGetErrorString(e)); }
        g_ctx[dev] = c;
    }
    *out = g_ctx[dev];
    return GBFIT_OK;
}

int ensure(Ctx* c, const JobLayout& L, size_t ntiles, size_t ngroups) {
    bool job_changed = false, scratch_changed = false;
    int rc;
    if ((rc = grow_dev(c->job, c->cap_job, L.end, job_changed))) return rc;
    if ((rc = grow_dev(c->tile_part_d, c->cap_tpd, ntiles * KMAX, scratch_changed))) return rc;
    if ((rc = grow_dev(c->group_part, c->cap_gp, ngroups * KMAX, scratch_changed))) return rc;
    if (job_changed) c->drop_graphs();
    return GBFIT_OK;
}

// Cooperative grid of a kernel set's loop kernel: every CTA resident.
int loop_grid(const Ctx* c, const KernelSet* ks, int prec) {
    int b = ks->blocks_per_sm[prec];
    return c->sms * (b < 1 ? 1 : b);
}

// The cooperative loop launch (pass constants at p0, then rounds) as a
// cached one-node graph.
int loop_graph(Ctx* c, const KernelSet* ks, int prec, cudaGraphExec_t* out) {
    auto key = std::make_pair(ks->id, prec);
    auto it = c->loop_exec.find(key);
    if (it == c->loop_exec.end()) {
        cudaGraph_t g;
        CUDA_TRY(cudaGraphCreate(&g, 0));
        Engine* Ed = c->eng_dev();
        int do_init = 1;
        void* args[] = {&Ed, &do_init};
        cudaKernelNodeParams kp = {};
        kp.func = (void*)ks->fit_loop[prec];
        kp.gridDim = dim3(loop_grid(c, ks, prec));
        kp.blockDim = dim3(EVAL_THREADS);
        kp.sharedMemBytes = (unsigned)ks->dyn_smem[prec];
        kp.kernelParams = args;
        cudaGraphNode_t node;
        cudaError_t e = cudaGraphAddKernelNode(&node, g, nullptr, 0, &kp);
        cudaLaunchAttributeValue v;
        memset(&v, 0, sizeof v);
        v.cooperative = 1;
        if (e == cudaSuccess) e = cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeCooperative, &v);
        cudaGraphExec_t ex = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(GBFIT_E_CUDA, "loop graph: %s", cudaGetErrorString(e));
        it = c->loop_exec.emplace(key, ex).first;
    }
    *out = it->second;
    return GBFIT_OK;
}

bool is_device_ptr(const void* p) {
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Tile of a single fit spread over a grid of `grid` CTAs: the fewest rounds
// k of at most TILE_MAX-point tiles per CTA, then tiles of m / (grid k)
// points, so that every CTA gets k or k - 1 tiles.
int choose_tile(int64_t m, int user, int grid) {
    if (user > 0) return ((user + EVAL_THREADS - 1) / EVAL_THREADS) * EVAL_THREADS;
    const int64_t G = grid > 0 ? grid : TILE_SPLIT;
    int64_t k = (m + G * TILE_MAX - 1) / (G * TILE_MAX);
    if (k < 1) k = 1;
    int64_t t = (m + G * k - 1) / (G * k);
    t = ((t + EVAL_THREADS - 1) / EVAL_THREADS) * EVAL_THREADS;
    if (t < TILE_MIN) t = TILE_MIN;
    if (t > TILE_MAX) t = TILE_MAX;
    return (int)t;
}

// ---- tile table of batched and served fits (gbfit_tune_*)
// Largest default / autotuned tile of mixed-precision fits: a fit that the
// precision guard moves to FP64 passes keeps its tiles, and an FP64 pass over
// a large FP32-sized tile holds one CTA for ~1 ms (FP64 issues at 1/64 of
// FP32 on GB300), lengthening that fit's chain of evaluations.
constexpr int MIXED_TILE_CAP = 4096;
std::mutex g_tune_mu;
gbfit_tune_table g_tune = [] {
    gbfit_tune_table t;
    for (int mo = 0; mo < GBFIT_NUM_MODELS; ++mo)
        for (int b = 0; b < GBFIT_TUNE_BUCKETS; ++b) {
            t.tile_points[mo][PREC_MIXED][b] = MIXED_TILE_CAP;
            t.tile_points[mo][PREC_FP64][b] = 4096;
            t.group_tiles[mo][PREC_MIXED][b] = t.group_tiles[mo][PREC_FP64][b] = GROUP_TILES;
        }
    return t;
}();

int tune_bucket(int64_t m) {
    int b = 0;
    while (b + 1 < GBFIT_TUNE_BUCKETS && (m >> (b + 1)) > 0) ++b;
    return b;
}

// Shape of a batched / served fit: user values where given, else the table;
// a fit smaller than its tile is one tile.
void multi_shape(int model, int prec, int64_t m, int user_tile, int user_group, int* tile, int* group) {
    int t = prec == PREC_MIXED ? MIXED_TILE_CAP : 4096, g = GROUP_TILES;   // user models: the table's defaults
    if (model >= 0 && model < GBFIT_NUM_MODELS) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        int b = tune_bucket(m);
        t = g_tune.tile_points[model][prec][b];
        g = g_tune.group_tiles[model][prec][b];
    }
    if (user_tile > 0) t = ((user_tile + EVAL_THREADS - 1) / EVAL_THREADS) * EVAL_THREADS;
    else if (t >= m) t = (int)(((m + EVAL_THREADS - 1) / EVAL_THREADS) * EVAL_THREADS);
    if (user_group > 0) g = user_group;
    *tile = t;
    *group = g;
}

struct FitArgs {
    int model, n, layout, dtype;
    int64_t m, grid_w;
    const void *x, *x2, *y, *sigma;
    const double *p0, *lb, *ub;
};

int check_params(const FitArgs& a, bool* bounded) {
    *bounded = false;
    for (int i = 0; i < a.n; ++i) {
        if (!std::isfinite(a.p0[i])) return fail(GBFIT_E_INVALID_ARG, "p0[%d] is not finite", i);
        double lo = a.lb ? a.lb[i] : -INFINITY, hi = a.ub ? a.ub[i] : INFINITY;
        if (std::isnan(lo) || std::isnan(hi)) return fail(GBFIT_E_INVALID_ARG, "bound %d is NaN", i);
        if (!(lo < hi)) return fail(GBFIT_E_INVALID_ARG, "lb[%d] >= ub[%d]", i, i);
        if (std::isfinite(lo) || std::isfinite(hi)) *bounded = true;
        if (!(a.p0[i] > lo && a.p0[i] < hi))
            return fail(GBFIT_E_INFEASIBLE_X0, "p0[%d] = %g is not strictly inside (%g, %g)", i, a.p0[i], lo, hi);
    }
    return GBFIT_OK;
}

int check_opts(const gbfit_options* o, int n) {
    if (!(o->ftol >= 0) || !(o->xtol >= 0) || !(o->gtol >= 0)) return fail(GBFIT_E_INVALID_ARG, "tolerances must be >= 0");
    if (o->precision != GBFIT_PREC_FP64 && o->precision != GBFIT_PREC_MIXED) return fail(GBFIT_E_INVALID_ARG, "unknown precision %d", o->precision);
    if (o->x_scale && !o->x_scale_jac)
        for (int i = 0; i < n; ++i)
            if (!(o->x_scale[i] > 0) || !std::isfinite(o->x_scale[i])) return fail(GBFIT_E_INVALID_ARG, "x_scale[%d] must be > 0", i);
    if (o->tile_points < 0 || o->tile_points > (1 << 24)) return fail(GBFIT_E_INVALID_ARG, "tile_points out of range");
    if (o->group_tiles < 0 || o->group_tiles > 1024) return fail(GBFIT_E_INVALID_ARG, "group_tiles out of range");
    if (o->loss < GBFIT_LOSS_LINEAR || o->loss > GBFIT_LOSS_ARCTAN) return fail(GBFIT_E_INVALID_ARG, "unknown loss %d", o->loss);
    if (!(o->f_scale >= 0) || !std::isfinite(o->f_scale)) return fail(GBFIT_E_INVALID_ARG, "f_scale must be > 0");
    if (std::isnan(o->guard_cond) || std::isnan(o->guard_floor))
        return fail(GBFIT_E_INVALID_ARG, "guard_cond and guard_floor must not be NaN");
    if (std::isnan(o->wait_limit_s) || o->wait_limit_s > 3600.0)
        return fail(GBFIT_E_INVALID_ARG, "wait_limit_s must be a number of seconds <= 3600");
    return GBFIT_OK;
}

gbfit_options defaults() {
    gbfit_options o;
    memset(&o, 0, sizeof o);
    o.ftol = o.xtol = o.gtol = 1e-8;
    o.precision = GBFIT_PREC_MIXED;
    o.f_scale = 1.0;
    o.guard_cond = GBFIT_GUARD_COND_DEFAULT;
    o.guard_floor = GBFIT_GUARD_FLOOR_DEFAULT;
    return o;
}

// Guard thresholds as used: <= 0 reads as the default, +inf is off.
double guard_value(double v, double dflt) { return v > 0.0 ? v : dflt; }

// Run nfits fits whose descriptors (data pointers already on the device) are
// in hd[]; writes per-fit results into hr[].  One host-to-device copy of the
// job buffer, one loop-kernel launch, one device-to-host copy of the results.
int run_fits(Ctx* c, const KernelSet* ks, int prec, std::vector<FitDesc>& hd, const std::vector<std::vector<double>>& p0s,
             std::vector<FitResult>& hr, cudaStream_t s, int* rounds_out) {
    NvtxRange nv("gbfit.run_fits");
    const auto t_host0 = std::chrono::steady_clock::now();
    size_t nf = hd.size();
    size_t ntiles = 0, ngroups = 0;
    int max_nfev = 1;
    bool any_cov = false;
    for (auto& d : hd) {
        d.tile_base = (int64_t)ntiles;
        d.group_base = (int64_t)ngroups;
        ntiles += d.n_tiles;
        ngroups += d.n_groups;
        if (d.max_nfev > max_nfev) max_nfev = d.max_nfev;
        any_cov = any_cov || d.cov;
    }
    JobLayout L(nf, ntiles, ngroups);
    int rc;
    if ((rc = ensure(c, L, ntiles, ngroups))) return rc;
    if ((rc = c->pinned(L.end))) return rc;
    char* hb = c->hbuf;
    memset(hb, 0, L.res_hdr + 32);                  // the job image plus a zeroed result header
    Engine E = c->engine(L);
    for (size_t f = 0; f < nf; ++f)                 // the launch's grid-wide waits: the smallest limit asked
        if (hd[f].wait_ns && (!E.wait_ns || hd[f].wait_ns < E.wait_ns)) E.wait_ns = hd[f].wait_ns;
    E.sc[0] = (int)ntiles;
    E.sc[1] = (int)nf;
    E.sc[2] = 0;
    E.sc[3] = any_cov ? 2 * max_nfev + 6 : max_nfev + 4;   // rounds per evaluation (2 for covariance fits), plus slack
    E.sc[4] = (int)nf;
    // few fits: each fit's combine and step stay on one CTA (warm code and state);
    // many fits: no lock-step rounds (a fit's tiles are re-armed by its own step)
    E.owner_mode = (nf <= OWNER_MAX_FITS && !any_cov) ? 1 : 0;
    E.queue_mode = (QUEUE_MODE && nf > OWNER_MAX_FITS && !any_cov) ? 1 : 0;
    memcpy(hb + L.eng, &E, sizeof E);
    memcpy(hb + L.desc, hd.data(), nf * sizeof(FitDesc));
    {
        unsigned* bits = (unsigned*)(hb + L.bits);     // every fit starts with all its tiles claimable
        for (size_t w = 0; w < (nf + 31) / 32; ++w)
            bits[w] = (w + 1) * 32 <= nf ? 0xffffffffu : ((1u << (nf % 32)) - 1u);
    }
    FitState* hs = (FitState*)(hb + L.state);
    WorkItem* hi = (WorkItem*)(hb + L.items);
    size_t k = 0;
    for (size_t f = 0; f < nf; ++f) {
        FitState& st = hs[f];
        st.run = RS_RUNNING;
        st.phase = PH_INIT;
        for (int i = 0; i < hd[f].n; ++i) { st.x[i] = p0s[f][i]; st.xt[i] = p0s[f][i]; st.scale_inv[i] = 1.0; }
        // covariance row items cost in proportion to their index: largest first
        for (int t = 0; t < hd[f].n_tiles; ++t) hi[k++] = WorkItem{(int)f, hd[f].cov ? hd[f].n_tiles - 1 - t : t};
    }
    // one upload: the image and the zeroed header words out[] (running, rounds, abort; busy / wait ns)
    CUDA_TRY(cudaMemcpyAsync(c->job, hb, L.res_hdr + 32, cudaMemcpyHostToDevice, s));
    double eval_ms = 0.0;
    int64_t eval_launches = 0;
    {
        cudaGraphExec_t ex;
        if ((rc = loop_graph(c, ks, prec, &ex))) return rc;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (g_profiling) {
            CUDA_TRY(cudaEventCreate(&e0));
            CUDA_TRY(cudaEventCreate(&e1));
            // the GPU stays busy while the launch is submitted: the events time the kernel
            CUDA_TRY(launch_hold(PROFILE_HOLD_NS, s));
            CUDA_TRY(cudaEventRecord(e0, s));
        }
        {
            NvtxRange nvl("gbfit.loop_launch");
            CUDA_TRY(cudaGraphLaunch(ex, s));
        }
        if (g_profiling) {
            CUDA_TRY(cudaEventRecord(e1, s));
            CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            eval_ms = ms;
            eval_launches = 1;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
    }
    CUDA_TRY(cudaMemcpyAsync(hb + L.res_hdr, c->job + L.res_hdr, L.end - L.res_hdr, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const int* outsc = (const int*)(hb + L.res_hdr);
    int running = outsc[0], rounds = outsc[1];
    if (outsc[2]) return fail(GBFIT_E_TIMEOUT, "a round barrier of the loop kernel timed out");
    const unsigned long long* acct = (const unsigned long long*)(hb + L.res_hdr) + 2;
    hr.resize(nf);
    memcpy(hr.data(), hb + L.res, nf * sizeof(FitResult));
    if (rounds_out) *rounds_out = rounds;
    {
        std::lock_guard<std::mutex> g(g_stats_mu);
        g_stats.calls += 1;
        g_stats.host_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_host0).count();
        g_stats.fits += (int64_t)nf;
        g_stats.kernel_launches += 1;
        g_stats.graph_rounds += rounds;
        g_stats.eval_ms += eval_ms;
        g_stats.eval_launches += eval_launches;
        g_stats.loop_busy_ms += acct[0] * 1e-6;
        g_stats.loop_wait_ms += acct[1] * 1e-6;
        g_stats.loop_ctas += loop_grid(c, ks, prec);
        for (size_t f = 0; f < nf; ++f) {
            for (int k = 0; k < 32; ++k) g_stats.phase_cycles[k] += hr[f].trace[k];
            g_stats.passes += hr[f].nfev;
            g_stats.point_passes += double(hd[f].m) * hr[f].nfev;
        }
    }
    if (!g_profiling && running != 0) return fail(GBFIT_E_TIMEOUT, "%d fit(s) still running after the round cap", running);
    return GBFIT_OK;
}

// Stage data arrays that live in host memory into the device buffer.
struct Staged {
    const void *x = nullptr, *x2 = nullptr, *y = nullptr, *sigma = nullptr;
};

int stage_data(Ctx* c, const void* x, size_t xbytes, const void* y, size_t ybytes, const void* sg, size_t sbytes,
               cudaStream_t s, Staged* out) {
    NvtxRange nv("gbfit.stage_data");
    bool hx = x && !is_device_ptr(x), hy = !is_device_ptr(y), hsg = sg && !is_device_ptr(sg);
    out->x = x; out->y = y; out->sigma = sg;
    size_t need = (hx ? xbytes + 256 : 0) + (hy ? ybytes + 256 : 0) + (hsg ? sbytes + 256 : 0);
    if (need == 0) return GBFIT_OK;
    bool changed = false;
    int rc = grow_dev(c->databuf, c->cap_data, need, changed);
    if (rc) return rc;
    size_t off = 0;
    auto put = [&](const void* src, size_t nb, const void** dst) -> int {
        char* d = c->databuf + off;
        CUDA_TRY(cudaMemcpyAsync(d, src, nb, cudaMemcpyHostToDevice, s));
        *dst = d;
        off += (nb + 255) / 256 * 256;
        return GBFIT_OK;
    };
    if (hx && (rc = put(x, xbytes, &out->x))) return rc;
    if (hy && (rc = put(y, ybytes, &out->y))) return rc;
    if (hsg && (rc = put(sg, sbytes, &out->sigma))) return rc;
    return GBFIT_OK;
}

// multi: the fit runs beside others (batched or served) and takes its shape
// from the tile table; otherwise its tiles spread over every SM.
int fill_desc(FitDesc& d, const FitArgs& a, const gbfit_options& o, bool bounded, int64_t m, bool multi,
              int grid = 0) {
    memset(&d, 0, sizeof d);
    d.model = a.model; d.n = a.n; d.layout = a.layout; d.dtype = a.dtype;
    d.prec = o.precision; d.bounded = bounded ? 1 : 0; d.jac_scale = o.x_scale_jac ? 1 : 0;
    d.m = m; d.grid_w = a.grid_w;
    if (multi) {
        multi_shape(a.model, o.precision, m, o.tile_points, o.group_tiles, &d.tile_points, &d.group_tiles);
    } else {
        d.tile_points = choose_tile(m, o.tile_points, grid);
        d.group_tiles = o.group_tiles > 0 ? o.group_tiles : GROUP_TILES;
    }
    d.n_tiles = (int)((m + d.tile_points - 1) / d.tile_points);
    d.n_groups = (d.n_tiles + d.group_tiles - 1) / d.group_tiles;
    d.max_nfev = o.max_nfev > 0 ? o.max_nfev : 100 * a.n;
    for (int i = 0; i < NMAX; ++i) {
        d.lb[i] = (a.lb && i < a.n) ? a.lb[i] : -INFINITY;
        d.ub[i] = (a.ub && i < a.n) ? a.ub[i] : INFINITY;
        d.xscale[i] = (o.x_scale && i < a.n && !o.x_scale_jac) ? o.x_scale[i] : 1.0;
    }
    d.ftol = o.ftol; d.xtol = o.xtol; d.gtol = o.gtol;
    d.absolute_sigma = o.absolute_sigma;
    d.loss = o.loss;
    d.f_scale = o.f_scale > 0 ? o.f_scale : 1.0;
    // precision guard: mixed path with the linear loss (make_cov turns it off)
    const bool gfit = o.precision == GBFIT_PREC_MIXED && o.loss == GBFIT_LOSS_LINEAR;
    d.guard_cond = gfit ? guard_value(o.guard_cond, GBFIT_GUARD_COND_DEFAULT) : INFINITY;
    d.guard_floor = gfit ? guard_value(o.guard_floor, GBFIT_GUARD_FLOOR_DEFAULT) : INFINITY;
    d.wait_ns = o.wait_limit_s > 0.0 ? (unsigned long long)std::max(1.0, o.wait_limit_s * 1e9) : 0ull;
    return GBFIT_OK;
}

// Set data pointers and weights of d (after staging); plain path stages w = 1/sigma.
int set_data(Ctx* c, FitDesc& d, const void* x, const void* x2, const void* y, const void* sigma,
             int64_t w_offset, cudaStream_t s) {
    d.x = x; d.x2 = x2; d.y = y;
    if (!sigma) { d.wkind = W_NONE; d.w = nullptr; return GBFIT_OK; }
    if (d.prec == PREC_MIXED) { d.wkind = W_SIGMA; d.w = sigma; return GBFIT_OK; }
    d.wkind = W_ARRAY;              // staged FP64 w = 1/sigma
    d.w = c->wbuf + w_offset;
    return GBFIT_OK;
}

// Full covariance (Appendix C): copy C to the device, factor C = L L^T and
// form X = L^-1 there (cov_kernels.cu), and turn the descriptor into a
// covariance fit: 32-point items, rounds alternating between evaluating
// points and reducing rows of X [h - y, J].  One D2H read of the factor's
// status word (a synchronisation) before the fit.
int stage_cov(Ctx* c, FitDesc& d, const double* cov, int64_t m, int n, cudaStream_t s) {
    NvtxRange nv("gbfit.stage_cov");
    bool ch = false;
    int rc;
    const size_t mp = cov_padded((int)m);
    const size_t mm = (size_t)m * (size_t)m;
    if ((rc = grow_dev(c->cov_a, c->cap_cov_a, mp * mp, ch))) return rc;
    if ((rc = grow_dev(c->cov_x, c->cap_cov_x, mp * mp, ch))) return rc;
    if ((rc = grow_dev(c->cov_rd, c->cap_cov_rd, mp * 32, ch))) return rc;
    if (d.prec == PREC_MIXED && (rc = grow_dev(c->cov_xf, c->cap_cov_xf, mm, ch))) return rc;
    if ((rc = grow_dev(c->cov_h, c->cap_cov_h, (size_t)(n + 2) * (size_t)m, ch))) return rc;
    if ((rc = grow_dev(c->cov_sync, c->cap_cov_sync, (size_t)4, ch))) return rc;
    const bool dev = is_device_ptr(cov);
    CUDA_TRY(cudaMemsetAsync(c->cov_a, 0, mp * mp * sizeof(double), s));
    CUDA_TRY(cudaMemcpy2DAsync(c->cov_a, mp * sizeof(double), cov, (size_t)m * sizeof(double),
                               (size_t)m * sizeof(double), (size_t)m,
                               dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemsetAsync(c->cov_x, 0, mp * mp * sizeof(double), s));
    CUDA_TRY(cudaMemsetAsync(c->cov_sync, 0, 4 * sizeof(int), s));
    // the compact FP64 inverse reuses the factor's storage (read before it is overwritten)
    CUDA_TRY(launch_cov_factor(c->cov_a, c->cov_rd, c->cov_x, c->cov_a, d.prec == PREC_MIXED ? c->cov_xf : nullptr,
                               (int)m, (unsigned*)c->cov_sync, c->cov_sync + 2, c->sms, s));
    int flag = 0;
    CUDA_TRY(cudaMemcpyAsync(&flag, c->cov_sync + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    {
        std::lock_guard<std::mutex> g(g_stats_mu);
        g_stats.kernel_launches += 3;
    }
    if (flag & 1) return fail(GBFIT_E_INVALID_ARG, "the covariance matrix is not positive definite");
    if (flag & 2) return fail(GBFIT_E_TIMEOUT, "a grid barrier of the covariance factorisation timed out");
    d.cov = 1;
    d.guard_cond = d.guard_floor = INFINITY;       // the guard's FP64 passes do not cover covariance fits
    d.xinv = d.prec == PREC_MIXED ? (const void*)c->cov_xf : (const void*)c->cov_a;
    d.hbuf = c->cov_h;
    d.wkind = W_NONE;
    d.w = nullptr;
    d.tile_points = COV_ROWS;
    d.n_tiles = (int)((m + COV_ROWS - 1) / COV_ROWS);
    d.n_groups = (d.n_tiles + d.group_tiles - 1) / d.group_tiles;
    return GBFIT_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

int gbfit_version(void) { return GBFIT_VERSION; }

const char* gbfit_last_error(void) { return g_err.c_str(); }

int gbfit_default_options(gbfit_options* opt) {
    if (!opt) return fail(GBFIT_E_INVALID_ARG, "opt is NULL");
    *opt = defaults();
    return GBFIT_OK;
}

int gbfit_model_info(int model_id, int* n_params, int* x_dims) {
    int n, xd;
    if (!model_shape(model_id, &n, &xd)) return fail(GBFIT_E_INVALID_ARG, "unknown model %d", model_id);
    if (n_params) *n_params = n;
    if (x_dims) *x_dims = xd;
    return GBFIT_OK;
}

static int check_common(int model_id, int x_layout, int dtype, const void* ydata, int* n) {
    int xd;
    if (!model_shape(model_id, n, &xd)) return fail(GBFIT_E_INVALID_ARG, "unknown model %d", model_id);
    if (dtype != GBFIT_F32 && dtype != GBFIT_F64) return fail(GBFIT_E_INVALID_ARG, "unknown dtype %d", dtype);
    if (xd == 1 && x_layout != GBFIT_X_VEC) return fail(GBFIT_E_INVALID_ARG, "1D model needs GBFIT_X_VEC");
    if (xd == 2 && x_layout != GBFIT_X_SOA2 && x_layout != GBFIT_X_GRID)
        return fail(GBFIT_E_INVALID_ARG, "2D model needs GBFIT_X_SOA2 or GBFIT_X_GRID");
    if (!ydata) return fail(GBFIT_E_INVALID_ARG, "ydata is NULL");
    return GBFIT_OK;
}

// Shared body of gbfit_curve_fit and gbfit_evaluate (single fit).
static int single_fit(int model_id, const void* xdata, int64_t m, int x_layout, const int64_t* grid_wh,
                      const void* ydata, const void* sigma, int dtype, const double* p0, const double* lb,
                      const double* ub, const gbfit_options* opt_in, FitResult* out, void* cuda_stream,
                      bool eval_only, const double* cov = nullptr) {
    int n, rc;
    if ((rc = check_common(model_id, x_layout, dtype, ydata, &n))) return rc;
    gbfit_options o = opt_in ? *opt_in : defaults();
    if ((rc = check_opts(&o, n))) return rc;
    if (m < n) return fail(GBFIT_E_INVALID_ARG, "m = %lld < n = %d", (long long)m, n);
    if (m > ((int64_t)1 << 40)) return fail(GBFIT_E_INVALID_ARG, "m too large");
    int64_t gw = 0;
    if (x_layout == GBFIT_X_GRID) {
        if (!grid_wh || grid_wh[0] <= 0 || grid_wh[1] <= 0 || grid_wh[0] * grid_wh[1] != m)
            return fail(GBFIT_E_INVALID_ARG, "grid_wh must give W*H == m");
        gw = grid_wh[0];
    } else if (!xdata) {
        return fail(GBFIT_E_INVALID_ARG, "xdata is NULL");
    }
    if (!p0) return fail(GBFIT_E_INVALID_ARG, "p0 is NULL");
    FitArgs a{model_id, n, x_layout, dtype, m, gw, xdata, nullptr, ydata, sigma, p0, lb, ub};
    bool bounded;
    if ((rc = check_params(a, &bounded))) return rc;
    if (eval_only) { bounded = false; o.max_nfev = 1; }
    if (cov) {
        if (m > GBFIT_COV_MAX_M) return fail(GBFIT_E_INVALID_ARG, "covariance fits take m <= %d", GBFIT_COV_MAX_M);
        if (o.loss != GBFIT_LOSS_LINEAR) return fail(GBFIT_E_UNSUPPORTED, "covariance fits take the linear loss");
        if (sigma) return fail(GBFIT_E_INVALID_ARG, "give sigma or a covariance matrix, not both");
    }
    const KernelSet* ks;
    if ((rc = kernels_for_model(model_id, &ks))) return rc;
    Ctx* c;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    size_t es = dtype == GBFIT_F64 ? 8 : 4;
    size_t xbytes = x_layout == GBFIT_X_GRID ? 0 : (size_t)m * es * (x_layout == GBFIT_X_SOA2 ? 2 : 1);
    Staged sd;
    if ((rc = stage_data(c, x_layout == GBFIT_X_GRID ? nullptr : xdata, xbytes, ydata, (size_t)m * es, sigma,
                         (size_t)m * es, s, &sd))) return rc;
    std::vector<FitDesc> hd(1);
    fill_desc(hd[0], a, o, bounded, m, false, loop_grid(c, ks, o.precision));
    hd[0].eval_only = eval_only ? 1 : 0;
    const void* x2 = (x_layout == GBFIT_X_SOA2) ? (const char*)sd.x + (size_t)m * es : nullptr;
    if (sigma && o.precision == GBFIT_PREC_FP64) {
        bool changed = false;
        if ((rc = grow_dev(c->wbuf, c->cap_w, (size_t)m, changed))) return rc;
        CUDA_TRY(launch_stage_weights(dtype == GBFIT_F64, sd.sigma, c->wbuf, m, c->sms * 8, s));
        { std::lock_guard<std::mutex> g(g_stats_mu); g_stats.kernel_launches += 1; }
    }
    set_data(c, hd[0], sd.x, x2, sd.y, sd.sigma, 0, s);
    if (cov && (rc = stage_cov(c, hd[0], cov, m, n, s))) return rc;
    std::vector<std::vector<double>> p0s(1, std::vector<double>(p0, p0 + n));
    std::vector<FitResult> hr;
    int rounds = 0;
    rc = run_fits(c, ks, o.precision, hd, p0s, hr, s, &rounds);
    if (rc) return rc;
    *out = hr[0];
    out->rounds = rounds;
    if (out->fit_status == -2) return fail(GBFIT_E_INVALID_ARG, "sigma <= 0 or non-finite x/y/sigma in the data");
    return GBFIT_OK;
}

int gbfit_curve_fit(int model_id, const void* xdata, int64_t m, int x_layout, const int64_t* grid_wh,
                    const void* ydata, const void* sigma, int dtype, const double* p0, const double* lb,
                    const double* ub, const gbfit_options* opt, double* popt, double* pcov, double* cost,
                    int* nfev, int* fit_status, void* cuda_stream) {
    FitResult r;
    int rc = single_fit(model_id, xdata, m, x_layout, grid_wh, ydata, sigma, dtype, p0, lb, ub, opt, &r,
                        cuda_stream, false);
    if (rc) return rc;
    int n = 0, xd = 0;
    model_shape(model_id, &n, &xd);
    if (popt) for (int i = 0; i < n; ++i) popt[i] = r.popt[i];
    if (pcov) for (int i = 0; i < n * n; ++i) pcov[i] = r.pcov[i];
    if (cost) *cost = r.cost;
    if (nfev) *nfev = r.nfev;
    if (fit_status) *fit_status = r.fit_status;
    return GBFIT_OK;
}

int gbfit_evaluate(int model_id, const void* xdata, int64_t m, int x_layout, const int64_t* grid_wh,
                   const void* ydata, const void* sigma, int dtype, const double* p, int precision,
                   int tile_points, double* out, void* cuda_stream) {
    gbfit_options o = defaults();
    o.precision = precision;
    o.tile_points = tile_points;
    FitResult r;
    int rc = single_fit(model_id, xdata, m, x_layout, grid_wh, ydata, sigma, dtype, p, nullptr, nullptr, &o, &r,
                        cuda_stream, true);
    if (rc) return rc;
    int n = 0, xd = 0;
    model_shape(model_id, &n, &xd);
    int K = n_tri(n) + n + 1;
    for (int k = 0; k < K; ++k) out[k] = r.tot[k];
    out[K - 1] = 0.5 * r.tot[K - 1];
    return GBFIT_OK;
}

int gbfit_curve_fit_cov(int model_id, const void* xdata, int64_t m, int x_layout, const int64_t* grid_wh,
                        const void* ydata, const double* cov, int dtype, const double* p0, const double* lb,
                        const double* ub, const gbfit_options* opt, double* popt, double* pcov, double* cost,
                        int* nfev, int* fit_status, void* cuda_stream) {
    if (!cov) return fail(GBFIT_E_INVALID_ARG, "cov is NULL");
    FitResult r;
    int rc = single_fit(model_id, xdata, m, x_layout, grid_wh, ydata, nullptr, dtype, p0, lb, ub, opt, &r,
                        cuda_stream, false, cov);
    if (rc) return rc;
    int n = 0, xd = 0;
    model_shape(model_id, &n, &xd);
    if (popt) for (int i = 0; i < n; ++i) popt[i] = r.popt[i];
    if (pcov) for (int i = 0; i < n * n; ++i) pcov[i] = r.pcov[i];
    if (cost) *cost = r.cost;
    if (nfev) *nfev = r.nfev;
    if (fit_status) *fit_status = r.fit_status;
    return GBFIT_OK;
}

int gbfit_evaluate_cov(int model_id, const void* xdata, int64_t m, int x_layout, const int64_t* grid_wh,
                       const void* ydata, const double* cov, int dtype, const double* p, int precision,
                       double* out, void* cuda_stream) {
    if (!cov) return fail(GBFIT_E_INVALID_ARG, "cov is NULL");
    gbfit_options o = defaults();
    o.precision = precision;
    FitResult r;
    int rc = single_fit(model_id, xdata, m, x_layout, grid_wh, ydata, nullptr, dtype, p, nullptr, nullptr, &o, &r,
                        cuda_stream, true, cov);
    if (rc) return rc;
    int n = 0, xd = 0;
    model_shape(model_id, &n, &xd);
    int K = n_tri(n) + n + 1;
    for (int k = 0; k < K; ++k) out[k] = r.tot[k];
    out[K - 1] = 0.5 * r.tot[K - 1];
    return GBFIT_OK;
}

int gbfit_curve_fit_batch(int model_id, int nfits, const int64_t* offsets, const void* xdata, int x_layout,
                          const void* ydata, const void* sigma, int dtype, const double* p0, const double* lb,
                          const double* ub, const gbfit_options* opt_in, double* popt, double* pcov, double* cost,
                          int* nfev, int* fit_status, void* cuda_stream) {
    int n, rc;
    if ((rc = check_common(model_id, x_layout, dtype, ydata, &n))) return rc;
    if (x_layout == GBFIT_X_GRID) return fail(GBFIT_E_UNSUPPORTED, "batched fits take explicit coordinates");
    if (nfits < 1 || !offsets || !xdata || !p0) return fail(GBFIT_E_INVALID_ARG, "bad batch arguments");
    gbfit_options o = opt_in ? *opt_in : defaults();
    if ((rc = check_opts(&o, n))) return rc;
    if (offsets[0] != 0) return fail(GBFIT_E_INVALID_ARG, "offsets[0] must be 0");
    for (int f = 0; f < nfits; ++f)
        if (offsets[f + 1] - offsets[f] < n) return fail(GBFIT_E_INVALID_ARG, "fit %d has fewer than n points", f);
    int64_t total = offsets[nfits];
    std::vector<bool> bnd(nfits);
    for (int f = 0; f < nfits; ++f) {
        FitArgs a{model_id, n, x_layout, dtype, offsets[f + 1] - offsets[f], 0, nullptr, nullptr, ydata, sigma,
                  p0 + (size_t)f * n, lb ? lb + (size_t)f * n : nullptr, ub ? ub + (size_t)f * n : nullptr};
        bool b;
        if ((rc = check_params(a, &b))) return fail(rc, "fit %d: %s", f, g_err.c_str());
        bnd[f] = b;
    }
    const KernelSet* ks;
    if ((rc = kernels_for_model(model_id, &ks))) return rc;
    Ctx* c;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    size_t es = dtype == GBFIT_F64 ? 8 : 4;
    size_t xbytes = (size_t)total * es * (x_layout == GBFIT_X_SOA2 ? 2 : 1);
    Staged sd;
    if ((rc = stage_data(c, xdata, xbytes, ydata, (size_t)total * es, sigma, (size_t)total * es, s, &sd))) return rc;
    if (sigma && o.precision == GBFIT_PREC_FP64) {
        bool changed = false;
        if ((rc = grow_dev(c->wbuf, c->cap_w, (size_t)total, changed))) return rc;
        CUDA_TRY(launch_stage_weights(dtype == GBFIT_F64, sd.sigma, c->wbuf, total, c->sms * 8, s));
        { std::lock_guard<std::mutex> g(g_stats_mu); g_stats.kernel_launches += 1; }
    }
    std::vector<FitDesc> hd(nfits);
    std::vector<std::vector<double>> p0s(nfits);
    for (int f = 0; f < nfits; ++f) {
        int64_t a0 = offsets[f], mf = offsets[f + 1] - offsets[f];
        FitArgs a{model_id, n, x_layout, dtype, mf, 0, nullptr, nullptr, ydata, sigma,
                  p0 + (size_t)f * n, lb ? lb + (size_t)f * n : nullptr, ub ? ub + (size_t)f * n : nullptr};
        fill_desc(hd[f], a, o, bnd[f], mf, true);
        const char* xb = (const char*)sd.x + a0 * es;
        const void* x2 = x_layout == GBFIT_X_SOA2 ? (const char*)sd.x + (total + a0) * es : nullptr;
        set_data(c, hd[f], xb, x2, (const char*)sd.y + a0 * es, sigma ? (const char*)sd.sigma + a0 * es : nullptr, a0, s);
        p0s[f].assign(p0 + (size_t)f * n, p0 + (size_t)(f + 1) * n);
    }
    std::vector<FitResult> hr;
    rc = run_fits(c, ks, o.precision, hd, p0s, hr, s, nullptr);
    if (rc) return rc;
    for (int f = 0; f < nfits; ++f) {
        const FitResult& r = hr[f];
        if (popt) for (int i = 0; i < n; ++i) popt[(size_t)f * n + i] = r.popt[i];
        if (pcov) for (int i = 0; i < n * n; ++i) pcov[(size_t)f * n * n + i] = r.pcov[i];
        if (cost) cost[f] = r.cost;
        if (nfev) nfev[f] = r.nfev;
        if (fit_status) fit_status[f] = r.fit_status;
    }
    return GBFIT_OK;
}

int gbfit_tune_get(gbfit_tune_table* out) {
    if (!out) return fail(GBFIT_E_INVALID_ARG, "out is NULL");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    *out = g_tune;
    return GBFIT_OK;
}

int gbfit_tune_set(const gbfit_tune_table* in) {
    if (!in) return fail(GBFIT_E_INVALID_ARG, "table is NULL");
    for (int mo = 0; mo < GBFIT_NUM_MODELS; ++mo)
        for (int p = 0; p < 2; ++p)
            for (int b = 0; b < GBFIT_TUNE_BUCKETS; ++b) {
                int t = in->tile_points[mo][p][b], g = in->group_tiles[mo][p][b];
                if (t < EVAL_THREADS || t > (1 << 24) || t % EVAL_THREADS)
                    return fail(GBFIT_E_INVALID_ARG, "tile_points[%d][%d][%d] = %d is not a multiple of %d in [%d, 2^24]",
                                mo, p, b, t, EVAL_THREADS, EVAL_THREADS);
                if (g < 1 || g > 1024) return fail(GBFIT_E_INVALID_ARG, "group_tiles[%d][%d][%d] = %d", mo, p, b, g);
            }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune = *in;
    return GBFIT_OK;
}

int gbfit_tune_shape(int model_id, int precision, int64_t m, int* tile_points, int* group_tiles) {
    if (model_id < 0 || model_id >= GBFIT_NUM_MODELS)
        return fail(GBFIT_E_INVALID_ARG, "model %d: the tile table covers the built-in models", model_id);
    if (precision != GBFIT_PREC_FP64 && precision != GBFIT_PREC_MIXED) return fail(GBFIT_E_INVALID_ARG, "unknown precision %d", precision);
    if (m < 1) return fail(GBFIT_E_INVALID_ARG, "m must be >= 1");
    int t, g;
    multi_shape(model_id, precision, m, 0, 0, &t, &g);
    if (tile_points) *tile_points = t;
    if (group_tiles) *group_tiles = g;
    return GBFIT_OK;
}

int gbfit_autotune(int model_id, int precision, int64_t m_max, int64_t points_per_run, gbfit_tune_table* out,
                   void* cuda_stream) {
    if (model_id < 0 || model_id >= GBFIT_NUM_MODELS)
        return fail(GBFIT_E_INVALID_ARG, "model %d: the tile table covers the built-in models", model_id);
    if (precision != GBFIT_PREC_FP64 && precision != GBFIT_PREC_MIXED) return fail(GBFIT_E_INVALID_ARG, "unknown precision %d", precision);
    if (m_max < 1 || m_max > ((int64_t)1 << 31)) return fail(GBFIT_E_INVALID_ARG, "m_max out of range");
    const int64_t ppr = points_per_run > 0 ? points_per_run : ((int64_t)1 << 25);
    const int n = model_nparams(model_id);
    const bool f64 = precision == GBFIT_PREC_FP64;
    const size_t es = f64 ? 8 : 4;
    const int layout = model_xdims(model_id) == 2 ? GBFIT_X_SOA2 : GBFIT_X_VEC;
    Ctx* c;
    int rc;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t cap = std::max(ppr, m_max);
    char *xb = nullptr, *yb = nullptr;
    cudaError_t e = cudaMalloc((void**)&xb, (size_t)cap * es * (layout == GBFIT_X_SOA2 ? 2 : 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&yb, (size_t)cap * es);
    if (e != cudaSuccess) {
        cudaFree(xb);
        return fail(GBFIT_E_OOM, "autotune calibration data: %s", cudaGetErrorString(e));
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto cleanup = [&](int r) { cudaFree(xb); cudaFree(yb); cudaEventDestroy(e0); cudaEventDestroy(e1); return r; };
    gbfit_tune_table tab;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tab = g_tune;
    }
    int first_b = -1;
    for (int b = 10; b < GBFIT_TUNE_BUCKETS; ++b) {
        const int64_t mb = (int64_t)3 << (b - 1);
        if (mb > m_max) break;
        const int64_t nf = std::max<int64_t>(1, std::min<int64_t>(4096, ppr / mb));
        // calibration parameters (the 2D centre and widths follow the grid side)
        double truth[NMAX] = {0};
        const double Wd = std::ceil(std::sqrt((double)mb));
        switch (model_id) {
            case 0: { double t[] = {5.0, 0.3, 1.2, 0.5}; std::copy(t, t + 4, truth); break; }
            case 1: { double t[] = {4.0, 0.8, 6.0, 9.0, 0.5}; std::copy(t, t + 5, truth); break; }
            case 2: { double t[] = {980.0, 0.5 * Wd, 0.48 * Wd, 0.06 * Wd, 0.035 * Wd, 0.4, 20.0}; std::copy(t, t + 7, truth); break; }
            default: { double t[] = {1.5, -0.7, 0.25}; std::copy(t, t + 3, truth); break; }
        }
        e = launch_synth_fill(model_id, f64, xb, layout == GBFIT_X_SOA2 ? xb + (size_t)cap * es : nullptr, yb,
                              nf * mb, mb, 1234u + (uint32_t)b, c->sms * 8, truth, s);
        if (e != cudaSuccess) return cleanup(fail(GBFIT_E_CUDA, "autotune data: %s", cudaGetErrorString(e)));
        std::vector<double> p0(n);
        for (int i = 0; i < n; ++i) p0[i] = truth[i] * 1.05;
        if (model_id == 2) { p0[1] = truth[1] + 1.0; p0[2] = truth[2] - 1.0; p0[5] = truth[5] + 0.02; }
        std::vector<std::vector<double>> p0s(nf, p0);
        gbfit_options o = defaults();
        o.precision = precision;
        o.ftol = o.xtol = o.gtol = 0.0;
        o.max_nfev = 4;
        // candidates: powers of two up to 2^18 below 2 m (mixed: up to
        // MIXED_TILE_CAP), and one tile per fit when that is within the cap
        const int64_t tmax = precision == GBFIT_PREC_MIXED ? MIXED_TILE_CAP : ((int64_t)1 << 18);
        std::vector<int> tiles;
        for (int k = 10; k <= 18; ++k)
            if (((int64_t)1 << k) < mb && ((int64_t)1 << k) <= tmax) tiles.push_back(1 << k);
        if (mb <= tmax) tiles.push_back((int)((mb + EVAL_THREADS - 1) / EVAL_THREADS * EVAL_THREADS));
        struct Cand { int tp, g; float ms; };
        std::vector<Cand> cands;
        for (int tp : tiles) {
            int64_t ntl = (mb + tp - 1) / tp;
            std::vector<int> groups = ntl > 8 ? std::vector<int>{8, 32, 128} : std::vector<int>{GROUP_TILES};
            for (int g : groups) {
                o.tile_points = tp;
                o.group_tiles = g;
                std::vector<FitDesc> hd(nf);
                for (int64_t f = 0; f < nf; ++f) {
                    FitArgs a{model_id, n, layout, f64 ? GBFIT_F64 : GBFIT_F32, mb, 0, nullptr, nullptr, nullptr, nullptr,
                              p0.data(), nullptr, nullptr};
                    fill_desc(hd[f], a, o, false, mb, true);
                    hd[f].x = xb + (size_t)(f * mb) * es;
                    hd[f].x2 = layout == GBFIT_X_SOA2 ? xb + (size_t)(cap + f * mb) * es : nullptr;
                    hd[f].y = yb + (size_t)(f * mb) * es;
                    hd[f].w = nullptr;
                    hd[f].wkind = W_NONE;
                }
                float ms = 0.0f;
                for (int rep = 0; rep < 2; ++rep) {
                    std::vector<FitResult> hr;
                    std::vector<FitDesc> hdc = hd;
                    e = cudaEventRecord(e0, s);
                    const KernelSet* kst = nullptr;
                    if ((rc = kernels_for_model(model_id, &kst))) return cleanup(rc);
                    if (e == cudaSuccess && (rc = run_fits(c, kst, precision, hdc, p0s, hr, s, nullptr))) return cleanup(rc);
                    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e != cudaSuccess) return cleanup(fail(GBFIT_E_CUDA, "autotune timing: %s", cudaGetErrorString(e)));
                }
                cands.push_back({tp, g, ms});
            }
        }
        // Among shapes within 3 % of the best throughput, the one with the
        // most tiles per fit: in a batch of mixed sizes the evaluation chains
        // of the largest fits set the launch time, and more tiles per fit
        // shorten each of their passes (calibration timings of near-equal
        // shapes differ by noise).
        float best = 1e30f;
        for (const Cand& q : cands) best = std::min(best, q.ms);
        int bt = tiles.back(), bg = GROUP_TILES;
        float bms = 1e30f;
        for (const Cand& q : cands)
            if (q.ms <= 1.03f * best && (q.tp < bt || (q.tp == bt && q.ms < bms))) { bt = q.tp; bg = q.g; bms = q.ms; }
        tab.tile_points[model_id][precision][b] = bt;
        tab.group_tiles[model_id][precision][b] = bg;
        if (first_b < 0) first_b = b;
    }
    if (first_b >= 0)
        for (int b = 0; b < first_b; ++b) {
            tab.tile_points[model_id][precision][b] = tab.tile_points[model_id][precision][first_b];
            tab.group_tiles[model_id][precision][b] = tab.group_tiles[model_id][precision][first_b];
        }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune = tab;
    }
    if (out) *out = tab;
    return cleanup(GBFIT_OK);
}

int gbfit_stats_reset(void) {
    std::lock_guard<std::mutex> g(g_stats_mu);
    memset(&g_stats, 0, sizeof g_stats);
    return GBFIT_OK;
}

int gbfit_stats_get(gbfit_stats* out) {
    if (!out) return fail(GBFIT_E_INVALID_ARG, "out is NULL");
    std::lock_guard<std::mutex> g(g_stats_mu);
    *out = g_stats;
    return GBFIT_OK;
}

int gbfit_check_rcp64(const double* x, double* y, int64_t n, void* cuda_stream) {
    if (n < 0) return fail(GBFIT_E_INVALID_ARG, "n < 0");
    if (n == 0) return GBFIT_OK;
    if (!x || !y) return fail(GBFIT_E_INVALID_ARG, "x and y must not be NULL");
    if (!is_device_ptr(x) || !is_device_ptr(y)) return fail(GBFIT_E_INVALID_ARG, "x and y must be device pointers");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    CUDA_TRY(launch_rcp64(x, y, n, 4 * 152, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return GBFIT_OK;
}

int gbfit_set_profiling(int on) {
    g_profiling = on ? 1 : 0;
    return GBFIT_OK;
}

int gbfit_tr_subproblem(int n, const double* B, const double* g, double Delta, double alpha0, double* p,
                        double* alpha, double* lam, void* cuda_stream) {
    if (n < 1 || n > NMAX || !B || !g || !p || !alpha || !lam) return fail(GBFIT_E_INVALID_ARG, "bad subproblem arguments");
    if (!(Delta > 0)) return fail(GBFIT_E_INVALID_ARG, "Delta must be > 0");
    Ctx* c;
    int rc;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double* d = c->small;
    if ((rc = c->pinned(256 * sizeof(double)))) return rc;
    double* h = (double*)c->hbuf;
    memcpy(h, B, n * n * sizeof(double));
    memcpy(h + 64, g, n * sizeof(double));
    CUDA_TRY(cudaMemcpyAsync(d, h, 72 * sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(launch_tr_subproblem(n, d, d + 64, Delta, alpha0, d + 80, d + 88, d + 96, s));
    CUDA_TRY(cudaMemcpyAsync(h + 80, d + 80, 24 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < n; ++i) { p[i] = h[80 + i]; lam[i] = h[96 + i]; }
    *alpha = h[88];
    return GBFIT_OK;
}

}  // extern "C"

// ====================================================================== allocation-free evaluation
// gbfit_evaluate_noalloc serves callers that may not allocate memory on the
// device when they call: applications whose memory manager owns all device
// memory (a pool sized at start-up), and loops that cannot take the implicit
// device-wide synchronisation of cudaMalloc / cudaFree.  The fused reduction
// pass needs scratch memory for its per-tile and per-group partial sums, its
// arrival counters and its one-fit job record; here all of it lives in the
// file-scope device array below, of fixed size, which every GPU that loads
// this library holds until the process exits.  The call is synchronous: it
// waits on the caller's stream for its result.
namespace {
constexpr int NOALLOC_MAX_TILES = 2048;                                   // reduction tiles per call
constexpr int NOALLOC_MAX_GROUPS = (NOALLOC_MAX_TILES + GROUP_TILES - 1) / GROUP_TILES;   // default groups

struct NoAllocLayout {
    static constexpr size_t eng = 0;
    static constexpr size_t desc = eng + ((sizeof(Engine) + 255) / 256) * 256;
    static constexpr size_t state = desc + ((sizeof(FitDesc) + 255) / 256) * 256;
    static constexpr size_t items = state + ((sizeof(FitState) + 255) / 256) * 256;
    static constexpr size_t gcnt = items + ((NOALLOC_MAX_TILES * sizeof(WorkItem) + 255) / 256) * 256;
    static constexpr size_t fcnt = gcnt + ((NOALLOC_MAX_GROUPS * sizeof(int) + 255) / 256) * 256;
    static constexpr size_t res_hdr = fcnt + 256;                          // end of the uploaded image
    static constexpr size_t res = res_hdr + 256;
    static constexpr size_t tpd = res + ((sizeof(FitResult) + 255) / 256) * 256;   // end of the result region
    static constexpr size_t gp = tpd + ((size_t(NOALLOC_MAX_TILES) * KMAX * sizeof(double) + 255) / 256) * 256;
    static constexpr size_t end = gp + ((size_t(NOALLOC_MAX_GROUPS) * KMAX * sizeof(double) + 255) / 256) * 256;
};
constexpr size_t NOALLOC_SCRATCH_BYTES = NoAllocLayout::end;             // about 0.9 MB

// Largest m a call takes: at the default tile choice, NOALLOC_MAX_TILES tiles
// of the largest tile; with the caller's tile_points, NOALLOC_MAX_TILES tiles
// of that size.
constexpr int64_t NOALLOC_MAX_M = int64_t(NOALLOC_MAX_TILES) * TILE_MAX;

// Tile size of an allocation-free call: the caller's, else the default
// choice for this grid, made coarser when that choice would need more tiles
// than the array holds.  For m <= NOALLOC_MAX_M the result never needs more
// than NOALLOC_MAX_TILES tiles, whatever the grid.
int noalloc_tile(int64_t m, int tile_points, int grid) {
    int tp = choose_tile(m, tile_points, grid);
    if (tile_points == 0 && (m + tp - 1) / tp > NOALLOC_MAX_TILES) {
        int64_t t = (m + NOALLOC_MAX_TILES - 1) / NOALLOC_MAX_TILES;
        t = ((t + EVAL_THREADS - 1) / EVAL_THREADS) * EVAL_THREADS;
        tp = (int)std::min<int64_t>(t, TILE_MAX);
    }
    return tp;
}

std::mutex g_noalloc_mu;
char* g_noalloc_dev[64] = {};                                            // device address, per device
alignas(256) char g_noalloc_host[NoAllocLayout::res_hdr];                // upload image (static, not heap)
alignas(256) char g_noalloc_result[NoAllocLayout::tpd - NoAllocLayout::res_hdr];
}  // namespace

// The scratch array.  In host code this name is only a host-side stand-in
// for the symbol; its device address is obtained with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

extern "C" int gbfit_evaluate_noalloc(int model_id, const void* xdata, int64_t m, int x_layout,
                                      const int64_t* grid_wh, const void* ydata, const void* sigma, int dtype,
                                      const double* p, int precision, int tile_points, double* out,
                                      void* cuda_stream) {
    int n, rc;
    if ((rc = check_common(model_id, x_layout, dtype, ydata, &n))) return rc;
    if (model_id >= GBFIT_NUM_MODELS) return fail(GBFIT_E_UNSUPPORTED, "the allocation-free entry point takes built-in models");
    if (!p || !out) return fail(GBFIT_E_INVALID_ARG, "p and out must not be NULL");
    if (precision != GBFIT_PREC_FP64 && precision != GBFIT_PREC_MIXED) return fail(GBFIT_E_INVALID_ARG, "unknown precision %d", precision);
    if (tile_points < 0 || tile_points > (1 << 24)) return fail(GBFIT_E_INVALID_ARG, "tile_points out of range");
    if (m < n) return fail(GBFIT_E_INVALID_ARG, "m = %lld < n = %d", (long long)m, n);
    int64_t gw = 0;
    if (x_layout == GBFIT_X_GRID) {
        if (!grid_wh || grid_wh[0] <= 0 || grid_wh[1] <= 0 || grid_wh[0] * grid_wh[1] != m)
            return fail(GBFIT_E_INVALID_ARG, "grid_wh must give W*H == m");
        gw = grid_wh[0];
    } else if (!xdata) {
        return fail(GBFIT_E_INVALID_ARG, "xdata is NULL");
    }
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return fail(GBFIT_E_INVALID_ARG, "p[%d] is not finite", i);
    // size limits first, from host arithmetic alone (no CUDA call yet)
    if (tile_points > 0) {
        const int tpu = choose_tile(m, tile_points, 0);
        const int64_t nt = (m + tpu - 1) / tpu;
        if (nt > NOALLOC_MAX_TILES)
            return fail(GBFIT_E_INVALID_ARG,
                        "m = %lld needs %lld reduction tiles of %d points; the allocation-free entry point holds at "
                        "most %d tiles (m <= %lld points at this tile size)",
                        (long long)m, (long long)nt, tpu, NOALLOC_MAX_TILES, (long long)NOALLOC_MAX_TILES * tpu);
    } else if (m > NOALLOC_MAX_M) {
        return fail(GBFIT_E_INVALID_ARG,
                    "m = %lld exceeds the allocation-free entry point's limit: it holds at most %d tiles "
                    "(m <= %lld points at the default tile size)",
                    (long long)m, NOALLOC_MAX_TILES, (long long)NOALLOC_MAX_M);
    }
    int nsm = 0, dev0 = 0;
    CUDA_TRY(cudaGetDevice(&dev0));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev0));
    const int grid_na = nsm * std::max(1, eval_blocks_per_sm(precision));
    const int tp = noalloc_tile(m, tile_points, grid_na);
    const int64_t ntiles = (m + tp - 1) / tp;
    if (ntiles > NOALLOC_MAX_TILES)                 // unreachable after the checks above
        return fail(GBFIT_E_INVALID_ARG, "m = %lld needs %lld tiles; at most %d fit", (long long)m,
                    (long long)ntiles, NOALLOC_MAX_TILES);
    if (!is_device_ptr(ydata) || (xdata && x_layout != GBFIT_X_GRID && !is_device_ptr(xdata)) ||
        (sigma && !is_device_ptr(sigma)))
        return fail(GBFIT_E_INVALID_ARG, "the allocation-free entry point needs device-resident data arrays");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(GBFIT_E_CUDA, "device ordinal %d out of range", dev);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    // From the first enqueue on, every return (error paths included) first
    // waits for this call's work on the stream, so that none of it can still
    // use the shared array once the lock is released (declared after the
    // lock: destroyed, and so synchronised, before the lock is let go).
    struct SyncOnExit {
        cudaStream_t s;
        bool armed;
        ~SyncOnExit() { if (armed) cudaStreamSynchronize(s); }
    } guard{s, false};
    if (!g_noalloc_dev[dev]) {
        // one-time set-up on this device (this device is current): the
        // device address of the scratch array
        void* ptr = nullptr;
        CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        g_noalloc_dev[dev] = (char*)ptr;
    }
    char* base = g_noalloc_dev[dev];
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int prec = precision;
    int bps = eval_blocks_per_sm(prec);
    if (bps < 1) bps = 1;
    // ---- the job image: engine header, descriptor, initial state, work
    //      items and zeroed arrival counters (everything that must start at
    //      zero is part of the upload)
    typedef NoAllocLayout LY;
    memset(g_noalloc_host, 0, sizeof g_noalloc_host);
    Engine E;
    memset(&E, 0, sizeof E);
    Engine* Ed = (Engine*)(base + LY::eng);
    E.results = (FitResult*)(base + LY::res);
    E.out = (int*)(base + LY::res_hdr);
    E.desc = (FitDesc*)(base + LY::desc);
    E.state = (FitState*)(base + LY::state);
    E.items = (WorkItem*)(base + LY::items);
    E.group_cnt = (int*)(base + LY::gcnt);
    E.fit_cnt = (int*)(base + LY::fcnt);
    E.tile_part_d = (double*)(base + LY::tpd);
    E.group_part = (double*)(base + LY::gp);
    E.n_items = &Ed->sc[0]; E.running = &Ed->sc[1]; E.rounds = &Ed->sc[2];
    E.max_rounds = &Ed->sc[3]; E.nfits_dev = &Ed->sc[4];
    E.sc[0] = (int)ntiles; E.sc[1] = 1; E.sc[2] = 0; E.sc[3] = 2; E.sc[4] = 1;
    memcpy(g_noalloc_host + LY::eng, &E, sizeof E);
    gbfit_options o = defaults();
    o.precision = prec;
    o.tile_points = tp;
    o.max_nfev = 1;
    FitArgs a{model_id, n, x_layout, dtype, m, gw, xdata, nullptr, ydata, sigma, p, nullptr, nullptr};
    FitDesc d;
    fill_desc(d, a, o, false, m, false, grid_na);
    d.eval_only = 1;
    size_t es = dtype == GBFIT_F64 ? 8 : 4;
    d.x = x_layout == GBFIT_X_GRID ? nullptr : xdata;
    d.x2 = (x_layout == GBFIT_X_SOA2) ? (const char*)xdata + (size_t)m * es : nullptr;
    d.y = ydata;
    d.w = sigma;
    d.wkind = sigma ? W_SIGMA : W_NONE;        // 1/sigma formed in the kernel: no staging buffer
    d.tile_base = 0;
    d.group_base = 0;
    memcpy(g_noalloc_host + LY::desc, &d, sizeof d);
    FitState* st = (FitState*)(g_noalloc_host + LY::state);
    st->run = RS_RUNNING;
    st->phase = PH_INIT;
    for (int i = 0; i < n; ++i) { st->x[i] = p[i]; st->xt[i] = p[i]; st->scale_inv[i] = 1.0; }
    WorkItem* items = (WorkItem*)(g_noalloc_host + LY::items);
    for (int t = 0; t < (int)ntiles; ++t) items[t] = WorkItem{0, t};
    guard.armed = true;
    CUDA_TRY(cudaMemcpyAsync(base, g_noalloc_host, LY::res_hdr, cudaMemcpyHostToDevice, s));
    void* args[] = {&Ed};
    CUDA_TRY(cudaLaunchKernel(kernel_init_fits(prec), dim3(1), dim3(32), args, 0, s));
    CUDA_TRY(cudaLaunchKernel(kernel_eval_round(prec), dim3(sms * bps), dim3(EVAL_THREADS), args,
                              eval_dyn_smem(prec), s));
    CUDA_TRY(cudaMemcpyAsync(g_noalloc_result, base + LY::res_hdr, sizeof g_noalloc_result,
                             cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    guard.armed = false;
    const FitResult* r = (const FitResult*)(g_noalloc_result + (LY::res - LY::res_hdr));
    if (r->fit_status == -2) return fail(GBFIT_E_INVALID_ARG, "sigma <= 0 or non-finite x/y/sigma in the data");
    const int K = n_tri(n) + n + 1;
    for (int k = 0; k < K; ++k) out[k] = r->tot[k];
    out[K - 1] = 0.5 * r->tot[K - 1];
    return GBFIT_OK;
}

// ====================================================================== serving (continuous batching)
#include <chrono>
#include <deque>
#include <map>

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, capacity) in arbitrary units, with coalescing.
struct RangeAlloc {
    std::map<size_t, size_t> free_;   // offset -> size
    size_t cap = 0, used = 0;
    void reset(size_t c) { free_.clear(); free_[0] = c; cap = c; used = 0; }
    bool alloc(size_t n, size_t align, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            size_t o = (it->first + align - 1) / align * align;
            size_t end = it->first + it->second;
            if (o + n <= end) {
                size_t fo = it->first, fs = it->second;
                free_.erase(it);
                if (o > fo) free_[fo] = o - fo;
                if (o + n < fo + fs) free_[o + n] = fo + fs - (o + n);
                *off = o;
                used += n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
        }
    }
};

struct SrvPending {
    gbfit_request req;
    uint64_t ticket;
    double t_submit;
    std::vector<unsigned char> resume;  // state prefix of a snapshot to continue from (empty: start at p0)
};

struct SrvSlot {
    bool used = false;
    uint64_t ticket = 0, tag = 0;
    size_t data_off = 0, data_bytes = 0, tile0 = 0, ntiles = 0, group0 = 0, ngroups = 0;
    double t_submit = 0, t_admit = 0;
    int n = 0, model = 0;
    int64_t m = 0;
    double p0[GBFIT_MAX_PARAMS] = {};
};

// Bytes of FitState a snapshot carries: everything before the trace counters.
constexpr size_t SNAP_STATE_BYTES = offsetof(FitState, trace);
static_assert(SNAP_STATE_BYTES <= GBFIT_SNAPSHOT_STATE_BYTES, "a fit's state must fit a snapshot");

// Each array of a request starts on a 256-byte boundary of its pool region
// (so that the bulk-copy ring can stream every array).
size_t arr_bytes(const gbfit_request& r) { return ((size_t)r.m * (r.dtype == GBFIT_F64 ? 8 : 4) + 255) / 256 * 256; }
size_t req_data_bytes(const gbfit_request& r) {
    size_t xs = r.x_layout == GBFIT_X_GRID ? 0 : (r.x_layout == GBFIT_X_SOA2 ? 2 : 1);
    return arr_bytes(r) * (xs + 1 + (r.sigma ? 1 : 0));
}

}  // namespace

struct gbfit_server {
    int device = 0, prec = PREC_MIXED, max_slots = 0, rounds = 4, grid = 0;
    double guard_cond = GBFIT_GUARD_COND_DEFAULT, guard_floor = GBFIT_GUARD_FLOOR_DEFAULT;
    size_t budget = 0;
    char* pool = nullptr;
    RangeAlloc pool_alloc, tile_alloc, group_alloc;
    size_t max_tiles = 0, max_groups = 0;
    double* tile_part_d = nullptr;
    double* group_part = nullptr;
    char* job = nullptr;
    JobLayout* L = nullptr;
    char* hbuf = nullptr;              // pinned staging (job image, results, flags)
    size_t hcap = 0;
    int* d_list = nullptr;             // device list of newly admitted slots
    cudaStream_t stream = nullptr;
    std::deque<SrvPending> queue;
    std::vector<SrvSlot> slots;
    std::deque<gbfit_result_rec> done;
    uint64_t next_ticket = 1;
    std::mutex mu;
};

extern "C" {

int gbfit_server_create(const gbfit_server_config* cfg_in, gbfit_server** out) {
    if (!out) return fail(GBFIT_E_INVALID_ARG, "out is NULL");
    gbfit_server_config cfg;
    memset(&cfg, 0, sizeof cfg);
    if (cfg_in) cfg = *cfg_in;
    if (cfg.hbm_budget_bytes == 0) cfg.hbm_budget_bytes = (size_t)1 << 30;
    if (cfg.max_slots <= 0) cfg.max_slots = 4096;
    if (cfg.rounds_per_step <= 0) cfg.rounds_per_step = 4;
    if (cfg.precision != GBFIT_PREC_FP64 && cfg.precision != GBFIT_PREC_MIXED)
        return fail(GBFIT_E_INVALID_ARG, "unknown precision %d", cfg.precision);
    gbfit_server* s = new gbfit_server();
    s->prec = cfg.precision;
    s->max_slots = cfg.max_slots;
    s->rounds = cfg.rounds_per_step;
    s->budget = cfg.hbm_budget_bytes;
    if (std::isnan(cfg.guard_cond) || std::isnan(cfg.guard_floor)) {
        delete s;
        return fail(GBFIT_E_INVALID_ARG, "guard_cond and guard_floor must not be NaN");
    }
    s->guard_cond = guard_value(cfg.guard_cond, GBFIT_GUARD_COND_DEFAULT);
    s->guard_floor = guard_value(cfg.guard_floor, GBFIT_GUARD_FLOOR_DEFAULT);
    auto bail = [&](int rc) { gbfit_server_destroy(s); return rc; };
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) return bail(fail(GBFIT_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e)));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    int bps = eval_blocks_per_sm(s->prec);
    s->grid = sms * (bps < 1 ? 1 : bps);
    // tile scratch: enough for the budget filled with the smallest tiles and
    // groups of the tile table (at 8 bytes per point)
    int min_tile = 1 << 24, min_group = 1024;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (int mo = 0; mo < GBFIT_NUM_MODELS; ++mo)
            for (int b = 0; b < GBFIT_TUNE_BUCKETS; ++b) {
                min_tile = std::min(min_tile, (int)g_tune.tile_points[mo][s->prec][b]);
                min_group = std::min(min_group, (int)g_tune.group_tiles[mo][s->prec][b]);
            }
    }
    s->max_tiles = s->budget / (size_t(min_tile) * 8) + (size_t)s->max_slots;
    s->max_groups = s->max_tiles / (size_t)min_group + (size_t)s->max_slots;
    s->L = new JobLayout((size_t)s->max_slots, s->max_tiles, s->max_groups);
    bool ch = false;
    size_t cap = 0;
    if (grow_dev(s->pool, cap, s->budget, ch)) return bail(GBFIT_E_OOM);
    cap = 0;
    if (grow_dev(s->job, cap, s->L->end, ch)) return bail(GBFIT_E_OOM);
    cap = 0;
    if (grow_dev(s->tile_part_d, cap, s->max_tiles * KMAX, ch)) return bail(GBFIT_E_OOM);
    cap = 0;
    if (grow_dev(s->group_part, cap, s->max_groups * KMAX, ch)) return bail(GBFIT_E_OOM);
    cap = 0;
    if (grow_dev(s->d_list, cap, (size_t)s->max_slots, ch)) return bail(GBFIT_E_OOM);
    s->hcap = s->L->end + (size_t)s->max_slots * 8 + 4096;   // + admit list, scalars, finished flags
    e = cudaMallocHost((void**)&s->hbuf, s->hcap);
    if (e != cudaSuccess) { s->hbuf = nullptr; return bail(fail(GBFIT_E_OOM, "cudaMallocHost: %s", cudaGetErrorString(e))); }
    e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(fail(GBFIT_E_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
    s->pool_alloc.reset(s->budget);
    s->tile_alloc.reset(s->max_tiles);
    s->group_alloc.reset(s->max_groups);
    s->slots.resize(s->max_slots);
    // device image: engine header and all slots marked done
    memset(s->hbuf, 0, s->L->res_hdr);
    Engine E;
    memset(&E, 0, sizeof E);
    char* job = s->job;
    Engine* Ed = (Engine*)job;
    E.results = (FitResult*)(job + s->L->res);
    E.out = (int*)(job + s->L->res_hdr);
    E.desc = (FitDesc*)(job + s->L->desc);
    E.state = (FitState*)(job + s->L->state);
    E.items = (WorkItem*)(job + s->L->items);
    E.group_cnt = (int*)(job + s->L->gcnt);
    E.fit_cnt = (int*)(job + s->L->fcnt);
    E.sm_cnt = (int*)(job + s->L->smcnt);
    E.tile_part_d = s->tile_part_d; E.group_part = s->group_part;
    E.n_items = &Ed->sc[0]; E.running = &Ed->sc[1]; E.rounds = &Ed->sc[2];
    E.max_rounds = &Ed->sc[3]; E.nfits_dev = &Ed->sc[4];
    E.sc[3] = 1 << 30;
    E.sc[4] = s->max_slots;
    memcpy(s->hbuf, &E, sizeof E);
    FitState* hs = (FitState*)(s->hbuf + s->L->state);
    for (int k = 0; k < s->max_slots; ++k) hs[k].run = RS_DONE;
    e = cudaMemcpyAsync(s->job, s->hbuf, s->L->res_hdr, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return bail(fail(GBFIT_E_CUDA, "server init: %s", cudaGetErrorString(e)));
    *out = s;
    return GBFIT_OK;
}

static int server_enqueue(gbfit_server* s, const gbfit_request* r, const gbfit_fit_snapshot* snap,
                          uint64_t* ticket) {
    if (!s || !r) return fail(GBFIT_E_INVALID_ARG, "server and request must not be NULL");
    int n, rc;
    if ((rc = check_common(r->model_id, r->x_layout, r->dtype, r->ydata, &n))) return rc;
    if (r->model_id >= GBFIT_NUM_MODELS) return fail(GBFIT_E_UNSUPPORTED, "serving takes built-in models");
    if (r->m < n) return fail(GBFIT_E_INVALID_ARG, "m = %lld < n = %d", (long long)r->m, n);
    if (r->x_layout == GBFIT_X_GRID && (r->grid_w <= 0 || r->grid_h <= 0 || r->grid_w * r->grid_h != r->m))
        return fail(GBFIT_E_INVALID_ARG, "grid_w * grid_h must equal m");
    if (r->x_layout != GBFIT_X_GRID && !r->xdata) return fail(GBFIT_E_INVALID_ARG, "xdata is NULL");
    FitArgs a{r->model_id, n, r->x_layout, r->dtype, r->m, r->grid_w, r->xdata, nullptr, r->ydata, r->sigma,
              r->p0, r->has_bounds ? r->lb : nullptr, r->has_bounds ? r->ub : nullptr};
    bool bounded;
    if ((rc = check_params(a, &bounded))) return rc;
    if (r->loss < GBFIT_LOSS_LINEAR || r->loss > GBFIT_LOSS_ARCTAN) return fail(GBFIT_E_INVALID_ARG, "unknown loss %d", r->loss);
    if (!(r->f_scale >= 0) || !std::isfinite(r->f_scale)) return fail(GBFIT_E_INVALID_ARG, "f_scale must be > 0");
    if (snap && (snap->magic != GBFIT_SNAPSHOT_MAGIC || snap->state_bytes != SNAP_STATE_BYTES ||
                 snap->model_id != r->model_id || snap->m != r->m || snap->precision != s->prec))
        return fail(GBFIT_E_INVALID_ARG, "the snapshot does not belong to this model, size and server precision");
    size_t need = req_data_bytes(*r);
    int tp, gt;
    multi_shape(r->model_id, s->prec, r->m, 0, 0, &tp, &gt);
    size_t nt = (size_t)((r->m + tp - 1) / tp);
    if (need > s->budget || nt > s->max_tiles)
        return fail(GBFIT_E_BUDGET, "request needs %zu bytes; the server's pool holds %zu", need, s->budget);
    std::lock_guard<std::mutex> g(s->mu);
    SrvPending p;
    p.req = *r;
    p.ticket = s->next_ticket++;
    p.t_submit = now_s();
    if (snap) p.resume.assign(snap->state, snap->state + SNAP_STATE_BYTES);
    s->queue.push_back(std::move(p));
    if (ticket) *ticket = s->queue.back().ticket;
    return GBFIT_OK;
}

int gbfit_server_submit(gbfit_server* s, const gbfit_request* r, uint64_t* ticket) {
    return server_enqueue(s, r, nullptr, ticket);
}

int gbfit_server_submit_resume(gbfit_server* s, const gbfit_request* r, const gbfit_fit_snapshot* snap,
                               uint64_t* ticket) {
    if (!snap) return fail(GBFIT_E_INVALID_ARG, "snap is NULL");
    return server_enqueue(s, r, snap, ticket);
}

// The device state of resident slot k (synchronous; between steps nothing runs).
static int server_read_state(gbfit_server* s, int k, void* out) {
    CUDA_TRY(cudaMemcpyAsync(out, s->job + s->L->state + (size_t)k * sizeof(FitState), SNAP_STATE_BYTES,
                             cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return GBFIT_OK;
}

static void server_release(gbfit_server* s, int k) {
    SrvSlot& sl = s->slots[k];
    s->pool_alloc.release(sl.data_off, sl.data_bytes);
    s->tile_alloc.release(sl.tile0, sl.ntiles);
    s->group_alloc.release(sl.group0, sl.ngroups);
    sl.used = false;
}

static int server_retire(gbfit_server* s) {
    NvtxRange nv("gbfit.server_retire");
    // which resident fits finished: the `run` word of every slot's state
    int* flags = (int*)(s->hbuf + s->L->end + (size_t)s->max_slots * 4 + 256);
    CUDA_TRY(cudaMemcpy2DAsync(flags, sizeof(int), s->job + s->L->state + offsetof(FitState, run), sizeof(FitState),
                               sizeof(int), (size_t)s->max_slots, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    FitResult* hr = (FitResult*)(s->hbuf + s->L->res);
    std::vector<int> fin;
    for (int k = 0; k < s->max_slots; ++k)
        if (s->slots[k].used && flags[k] == RS_DONE) {
            fin.push_back(k);
            CUDA_TRY(cudaMemcpyAsync(hr + k, s->job + s->L->res + (size_t)k * sizeof(FitResult), sizeof(FitResult),
                                     cudaMemcpyDeviceToHost, s->stream));
        }
    if (fin.empty()) return GBFIT_OK;
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    double t = now_s();
    for (int k : fin) {
        SrvSlot& sl = s->slots[k];
        gbfit_result_rec rec;
        memset(&rec, 0, sizeof rec);
        rec.ticket = sl.ticket;
        rec.tag = sl.tag;
        rec.fit_status = hr[k].fit_status;
        rec.status = hr[k].fit_status == -2 ? GBFIT_E_INVALID_ARG : GBFIT_OK;
        rec.nfev = hr[k].nfev;
        rec.n_params = sl.n;
        rec.cost = hr[k].cost;
        for (int i = 0; i < sl.n; ++i) rec.popt[i] = hr[k].popt[i];
        rec.t_submit = sl.t_submit;
        rec.t_admit = sl.t_admit;
        rec.t_done = t;
        s->done.push_back(rec);
        server_release(s, k);
    }
    return GBFIT_OK;
}

int gbfit_server_step(gbfit_server* s, int* n_active, int* n_queued) {
    if (!s) return fail(GBFIT_E_INVALID_ARG, "server is NULL");
    NvtxRange nv("gbfit.server_step");
    std::lock_guard<std::mutex> g(s->mu);
    int rc;
    if ((rc = server_retire(s))) return rc;
    // ---- admit in arrival order while a slot and memory are free
    std::vector<int> admitted, fresh;            // fresh: start at p0 (pass constants computed on the device)
    int free_slot = 0;
    while (!s->queue.empty()) {
        SrvPending& p = s->queue.front();
        const gbfit_request& r = p.req;
        while (free_slot < s->max_slots && s->slots[free_slot].used) ++free_slot;
        if (free_slot >= s->max_slots) break;
        int n = model_nparams(r.model_id);
        size_t need = req_data_bytes(r);
        gbfit_options o = defaults();
        o.precision = s->prec;
        o.ftol = r.ftol > 0 ? r.ftol : 1e-8;
        o.xtol = r.xtol > 0 ? r.xtol : 1e-8;
        o.gtol = r.gtol > 0 ? r.gtol : 1e-8;
        o.max_nfev = r.max_nfev;
        o.loss = r.loss;
        o.f_scale = r.f_scale;
        o.guard_cond = s->guard_cond;
        o.guard_floor = s->guard_floor;
        FitArgs a{r.model_id, n, r.x_layout, r.dtype, r.m, r.grid_w, nullptr, nullptr, nullptr, nullptr,
                  r.p0, r.has_bounds ? r.lb : nullptr, r.has_bounds ? r.ub : nullptr};
        bool bounded = false;
        for (int i = 0; i < n && r.has_bounds; ++i)
            if (std::isfinite(r.lb[i]) || std::isfinite(r.ub[i])) bounded = true;
        FitDesc d;
        fill_desc(d, a, o, bounded, r.m, true);
        size_t nt = (size_t)d.n_tiles, ng = (size_t)d.n_groups;
        size_t off, t0, g0;
        if (!s->pool_alloc.alloc(need, 256, &off)) break;
        if (!s->tile_alloc.alloc(nt, 1, &t0)) { s->pool_alloc.release(off, need); break; }
        if (!s->group_alloc.alloc(ng, 1, &g0)) { s->pool_alloc.release(off, need); s->tile_alloc.release(t0, nt); break; }
        // copy the data into the pool: x rows, y, sigma
        size_t es = r.dtype == GBFIT_F64 ? 8 : 4;
        size_t xs = r.x_layout == GBFIT_X_GRID ? 0 : (r.x_layout == GBFIT_X_SOA2 ? 2 : 1);
        char* base = s->pool + off;
        size_t ab = arr_bytes(r), raw = (size_t)r.m * es;
        size_t bx = ab * xs, by = ab;
        for (size_t k = 0; k < xs; ++k)     // caller's x is [xs][m] contiguous
            CUDA_TRY(cudaMemcpyAsync(base + k * ab, (const char*)r.xdata + k * raw, raw, cudaMemcpyDefault, s->stream));
        CUDA_TRY(cudaMemcpyAsync(base + bx, r.ydata, raw, cudaMemcpyDefault, s->stream));
        if (r.sigma) CUDA_TRY(cudaMemcpyAsync(base + bx + by, r.sigma, raw, cudaMemcpyDefault, s->stream));
        d.x = xs ? base : nullptr;
        d.x2 = xs == 2 ? base + ab : nullptr;
        d.y = base + bx;
        d.w = r.sigma ? base + bx + by : nullptr;
        d.wkind = r.sigma ? W_SIGMA : W_NONE;    // 1/sigma formed in the kernel
        d.tile_base = (int64_t)t0;
        d.group_base = (int64_t)g0;
        FitState* st = (FitState*)(s->hbuf + s->L->state) + free_slot;
        memset(st, 0, sizeof(FitState));
        const bool resumed = !p.resume.empty();
        if (resumed) {
            // the snapshot's state, pass constants for its pending evaluation included
            memcpy(st, p.resume.data(), p.resume.size());
            st->run = RS_RUNNING;
        } else {
            st->run = RS_RUNNING;
            st->phase = PH_INIT;
            for (int i = 0; i < n; ++i) { st->x[i] = r.p0[i]; st->xt[i] = r.p0[i]; st->scale_inv[i] = 1.0; }
        }
        FitDesc* hd = (FitDesc*)(s->hbuf + s->L->desc) + free_slot;
        *hd = d;
        CUDA_TRY(cudaMemcpyAsync(s->job + s->L->desc + (size_t)free_slot * sizeof(FitDesc), hd, sizeof(FitDesc),
                                 cudaMemcpyHostToDevice, s->stream));
        CUDA_TRY(cudaMemcpyAsync(s->job + s->L->state + (size_t)free_slot * sizeof(FitState), st, sizeof(FitState),
                                 cudaMemcpyHostToDevice, s->stream));
        SrvSlot& sl = s->slots[free_slot];
        sl.used = true;
        sl.ticket = p.ticket;
        sl.tag = r.tag;
        sl.data_off = off; sl.data_bytes = need;
        sl.tile0 = t0; sl.ntiles = nt; sl.group0 = g0; sl.ngroups = ng;
        sl.t_submit = p.t_submit;
        sl.t_admit = now_s();
        sl.n = n;
        sl.m = r.m;
        sl.model = r.model_id;
        for (int i = 0; i < n; ++i) sl.p0[i] = r.p0[i];
        admitted.push_back(free_slot);
        if (!resumed) fresh.push_back(free_slot);
        s->queue.pop_front();
    }
    // ---- counters of new fits start at zero; pass constants at p0
    Engine* Ed = (Engine*)s->job;
    for (int k : admitted) {
        SrvSlot& sl = s->slots[k];
        CUDA_TRY(cudaMemsetAsync(s->job + s->L->gcnt + sl.group0 * sizeof(int), 0, sl.ngroups * sizeof(int), s->stream));
        CUDA_TRY(cudaMemsetAsync(s->job + s->L->fcnt + (size_t)k * sizeof(int), 0, sizeof(int), s->stream));
    }
    if (!fresh.empty()) {
        int* hl = (int*)(s->hbuf + s->L->end);
        for (size_t k = 0; k < fresh.size(); ++k) hl[k] = fresh[k];
        CUDA_TRY(cudaMemcpyAsync(s->d_list, hl, fresh.size() * sizeof(int), cudaMemcpyHostToDevice, s->stream));
        int cnt = (int)fresh.size();
        void* a_init[] = {&Ed, &s->d_list, &cnt};
        CUDA_TRY(cudaLaunchKernel(kernel_init_slots(s->prec), dim3(cnt < 1024 ? cnt : 1024), dim3(32), a_init, 0, s->stream));
    }
    // ---- compacted work list of every resident fit, then the shared rounds
    int active = 0;
    WorkItem* hi = (WorkItem*)(s->hbuf + s->L->items);
    size_t ni = 0;
    for (int k = 0; k < s->max_slots; ++k)
        if (s->slots[k].used) {
            ++active;
            for (size_t t = 0; t < s->slots[k].ntiles; ++t) hi[ni++] = WorkItem{k, (int)t};
        }
    if (active > 0) {
        CUDA_TRY(cudaMemcpyAsync(s->job + s->L->items, hi, ni * sizeof(WorkItem), cudaMemcpyHostToDevice, s->stream));
        // loop scalars: items, running, rounds done, round cap, fits, barrier (count, generation, control)
        int sc8[8] = {(int)ni, active, 0, s->rounds, s->max_slots, 0, 0, 0};
        int* hsc = (int*)(s->hbuf + s->L->end + (size_t)s->max_slots * 4);
        memcpy(hsc, sc8, sizeof sc8);
        CUDA_TRY(cudaMemcpyAsync(&Ed->sc[0], hsc, sizeof sc8, cudaMemcpyHostToDevice, s->stream));
        CUDA_TRY(cudaMemsetAsync(s->job + s->L->res_hdr, 0, 32, s->stream));
        // per-SM CTA counters start at zero (a launch that aborted at its
        // set-up barrier leaves them as they were)
        CUDA_TRY(cudaMemsetAsync(s->job + s->L->smcnt, 0, (SM_IDS + 1) * sizeof(int), s->stream));
        int do_init = 0;
        void* a_loop[] = {&Ed, &do_init};
        CUDA_TRY(cudaLaunchCooperativeKernel(kernel_fit_loop(s->prec), dim3(s->grid), dim3(EVAL_THREADS), a_loop,
                                             eval_dyn_smem(s->prec), s->stream));
        int* hout = hsc + 8;
        CUDA_TRY(cudaMemcpyAsync(hout, s->job + s->L->res_hdr, 3 * sizeof(int), cudaMemcpyDeviceToHost, s->stream));
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        if (hout[2]) return fail(GBFIT_E_TIMEOUT, "a round barrier of the loop kernel timed out");
        {
            std::lock_guard<std::mutex> gs(g_stats_mu);
            g_stats.kernel_launches += 1 + (fresh.empty() ? 0 : 1);
        }
    }
    if ((rc = server_retire(s))) return rc;
    int act = 0;
    for (int k = 0; k < s->max_slots; ++k) act += s->slots[k].used;
    if (n_active) *n_active = act;
    if (n_queued) *n_queued = (int)s->queue.size();
    return GBFIT_OK;
}

int gbfit_server_poll(gbfit_server* s, gbfit_result_rec* out, int max, int* count) {
    if (!s || (!out && max > 0)) return fail(GBFIT_E_INVALID_ARG, "bad poll arguments");
    std::lock_guard<std::mutex> g(s->mu);
    int c = 0;
    while (c < max && !s->done.empty()) { out[c++] = s->done.front(); s->done.pop_front(); }
    if (count) *count = c;
    return GBFIT_OK;
}

int gbfit_server_cancel(gbfit_server* s, uint64_t ticket) {
    if (!s) return fail(GBFIT_E_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    gbfit_result_rec rec;
    memset(&rec, 0, sizeof rec);
    rec.ticket = ticket;
    rec.status = GBFIT_E_CANCELLED;
    rec.fit_status = FS_MAX_NFEV;
    rec.t_done = now_s();
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
        if (it->ticket == ticket) {                         // never started: p0, no evaluation
            const gbfit_request& r = it->req;
            rec.tag = r.tag;
            rec.n_params = model_nparams(r.model_id);
            for (int i = 0; i < rec.n_params; ++i) rec.popt[i] = r.p0[i];
            rec.cost = NAN;
            rec.t_submit = rec.t_admit = it->t_submit;
            s->queue.erase(it);
            s->done.push_back(rec);
            return GBFIT_OK;
        }
    for (int k = 0; k < s->max_slots; ++k) {
        SrvSlot& sl = s->slots[k];
        if (!sl.used || sl.ticket != ticket) continue;
        FitState st;
        int rc = server_read_state(s, k, &st);
        if (rc) return rc;
        rec.tag = sl.tag;
        rec.n_params = sl.n;
        for (int i = 0; i < sl.n; ++i) rec.popt[i] = (st.nfev > 0) ? st.x[i] : sl.p0[i];
        rec.cost = (st.nfev > 0) ? st.f : NAN;
        rec.nfev = st.nfev;
        rec.t_submit = sl.t_submit;
        rec.t_admit = sl.t_admit;
        s->done.push_back(rec);
        server_release(s, k);
        return GBFIT_OK;
    }
    return fail(GBFIT_E_INVALID_ARG, "ticket %llu is neither queued nor resident", (unsigned long long)ticket);
}

int gbfit_server_snapshot(gbfit_server* s, uint64_t ticket, gbfit_fit_snapshot* out) {
    if (!s || !out) return fail(GBFIT_E_INVALID_ARG, "server and out must not be NULL");
    std::lock_guard<std::mutex> g(s->mu);
    for (int k = 0; k < s->max_slots; ++k) {
        SrvSlot& sl = s->slots[k];
        if (!sl.used || sl.ticket != ticket) continue;
        memset(out, 0, sizeof *out);
        int rc = server_read_state(s, k, out->state);
        if (rc) return rc;
        out->magic = GBFIT_SNAPSHOT_MAGIC;
        out->state_bytes = (uint32_t)SNAP_STATE_BYTES;
        out->model_id = sl.model;
        out->precision = s->prec;
        out->m = sl.m;
        return GBFIT_OK;
    }
    return fail(GBFIT_E_INVALID_ARG, "ticket %llu is not resident (queued, finished or unknown)",
                (unsigned long long)ticket);
}

int gbfit_server_destroy(gbfit_server* s) {
    if (!s) return GBFIT_OK;
    if (s->stream) { cudaStreamSynchronize(s->stream); cudaStreamDestroy(s->stream); }
    if (s->pool) cudaFree(s->pool);
    if (s->job) cudaFree(s->job);
    if (s->tile_part_d) cudaFree(s->tile_part_d);
    if (s->group_part) cudaFree(s->group_part);
    if (s->d_list) cudaFree(s->d_list);
    if (s->hbuf) cudaFreeHost(s->hbuf);
    delete s->L;
    delete s;
    return GBFIT_OK;
}

}  // extern "C"

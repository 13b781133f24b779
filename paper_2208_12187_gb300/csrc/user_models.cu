// User-defined models: run-time compilation (NVRTC) of the library's loop
// kernels for a model given as source text, and the kernel sets the engine
// launches (built-in registry or one user model).
//
// The generated program includes the same device headers the library is
// built from (embedded at build time), the user's source in a namespace of
// its own, and the adapter of user_model.cuh; it instantiates
// fit_loop_kernel<precision, SingleModel<MUser<Def>>> for both precisions.
// NVRTC is opened with dlopen on first use, so the library itself does not
// depend on it.
#include <dlfcn.h>
#include <cctype>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gbfit.h"
#include "gbfit_internal.cuh"
#include "kernels.cuh"
#include "models.cuh"
#include "user_models.h"
#include "rtc_headers.inc"   // generated by the build: k_rtc_count, k_rtc_names[], k_rtc_srcs[]

namespace gbfit {
int set_error(int code, const char* msg);   // engine.cu: the thread's last error

namespace {

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_error(code, buf);
}

// ---- NVRTC entry points (nvrtcResult is an int enum, nvrtcProgram a pointer)
struct Nvrtc {
    typedef int (*create_t)(void**, const char*, const char*, int, const char* const*, const char* const*);
    typedef int (*compile_t)(void*, int, const char* const*);
    typedef int (*size_t_t)(void*, size_t*);
    typedef int (*get_t)(void*, char*);
    typedef int (*addname_t)(void*, const char*);
    typedef int (*lowered_t)(void*, const char*, const char**);
    typedef int (*destroy_t)(void**);
    typedef const char* (*errstr_t)(int);
    create_t create = nullptr;
    compile_t compile = nullptr;
    size_t_t log_size = nullptr, cubin_size = nullptr;
    get_t log = nullptr, cubin = nullptr;
    addname_t add_name = nullptr;
    lowered_t lowered = nullptr;
    destroy_t destroy = nullptr;
    errstr_t errstr = nullptr;
    bool tried = false, ok = false;
    std::string why;
};
Nvrtc g_nv;

bool open_nvrtc() {
    if (g_nv.tried) return g_nv.ok;
    g_nv.tried = true;
    std::vector<std::string> cand = {"libnvrtc.so.13", "libnvrtc.so"};
    for (const char* env : {"CUDA_HOME", "CUDA_PATH"})
        if (const char* h = getenv(env)) { cand.push_back(std::string(h) + "/lib64/libnvrtc.so.13"); cand.push_back(std::string(h) + "/lib64/libnvrtc.so"); }
    cand.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
    cand.push_back("/usr/local/cuda/lib64/libnvrtc.so");
    void* h = nullptr;
    for (auto& c : cand)
        if ((h = dlopen(c.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) { g_nv.why = "libnvrtc (CUDA toolkit) not found"; return false; }
    g_nv.create = (Nvrtc::create_t)dlsym(h, "nvrtcCreateProgram");
    g_nv.compile = (Nvrtc::compile_t)dlsym(h, "nvrtcCompileProgram");
    g_nv.log_size = (Nvrtc::size_t_t)dlsym(h, "nvrtcGetProgramLogSize");
    g_nv.log = (Nvrtc::get_t)dlsym(h, "nvrtcGetProgramLog");
    g_nv.cubin_size = (Nvrtc::size_t_t)dlsym(h, "nvrtcGetCUBINSize");
    g_nv.cubin = (Nvrtc::get_t)dlsym(h, "nvrtcGetCUBIN");
    g_nv.add_name = (Nvrtc::addname_t)dlsym(h, "nvrtcAddNameExpression");
    g_nv.lowered = (Nvrtc::lowered_t)dlsym(h, "nvrtcGetLoweredName");
    g_nv.destroy = (Nvrtc::destroy_t)dlsym(h, "nvrtcDestroyProgram");
    g_nv.errstr = (Nvrtc::errstr_t)dlsym(h, "nvrtcGetErrorString");
    g_nv.ok = g_nv.create && g_nv.compile && g_nv.log_size && g_nv.log && g_nv.cubin_size && g_nv.cubin &&
              g_nv.add_name && g_nv.lowered && g_nv.destroy && g_nv.errstr;
    if (!g_nv.ok) g_nv.why = "libnvrtc lacks an expected entry point";
    return g_nv.ok;
}

struct UserModel {
    int id = 0, n = 0, dims = 1;
    std::vector<char> cubin;
    std::string lowered[2];        // mangled names of the loop kernel per precision
    bool loaded = false;
    cudaLibrary_t lib = nullptr;
    KernelSet ks{};
};

std::mutex g_um_mu;
UserModel* g_um[GBFIT_MAX_USER_MODELS] = {};
int g_um_count = 0;
std::string g_um_log;

KernelSet make_builtin() {
    KernelSet k{};
    k.id = 0;
    for (int p = 0; p < 2; ++p) {
        k.fit_loop[p] = kernel_fit_loop(p);
        k.blocks_per_sm[p] = eval_blocks_per_sm(p);
        k.dyn_smem[p] = eval_dyn_smem(p);
    }
    return k;
}

bool valid_name(const char* s) {
    if (!s || !*s || !(isalpha((unsigned char)s[0]) || s[0] == '_')) return false;
    for (const char* c = s; *c; ++c)
        if (!(isalnum((unsigned char)*c) || *c == '_')) return false;
    return strlen(s) < 64;
}

}  // namespace

const KernelSet* builtin_kernels() {
    static std::once_flag once;
    static KernelSet k;
    std::call_once(once, [] { k = make_builtin(); });
    return &k;
}

bool is_user_model(int id) {
    int k = id - GBFIT_USER_MODEL_BASE;
    if (k < 0 || k >= GBFIT_MAX_USER_MODELS) return false;
    std::lock_guard<std::mutex> g(g_um_mu);
    return g_um[k] != nullptr;
}

bool model_shape(int id, int* n, int* dims) {
    if (id >= 0 && id < GBFIT_NUM_MODELS) {
        *n = model_nparams(id);
        *dims = model_xdims(id);
        return true;
    }
    int k = id - GBFIT_USER_MODEL_BASE;
    if (k < 0 || k >= GBFIT_MAX_USER_MODELS) return false;
    std::lock_guard<std::mutex> g(g_um_mu);
    if (!g_um[k]) return false;
    *n = g_um[k]->n;
    *dims = g_um[k]->dims;
    return true;
}

// A built-in model's own kernel set: the mixed loop kernel compiled for that
// model alone, the all-model FP64 kernel (ids -1 - model keep the engine's
// cached graphs apart from the registry's).  Models without a single-model
// instantiation use the registry's set.
const KernelSet* builtin_single_kernels(int model) {
    static std::once_flag once[GBFIT_NUM_MODELS];
    static KernelSet k[GBFIT_NUM_MODELS];
    std::call_once(once[model], [model] {
        const KernelSet* all = builtin_kernels();
        k[model] = *all;
        const void* f = kernel_fit_loop_single_mixed(model);
        const int b = f ? blocks_per_sm_single_mixed(model) : 0;
        // the single-model grid must not exceed the all-model kernel's (both fit its scratch)
        if (f && b >= 1 && b <= all->blocks_per_sm[PREC_MIXED]) {
            k[model].id = -1 - model;
            k[model].fit_loop[PREC_MIXED] = f;
            k[model].blocks_per_sm[PREC_MIXED] = b;
        }
    });
    return &k[model];
}

int kernels_for_model(int id, const KernelSet** out) {
    if (id >= 0 && id < GBFIT_NUM_MODELS) { *out = builtin_single_kernels(id); return GBFIT_OK; }
    int k = id - GBFIT_USER_MODEL_BASE;
    if (k < 0 || k >= GBFIT_MAX_USER_MODELS) return fail(GBFIT_E_INVALID_ARG, "unknown model %d", id);
    std::lock_guard<std::mutex> g(g_um_mu);
    UserModel* u = g_um[k];
    if (!u) return fail(GBFIT_E_INVALID_ARG, "unknown model %d", id);
    if (!u->loaded) {
        cudaError_t e = cudaLibraryLoadData(&u->lib, u->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
        if (e != cudaSuccess) return fail(GBFIT_E_CUDA, "loading user model %d: %s", id, cudaGetErrorString(e));
        u->ks.id = id;
        for (int p = 0; p < 2; ++p) {
            cudaKernel_t kern;
            e = cudaLibraryGetKernel(&kern, u->lib, u->lowered[p].c_str());
            if (e != cudaSuccess) return fail(GBFIT_E_CUDA, "user model %d kernel: %s", id, cudaGetErrorString(e));
            const void* f = (const void*)kern;
            const int dyn = (int)eval_dyn_smem(p);
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
            if (e == cudaSuccess && p == PREC_MIXED)     // two CTAs with their bulk-copy rings per SM
                e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
            int b = 0;
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, EVAL_THREADS, dyn);
            if (e != cudaSuccess) return fail(GBFIT_E_CUDA, "user model %d occupancy: %s", id, cudaGetErrorString(e));
            if (b < 1) return fail(GBFIT_E_CUDA, "user model %d: its loop kernel does not fit on an SM", id);
            u->ks.fit_loop[p] = f;
            u->ks.blocks_per_sm[p] = b;
            u->ks.dyn_smem[p] = (size_t)dyn;
        }
        u->loaded = true;
    }
    *out = &u->ks;
    return GBFIT_OK;
}

}  // namespace gbfit

using namespace gbfit;

extern "C" int gbfit_model_register(const char* source, const char* func_name, int n_params, int x_dims,
                                    int* model_id) {
    if (!source || !model_id) return fail(GBFIT_E_INVALID_ARG, "source and model_id must not be NULL");
    if (n_params < 1 || n_params > GBFIT_MAX_PARAMS)
        return fail(GBFIT_E_INVALID_ARG, "n_params must be in [1, %d]", GBFIT_MAX_PARAMS);
    if (x_dims != 1 && x_dims != 2) return fail(GBFIT_E_INVALID_ARG, "x_dims must be 1 or 2");
    const char* fname = func_name ? func_name : "model";
    if (!valid_name(fname)) return fail(GBFIT_E_INVALID_ARG, "func_name must be a C identifier");
    {
        std::lock_guard<std::mutex> g(g_um_mu);
        if (g_um_count >= GBFIT_MAX_USER_MODELS) return fail(GBFIT_E_OOM, "at most %d user models", GBFIT_MAX_USER_MODELS);
    }
    static std::mutex compile_mu;          // one compilation at a time (NVRTC state and the log)
    std::lock_guard<std::mutex> cg(compile_mu);
    if (!open_nvrtc()) return fail(GBFIT_E_UNSUPPORTED, "user models need NVRTC: %s", g_nv.why.c_str());

    std::string src;
    src += "#include \"round_kernels.cuh\"\n#include \"user_model.cuh\"\n";
    src += "namespace gbfit_user_src {\n#line 1 \"user_source\"\n";
    src += source;
    src += "\n}\n";
    char def[512];
    snprintf(def, sizeof def,
             "struct GbfitUserDef {\n"
             "    static constexpr int N = %d;\n"
             "    static constexpr int DIM = %d;\n"
             "    template <class T, class S> __device__ static T h(const T* p, S x, S x2) {\n"
             "        return gbfit_user_src::%s<T, S>(p, x, x2);\n"
             "    }\n"
             "};\n"
             "using GbfitUserSet = gbfit::SingleModel<gbfit::MUser<GbfitUserDef>>;\n",
             n_params, x_dims, fname);
    src += def;

    void* prog = nullptr;
    int r = g_nv.create(&prog, src.c_str(), "gbfit_user_model.cu", k_rtc_count, k_rtc_srcs, k_rtc_names);
    if (r != 0) return fail(GBFIT_E_UNSUPPORTED, "nvrtcCreateProgram: %s", g_nv.errstr(r));
    std::string names[2] = {"&gbfit::fit_loop_kernel<0, GbfitUserSet>", "&gbfit::fit_loop_kernel<1, GbfitUserSet>"};
    for (auto& nm : names) g_nv.add_name(prog, nm.c_str());
    char words[64];
    snprintf(words, sizeof words, "-DGBFIT_STATE_WORDS=%d", (int)(offsetof(FitState, trace) / 16));
    const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", "-lineinfo", words};
    r = g_nv.compile(prog, (int)(sizeof opts / sizeof opts[0]), opts);
    size_t ls = 0;
    g_nv.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) g_nv.log(prog, &log[0]);
    while (!log.empty() && log.back() == '\0') log.pop_back();
    {
        std::lock_guard<std::mutex> g(g_um_mu);
        g_um_log = log;
    }
    if (r != 0) {
        g_nv.destroy(&prog);
        return fail(GBFIT_E_INVALID_ARG, "user model does not compile: %.400s", log.c_str());
    }
    UserModel* u = new UserModel();
    u->n = n_params;
    u->dims = x_dims;
    size_t cs = 0;
    g_nv.cubin_size(prog, &cs);
    u->cubin.resize(cs);
    g_nv.cubin(prog, u->cubin.data());
    for (int p = 0; p < 2; ++p) {
        const char* low = nullptr;
        if (g_nv.lowered(prog, names[p].c_str(), &low) != 0 || !low) {
            g_nv.destroy(&prog);
            delete u;
            return fail(GBFIT_E_UNSUPPORTED, "nvrtcGetLoweredName failed");
        }
        u->lowered[p] = low;
    }
    g_nv.destroy(&prog);
    std::lock_guard<std::mutex> g(g_um_mu);
    if (g_um_count >= GBFIT_MAX_USER_MODELS) { delete u; return fail(GBFIT_E_OOM, "at most %d user models", GBFIT_MAX_USER_MODELS); }
    u->id = GBFIT_USER_MODEL_BASE + g_um_count;
    g_um[g_um_count++] = u;
    *model_id = u->id;
    return GBFIT_OK;
}

extern "C" int gbfit_model_log(char* buf, size_t cap, size_t* len) {
    std::lock_guard<std::mutex> g(g_um_mu);
    if (len) *len = g_um_log.size();
    if (buf && cap) {
        size_t k = g_um_log.size() < cap - 1 ? g_um_log.size() : cap - 1;
        memcpy(buf, g_um_log.data(), k);
        buf[k] = '\0';
    }
    return GBFIT_OK;
}

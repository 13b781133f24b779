// Staging of a full-covariance fit (Appendix C, Eq. covariance): the
// Cholesky factor C = L L^T and the inverse factor X = L^-1, in FP64 on the
// device.  The fit's passes then reduce rows of X [h - y, J] (the weighted
// residual and Jacobian of Eqs. slsq1, slsq2).
//
// Matrices are column-major (element (i, j) at [j ld + i]); a symmetric C
// reads the same in either order.  The factorisation works on C padded to
// mp = 32 ceil(m / 32) with the identity in the padding (its factor and
// inverse are then the padded L and X), in 32 x 32 blocks:
//   Cholesky, per block column kb (three grid barriers):
//     1. one CTA factors the diagonal block (unblocked, in shared memory)
//        and inverts its factor;
//     2. the blocks below it: A_ib,kb <- A_ib,kb L_kk^-T;
//     3. the trailing blocks: A_ib,jb -= A_ib,kb A_jb,kb^T (kb < jb <= ib).
//   Inverse, right-looking over block rows kb (two grid barriers):
//     1. X_kb,jb <- L_kk^-1 T_kb,jb for jb <= kb (T starts as I);
//     2. T_ib,jb -= L_ib,kb X_kb,jb for ib > kb, jb <= kb.
// Every step is a set of independent 32 x 32 x 32 block products spread over
// the cooperative grid.
#include "gbfit_internal.cuh"
#include "sync_device.cuh"
#include "kernels.cuh"

namespace gbfit {
namespace {

constexpr unsigned long long COV_WAIT_LIMIT_NS = 10ull * 1000 * 1000 * 1000;
constexpr int COV_THREADS = 256;           // 8 warps: a thread owns row (t & 31), columns (t >> 5) + 8 u
constexpr int NB = 32;                     // block size
constexpr int LDS = NB + 1;                // shared-memory column stride (no bank conflicts)
constexpr size_t COV_BLOCK_SMEM = 3 * NB * LDS * sizeof(double);

// Grid-wide barrier of a cooperative launch, bounded in time: false (and
// flag bit 2) when the wait gave up.  sync: {arrivals, generation}.
__device__ bool coop_sync(unsigned* sync, int* flag) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        unsigned* cnt = sync;
        unsigned* gen = sync + 1;
        const unsigned g = ld_acquire_u32(gen);
        unsigned old;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(cnt) : "memory");
        if (old == gridDim.x - 1) {
            *(volatile unsigned*)cnt = 0;
            st_release_u32(gen, g + 1);
        } else {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_u32(gen) == g) {
                __nanosleep(64);
                if (global_ns() - t0 > COV_WAIT_LIMIT_NS) {
                    ok = 0;
                    atomicOr(flag, 2);
                    break;
                }
            }
        }
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ int read_flag(const int* flag) {
    return (int)ld_acquire_u32(reinterpret_cast<const unsigned*>(flag));
}

// Block (rb, cb) of a column-major matrix (leading dimension ld) into shared
// memory s (column-major, stride LDS); L2 loads (other CTAs wrote it).
__device__ __forceinline__ void load_blk(double* s, const double* A, int64_t ld, int rb, int cb) {
    const int r = threadIdx.x & 31, c0 = threadIdx.x >> 5;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int c = c0 + 8 * u;
        s[c * LDS + r] = __ldcg(A + (int64_t)(cb * NB + c) * ld + rb * NB + r);
    }
}

// acc_u = sum_k a(r, k) b(k, c_u) for this thread's r and c_u: a from As
// (column-major); b(k, c) = Bs[k LDS + c] when BT (B given as its
// transpose's storage), else Bs[c LDS + k].
template <bool BT>
__device__ __forceinline__ void blk_mm(const double* As, const double* Bs, double (&acc)[4]) {
    const int r = threadIdx.x & 31, c0 = threadIdx.x >> 5;
#pragma unroll 8
    for (int k = 0; k < NB; ++k) {
        const double a = As[k * LDS + r];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = c0 + 8 * u;
            acc[u] = fma(a, BT ? Bs[k * LDS + c] : Bs[c * LDS + k], acc[u]);
        }
    }
}

__device__ __forceinline__ void store_blk(double* A, int64_t ld, int rb, int cb, const double (&v)[4]) {
    const int r = threadIdx.x & 31, c0 = threadIdx.x >> 5;
#pragma unroll
    for (int u = 0; u < 4; ++u) A[(int64_t)(cb * NB + c0 + 8 * u) * ld + rb * NB + r] = v[u];
}

// A: [mp][mp] C padded with the identity (the padding's diagonal is set
// here); on exit its lower triangle holds L (strict upper blocks untouched,
// upper triangles of diagonal blocks zero).  W: [mp / 32][32][32] the
// inverses of the diagonal blocks of L.  flag bit 1: a pivot was not
// positive (C not positive definite); every CTA reads the flag after the
// same barrier and leaves.
__global__ void __launch_bounds__(COV_THREADS) chol_blocked_kernel(double* A, double* W, int m, int mp,
                                                                   unsigned* sync, int* flag) {
    extern __shared__ double smem[];
    double* S0 = smem;
    double* S1 = smem + NB * LDS;
    double* S2 = smem + 2 * NB * LDS;
    const int t = threadIdx.x;
    const int nb = mp / NB;
    for (int i = m + blockIdx.x * COV_THREADS + t; i < mp; i += gridDim.x * COV_THREADS) A[(int64_t)i * mp + i] = 1.0;
    if (!coop_sync(sync, flag)) return;
    for (int kb = 0; kb < nb; ++kb) {
        // 1. the diagonal block and its inverse (CTA 0)
        if (blockIdx.x == 0) {
            load_blk(S0, A, mp, kb, kb);
            __shared__ double dk;
            for (int k = 0; k < NB; ++k) {
                __syncthreads();
                if (t == 0) {
                    const double piv = S0[k * LDS + k];
                    const bool ok = piv > 0.0 && isfinite(piv);
                    if (!ok) atomicOr(flag, 1);
                    dk = ok ? sqrt(piv) : 1.0;
                    S0[k * LDS + k] = dk;
                }
                __syncthreads();
                if (t > k && t < NB) S0[k * LDS + t] /= dk;
                __syncthreads();
                for (int e = t; e < NB * NB; e += COV_THREADS) {
                    const int r = e & 31, c = e >> 5;
                    if (c > k && r >= c) S0[c * LDS + r] = fma(-S0[k * LDS + r], S0[k * LDS + c], S0[c * LDS + r]);
                }
            }
            __syncthreads();
            // write L_kk (zero above the diagonal); reciprocal diagonal in S2
            for (int e = t; e < NB * NB; e += COV_THREADS) {
                const int r = e & 31, c = e >> 5;
                A[(int64_t)(kb * NB + c) * mp + kb * NB + r] = (r >= c) ? S0[c * LDS + r] : 0.0;
            }
            if (t < NB) S2[t] = 1.0 / S0[t * LDS + t];
            __syncthreads();
            // inverse of L_kk: thread c forward-substitutes column c
            if (t < NB) {
                const int c = t;
                for (int r = 0; r < NB; ++r) {
                    double v = 0.0;
                    if (r >= c) {
                        double s = (r == c) ? 1.0 : 0.0;
                        for (int k = c; k < r; ++k) s = fma(-S0[k * LDS + r], S1[c * LDS + k], s);
                        v = s * S2[r];
                    }
                    S1[c * LDS + r] = v;
                }
            }
            __syncthreads();
            double* Wk = W + (int64_t)kb * NB * NB;
            for (int e = t; e < NB * NB; e += COV_THREADS) {
                const int r = e & 31, c = e >> 5;
                Wk[c * NB + r] = S1[c * LDS + r];
            }
        }
        if (!coop_sync(sync, flag)) return;
        if (read_flag(flag) & 1) return;
        // 2. the panel below: A_ib,kb <- A_ib,kb L_kk^-T
        const double* Wk = W + (int64_t)kb * NB * NB;
        for (int ib = kb + 1 + blockIdx.x; ib < nb; ib += gridDim.x) {
            __syncthreads();
            load_blk(S0, A, mp, ib, kb);
            load_blk(S1, Wk, NB, 0, 0);
            __syncthreads();
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            blk_mm<true>(S0, S1, acc);             // b(k, c) = L_kk^-1(c, k)
            __syncthreads();
            store_blk(A, mp, ib, kb, acc);
        }
        if (!coop_sync(sync, flag)) return;
        // 3. the trailing blocks: A_ib,jb -= A_ib,kb A_jb,kb^T, kb < jb <= ib
        const int tb = nb - kb - 1;
        const int64_t pairs = (int64_t)tb * (tb + 1) / 2;
        for (int64_t q = blockIdx.x; q < pairs; q += gridDim.x) {
            int a = (int)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
            while ((int64_t)(a + 1) * (a + 2) / 2 <= q) ++a;
            while ((int64_t)a * (a + 1) / 2 > q) --a;
            const int b = (int)(q - (int64_t)a * (a + 1) / 2);
            const int ib = kb + 1 + a, jb = kb + 1 + b;
            __syncthreads();
            load_blk(S0, A, mp, ib, kb);
            load_blk(S1, A, mp, jb, kb);
            load_blk(S2, A, mp, ib, jb);
            __syncthreads();
            double acc[4];
            const int r = t & 31, c0 = t >> 5;
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = -S2[(c0 + 8 * u) * LDS + r];
            blk_mm<true>(S0, S1, acc);             // -(C - A_ik A_jk^T)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = -acc[u];
            store_blk(A, mp, ib, jb, acc);
        }
        if (!coop_sync(sync, flag)) return;
    }
}

// X = L^-1 ([mp][mp], zeroed by the host): right-looking block forward
// substitution with the diagonal blocks' inverses W.
__global__ void __launch_bounds__(COV_THREADS) trinv_blocked_kernel(const double* L, const double* W, double* X,
                                                                    int mp, unsigned* sync, int* flag) {
    extern __shared__ double smem[];
    double* S0 = smem;
    double* S1 = smem + NB * LDS;
    const int t = threadIdx.x;
    const int nb = mp / NB;
    if (read_flag(flag)) return;             // the factorisation failed: every CTA leaves here
    for (int i = blockIdx.x * COV_THREADS + t; i < mp; i += gridDim.x * COV_THREADS) X[(int64_t)i * mp + i] = 1.0;
    if (!coop_sync(sync, flag)) return;
    for (int kb = 0; kb < nb; ++kb) {
        // 1. X_kb,jb <- L_kk^-1 T_kb,jb
        const double* Wk = W + (int64_t)kb * NB * NB;
        for (int jb = blockIdx.x; jb <= kb; jb += gridDim.x) {
            __syncthreads();
            load_blk(S0, Wk, NB, 0, 0);
            load_blk(S1, X, mp, kb, jb);
            __syncthreads();
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            blk_mm<false>(S0, S1, acc);            // b(k, c) = T(k, c)
            __syncthreads();
            store_blk(X, mp, kb, jb, acc);
        }
        if (!coop_sync(sync, flag)) return;
        // 2. T_ib,jb -= L_ib,kb X_kb,jb
        const int64_t pairs = (int64_t)(nb - kb - 1) * (kb + 1);
        for (int64_t q = blockIdx.x; q < pairs; q += gridDim.x) {
            const int ib = kb + 1 + (int)(q / (kb + 1)), jb = (int)(q % (kb + 1));
            __syncthreads();
            load_blk(S0, L, mp, ib, kb);
            load_blk(S1, X, mp, kb, jb);
            __syncthreads();
            double acc[4];
            const int r = t & 31, c0 = t >> 5;
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = -__ldcg(X + (int64_t)(jb * NB + c0 + 8 * u) * mp + ib * NB + r);
            blk_mm<false>(S0, S1, acc);            // -(T - L X)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = -acc[u];
            store_blk(X, mp, ib, jb, acc);
        }
        if (!coop_sync(sync, flag)) return;
    }
}

// The top-left m x m of X ([mp][mp]) into Xc ([m][m], FP64) and Xf (FP32, optional).
__global__ void compact_kernel(const double* X, int mp, int m, double* Xc, float* Xf) {
    const int64_t n = (int64_t)m * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / m, i = e - j * m;
        const double v = X[j * mp + i];
        Xc[e] = v;
        if (Xf) Xf[e] = float(v);
    }
}

int coop_grid(const void* k, int sms, int want) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, COV_THREADS, COV_BLOCK_SMEM) != cudaSuccess)
        return 0;
    int g = sms * (per_sm < 1 ? 0 : per_sm);
    return g < want ? g : want;
}

}  // namespace

size_t cov_padded(int m) { return (size_t)((m + NB - 1) / NB) * NB; }

cudaError_t launch_cov_factor(double* A, double* W, double* X, double* Xc, float* Xf, int m, unsigned* sync,
                              int* flag, int sms, cudaStream_t s) {
    const int mp = (int)cov_padded(m);
    const int nb = mp / NB;
    cudaError_t e = cudaFuncSetAttribute(chol_blocked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)COV_BLOCK_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(trinv_blocked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)COV_BLOCK_SMEM);
    if (e != cudaSuccess) return e;
    // enough CTAs for the widest step (nb (nb + 1) / 2 trailing blocks), every one resident
    const int want = nb * (nb + 1) / 2 > 1 ? nb * (nb + 1) / 2 : 1;
    int g1 = coop_grid((const void*)chol_blocked_kernel, sms, want);
    int g2 = coop_grid((const void*)trinv_blocked_kernel, sms, want);
    if (g1 < 1 || g2 < 1) return cudaErrorLaunchOutOfResources;
    void* a1[] = {&A, &W, &m, (void*)&mp, &sync, &flag};
    e = cudaLaunchCooperativeKernel((const void*)chol_blocked_kernel, dim3(g1), dim3(COV_THREADS), a1,
                                    COV_BLOCK_SMEM, s);
    if (e != cudaSuccess) return e;
    const double* Lc = A;
    const double* Wc = W;
    void* a2[] = {(void*)&Lc, (void*)&Wc, &X, (void*)&mp, &sync, &flag};
    e = cudaLaunchCooperativeKernel((const void*)trinv_blocked_kernel, dim3(g2), dim3(COV_THREADS), a2,
                                    COV_BLOCK_SMEM, s);
    if (e != cudaSuccess) return e;
    compact_kernel<<<sms * 4, 256, 0, s>>>(X, mp, m, Xc, Xf);
    return cudaGetLastError();
}

}  // namespace gbfit

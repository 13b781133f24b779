// Staging of a full-covariance fit (Appendix C, Eq. covariance): the
// Cholesky factor C = L L^T and the inverse factor X = L^-1, both in FP64 on
// the device.  The fit's passes then reduce rows of X [h - y, J] (the
// weighted residual and Jacobian of Eqs. slsq1, slsq2).
//
// Matrices are [m][m] column-major (element (i, j) at [j m + i]); a
// symmetric C reads the same in either order.
#include "gbfit_internal.cuh"
#include "sync_device.cuh"
#include "kernels.cuh"

namespace gbfit {
namespace {

constexpr unsigned long long COV_WAIT_LIMIT_NS = 10ull * 1000 * 1000 * 1000;
constexpr int COV_THREADS = 256;

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

// Right-looking Cholesky without square roots in the loop: step k subtracts
// A_ik A_jk / A_kk from every A_ij, k < j <= i (the Schur complement); one
// grid barrier per step.  Afterwards column k is scaled by 1/sqrt(A_kk).
// flag bit 1: a pivot was not positive (C not positive definite).  Every
// CTA reads the same pivot after the barrier, so all leave together.
// rdiag[k] = 1 / L_kk for the inverse.
__global__ void __launch_bounds__(COV_THREADS) chol_kernel(double* A, double* rdiag, int m, unsigned* sync,
                                                           int* flag) {
    for (int k = 0; k < m; ++k) {
        const double piv = __ldcg(A + (int64_t)k * m + k);
        if (!(piv > 0.0) || !isfinite(piv)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(flag, 1);
            return;
        }
        const double ip = 1.0 / piv;
        const double* ck = A + (int64_t)k * m;
        for (int j = k + 1 + blockIdx.x; j < m; j += gridDim.x) {
            const double f = __ldcg(ck + j) * ip;
            double* col = A + (int64_t)j * m;
            for (int i = j + threadIdx.x; i < m; i += blockDim.x) col[i] = fma(-__ldcg(ck + i), f, __ldcg(col + i));
        }
        if (!coop_sync(sync, flag)) return;
    }
    for (int k = blockIdx.x; k < m; k += gridDim.x) {
        double* col = A + (int64_t)k * m;
        const double piv = __ldcg(col + k);
        __syncthreads();                          // every thread has the pivot before it is overwritten
        const double s = 1.0 / sqrt(piv);
        for (int i = threadIdx.x; i < m; i += blockDim.x) col[i] = (i < k) ? 0.0 : __ldcg(col + i) * s;
        if (threadIdx.x == 0) rdiag[k] = s;       // 1 / L_kk
        __syncthreads();
    }
}

// X = L^-1 by forward substitution, one column per CTA at a time:
// x_j = 1 / L_jj, x_i = -(sum_{k=j}^{i-1} L_ik x_k) / L_ii, right-looking
// (after x_k is known, every later row's running sum takes L_ik x_k).
// Dynamic shared memory: m doubles of running sums.
__global__ void __launch_bounds__(COV_THREADS) trinv_kernel(const double* L, const double* rdiag, double* X, int m) {
    extern __shared__ double sums[];
    __shared__ double xk;
    for (int j = blockIdx.x; j < m; j += gridDim.x) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) sums[i] = 0.0;
        __syncthreads();
        double* xc = X + (int64_t)j * m;
        for (int k = j; k < m; ++k) {
            if (threadIdx.x == 0) {
                xk = ((k == j ? 1.0 : 0.0) - sums[k]) * rdiag[k];
                xc[k] = xk;
            }
            __syncthreads();
            const double v = xk;
            const double* lk = L + (int64_t)k * m;
            for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) sums[i] = fma(lk[i], v, sums[i]);
            __syncthreads();
        }
        for (int i = threadIdx.x; i < j; i += blockDim.x) xc[i] = 0.0;
        __syncthreads();
    }
}

__global__ void to_f32_kernel(const double* a, float* b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = float(a[i]);
}

}  // namespace

cudaError_t launch_cov_factor(double* A, double* rdiag, double* X, float* Xf, int m, unsigned* sync, int* flag,
                              int sms, cudaStream_t s) {
    // the cooperative grid: every CTA resident
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_kernel, COV_THREADS, 0);
    if (e != cudaSuccess) return e;
    int grid = sms * (per_sm < 1 ? 1 : per_sm);
    if (grid > m) grid = m > 0 ? m : 1;
    void* a1[] = {&A, &rdiag, &m, &sync, &flag};
    e = cudaLaunchCooperativeKernel((const void*)chol_kernel, dim3(grid), dim3(COV_THREADS), a1, 0, s);
    if (e != cudaSuccess) return e;
    const size_t dyn = (size_t)m * sizeof(double);
    if (dyn > 48 * 1024) {
        e = cudaFuncSetAttribute(trinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    int g2 = sms * 2 < m ? sms * 2 : m;
    trinv_kernel<<<g2, COV_THREADS, dyn, s>>>(A, rdiag, X, m);
    e = cudaGetLastError();
    if (e != cudaSuccess || !Xf) return e;
    to_f32_kernel<<<sms * 4, 256, 0, s>>>(X, Xf, (int64_t)m * m);
    return cudaGetLastError();
}

}  // namespace gbfit

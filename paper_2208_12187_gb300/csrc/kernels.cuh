// Kernel declarations shared between kernels.cu and the host engine.
#pragma once
#include "gbfit_internal.cuh"
#include "trf_device.cuh"

namespace gbfit {
// Host-side handles to the kernels of kernels*.cu (kept non-template so that
// the host engine never names a template kernel of another translation unit).
void* kernel_eval_round_mixed();
void* kernel_eval_round_fp64();
void* kernel_init_fits_mixed();
void* kernel_init_fits_fp64();
void* kernel_fit_loop_mixed();
void* kernel_fit_loop_fp64();
void* kernel_init_slots_mixed();
void* kernel_init_slots_fp64();
int eval_blocks_per_sm_mixed();
int eval_blocks_per_sm_fp64();
int eval_round_blocks_per_sm_mixed();      // resident CTAs per SM of the single-round kernel alone
int eval_round_blocks_per_sm_fp64();
size_t eval_dyn_smem_mixed();
size_t eval_dyn_smem_fp64();
void* kernel_eval_round(int prec);
void* kernel_init_fits(int prec);
void* kernel_init_slots(int prec);
void* kernel_fit_loop(int prec);
int eval_blocks_per_sm(int prec);
size_t eval_dyn_smem(int prec);
cudaError_t launch_stage_weights(bool f64, const void* sigma, double* w, int64_t m, int blocks, cudaStream_t s);
cudaError_t launch_synth_fill(int model, bool f64, void* x, void* x2, void* y, int64_t total, int64_t period,
                              uint32_t seed, int blocks, const double* truth, cudaStream_t s);
// Full covariance: A ([mp][mp] FP64 column-major, mp = cov_padded(m), C in
// the top-left m x m, zeros elsewhere) is factored in place into L; X
// ([mp][mp], zeroed) receives L^-1; W ([mp][32]) the diagonal blocks'
// inverses; Xc ([m][m] FP64, may alias A) and Xf ([m][m] FP32, optional)
// the compact inverse.  flag: bit 1 not positive definite, bit 2 a grid
// barrier gave up.  sync: two zeroed words.
size_t cov_padded(int m);
cudaError_t launch_cov_factor(double* A, double* W, double* X, double* Xc, float* Xf, int m, unsigned* sync,
                              int* flag, int sms, cudaStream_t s);
cudaError_t launch_tr_subproblem(int n, const double* B, const double* g, double Delta, double alpha0,
                                 double* p_out, double* alpha_out, double* lam_out, cudaStream_t s);
cudaError_t launch_rcp64(const double* x, double* y, int64_t n, int blocks, cudaStream_t s);
// Keeps the stream busy for about ns nanoseconds (profiling: queued before a timed launch).
cudaError_t launch_hold(unsigned long long ns, cudaStream_t s);
// The mixed loop kernel compiled for built-in model `model` alone (the 1D
// Gaussian; null for the others) and its resident CTAs per SM
// (kernels_single.cu).
const void* kernel_fit_loop_single_mixed(int model);
int blocks_per_sm_single_mixed(int model);
}  // namespace gbfit

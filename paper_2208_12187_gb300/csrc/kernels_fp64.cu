// The plain FP64 instantiation of the loop kernel (one translation unit per
// precision and kernel, so that they compile in parallel; the single-round
// kernel of the allocation-free entry point is in kernels_fp64_eval.cu).
#include "round_kernels.cuh"
#include "kernels.cuh"

namespace gbfit {

void* kernel_init_fits_fp64() { return (void*)init_fits_kernel<PREC_FP64, BuiltinModels>; }
void* kernel_fit_loop_fp64() { return (void*)fit_loop_kernel<PREC_FP64, BuiltinModels>; }
void* kernel_init_slots_fp64() { return (void*)init_slots_kernel<PREC_FP64, BuiltinModels>; }

// Resident CTAs per SM of the round kernels (the loop kernel's cooperative
// grid is this times the SM count, so both kernels must fit it).
int eval_blocks_per_sm_fp64() {
    const int dyn = (int)(COV_SMEM_BYTES);          // scratch of the covariance row rounds
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(fit_loop_kernel<PREC_FP64, BuiltinModels>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        attr_set = true;
    }
    int b2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, fit_loop_kernel<PREC_FP64, BuiltinModels>, EVAL_THREADS, dyn);
    const int b = eval_round_blocks_per_sm_fp64();
    return b < b2 ? b : b2;
}
size_t eval_dyn_smem_fp64() { return COV_SMEM_BYTES; }

}  // namespace gbfit

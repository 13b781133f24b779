// The plain FP64 instantiation of the single-round kernel (the
// allocation-free entry point's), in a translation unit of its own so that it
// compiles in parallel with the loop kernel's.
#include "round_kernels.cuh"
#include "kernels.cuh"

namespace gbfit {

void* kernel_eval_round_fp64() { return (void*)eval_round_kernel<PREC_FP64, BuiltinModels>; }

int eval_round_blocks_per_sm_fp64() {
    const int dyn = (int)(COV_SMEM_BYTES);          // scratch of the covariance row rounds
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(eval_round_kernel<PREC_FP64, BuiltinModels>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        attr_set = true;
    }
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, eval_round_kernel<PREC_FP64, BuiltinModels>, EVAL_THREADS, dyn);
    return b;
}

}  // namespace gbfit

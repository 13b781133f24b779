// The mixed-precision instantiation of the single-round kernel (the
// allocation-free entry point's), in a translation unit of its own so that it
// compiles in parallel with the loop kernel's.
#include "round_kernels.cuh"
#include "kernels.cuh"

namespace gbfit {

void* kernel_eval_round_mixed() { return (void*)eval_round_kernel<PREC_MIXED, BuiltinModels>; }

int eval_round_blocks_per_sm_mixed() {
    const int dyn = (int)(RING_BYTES);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(eval_round_kernel<PREC_MIXED, BuiltinModels>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        cudaFuncSetAttribute(eval_round_kernel<PREC_MIXED, BuiltinModels>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        attr_set = true;
    }
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, eval_round_kernel<PREC_MIXED, BuiltinModels>, EVAL_THREADS, dyn);
    return b;
}

}  // namespace gbfit

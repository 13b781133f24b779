// The mixed-precision instantiation of the loop kernel (one translation unit
// per precision and kernel, so that they compile in parallel; the single-round
// kernel of the allocation-free entry point is in kernels_mixed_eval.cu).
#include "round_kernels.cuh"
#include "kernels.cuh"

namespace gbfit {

void* kernel_init_fits_mixed() { return (void*)init_fits_kernel<PREC_MIXED, BuiltinModels>; }
void* kernel_fit_loop_mixed() { return (void*)fit_loop_kernel<PREC_MIXED, BuiltinModels>; }
void* kernel_init_slots_mixed() { return (void*)init_slots_kernel<PREC_MIXED, BuiltinModels>; }

// Resident CTAs per SM of the round kernels (the loop kernel's cooperative
// grid is this times the SM count, so both kernels must fit it).
int eval_blocks_per_sm_mixed() {
    const int dyn = (int)(RING_BYTES);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(fit_loop_kernel<PREC_MIXED, BuiltinModels>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        // the whole unified L1 / shared array as shared memory: two CTAs with their rings per SM
        cudaFuncSetAttribute(fit_loop_kernel<PREC_MIXED, BuiltinModels>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        attr_set = true;
    }
    int b2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, fit_loop_kernel<PREC_MIXED, BuiltinModels>, EVAL_THREADS, dyn);
    const int b = eval_round_blocks_per_sm_mixed();
    return b < b2 ? b : b2;
}
size_t eval_dyn_smem_mixed() { return RING_BYTES; }

}  // namespace gbfit

// Single-model instantiation of the mixed-precision loop kernel for the 1D
// Gaussian.  A launch whose fits are all 1D Gaussians (a single fit, a batch,
// an evaluation) runs the kernel compiled for that model alone: its code and
// register allocation carry only that model's paths (24 B of stack and 32 B
// of spills against ~1 KB and ~0.7 KB for the all-model kernel; measured:
// a 5e7-point pass 164 -> 155 us, a 1e6-point fit 132 -> 118 us).  The same
// instantiation for the 2D Gaussian spills ~6 KB in its streaming loop and
// the double exponential's runs slower than the all-model kernel, so those
// models, and serving (models mixed in one launch), keep the all-model kernel.
#include "round_kernels.cuh"
#include "user_model.cuh"
#include "kernels.cuh"

namespace gbfit {

namespace {
template <class M>
const void* loop_mixed() { return (const void*)fit_loop_kernel<PREC_MIXED, SingleModel<M>>; }

template <class M>
int blocks_mixed() {
    const void* f = loop_mixed<M>();
    const int dyn = (int)RING_BYTES;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
        cudaSuccess)
        return 0;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, EVAL_THREADS, dyn) != cudaSuccess) return 0;
    return b;
}
}  // namespace

const void* kernel_fit_loop_single_mixed(int model) { return model == 0 ? loop_mixed<MGauss1D>() : nullptr; }

int blocks_per_sm_single_mixed(int model) { return model == 0 ? blocks_mixed<MGauss1D>() : 0; }

}  // namespace gbfit

// Kernel sets of libgbfit and the registry of user-defined models (host side).
#pragma once
#include <cstddef>

namespace gbfit {

// The persistent loop kernels of one model set: the built-in registry (id 0)
// or one user-defined model compiled at run time (id = its model id).
struct KernelSet {
    int id;
    const void* fit_loop[2];    // [precision]
    int blocks_per_sm[2];
    size_t dyn_smem[2];
};

const KernelSet* builtin_kernels();
bool is_user_model(int id);
// n and coordinate dimensions of any model id; false when the id is unknown
bool model_shape(int id, int* n, int* dims);
// kernels for a model id, loading a user model's compiled code on first use
int kernels_for_model(int id, const KernelSet** out);

}  // namespace gbfit

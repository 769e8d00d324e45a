// sp_step_bf16.cu -- step kernels instantiated for bf16 storage.
#include "sp_step_launch.cuh"

namespace sp {

cudaError_t launch_step_bf16(int model, int stencil, const StepArgs &a, cudaStream_t s, int n_sm, int k) {
    return launch_step_dispatch<bf16>(model, stencil, a, s, n_sm, k);
}

}  // namespace sp

// sp_step_f32.cu -- step kernels instantiated for float storage.
#include "sp_step_launch.cuh"

namespace sp {

cudaError_t launch_step_f32(int model, int stencil, const StepArgs &a, cudaStream_t s, int n_sm, int k) {
    return launch_step_dispatch<float>(model, stencil, a, s, n_sm, k);
}

}  // namespace sp

// sp_step_f64.cu -- step kernels instantiated for double storage.
#include "sp_step_launch.cuh"

namespace sp {

cudaError_t launch_step_f64(int model, int stencil, const StepArgs &a, cudaStream_t s, int n_sm, int k) {
    return launch_step_dispatch<double>(model, stencil, a, s, n_sm, k);
}

}  // namespace sp

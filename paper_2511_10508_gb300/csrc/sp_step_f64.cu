// sp_step_f64.cu -- step kernels instantiated for double storage.
#include "sp_step_launch.cuh"

namespace sp {

cudaError_t launch_step_f64(int model, int stencil, const StepArgs &a, cudaStream_t s, int n_sm, int k) {
    return launch_step_dispatch<double>(model, stencil, a, s, n_sm, k);
}

cudaError_t launch_planes27_f64(int model, const StepArgs &a, void *mu, cudaStream_t s, int n_sm) {
    Planes27Args p;
    p.nx = a.nx;
    p.ny = a.ny;
    p.nz = a.nz;
    p.k = a.k;
    p.centre = nullptr;
    const double *in0 = static_cast<const double *>(a.in0), *in1 = static_cast<const double *>(a.in1);
    double *out0 = static_cast<double *>(a.out0), *out1 = static_cast<double *>(a.out1);
    switch (model) {
    case CH: {
        if (!mu) return cudaErrorInvalidValue;
        p.in[0] = p.in[1] = in0;
        p.out[0] = p.out[1] = static_cast<double *>(mu);
        const cudaError_t e = launch_planes27_mode<0>(p, s, n_sm);
        if (e != cudaSuccess) return e;
        p.in[0] = p.in[1] = static_cast<const double *>(mu);
        p.centre = in0;
        p.out[0] = p.out[1] = out0;
        return launch_planes27_mode<1>(p, s, n_sm);
    }
    case AC:
        p.in[0] = p.in[1] = in0;
        p.out[0] = p.out[1] = out0;
        return launch_planes27_mode<2>(p, s, n_sm);
    case GS:
        p.in[0] = in0;
        p.in[1] = in1;
        p.out[0] = out0;
        p.out[1] = out1;
        return launch_planes27_mode<3>(p, s, n_sm);
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ch_twopass_f64(int stencil, const StepArgs &a, void *mu, cudaStream_t s, int n_sm) {
    if (!mu) return cudaErrorInvalidValue;
    Planes27Args p;
    p.nx = a.nx;
    p.ny = a.ny;
    p.nz = a.nz;
    p.k = a.k;
    const double *phi = static_cast<const double *>(a.in0);
    p.in[0] = p.in[1] = phi;
    p.centre = nullptr;
    p.out[0] = p.out[1] = static_cast<double *>(mu);
    auto run = [&](auto mu_pass, auto update_pass) -> cudaError_t {
        cudaError_t e = mu_pass(p, s, n_sm);
        if (e != cudaSuccess) return e;
        p.in[0] = p.in[1] = static_cast<const double *>(mu);
        p.centre = phi;
        p.out[0] = p.out[1] = static_cast<double *>(a.out0);
        return update_pass(p, s, n_sm);
    };
    switch (stencil) {
    case L7: return run(launch_ring2pass_mode<L7, 0>, launch_ring2pass_mode<L7, 1>);
    case L13X4: return run(launch_ring2pass_mode<L13X4, 0>, launch_ring2pass_mode<L13X4, 1>);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace sp

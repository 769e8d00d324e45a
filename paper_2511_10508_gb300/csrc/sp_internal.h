// sp_internal.h -- declarations shared by the library's translation units
// (kernels, launchers and the C-ABI runtime).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sp.h"
#include "sp_common.cuh"

namespace sp {

constexpr int kMaxPatches = 2048;       // Gray-Scott seeded patches per grid
constexpr int kReduceThreads = 256;
constexpr int kReduceBlocksPerSM = 2;

struct ReduceGeom {
    int nx, ny, nz, dims;
    double h, cell_volume, c1, c2;
};

// Step launchers, one per storage type (sp_step_f64.cu, sp_step_f32.cu,
// sp_step_bf16.cu).  One forward-Euler step from a.in* to a.out*.
cudaError_t launch_step_f64(int model, int stencil, const StepArgs &a, cudaStream_t s, int n_sm);
cudaError_t launch_step_f32(int model, int stencil, const StepArgs &a, cudaStream_t s, int n_sm);
cudaError_t launch_step_bf16(int model, int stencil, const StepArgs &a, cudaStream_t s, int n_sm);

cudaError_t launch_ic(int dtype, void *u, void *v, int model, int dims, int nx, int ny, int nz,
                      uint64_t seed, int ic_kind, double mean, double amp, int patches, int patch,
                      cudaStream_t s, int n_sm);

int reduce_blocks(uint64_t N, int n_sm);
cudaError_t launch_reduce(int dtype, int what, const void *f, const ReduceGeom &g, double *partials,
                          int nblocks, double *out, cudaStream_t s);

// Element-wise conversion between FP64 staging and the storage type.
cudaError_t launch_convert_from_f64(int dtype, const double *src, void *dst, uint64_t n, cudaStream_t s);
cudaError_t launch_convert_to_f64(int dtype, const void *src, double *dst, uint64_t n, cudaStream_t s);

}  // namespace sp

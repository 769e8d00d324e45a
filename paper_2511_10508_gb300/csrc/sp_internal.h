// sp_internal.h -- declarations shared by the library's translation units
// (kernels, launchers and the C-ABI runtime).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sp.h"
#include "sp_common.cuh"

namespace sp {

constexpr int kMaxPatches = 2048;       // Gray-Scott seeded patches per grid
constexpr int kReduceThreads = 256;
constexpr int kReduceBlocksPerSM = 2;

struct ReduceGeom {
    int nx, ny, nz, dims;
    double h, cell_volume, c1, c2;
    double c3 = 0.0;            // Model C free energy: coupling
    const void *rho = nullptr;  // Model C free energy: the density field (else null)
    const void *jq[3] = {nullptr, nullptr, nullptr};  // Model H free energy: |j|^2/2 terms
    int nq = 0;
};

// Step launchers, one per storage type (sp_step_f64.cu, sp_step_f32.cu,
// sp_step_bf16.cu).  k forward-Euler steps from a.in* to a.out* in one launch;
// k must be 1, or the value of steps_per_launch() for this model/stencil/dtype.
cudaError_t launch_step_f64(int model, int stencil, const StepArgs &a, cudaStream_t s, int n_sm, int k);
cudaError_t launch_step_f32(int model, int stencil, const StepArgs &a, cudaStream_t s, int n_sm, int k);
cudaError_t launch_step_bf16(int model, int stencil, const StepArgs &a, cudaStream_t s, int n_sm, int k);

// Steps fused per launch (temporal blocking) for a request of `requested`
// (0 = the library's choice, 1 = none): 2D grids support 2 and 4 (FP64 on small
// tiles, where a launch is short enough for its fixed cost to matter); 3D grids
// see steps_per_launch_3d.  The library's choice follows measurement on GB300:
// blocking pays where the one-step tile kernel is at the HBM bound (FP32
// Gray-Scott 32768^2: 1 step 0.99 of the copy bandwidth, 2 steps 1.31
// effective, 4 steps 1.19); Cahn-Hilliard and BF16 storage are limited by
// on-chip work and FP64 by the FP64 pipe, so there extra halo work only slows
// large grids (the autotuner tries it on small FP64 grids).
// Kernel variant chosen per launch: 0 = the default for the grid, 1 (and 2) =
// alternative families (2D FP64: small tiles instead of strips, or strips instead
// of small tiles for grids up to 1024^2, and 2 / 4 = strips of 64 threads / of
// half the rows per batch; 2D FP32/BF16 single steps: shared-
// memory tiles instead of warp strips; 3D FP32/BF16: 1 = cp.async plane ring,
// 2 = register-staged plane rings, instead of warp rows; 3D FP64 27-point:
// shared-memory plane rings instead of z-streaming).  Set around each launch by
// the runtime.
extern thread_local int g_step_variant;

// Number of equal z segments for a lockstep schedule of `tiles` x segments work
// items over `wave` resident CTAs: minimises rounds x (planes per segment +
// halo planes), the time of the slowest CTA.
inline int lockstep_segments(long long tiles, int nz, int halo, long long wave) {
    int best = 1;
    double best_cost = 0;
    for (int sgs = 1; sgs <= std::min(nz, 64); ++sgs) {
        const long long rounds = (tiles * sgs + wave - 1) / wave;
        const double cost = (double)rounds * ((double)nz / sgs + halo);
        if (sgs == 1 || cost < best_cost * 0.999) {
            best = sgs;
            best_cost = cost;
        }
    }
    return best;
}

// FP64 2D grids up to 1024^2 use small tiles by default (and may fuse steps).
constexpr long long kSmallGrid2d = 1LL << 20;

// 3D: two steps per launch for FP32 / BF16 Allen-Cahn, Gray-Scott and Model C
// (plane rings, grids with nx a multiple of 4), when asked for or autotuned.
inline int steps_per_launch_3d(int dtype, int model, int nx, int requested) {
    const bool ok = dtype != SP_F64 && (model == SP_ALLEN_CAHN || model == SP_GRAY_SCOTT || model == SP_MODEL_C) &&
                    nx % 4 == 0;
    return (ok && requested >= 2) ? 2 : 1;
}

inline int steps_per_launch(int dims, int dtype, int model, int requested) {
    if (dims != 2 || model == SP_MODEL_H) return 1;
    if (requested == 0) return (dtype == SP_F32 && model != CH) ? 2 : 1;
    if (requested >= 4) return 4;
    if (requested >= 2) return 2;
    return 1;
}

// 3D FP64 27-point Allen-Cahn, Cahn-Hilliard (two passes through `mu`, N
// doubles) and Gray-Scott with x-pair sums shared between y neighbours: kernel
// family 0 of these grids.  Family 2 is then the z-streaming kernel with plane
// sums in registers (step3d_zreg_kernel, family 0 of launch_step_f64), family 1
// the accessor-based plane ring.
constexpr int kZregFamily = 2;
cudaError_t launch_planes27_f64(int model, const StepArgs &a, void *mu, cudaStream_t s, int n_sm);
// 3D FP64 Cahn-Hilliard with the 7- and 13-point stencils in two passes through
// `mu` (N doubles): kernel family 0 of these grids; family kFusedFamily is the
// one-pass plane ring with mu on a halo ring (launch_step_f64's family 0).
constexpr int kFusedFamily = 2;
cudaError_t launch_ch_twopass_f64(int stencil, const StepArgs &a, void *mu, cudaStream_t s, int n_sm);
inline bool twopass_applies(int dims, int dtype, int stencil, int model) {
    return dims == 3 && dtype == SP_F64 && (stencil == SP_LAP_7 || stencil == SP_LAP_13CROSS4) && model == SP_CAHN_HILLIARD;
}
inline bool planes27_applies(int dims, int dtype, int stencil, int model) {
    return dims == 3 && dtype == SP_F64 && stencil == SP_LAP_27 &&
           (model == SP_ALLEN_CAHN || model == SP_CAHN_HILLIARD || model == SP_GRAY_SCOTT);
}

// Tensor-map (TMA) plane loads (sp_tma.cu): kernel family kTmaFamily of 3D
// FP32/BF16 Allen-Cahn, Cahn-Hilliard and Gray-Scott grids with nx a multiple of
// 16 bytes' worth of cells.  encode_plane_maps describes fields f0 and f1 (f1 may
// equal f0) as nx x ny x nz tensors with box_x x box_y x 1 boxes.
constexpr int kTmaFamily = 6;
bool tma_available();
cudaError_t encode_plane_maps(TmaMaps *maps, bool bf16, const void *f0, const void *f1, int nx, int ny, int nz,
                              int box_x, int box_y);

// Generated cross stencils (sp_generated.cu), radius up to kMaxGenRadius.
constexpr int kMaxGenRadius = 4;
int generated_weights(int order, int dims, double *wk, double *lambda_max);
cudaError_t launch_generated(int model, int dtype, int order, int dims, const double *wk, const StepArgs &a, void *mu,
                             cudaStream_t s, int n_sm);

// Model H (sp_model_h.cu): one step from in[0..nf) to out[0..nf) (m, then the
// components of j; unused entries null) through the mu buffer of N compute-
// precision values; c3g = c3 times the central-difference scale.
cudaError_t launch_model_h(int dtype, int stencil, void *const in[4], void *const out[4], void *mu, int nx, int ny,
                           int nz, const StepConsts &k, double c3g, cudaStream_t s, int n_sm);
cudaError_t launch_ic_currents(int dtype, void *const j[3], int dims, uint64_t N, uint64_t seed, int ic_kind, double amp,
                               cudaStream_t s, int n_sm);

// Unfused Cahn-Hilliard step (ablation only, kernel family kUnfusedFamily): mu
// into the caller's temporary of N compute-precision values, then the update.
constexpr int kUnfusedFamily = 3;
cudaError_t launch_unfused_ch(int dtype, int stencil, const StepArgs &a, void *mu, cudaStream_t s, int n_sm);

// Semi-implicit Fourier spectral scheme (sp_spectral.cu, with its own FFTs): a
// plan holds the twiddle tables, the resident spectrum and the transform
// buffer.  Functions return SP_* status codes.  spectral_step with `more` set
// also transforms the cubic term of the new field for the step that follows.
struct SpectralPlan;
int spectral_create(int dtype, int dims, int nx, int ny, int nz, SpectralPlan **out);
void spectral_destroy(SpectralPlan *P);
size_t spectral_bytes(const SpectralPlan *P);
int spectral_load(SpectralPlan *P, const void *phi, cudaStream_t s);
int spectral_step(SpectralPlan *P, int model, void *phi, void *nbuf, double h, double dt, double c1, double c2,
                  double kappa, cudaStream_t s, int n_sm, bool more);
const char *spectral_last_error();

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

// sp_step_launch.cuh -- host-side launch of the step kernels: tile choices per
// storage type and stencil radius, and the grid size.
//
// Grid sizing: a CTA owns a column strip (2D: TW columns; 3D: a TX x TY tile)
// and a run of rows/planes along the slowest axis.  The run length is chosen
// so that the whole grid is one wave of resident CTAs (SMs x occupancy), but
// never shorter than kMinRun slices, which bounds the redundant halo slices
// (2*RIN per run) at a few percent.
#pragma once

#include <algorithm>

#include "sp_internal.h"
#include "sp_step.cuh"

namespace sp {

template <typename T> struct Tiles;
template <> struct Tiles<double> {
    static constexpr int NT2 = 128, V2 = 2;                  // 2D: 256 columns per strip
    template <int r> struct T3 { static constexpr int TX = (r == 1) ? 64 : 32, TY = 32, NT = 256; };
};
template <> struct Tiles<float> {
    static constexpr int NT2 = 128, V2 = 4;                  // 2D: 512 columns per strip
    template <int r> struct T3 { static constexpr int TX = 64, TY = 16, NT = 256; };
};
template <> struct Tiles<bf16> {
    static constexpr int NT2 = 128, V2 = 8;                  // 2D: 1024 columns per strip
    template <int r> struct T3 { static constexpr int TX = 64, TY = 16, NT = 256; };
};

constexpr int kMinRun = 32;

inline int run_length(int n_slow, long long strips, int ctas_per_sm, int n_sm) {
    const long long wave = (long long)n_sm * std::max(ctas_per_sm, 1);
    long long chunks = (wave + strips - 1) / strips;
    chunks = std::max<long long>(1, std::min<long long>(chunks, (n_slow + kMinRun - 1) / kMinRun));
    return (int)((n_slow + chunks - 1) / chunks);
}

template <int MODEL, int ST, typename T>
cudaError_t launch_step_t(const StepArgs &a, cudaStream_t s, int n_sm) {
    if constexpr (StencilInfo<ST>::dims == 2) {
        constexpr int NT = Tiles<T>::NT2, V = Tiles<T>::V2, TW = NT * V;
        auto kern = step2d_kernel<MODEL, ST, T, NT, V>;
        static const int occ = [&] {
            int o = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, NT, 0);
            return o;
        }();
        const int strips = (a.nx + TW - 1) / TW;
        const int TH = run_length(a.ny, strips, occ, n_sm);
        dim3 grid(strips, (a.ny + TH - 1) / TH);
        kern<<<grid, NT, 0, s>>>(a, TH);
    } else {
        typedef typename Tiles<T>::template T3<StencilInfo<ST>::r> TT;
        typedef Step3dShape<MODEL, ST, T, TT::TX, TT::TY, TT::NT> Sh;
        auto kern = step3d_kernel<MODEL, ST, T, TT::TX, TT::TY, TT::NT>;
        static const int occ = [&] {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
            int o = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, TT::NT, Sh::smem_bytes);
            return o;
        }();
        const long long strips = (long long)((a.nx + TT::TX - 1) / TT::TX) * ((a.ny + TT::TY - 1) / TT::TY);
        const int TZ = run_length(a.nz, strips, occ, n_sm);
        dim3 grid((a.nx + TT::TX - 1) / TT::TX, (a.ny + TT::TY - 1) / TT::TY, (a.nz + TZ - 1) / TZ);
        kern<<<grid, TT::NT, Sh::smem_bytes, s>>>(a, TZ);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step_dispatch(int model, int stencil, const StepArgs &a, cudaStream_t s, int n_sm) {
#define SP_STENCILS(M)                                                   \
    switch (stencil) {                                                   \
    case L5: return launch_step_t<M, L5, T>(a, s, n_sm);                 \
    case L9BOX: return launch_step_t<M, L9BOX, T>(a, s, n_sm);           \
    case L9X4: return launch_step_t<M, L9X4, T>(a, s, n_sm);             \
    case L7: return launch_step_t<M, L7, T>(a, s, n_sm);                 \
    case L27: return launch_step_t<M, L27, T>(a, s, n_sm);               \
    case L13X4: return launch_step_t<M, L13X4, T>(a, s, n_sm);           \
    }                                                                    \
    break;
    switch (model) {
    case AC: SP_STENCILS(AC)
    case CH: SP_STENCILS(CH)
    case GS: SP_STENCILS(GS)
    }
#undef SP_STENCILS
    return cudaErrorInvalidValue;
}

}  // namespace sp

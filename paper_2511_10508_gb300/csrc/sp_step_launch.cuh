// sp_step_launch.cuh -- host-side launch of the step kernels: tile choices per
// storage type and stencil radius, and the grid size.
//
// Grid sizing: every kernel is persistent.  The work is the flattened space of
// (column strip or xy tile, row or plane) pairs; the grid is one resident wave
// and each CTA (2D FP32/BF16: each warp) takes an equal contiguous share, so no
// SM waits for a tail of long-running CTAs.
#pragma once

#include <algorithm>
#include <type_traits>

#include "sp_internal.h"
#include "sp_step.cuh"

namespace sp {

// 3D tiles (x, y) per storage type and stencil radius.
template <typename T> struct Tiles;
template <> struct Tiles<double> {
    template <int r> struct T3 { static constexpr int TX = (r == 1) ? 64 : 32, TY = 32, NT = 256; };
};
template <> struct Tiles<float> {
    template <int r> struct T3 { static constexpr int TX = 64, TY = 16, NT = 256; };
};
template <> struct Tiles<bf16> {
    template <int r> struct T3 { static constexpr int TX = 64, TY = 16, NT = 256; };
};

constexpr int kMinRun = 32;
constexpr size_t kMaxSmemPerCta = 227 * 1024;  // opt-in maximum of dynamic shared memory per CTA

// Persistent grids: one resident wave of CTAs (SMs x occupancy), each owning an
// equal share of the flattened (tile, slow-axis) work, but at least kMinRun
// slices per CTA so that the halo slices of each segment stay a small fraction.
inline long long persistent_ctas(long long total_slices, int ctas_per_sm, int n_sm) {
    const long long wave = (long long)n_sm * std::max(ctas_per_sm, 1);
    return std::max(1LL, std::min(wave, total_slices / kMinRun));
}

// Launch with programmatic stream serialisation (the kernel calls pdl_enter()
// before touching global memory): used where a launch is a few microseconds
// long, so that the next step's CTAs are resident when this one completes.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Batched persistent 2D kernel (FP64): rows per batch and CTAs per SM.
template <int MODEL> struct Batch2d { static constexpr int NT = 128, RB = (MODEL == CH) ? 8 : (MODEL == AC ? 4 : 2), CPS = 4; };

// The FP64 2D strip kernel with NT threads, RB rows per batch, at most CPS CTAs
// per SM; persistent grid with equal rows per CTA.
template <int MODEL, int ST, typename T, int NT, int RB, int CPS>
cudaError_t launch_strips(const StepArgs &a, cudaStream_t s, int n_sm) {
    typedef Step2dBatchShape<MODEL, ST, T, NT, RB> Sh;
    auto kern = step2d_batch_kernel<MODEL, ST, T, NT, RB>;
    static const int occ = [&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
        int o = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, NT, Sh::smem_bytes);
        return o;
    }();
    const int strips = (a.nx + Sh::TW - 1) / Sh::TW;
    const long long total = (long long)strips * a.ny;
    // equal rows per CTA; at least 4*RB rows each so that the ring warm-up stays small
    long long ctas = (long long)n_sm * std::max(1, std::min(occ, CPS));
    ctas = std::max(1LL, std::min(ctas, total / (4 * RB)));
    const long long rows = (total + ctas - 1) / ctas;
    ctas = (total + rows - 1) / rows;
    kern<<<(unsigned)ctas, NT, Sh::smem_bytes, s>>>(a, strips, rows);
    return cudaGetLastError();
}

// Temporally blocked 2D tile kernel: K steps per launch.  FP32 / BF16 tiles of
// 128 x 16; FP64 (small grids, where the fixed cost of a launch matters) tiles
// of 32 x 14, so that a 256^2 grid spreads over 8 x 19 = 152 CTAs, one per SM.
template <int MODEL, int ST, typename T, int K>
cudaError_t launch_tb(const StepArgs &a, cudaStream_t s) {
    constexpr bool f64 = std::is_same<T, double>::value;
    constexpr int BX = f64 ? 32 : 128, BY = f64 ? 14 : 16, NT = f64 ? 128 : 256;
    typedef Step2dTbShape<MODEL, ST, T, BX, BY, K> Sh;
    auto kern = step2d_tb_kernel<MODEL, ST, T, BX, BY, K, NT>;
    static const bool attr = [&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
        return true;
    }();
    (void)attr;
    dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY);
    if constexpr (f64) return launch_pdl(kern, grid, dim3(NT), Sh::smem_bytes, s, a);  // small grids
    kern<<<grid, NT, Sh::smem_bytes, s>>>(a);
    return cudaGetLastError();
}

// 3D FP32 / BF16 Allen-Cahn and Gray-Scott with a plane ring per time level: K
// steps per pass (temporal blocking for K = 2) on warp-row tiles of 120 x TY
// outputs; lockstep z segments.  Needs nx a multiple of 4 and 16-byte aligned
// fields (the runtime offers these families only then).
template <int MODEL, int ST, typename T, int TY, int K>
cudaError_t launch_tbs(const StepArgs &a, cudaStream_t s, int n_sm) {
    typedef Step3dTbsShape<MODEL, ST, T, TY, K> Sh;
    auto kern = step3d_tbs_kernel<MODEL, ST, T, TY, K>;
    static const int occ = [&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
        int o = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, Sh::NT, Sh::smem_bytes);
        return o;
    }();
    const int tx = (a.nx + Sh::TX - 1) / Sh::TX, ty = (a.ny + TY - 1) / TY;
    const long long wave = (long long)n_sm * std::max(occ, 1);
    const int segs = lockstep_segments((long long)tx * ty, a.nz, 2 * K * Sh::r, wave);
    const long long items = (long long)tx * ty * segs;
    kern<<<(unsigned)std::min(items, wave), Sh::NT, Sh::smem_bytes, s>>>(a, tx, ty, segs);
    return cudaGetLastError();
}

// FP64 27-point: z-streaming kernel with per-plane partial sums in registers.
template <int MODEL, typename T>
cudaError_t launch_zreg(const StepArgs &a, cudaStream_t s, int n_sm) {
    constexpr int TX = 32, TY = 32, NT = 256;
    typedef Step3dZregShape<MODEL, TX, TY, NT> Sh;
    auto kern = step3d_zreg_kernel<MODEL, TX, TY, NT>;
    static const int occ = [&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
        int o = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, NT, Sh::smem_bytes);
        return o;
    }();
    const int tx = (a.nx + TX - 1) / TX, ty = (a.ny + TY - 1) / TY;
    const long long ctas = persistent_ctas((long long)tx * ty * a.nz, occ, n_sm);
    const long long planes = ((long long)tx * ty * a.nz + ctas - 1) / ctas;
    kern<<<(unsigned)(((long long)tx * ty * a.nz + planes - 1) / planes), NT, Sh::smem_bytes, s>>>(a, tx, ty, planes);
    return cudaGetLastError();
}

// FP64 27-point with shared pair sums: one pass per mode (Cahn-Hilliard: mode 0
// then mode 1 through the mu buffer).
template <int MODE>
cudaError_t launch_planes27_mode(const Planes27Args &a, cudaStream_t s, int n_sm) {
    typedef Planes27Shape<MODE> Sh;
    auto kern = planes27_kernel<MODE>;
    static const int occ = [&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
        int o = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, Sh::NT, Sh::smem_bytes);
        return o;
    }();
    const int tx = (a.nx + Sh::TX - 1) / Sh::TX, ty = (a.ny + Sh::TY - 1) / Sh::TY;
    const long long total = (long long)tx * ty * a.nz;
    const long long ctas = persistent_ctas(total, occ, n_sm);
    const long long planes = (total + ctas - 1) / ctas;
    kern<<<(unsigned)((total + planes - 1) / planes), Sh::NT, Sh::smem_bytes, s>>>(a, tx, planes, total);
    return cudaGetLastError();
}

template <int ST, int MODE>
cudaError_t launch_ring2pass_mode(const Planes27Args &a, cudaStream_t s, int n_sm) {
    typedef Ring2PassShape<ST> Sh;
    auto kern = ring2pass_kernel<ST, MODE>;
    static const int occ = [&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
        int o = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, Sh::NT, Sh::smem_bytes);
        return o;
    }();
    const int tx = (a.nx + Sh::TX - 1) / Sh::TX, ty = (a.ny + Sh::TY - 1) / Sh::TY;
    const long long total = (long long)tx * ty * a.nz;
    const long long ctas = persistent_ctas(total, occ, n_sm);
    const long long planes = (total + ctas - 1) / ctas;
    kern<<<(unsigned)((total + planes - 1) / planes), Sh::NT, Sh::smem_bytes, s>>>(a, tx, planes, total);
    return cudaGetLastError();
}

template <int MODEL, int ST, typename T>
cudaError_t launch_step_t(const StepArgs &a, cudaStream_t s, int n_sm, int k) {
    if constexpr (StencilInfo<ST>::dims == 2) {
        if (k == 4) return launch_tb<MODEL, ST, T, 4>(a, s);
        if (k == 2) return launch_tb<MODEL, ST, T, 2>(a, s);
    }
    if constexpr (StencilInfo<ST>::dims == 2 && std::is_same<T, double>::value) {
        const bool small = (long long)a.nx * a.ny <= kSmallGrid2d;
        const bool strip_shape = g_step_variant == 2 || g_step_variant == 4;
        if (!strip_shape && small != (g_step_variant == 1)) {
            // small grids are latency bound: many small tiles instead of a few long strips
            constexpr int BX = 32, BY = 16, NT = 128;
            typedef Step2dTileShape<MODEL, ST, T, BX, BY> Sh;
            auto kern = step2d_tile_kernel<MODEL, ST, T, BX, BY, NT>;
            static const bool attr = [&] {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
                return true;
            }();
            (void)attr;
            return launch_pdl(kern, dim3((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY), dim3(NT), Sh::smem_bytes, s, a);
        }
        // strip families: 0 the default shape, 2 narrower CTAs (64 threads), 4 half
        // the rows per batch; the autotuner picks per grid
        typedef Batch2d<MODEL> B;
        if (g_step_variant == 2) return launch_strips<MODEL, ST, T, 64, B::RB, 2 * B::CPS>(a, s, n_sm);
        if (g_step_variant == 4)
            return launch_strips<MODEL, ST, T, B::NT, (B::RB > 1 ? B::RB / 2 : 1), 2 * B::CPS>(a, s, n_sm);
        return launch_strips<MODEL, ST, T, B::NT, B::RB, B::CPS>(a, s, n_sm);
    } else if constexpr (StencilInfo<ST>::dims == 2) {
        typedef Step2dWarpShape<MODEL, ST, T> WS;
        const bool aligned = ((uintptr_t)a.in0 | (uintptr_t)a.in1 | (uintptr_t)a.out0 | (uintptr_t)a.out1) % 16 == 0;
        if (g_step_variant == 0 && a.nx % WS::V == 0 && aligned) {
            // FP32 / BF16: one warp per column strip, up to 8 adjacent strips per
            // CTA, persistent equal shares of (strip group, row)
            constexpr int NT = 256;
            auto kern = step2d_warp_kernel<MODEL, ST, T, NT>;
            static const bool attr = [&] {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(WS::warp_smem * (NT / 32)));
                return true;
            }();
            (void)attr;
            const int strips = (a.nx + WS::OUT_COLS - 1) / WS::OUT_COLS;
            const int wpc = std::min(NT / 32, strips);
            const size_t smem = WS::warp_smem * wpc;
            int occ = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * wpc, smem);
            const int groups = (strips + wpc - 1) / wpc;
            const long long total = (long long)groups * a.ny;
            long long ctas = (long long)n_sm * std::max(occ, 1);
            ctas = std::max(1LL, std::min(ctas, total / kMinRun));
            const long long rows = (total + ctas - 1) / ctas;
            ctas = (total + rows - 1) / rows;
            kern<<<(unsigned)ctas, 32 * wpc, smem, s>>>(a, strips, groups, rows);
            return cudaGetLastError();
        }
        // FP32 / BF16: one CTA per 128 x 32 tile
        constexpr int BX = 128, BY = 32, NT = 256;
        typedef Step2dTileShape<MODEL, ST, T, BX, BY> Sh;
        auto kern = step2d_tile_kernel<MODEL, ST, T, BX, BY, NT>;
        static const bool attr = [&] {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
            return true;
        }();
        (void)attr;
        dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY);
        kern<<<grid, NT, Sh::smem_bytes, s>>>(a);
    } else if constexpr (!std::is_same<T, double>::value && MODEL == MC) {
        // Model C, FP32 / BF16 3D: plane rings (two steps per launch: families 0 and 1,
        // tiles of 8 and 16 rows; one step: families 4 and 5) where nx and the
        // alignment allow, else one CTA per box (the accessor-based box code)
        const bool al = ((uintptr_t)a.in0 | (uintptr_t)a.in1 | (uintptr_t)a.out0 | (uintptr_t)a.out1) % 16 == 0;
        if (a.nx % 4 == 0 && al) {
            constexpr bool tall2 = Step3dTbsShape<MODEL, ST, T, 16, 2>::smem_bytes <= kMaxSmemPerCta;
            if (k == 2 && g_step_variant == 1 && tall2) return launch_tbs<MODEL, ST, T, (tall2 ? 16 : 8), 2>(a, s, n_sm);
            if (k == 2) return launch_tbs<MODEL, ST, T, 8, 2>(a, s, n_sm);
            if (g_step_variant == 5) return launch_tbs<MODEL, ST, T, 16, 1>(a, s, n_sm);
            if (g_step_variant == 4) return launch_tbs<MODEL, ST, T, 8, 1>(a, s, n_sm);
        }
        constexpr int BX = 32, BY = 8, BZ = 8, NT = 256;
        typedef Step3dBoxShape<MODEL, ST, T, BX, BY, BZ> Sh;
        auto kern = step3d_box_kernel<MODEL, ST, T, BX, BY, BZ, NT>;
        static const bool attr = [&] {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
            return true;
        }();
        (void)attr;
        const int bx = (a.nx + BX - 1) / BX, by = (a.ny + BY - 1) / BY, bz = (a.nz + BZ - 1) / BZ;
        kern<<<dim3((unsigned)bx, (unsigned)by, (unsigned)bz), NT, Sh::smem_bytes, s>>>(a);
    } else if constexpr (!std::is_same<T, double>::value) {
        if constexpr (MODEL == AC || MODEL == GS) {
            // two steps per launch with a plane ring per time level (families 0 and 1:
            // tiles of 8 and 16 rows; the taller ones only where their rings fit)
            constexpr bool tall2 = Step3dTbsShape<MODEL, ST, T, 16, 2>::smem_bytes <= kMaxSmemPerCta;
            if (k == 2 && g_step_variant == 1 && tall2) return launch_tbs<MODEL, ST, T, (tall2 ? 16 : 8), 2>(a, s, n_sm);
            if (k == 2) return launch_tbs<MODEL, ST, T, 8, 2>(a, s, n_sm);
        }
        constexpr int ATX = 16, ATY = 16;
        typedef Step3dAsyncShape<MODEL, ST, T, ATX, ATY> AS;
        const bool aligned = ((uintptr_t)a.in0 | (uintptr_t)a.in1 | (uintptr_t)a.out0 | (uintptr_t)a.out1) % 16 == 0;
        constexpr int WTY = 8;
        typedef Step3dWrShape<MODEL, ST, T, WTY> WS;
        auto wkern = step3d_wr_kernel<MODEL, ST, T, WTY>;
        // the warp-row kernel is the default unless its register queues spill
        // (a spill of a few words outside the queues costs nothing measurable)
        static const bool wr_spills = [&] {
            cudaFuncAttributes fa{};
            return cudaFuncGetAttributes(&fa, wkern) != cudaSuccess || fa.localSizeBytes > 16;
        }();
        const int fam = (g_step_variant == 0 && wr_spills) ? 1 : g_step_variant;
        if (fam == 0 && a.nx % WS::V == 0 && aligned) {
            // FP32 / BF16 3D: warp per tile row, z neighbours in registers
            auto kern = wkern;
            static const int occ = [&] {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WS::smem_bytes);
                int o = 1;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, WS::NT, WS::smem_bytes);
                return o;
            }();
            const int tx = (a.nx + WS::TX - 1) / WS::TX, ty = (a.ny + WTY - 1) / WTY;
            const long long wave = (long long)n_sm * std::max(occ, 1);
            const int segs = lockstep_segments((long long)tx * ty, a.nz, 2 * WS::R, wave);
            const long long items = (long long)tx * ty * segs;
            kern<<<(unsigned)std::min(items, wave), WS::NT, WS::smem_bytes, s>>>(a, tx, ty, segs);
            return cudaGetLastError();
        }
        if (fam == kTmaFamily && a.nx % AS::V == 0 && aligned) {
            // FP32 / BF16 3D: the plane ring with tensor-map plane loads
            TmaMaps maps;
            const cudaError_t e = encode_plane_maps(&maps, sizeof(T) == 2, a.in0, a.in1, a.nx, a.ny, a.nz, AS::SW,
                                                    AS::HIN);
            if (e != cudaSuccess) return e;
            auto kern = step3d_async_kernel<MODEL, ST, T, ATX, ATY, true>;
            static const int occ = [&] {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AS::smem_bytes);
                int o = 1;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, AS::NT, AS::smem_bytes);
                return o;
            }();
            const int tx = (a.nx + AS::TX - 1) / AS::TX, ty = (a.ny + ATY - 1) / ATY;
            const long long wave = (long long)n_sm * std::max(occ, 1);
            const int segs = lockstep_segments((long long)tx * ty, a.nz, 2 * AS::R, wave);
            const long long items = (long long)tx * ty * segs;
            kern<<<(unsigned)std::min(items, wave), AS::NT, AS::smem_bytes, s>>>(a, tx, ty, segs, maps);
            return cudaGetLastError();
        }
        if (fam != 2 && a.nx % AS::V == 0 && aligned) {
            // FP32 / BF16 3D: cp.async plane ring with planes in flight
            auto kern = step3d_async_kernel<MODEL, ST, T, ATX, ATY, false>;
            static const int occ = [&] {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AS::smem_bytes);
                int o = 1;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, AS::NT, AS::smem_bytes);
                return o;
            }();
            const int tx = (a.nx + AS::TX - 1) / AS::TX, ty = (a.ny + ATY - 1) / ATY;
            const long long wave = (long long)n_sm * std::max(occ, 1);
            const int segs = lockstep_segments((long long)tx * ty, a.nz, 2 * AS::R, wave);
            const long long items = (long long)tx * ty * segs;
            kern<<<(unsigned)std::min(items, wave), AS::NT, AS::smem_bytes, s>>>(a, tx, ty, segs, TmaMaps{});
            return cudaGetLastError();
        }
        // FP32 / BF16 3D, any nx: vectorised plane kernel, 64 x 32 tiles
        constexpr int TXT = 16, TYT = 32;
        typedef Step3dVecShape<MODEL, ST, T, TXT, TYT> Sh;
        auto kern = step3d_vec_kernel<MODEL, ST, T, TXT, TYT>;
        static const int occ = [&] {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
            int o = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, Sh::NT, Sh::smem_bytes);
            return o;
        }();
        const int tx = (a.nx + Sh::TX - 1) / Sh::TX, ty = (a.ny + Sh::TY - 1) / Sh::TY;
        const long long ctas = persistent_ctas((long long)tx * ty * a.nz, occ, n_sm);
        const long long planes = ((long long)tx * ty * a.nz + ctas - 1) / ctas;
        kern<<<(unsigned)(((long long)tx * ty * a.nz + planes - 1) / planes), Sh::NT, Sh::smem_bytes, s>>>(
            a, tx, ty, planes);
    } else {
        if constexpr (MODEL != MC) {
            if (ST == L27 && g_step_variant == 0) return launch_zreg<MODEL, T>(a, s, n_sm);
        }
        typedef typename Tiles<T>::template T3<StencilInfo<ST>::r> TT;
        typedef Step3dShape<MODEL, ST, T, TT::TX, TT::TY, TT::NT> Sh;
        auto kern = step3d_kernel<MODEL, ST, T, TT::TX, TT::TY, TT::NT>;
        static const int occ = [&] {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
            int o = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, TT::NT, Sh::smem_bytes);
            return o;
        }();
        const int tx = (a.nx + TT::TX - 1) / TT::TX, ty = (a.ny + TT::TY - 1) / TT::TY;
        const long long ctas = persistent_ctas((long long)tx * ty * a.nz, occ, n_sm);
        const long long planes = ((long long)tx * ty * a.nz + ctas - 1) / ctas;
        kern<<<(unsigned)(((long long)tx * ty * a.nz + planes - 1) / planes), TT::NT, Sh::smem_bytes, s>>>(
            a, tx, ty, planes);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step_dispatch(int model, int stencil, const StepArgs &a, cudaStream_t s, int n_sm, int k) {
#define SP_STENCILS(M)                                                   \
    switch (stencil) {                                                   \
    case L5: return launch_step_t<M, L5, T>(a, s, n_sm, k);              \
    case L9BOX: return launch_step_t<M, L9BOX, T>(a, s, n_sm, k);        \
    case L9X4: return launch_step_t<M, L9X4, T>(a, s, n_sm, k);          \
    case L7: return launch_step_t<M, L7, T>(a, s, n_sm, k);              \
    case L27: return launch_step_t<M, L27, T>(a, s, n_sm, k);            \
    case L13X4: return launch_step_t<M, L13X4, T>(a, s, n_sm, k);        \
    }                                                                    \
    break;
    switch (model) {
    case AC: SP_STENCILS(AC)
    case CH: SP_STENCILS(CH)
    case GS: SP_STENCILS(GS)
    case MC: SP_STENCILS(MC)
    }
#undef SP_STENCILS
    return cudaErrorInvalidValue;
}

}  // namespace sp

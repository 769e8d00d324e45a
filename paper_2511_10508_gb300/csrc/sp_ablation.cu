// sp_ablation.cu -- the unfused Cahn-Hilliard step, kept only as an ablation of
// the fused kernels (never chosen by the autotuner).
//
// The paper's solver evaluates the chemical potential into a temporary field in
// global memory and applies the outer Laplacian in a second pass (Sec.
// "Benchmarks", Table 2 with one temporary).  Here: pass 1 reads phi and writes
// mu for every point (compute precision), pass 2 reads mu and phi and writes
// phi'; 5 field accesses per update instead of the fused kernels' 2.  Both
// passes evaluate the same expressions in the same order as the fused kernels,
// so the results are identical bit for bit.  One thread per point, a block per
// 256-point row segment; neighbours come through L1/L2.
#include "sp_internal.h"

namespace sp {

// Stencil sum at (x, y, z): the wrapped offsets of the 2r+1 planes and rows
// around the segment are computed once per segment.
template <int ST>
struct Taps {
    static constexpr int r = StencilInfo<ST>::r;
    size_t zb[2 * r + 1], yb[2 * r + 1];
    __device__ __forceinline__ Taps(int y, int z, int nx, int ny, int nz) {
#pragma unroll
        for (int d = -r; d <= r; ++d) {
            zb[d + r] = (size_t)wrap_idx(z + d, nz) * ny * nx;
            yb[d + r] = (size_t)wrap_idx(y + d, ny) * nx;
        }
    }
};

template <int ST, typename T, typename U>
__device__ __forceinline__ typename Cmp<U>::type ablation_sum(const U *f, const Taps<ST> &tp, int x, int nx) {
    typedef typename Cmp<U>::type C;
    auto P = [&](int dx, int dy, int dz) -> C {
        constexpr int r = StencilInfo<ST>::r;
        return to_c(f[tp.zb[dz + r] + tp.yb[dy + r] + wrap_idx(x + dx, nx)]);
    };
    return stencil_sum<ST, C>(P);
}

// Work unit: a 256-point segment of one row (x fastest); units are handed out
// grid-stride, so index arithmetic is per segment, not per point.
struct RowSeg {
    int x, y, z;
    size_t row;  // offset of the row start
};
__device__ __forceinline__ RowSeg row_seg(long long u, int segs, const StepArgs &a) {
    const long long r = u / segs;
    RowSeg q;
    q.x = (int)(u - r * segs) * 256 + (int)threadIdx.x;
    q.y = (int)(r % a.ny);
    q.z = (int)(r / a.ny);
    q.row = (size_t)r * a.nx;
    return q;
}

// pass 1: mu = c2 phi^3 - c1 phi - kappa L phi (Eq. model-b's chemical potential)
template <int ST, typename T>
__global__ void __launch_bounds__(256) unfused_mu_kernel(const T *phi, typename Cmp<T>::type *mu, StepArgs a,
                                                         int segs) {
    typedef typename Cmp<T>::type C;
    const ConstsC<C> k(a.k, a.kf);
    const long long units = (long long)a.ny * a.nz * segs;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const RowSeg q = row_seg(u, segs, a);
        const Taps<ST> tp(q.y, q.z, a.nx, a.ny, a.nz);
        if (q.x < a.nx) mu[q.row + q.x] = ch_mu<C>(to_c(phi[q.row + q.x]), ablation_sum<ST, T>(phi, tp, q.x, a.nx), k);
    }
}

// pass 2: phi' = phi + dt L mu
template <int ST, typename T>
__global__ void __launch_bounds__(256) unfused_update_kernel(const T *phi, const typename Cmp<T>::type *mu, T *out,
                                                             StepArgs a, int segs) {
    typedef typename Cmp<T>::type C;
    const ConstsC<C> k(a.k, a.kf);
    const long long units = (long long)a.ny * a.nz * segs;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const RowSeg q = row_seg(u, segs, a);
        const Taps<ST> tp(q.y, q.z, a.nx, a.ny, a.nz);
        if (q.x < a.nx)
            out[q.row + q.x] = from_c<T>(ch_update<C>(to_c(phi[q.row + q.x]), ablation_sum<ST, C>(mu, tp, q.x, a.nx), k));
    }
}

template <int ST, typename T>
static cudaError_t launch_unfused_t(const StepArgs &a, void *mu, cudaStream_t s, int n_sm) {
    typedef typename Cmp<T>::type C;
    const int segs = (a.nx + 255) / 256;
    const long long units = (long long)a.ny * a.nz * segs;
    const unsigned blocks = (unsigned)std::min<long long>(units, (long long)n_sm * 8);
    unfused_mu_kernel<ST, T><<<blocks, 256, 0, s>>>(static_cast<const T *>(a.in0), static_cast<C *>(mu), a, segs);
    unfused_update_kernel<ST, T><<<blocks, 256, 0, s>>>(static_cast<const T *>(a.in0), static_cast<const C *>(mu),
                                                         static_cast<T *>(a.out0), a, segs);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_unfused_st(int stencil, const StepArgs &a, void *mu, cudaStream_t s, int n_sm) {
    switch (stencil) {
    case L5: return launch_unfused_t<L5, T>(a, mu, s, n_sm);
    case L9BOX: return launch_unfused_t<L9BOX, T>(a, mu, s, n_sm);
    case L9X4: return launch_unfused_t<L9X4, T>(a, mu, s, n_sm);
    case L7: return launch_unfused_t<L7, T>(a, mu, s, n_sm);
    case L27: return launch_unfused_t<L27, T>(a, mu, s, n_sm);
    default: return launch_unfused_t<L13X4, T>(a, mu, s, n_sm);
    }
}

cudaError_t launch_unfused_ch(int dtype, int stencil, const StepArgs &a, void *mu, cudaStream_t s, int n_sm) {
    switch (dtype) {
    case SP_F64: return launch_unfused_st<double>(stencil, a, mu, s, n_sm);
    case SP_F32: return launch_unfused_st<float>(stencil, a, mu, s, n_sm);
    default: return launch_unfused_st<bf16>(stencil, a, mu, s, n_sm);
    }
}

}  // namespace sp

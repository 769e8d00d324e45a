// sp_reduce.cu -- FP64 reductions over a resident field: mass, discrete Landau
// free energy, sums, sum of squares, min and max.
//
// Mass M = h^d sum phi (conserved by Model B, Eq. (model-b)); free energy
// F_h = h^d sum [1/2 sum_axes ((phi_{i+e} - phi_i)/h)^2 - c1/2 phi^2 + c2/4 phi^4],
// the Landau density whose functional derivative (Eq. (2) of the paper, first-
// order case) gives Models A and B, with forward differences.
//
// Two passes, deterministic for a fixed grid size: every thread keeps a
// Neumaier-compensated (sum, correction) pair over a grid-stride range (fed
// with FP64 sums of 16-value blocks); warps combine pairs with shuffles,
// blocks through shared memory, and each block writes its pair to a scratch
// array; a single block then combines the block pairs in index order and
// writes the scaled result.
#include <type_traits>

#include "sp_internal.h"

namespace sp {

__device__ __forceinline__ void neu_add(double &s, double &c, double x) {
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
}

__device__ __forceinline__ void neu_merge(double &s, double &c, double s2, double c2) {
    neu_add(s, c, s2);
    c += c2;
}

template <int WHAT>
__device__ __forceinline__ void combine(double &s, double &c, double s2, double c2) {
    if constexpr (WHAT == SP_MIN_U) s = fmin(s, s2);
    else if constexpr (WHAT == SP_MAX_U) s = fmax(s, s2);
    else neu_merge(s, c, s2, c2);
}

template <int WHAT>
__device__ __forceinline__ void block_combine(double &s, double &c) {
    __shared__ double ws[32], wc[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double s2 = __shfl_down_sync(0xffffffffu, s, off);
        const double c2 = __shfl_down_sync(0xffffffffu, c, off);
        combine<WHAT>(s, c, s2, c2);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) { ws[warp] = s; wc[warp] = c; }
    __syncthreads();
    if (warp == 0) {
        s = lane < nw ? ws[lane] : ((WHAT == SP_MIN_U) ? INFINITY : (WHAT == SP_MAX_U ? -INFINITY : 0.0));
        c = lane < nw ? wc[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double s2 = __shfl_down_sync(0xffffffffu, s, off);
            const double c2 = __shfl_down_sync(0xffffffffu, c, off);
            combine<WHAT>(s, c, s2, c2);
        }
    }
}

// Point value of a plain reduction (sum, mass, sum of squares) in FP64.
template <int WHAT> __device__ __forceinline__ double point_value(double p) {
    if constexpr (WHAT == SP_SUMSQ_U) return p * p;
    else return p;
}

// Free-energy density at linear index i (forward differences, periodic).
// With rho (Model C) the density adds rho^2/2 - c3 phi^2 rho; with currents
// (Model H, nq components) it adds (j_x^2 + j_y^2 [+ j_z^2]) / 2.
template <typename T>
__device__ __forceinline__ double fe_density(const T *__restrict__ f, const T *__restrict__ rho, const T *const *jq,
                                             int nq, uint64_t i, int nx, int ny, int nz, int dims, double h, double c1,
                                             double c2, double c3) {
    const double p = (double)to_c(f[i]);
    const int x = (int)(i % (uint64_t)nx);
    const int y = (int)((i / (uint64_t)nx) % (uint64_t)ny);
    const uint64_t row = i - (uint64_t)x;
    const uint64_t zbase = row - (uint64_t)y * nx;
    const double px = (double)to_c(f[row + (x + 1 == nx ? 0 : x + 1)]);
    const double py = (double)to_c(f[zbase + (uint64_t)(y + 1 == ny ? 0 : y + 1) * nx + x]);
    const double gx = (px - p) / h;
    const double gy = (py - p) / h;
    double g2 = gx * gx + gy * gy;
    if (dims == 3) {
        const int z = (int)(i / ((uint64_t)nx * ny));
        const uint64_t plane = (uint64_t)nx * ny;
        const double pz = (double)to_c(f[(uint64_t)(z + 1 == nz ? 0 : z + 1) * plane + (i - (uint64_t)z * plane)]);
        const double gz = (pz - p) / h;
        g2 = g2 + gz * gz;
    }
    const double p2 = p * p;
    if (nq > 0) {
        double q = (double)to_c(jq[0][i]) * (double)to_c(jq[0][i]) + (double)to_c(jq[1][i]) * (double)to_c(jq[1][i]);
        if (nq == 3) q = q + (double)to_c(jq[2][i]) * (double)to_c(jq[2][i]);
        return (0.5 * g2 - 0.5 * c1 * p2 + 0.25 * c2 * p2 * p2) + 0.5 * q;
    }
    if (rho) {
        const double r = (double)to_c(rho[i]);
        return 0.5 * g2 - 0.5 * c1 * p2 + 0.25 * c2 * p2 * p2 + 0.5 * r * r - c3 * p2 * r;
    }
    return 0.5 * g2 - 0.5 * c1 * p2 + 0.25 * c2 * p2 * p2;
}

// Sum of a block of 32 FP32 values (BF16 values widen to FP32 exactly) in
// fixed point, with integer arithmetic only.  A value with biased exponent e
// and 24-bit significand m is m * 2^(max(e,1) - 150).  With E the largest
// exponent of the block, every value is expressed in units of 2^(E - 150 - K),
// K = 33: v = floor(m * 2^(K - (E - max(e,1)))), so the block's largest values
// keep every bit and values more than 2^33 times smaller lose the bits below
// the unit (an error below 2^-56 max|x| each, at most 2^-51 max|x| per block).
// 32 values of at most 24 + 33 bits sum exactly in 62 bits.  The integer sum is
// converted to FP64 once (one rounding) and scaled by the exact power of two.
// A block holding an infinity or a NaN (E = 255) is summed in FP64 instead, so
// that those propagate as in plain summation.
__device__ __forceinline__ double fixed_block_sum32(const float *x) {
    constexpr int K = 33;
    uint32_t b[32];
    int emax = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        b[j] = __float_as_uint(x[j]);
        emax = max(emax, (int)((b[j] >> 23) & 0xffu));
    }
    if (emax == 255) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < 32; ++j) s += (double)x[j];
        return s;
    }
    const int em = max(emax, 1);
    long long acc = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const int e = (int)((b[j] >> 23) & 0xffu);
        const unsigned long long m = (unsigned long long)((b[j] & 0x7fffffu) | (e ? 0x800000u : 0u));
        const int sh = min(em - max(e, 1), 63);
        const long long v = (long long)((m << K) >> sh);
        const long long sgn = -(long long)(b[j] >> 31);  // 0 or -1
        acc += (v ^ sgn) - sgn;
    }
    // 2^(em - 150 - K) as an FP64 power of two (em - 183 >= -182: a normal number)
    const double unit = __longlong_as_double((long long)(em - 150 - K + 1023) << 52);
    return __ll2double_rn(acc) * unit;
}

// Block partials.  Sums: each thread reads 16-byte vectors in a grid-stride
// loop.  FP32 / BF16 mass and plain sums: the vectors are taken in groups of
// 32 values per thread (a warp's group interleaves its lanes, so every load
// instruction is coalesced), each group is summed exactly in fixed point
// (fixed_block_sum32) and folded into the thread's Neumaier pair, so the FP64
// pipe (slow on this part) sees ~0.3 operations per value; error bound u|S| +
// 5u sum|x| per thread (truncation 4u, conversion u).  FP64 fields and sums of
// squares: plain FP64 additions over blocks of 16 values folded into the
// Neumaier pair, ~2 FP64 operations per value, bound u|S| + 15u sum|x|.  The
// remaining vectors and the scalar tail take the FP64 block path.  Min / max run
// in the compute type.  The free energy keeps a per-point Neumaier update.
template <typename T, int WHAT>
__global__ void __launch_bounds__(kReduceThreads)
reduce_partial_kernel(const T *__restrict__ f, const T *__restrict__ rho, const T *j0, const T *j1, const T *j2, int nq,
                      int nx, int ny, int nz, int dims, double h, double c1, double c2, double c3,
                      double *__restrict__ partials) {
    typedef typename Cmp<T>::type C;
    constexpr int VE = 16 / sizeof(T);       // values per vector
    constexpr int kBlockVecs = (16 + VE - 1) / VE;
    const uint64_t N = (uint64_t)nx * ny * nz;
    double s = (WHAT == SP_MIN_U) ? INFINITY : (WHAT == SP_MAX_U ? -INFINITY : 0.0), c = 0.0;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if constexpr (WHAT == SP_FREE_ENERGY) {
        const T *jq[3] = {j0, j1, j2};
        for (uint64_t i = tid; i < N; i += stride)
            neu_add(s, c, fe_density(f, rho, jq, nq, i, nx, ny, nz, dims, h, c1, c2, c3));
    } else {
        // vector part when the base is 16-byte aligned (library buffers always are;
        // a caller's pointer may not be), then the scalar tail
        const bool aligned = (reinterpret_cast<uintptr_t>(f) & 15u) == 0;
        const uint64_t NV = aligned ? N / VE : 0;
        C mn = C(INFINITY), mx = C(-INFINITY);
        double blk = 0.0;
        int nb = 0;
        uint64_t v0 = 0;  // first vector of the FP64 block path
        if constexpr (!std::is_same<T, double>::value && (WHAT == SP_MASS || WHAT == SP_SUM_U)) {
            constexpr int G = 32 / VE;  // vectors per thread per group
            const uint64_t lane = threadIdx.x & 31u, warp = tid >> 5;
            const uint64_t nwarps = stride >> 5;
            const uint64_t ngroups = NV / (32u * G);
            for (uint64_t gi = warp; gi < ngroups; gi += nwarps) {
                float x[32];
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    C xv[VE];
                    load_vec<T, VE>(f + ((gi * G + j) * 32u + lane) * VE, xv);
#pragma unroll
                    for (int q = 0; q < VE; ++q) x[j * VE + q] = xv[q];
                }
                neu_add(s, c, fixed_block_sum32(x));
            }
            v0 = ngroups * 32u * G;
        }
        for (uint64_t v = v0 + tid; v < NV; v += stride) {
            C x[VE];
            load_vec<T, VE>(f + v * VE, x);
            if constexpr (WHAT == SP_MIN_U) {
#pragma unroll
                for (int j = 0; j < VE; ++j) mn = fmin(mn, x[j]);
            } else if constexpr (WHAT == SP_MAX_U) {
#pragma unroll
                for (int j = 0; j < VE; ++j) mx = fmax(mx, x[j]);
            } else {
#pragma unroll
                for (int j = 0; j < VE; ++j) blk += point_value<WHAT>((double)x[j]);
                if (++nb == kBlockVecs) {
                    neu_add(s, c, blk);
                    blk = 0.0;
                    nb = 0;
                }
            }
        }
        for (uint64_t i = NV * VE + tid; i < N; i += stride) {
            const C x = to_c(f[i]);
            if constexpr (WHAT == SP_MIN_U) mn = fmin(mn, x);
            else if constexpr (WHAT == SP_MAX_U) mx = fmax(mx, x);
            else blk += point_value<WHAT>((double)x);
        }
        if constexpr (WHAT == SP_MIN_U) s = (double)mn;
        else if constexpr (WHAT == SP_MAX_U) s = (double)mx;
        else neu_add(s, c, blk);
    }
    block_combine<WHAT>(s, c);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = s;
        partials[2 * blockIdx.x + 1] = c;
    }
}

template <int WHAT>
__global__ void __launch_bounds__(kReduceThreads)
reduce_final_kernel(const double *__restrict__ partials, int nblocks, double scale, double *__restrict__ out) {
    double s = (WHAT == SP_MIN_U) ? INFINITY : (WHAT == SP_MAX_U ? -INFINITY : 0.0), c = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) combine<WHAT>(s, c, partials[2 * b], partials[2 * b + 1]);
    block_combine<WHAT>(s, c);
    if (threadIdx.x == 0) {
        if constexpr (WHAT == SP_MIN_U || WHAT == SP_MAX_U) out[0] = s;
        else out[0] = scale * (isfinite(s) ? s + c : s);  // an infinite sum keeps its sign (c is NaN then)
    }
}

template <typename T, int WHAT>
static cudaError_t launch_reduce_t(const void *f, const ReduceGeom &g, double *partials, int nblocks,
                                   double *out, cudaStream_t s) {
    const double scale = (WHAT == SP_MASS || WHAT == SP_FREE_ENERGY) ? g.cell_volume : 1.0;
    reduce_partial_kernel<T, WHAT><<<nblocks, kReduceThreads, 0, s>>>(
        static_cast<const T *>(f), static_cast<const T *>(g.rho), static_cast<const T *>(g.jq[0]),
        static_cast<const T *>(g.jq[1]), static_cast<const T *>(g.jq[2]), g.nq, g.nx, g.ny, g.nz, g.dims, g.h, g.c1,
        g.c2, g.c3, partials);
    reduce_final_kernel<WHAT><<<1, kReduceThreads, 0, s>>>(partials, nblocks, scale, out);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_reduce_dt(int what, const void *f, const ReduceGeom &g, double *partials, int nblocks,
                                    double *out, cudaStream_t s) {
    switch (what) {
    case SP_MASS: return launch_reduce_t<T, SP_MASS>(f, g, partials, nblocks, out, s);
    case SP_FREE_ENERGY: return launch_reduce_t<T, SP_FREE_ENERGY>(f, g, partials, nblocks, out, s);
    case SP_SUM_U:
    case SP_SUM_V: return launch_reduce_t<T, SP_SUM_U>(f, g, partials, nblocks, out, s);
    case SP_MIN_U: return launch_reduce_t<T, SP_MIN_U>(f, g, partials, nblocks, out, s);
    case SP_MAX_U: return launch_reduce_t<T, SP_MAX_U>(f, g, partials, nblocks, out, s);
    case SP_SUMSQ_U: return launch_reduce_t<T, SP_SUMSQ_U>(f, g, partials, nblocks, out, s);
    }
    return cudaErrorInvalidValue;
}

int reduce_blocks(uint64_t N, int n_sm) {
    const uint64_t want = (N + kReduceThreads - 1) / kReduceThreads;
    const uint64_t cap = (uint64_t)n_sm * kReduceBlocksPerSM;
    const uint64_t b = want < cap ? want : cap;
    return (int)(b > 0 ? b : 1);
}

cudaError_t launch_reduce(int dtype, int what, const void *f, const ReduceGeom &g, double *partials,
                          int nblocks, double *out, cudaStream_t s) {
    switch (dtype) {
    case SP_F64: return launch_reduce_dt<double>(what, f, g, partials, nblocks, out, s);
    case SP_F32: return launch_reduce_dt<float>(what, f, g, partials, nblocks, out, s);
    default: return launch_reduce_dt<bf16>(what, f, g, partials, nblocks, out, s);
    }
}

}  // namespace sp

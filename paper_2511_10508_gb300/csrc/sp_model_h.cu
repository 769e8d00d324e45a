// sp_model_h.cu -- Model H (Sec. "Model H", transverse projector at unity), a
// conserved scalar m and a d-vector current j, signs of the paper's listing:
//   mu    = -kappa lap m - c1 m + c2 m^3
//   dm/dt = lap mu - c3 div(m j)
//   dj/dt = lap j - c3 m grad mu
// grad and div are central differences of the Laplacian stencil's order.
//
// Like the paper's solver (one temporary for Model H, Table 2), the per-point
// kernels take two passes: mu for every point into a compute-precision buffer,
// then the update of m and of each component of j, which reads mu, m and j
// through periodic taps (the flux m j_a is formed at each tap, with the
// rounding of the product m * j_a).  2D FP32 / BF16 grids instead use one
// shared-memory tile pass with mu kept on chip (FP64 is bound by the FP64
// pipe, where the halo mu of a tile costs more than the buffer).  Fixed order per point (FP64 results equal the oracle's bit for bit):
//   mu  = fma(m, fma(c2, m*m, -c1), -((kappa/q_h2) * S(m)))
//   div = (D_x(m j_x) + D_y(m j_y)) [+ D_z(m j_z)]
//   m'  = fma(dt, fma(1/q_h2, S(mu), -(c3g * div)), m)
//   j_a' = fma(dt, fma(1/q_h2, S(j_a), -(c3g * (m * D_a mu))), j_a)
// with D f = f(+1) - f(-1) (radius-1 stencils) or fma(8, f(+1) - f(-1),
// -(f(+2) - f(-2))) (radius 2) and c3g = c3 / (2h) or c3 / (12h).
#include <type_traits>

#include "sp_internal.h"

namespace sp {

// Wrapped offsets of the planes and rows within the stencil radius around a
// 256-point row segment (computed once per segment).
template <int R>
struct TapRows {
    size_t zb[2 * R + 1], yb[2 * R + 1];
    __device__ __forceinline__ TapRows(int y, int z, int nx, int ny, int nz) {
#pragma unroll
        for (int d = -R; d <= R; ++d) {
            zb[d + R] = (size_t)wrap_idx(z + d, nz) * ny * nx;
            yb[d + R] = (size_t)wrap_idx(y + d, ny) * nx;
        }
    }
    __device__ __forceinline__ size_t at(int x, int nx, int dx, int dy, int dz) const {
        return zb[dz + R] + yb[dy + R] + wrap_idx(x + dx, nx);
    }
};

struct MhArgs {
    const void *m, *j[3];
    void *mo, *jo[3];
    void *mu;
    int nx, ny, nz;
    StepConsts k;
    StepConstsF kf;
};

__device__ __forceinline__ void mh_seg(long long u, int segs, const MhArgs &a, int &x, int &y, int &z, size_t &row) {
    const long long r = u / segs;
    x = (int)(u - r * segs) * 256 + (int)threadIdx.x;
    y = (int)(r % a.ny);
    z = (int)(r / a.ny);
    row = (size_t)r * a.nx;
}

// central difference along axis A of f at the tap origin
template <int R, int A, typename Fn>
__device__ __forceinline__ auto central(const Fn &f) -> decltype(f(0, 0, 0)) {
    constexpr int ex = (A == 0), ey = (A == 1), ez = (A == 2);
    const auto d1 = f(ex, ey, ez) - f(-ex, -ey, -ez);
    if constexpr (R == 1) {
        return d1;
    } else {
        const auto d2 = f(2 * ex, 2 * ey, 2 * ez) - f(-2 * ex, -2 * ey, -2 * ez);
        return FMA(decltype(d1)(8), d1, -d2);
    }
}

template <int ST, typename T>
__global__ void __launch_bounds__(256) mh_mu_kernel(MhArgs a, int segs) {
    typedef typename Cmp<T>::type C;
    constexpr int R = StencilInfo<ST>::r;
    const ConstsC<C> k(a.k, a.kf);
    const T *m = static_cast<const T *>(a.m);
    C *mu = static_cast<C *>(a.mu);
    const long long units = (long long)a.ny * a.nz * segs;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        int x, y, z;
        size_t row;
        mh_seg(u, segs, a, x, y, z, row);
        const TapRows<R> tp(y, z, a.nx, a.ny, a.nz);
        if (x >= a.nx) continue;
        auto P = [&](int dx, int dy, int dz) -> C { return to_c(m[tp.at(x, a.nx, dx, dy, dz)]); };
        mu[row + x] = ch_mu<C>(to_c(m[row + x]), stencil_sum<ST, C>(P), k);
    }
}

template <int ST, typename T, int DIMS>
__global__ void __launch_bounds__(256) mh_update_kernel(MhArgs a, int segs, typename Cmp<T>::type c3g) {
    typedef typename Cmp<T>::type C;
    constexpr int R = StencilInfo<ST>::r;
    const ConstsC<C> k(a.k, a.kf);
    const T *m = static_cast<const T *>(a.m);
    const C *mu = static_cast<const C *>(a.mu);
    const T *j[3] = {static_cast<const T *>(a.j[0]), static_cast<const T *>(a.j[1]), static_cast<const T *>(a.j[2])};
    T *jo[3] = {static_cast<T *>(a.jo[0]), static_cast<T *>(a.jo[1]), static_cast<T *>(a.jo[2])};
    const long long units = (long long)a.ny * a.nz * segs;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        int x, y, z;
        size_t row;
        mh_seg(u, segs, a, x, y, z, row);
        const TapRows<R> tp(y, z, a.nx, a.ny, a.nz);
        if (x >= a.nx) continue;
        const size_t i = row + x;
        auto Pmu = [&](int dx, int dy, int dz) -> C { return mu[tp.at(x, a.nx, dx, dy, dz)]; };
        auto flux = [&](int ax) {
            return [&, ax](int dx, int dy, int dz) -> C {
                const size_t t = tp.at(x, a.nx, dx, dy, dz);
                return to_c(m[t]) * to_c(j[ax][t]);
            };
        };
        C div = central<R, 0>(flux(0)) + central<R, 1>(flux(1));
        if constexpr (DIMS == 3) div = div + central<R, 2>(flux(2));
        const C mi = to_c(m[i]);
        static_cast<T *>(a.mo)[i] = from_c<T>(FMA(k.dt, FMA(k.sAC, stencil_sum<ST, C>(Pmu), -(c3g * div)), mi));
#pragma unroll
        for (int ax = 0; ax < DIMS; ++ax) {
            C gm;
            if (ax == 0) gm = central<R, 0>(Pmu);
            else if (ax == 1) gm = central<R, 1>(Pmu);
            else gm = central<R, 2>(Pmu);
            auto Pj = [&](int dx, int dy, int dz) -> C { return to_c(j[ax][tp.at(x, a.nx, dx, dy, dz)]); };
            jo[ax][i] = from_c<T>(FMA(k.dt, FMA(k.sAC, stencil_sum<ST, C>(Pj), -(c3g * (mi * gm))), to_c(j[ax][i])));
        }
    }
}

// 2D tiles (FP32 / BF16 storage): one BX x BY output tile per CTA.  m and the
// components of j are fetched once with a 2R halo (x padded to whole 16-byte
// chunks), mu is evaluated on the tile grown by R into shared memory, and the
// update reads everything from shared memory: one pass over HBM instead of two
// plus the mu buffer.  The same expressions as the per-point kernels, so the
// results are identical to theirs.
template <int ST, typename T, int BX, int BY>
struct MhTile2dShape {
    typedef typename Cmp<T>::type C;
    static constexpr int R = StencilInfo<ST>::r;
    static constexpr int RIN = 2 * R;
    static constexpr int CK = 16 / sizeof(T);
    static constexpr int HC = (RIN + CK - 1) / CK;
    static constexpr int NCK = BX / CK + 2 * HC;
    static constexpr int SW = NCK * CK, X0 = HC * CK;
    static constexpr int HIN = BY + 2 * RIN;
    static constexpr int NF = 3;  // m, j_x, j_y
    static constexpr int WMU = BX + 2 * R, HMU = BY + 2 * R;
    static constexpr size_t bytes_in = sizeof(T) * (size_t)NF * HIN * SW;
    static constexpr size_t smem_bytes = bytes_in + sizeof(C) * (size_t)WMU * HMU;
    static_assert(bytes_in % 16 == 0, "mu array alignment");
};

template <int ST, typename T, int BX, int BY, int NT>
__global__ void __launch_bounds__(NT) mh_tile2d_kernel(MhArgs a, typename Cmp<T>::type c3g) {
    typedef MhTile2dShape<ST, T, BX, BY> Sh;
    typedef typename Sh::C C;
    constexpr int R = Sh::R, RIN = Sh::RIN, CK = Sh::CK, NCK = Sh::NCK, SW = Sh::SW, X0 = Sh::X0;
    constexpr int HIN = Sh::HIN, NF = Sh::NF, WMU = Sh::WMU, HMU = Sh::HMU;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_in = reinterpret_cast<T *>(smem_raw);                 // [NF][HIN][SW]: m, j_x, j_y
    C *s_mu = reinterpret_cast<C *>(smem_raw + Sh::bytes_in);  // [HMU][WMU]
    const ConstsC<C> k(a.k, a.kf);
    const int nx = a.nx, ny = a.ny, t = threadIdx.x;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const bool vec_ok = (nx % CK) == 0;
    const T *in[NF] = {static_cast<const T *>(a.m), static_cast<const T *>(a.j[0]), static_cast<const T *>(a.j[1])};
    T *out[NF] = {static_cast<T *>(a.mo), static_cast<T *>(a.jo[0]), static_cast<T *>(a.jo[1])};

    // chunk c of shared row i holds columns x0 - X0 + c*CK .. +CK-1 of grid row y0 - RIN + i
    for (int q = t; q < HIN * NCK; q += NT) {
        const int i = q / NCK, c = q - i * NCK;
        const int y = wrap_idx(y0 - RIN + i, ny);
        const int x = x0 - X0 + c * CK;
        const size_t row = (size_t)y * (size_t)nx;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T *dst = s_in + ((size_t)f * HIN + i) * SW + c * CK;
            if (vec_ok && x >= 0 && x + CK <= nx) {
                cp_async16(dst, in[f] + row + x);
            } else {
#pragma unroll
                for (int jj = 0; jj < CK; ++jj) dst[jj] = in[f][row + wrap_idx(x + jj, nx)];
            }
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();

    // field f at tile coordinates (i, j), -RIN <= i < BY + RIN, -X0 <= j < BX + X0
    auto fld = [&](int f, int i, int j) -> C { return to_c(s_in[((size_t)f * HIN + i + RIN) * SW + j + X0]); };
    for (int q = t; q < HMU * WMU; q += NT) {
        const int i = q / WMU - R, j = q % WMU - R;
        auto P = [&](int dx, int dy, int) -> C { return fld(0, i + dy, j + dx); };
        s_mu[q] = ch_mu<C>(fld(0, i, j), stencil_sum<ST, C>(P), k);
    }
    __syncthreads();
    for (int q = t; q < BY * BX; q += NT) {
        const int i = q / BX, j = q - i * BX;
        const int y = y0 + i, x = x0 + j;
        if (y >= ny || x >= nx) continue;
        const size_t o = (size_t)y * (size_t)nx + x;
        auto Pmu = [&](int dx, int dy, int) -> C { return s_mu[(i + R + dy) * WMU + (j + R + dx)]; };
        auto flux = [&](int ax) {
            return [&, ax](int dx, int dy, int) -> C { return fld(0, i + dy, j + dx) * fld(1 + ax, i + dy, j + dx); };
        };
        const C div = central<R, 0>(flux(0)) + central<R, 1>(flux(1));
        const C mi = fld(0, i, j);
        out[0][o] = from_c<T>(FMA(k.dt, FMA(k.sAC, stencil_sum<ST, C>(Pmu), -(c3g * div)), mi));
#pragma unroll
        for (int ax = 0; ax < 2; ++ax) {
            const C gm = (ax == 0) ? central<R, 0>(Pmu) : central<R, 1>(Pmu);
            auto Pj = [&](int dx, int dy, int) -> C { return fld(1 + ax, i + dy, j + dx); };
            out[1 + ax][o] = from_c<T>(FMA(k.dt, FMA(k.sAC, stencil_sum<ST, C>(Pj), -(c3g * (mi * gm))), fld(1 + ax, i, j)));
        }
    }
}

// 3D FP32 / BF16: xy tiles streamed along z.  Each loaded plane (tile plus a 2R
// halo, all four fields, widened to FP32) enters a ring of D = 3R + 2 planes in
// shared memory; mu of plane i - R (tile grown by R) goes to a ring of 2R + 1
// planes; the update of plane i - 2R then reads m and j on planes i - 3R .. i - R
// and mu from the rings.  The ring depth keeps the plane committed at iteration i
// clear of every plane a thread still in iteration i - 1 may read.  Work items
// are (z segment, tile) pairs handed out round by round, segment-major, so the
// resident CTAs stream the same z range together and the halo rows and columns
// that neighbouring tiles share are still in L2 when the second tile reads them.
// The same expressions as the per-point kernels, so the results are identical.
template <int ST, typename T, int TX, int TY>
struct MhRing3dShape {
    static constexpr int R = StencilInfo<ST>::r;
    static constexpr int RIN = 2 * R;
    static constexpr int WIN = TX + 2 * RIN, HIN = TY + 2 * RIN, AIN = WIN * HIN;
    static constexpr int D = 3 * R + 2;
    static constexpr int NF = 4;  // m, j_x, j_y, j_z
    static constexpr int WMU = TX + 2 * R, HMU = TY + 2 * R, AMU = WMU * HMU, DMU = 2 * R + 1;
    static constexpr size_t smem_bytes = sizeof(float) * ((size_t)NF * D * AIN + (size_t)DMU * AMU);
};

template <int ST, typename T, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) mh_ring3d_kernel(MhArgs a, float c3g, int tiles_x, int tiles_y, int segs) {
    typedef float C;
    typedef MhRing3dShape<ST, T, TX, TY> Sh;
    constexpr int R = Sh::R, RIN = Sh::RIN, WIN = Sh::WIN, AIN = Sh::AIN, D = Sh::D, NF = Sh::NF;
    constexpr int WMU = Sh::WMU, AMU = Sh::AMU, DMU = Sh::DMU;
    constexpr int EPT = (AIN + NT - 1) / NT;  // loaded cells per thread per field
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s_in = reinterpret_cast<C *>(smem_raw);  // [NF][D][AIN]
    C *s_mu = s_in + (size_t)NF * D * AIN;      // [DMU][AMU]
    const ConstsC<C> k(a.k, a.kf);
    const int nx = a.nx, ny = a.ny, nz = a.nz, t = threadIdx.x;
    const size_t plane = (size_t)nx * (size_t)ny;
    const T *in[NF] = {static_cast<const T *>(a.m), static_cast<const T *>(a.j[0]), static_cast<const T *>(a.j[1]),
                       static_cast<const T *>(a.j[2])};
    T *out[NF] = {static_cast<T *>(a.mo), static_cast<T *>(a.jo[0]), static_cast<T *>(a.jo[1]),
                  static_cast<T *>(a.jo[2])};
    auto S_in = [&](int f, int i) -> const C * { return s_in + ((size_t)f * D + (i % D)) * AIN; };

    const int tiles = tiles_x * tiles_y;
    for (long long it = blockIdx.x; it < (long long)tiles * segs; it += gridDim.x) {
        const int seg = (int)(it / tiles), tile = (int)(it - (long long)seg * tiles);
        const int z0 = (int)((long long)seg * nz / segs), z1 = (int)((long long)(seg + 1) * nz / segs);
        const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
        const int nplanes = (z1 - z0) + 2 * RIN;  // loaded plane i is z = z0 - RIN + i

        int loff[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int c = t + e * NT;
            if (c < AIN) {
                const int yi = c / WIN, xi = c - yi * WIN;
                loff[e] = wrap_idx(y0 - RIN + yi, ny) * nx + wrap_idx(x0 - RIN + xi, nx);
            } else {
                loff[e] = -1;
            }
        }
        C pf[NF][EPT];
        auto fetch = [&](int i) {
            const size_t zoff = (size_t)wrap_idx(z0 - RIN + i, nz) * plane;
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
                for (int e = 0; e < EPT; ++e)
                    if (loff[e] >= 0) pf[f][e] = to_c(in[f][zoff + loff[e]]);
        };
        auto commit = [&](int i) {
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
                for (int e = 0; e < EPT; ++e)
                    if (loff[e] >= 0) s_in[((size_t)f * D + (i % D)) * AIN + t + e * NT] = pf[f][e];
        };

        fetch(0);
        for (int i = 0; i < nplanes; ++i) {
            commit(i);
            if (i + 1 < nplanes) fetch(i + 1);
            __syncthreads();
            if (i >= 2 * R) {
                // mu of plane i - R over the tile grown by R
                C *mu = s_mu + (size_t)((i - R) % DMU) * AMU;
                for (int c = t; c < AMU; c += NT) {
                    const int ym = c / WMU, xm = c - ym * WMU;
                    const int base = (ym + R) * WIN + (xm + R);
                    auto P = [&](int dx, int dy, int dz) -> C { return S_in(0, i - R + dz)[base + dy * WIN + dx]; };
                    mu[c] = ch_mu<C>(S_in(0, i - R)[base], stencil_sum<ST, C>(P), k);
                }
            }
            __syncthreads();
            if (i >= 4 * R) {
                const int o = i - 2 * R;  // loaded index of the output plane
                const size_t zo = (size_t)(z0 + o - RIN) * plane;
                for (int c = t; c < TX * TY; c += NT) {
                    const int yy = c / TX, xx = c - yy * TX;
                    const int x = x0 + xx, y = y0 + yy;
                    if (x >= nx || y >= ny) continue;
                    const int b = (yy + RIN) * WIN + xx + RIN;
                    const int mb = (yy + R) * WMU + (xx + R);
                    auto Pmu = [&](int dx, int dy, int dz) -> C {
                        return s_mu[(size_t)((o + dz) % DMU) * AMU + mb + dy * WMU + dx];
                    };
                    auto fld = [&](int f, int dx, int dy, int dz) -> C { return S_in(f, o + dz)[b + dy * WIN + dx]; };
                    auto flux = [&](int ax) {
                        return [&, ax](int dx, int dy, int dz) -> C { return fld(0, dx, dy, dz) * fld(1 + ax, dx, dy, dz); };
                    };
                    const C div = (central<R, 0>(flux(0)) + central<R, 1>(flux(1))) + central<R, 2>(flux(2));
                    const C mi = fld(0, 0, 0, 0);
                    const size_t oi = zo + (size_t)y * nx + x;
                    out[0][oi] = from_c<T>(FMA(k.dt, FMA(k.sAC, stencil_sum<ST, C>(Pmu), -(c3g * div)), mi));
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        const C gm = (ax == 0) ? central<R, 0>(Pmu) : (ax == 1 ? central<R, 1>(Pmu) : central<R, 2>(Pmu));
                        auto Pj = [&](int dx, int dy, int dz) -> C { return fld(1 + ax, dx, dy, dz); };
                        out[1 + ax][oi] =
                            from_c<T>(FMA(k.dt, FMA(k.sAC, stencil_sum<ST, C>(Pj), -(c3g * (mi * gm))), fld(1 + ax, 0, 0, 0)));
                    }
                }
            }
        }
        __syncthreads();  // the rings are reused by the next segment
    }
}

template <int ST, typename T>
static cudaError_t launch_mh_t(const MhArgs &a, double c3g, cudaStream_t s, int n_sm) {
    typedef typename Cmp<T>::type C;
    if constexpr (StencilInfo<ST>::dims == 2 && !std::is_same<T, double>::value) {
        // family 0: shared-memory tiles; family 1: the two per-point passes
        if (g_step_variant != 1) {
            constexpr int BX = 128, BY = 16, NT = 256;
            typedef MhTile2dShape<ST, T, BX, BY> Sh;
            auto kern = mh_tile2d_kernel<ST, T, BX, BY, NT>;
            static const bool attr = [&] {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
                return true;
            }();
            (void)attr;
            kern<<<dim3((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY), NT, Sh::smem_bytes, s>>>(a, (C)c3g);
            return cudaGetLastError();
        }
    }
    if constexpr (StencilInfo<ST>::dims == 3 && !std::is_same<T, double>::value) {
        // family 0: z-streaming tiles; family 1: the two per-point passes
        if (g_step_variant != 1) {
            constexpr int TX = 32, TY = 16, NT = 256;
            typedef MhRing3dShape<ST, T, TX, TY> Sh;
            auto kern = mh_ring3d_kernel<ST, T, TX, TY, NT>;
            static const int occ = [&] {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
                int o = 1;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, NT, Sh::smem_bytes);
                return o;
            }();
            const int tx = (a.nx + TX - 1) / TX, ty = (a.ny + TY - 1) / TY;
            const long long wave = (long long)n_sm * std::max(occ, 1);
            const int segs = lockstep_segments((long long)tx * ty, a.nz, 2 * Sh::RIN, wave);
            const long long items = (long long)tx * ty * segs;
            kern<<<(unsigned)std::min(items, wave), NT, Sh::smem_bytes, s>>>(a, (C)c3g, tx, ty, segs);
            return cudaGetLastError();
        }
    }
    const int segs = (a.nx + 255) / 256;
    const long long units = (long long)a.ny * a.nz * segs;
    const unsigned blocks = (unsigned)std::min<long long>(units, (long long)n_sm * 8);
    mh_mu_kernel<ST, T><<<blocks, 256, 0, s>>>(a, segs);
    if constexpr (StencilInfo<ST>::dims == 2)
        mh_update_kernel<ST, T, 2><<<blocks, 256, 0, s>>>(a, segs, (C)c3g);
    else
        mh_update_kernel<ST, T, 3><<<blocks, 256, 0, s>>>(a, segs, (C)c3g);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_mh_st(int stencil, const MhArgs &a, double c3g, cudaStream_t s, int n_sm) {
    switch (stencil) {
    case L5: return launch_mh_t<L5, T>(a, c3g, s, n_sm);
    case L9BOX: return launch_mh_t<L9BOX, T>(a, c3g, s, n_sm);
    case L9X4: return launch_mh_t<L9X4, T>(a, c3g, s, n_sm);
    case L7: return launch_mh_t<L7, T>(a, c3g, s, n_sm);
    case L27: return launch_mh_t<L27, T>(a, c3g, s, n_sm);
    default: return launch_mh_t<L13X4, T>(a, c3g, s, n_sm);
    }
}

cudaError_t launch_model_h(int dtype, int stencil, void *const in[4], void *const out[4], void *mu, int nx, int ny,
                           int nz, const StepConsts &k, double c3g, cudaStream_t s, int n_sm) {
    MhArgs a;
    a.m = in[0];
    a.mo = out[0];
    for (int c = 0; c < 3; ++c) {
        a.j[c] = in[1 + c] ? in[1 + c] : in[1];
        a.jo[c] = out[1 + c] ? out[1 + c] : out[1];
    }
    a.mu = mu;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.k = k;
    a.kf = to_float(k);
    switch (dtype) {
    case SP_F64: return launch_mh_st<double>(stencil, a, c3g, s, n_sm);
    case SP_F32: return launch_mh_st<float>(stencil, a, c3g, s, n_sm);
    default: return launch_mh_st<bf16>(stencil, a, c3g, s, n_sm);
    }
}

}  // namespace sp

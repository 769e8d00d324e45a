// sp_step.cuh -- fused explicit time-step kernels (one forward-Euler step per
// launch) for Allen-Cahn, Cahn-Hilliard and Gray-Scott on periodic grids.
//
// One pass per step (the paper, Sec. "Benchmarks", stores phi^3 in a temporary
// field for conserved dynamics; here the chemical potential never leaves the
// chip): each CTA owns a column strip of the grid and streams along the slowest
// axis (rows in 2D, z-planes in 3D).  Input slices enter a shared-memory ring
// with a periodic halo; Cahn-Hilliard computes mu for the slice plus an r-wide
// halo into a second ring, then applies the outer Laplacian to mu.  The next
// slice is fetched into registers while the current one is computed.  HBM
// traffic per point and step: one read and one write of each field.
#pragma once

#include "sp_common.cuh"

namespace sp {

// ===================================================================== 2D ==
//
// CTA: NT threads, each owning V consecutive x points; tile width TW = NT*V.
// Rows y0 .. y1-1 of strip [x0, x0+TW) are produced; rows are streamed from
// y0-RIN to y1+RIN-1 (RIN = r, or 2r for Cahn-Hilliard).
template <int MODEL, int ST, typename T, int NT, int V>
__global__ void __launch_bounds__(NT) step2d_kernel(StepArgs a, int TH) {
    typedef typename Cmp<T>::type C;
    constexpr int r = StencilInfo<ST>::r;
    constexpr int RIN = (MODEL == CH) ? 2 * r : r;
    constexpr int TW = NT * V;
    constexpr int WIN = TW + 2 * RIN;
    constexpr int DIN = 2 * r + 2;
    constexpr int NF = (MODEL == GS) ? 2 : 1;
    constexpr int WMU = (MODEL == CH) ? TW + 2 * r : 1;
    constexpr int DMU = (MODEL == CH) ? 2 * r + 1 : 1;
    __shared__ C s_in[NF][DIN][WIN];
    __shared__ C s_mu[DMU][WMU];

    const ConstsC<C> k(a.k);
    const int nx = a.nx, ny = a.ny;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * TW;
    const int y0 = blockIdx.y * TH;
    const int y1 = min(y0 + TH, ny);
    if (y0 >= y1) return;  // uniform per CTA
    const int nrows = (y1 - y0) + 2 * RIN;
    const bool vec = (nx % V) == 0;
    const int xg = x0 + t * V;
    const T *in[2] = {static_cast<const T *>(a.in0), static_cast<const T *>(a.in1)};
    T *out[2] = {static_cast<T *>(a.out0), static_cast<T *>(a.out1)};

    // halo column handled by this thread (threads 0 .. 2*RIN-1)
    const int hxi = (t < RIN) ? t : TW + t;  // smem column
    const int hx = wrap_idx(x0 - RIN + hxi, nx);

    C pf[NF][V];
    C ph[NF];
    auto fetch = [&](int y) {
        const size_t row = (size_t)wrap_idx(y, ny) * (size_t)nx;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const T *src = in[f] + row;
            if (vec && xg + V <= nx) {
                load_vec<T, V>(src + xg, pf[f]);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) pf[f][v] = load_one(src + wrap_idx(xg + v, nx));
            }
            if (t < 2 * RIN) ph[f] = load_one(src + hx);
        }
    };
    auto commit = [&](int slot) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
#pragma unroll
            for (int v = 0; v < V; ++v) s_in[f][slot][RIN + t * V + v] = pf[f][v];
            if (t < 2 * RIN) s_in[f][slot][hxi] = ph[f];
        }
    };
    auto store = [&](int f, int y, const C (&vals)[V]) {
        T *dst = out[f] + (size_t)y * (size_t)nx;
        if (vec && xg + V <= nx) {
            store_vec<T, V>(dst + xg, vals);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (xg + v < nx) dst[xg + v] = from_c<T>(vals[v]);
        }
    };

    fetch(y0 - RIN);
    for (int j = 0; j < nrows; ++j) {
        commit(j % DIN);
        if (j + 1 < nrows) fetch(y0 - RIN + j + 1);
        __syncthreads();
        if constexpr (MODEL == CH) {
            if (j >= 2 * r) {
                // mu of row y0 - r + (j - 2r) over columns x0-r .. x0+TW+r-1
                const int jm = j - 2 * r;
                auto mu_at = [&](int xm) {
                    auto P = [&](int dx, int dy, int) -> C {
                        return s_in[0][(j - r + dy) % DIN][xm + r + dx];
                    };
                    const C S = stencil_sum<ST, C>(P);
                    const C p = s_in[0][(j - r) % DIN][xm + r];
                    s_mu[jm % DMU][xm] = ch_mu<C>(p, S, k);
                };
#pragma unroll
                for (int v = 0; v < V; ++v) mu_at(t * V + v);
                if (t < 2 * r) mu_at(TW + t);
            }
            __syncthreads();
            if (j >= 4 * r) {
                const int yo = y0 + j - 4 * r;
                C o[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int xm = t * V + v + r;
                    auto Pm = [&](int dx, int dy, int) -> C {
                        return s_mu[(j - 3 * r + dy) % DMU][xm + dx];
                    };
                    const C Smu = stencil_sum<ST, C>(Pm);
                    o[v] = ch_update<C>(s_in[0][(j - 2 * r) % DIN][RIN + t * V + v], Smu, k);
                }
                store(0, yo, o);
            }
        } else {
            if (j >= 2 * r) {
                const int yo = y0 + j - 2 * r;
                C o0[V], o1[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int xi = RIN + t * V + v;
                    auto P0 = [&](int dx, int dy, int) -> C {
                        return s_in[0][(j - r + dy) % DIN][xi + dx];
                    };
                    const C S0 = stencil_sum<ST, C>(P0);
                    const C p0 = s_in[0][(j - r) % DIN][xi];
                    if constexpr (MODEL == AC) {
                        o0[v] = ac_update<C>(p0, S0, k);
                    } else {
                        auto P1 = [&](int dx, int dy, int) -> C {
                            return s_in[NF - 1][(j - r + dy) % DIN][xi + dx];
                        };
                        const C S1 = stencil_sum<ST, C>(P1);
                        const C p1 = s_in[NF - 1][(j - r) % DIN][xi];
                        gs_update<C>(p0, p1, S0, S1, k, o0[v], o1[v]);
                    }
                }
                store(0, yo, o0);
                if constexpr (MODEL == GS) store(1, yo, o1);
            }
        }
    }
}

// ===================================================================== 3D ==
//
// CTA: NT threads; tile TX x TY of (x, y); planes z0 .. z1-1 produced, planes
// streamed from z0-RIN to z1+RIN-1.  Plane slices are (TY+2RIN) x (TX+2RIN)
// cells, loaded by a flat loop (consecutive threads, consecutive x).
template <int MODEL, int ST, typename T, int TX, int TY, int NT>
struct Step3dShape {
    typedef typename Cmp<T>::type C;
    static constexpr int r = StencilInfo<ST>::r;
    static constexpr int RIN = (MODEL == CH) ? 2 * r : r;
    static constexpr int WIN = TX + 2 * RIN, HIN = TY + 2 * RIN, AIN = WIN * HIN;
    static constexpr int DIN = 2 * r + 2;
    static constexpr int NF = (MODEL == GS) ? 2 : 1;
    static constexpr int WMU = TX + 2 * r, HMU = TY + 2 * r, AMU = WMU * HMU;
    static constexpr int DMU = (MODEL == CH) ? 2 * r + 1 : 0;
    static constexpr int EPT = (AIN + NT - 1) / NT;  // loaded cells per thread per field
    static constexpr size_t smem_bytes = sizeof(C) * ((size_t)NF * DIN * AIN + (size_t)DMU * AMU);
};

template <int MODEL, int ST, typename T, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) step3d_kernel(StepArgs a, int TZ) {
    typedef Step3dShape<MODEL, ST, T, TX, TY, NT> Sh;
    typedef typename Sh::C C;
    constexpr int r = Sh::r, RIN = Sh::RIN, WIN = Sh::WIN, AIN = Sh::AIN, DIN = Sh::DIN, NF = Sh::NF;
    constexpr int WMU = Sh::WMU, AMU = Sh::AMU, DMU = Sh::DMU, EPT = Sh::EPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s_in = reinterpret_cast<C *>(smem_raw);            // [NF][DIN][AIN]
    C *s_mu = s_in + (size_t)NF * DIN * AIN;               // [DMU][AMU]

    const ConstsC<C> k(a.k);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * TZ;
    const int z1 = min(z0 + TZ, nz);
    if (z0 >= z1) return;
    const int nplanes = (z1 - z0) + 2 * RIN;
    const size_t plane = (size_t)nx * (size_t)ny;
    const T *in[2] = {static_cast<const T *>(a.in0), static_cast<const T *>(a.in1)};
    T *out[2] = {static_cast<T *>(a.out0), static_cast<T *>(a.out1)};

    // per-thread load offsets within a plane (independent of z)
    int loff[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int c = t + e * NT;
        if (c < AIN) {
            const int yi = c / WIN, xi = c - yi * WIN;
            const int y = wrap_idx(y0 - RIN + yi, ny), x = wrap_idx(x0 - RIN + xi, nx);
            loff[e] = y * nx + x;
        } else {
            loff[e] = -1;
        }
    }
    C pf[NF][EPT];
    auto fetch = [&](int z) {
        const size_t zoff = (size_t)wrap_idx(z, nz) * plane;
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int e = 0; e < EPT; ++e)
                if (loff[e] >= 0) pf[f][e] = load_one(in[f] + zoff + loff[e]);
    };
    auto commit = [&](int slot) {
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int e = 0; e < EPT; ++e)
                if (loff[e] >= 0) s_in[((size_t)f * DIN + slot) * AIN + t + e * NT] = pf[f][e];
    };
    auto S_in = [&](int f, int slot) -> const C * { return s_in + ((size_t)f * DIN + slot) * AIN; };

    fetch(z0 - RIN);
    for (int j = 0; j < nplanes; ++j) {
        commit(j % DIN);
        if (j + 1 < nplanes) fetch(z0 - RIN + j + 1);
        __syncthreads();
        if constexpr (MODEL == CH) {
            if (j >= 2 * r) {
                // mu of plane z0 - r + (j - 2r) over the (TY+2r) x (TX+2r) region
                const int jm = j - 2 * r;
                C *mu = s_mu + (size_t)(jm % DMU) * AMU;
                for (int c = t; c < AMU; c += NT) {
                    const int ym = c / WMU, xm = c - ym * WMU;
                    const int base = (ym + r) * WIN + (xm + r);
                    auto P = [&](int dx, int dy, int dz) -> C {
                        return S_in(0, (j - r + dz) % DIN)[base + dy * WIN + dx];
                    };
                    const C S = stencil_sum<ST, C>(P);
                    mu[c] = ch_mu<C>(S_in(0, (j - r) % DIN)[base], S, k);
                }
            }
            __syncthreads();
            if (j >= 4 * r) {
                const int zo = z0 + j - 4 * r;
                T *dst = out[0] + (size_t)zo * plane;
                for (int c = t; c < TX * TY; c += NT) {
                    const int yy = c / TX, xx = c - yy * TX;
                    const int x = x0 + xx, y = y0 + yy;
                    if (x >= nx || y >= ny) continue;
                    const int mb = (yy + r) * WMU + (xx + r);
                    auto Pm = [&](int dx, int dy, int dz) -> C {
                        return s_mu[(size_t)((j - 3 * r + dz) % DMU) * AMU + mb + dy * WMU + dx];
                    };
                    const C Smu = stencil_sum<ST, C>(Pm);
                    const C p = S_in(0, (j - 2 * r) % DIN)[(yy + RIN) * WIN + xx + RIN];
                    dst[(size_t)y * nx + x] = from_c<T>(ch_update<C>(p, Smu, k));
                }
            }
        } else {
            if (j >= 2 * r) {
                const int zo = z0 + j - 2 * r;
                for (int c = t; c < TX * TY; c += NT) {
                    const int yy = c / TX, xx = c - yy * TX;
                    const int x = x0 + xx, y = y0 + yy;
                    if (x >= nx || y >= ny) continue;
                    const int b = (yy + RIN) * WIN + xx + RIN;
                    const size_t o = (size_t)zo * plane + (size_t)y * nx + x;
                    auto P0 = [&](int dx, int dy, int dz) -> C {
                        return S_in(0, (j - r + dz) % DIN)[b + dy * WIN + dx];
                    };
                    const C S0 = stencil_sum<ST, C>(P0);
                    const C p0 = S_in(0, (j - r) % DIN)[b];
                    if constexpr (MODEL == AC) {
                        out[0][o] = from_c<T>(ac_update<C>(p0, S0, k));
                    } else {
                        auto P1 = [&](int dx, int dy, int dz) -> C {
                            return S_in(NF - 1, (j - r + dz) % DIN)[b + dy * WIN + dx];
                        };
                        const C S1 = stencil_sum<ST, C>(P1);
                        const C p1 = S_in(NF - 1, (j - r) % DIN)[b];
                        C un, vn;
                        gs_update<C>(p0, p1, S0, S1, k, un, vn);
                        out[0][o] = from_c<T>(un);
                        out[NF - 1][o] = from_c<T>(vn);
                    }
                }
            }
        }
    }
}

}  // namespace sp

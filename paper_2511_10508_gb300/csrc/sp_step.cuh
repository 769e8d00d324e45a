// sp_step.cuh -- fused explicit time-step kernels (one forward-Euler step per
// launch, or K steps for the temporally blocked 2D tiles) for Allen-Cahn,
// Cahn-Hilliard, Gray-Scott and Model C on periodic grids.
//
// One pass per step (the paper, Sec. "Benchmarks", stores phi^3 in a temporary
// field for conserved dynamics; here the chemical potential never leaves the
// chip).  Every kernel streams along the slowest axis (rows in 2D, z-planes in
// 3D) and keeps the slices it still needs on chip, so HBM traffic per point and
// step is one read and one write of each field:
//   step2d_batch_kernel  2D, FP64: shared-memory rings, batches of rows
//   step2d_tile_kernel   2D: one CTA per tile, tile + halo fetched with cp.async
//                        (FP64 small grids, FP32/BF16 alternative family, serving)
//   step2d_tb_kernel     2D: K steps per launch on a tile grown by the K-step halo
//   step2d_warp_kernel   2D, FP32/BF16: one warp per column strip, rows in registers
//   step3d_kernel        3D, FP64: shared-memory plane rings
//   step3d_zreg_kernel   3D, FP64, 27-point: z-streaming with register queues
//   step3d_wr_kernel     3D, FP32/BF16: warp per tile row, z in register queues
//   step3d_tbs_kernel    3D, FP32/BF16 Allen-Cahn / Gray-Scott / Model C: 2 steps
//                        per pass (Model C also 1), warp rows, a plane ring per level
//   step3d_async_kernel  3D, FP32/BF16: cp.async plane ring, planes in flight
//   step3d_vec_kernel    3D, FP32/BF16: plane rings of 16-byte chunks (any nx)
//   step3d_box_kernel    3D, FP32/BF16 Model C: one CTA per box
#pragma once

#include "sp_common.cuh"

namespace sp {

// ========================================================== 2D, batched ==
//
// Shared-memory ring kernel used for FP64 (bound by the FP64 pipe, so every
// wasted FP64 lane counts).  CTA: NT threads; strip of TW = 2*NT columns,
// thread t owns columns t and t+NT (consecutive threads, consecutive doubles:
// no bank conflicts).  Rows are processed in batches of RB: a batch loads RB
// new rows, computes RB new rows of mu (Cahn-Hilliard) as one flat work list
// over all threads, then RB output rows.  Rows of mu and phi needed by the
// next batch stay in the rings.  The grid is persistent: CTA c processes the
// rows [c*R, (c+1)*R) of the flattened (strip, row) space, so every CTA has the
// same work; a range that crosses a strip boundary is processed as two
// segments.
template <int MODEL, int ST, typename T, int NT, int RB>
struct Step2dBatchShape {
    typedef typename Cmp<T>::type C;
    static constexpr int r = StencilInfo<ST>::r;
    static constexpr int RIN = (MODEL == CH) ? 2 * r : r;
    static constexpr int TW = 2 * NT;
    static constexpr int WIN = TW + 2 * RIN;
    // phi ring: a batch uses RB + 2r rows (CH: rows [yb, yb+RB+2r); AC/GS:
    // [yb-r, yb+RB+r)); the next batch's RB rows are committed while slow threads
    // may still read this batch's rows, which stays collision-free when the ring
    // has 2*RB + 2r slots (row differences lie in [1, 2RB+2r-1]).
    static constexpr int DIN = 2 * RB + 2 * r;
    static constexpr int NF = num_fields<MODEL>();
    // Model C: the density's chemical potential of every committed point, kept
    // in the ring as one more field (evaluated once per point, not per tap)
    static constexpr int NRING = NF + (MODEL == MC ? 1 : 0);
    // mu ring: a batch reads mu rows [yb-r, yb+RB+r); the next batch's rows are
    // written only after a barrier that follows this batch's output.
    static constexpr int WMU = (MODEL == CH) ? TW + 2 * r : 0;
    static constexpr int DMU = (MODEL == CH) ? RB + 2 * r : 0;
    static constexpr size_t smem_bytes = sizeof(C) * ((size_t)NRING * DIN * WIN + (size_t)DMU * WMU);
};

template <int MODEL, int ST, typename T, int NT, int RB>
__global__ void __launch_bounds__(NT) step2d_batch_kernel(StepArgs a, int strips, long long rows_per_cta) {
    typedef Step2dBatchShape<MODEL, ST, T, NT, RB> Sh;
    typedef typename Sh::C C;
    constexpr int r = Sh::r, RIN = Sh::RIN, TW = Sh::TW, WIN = Sh::WIN, DIN = Sh::DIN, NF = Sh::NF;
    constexpr int WMU = Sh::WMU, DMU = Sh::DMU;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C (*s_in)[DIN][WIN] = reinterpret_cast<C (*)[DIN][WIN]>(smem_raw);                  // [NRING][DIN][WIN]
    C (*s_mu)[WMU > 0 ? WMU : 1] =
        reinterpret_cast<C (*)[WMU > 0 ? WMU : 1]>(smem_raw + sizeof(C) * (size_t)Sh::NRING * DIN * WIN);  // [DMU][WMU]

    const ConstsC<C> k(a.k, a.kf);
    const int nx = a.nx, ny = a.ny;
    const int t = threadIdx.x;
    const T *in[2] = {static_cast<const T *>(a.in0), static_cast<const T *>(a.in1)};
    T *out[2] = {static_cast<T *>(a.out0), static_cast<T *>(a.out1)};

    long long g0 = (long long)blockIdx.x * rows_per_cta;
    const long long gend = min(g0 + rows_per_cta, (long long)strips * ny);
    while (g0 < gend) {
        const int strip = (int)(g0 / ny);
        const int y0 = (int)(g0 - (long long)strip * ny);
        const int y1 = (int)min((long long)ny, (long long)y0 + (gend - g0));
        g0 += y1 - y0;
        const int x0 = strip * TW;
        // columns of this thread (global, wrapped) and the halo column it loads
        const int xa = wrap_idx(x0 + t, nx), xb = wrap_idx(x0 + t + NT, nx);
        const bool has_halo = t < 2 * RIN;
        const int hxi = (t < RIN) ? t : TW + t;
        const int hx = wrap_idx(x0 - RIN + hxi, nx);

        // ring slot of global row y (rows relative to y0 - RIN, always >= 0)
        auto slot_in = [&](int y) { return (y - y0 + RIN) % DIN; };
        auto slot_mu = [&](int y) { return (y - y0 + r) % DMU; };

        C pa[NF][RB], pb[NF][RB], ph[NF][RB];
        // fetch `n` rows starting at global row y (wrapped) into registers
        auto fetch = [&](int y, int n) {
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                if (i < n) {
                    const size_t row = (size_t)wrap_idx(y + i, ny) * (size_t)nx;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        pa[f][i] = load_one(in[f] + row + xa);
                        pb[f][i] = load_one(in[f] + row + xb);
                        if (has_halo) ph[f][i] = load_one(in[f] + row + hx);
                    }
                }
            }
        };
        auto commit = [&](int y, int n) {
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                if (i < n) {
                    const int sl = slot_in(y + i);
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        s_in[f][sl][RIN + t] = pa[f][i];
                        s_in[f][sl][RIN + t + NT] = pb[f][i];
                        if (has_halo) s_in[f][sl][hxi] = ph[f][i];
                    }
                    if constexpr (MODEL == MC) {
                        s_in[NF][sl][RIN + t] = mc_mu<C>(pa[0][i], pa[1][i], k);
                        s_in[NF][sl][RIN + t + NT] = mc_mu<C>(pb[0][i], pb[1][i], k);
                        if (has_halo) s_in[NF][sl][hxi] = mc_mu<C>(ph[0][i], ph[1][i], k);
                    }
                }
            }
        };
        // mu rows [ya, ya + n) as one flat work list
        auto compute_mu = [&](int ya, int n) {
            if constexpr (MODEL == CH) {
                const int items = n * WMU;
                for (int q = t; q < items; q += NT) {
                    const int i = q / WMU, c = q - i * WMU;
                    const int y = ya + i;
                    auto P = [&](int dx, int dy, int) -> C { return s_in[0][slot_in(y + dy)][c + r + dx]; };
                    const C S = stencil_sum<ST, C>(P);
                    s_mu[slot_mu(y)][c] = ch_mu<C>(s_in[0][slot_in(y)][c + r], S, k);
                }
            }
        };
        auto output = [&](int ya, int n) {
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                if (i < n) {
                    const int y = ya + i;
                    const size_t row = (size_t)y * (size_t)nx;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int c = t + h * NT;  // column within the strip
                        const int x = x0 + c;
                        C o0, o1 = C(0);
                        if constexpr (MODEL == CH) {
                            auto Pm = [&](int dx, int dy, int) -> C { return s_mu[slot_mu(y + dy)][c + r + dx]; };
                            o0 = ch_update<C>(s_in[0][slot_in(y)][c + RIN], stencil_sum<ST, C>(Pm), k);
                        } else {
                            auto P0 = [&](int dx, int dy, int) -> C { return s_in[0][slot_in(y + dy)][c + RIN + dx]; };
                            const C S0 = stencil_sum<ST, C>(P0);
                            const C p0 = s_in[0][slot_in(y)][c + RIN];
                            if constexpr (MODEL == AC) {
                                o0 = ac_update<C>(p0, S0, k);
                            } else {
                                auto P1 = [&](int dx, int dy, int) -> C {
                                    return s_in[NF - 1][slot_in(y + dy)][c + RIN + dx];
                                };
                                C S1;
                                if constexpr (MODEL == MC) {
                                    auto Pr = [&](int dx, int dy, int) -> C {
                                        return s_in[NF][slot_in(y + dy)][c + RIN + dx];
                                    };
                                    S1 = stencil_sum<ST, C>(Pr);  // = second_sum, mu_rho read, not re-evaluated
                                } else {
                                    S1 = second_sum<MODEL, ST, C>(P0, P1, k);
                                }
                                two_field_update<MODEL, C>(p0, s_in[NF - 1][slot_in(y)][c + RIN], S0, S1, k, o0, o1);
                            }
                        }
                        if (x < nx) {
                            out[0][row + x] = from_c<T>(o0);
                            if constexpr (num_fields<MODEL>() == 2) out[1][row + x] = from_c<T>(o1);
                        }
                    }
                }
            }
        };

        // prologue: rows [y0 - RIN, y0 + RIN - ...) that precede the first batch
        constexpr int PRO = (MODEL == CH) ? 4 * r : 2 * r;  // phi rows before the first batch's new rows
        {
            int y = y0 - RIN;
            for (int left = PRO; left > 0; left -= RB) {
                const int n = left < RB ? left : RB;
                fetch(y, n);
                commit(y, n);
                y += n;
            }
        }
        __syncthreads();
        if constexpr (MODEL == CH) {
            compute_mu(y0 - r, 2 * r);  // mu rows carried into the first batch
        }
        // first batch's new rows
        int ynew = y0 - RIN + PRO;   // = y0 + RIN (CH: y0 + 2r; AC/GS: y0 + r)
        int nb = min(RB, y1 - y0);
        fetch(ynew, nb);
        for (int yb = y0; yb < y1; yb += RB) {
            const int n = min(RB, y1 - yb);
            commit(ynew, n);
            ynew += n;
            const int nn = min(RB, y1 - (yb + RB));
            if (nn > 0) fetch(ynew, nn);
            __syncthreads();
            if constexpr (MODEL == CH) {
                compute_mu(yb + r, n);
                __syncthreads();
            }
            output(yb, n);
        }
        __syncthreads();  // the rings are reused by the next segment
    }
}

// ============================================================= 2D, tiles ==
//
// Tile kernel for FP32 and BF16 storage (bound by HBM), also the 2D work unit
// of the batched serving kernel.  One CTA per BX x BY output tile: the tile
// plus an R-wide halo (R = r, or 2r for Cahn-Hilliard) is fetched in one shot
// as 16-byte chunks with cp.async (rows padded to whole chunks: HC chunks of
// halo on each side), Cahn-Hilliard computes mu on the tile plus an r-wide
// ring, then every point of the tile is updated.  Many small CTAs are
// resident per SM, so the loads of one CTA overlap the arithmetic of the
// others; halo reads of neighbouring tiles hit L2.
template <int MODEL, int ST, typename T, int BX, int BY>
struct Step2dTileShape {
    typedef typename Cmp<T>::type C;
    static constexpr int r = StencilInfo<ST>::r;
    static constexpr int R = (MODEL == CH) ? 2 * r : r;
    static constexpr int CK = 16 / sizeof(T);          // elements per 16-byte chunk
    static constexpr int HC = (R + CK - 1) / CK;       // halo chunks on each side
    static constexpr int NCK = BX / CK + 2 * HC;       // chunks per row
    static constexpr int SW = NCK * CK;                // row stride (elements of T)
    static constexpr int X0 = HC * CK;                 // smem column of the tile's first column
    static constexpr int HIN = BY + 2 * R;             // rows
    static constexpr int NF = num_fields<MODEL>();
    static constexpr int WMU = (MODEL == CH) ? BX + 2 * r : 0, HMU = (MODEL == CH) ? BY + 2 * r : 0;
    static constexpr size_t bytes_in = sizeof(T) * (size_t)NF * HIN * SW;
    static constexpr size_t smem_bytes = bytes_in + sizeof(C) * (size_t)WMU * HMU;
};

// One BX x BY tile with origin (x0, y0) of one grid; smem as in Step2dTileShape.
template <int MODEL, int ST, typename T, int BX, int BY, int NT>
__device__ __forceinline__ void tile2d(const T *in0, const T *in1, T *out0, T *out1, int nx, int ny,
                                       const ConstsC<typename Cmp<T>::type> &k, int x0, int y0,
                                       unsigned char *smem_raw) {
    typedef Step2dTileShape<MODEL, ST, T, BX, BY> Sh;
    typedef typename Sh::C C;
    constexpr int r = Sh::r, R = Sh::R, CK = Sh::CK, NCK = Sh::NCK, SW = Sh::SW, X0 = Sh::X0, HIN = Sh::HIN;
    constexpr int NF = Sh::NF, WMU = Sh::WMU, HMU = Sh::HMU;
    T *s_in = reinterpret_cast<T *>(smem_raw);                   // [NF][HIN][SW]
    C *s_mu = reinterpret_cast<C *>(smem_raw + Sh::bytes_in);    // [HMU][WMU]
    const int t = threadIdx.x;
    const bool vec_ok = (nx % CK) == 0;
    const T *in[2] = {in0, in1};
    T *out[2] = {out0, out1};

    // fetch: chunk c of row i covers columns x0 - X0 + c*CK .. +CK-1
    for (int q = t; q < HIN * NCK; q += NT) {
        const int i = q / NCK, c = q - i * NCK;
        const int y = wrap_idx(y0 - R + i, ny);
        const int x = x0 - X0 + c * CK;
        const size_t row = (size_t)y * (size_t)nx;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T *dst = s_in + ((size_t)f * HIN + i) * SW + c * CK;
            if (vec_ok && x >= 0 && x + CK <= nx) {
                cp_async16(dst, in[f] + row + x);
            } else {
#pragma unroll
                for (int j = 0; j < CK; ++j) dst[j] = in[f][row + wrap_idx(x + j, nx)];
            }
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();

    auto phi = [&](int f, int i, int j) -> C { return to_c(s_in[((size_t)f * HIN + i) * SW + j]); };
    if constexpr (MODEL == CH) {
        // mu at (y0 - r + i, x0 - r + j), i < HMU, j < WMU
        for (int q = t; q < HMU * WMU; q += NT) {
            const int i = q / WMU, j = q - i * WMU;
            const int ii = i + (R - r), jj = j + (X0 - r);
            auto P = [&](int dx, int dy, int) -> C { return phi(0, ii + dy, jj + dx); };
            s_mu[q] = ch_mu<C>(phi(0, ii, jj), stencil_sum<ST, C>(P), k);
        }
        __syncthreads();
    }
    for (int q = t; q < BY * BX; q += NT) {
        const int i = q / BX, j = q - i * BX;
        const int y = y0 + i, x = x0 + j;
        if (y >= ny || x >= nx) continue;
        const size_t o = (size_t)y * (size_t)nx + x;
        if constexpr (MODEL == CH) {
            auto Pm = [&](int dx, int dy, int) -> C { return s_mu[(i + r + dy) * WMU + (j + r + dx)]; };
            out[0][o] = from_c<T>(ch_update<C>(phi(0, i + R, j + X0), stencil_sum<ST, C>(Pm), k));
        } else {
            auto P0 = [&](int dx, int dy, int) -> C { return phi(0, i + R + dy, j + X0 + dx); };
            const C S0 = stencil_sum<ST, C>(P0);
            if constexpr (MODEL == AC) {
                out[0][o] = from_c<T>(ac_update<C>(phi(0, i + R, j + X0), S0, k));
            } else {
                auto P1 = [&](int dx, int dy, int) -> C { return phi(NF - 1, i + R + dy, j + X0 + dx); };
                C un, vn;
                two_field_update<MODEL, C>(phi(0, i + R, j + X0), phi(NF - 1, i + R, j + X0), S0,
                                           second_sum<MODEL, ST, C>(P0, P1, k), k, un, vn);
                out[0][o] = from_c<T>(un);
                out[NF - 1][o] = from_c<T>(vn);
            }
        }
    }
}

template <int MODEL, int ST, typename T, int BX, int BY, int NT>
__global__ void __launch_bounds__(NT) step2d_tile_kernel(StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_enter();
    const ConstsC<typename Cmp<T>::type> k(a.k, a.kf);
    tile2d<MODEL, ST, T, BX, BY, NT>(static_cast<const T *>(a.in0), static_cast<const T *>(a.in1),
                                     static_cast<T *>(a.out0), static_cast<T *>(a.out1), a.nx, a.ny, k,
                                     blockIdx.x * BX, blockIdx.y * BY, smem_raw);
}

// ================================================== 2D, temporal blocking ==
//
// K time steps per launch on one BX x BY tile (FP32 / BF16 storage): the tile
// plus a K*R halo is fetched once (cp.async, rows padded to whole 16-byte
// chunks), then step s = 0 .. K-1 updates the tile grown by the margin
// m_s = R*(K-1-s) from one shared-memory buffer into the other; each step's
// region is one halo width smaller than the region it reads, so every value it
// uses was produced by the previous step (or loaded).  Intermediate values are
// kept in the storage type, rounded exactly as a global store would round
// them, so K blocked steps equal K single steps bit for bit.  Only the last
// step writes to global memory: HBM traffic per point is one read and one
// write per K steps.
template <int MODEL, int ST, typename T, int BX, int BY, int K>
struct Step2dTbShape {
    typedef typename Cmp<T>::type C;
    static constexpr int r = StencilInfo<ST>::r;
    static constexpr int R = (MODEL == CH) ? 2 * r : r;
    static constexpr int KR = K * R;                    // loaded halo
    static constexpr int CK = 16 / sizeof(T);
    static constexpr int HC = (KR + CK - 1) / CK;
    static constexpr int NCK = BX / CK + 2 * HC;
    static constexpr int SW = NCK * CK, X0 = HC * CK;
    static constexpr int HIN = BY + 2 * KR;
    static constexpr int NF = num_fields<MODEL>();
    static constexpr int MMU = R * (K - 1) + r;         // widest mu margin
    static constexpr int WMU = (MODEL == CH) ? BX + 2 * MMU : 0, HMU = (MODEL == CH) ? BY + 2 * MMU : 0;
    static constexpr size_t buf_elems = (size_t)HIN * SW;
    static constexpr size_t bytes_in = sizeof(T) * (size_t)2 * NF * buf_elems;  // two levels per field
    static constexpr size_t smem_bytes = bytes_in + sizeof(C) * (size_t)WMU * HMU;
};

template <int MODEL, int ST, typename T, int BX, int BY, int K, int NT>
__global__ void __launch_bounds__(NT) step2d_tb_kernel(StepArgs a) {
    typedef Step2dTbShape<MODEL, ST, T, BX, BY, K> Sh;
    typedef typename Sh::C C;
    constexpr int r = Sh::r, R = Sh::R, KR = Sh::KR, CK = Sh::CK, NCK = Sh::NCK, SW = Sh::SW, X0 = Sh::X0;
    constexpr int HIN = Sh::HIN, NF = Sh::NF, WMU = Sh::WMU;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf = reinterpret_cast<T *>(smem_raw);                  // [2 levels][NF][HIN][SW]
    C *s_mu = reinterpret_cast<C *>(smem_raw + Sh::bytes_in);  // [HMU][WMU]
    pdl_enter();
    const ConstsC<C> k(a.k, a.kf);
    const int nx = a.nx, ny = a.ny;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const bool vec_ok = (nx % CK) == 0;
    const T *in[2] = {static_cast<const T *>(a.in0), static_cast<const T *>(a.in1)};
    T *out[2] = {static_cast<T *>(a.out0), static_cast<T *>(a.out1)};
    // element (i, j) of the tile frame (i in [-KR, BY+KR), j in [-X0, BX+X0)) of field f, level l
    auto at = [&](int l, int f, int i, int j) -> T & {
        return buf[((size_t)(l * NF + f) * HIN + (i + KR)) * SW + (j + X0)];
    };

    for (int q = t; q < HIN * NCK; q += NT) {
        const int i = q / NCK, c = q - i * NCK;
        const int y = wrap_idx(y0 - KR + i, ny);
        const int x = x0 - X0 + c * CK;
        const size_t row = (size_t)y * (size_t)nx;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T *dst = buf + ((size_t)f * HIN + i) * SW + c * CK;
            if (vec_ok && x >= 0 && x + CK <= nx) {
                cp_async16(dst, in[f] + row + x);
            } else {
#pragma unroll
                for (int j = 0; j < CK; ++j) dst[j] = in[f][row + wrap_idx(x + j, nx)];
            }
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();

#pragma unroll
    for (int s = 0; s < K; ++s) {
        const int src = s & 1, dst = src ^ 1;
        const int m = R * (K - 1 - s);  // margin of this step's output region
        if constexpr (MODEL == CH) {
            // mu on the region grown by m + r
            const int mm = m + r, W = BX + 2 * mm, H = BY + 2 * mm;
            for (int q = t; q < H * W; q += NT) {
                const int i = q / W - mm, j = q % W - mm;
                auto P = [&](int dx, int dy, int) -> C { return to_c(at(src, 0, i + dy, j + dx)); };
                s_mu[(i + Sh::MMU) * WMU + (j + Sh::MMU)] = ch_mu<C>(to_c(at(src, 0, i, j)), stencil_sum<ST, C>(P), k);
            }
            __syncthreads();
        }
        const int W = BX + 2 * m, H = BY + 2 * m;
        for (int q = t; q < H * W; q += NT) {
            const int i = q / W - m, j = q % W - m;
            C o0, o1 = C(0);
            if constexpr (MODEL == CH) {
                auto Pm = [&](int dx, int dy, int) -> C {
                    return s_mu[(i + dy + Sh::MMU) * WMU + (j + dx + Sh::MMU)];
                };
                o0 = ch_update<C>(to_c(at(src, 0, i, j)), stencil_sum<ST, C>(Pm), k);
            } else {
                auto P0 = [&](int dx, int dy, int) -> C { return to_c(at(src, 0, i + dy, j + dx)); };
                const C S0 = stencil_sum<ST, C>(P0);
                if constexpr (MODEL == AC) {
                    o0 = ac_update<C>(to_c(at(src, 0, i, j)), S0, k);
                } else {
                    auto P1 = [&](int dx, int dy, int) -> C { return to_c(at(src, NF - 1, i + dy, j + dx)); };
                    two_field_update<MODEL, C>(to_c(at(src, 0, i, j)), to_c(at(src, NF - 1, i, j)), S0,
                                               second_sum<MODEL, ST, C>(P0, P1, k), k, o0, o1);
                }
            }
            if (s + 1 < K) {
                at(dst, 0, i, j) = from_c<T>(o0);
                if constexpr (num_fields<MODEL>() == 2) at(dst, 1, i, j) = from_c<T>(o1);
            } else {
                const int y = y0 + i, x = x0 + j;
                if (y < ny && x < nx) {
                    const size_t o = (size_t)y * (size_t)nx + x;
                    out[0][o] = from_c<T>(o0);
                    if constexpr (num_fields<MODEL>() == 2) out[1][o] = from_c<T>(o1);
                }
            }
        }
        if (s + 1 < K) __syncthreads();
    }
}

// ============================================================== 3D, boxes ==
//
// 3D work unit of the batched serving kernel: one BX x BY x BZ box per CTA,
// fetched with its R-wide halo in one shot (x padded to whole 16-byte chunks),
// mu of Cahn-Hilliard on the box plus an r-wide shell, then the update.  Used
// for the small 3D grids of the serving mix, where one box is a sizeable part
// of a grid; large single grids use the plane-streaming kernels below.
template <int MODEL, int ST, typename T, int BX, int BY, int BZ>
struct Step3dBoxShape {
    typedef typename Cmp<T>::type C;
    static constexpr int r = StencilInfo<ST>::r;
    static constexpr int R = (MODEL == CH) ? 2 * r : r;
    static constexpr int CK = 16 / sizeof(T);
    static constexpr int HC = (R + CK - 1) / CK;
    static constexpr int NCK = BX / CK + 2 * HC;
    static constexpr int SW = NCK * CK, X0 = HC * CK;
    static constexpr int HIN = BY + 2 * R, DIN = BZ + 2 * R;
    static constexpr int NF = num_fields<MODEL>();
    static constexpr int WMU = (MODEL == CH) ? BX + 2 * r : 0, HMU = (MODEL == CH) ? BY + 2 * r : 0,
                         DMU = (MODEL == CH) ? BZ + 2 * r : 0;
    static constexpr size_t bytes_in = sizeof(T) * (size_t)NF * DIN * HIN * SW;
    static constexpr size_t smem_bytes = bytes_in + sizeof(C) * (size_t)WMU * HMU * DMU;
};

template <int MODEL, int ST, typename T, int BX, int BY, int BZ, int NT>
__device__ __forceinline__ void box3d(const T *in0, const T *in1, T *out0, T *out1, int nx, int ny, int nz,
                                      const ConstsC<typename Cmp<T>::type> &k, int x0, int y0, int z0,
                                      unsigned char *smem_raw) {
    typedef Step3dBoxShape<MODEL, ST, T, BX, BY, BZ> Sh;
    typedef typename Sh::C C;
    constexpr int r = Sh::r, R = Sh::R, CK = Sh::CK, NCK = Sh::NCK, SW = Sh::SW, X0 = Sh::X0;
    constexpr int HIN = Sh::HIN, DIN = Sh::DIN, NF = Sh::NF, WMU = Sh::WMU, HMU = Sh::HMU, DMU = Sh::DMU;
    T *s_in = reinterpret_cast<T *>(smem_raw);                   // [NF][DIN][HIN][SW]
    C *s_mu = reinterpret_cast<C *>(smem_raw + Sh::bytes_in);    // [DMU][HMU][WMU]
    const int t = threadIdx.x;
    const bool vec_ok = (nx % CK) == 0;
    const size_t plane = (size_t)nx * (size_t)ny;
    const T *in[2] = {in0, in1};
    T *out[2] = {out0, out1};

    for (int q = t; q < DIN * HIN * NCK; q += NT) {
        const int zi = q / (HIN * NCK), rem = q - zi * (HIN * NCK);
        const int i = rem / NCK, c = rem - i * NCK;
        const int z = wrap_idx(z0 - R + zi, nz), y = wrap_idx(y0 - R + i, ny);
        const int x = x0 - X0 + c * CK;
        const size_t row = (size_t)z * plane + (size_t)y * (size_t)nx;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T *dst = s_in + (((size_t)f * DIN + zi) * HIN + i) * SW + c * CK;
            if (vec_ok && x >= 0 && x + CK <= nx) {
                cp_async16(dst, in[f] + row + x);
            } else {
#pragma unroll
                for (int j = 0; j < CK; ++j) dst[j] = in[f][row + wrap_idx(x + j, nx)];
            }
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();

    auto phi = [&](int f, int zi, int i, int j) -> C {
        return to_c(s_in[(((size_t)f * DIN + zi) * HIN + i) * SW + j]);
    };
    if constexpr (MODEL == CH) {
        for (int q = t; q < DMU * HMU * WMU; q += NT) {
            const int zm = q / (HMU * WMU), rem = q - zm * (HMU * WMU);
            const int i = rem / WMU, j = rem - i * WMU;
            const int zz = zm + (R - r), ii = i + (R - r), jj = j + (X0 - r);
            auto P = [&](int dx, int dy, int dz) -> C { return phi(0, zz + dz, ii + dy, jj + dx); };
            s_mu[q] = ch_mu<C>(phi(0, zz, ii, jj), stencil_sum<ST, C>(P), k);
        }
        __syncthreads();
    }
    for (int q = t; q < BZ * BY * BX; q += NT) {
        const int zb = q / (BY * BX), rem = q - zb * (BY * BX);
        const int i = rem / BX, j = rem - i * BX;
        const int z = z0 + zb, y = y0 + i, x = x0 + j;
        if (z >= nz || y >= ny || x >= nx) continue;
        const size_t o = (size_t)z * plane + (size_t)y * (size_t)nx + x;
        if constexpr (MODEL == CH) {
            auto Pm = [&](int dx, int dy, int dz) -> C {
                return s_mu[((zb + r + dz) * HMU + (i + r + dy)) * WMU + (j + r + dx)];
            };
            out[0][o] = from_c<T>(ch_update<C>(phi(0, zb + R, i + R, j + X0), stencil_sum<ST, C>(Pm), k));
        } else {
            auto P0 = [&](int dx, int dy, int dz) -> C { return phi(0, zb + R + dz, i + R + dy, j + X0 + dx); };
            const C S0 = stencil_sum<ST, C>(P0);
            if constexpr (MODEL == AC) {
                out[0][o] = from_c<T>(ac_update<C>(phi(0, zb + R, i + R, j + X0), S0, k));
            } else {
                auto P1 = [&](int dx, int dy, int dz) -> C {
                    return phi(NF - 1, zb + R + dz, i + R + dy, j + X0 + dx);
                };
                C un, vn;
                two_field_update<MODEL, C>(phi(0, zb + R, i + R, j + X0), phi(NF - 1, zb + R, i + R, j + X0), S0,
                                           second_sum<MODEL, ST, C>(P0, P1, k), k, un, vn);
                out[0][o] = from_c<T>(un);
                out[NF - 1][o] = from_c<T>(vn);
            }
        }
    }
}

// One CTA per BX x BY x BZ box of a single grid (Model C, FP32 / BF16 3D).
template <int MODEL, int ST, typename T, int BX, int BY, int BZ, int NT>
__global__ void __launch_bounds__(NT) step3d_box_kernel(StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const ConstsC<typename Cmp<T>::type> k(a.k, a.kf);
    box3d<MODEL, ST, T, BX, BY, BZ, NT>(static_cast<const T *>(a.in0), static_cast<const T *>(a.in1),
                                        static_cast<T *>(a.out0), static_cast<T *>(a.out1), a.nx, a.ny, a.nz, k,
                                        blockIdx.x * BX, blockIdx.y * BY, blockIdx.z * BZ, smem_raw);
}

// ===================================================== 2D, warp rows ==
//
// FP32 / BF16-storage 2D kernel without shared memory or barriers.  A warp
// owns a strip of 32 x V columns (V = one 16-byte vector per lane) and streams
// down the rows of a segment.  Lanes 0 and 31 only supply halo columns; lanes
// 1..30 produce the 30 x V output columns of the strip.  The x neighbours of a
// lane's vector come from the adjacent lanes by warp shuffles, the y
// neighbours from a register window of the last 2r+1 rows (phi, and mu for
// Cahn-Hilliard).  The row loop is unrolled by the window length so that the
// window rotates by renaming registers.  Rows arrive through a per-warp ring of
// D rows in shared memory filled by cp.async (each lane copies and later reads
// only its own 16 bytes, so no barrier is needed), keeping D-1 rows of loads in
// flight per warp.  Same expressions in the same order as the other FP32
// kernels, so results are identical to them bit for bit.
//
// Requirements (checked by the launcher): nx a multiple of V and 16-byte
// aligned field pointers, so that every vector, wrapped or not, is aligned.
template <int MODEL, int ST, typename T>
struct Step2dWarpShape {
    typedef typename Cmp<T>::type C;
    static constexpr int r = StencilInfo<ST>::r;
    static constexpr int V = 16 / (int)sizeof(T);
    static constexpr int RIN = (MODEL == CH) ? 2 * r : r;
    static constexpr int NF = num_fields<MODEL>();
    static constexpr int U = 2 * r + 1;        // window rows = unroll = prefetch depth
    static constexpr int XW = V + 2 * r;       // a row of the window: own vector plus r halo each side
    static constexpr int OUT_COLS = 30 * V;    // output columns per strip
    static constexpr int D = (NF == 1 && sizeof(T) == 2) ? 12 : 8;  // rows in the per-warp load ring
    static constexpr size_t warp_smem = (size_t)D * NF * 32 * 16;
    static_assert(V >= 2 * r, "the halo lanes must cover the mu halo");
};

template <int MODEL, int ST, typename T, int NT>
__global__ void __launch_bounds__(NT) step2d_warp_kernel(StepArgs a, int strips, int groups, long long rows_per_cta) {
    typedef Step2dWarpShape<MODEL, ST, T> Sh;
    typedef typename Sh::C C;
    typedef uint4 W;
    constexpr int r = Sh::r, V = Sh::V, RIN = Sh::RIN, NF = Sh::NF, U = Sh::U, XW = Sh::XW, D = Sh::D;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    W *ring = reinterpret_cast<W *>(smem_raw) + (size_t)(threadIdx.x >> 5) * D * NF * 32;  // [D][NF][32]

    const ConstsC<C> k(a.k, a.kf);
    const ConstsF2 k2(k);
    const int nx = a.nx, ny = a.ny;
    const int lane = threadIdx.x & 31;
    // The warps of a CTA take adjacent strips (a group) over the same rows, so a
    // CTA reads contiguous spans of each row and the strips' overlapping halo
    // columns are shared through the caches.  CTAs own equal shares of the
    // flattened (group, row) space.
    const int wpc = blockDim.x >> 5, warp = threadIdx.x >> 5;
    const T *in[2] = {static_cast<const T *>(a.in0), static_cast<const T *>(a.in1)};
    T *out[2] = {static_cast<T *>(a.out0), static_cast<T *>(a.out1)};

    long long g0 = (long long)blockIdx.x * rows_per_cta;
    const long long gend = min(g0 + rows_per_cta, (long long)groups * ny);
    while (g0 < gend) {
        const int group = (int)(g0 / ny);
        const int y0 = (int)(g0 - (long long)group * ny);
        const int y1 = (int)min((long long)ny, (long long)y0 + (gend - g0));
        g0 += y1 - y0;
        const int strip = group * wpc + warp;
        if (strip >= strips) continue;
        const int col = strip * Sh::OUT_COLS + (lane - 1) * V;  // first column of this lane
        const int colw = wrap_idx(col, nx);
        const bool store = lane >= 1 && lane <= 30 && col < nx;
        const int jbeg = y0 - RIN;
        const int n = (y1 - y0) + 2 * RIN;

        // row i of the segment goes to ring slot i % D; one cp.async group per row
        auto issue = [&](int i) {
            if (i < n) {
                const size_t off = (size_t)wrap_idx(jbeg + i, ny) * nx + colw;
#pragma unroll
                for (int f = 0; f < NF; ++f) cp_async16(&ring[((i % D) * NF + f) * 32 + lane], in[f] + off);
            }
            cp_async_commit();  // empty groups keep the count uniform
        };
#pragma unroll
        for (int s = 0; s < D - 1; ++s) issue(s);

        C ph[NF][U][XW];
        C mu[MODEL == CH ? U : 1][XW];
        (void)mu;
        for (int i0 = 0; i0 < n; i0 += U) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u;
                if (i < n) {
                    const int j = jbeg + i;
                    // the slot read in the previous iteration is refilled; row i has landed
                    issue(i + D - 1);
                    cp_async_wait<D - 1>();
                    // unpack row j and extend it with the neighbouring lanes' edge values
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        union { W w; T t[V]; } raw;
                        raw.w = ring[((i % D) * NF + f) * 32 + lane];
                        C *row = ph[f][u];
#pragma unroll
                        for (int c = 0; c < V; ++c) row[r + c] = to_c(raw.t[c]);
#pragma unroll
                        for (int h = 0; h < r; ++h) {
                            row[h] = __shfl_up_sync(FULL, row[V + h], 1);
                            row[r + V + h] = __shfl_down_sync(FULL, row[r + h], 1);
                        }
                    }
                    // window slot of the row `m` iterations back
#define SLOT(m) ((u - (m) + 4 * U) % U)
                    if constexpr (MODEL == CH) {
                        if (i >= 2 * r) {
                            // mu of row j - r, two cells per instruction (packed pairs:
                            // BF16 0.68 -> 0.74 of HBM on 16384^2)
                            C *m = mu[u];
                            auto P = [&](int dx, int dy, int c) -> C { return ph[0][SLOT(r - dy)][r + c + dx]; };
#pragma unroll
                            for (int c = 0; c < V; c += 2) {
                                const float2 m2 = ch_mu2(make_float2(ph[0][SLOT(r)][r + c], ph[0][SLOT(r)][r + c + 1]),
                                                         stencil_sum2_2d<ST>(P, c), k2);
                                m[r + c] = m2.x;
                                m[r + c + 1] = m2.y;
                            }
#pragma unroll
                            for (int h = 0; h < r; ++h) {
                                m[h] = __shfl_up_sync(FULL, m[V + h], 1);
                                m[r + V + h] = __shfl_down_sync(FULL, m[r + h], 1);
                            }
                            if (i >= 4 * r) {
                                // output row j - 2r from mu rows j - 3r .. j - r
                                C o[V];
                                auto Pm = [&](int dx, int dy, int c) -> C { return mu[SLOT(r - dy)][r + c + dx]; };
#pragma unroll
                                for (int c = 0; c < V; c += 2) {
                                    const float2 o2 = ch_update2(
                                        make_float2(ph[0][SLOT(2 * r)][r + c], ph[0][SLOT(2 * r)][r + c + 1]),
                                        stencil_sum2_2d<ST>(Pm, c), k2);
                                    o[c] = o2.x;
                                    o[c + 1] = o2.y;
                                }
                                if (store) store_vec<T, V>(out[0] + (size_t)(j - 2 * r) * nx + col, o);
                            }
                        }
                    } else {
                        if (i >= 2 * r) {
                            // output row j - r
                            C o0[V], o1[V];
                            // (scalar: packed pairs measured slower for these models)
#pragma unroll
                            for (int c = 0; c < V; ++c) {
                                auto P0 = [&](int dx, int dy, int) -> C { return ph[0][SLOT(r - dy)][r + c + dx]; };
                                const C S0 = stencil_sum<ST, C>(P0);
                                const C p0 = ph[0][SLOT(r)][r + c];
                                if constexpr (MODEL == AC) {
                                    o0[c] = ac_update<C>(p0, S0, k);
                                } else {
                                    auto P1 = [&](int dx, int dy, int) -> C {
                                        return ph[NF - 1][SLOT(r - dy)][r + c + dx];
                                    };
                                    two_field_update<MODEL, C>(p0, ph[NF - 1][SLOT(r)][r + c], S0,
                                                               second_sum<MODEL, ST, C>(P0, P1, k), k, o0[c], o1[c]);
                                }
                            }
                            if (store) {
                                const size_t o = (size_t)(j - r) * nx + col;
                                store_vec<T, V>(out[0] + o, o0);
                                if constexpr (num_fields<MODEL>() == 2) store_vec<T, V>(out[NF - 1] + o, o1);
                            }
                        }
                    }
#undef SLOT
                }
            }
        }
        cp_async_wait<0>();  // the ring is reused by the next segment
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
    static constexpr int NF = num_fields<MODEL>();
    // Model C: the density's chemical potential of every loaded point, kept in
    // the ring as one more field (evaluated once per point, not per tap)
    static constexpr int NRING = NF + (MODEL == MC ? 1 : 0);
    static constexpr int WMU = TX + 2 * r, HMU = TY + 2 * r, AMU = WMU * HMU;
    static constexpr int DMU = (MODEL == CH) ? 2 * r + 1 : 0;
    static constexpr int EPT = (AIN + NT - 1) / NT;  // loaded cells per thread per field
    static constexpr size_t smem_bytes = sizeof(C) * ((size_t)NRING * DIN * AIN + (size_t)DMU * AMU);
};

template <int MODEL, int ST, typename T, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) step3d_kernel(StepArgs a, int tiles_x, int tiles_y, long long planes_per_cta) {
    typedef Step3dShape<MODEL, ST, T, TX, TY, NT> Sh;
    typedef typename Sh::C C;
    constexpr int r = Sh::r, RIN = Sh::RIN, WIN = Sh::WIN, AIN = Sh::AIN, DIN = Sh::DIN, NF = Sh::NF;
    constexpr int WMU = Sh::WMU, AMU = Sh::AMU, DMU = Sh::DMU, EPT = Sh::EPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s_in = reinterpret_cast<C *>(smem_raw);            // [NRING][DIN][AIN]
    C *s_mu = s_in + (size_t)Sh::NRING * DIN * AIN;        // [DMU][AMU]

    const ConstsC<C> k(a.k, a.kf);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int t = threadIdx.x;
    const size_t plane = (size_t)nx * (size_t)ny;
    const T *in[2] = {static_cast<const T *>(a.in0), static_cast<const T *>(a.in1)};
    T *out[2] = {static_cast<T *>(a.out0), static_cast<T *>(a.out1)};
    // Persistent schedule: CTA c owns planes [c*P, (c+1)*P) of the flattened
    // (tile, z) space, one segment per tile it touches.
    long long g0 = (long long)blockIdx.x * planes_per_cta;
    const long long gend = min(g0 + planes_per_cta, (long long)tiles_x * tiles_y * nz);
    while (g0 < gend) {
    const int tile = (int)(g0 / nz);
    const int z0 = (int)(g0 - (long long)tile * nz);
    const int z1 = (int)min((long long)nz, (long long)z0 + (gend - g0));
    g0 += z1 - z0;
    const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
    const int nplanes = (z1 - z0) + 2 * RIN;

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
        if constexpr (MODEL == MC) {
#pragma unroll
            for (int e = 0; e < EPT; ++e)
                if (loff[e] >= 0) s_in[((size_t)NF * DIN + slot) * AIN + t + e * NT] = mc_mu<C>(pf[0][e], pf[1][e], k);
        }
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
                        C S1;
                        if constexpr (MODEL == MC) {
                            auto Pr = [&](int dx, int dy, int dz) -> C {
                                return S_in(NF, (j - r + dz) % DIN)[b + dy * WIN + dx];
                            };
                            S1 = stencil_sum<ST, C>(Pr);  // = second_sum, mu_rho read, not re-evaluated
                        } else {
                            S1 = second_sum<MODEL, ST, C>(P0, P1, k);
                        }
                        const C p1 = S_in(NF - 1, (j - r) % DIN)[b];
                        C un, vn;
                        two_field_update<MODEL, C>(p0, p1, S0, S1, k, un, vn);
                        out[0][o] = from_c<T>(un);
                        out[NF - 1][o] = from_c<T>(vn);
                    }
                }
            }
        }
    }
    __syncthreads();  // the rings are reused by the next segment
    }  // segments
}

// ================================================= 3D, 27-point, FP64 ==
//
// The 27-point stencil's fixed order (see sp_common.cuh) is built from per-plane
// partial sums: the in-plane cross sum Cz and diagonal sum Dz of each of the
// three planes.  Each thread owns fixed (x, y) points of a TX x TY tile and
// streams along z, keeping the value, Cz and Dz of its points for the two
// previous planes in registers; a plane's partial sums are then computed once
// per point instead of once per use (14 instead of 26 FP64 operations per
// stencil application, with the same operations in the same order, so results
// are unchanged bit for bit).  Only the newest plane is read from shared
// memory, so the input needs two plane buffers and mu (Cahn-Hilliard) one.
//
// Cahn-Hilliard per input plane j (z = z0 - 2 + j): mu of plane j-1 over the
// tile plus one halo cell, then the output of plane j-2 from the mu partial
// sums of planes j-3 .. j-1.  Allen-Cahn / Gray-Scott: output of plane j-1.
// Barriers: after the commit of plane j, and (Cahn-Hilliard) after mu.
template <int MODEL, int TX, int TY, int NT>
struct Step3dZregShape {
    static constexpr int r = 1;
    static constexpr int RIN = (MODEL == CH) ? 2 : 1;
    static constexpr int WIN = TX + 2 * RIN, HIN = TY + 2 * RIN, AIN = WIN * HIN;
    static constexpr int NF = num_fields<MODEL>();
    static constexpr int WMU = TX + 2, HMU = TY + 2, AMU = (MODEL == CH) ? WMU * HMU : 0;
    static constexpr int EPT = (AIN + NT - 1) / NT;       // loaded cells per thread per field
    static constexpr int EMU = (AMU + NT - 1) / NT;       // mu points per thread
    static constexpr int EOUT = TX * TY / NT;             // output points per thread
    static_assert(TX * TY % NT == 0 && NT % TX == 0, "tile rows must map to whole threads");
    static constexpr size_t smem_bytes = sizeof(double) * ((size_t)2 * NF * AIN + (size_t)AMU);
};

// in-plane cross and diagonal sums of the 27-point stencil at p (row pitch W)
__device__ __forceinline__ void plane_sums27(const double *p, int W, double &Cz, double &Dz) {
    Cz = (p[-1] + p[1]) + (p[-W] + p[W]);
    Dz = (p[-W - 1] + p[-W + 1]) + (p[W - 1] + p[W + 1]);
}

// stencil sum from the centre value, its z neighbours and the three planes'
// partial sums (m = z-1, 0 = z, p = z+1)
__device__ __forceinline__ double combine27(double fm, double f0, double fp, double Cm, double C0, double Cp,
                                            double Dm, double D0, double Dp) {
    const double F = C0 + (fm + fp);
    const double E = D0 + (Cm + Cp);
    const double K = Dm + Dp;
    return FMA(-128.0, f0, FMA(14.0, F, FMA(3.0, E, K)));
}

template <int MODEL, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) step3d_zreg_kernel(StepArgs a, int tiles_x, int tiles_y,
                                                         long long planes_per_cta) {
    static_assert(MODEL != MC, "Model C runs on the accessor-based kernels");
    typedef Step3dZregShape<MODEL, TX, TY, NT> Sh;
    typedef double C;
    constexpr int RIN = Sh::RIN, WIN = Sh::WIN, AIN = Sh::AIN, NF = Sh::NF;
    constexpr int WMU = Sh::WMU, AMU = Sh::AMU, EPT = Sh::EPT, EMU = Sh::EMU, EOUT = Sh::EOUT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s_in = reinterpret_cast<C *>(smem_raw);  // [2][NF][AIN]
    C *s_mu = s_in + (size_t)2 * NF * AIN;      // [AMU]

    const ConstsC<C> k(a.k, a.kf);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int t = threadIdx.x;
    const size_t plane = (size_t)nx * (size_t)ny;
    const double *in[2] = {static_cast<const double *>(a.in0), static_cast<const double *>(a.in1)};
    double *out[2] = {static_cast<double *>(a.out0), static_cast<double *>(a.out1)};
    // output points of this thread: rows oy + e * (NT / TX), column ox
    const int ox = t % TX, oy = t / TX;
    constexpr int OSTEP = NT / TX;

    long long g0 = (long long)blockIdx.x * planes_per_cta;
    const long long gend = min(g0 + planes_per_cta, (long long)tiles_x * tiles_y * nz);
    while (g0 < gend) {
        const int tile = (int)(g0 / nz);
        const int z0 = (int)(g0 - (long long)tile * nz);
        const int z1 = (int)min((long long)nz, (long long)z0 + (gend - g0));
        g0 += z1 - z0;
        const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
        const int nplanes = (z1 - z0) + 2 * RIN;

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
        auto fetch = [&](int z) {
            const size_t zoff = (size_t)wrap_idx(z, nz) * plane;
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
                for (int e = 0; e < EPT; ++e)
                    if (loff[e] >= 0) pf[f][e] = load_one(in[f] + zoff + loff[e]);
        };

        // register queues: index 0 = plane j-2, 1 = plane j-1 (of the streamed quantity)
        C qf[NF][EOUT][2], qC[NF][EOUT][2], qD[NF][EOUT][2];
        constexpr int EM = EMU > 0 ? EMU : 1;
        C mf[EM][2], mC[EM][2], mD[EM][2];  // Cahn-Hilliard: phi partials at mu points
        C pq[EOUT][2];                          // Cahn-Hilliard: phi at output points
        (void)mf; (void)mC; (void)mD; (void)pq;

        fetch(z0 - RIN);
        for (int j = 0; j < nplanes; ++j) {
            C *buf = s_in + (size_t)(j & 1) * NF * AIN;
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
                for (int e = 0; e < EPT; ++e)
                    if (loff[e] >= 0) buf[(size_t)f * AIN + t + e * NT] = pf[f][e];
            if (j + 1 < nplanes) fetch(z0 - RIN + j + 1);
            __syncthreads();
            if constexpr (MODEL == CH) {
                // mu of plane j-1 at the tile points plus one halo cell
#pragma unroll
                for (int e = 0; e < EMU; ++e) {
                    const int c = t + e * NT;
                    if (c < AMU) {
                        const int ym = c / WMU, xm = c - ym * WMU;
                        const C *p = buf + (ym + 1) * WIN + (xm + 1);
                        C Cz, Dz;
                        plane_sums27(p, WIN, Cz, Dz);
                        const C f0 = p[0];
                        if (j >= 2) {
                            const C S = combine27(mf[e][0], mf[e][1], f0, mC[e][0], mC[e][1], Cz, mD[e][0], mD[e][1], Dz);
                            s_mu[c] = ch_mu<C>(mf[e][1], S, k);
                        }
                        mf[e][0] = mf[e][1], mf[e][1] = f0;
                        mC[e][0] = mC[e][1], mC[e][1] = Cz;
                        mD[e][0] = mD[e][1], mD[e][1] = Dz;
                    }
                }
                C pnow[EOUT];
#pragma unroll
                for (int e = 0; e < EOUT; ++e) pnow[e] = buf[(oy + e * OSTEP + RIN) * WIN + ox + RIN];
                __syncthreads();
                if (j >= 2) {
                    // mu partial sums of plane j-1; output of plane j-2
                    const int zo = z0 - 4 + j;
#pragma unroll
                    for (int e = 0; e < EOUT; ++e) {
                        const int yy = oy + e * OSTEP;
                        const C *m = s_mu + (yy + 1) * WMU + (ox + 1);
                        C Cz, Dz;
                        plane_sums27(m, WMU, Cz, Dz);
                        const C m0 = m[0];
                        if (j >= 4) {
                            const C S = combine27(qf[0][e][0], qf[0][e][1], m0, qC[0][e][0], qC[0][e][1], Cz,
                                                  qD[0][e][0], qD[0][e][1], Dz);
                            const int x = x0 + ox, y = y0 + yy;
                            if (x < nx && y < ny)
                                out[0][(size_t)zo * plane + (size_t)y * nx + x] = ch_update<C>(pq[e][0], S, k);
                        }
                        qf[0][e][0] = qf[0][e][1], qf[0][e][1] = m0;
                        qC[0][e][0] = qC[0][e][1], qC[0][e][1] = Cz;
                        qD[0][e][0] = qD[0][e][1], qD[0][e][1] = Dz;
                    }
                }
#pragma unroll
                for (int e = 0; e < EOUT; ++e) pq[e][0] = pq[e][1], pq[e][1] = pnow[e];
            } else {
                // output of plane j-1
                const int zo = z0 - 2 + j;
#pragma unroll
                for (int e = 0; e < EOUT; ++e) {
                    const int yy = oy + e * OSTEP;
                    C f0[NF], S[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const C *p = buf + (size_t)f * AIN + (yy + 1) * WIN + (ox + 1);
                        C Cz, Dz;
                        plane_sums27(p, WIN, Cz, Dz);
                        f0[f] = p[0];
                        if (j >= 2)
                            S[f] = combine27(qf[f][e][0], qf[f][e][1], f0[f], qC[f][e][0], qC[f][e][1], Cz,
                                             qD[f][e][0], qD[f][e][1], Dz);
                        qC[f][e][0] = qC[f][e][1], qC[f][e][1] = Cz;
                        qD[f][e][0] = qD[f][e][1], qD[f][e][1] = Dz;
                    }
                    if (j >= 2) {
                        const int x = x0 + ox, y = y0 + yy;
                        if (x < nx && y < ny) {
                            const size_t o = (size_t)zo * plane + (size_t)y * nx + x;
                            if constexpr (MODEL == AC) {
                                out[0][o] = ac_update<C>(qf[0][e][1], S[0], k);
                            } else {
                                C un, vn;
                                gs_update<C>(qf[0][e][1], qf[NF - 1][e][1], S[0], S[NF - 1], k, un, vn);
                                out[0][o] = un;
                                out[NF - 1][o] = vn;
                            }
                        }
                    }
#pragma unroll
                    for (int f = 0; f < NF; ++f) qf[f][e][0] = qf[f][e][1], qf[f][e][1] = f0[f];
                }
            }
        }
        __syncthreads();  // the buffers are reused by the next segment
    }  // segments
}

// ------------------------------------- 3D, 27-point, FP64, shared pair sums --
//
// The same fixed order with the x-pair sums shared between y neighbours: in
// row y, P(y) = f(x-1, y) + f(x+1, y); the in-plane sums are then
// C = P(y) + (f(y-1) + f(y+1)) and D = P(y-1) + P(y+1) (exactly the groupings
// of plane_sums27).  Each plane's P is formed once per point in shared memory
// (rows -1 .. TY of the tile), so a stencil application costs 12 FP64
// operations (P 1, C 2, D 1, combine 8) instead of 14; value, C and D of the
// two previous planes stay in registers as in step3d_zreg_kernel.
//
// Cahn-Hilliard runs as two passes through a mu buffer (mode 0: mu of every
// point; mode 1: the update from mu and the centre phi), so mu is evaluated
// once per point rather than on a halo ring as well; the buffer's HBM traffic
// (16 bytes per point) is cheap next to the FP64 work on this part.  Allen-Cahn
// (mode 2) and Gray-Scott (mode 3) take one pass.  Same operations in the same
// order as every other family, so the results are identical bit for bit.
// The default for these grids; measured on GB300 against step3d_zreg_kernel:
// Cahn-Hilliard 1024^3 17.5 vs 13.6 GLUPS, Allen-Cahn 512^3 29.6 vs 27.0,
// Gray-Scott 512^3 14.9 vs 13.3.
struct Planes27Args {
    const double *in[2];   // streamed fields (mode 1: mu)
    const double *centre;  // mode 1: phi at the output points
    double *out[2];        // mode 0: mu
    int nx, ny, nz;
    StepConsts k;
};

template <int MODE>
struct Planes27Shape {
    static constexpr int NF = (MODE == 3) ? 2 : 1;
    static constexpr int TX = 32, TY = 32, NT = 256;
    static constexpr int WIN = TX + 2, HIN = TY + 2, AIN = WIN * HIN;
    static constexpr int AP = HIN * TX;                // pair sums of rows -1 .. TY
    static constexpr int EPT = (AIN + NT - 1) / NT;    // loaded cells per thread per field
    static constexpr int EOUT = TX * TY / NT, OSTEP = NT / TX;
    static constexpr size_t smem_bytes = sizeof(double) * ((size_t)2 * NF * AIN + (size_t)NF * AP);
};

template <int MODE>
__global__ void __launch_bounds__(256, MODE == 3 ? 1 : 2)
    planes27_kernel(Planes27Args a, int tiles_x, long long planes_per_cta, long long total) {
    typedef Planes27Shape<MODE> Sh;
    constexpr int NF = Sh::NF, TX = Sh::TX, TY = Sh::TY, NT = Sh::NT, WIN = Sh::WIN, AIN = Sh::AIN, AP = Sh::AP;
    constexpr int EPT = Sh::EPT, EOUT = Sh::EOUT, OSTEP = Sh::OSTEP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *s_in = reinterpret_cast<double *>(smem_raw);  // [2][NF][AIN]
    double *s_P = s_in + (size_t)2 * NF * AIN;            // [NF][AP]
    const ConstsC<double> k(a.k, StepConstsF{});
    const int nx = a.nx, ny = a.ny, nz = a.nz, t = threadIdx.x;
    const size_t plane = (size_t)nx * (size_t)ny;
    const int ox = t % TX, oy = t / TX;  // output points (ox, oy + e OSTEP)

    long long g0 = (long long)blockIdx.x * planes_per_cta;
    const long long gend = min(g0 + planes_per_cta, total);
    while (g0 < gend) {
        const int tile = (int)(g0 / nz);
        const int z0 = (int)(g0 - (long long)tile * nz);
        const int z1 = (int)min((long long)nz, (long long)z0 + (gend - g0));
        g0 += z1 - z0;
        const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
        const int nplanes = (z1 - z0) + 2;  // loaded plane j is z = z0 - 1 + j

        int loff[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int c = t + e * NT;
            if (c < AIN) {
                const int yi = c / WIN, xi = c - yi * WIN;
                loff[e] = wrap_idx(y0 - 1 + yi, ny) * nx + wrap_idx(x0 - 1 + xi, nx);
            } else {
                loff[e] = -1;
            }
        }
        double pf[NF][EPT];
        auto fetch = [&](int z) {
            const size_t zoff = (size_t)wrap_idx(z, nz) * plane;
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
                for (int e = 0; e < EPT; ++e)
                    if (loff[e] >= 0) pf[f][e] = load_one(a.in[f] + zoff + loff[e]);
        };
        // register queues: index 0 = plane j-2, 1 = plane j-1
        double qf[NF][EOUT][2], qC[NF][EOUT][2], qD[NF][EOUT][2];

        fetch(z0 - 1);
        for (int j = 0; j < nplanes; ++j) {
            double *buf = s_in + (size_t)(j & 1) * NF * AIN;
#pragma unroll
            for (int f = 0; f < NF; ++f)
#pragma unroll
                for (int e = 0; e < EPT; ++e)
                    if (loff[e] >= 0) buf[(size_t)f * AIN + t + e * NT] = pf[f][e];
            if (j + 1 < nplanes) fetch(z0 + j);
            __syncthreads();
#pragma unroll
            for (int f = 0; f < NF; ++f)
                for (int q = t; q < AP; q += NT) {
                    const int r = q / TX, c = q - r * TX;
                    const double *row = buf + (size_t)f * AIN + r * WIN + c;
                    s_P[(size_t)f * AP + q] = row[0] + row[2];
                }
            __syncthreads();
            const int zo = z0 - 2 + j;  // output plane (j >= 2)
#pragma unroll
            for (int e = 0; e < EOUT; ++e) {
                const int yy = oy + e * OSTEP;
                double S[NF], fc[NF];
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const double *p = buf + (size_t)f * AIN + (yy + 1) * WIN + (ox + 1);
                    const double *P = s_P + (size_t)f * AP + (yy + 1) * TX + ox;
                    const double Cz = P[0] + (p[-WIN] + p[WIN]);
                    const double Dz = P[-TX] + P[TX];
                    const double f0 = p[0];
                    S[f] = (j >= 2) ? combine27(qf[f][e][0], qf[f][e][1], f0, qC[f][e][0], qC[f][e][1], Cz,
                                                qD[f][e][0], qD[f][e][1], Dz)
                                    : 0.0;
                    fc[f] = qf[f][e][1];
                    qf[f][e][0] = qf[f][e][1], qf[f][e][1] = f0;
                    qC[f][e][0] = qC[f][e][1], qC[f][e][1] = Cz;
                    qD[f][e][0] = qD[f][e][1], qD[f][e][1] = Dz;
                }
                const int x = x0 + ox, y = y0 + yy;
                if (j >= 2 && x < nx && y < ny) {
                    const size_t o = (size_t)zo * plane + (size_t)y * nx + x;
                    if constexpr (MODE == 0) {
                        a.out[0][o] = ch_mu<double>(fc[0], S[0], k);
                    } else if constexpr (MODE == 1) {
                        a.out[0][o] = ch_update<double>(a.centre[o], S[0], k);
                    } else if constexpr (MODE == 2) {
                        a.out[0][o] = ac_update<double>(fc[0], S[0], k);
                    } else {
                        double un, vn;
                        gs_update<double>(fc[0], fc[1], S[0], S[1], k, un, vn);
                        a.out[0][o] = un;
                        a.out[1][o] = vn;
                    }
                }
            }
        }
        __syncthreads();  // the buffers are reused by the next tile
    }
}

// --------------------- 3D FP64 Cahn-Hilliard, 7- and 13-point, two passes --
//
// Cahn-Hilliard through a mu buffer, as for the 27-point stencil: pass 0 writes
// mu = ch_mu(phi, S(phi)) of every point, pass 1 phi' = ch_update(phi, S(mu)).
// Each pass streams TX x TY tiles along z; the input planes (tile + R halo)
// enter a shared-memory ring of 2R + 2 planes (one barrier per plane: the plane
// committed at iteration j is never one a thread still in iteration j - 1
// reads), and the stencil sum of plane j - R is taken from the ring in the
// fixed order.  The FP64 operations are exactly the counted ones (S + 4, then
// S + 1): the fused kernel also evaluates mu on a halo ring of the tile.  The
// default for these grids; measured on GB300 at 1024^3 against the fused
// kernel: 7-point 29.6 vs 27.2 GLUPS, 13-point 17.7 vs 14.3.
template <int ST>
struct Ring2PassShape {
    static constexpr int R = StencilInfo<ST>::r;
    static constexpr int TX = 32, TY = 32, NT = 256;
    static constexpr int WIN = TX + 2 * R, HIN = TY + 2 * R, AIN = WIN * HIN;
    static constexpr int D = 2 * R + 2;
    static constexpr int EPT = (AIN + NT - 1) / NT;
    static constexpr int EOUT = TX * TY / NT, OSTEP = NT / TX;
    static constexpr size_t smem_bytes = sizeof(double) * (size_t)D * AIN;
};

template <int ST, int MODE>
__global__ void __launch_bounds__(256, 2)
    ring2pass_kernel(Planes27Args a, int tiles_x, long long planes_per_cta, long long total) {
    typedef Ring2PassShape<ST> Sh;
    constexpr int R = Sh::R, TX = Sh::TX, NT = Sh::NT, WIN = Sh::WIN, AIN = Sh::AIN, D = Sh::D;
    constexpr int EPT = Sh::EPT, EOUT = Sh::EOUT, OSTEP = Sh::OSTEP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *s_in = reinterpret_cast<double *>(smem_raw);  // [D][AIN]
    const ConstsC<double> k(a.k, StepConstsF{});
    const int nx = a.nx, ny = a.ny, nz = a.nz, t = threadIdx.x;
    const size_t plane = (size_t)nx * (size_t)ny;
    const int ox = t % TX, oy = t / TX;

    long long g0 = (long long)blockIdx.x * planes_per_cta;
    const long long gend = min(g0 + planes_per_cta, total);
    while (g0 < gend) {
        const int tile = (int)(g0 / nz);
        const int z0 = (int)(g0 - (long long)tile * nz);
        const int z1 = (int)min((long long)nz, (long long)z0 + (gend - g0));
        g0 += z1 - z0;
        const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * Sh::TY;
        const int nplanes = (z1 - z0) + 2 * R;  // loaded plane j is z = z0 - R + j

        int loff[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int c = t + e * NT;
            if (c < AIN) {
                const int yi = c / WIN, xi = c - yi * WIN;
                loff[e] = wrap_idx(y0 - R + yi, ny) * nx + wrap_idx(x0 - R + xi, nx);
            } else {
                loff[e] = -1;
            }
        }
        double pf[EPT];
        auto fetch = [&](int z) {
            const size_t zoff = (size_t)wrap_idx(z, nz) * plane;
#pragma unroll
            for (int e = 0; e < EPT; ++e)
                if (loff[e] >= 0) pf[e] = load_one(a.in[0] + zoff + loff[e]);
        };

        fetch(z0 - R);
        for (int j = 0; j < nplanes; ++j) {
            double *slot = s_in + (size_t)(j % D) * AIN;
#pragma unroll
            for (int e = 0; e < EPT; ++e)
                if (loff[e] >= 0) slot[t + e * NT] = pf[e];
            if (j + 1 < nplanes) fetch(z0 - R + j + 1);
            __syncthreads();
            if (j >= 2 * R) {
                const int c = j - R;  // loaded index of the output plane
                const int zo = z0 - R + c;
                const double *pl[2 * R + 1];
#pragma unroll
                for (int dz = -R; dz <= R; ++dz) pl[dz + R] = s_in + (size_t)((c + dz) % D) * AIN;
#pragma unroll
                for (int e = 0; e < EOUT; ++e) {
                    const int yy = oy + e * OSTEP;
                    const int x = x0 + ox, y = y0 + yy;
                    const int b = (yy + R) * WIN + ox + R;
                    auto P = [&](int dx, int dy, int dz) -> double { return pl[dz + R][b + dy * WIN + dx]; };
                    const double S = stencil_sum<ST, double>(P);
                    if (x < nx && y < ny) {
                        const size_t o = (size_t)zo * plane + (size_t)y * nx + x;
                        if constexpr (MODE == 0)
                            a.out[0][o] = ch_mu<double>(P(0, 0, 0), S, k);
                        else
                            a.out[0][o] = ch_update<double>(a.centre[o], S, k);
                    }
                }
            }
        }
        __syncthreads();  // the ring is reused by the next tile
    }
}

// ===================================================== 3D, warp rows ==
//
// FP32 / BF16-storage 3D kernel built like the 2D warp-strip kernel.  Warp w
// of a CTA owns input row w of a tile (TY output rows plus R halo rows on each
// side) and lane l the chunk l of 4 cells of that row (16 bytes FP32, 8 bytes
// BF16): lanes 1..30 are the tile's 30 chunks, lanes 0 and 31 halo chunks.
// Planes stream along z through a ring of P+1 planes in shared memory filled by
// cp.async (each thread copies its own chunk; one base pointer per plane, the
// global source and destination offsets advance by a plane each step).
// Neighbours: x from the adjacent lanes (warp shuffles), y from the rows above
// and below in shared memory, z from per-thread register queues of the previous
// planes' values and in-plane partial sums, held as pairs of cells (the
// stencil's fixed order is a sum over planes of in-plane partial sums, see
// sp_common.cuh); the combine, mu and the updates run two cells per instruction
// (packed f32x2).  Cahn-Hilliard keeps mu in the register queues and shares each
// mu plane through one of two mu buffers in shared memory; its output stage runs
// one plane behind mu, so one barrier per plane suffices.  The plane loop is
// unrolled by the queue length so that queues rotate by renaming registers.
// Same expressions in the same order as the other FP32 kernels: identical
// results bit for bit.
//
// Requirements (checked by the launcher): nx a multiple of 4 and 16-byte
// aligned field pointers.

// Number of in-plane partial sums per plane.
template <int ST> struct Planar { static constexpr int NP = (ST == L7) ? 1 : 2; };

// In-plane partial sums of plane z for the V cells of a chunk.  row(dy) points
// at a row extended by r cells on each side (index r + c is cell c).
template <int ST, int V, int XW, typename RowFn>
__device__ __forceinline__ void planar_sums(const RowFn &row, float (&ps)[Planar<ST>::NP][V]) {
    const float *w0 = row(0);
#pragma unroll
    for (int c = 0; c < V; ++c) {
        const int x = StencilInfo<ST>::r + c;
        if constexpr (ST == L7) {
            ps[0][c] = (w0[x - 1] + w0[x + 1]) + (row(-1)[x] + row(1)[x]);
        } else if constexpr (ST == L27) {
            const float *wm = row(-1), *wp = row(1);
            ps[0][c] = (w0[x - 1] + w0[x + 1]) + (wm[x] + wp[x]);
            ps[1][c] = (wm[x - 1] + wm[x + 1]) + (wp[x - 1] + wp[x + 1]);
        } else {  // L13X4
            ps[0][c] = (w0[x - 1] + w0[x + 1]) + (row(-1)[x] + row(1)[x]);
            ps[1][c] = (w0[x - 2] + w0[x + 2]) + (row(-2)[x] + row(2)[x]);
        }
    }
}

// Stencil sum at the centre plane from the values f[k] and partial sums p[k]
// of planes k = 0 .. 2r (z offsets -r .. r), for the pair of cells q (cells 2q
// and 2q+1), two cells per instruction.
template <int ST, typename FA, typename PA>
__device__ __forceinline__ float2 planar_combine2(const FA &f, const PA &p, int q) {
    if constexpr (ST == L7) {
        return fma2(splat2(-6.f), f(1)[q], add2(p(1)[0][q], add2(f(0)[q], f(2)[q])));
    } else if constexpr (ST == L27) {
        const float2 F = add2(p(1)[0][q], add2(f(0)[q], f(2)[q]));
        const float2 E = add2(p(1)[1][q], add2(p(0)[0][q], p(2)[0][q]));
        const float2 K = add2(p(0)[1][q], p(2)[1][q]);
        return fma2(splat2(-128.f), f(1)[q], fma2(splat2(14.f), F, fma2(splat2(3.f), E, K)));
    } else {  // L13X4
        const float2 F1 = add2(p(2)[0][q], add2(f(1)[q], f(3)[q]));
        const float2 F2 = add2(p(2)[1][q], add2(f(0)[q], f(4)[q]));
        return fma2(splat2(-90.f), f(2)[q], fma2(splat2(16.f), F1, neg2(F2)));
    }
}

template <int MODEL, int ST, typename T, int TY>
struct Step3dWrShape {
    typedef typename Cmp<T>::type C;
    static constexpr int V = 4;                       // cells per lane (16 bytes FP32, 8 bytes BF16)
    static constexpr int CB = V * (int)sizeof(T);     // chunk bytes
    static constexpr int r = StencilInfo<ST>::r;
    static constexpr int R = (MODEL == CH) ? 2 * r : r;
    static_assert(V >= 2 * r, "a lane's chunk must cover the halo");
    static constexpr int TXC = 30;                    // output chunks per tile row
    static constexpr int TX = TXC * V;
    static constexpr int HIN = TY + 2 * R;            // warps = input rows
    static constexpr int NT = 32 * HIN;
    static constexpr int XW = V + 2 * r;
    static constexpr int NP = Planar<ST>::NP;
    static constexpr int Q = 2 * r + 1;               // planes in a queue (incl. the newest)
    static constexpr int P = 3;                       // planes in flight
    static constexpr int NF = num_fields<MODEL>();
    static constexpr size_t plane_bytes = (size_t)HIN * 32 * CB;
    static constexpr size_t in_bytes = (size_t)(P + 1) * NF * plane_bytes;
    // Cahn-Hilliard: two mu planes (plane j - r is written while the output stage
    // reads plane j - 1 - r), so one barrier per plane suffices
    static constexpr size_t mu_plane = (size_t)HIN * 32 * V;
    static constexpr size_t mu_bytes = (MODEL == CH) ? 2 * mu_plane * sizeof(float) : 0;
    static constexpr size_t smem_bytes = in_bytes + mu_bytes;
    // resident CTAs per SM asked of the register allocator (measured on GB300:
    // Allen-Cahn with radius-1 stencils gains from a third CTA; Cahn-Hilliard
    // 7-point needs two; elsewhere a bound would make the queues spill)
    static constexpr int MINB = (MODEL == AC && r == 1) ? 3 : ((MODEL == CH && ST == L7) ? 2 : 1);
};

template <int MODEL, int ST, typename T, int TY>
__global__ void __launch_bounds__(Step3dWrShape<MODEL, ST, T, TY>::NT, Step3dWrShape<MODEL, ST, T, TY>::MINB)
    step3d_wr_kernel(StepArgs a, int tiles_x, int tiles_y, int segs) {
    static_assert(MODEL != MC, "Model C runs on the accessor-based kernels");
    typedef Step3dWrShape<MODEL, ST, T, TY> Sh;
    typedef float C;
    constexpr int V = Sh::V, r = Sh::r, R = Sh::R, HIN = Sh::HIN, XW = Sh::XW, NP = Sh::NP, Q = Sh::Q;
    constexpr int P = Sh::P, NF = Sh::NF, CB = Sh::CB;
    constexpr unsigned FULL = 0xffffffffu;
    typedef typename VecT<CB>::type W;                                      // one chunk
    extern __shared__ __align__(16) unsigned char smem_raw[];
    W *s_in = reinterpret_cast<W *>(smem_raw);                              // [P+1][NF][HIN][32]
    float *s_mu = reinterpret_cast<float *>(smem_raw + Sh::in_bytes);      // [2][HIN][32][V]

    const ConstsF2 k2(ConstsC<C>(a.k, a.kf));
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t plane = (size_t)nx * (size_t)ny;
    const T *in[2] = {static_cast<const T *>(a.in0), static_cast<const T *>(a.in1)};
    T *out[2] = {static_cast<T *>(a.out0), static_cast<T *>(a.out1)};
    const bool mu_row = (MODEL == CH) && w >= r && w < HIN - r;
    const bool out_row = w >= R && w < HIN - R;

    // this lane's chunk of its own row in ring slot 0 (field 0); other slots,
    // fields and rows lie at fixed offsets, so each plane needs one base pointer
    constexpr int D = P + 1;  // ring slots
    static_assert((D & (D - 1)) == 0, "ring slots must be a power of two");
    constexpr size_t SLOT = (size_t)NF * HIN * 32, FLD = (size_t)HIN * 32;
    W *const s_own = s_in + (size_t)w * 32 + lane;
    float *const mu_own = s_mu + ((size_t)w * 32 + lane) * V;
    // chunk at row offset dy of field f in the slot starting at `base`, widened
    auto ring_chunk = [&](const W *base, int f, int dy, float *dst) {
        union { W q; T t[V]; } u;
        u.q = base[f * FLD + dy * 32];
#pragma unroll
        for (int i = 0; i < V; ++i) dst[i] = to_c(u.t[i]);
    };
    // extend a row chunk held in ext[r .. r+V) with r cells from each neighbouring lane
    auto extend = [&](float *ext) {
#pragma unroll
        for (int h = 0; h < r; ++h) {
            ext[h] = __shfl_up_sync(FULL, ext[V + h], 1);
            ext[r + V + h] = __shfl_down_sync(FULL, ext[r + h], 1);
        }
    };

    const int tiles = tiles_x * tiles_y;
    for (long long it = blockIdx.x; it < (long long)tiles * segs; it += gridDim.x) {
        const int seg = (int)(it / tiles), tile = (int)(it - (long long)seg * tiles);
        const int z0 = (int)((long long)seg * nz / segs), z1 = (int)((long long)(seg + 1) * nz / segs);
        const int x0 = (tile % tiles_x) * Sh::TX, y0 = (tile / tiles_x) * TY;
        const int n = (z1 - z0) + 2 * R;                           // planes fetched
        const int niter = n + (MODEL == CH ? 1 : 0);              // CH: the output stage lags one plane
        const int col = x0 + (lane - 1) * V;                       // first cell of this lane's chunk
        const size_t goff = (size_t)wrap_idx(y0 - R + w, ny) * nx + wrap_idx(col, nx);
        const int yo = y0 - R + w;                                 // output row (if out_row)
        const bool store = out_row && lane >= 1 && lane <= 30 && col < nx && yo < ny;
        // element offsets: next plane to fetch (plane jn, wrapped z zn) and next output
        int jn = 0, zn = wrap_idx(z0 - R, nz);
        size_t src = (size_t)zn * plane + goff;
        size_t dst_off = (size_t)z0 * plane + (size_t)yo * nx + col;

        auto issue = [&]() {
            if (jn < n) {
                W *dst = s_own + (size_t)(jn & (D - 1)) * SLOT;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    if constexpr (CB == 16) cp_async16(dst + f * FLD, in[f] + src);
                    else cp_async8(dst + f * FLD, in[f] + src);
                }
                src += plane;
                if (++zn == nz) {
                    zn = 0;
                    src -= (size_t)nz * plane;
                }
            }
            ++jn;
            cp_async_commit();
        };
#pragma unroll
        for (int j = 0; j < P; ++j) issue();

        // queues, slot (j % Q) holds plane j: values and partial sums, as pairs of cells
        constexpr int V2 = V / 2;
        float2 qf[NF][Q][V2], qp[NF][Q][NP][V2];
        float2 qm[MODEL == CH ? Q : 1][V2], qmp[MODEL == CH ? Q : 1][NP][V2];
        (void)qm; (void)qmp;
        // in-plane partial sums of a row triple into queue slot dst
        auto sums_into = [&](const float (*ext)[XW], float2 (&dst)[NP][V2]) {
            float ps[NP][V];
            auto row = [&](int dy) -> const float * { return ext[r + dy]; };
            planar_sums<ST, V, XW>(row, ps);
#pragma unroll
            for (int n2 = 0; n2 < NP; ++n2)
#pragma unroll
                for (int q = 0; q < V2; ++q) dst[n2][q] = make_float2(ps[n2][2 * q], ps[n2][2 * q + 1]);
        };

        for (int j0 = 0; j0 < niter; j0 += Q) {
#pragma unroll
            for (int u = 0; u < Q; ++u) {
                const int j = j0 + u;
                if (j < niter) {
                    cp_async_wait<P - 1>();
                    // plane j published; plane j-1's slot is free; CH: mu plane j-1-r
                    // published and the mu buffer of plane j-2-r free
                    __syncthreads();
                    issue();          // plane j + P into plane j-1's slot
                    const W *cur = s_own + (size_t)(j & (D - 1)) * SLOT;
#define QS(m) ((u - (m) + 4 * Q) % Q)   /* queue slot of plane j - m */
                    if constexpr (MODEL == CH) {
                        // output stage on mu plane j - 1 - r (written in the previous
                        // iteration, published by this iteration's barrier); it runs
                        // first because phi of its output plane j - 1 - 2r and the mu
                        // of plane j - 1 - 3r sit in the queue slots that plane j and
                        // mu plane j - r take below
                        if (out_row && j >= 2 * r + 1) {
                            const float2 *mu = qm[QS(1)];
                            const float *mu_prev = mu_own + (size_t)((j - 1) & 1) * Sh::mu_plane;
                            float ext[2 * r + 1][XW];
#pragma unroll
                            for (int q = 0; q < V2; ++q) {
                                ext[r][r + 2 * q] = mu[q].x;
                                ext[r][r + 2 * q + 1] = mu[q].y;
                            }
                            extend(ext[r]);
#pragma unroll
                            for (int dy = -r; dy <= r; ++dy) {
                                if (dy == 0) continue;
                                const float *src_mu = mu_prev + dy * 32 * V;
#pragma unroll
                                for (int i = 0; i < V; i += 4) {
                                    const float4 v4 = *reinterpret_cast<const float4 *>(src_mu + i);
                                    ext[r + dy][r + i] = v4.x;
                                    ext[r + dy][r + i + 1] = v4.y;
                                    ext[r + dy][r + i + 2] = v4.z;
                                    ext[r + dy][r + i + 3] = v4.w;
                                }
                                if constexpr (ST == L27) extend(ext[r + dy]);
                            }
                            sums_into(ext, qmp[QS(0)]);
                            if (j >= 4 * r + 1) {
                                // output plane j - 1 - 2r: mu planes j - 1 - 3r .. j - 1 - r in mu
                                // queue slots of iterations j - 2r - 1 .. j - 1 (values) and
                                // j - 2r .. j (partial sums); its phi in the slot of iteration j - 1 - 2r
                                auto mf = [&](int kk) -> const float2 * { return qm[QS(2 * r + 1 - kk)]; };
                                auto mp = [&](int kk) -> const float2(*)[V2] { return qmp[QS(2 * r - kk)]; };
                                float o[V];
#pragma unroll
                                for (int q = 0; q < V2; ++q) {
                                    const float2 o2 =
                                        ch_update2(qf[0][QS(2 * r + 1)][q], planar_combine2<ST>(mf, mp, q), k2);
                                    o[2 * q] = o2.x;
                                    o[2 * q + 1] = o2.y;
                                }
                                if (store) store_vec<T, V>(out[0] + dst_off, o);
                                dst_off += plane;
                            }
                        }
                    }
                    if (j < n && ((MODEL == CH && mu_row) || (MODEL != CH && out_row))) {
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            float ext[2 * r + 1][XW];
                            ring_chunk(cur, f, 0, ext[r] + r);
                            extend(ext[r]);
#pragma unroll
                            for (int dy = 1; dy <= r; ++dy) {
                                ring_chunk(cur, f, -dy, ext[r - dy] + r);
                                ring_chunk(cur, f, dy, ext[r + dy] + r);
                                if constexpr (ST == L27) {
                                    extend(ext[r - dy]);
                                    extend(ext[r + dy]);
                                }
                            }
                            sums_into(ext, qp[f][QS(0)]);
#pragma unroll
                            for (int q = 0; q < V2; ++q)
                                qf[f][QS(0)][q] = make_float2(ext[r][r + 2 * q], ext[r][r + 2 * q + 1]);
                        }
                    }
                    // stencil of plane j - r from the queues (planes j - 2r .. j)
                    auto f0q = [&](int kk) -> const float2 * { return qf[0][QS(2 * r - kk)]; };
                    auto p0q = [&](int kk) -> const float2(*)[V2] { return qp[0][QS(2 * r - kk)]; };
                    auto f1q = [&](int kk) -> const float2 * { return qf[NF - 1][QS(2 * r - kk)]; };
                    auto p1q = [&](int kk) -> const float2(*)[V2] { return qp[NF - 1][QS(2 * r - kk)]; };
                    (void)f1q; (void)p1q;
                    if constexpr (MODEL == CH) {
                        // mu of plane j - r into the queue and the mu buffer of this iteration
                        if (mu_row && j >= 2 * r && j < n) {
                            float2 *mu = qm[QS(0)];
#pragma unroll
                            for (int q = 0; q < V2; ++q)
                                mu[q] = ch_mu2(qf[0][QS(r)][q], planar_combine2<ST>(f0q, p0q, q), k2);
                            float *dst_mu = mu_own + (size_t)(j & 1) * Sh::mu_plane;
#pragma unroll
                            for (int q = 0; q < V2; q += 2)
                                *reinterpret_cast<float4 *>(dst_mu + 2 * q) =
                                    make_float4(mu[q].x, mu[q].y, mu[q + 1].x, mu[q + 1].y);
                        }
                    } else {
                        if (out_row && j >= 2 * r) {
                            float o0[V], o1[V];
#pragma unroll
                            for (int q = 0; q < V2; ++q) {
                                const float2 S0 = planar_combine2<ST>(f0q, p0q, q);
                                const float2 p0 = qf[0][QS(r)][q];
                                float2 a0, a1 = make_float2(0.f, 0.f);
                                if constexpr (MODEL == AC) {
                                    a0 = ac_update2(p0, S0, k2);
                                } else {
                                    gs_update2(p0, qf[NF - 1][QS(r)][q], S0, planar_combine2<ST>(f1q, p1q, q), k2, a0,
                                               a1);
                                }
                                o0[2 * q] = a0.x;
                                o0[2 * q + 1] = a0.y;
                                o1[2 * q] = a1.x;
                                o1[2 * q + 1] = a1.y;
                            }
                            if (store) {
                                store_vec<T, V>(out[0] + dst_off, o0);
                                if constexpr (num_fields<MODEL>() == 2) store_vec<T, V>(out[NF - 1] + dst_off, o1);
                            }
                            dst_off += plane;
                        }
                    }
#undef QS
                }
            }
        }
        cp_async_wait<0>();
        __syncthreads();  // the ring is reused by the next item
    }
}

// Stencil sum of the 4 cells of this lane's chunk, two cells per instruction,
// in the fixed order of stencil_sum (sp_common.cuh).  row(dz, dy, dst) loads
// the chunk at plane offset dz and row offset dy; `ext` helpers shuffle in the
// x halo.
template <int ST, typename RowFn, typename ExtFn>
__device__ __forceinline__ void ring_stencil(const RowFn &row, const ExtFn &extend, float (&S)[4], float (&cen)[4]) {
    constexpr int r = StencilInfo<ST>::r, V = 4, XW = V + 2 * r;
    auto pr = [](const float *a, int c0) { return make_float2(a[c0], a[c0 + 1]); };
    if constexpr (ST == L27) {
        // per plane dz: cross C and diagonal D sums of the 3 x 3 in-plane neighbourhood
        float2 Cz[3][2], Dz[3][2];
        float ctr[3][V];
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            float e[3][XW];
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                row(dz, dy, e[dy + 1] + r);
                extend(e[dy + 1]);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int c0 = 2 * q, x = r + c0;
                const float2 xs = make_float2(e[1][x - 1] + e[1][x + 1], e[1][x] + e[1][x + 2]);
                Cz[dz + 1][q] = add2(xs, add2(pr(e[0] + r, c0), pr(e[2] + r, c0)));
                const float2 dm = make_float2(e[0][x - 1] + e[0][x + 1], e[0][x] + e[0][x + 2]);
                const float2 dp = make_float2(e[2][x - 1] + e[2][x + 1], e[2][x] + e[2][x + 2]);
                Dz[dz + 1][q] = add2(dm, dp);
            }
#pragma unroll
            for (int c = 0; c < V; ++c) ctr[dz + 1][c] = e[1][r + c];
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int c0 = 2 * q;
            const float2 F = add2(Cz[1][q], add2(pr(ctr[0], c0), pr(ctr[2], c0)));
            const float2 E = add2(Dz[1][q], add2(Cz[0][q], Cz[2][q]));
            const float2 K = add2(Dz[0][q], Dz[2][q]);
            const float2 s2 =
                fma2(splat2(-128.f), pr(ctr[1], c0), fma2(splat2(14.f), F, fma2(splat2(3.f), E, K)));
            S[c0] = s2.x;
            S[c0 + 1] = s2.y;
            cen[c0] = ctr[1][c0];
            cen[c0 + 1] = ctr[1][c0 + 1];
        }
    } else {
        float ext[XW], ym[r][V], yp[r][V], zm[r][V], zp[r][V];
        row(0, 0, ext + r);
        extend(ext);
#pragma unroll
        for (int d = 1; d <= r; ++d) {
            row(0, -d, ym[d - 1]);
            row(0, d, yp[d - 1]);
            row(-d, 0, zm[d - 1]);
            row(d, 0, zp[d - 1]);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int c0 = 2 * q, x = r + c0;
            const float2 xs1 = make_float2(ext[x - 1] + ext[x + 1], ext[x] + ext[x + 2]);
            const float2 F1 =
                add2(add2(xs1, add2(pr(ym[0], c0), pr(yp[0], c0))), add2(pr(zm[0], c0), pr(zp[0], c0)));
            float2 s2;
            if constexpr (ST == L7) {
                s2 = fma2(splat2(-6.f), make_float2(ext[x], ext[x + 1]), F1);
            } else {
                const float2 xs2 = make_float2(ext[x - 2] + ext[x + 2], ext[x - 1] + ext[x + 3]);
                const float2 F2 = add2(add2(xs2, add2(pr(ym[r - 1], c0), pr(yp[r - 1], c0))),
                                       add2(pr(zm[r - 1], c0), pr(zp[r - 1], c0)));
                s2 = fma2(splat2(-90.f), make_float2(ext[x], ext[x + 1]), fma2(splat2(16.f), F1, neg2(F2)));
            }
            S[c0] = s2.x;
            S[c0 + 1] = s2.y;
            cen[c0] = ext[x];
            cen[c0 + 1] = ext[x + 1];
        }
    }
}

// ====================================== 3D, plane rings, K steps per pass ==
//
// Temporal blocking in 3D: K forward-Euler steps (K = 1: the plain step) of
// Allen-Cahn, Gray-Scott or Model C per HBM round trip, with
// every time level kept as a ring of planes in shared memory instead of
// register queues, so that a thread holds no per-level state and more warps fit
// on an SM.  Warp w owns row w of a tile (TY output rows plus K*r halo rows on
// each side), lane l the chunk of 4 cells l (lanes 1..30 the tile's 120 cells,
// lanes 0 and 31 halo chunks covering the K*r halo cells).  Input planes stream
// along z through a cp.async ring.  Level s (1..K) produces plane j-(s-1)-s*r
// at iteration j from planes of level s-1 that earlier iterations published
// (the x neighbours by warp shuffles, y and z neighbours from the ring of level
// s-1); levels 1..K-1 write their plane into their own ring, level K to global
// memory.  One barrier per iteration.  Level s is valid on the rows and cells of
// level s-1 shrunk by r, so after K levels exactly the tile remains.
// Intermediate planes are rounded to the storage type as a global store would
// round them, and every level evaluates the single-step expressions in the same
// order, so K blocked steps equal K single steps bit for bit.
//
// Requirements (checked by the launcher): nx a multiple of 4 and 16-byte
// aligned field pointers.
template <int MODEL, int ST, typename T, int TY, int K>
struct Step3dTbsShape {
    static constexpr int V = 4;
    static constexpr int CB = V * (int)sizeof(T);
    static constexpr int r = StencilInfo<ST>::r;
    static_assert(K * r <= V, "the halo lanes must cover K*r cells");
    static constexpr int TXC = 30;
    static constexpr int TX = TXC * V;
    static constexpr int HIN = TY + 2 * K * r;
    static constexpr int NT = 32 * HIN;
    static constexpr int NF = num_fields<MODEL>();
    static constexpr int P = 2;                        // input planes in flight
    static constexpr int D0 = 2 * r + 1 + P;           // input ring: planes read by level 1, plus in flight
    static constexpr int DL = 2 * r + 2;               // level ring: planes read by the next level, plus the new one
    static constexpr size_t in_plane = (size_t)HIN * 32 * CB;              // bytes, one field
    static constexpr size_t lv_plane = (size_t)HIN * 32 * V * sizeof(float);
    static constexpr size_t in_bytes = (size_t)D0 * NF * in_plane;
    static constexpr size_t smem_bytes = in_bytes + (size_t)(K - 1) * DL * NF * lv_plane;
};

template <int MODEL, int ST, typename T, int TY, int K>
__global__ void __launch_bounds__(Step3dTbsShape<MODEL, ST, T, TY, K>::NT)
    step3d_tbs_kernel(StepArgs a, int tiles_x, int tiles_y, int segs) {
    static_assert(MODEL == AC || MODEL == GS || MODEL == MC, "Allen-Cahn, Gray-Scott and Model C");
    typedef Step3dTbsShape<MODEL, ST, T, TY, K> Sh;
    constexpr int V = Sh::V, r = Sh::r, HIN = Sh::HIN, NF = Sh::NF, CB = Sh::CB, V2 = V / 2;
    const ConstsC<float> kc(a.k, a.kf);
    constexpr int D0 = Sh::D0, DL = Sh::DL, P = Sh::P;
    constexpr unsigned FULL = 0xffffffffu;
    typedef typename VecT<CB>::type W;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const ConstsF2 k2(ConstsC<float>(a.k, a.kf));
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t plane = (size_t)nx * (size_t)ny;
    const T *in[2] = {static_cast<const T *>(a.in0), static_cast<const T *>(a.in1)};
    T *out[2] = {static_cast<T *>(a.out0), static_cast<T *>(a.out1)};
    // this lane's chunk of its own row: input ring [D0][NF][HIN][32] chunks,
    // level rings [K-1][DL][NF][HIN][32][V] floats
    W *const in_own = reinterpret_cast<W *>(smem_raw) + (size_t)w * 32 + lane;
    float *const lv_own = reinterpret_cast<float *>(smem_raw + Sh::in_bytes) + ((size_t)w * 32 + lane) * V;
    constexpr size_t IN_FLD = (size_t)HIN * 32, IN_SLOT = NF * IN_FLD;   // chunks
    constexpr size_t LV_FLD = (size_t)HIN * 32 * V, LV_SLOT = NF * LV_FLD, LV_LEVEL = DL * LV_SLOT;  // floats
    auto extend = [&](float *ext) {
#pragma unroll
        for (int h = 0; h < r; ++h) {
            ext[h] = __shfl_up_sync(FULL, ext[V + h], 1);
            ext[r + V + h] = __shfl_down_sync(FULL, ext[r + h], 1);
        }
    };
    // V cells of field f at row offset dy of level-s plane q (s = 0: the input ring)
    auto chunk = [&](int s, int q, int f, int dy, float *dst) {
        if (s == 0) {
            union { W c; T t[V]; } u;
            u.c = in_own[(size_t)(q % D0) * IN_SLOT + f * IN_FLD + dy * 32];
#pragma unroll
            for (int i = 0; i < V; ++i) dst[i] = to_c(u.t[i]);
        } else {
            const float4 v4 = *reinterpret_cast<const float4 *>(
                lv_own + (size_t)(s - 1) * LV_LEVEL + (size_t)(q % DL) * LV_SLOT + f * LV_FLD + dy * 32 * V);
            dst[0] = v4.x;
            dst[1] = v4.y;
            dst[2] = v4.z;
            dst[3] = v4.w;
        }
    };

    const int tiles = tiles_x * tiles_y;
    for (long long it = blockIdx.x; it < (long long)tiles * segs; it += gridDim.x) {
        const int seg = (int)(it / tiles), tile = (int)(it - (long long)seg * tiles);
        const int z0 = (int)((long long)seg * nz / segs), z1 = (int)((long long)(seg + 1) * nz / segs);
        const int x0 = (tile % tiles_x) * Sh::TX, y0 = (tile / tiles_x) * TY;
        const int n = (z1 - z0) + 2 * K * r;
        const int niter = n + K - 1;
        const int col = x0 + (lane - 1) * V;
        const size_t goff = (size_t)wrap_idx(y0 - K * r + w, ny) * nx + wrap_idx(col, nx);
        const int yo = y0 - K * r + w;
        const bool store = w >= K * r && w < HIN - K * r && lane >= 1 && lane <= 30 && col < nx && yo < ny;
        int jn = 0, zn = wrap_idx(z0 - K * r, nz);
        size_t src = (size_t)zn * plane + goff;
        size_t dst_off = (size_t)z0 * plane + (size_t)yo * nx + col;
        auto issue = [&]() {
            if (jn < n) {
                W *dst = in_own + (size_t)(jn % D0) * IN_SLOT;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    if constexpr (CB == 16) cp_async16(dst + f * IN_FLD, in[f] + src);
                    else cp_async8(dst + f * IN_FLD, in[f] + src);
                }
                src += plane;
                if (++zn == nz) {
                    zn = 0;
                    src -= (size_t)nz * plane;
                }
            }
            ++jn;
            cp_async_commit();
        };
#pragma unroll
        for (int j = 0; j < P; ++j) issue();

        for (int j = 0; j < niter; ++j) {
            cp_async_wait<P - 1>();
            // input plane j and the level planes of iteration j-1 published; the
            // slots written below are no longer read
            __syncthreads();
            issue();
#pragma unroll
            for (int s = 1; s <= K; ++s) {
                const int t = j - (s - 1) - s * r;                 // plane of level s produced now
                if (w >= s * r && w < HIN - s * r && t >= s * r && t < n - s * r) {
                    float S[NF][V], cen[NF][V], res[NF][V];
                    if constexpr (MODEL == MC) {
                        // phi's stencil, and that of the density's chemical potential
                        // m = mc_mu(phi, rho) formed at every tap (per lane, then shuffled)
                        auto row0 = [&](int dz, int dy, float *dst) { chunk(s - 1, t + dz, 0, dy, dst); };
                        ring_stencil<ST>(row0, extend, S[0], cen[0]);
                        auto rowm = [&](int dz, int dy, float *dst) {
                            float u4[V], v4[V];
                            chunk(s - 1, t + dz, 0, dy, u4);
                            chunk(s - 1, t + dz, 1, dy, v4);
#pragma unroll
                            for (int c = 0; c < V; ++c) dst[c] = mc_mu<float>(u4[c], v4[c], kc);
                        };
                        ring_stencil<ST>(rowm, extend, S[1], cen[1]);
                        float vc[V];
                        chunk(s - 1, t, 1, 0, vc);
#pragma unroll
                        for (int c = 0; c < V; ++c)
                            mc_update<float>(cen[0][c], vc[c], S[0][c], S[1][c], kc, res[0][c], res[1][c]);
                    } else {
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        auto row = [&](int dz, int dy, float *dst) { chunk(s - 1, t + dz, f, dy, dst); };
                        ring_stencil<ST>(row, extend, S[f], cen[f]);
                    }
#pragma unroll
                    for (int q = 0; q < V2; ++q) {
                        const int c0 = 2 * q;
                        auto pr = [&](const float *a) { return make_float2(a[c0], a[c0 + 1]); };
                        float2 a0, a1 = make_float2(0.f, 0.f);
                        if constexpr (MODEL == AC) a0 = ac_update2(pr(cen[0]), pr(S[0]), k2);
                        else gs_update2(pr(cen[0]), pr(cen[NF - 1]), pr(S[0]), pr(S[NF - 1]), k2, a0, a1);
                        res[0][c0] = a0.x;
                        res[0][c0 + 1] = a0.y;
                        res[NF - 1][c0] = NF == 2 ? a1.x : a0.x;
                        res[NF - 1][c0 + 1] = NF == 2 ? a1.y : a0.y;
                    }
                    }
                    if (s < K) {
#pragma unroll
                        for (int f = 0; f < NF; ++f)
                            *reinterpret_cast<float4 *>(lv_own + (size_t)(s - 1) * LV_LEVEL +
                                                        (size_t)(t % DL) * LV_SLOT + f * LV_FLD) =
                                make_float4(to_c(from_c<T>(res[f][0])), to_c(from_c<T>(res[f][1])),
                                            to_c(from_c<T>(res[f][2])), to_c(from_c<T>(res[f][3])));
                    } else {
                        if (store) {
                            store_vec<T, V>(out[0] + dst_off, res[0]);
                            if constexpr (NF == 2) store_vec<T, V>(out[NF - 1] + dst_off, res[NF - 1]);
                        }
                        dst_off += plane;
                    }
                }
            }
        }
        cp_async_wait<0>();
        __syncthreads();
    }
}

// ================================================== 3D, asynchronous ring ==
//
// FP32 / BF16-storage 3D kernel.  A thread owns one 16-byte chunk of V cells
// (V = 4 for FP32, 8 for BF16) of a TX x TY tile and the CTA streams along z.
// Input planes (tile plus halo: HIN rows of NCH = TX/V + 2 chunks, kept in the
// storage type) arrive through a ring of D planes in shared memory filled by
// cp.async, P planes ahead of the one being computed; each thread copies its
// own chunks and a barrier per plane publishes them.  Cahn-Hilliard computes mu
// chunk-wise over the tile rows plus r halo rows and the two halo chunks (FP32,
// a ring of 2r+1 planes) behind a second barrier.  Stencil rows are read only
// where the stencil has taps (x halos only on the centre row of the cross
// stencils).  The same expressions in the same order as the other FP32
// kernels, so results are identical to them bit for bit.
//
// Requirements (checked by the launcher): nx a multiple of V and 16-byte
// aligned field pointers, so that every chunk, wrapped or not, is one aligned
// 16-byte copy.
template <int MODEL, int ST, typename T, int TXT, int TY>
struct Step3dAsyncShape {
    typedef typename Cmp<T>::type C;
    static constexpr int V = 16 / (int)sizeof(T);
    static constexpr int r = StencilInfo<ST>::r;
    static constexpr int R = (MODEL == CH) ? 2 * r : r;
    static_assert(R <= V, "halo wider than one chunk");
    static_assert(MODEL != CH || V >= 2 * r, "halo chunk must cover the mu halo");
    static constexpr int TX = TXT * V, NT = TXT * TY;
    static constexpr int NCH = TXT + 2;              // chunks per row (one halo chunk each side)
    static constexpr int SW = NCH * V;               // row stride (cells)
    static constexpr int HIN = TY + 2 * R, PIN = HIN * SW;
    static constexpr int P = 3;                      // planes in flight
    static constexpr int D = P + 2 * r + 1;          // input ring slots
    static constexpr int HMU = TY + 2 * r, PMU = HMU * SW;
    static constexpr int DMU = (MODEL == CH) ? 2 * r + 1 : 0;
    static constexpr int NF = num_fields<MODEL>();
    static constexpr int EPT = (HIN * NCH + NT - 1) / NT;  // chunk copies per thread per field
    // plane slots start on 128-byte boundaries (tensor-map destinations)
    static constexpr int PINS = (int)(((size_t)PIN * sizeof(T) + 127) / 128 * 128 / sizeof(T));
    static constexpr int GUARD = 128;                // bytes before and after each region
    static constexpr size_t in_bytes = sizeof(T) * (size_t)NF * D * PINS;
    static constexpr size_t mu_off = GUARD + in_bytes + GUARD;
    static constexpr size_t bar_off = (mu_off + sizeof(C) * (size_t)DMU * PMU + GUARD + 7) / 8 * 8;
    // + D mbarriers + slack to align the dynamic shared memory base to 128 bytes
    static constexpr size_t smem_bytes = bar_off + 8 * (size_t)D + 128;
    static constexpr unsigned box_bytes = (unsigned)(sizeof(T) * (size_t)PIN);  // one field's plane box
};

// The V cells at p (16-byte aligned, a multiple of 16 bytes), widened to float.
template <typename T, int V>
__device__ __forceinline__ void lds_chunk(const T *p, float *w) {
    constexpr int NQ = V * (int)sizeof(T) / 16;
    static_assert(NQ * 16 == V * (int)sizeof(T), "whole 16-byte pieces");
    union { uint4 q[NQ]; T t[V]; } u;
#pragma unroll
    for (int i = 0; i < NQ; ++i) u.q[i] = reinterpret_cast<const uint4 *>(p)[i];
#pragma unroll
    for (int i = 0; i < V; ++i) w[i] = to_c(u.t[i]);
}

// Stencil sums and centre values of the V cells of chunk ci on row `row` of the
// planes pl[0 .. 2r] (z offsets -r .. r), row stride SW cells.
template <int ST, typename T, int V, int SW>
__device__ __forceinline__ void async_chunk_sums(const T *const (&pl)[2 * StencilInfo<ST>::r + 1], int row, int ci,
                                                 float (&S)[V], float (&ctr)[V]) {
    constexpr int r = StencilInfo<ST>::r;
    constexpr int W = V + 2 * r;
    float w[2 * r + 1][2 * r + 1][W];
#pragma unroll
    for (int dz = -r; dz <= r; ++dz)
#pragma unroll
        for (int dy = -r; dy <= r; ++dy) {
            const bool full = (ST == L27) || (dz == 0 && dy == 0);  // x taps on this row
            if (ST == L27 || dz == 0 || dy == 0) {
                const T *p = pl[dz + r] + (row + dy) * SW + ci * V;
                float *wr = w[dz + r][dy + r];
                lds_chunk<T, V>(p, wr + r);
                if (full && r > 0) {
                    float lq[V], rq[V];
                    lds_chunk<T, V>(p - V, lq);
                    lds_chunk<T, V>(p + V, rq);
#pragma unroll
                    for (int d = 0; d < r; ++d) {
                        wr[d] = lq[V - r + d];
                        wr[r + V + d] = rq[d];
                    }
                }
            }
        }
#pragma unroll
    for (int j = 0; j < V; ++j) {
        auto Pf = [&](int dx, int dy, int dz) -> float { return w[dz + r][dy + r][r + j + dx]; };
        S[j] = stencil_sum<ST, float>(Pf);
        ctr[j] = w[r][r][r + j];
    }
}

// TMA (family 6): the same kernel with each input plane box (tile + halo, all
// in-grid columns and rows) moved by one tensor-map load per field, issued by
// one thread into the ring slot and completed on the slot's mbarrier; chunks of
// the box outside the grid (periodic wrap, zero-filled by the load) are copied
// from their wrapped positions with plain loads, fetched one plane ahead, once
// the box has landed.  Waits are bounded: if one expires, every thread leaves
// together after the copies in flight have landed (again bounded), and the
// kernel sets *a.flag.
template <int MODEL, int ST, typename T, int TXT, int TY, bool TMA>
__global__ void __launch_bounds__(TXT * TY) step3d_async_kernel(StepArgs a, int tiles_x, int tiles_y, int segs,
                                                                const __grid_constant__ TmaMaps maps) {
    static_assert(MODEL != MC, "Model C runs on the accessor-based kernels");
    typedef Step3dAsyncShape<MODEL, ST, T, TXT, TY> Sh;
    typedef typename Sh::C C;
    constexpr int V = Sh::V, r = Sh::r, R = Sh::R, TX = Sh::TX, NT = Sh::NT, NCH = Sh::NCH, SW = Sh::SW;
    constexpr int HIN = Sh::HIN, PIN = Sh::PINS, P = Sh::P, D = Sh::D, HMU = Sh::HMU, PMU = Sh::PMU;
    constexpr int DMU = Sh::DMU, NF = Sh::NF, EPT = Sh::EPT;
    static_assert(D <= 32, "one phase bit per slot");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *sbase = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    T *s_in = reinterpret_cast<T *>(sbase + Sh::GUARD);      // [NF][D][PIN]
    C *s_mu = reinterpret_cast<C *>(sbase + Sh::mu_off);     // [DMU][PMU]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sbase + Sh::bar_off);  // [D] (TMA)
    const long long polls = a.wait_polls == 0 ? kDefaultWaitPolls : (a.wait_polls < 0 ? 0 : a.wait_polls);
    unsigned phase = 0;  // TMA: parity of the next completion of each slot's barrier
    if constexpr (TMA) {
        if (threadIdx.x == 0) {
            for (int i = 0; i < D; ++i) mbar_init(&bars[i], 1);
            mbar_init_fence();
        }
        __syncthreads();
    }

    const ConstsC<C> k(a.k, a.kf);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int t = threadIdx.x;
    const size_t plane = (size_t)nx * (size_t)ny;
    const T *in[2] = {static_cast<const T *>(a.in0), static_cast<const T *>(a.in1)};
    T *out[2] = {static_cast<T *>(a.out0), static_cast<T *>(a.out1)};
    const int tc = t % TXT, ty = t / TXT;  // output chunk of this thread

    // Work items (z segment, tile), segment-major, handed out round by round:
    // all CTAs stream the same z range at the same time, so the halo rows that
    // neighbouring tiles share are still in L2 when the second tile reads them.
    const int tiles = tiles_x * tiles_y;
    for (long long it = blockIdx.x; it < (long long)tiles * segs; it += gridDim.x) {
        const int seg = (int)(it / tiles), tile = (int)(it - (long long)seg * tiles);
        const int z0 = (int)((long long)seg * nz / segs), z1 = (int)((long long)(seg + 1) * nz / segs);
        const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
        const int nplanes = (z1 - z0) + 2 * R;

        // global (plane-relative) offsets of this thread's chunk copies, or -1; TMA:
        // only chunks outside the grid (the box's zero fill) are copied by threads
        int goff[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int q = t + e * NT;
            goff[e] = -1;
            if (q < HIN * NCH) {
                const int yi = q / NCH, ci = q - yi * NCH;
                const int y = y0 - R + yi, x = x0 - V + ci * V;
                if (!TMA || y < 0 || y >= ny || x < 0 || x + V > nx)
                    goff[e] = wrap_idx(y, ny) * nx + wrap_idx(x, nx);
            }
        }
        uint4 fx[NF][EPT];  // TMA: wrapped chunks of the next plane
        auto fetch_fix = [&](int j) {
            if (TMA && j < nplanes) {
                const size_t zoff = (size_t)wrap_idx(z0 - R + j, nz) * plane;
#pragma unroll
                for (int f = 0; f < NF; ++f)
#pragma unroll
                    for (int e = 0; e < EPT; ++e)
                        if (goff[e] >= 0) fx[f][e] = __ldg(reinterpret_cast<const uint4 *>(in[f] + zoff + goff[e]));
            }
        };
        auto put_fix = [&](int j) {
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                T *slot = s_in + ((size_t)f * D + j % D) * PIN;
#pragma unroll
                for (int e = 0; e < EPT; ++e)
                    if (goff[e] >= 0) *reinterpret_cast<uint4 *>(slot + (t + e * NT) * V) = fx[f][e];
            }
        };
        auto issue_tma = [&](int j) {
            if (t == 0 && j < nplanes) {
                fence_proxy_async_smem();  // the slot's earlier reads and writes come first
                const int sl = j % D;
                mbar_arrive_expect_tx(&bars[sl], NF * Sh::box_bytes);
                const int zc = wrap_idx(z0 - R + j, nz);
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    tma_load_3d(s_in + ((size_t)f * D + sl) * PIN, &maps.m[f], x0 - V, y0 - R, zc, &bars[sl]);
            }
        };
        auto issue = [&](int j) {
            if (TMA) {
                issue_tma(j);
                return;
            }
            if (j < nplanes) {
                const size_t zoff = (size_t)wrap_idx(z0 - R + j, nz) * plane;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    T *slot = s_in + ((size_t)f * D + j % D) * PIN;
#pragma unroll
                    for (int e = 0; e < EPT; ++e)
                        if (goff[e] >= 0) cp_async16(slot + (t + e * NT) * V, in[f] + zoff + goff[e]);
                }
            }
            cp_async_commit();  // empty groups keep the count uniform
        };
        auto in_plane = [&](int f, int j) -> const T * { return s_in + ((size_t)f * D + j % D) * PIN; };

#pragma unroll
        for (int j = 0; j < P; ++j) issue(j);
        fetch_fix(0);
        for (int j = 0; j < nplanes; ++j) {
            if constexpr (TMA) {
                const int sl = j % D;
                const bool ok = mbar_wait_bounded(&bars[sl], (phase >> sl) & 1u, polls);
                if (ok) put_fix(j);
                if (__syncthreads_or(!ok)) {  // plane j complete for every thread, or give up together
                    if (t == 0 && a.flag) atomicExch(a.flag, 1);
                    if (t == 0)
                        for (int g = j; g < j + P && g < nplanes; ++g)  // copies still in flight
                            mbar_wait_bounded(&bars[g % D], (phase >> (g % D)) & 1u, kDefaultWaitPolls);
                    __syncthreads();
                    return;
                }
                phase ^= 1u << sl;
                fetch_fix(j + 1);
            } else {
                cp_async_wait<P - 1>();
                __syncthreads();  // plane j complete for every thread; planes <= j-1 no longer read
            }
            issue(j + P);
            if constexpr (MODEL == CH) {
                if (j >= 2 * r) {
                    // mu of plane j - r over the tile rows plus r halo rows and the halo chunks
                    C *mu = s_mu + (size_t)((j - r) % DMU) * PMU;
                    const T *pl[2 * r + 1];
#pragma unroll
                    for (int d = 0; d <= 2 * r; ++d) pl[d] = in_plane(0, j - 2 * r + d);
                    for (int q = t; q < HMU * NCH; q += NT) {
                        const int ym = q / NCH, ci = q - ym * NCH;
                        float S[V], p[V];
                        async_chunk_sums<ST, T, V, SW>(pl, ym + r, ci, S, p);
                        float m[V];
#pragma unroll
                        for (int i = 0; i < V; ++i) m[i] = ch_mu<C>(p[i], S[i], k);
#pragma unroll
                        for (int i = 0; i < V; i += 4)
                            *reinterpret_cast<float4 *>(mu + ym * SW + ci * V + i) =
                                make_float4(m[i], m[i + 1], m[i + 2], m[i + 3]);
                    }
                }
                __syncthreads();
                if (j >= 4 * r) {
                    // output plane j - 2r from mu planes j - 3r .. j - r
                    const int zo = z0 - 4 * r + j;
                    const int x = x0 + tc * V, y = y0 + ty;
                    if (x < nx && y < ny) {
                        const C *plm[2 * r + 1];
#pragma unroll
                        for (int d = 0; d <= 2 * r; ++d) plm[d] = s_mu + (size_t)((j - 3 * r + d) % DMU) * PMU;
                        float S[V], dummy[V], p[V], o[V];
                        async_chunk_sums<ST, C, V, SW>(plm, ty + r, tc + 1, S, dummy);
                        lds_chunk<T, V>(in_plane(0, j - 2 * r) + (ty + R) * SW + (tc + 1) * V, p);
#pragma unroll
                        for (int i = 0; i < V; ++i) o[i] = ch_update<C>(p[i], S[i], k);
                        store_vec<T, V>(out[0] + (size_t)zo * plane + (size_t)y * nx + x, o);
                    }
                }
            } else {
                if (j >= 2 * r) {
                    // output plane j - r
                    const int zo = z0 - 2 * r + j;
                    const int x = x0 + tc * V, y = y0 + ty;
                    if (x < nx && y < ny) {
                        const T *pl0[2 * r + 1];
#pragma unroll
                        for (int d = 0; d <= 2 * r; ++d) pl0[d] = in_plane(0, j - 2 * r + d);
                        float S0[V], p0[V], o0[V], o1[V];
                        async_chunk_sums<ST, T, V, SW>(pl0, ty + r, tc + 1, S0, p0);
                        if constexpr (MODEL == AC) {
#pragma unroll
                            for (int i = 0; i < V; ++i) o0[i] = ac_update<C>(p0[i], S0[i], k);
                        } else {
                            const T *pl1[2 * r + 1];
#pragma unroll
                            for (int d = 0; d <= 2 * r; ++d) pl1[d] = in_plane(NF - 1, j - 2 * r + d);
                            float S1[V], p1[V];
                            async_chunk_sums<ST, T, V, SW>(pl1, ty + r, tc + 1, S1, p1);
#pragma unroll
                            for (int i = 0; i < V; ++i) gs_update<C>(p0[i], p1[i], S0[i], S1[i], k, o0[i], o1[i]);
                        }
                        const size_t o = (size_t)zo * plane + (size_t)y * nx + x;
                        store_vec<T, V>(out[0] + o, o0);
                        if constexpr (num_fields<MODEL>() == 2) store_vec<T, V>(out[NF - 1] + o, o1);
                    }
                }
            }
        }
        if constexpr (!TMA) cp_async_wait<0>();
        __syncthreads();  // the rings are reused by the next segment
    }  // segments
}

// ======================================================== 3D, vectorised ==
//
// FP32 / BF16-storage 3D kernel.  A thread owns V = 4 consecutive x cells of
// one row of a TX x TY tile (TX = 4*TXT, TY = TYT) and streams along z.  Plane
// slices live in shared memory as rows of NCH = TX/4 + 2 chunks of 4 cells
// (one halo chunk on each side, so any stencil radius up to 4 fits); all
// shared-memory traffic is aligned 16-byte chunks.  Cahn-Hilliard computes mu
// chunk-wise on the tile rows plus r halo rows and the two halo chunks; the
// cells of a halo chunk beyond the needed r columns read neighbours outside
// the row (kept inside the allocation by guard chunks) and are never used.
template <int MODEL, int ST, typename T, int TXT, int TYT>
struct Step3dVecShape {
    typedef typename Cmp<T>::type C;
    static constexpr int V = 4;
    static constexpr int r = StencilInfo<ST>::r;
    static constexpr int R = (MODEL == CH) ? 2 * r : r;
    static_assert(R <= V, "halo wider than one chunk");
    static constexpr int TX = TXT * V, TY = TYT, NT = TXT * TYT;
    static constexpr int NCH = TXT + 2;          // chunks per row
    static constexpr int SW = NCH * V;           // row stride (cells)
    static constexpr int HIN = TY + 2 * R;       // rows of an input plane
    static constexpr int PIN = HIN * SW;
    static constexpr int HMU = TY + 2 * r;       // rows of a mu plane
    static constexpr int PMU = HMU * SW;
    static constexpr int DIN = 2 * r + 2;
    static constexpr int DMU = (MODEL == CH) ? 2 * r + 1 : 0;
    static constexpr int NF = num_fields<MODEL>();
    static constexpr int GUARD = 2 * V;          // cells before and after the planes
    static constexpr int EPT = (HIN * NCH + NT - 1) / NT;  // input chunks per thread per field
    static constexpr size_t smem_bytes = sizeof(C) * ((size_t)2 * GUARD + (size_t)NF * DIN * PIN + (size_t)DMU * PMU);
};

// Cells [-r, V+r) around the 4-cell chunk at p (16-byte aligned) into w.
template <int r, int W>
__device__ __forceinline__ void chunk_row(const float *p, float (&w)[W]) {
    const float4 c = *reinterpret_cast<const float4 *>(p);
    w[r + 0] = c.x; w[r + 1] = c.y; w[r + 2] = c.z; w[r + 3] = c.w;
    if constexpr (r > 0) {
        const float4 lq = *reinterpret_cast<const float4 *>(p - 4);
        const float4 rq = *reinterpret_cast<const float4 *>(p + 4);
        const float l[4] = {lq.x, lq.y, lq.z, lq.w}, rr[4] = {rq.x, rq.y, rq.z, rq.w};
#pragma unroll
        for (int d = 0; d < r; ++d) {
            w[d] = l[4 - r + d];
            w[r + 4 + d] = rr[d];
        }
    }
}

// Stencil sums S and centre values of the 4 cells of the chunk at row `row`,
// chunk `ci` of the planes pl[0 .. 2r] (plane offsets -r .. r), row stride SW.
template <int ST, int SW>
__device__ __forceinline__ void chunk_sums(const float *const (&pl)[2 * StencilInfo<ST>::r + 1], int row, int ci,
                                           float (&S)[4], float (&ctr)[4]) {
    constexpr int r = StencilInfo<ST>::r;
    constexpr int W = 4 + 2 * r;
    float w[2 * r + 1][2 * r + 1][W];
#pragma unroll
    for (int dz = -r; dz <= r; ++dz)
#pragma unroll
        for (int dy = -r; dy <= r; ++dy)
            if (ST == L27 || dz == 0 || dy == 0)  // cross stencils only read the axes
                chunk_row<r, W>(pl[dz + r] + (row + dy) * SW + ci * 4, w[dz + r][dy + r]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        auto P = [&](int dx, int dy, int dz) -> float { return w[dz + r][dy + r][r + j + dx]; };
        S[j] = stencil_sum<ST, float>(P);
        ctr[j] = w[r][r][r + j];
    }
}

template <int MODEL, int ST, typename T, int TXT, int TYT>
__global__ void __launch_bounds__(TXT * TYT) step3d_vec_kernel(StepArgs a, int tiles_x, int tiles_y,
                                                               long long planes_per_cta) {
    static_assert(MODEL != MC, "Model C runs on the accessor-based kernels");
    typedef Step3dVecShape<MODEL, ST, T, TXT, TYT> Sh;
    typedef typename Sh::C C;
    constexpr int V = Sh::V, r = Sh::r, R = Sh::R, TX = Sh::TX, TY = Sh::TY, NT = Sh::NT;
    constexpr int NCH = Sh::NCH, SW = Sh::SW, HIN = Sh::HIN, PIN = Sh::PIN, HMU = Sh::HMU, PMU = Sh::PMU;
    constexpr int DIN = Sh::DIN, DMU = Sh::DMU, NF = Sh::NF, EPT = Sh::EPT;
    typedef float4 Q;  // one chunk in shared memory (C is float here)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s_in = reinterpret_cast<C *>(smem_raw) + Sh::GUARD;   // [NF][DIN][PIN]
    C *s_mu = s_in + (size_t)NF * DIN * PIN;                // [DMU][PMU]

    const ConstsC<C> k(a.k, a.kf);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int t = threadIdx.x;
    const size_t plane = (size_t)nx * (size_t)ny;
    const bool vec_ok = (nx % V) == 0;
    const T *in[2] = {static_cast<const T *>(a.in0), static_cast<const T *>(a.in1)};
    T *out[2] = {static_cast<T *>(a.out0), static_cast<T *>(a.out1)};
    // Persistent schedule over the flattened (tile, z) space (see step3d_kernel).
    long long g0 = (long long)blockIdx.x * planes_per_cta;
    const long long gend = min(g0 + planes_per_cta, (long long)tiles_x * tiles_y * nz);
    while (g0 < gend) {
    const int tile = (int)(g0 / nz);
    const int z0 = (int)(g0 - (long long)tile * nz);
    const int z1 = (int)min((long long)nz, (long long)z0 + (gend - g0));
    g0 += z1 - z0;
    const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
    const int nplanes = (z1 - z0) + 2 * R;

    // input chunks of this thread: plane-relative offset of the first cell, or -1
    int goff[EPT];
    bool gvec[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int q = t + e * NT;
        goff[e] = -1;
        gvec[e] = false;
        if (q < HIN * NCH) {
            const int yi = q / NCH, ci = q - yi * NCH;
            const int y = wrap_idx(y0 - R + yi, ny);
            const int x = x0 - V + ci * V;
            gvec[e] = vec_ok && x >= 0 && x + V <= nx;
            goff[e] = y * nx + (gvec[e] ? x : 0);
        }
    }
    C pf[NF][EPT][V];
    auto fetch = [&](int z) {
        const size_t zoff = (size_t)wrap_idx(z, nz) * plane;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            if (goff[e] < 0) continue;
            const int q = t + e * NT;
            const int ci = q % NCH;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                if (gvec[e]) {
                    load_vec<T, V>(in[f] + zoff + goff[e], pf[f][e]);
                } else {
                    const int x = x0 - V + ci * V;
#pragma unroll
                    for (int j = 0; j < V; ++j) pf[f][e][j] = load_one(in[f] + zoff + goff[e] + wrap_idx(x + j, nx));
                }
            }
        }
    };
    auto commit = [&](int slot) {
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            if (goff[e] < 0) continue;
            const int q = t + e * NT;
#pragma unroll
            for (int f = 0; f < NF; ++f)
                *reinterpret_cast<Q *>(s_in + ((size_t)f * DIN + slot) * PIN + q * V) =
                    make_float4(pf[f][e][0], pf[f][e][1], pf[f][e][2], pf[f][e][3]);
        }
    };
    fetch(z0 - R);
    for (int jz = 0; jz < nplanes; ++jz) {
        commit(jz % DIN);
        if (jz + 1 < nplanes) fetch(z0 - R + jz + 1);
        __syncthreads();
        if constexpr (MODEL == CH) {
            if (jz >= 2 * r) {
                C *mu = s_mu + (size_t)((jz - 2 * r) % DMU) * PMU;
                const C *pl[2 * r + 1];
#pragma unroll
                for (int d = 0; d <= 2 * r; ++d) pl[d] = s_in + (size_t)((jz - 2 * r + d) % DIN) * PIN;
                for (int q = t; q < HMU * NCH; q += NT) {
                    const int ym = q / NCH, ci = q - ym * NCH;
                    C S[V], p[V], m[V];
                    chunk_sums<ST, SW>(pl, ym + r, ci, S, p);
#pragma unroll
                    for (int j = 0; j < V; ++j) m[j] = ch_mu<C>(p[j], S[j], k);
                    *reinterpret_cast<Q *>(mu + ym * SW + ci * V) = make_float4(m[0], m[1], m[2], m[3]);
                }
            }
            __syncthreads();
            if (jz >= 4 * r) {
                const int zo = z0 + jz - 4 * r;
                const int tx = t % TXT, ty = t / TXT;
                const int x = x0 + tx * V, y = y0 + ty;
                if (y < ny && x < nx) {
                    const C *plm[2 * r + 1];
#pragma unroll
                    for (int d = 0; d <= 2 * r; ++d) plm[d] = s_mu + (size_t)((jz - 4 * r + d) % DMU) * PMU;
                    C S[V], dummy[V], o[V];
                    chunk_sums<ST, SW>(plm, ty + r, tx + 1, S, dummy);
                    const C *pc = s_in + (size_t)((jz - 2 * r) % DIN) * PIN + (ty + R) * SW + (tx + 1) * V;
                    const Q c = *reinterpret_cast<const Q *>(pc);
                    const C p[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
                    for (int j = 0; j < V; ++j) o[j] = ch_update<C>(p[j], S[j], k);
                    T *dst = out[0] + (size_t)zo * plane + (size_t)y * nx;
                    if (vec_ok && x + V <= nx) store_vec<T, V>(dst + x, o);
                    else
                        for (int j = 0; j < V; ++j)
                            if (x + j < nx) dst[x + j] = from_c<T>(o[j]);
                }
            }
        } else {
            if (jz >= 2 * r) {
                const int zo = z0 + jz - 2 * r;
                const int tx = t % TXT, ty = t / TXT;
                const int x = x0 + tx * V, y = y0 + ty;
                if (y < ny && x < nx) {
                    const C *pl0[2 * r + 1];
#pragma unroll
                    for (int d = 0; d <= 2 * r; ++d) pl0[d] = s_in + (size_t)((jz - 2 * r + d) % DIN) * PIN;
                    C S0[V], p0[V], o0[V], o1[V];
                    chunk_sums<ST, SW>(pl0, ty + r, tx + 1, S0, p0);
                    if constexpr (MODEL == AC) {
#pragma unroll
                        for (int j = 0; j < V; ++j) o0[j] = ac_update<C>(p0[j], S0[j], k);
                    } else {
                        const C *pl1[2 * r + 1];
#pragma unroll
                        for (int d = 0; d <= 2 * r; ++d)
                            pl1[d] = s_in + ((size_t)(NF - 1) * DIN + (jz - 2 * r + d) % DIN) * PIN;
                        C S1[V], p1[V];
                        chunk_sums<ST, SW>(pl1, ty + r, tx + 1, S1, p1);
#pragma unroll
                        for (int j = 0; j < V; ++j) gs_update<C>(p0[j], p1[j], S0[j], S1[j], k, o0[j], o1[j]);
                    }
                    const size_t o = (size_t)zo * plane + (size_t)y * nx;
                    T *dst0 = out[0] + o;
                    if (vec_ok && x + V <= nx) store_vec<T, V>(dst0 + x, o0);
                    else
                        for (int j = 0; j < V; ++j)
                            if (x + j < nx) dst0[x + j] = from_c<T>(o0[j]);
                    if constexpr (num_fields<MODEL>() == 2) {
                        T *dst1 = out[1] + o;
                        if (vec_ok && x + V <= nx) store_vec<T, V>(dst1 + x, o1);
                        else
                            for (int j = 0; j < V; ++j)
                                if (x + j < nx) dst1[x + j] = from_c<T>(o1[j]);
                    }
                }
            }
        }
    }
    __syncthreads();  // the rings are reused by the next segment
    }  // segments
}

}  // namespace sp

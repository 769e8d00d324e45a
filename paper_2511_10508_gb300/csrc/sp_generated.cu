// sp_generated.cu -- cross Laplacians of any even accuracy order, generated at
// run time (the paper generates stencils from polynomial interpolation, Sec.
// "Compile-Time Stencil Generation"), and the step kernels that use them.
//
// Weights: on the points -r..r (r = order/2) the symmetric weights w_0..w_r of
// the central second derivative make it exact on polynomials of degree <= 2r+1:
//   sum_{j>=1} w_j j^(2m) = [m == 1]  (m = 1..r),   w_0 = -2 sum_{j>=1} w_j.
// The system is solved exactly in rational arithmetic and each weight is then
// rounded once to FP64, so the values do not depend on the solver.  In d
// dimensions the cross Laplacian is (1/h^2) [d w_0 f_0 + sum_j w_j P_j] with
// P_j = ((f(+j e_x) + f(-j e_x)) + (f(+j e_y) + f(-j e_y))) [+ (z pair)], in the
// fixed order  acc = w_r P_r; acc = fma(w_j, P_j, acc) for j = r-1..1;
// S = fma(d w_0, f_0, acc).  2D FP32 / BF16 grids use shared-memory tiles (one
// pass, mu in shared memory); FP64 (bound by the FP64 pipe, where the halo mu
// of a tile would cost more than it saves) and 3D grids use per-point kernels
// (a block per 256-point row segment, tap offsets computed once per segment;
// Cahn-Hilliard takes two passes through a mu buffer).
#include <cstdint>
#include <cstdlib>
#include <type_traits>

#include "sp_internal.h"

namespace sp {

// ------------------------------------------------------ exact weights --

namespace {
struct Rat {
    __int128 p, q;  // q > 0, gcd(p, q) = 1
};
__int128 gcd128(__int128 a, __int128 b) {
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b) {
        const __int128 t = a % b;
        a = b;
        b = t;
    }
    return a ? a : 1;
}
Rat mk(__int128 p, __int128 q) {
    if (q < 0) p = -p, q = -q;
    const __int128 g = gcd128(p, q);
    return {p / g, q / g};
}
Rat add(Rat a, Rat b) { return mk(a.p * b.q + b.p * a.q, a.q * b.q); }
Rat sub(Rat a, Rat b) { return mk(a.p * b.q - b.p * a.q, a.q * b.q); }
Rat mul(Rat a, Rat b) { return mk(a.p * b.p, a.q * b.q); }
Rat dvd(Rat a, Rat b) { return mk(a.p * b.q, a.q * b.p); }
}  // namespace

// Exact weights w_0..w_r of the central second derivative of accuracy `order`
// (even, 2..8) as numerator / denominator pairs.
static bool exact_weights(int order, Rat *w) {
    if (order < 2 || order > 2 * kMaxGenRadius || order % 2) return false;
    const int r = order / 2;
    Rat A[kMaxGenRadius][kMaxGenRadius + 1];
    for (int m = 1; m <= r; ++m) {
        for (int j = 1; j <= r; ++j) {
            __int128 v = 1;
            for (int e = 0; e < 2 * m; ++e) v *= j;
            A[m - 1][j - 1] = mk(v, 1);
        }
        A[m - 1][r] = mk(m == 1 ? 1 : 0, 1);
    }
    for (int c = 0; c < r; ++c) {  // Gauss-Jordan elimination
        int piv = c;
        while (piv < r && A[piv][c].p == 0) ++piv;
        if (piv == r) return false;
        if (piv != c)
            for (int k = 0; k <= r; ++k) std::swap(A[c][k], A[piv][k]);
        const Rat pv = A[c][c];
        for (int k = 0; k <= r; ++k) A[c][k] = dvd(A[c][k], pv);
        for (int i = 0; i < r; ++i)
            if (i != c && A[i][c].p != 0) {
                const Rat f = A[i][c];
                for (int k = 0; k <= r; ++k) A[i][k] = sub(A[i][k], mul(f, A[c][k]));
            }
    }
    Rat s = mk(0, 1);
    for (int j = 1; j <= r; ++j) {
        w[j] = A[j - 1][r];
        s = add(s, w[j]);
    }
    w[0] = mul(mk(-2, 1), s);
    return true;
}

// p/q rounded once to FP64 (p and q are far below 2^53 for these orders)
static double to_double(Rat a) { return (double)(long long)a.p / (double)(long long)a.q; }

int generated_weights(int order, int dims, double *wk, double *lambda_max) {
    Rat w[kMaxGenRadius + 1];
    if (!exact_weights(order, w) || (dims != 2 && dims != 3)) return SP_EINVAL;
    const int r = order / 2;
    wk[0] = to_double(mul(mk(dims, 1), w[0]));
    for (int j = 1; j <= r; ++j) wk[j] = to_double(w[j]);
    if (lambda_max) {  // largest eigenvalue of -h^2 L_h: theta = pi on every axis
        Rat one = w[0];
        for (int j = 1; j <= r; ++j) one = add(one, mul(mk(j % 2 ? -2 : 2, 1), w[j]));
        *lambda_max = to_double(mul(mk(-dims, 1), one));
    }
    return SP_OK;
}

// -------------------------------------------------------------- kernels --

struct GenW {
    double w[kMaxGenRadius + 1];  // d w_0, w_1, ..., w_r
    float wf[kMaxGenRadius + 1];
};

template <int R>
struct GenTaps {
    size_t zb[2 * R + 1], yb[2 * R + 1];
    __device__ __forceinline__ GenTaps(int y, int z, int nx, int ny, int nz) {
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

template <typename C> __device__ __forceinline__ C gw(const GenW &W, int j);
template <> __device__ __forceinline__ double gw<double>(const GenW &W, int j) { return W.w[j]; }
template <> __device__ __forceinline__ float gw<float>(const GenW &W, int j) { return W.wf[j]; }

// S of the generated cross stencil from an accessor P(dx, dy, dz)
template <int R, int DIMS, typename C, typename Acc>
__device__ __forceinline__ C gen_sum(const Acc &P, const GenW &W) {
    C acc = C(0);
#pragma unroll
    for (int j = R; j >= 1; --j) {
        C pj = (P(j, 0, 0) + P(-j, 0, 0)) + (P(0, j, 0) + P(0, -j, 0));
        if constexpr (DIMS == 3) pj = pj + (P(0, 0, j) + P(0, 0, -j));
        acc = (j == R) ? gw<C>(W, j) * pj : FMA(gw<C>(W, j), pj, acc);
    }
    return FMA(gw<C>(W, 0), P(0, 0, 0), acc);
}

struct GenArgs {
    StepArgs a;
    GenW W;
    void *mu;
};

__device__ __forceinline__ void gen_seg(long long u, int segs, const StepArgs &a, int &x, int &y, int &z,
                                        size_t &row) {
    const long long r = u / segs;
    x = (int)(u - r * segs) * 256 + (int)threadIdx.x;
    y = (int)(r % a.ny);
    z = (int)(r / a.ny);
    row = (size_t)r * a.nx;
}

// Cahn-Hilliard pass 1: mu of every point
template <int R, int DIMS, typename T>
__global__ void __launch_bounds__(256) gen_mu_kernel(GenArgs g, int segs) {
    typedef typename Cmp<T>::type C;
    const StepArgs &a = g.a;
    const ConstsC<C> k(a.k, a.kf);
    const T *p = static_cast<const T *>(a.in0);
    C *mu = static_cast<C *>(g.mu);
    const long long units = (long long)a.ny * a.nz * segs;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        int x, y, z;
        size_t row;
        gen_seg(u, segs, a, x, y, z, row);
        const GenTaps<R> tp(y, z, a.nx, a.ny, a.nz);
        if (x >= a.nx) continue;
        auto P = [&](int dx, int dy, int dz) -> C { return to_c(p[tp.at(x, a.nx, dx, dy, dz)]); };
        mu[row + x] = ch_mu<C>(to_c(p[row + x]), gen_sum<R, DIMS, C>(P, g.W), k);
    }
}

// one step of the model (Cahn-Hilliard: pass 2, from mu)
template <int MODEL, int R, int DIMS, typename T>
__global__ void __launch_bounds__(256) gen_step_kernel(GenArgs g, int segs) {
    typedef typename Cmp<T>::type C;
    const StepArgs &a = g.a;
    const ConstsC<C> k(a.k, a.kf);
    const T *i0 = static_cast<const T *>(a.in0), *i1 = static_cast<const T *>(a.in1);
    T *o0 = static_cast<T *>(a.out0), *o1 = static_cast<T *>(a.out1);
    const long long units = (long long)a.ny * a.nz * segs;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        int x, y, z;
        size_t row;
        gen_seg(u, segs, a, x, y, z, row);
        const GenTaps<R> tp(y, z, a.nx, a.ny, a.nz);
        if (x >= a.nx) continue;
        const size_t i = row + x;
        auto P0 = [&](int dx, int dy, int dz) -> C { return to_c(i0[tp.at(x, a.nx, dx, dy, dz)]); };
        if constexpr (MODEL == CH) {
            const C *mu = static_cast<const C *>(g.mu);
            auto Pm = [&](int dx, int dy, int dz) -> C { return mu[tp.at(x, a.nx, dx, dy, dz)]; };
            o0[i] = from_c<T>(ch_update<C>(to_c(i0[i]), gen_sum<R, DIMS, C>(Pm, g.W), k));
        } else if constexpr (MODEL == AC) {
            o0[i] = from_c<T>(ac_update<C>(to_c(i0[i]), gen_sum<R, DIMS, C>(P0, g.W), k));
        } else {
            auto P1 = [&](int dx, int dy, int dz) -> C { return to_c(i1[tp.at(x, a.nx, dx, dy, dz)]); };
            C S1;
            if constexpr (MODEL == MC) {
                auto Pm = [&](int dx, int dy, int dz) -> C { return mc_mu<C>(P0(dx, dy, dz), P1(dx, dy, dz), k); };
                S1 = gen_sum<R, DIMS, C>(Pm, g.W);
            } else {
                S1 = gen_sum<R, DIMS, C>(P1, g.W);
            }
            C a0, a1;
            two_field_update<MODEL, C>(to_c(i0[i]), to_c(i1[i]), gen_sum<R, DIMS, C>(P0, g.W), S1, k, a0, a1);
            o0[i] = from_c<T>(a0);
            o1[i] = from_c<T>(a1);
        }
    }
}

// Stencil sums of RY cells of one column (rows i0 .. i0+RY-1, column j) of the
// field read by Vf(i, j): the column's values on rows i0-R .. i0+RY-1+R are read
// once into registers (rows outside [lo, hi] are clamped there: their sums are
// not used), the x taps per cell.  Each sum is gen_sum's, with the same taps in
// the same order.
template <int R, int RY, typename Val>
__device__ __forceinline__ void gen_column_sums(const Val &Vf, int i0, int j, int lo, int hi, const GenW &W,
                                                float (&S)[RY], float (&ctr)[RY]) {
    float col[RY + 2 * R];
#pragma unroll
    for (int a = 0; a < RY + 2 * R; ++a) col[a] = Vf(min(max(i0 - R + a, lo), hi), j);
#pragma unroll
    for (int b = 0; b < RY; ++b) {
        const int i = min(max(i0 + b, lo), hi);
        auto P = [&](int dx, int dy, int) -> float { return dx == 0 ? col[b + R + dy] : Vf(i, j + dx); };
        S[b] = gen_sum<R, 2, float>(P, W);
        ctr[b] = col[b + R];
    }
}

// 2D tiles (FP32 / BF16 storage): one BX x BY output tile per CTA; the tile and
// its halo (2R for Cahn-Hilliard, whose mu is evaluated on the tile grown by R,
// else R; x padded to whole 16-byte chunks) are fetched once into shared
// memory, and mu stays in shared memory, so the step is one pass over HBM.  The
// same expressions as the per-point kernels, so the results are identical.
template <int MODEL, int R, typename T, int BX, int BY>
struct GenTile2dShape {
    typedef typename Cmp<T>::type C;
    static constexpr int RIN = (MODEL == CH) ? 2 * R : R;
    static constexpr int CK = 16 / sizeof(T);
    static constexpr int HC = (RIN + CK - 1) / CK;
    static constexpr int NCK = BX / CK + 2 * HC;
    static constexpr int SW = NCK * CK, X0 = HC * CK;
    static constexpr int HIN = BY + 2 * RIN;
    static constexpr int NF = num_fields<MODEL>();
    static constexpr int WMU = (MODEL == CH) ? BX + 2 * R : 0, HMU = (MODEL == CH) ? BY + 2 * R : 0;
    static constexpr size_t bytes_in = sizeof(T) * (size_t)NF * HIN * SW;
    static constexpr size_t smem_bytes = bytes_in + sizeof(C) * (size_t)WMU * HMU;
    static_assert(bytes_in % 16 == 0, "mu array alignment");
};

template <int MODEL, int R, typename T, int BX, int BY, int NT>
__global__ void __launch_bounds__(NT) gen_tile2d_kernel(GenArgs g) {
    typedef GenTile2dShape<MODEL, R, T, BX, BY> Sh;
    typedef typename Sh::C C;
    constexpr int RIN = Sh::RIN, CK = Sh::CK, NCK = Sh::NCK, SW = Sh::SW, X0 = Sh::X0, HIN = Sh::HIN;
    constexpr int NF = Sh::NF, WMU = Sh::WMU, HMU = Sh::HMU;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_in = reinterpret_cast<T *>(smem_raw);                 // [NF][HIN][SW]
    C *s_mu = reinterpret_cast<C *>(smem_raw + Sh::bytes_in);  // [HMU][WMU]
    const StepArgs &a = g.a;
    const ConstsC<C> k(a.k, a.kf);
    const int nx = a.nx, ny = a.ny, t = threadIdx.x;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const bool vec_ok = (nx % CK) == 0;
    const T *in[2] = {static_cast<const T *>(a.in0), static_cast<const T *>(a.in1)};
    T *out[2] = {static_cast<T *>(a.out0), static_cast<T *>(a.out1)};

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
                for (int j = 0; j < CK; ++j) dst[j] = in[f][row + wrap_idx(x + j, nx)];
            }
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();

    // value of field f at tile coordinates (i, j), -RIN <= i < BY + RIN, -X0 <= j < BX + X0
    auto phi = [&](int f, int i, int j) -> C { return to_c(s_in[((size_t)f * HIN + i + RIN) * SW + j + X0]); };
    // Each work item is a column of RY cells (register-blocked along y, see
    // gen_column_sums); consecutive threads take consecutive columns.
    constexpr int RY = 8;
    if constexpr (MODEL == CH) {
        constexpr int NB = (HMU + RY - 1) / RY;  // row blocks of the mu region
        auto phi0 = [&](int i, int j) -> C { return phi(0, i, j); };
        for (int q = t; q < NB * WMU; q += NT) {
            const int b = q / WMU, j = q - b * WMU - R;
            const int i0 = b * RY - R;
            float S[RY], p[RY];
            gen_column_sums<R, RY>(phi0, i0, j, -RIN, BY + RIN - 1, g.W, S, p);
#pragma unroll
            for (int c = 0; c < RY; ++c)
                if (i0 + c < BY + R) s_mu[(i0 + c + R) * WMU + (j + R)] = ch_mu<C>(p[c], S[c], k);
        }
        __syncthreads();
    }
    constexpr int NBO = (BY + RY - 1) / RY;  // row blocks of the output tile
    for (int q = t; q < NBO * BX; q += NT) {
        const int b = q / BX, j = q - b * BX;
        const int i0 = b * RY;
        const int x = x0 + j;
        float o0[RY], o1[RY];
        if constexpr (MODEL == CH) {
            auto mu = [&](int i, int jj) -> C { return s_mu[(i + R) * WMU + (jj + R)]; };
            float S[RY], dummy[RY];
            gen_column_sums<R, RY>(mu, i0, j, -R, BY + R - 1, g.W, S, dummy);
#pragma unroll
            for (int c = 0; c < RY; ++c) o0[c] = ch_update<C>(phi(0, min(i0 + c, BY - 1), j), S[c], k);
        } else {
            auto phi0 = [&](int i, int jj) -> C { return phi(0, i, jj); };
            float S0[RY], p0[RY];
            gen_column_sums<R, RY>(phi0, i0, j, -RIN, BY + RIN - 1, g.W, S0, p0);
            if constexpr (MODEL == AC) {
#pragma unroll
                for (int c = 0; c < RY; ++c) o0[c] = ac_update<C>(p0[c], S0[c], k);
            } else {
                float S1[RY], p1[RY];
                if constexpr (MODEL == MC) {
                    auto m = [&](int i, int jj) -> C { return mc_mu<C>(phi(0, i, jj), phi(NF - 1, i, jj), k); };
                    gen_column_sums<R, RY>(m, i0, j, -RIN, BY + RIN - 1, g.W, S1, p1);
                } else {
                    auto phi1 = [&](int i, int jj) -> C { return phi(NF - 1, i, jj); };
                    gen_column_sums<R, RY>(phi1, i0, j, -RIN, BY + RIN - 1, g.W, S1, p1);
                }
#pragma unroll
                for (int c = 0; c < RY; ++c)
                    two_field_update<MODEL, C>(p0[c], phi(NF - 1, min(i0 + c, BY - 1), j), S0[c], S1[c], k, o0[c],
                                               o1[c]);
            }
        }
        if (x < nx) {
#pragma unroll
            for (int c = 0; c < RY; ++c) {
                const int y = y0 + i0 + c;
                if (i0 + c < BY && y < ny) {
                    const size_t o = (size_t)y * (size_t)nx + x;
                    out[0][o] = from_c<T>(o0[c]);
                    if constexpr (NF == 2) out[NF - 1][o] = from_c<T>(o1[c]);
                }
            }
        }
    }
}

template <int MODEL, int R, int DIMS, typename T>
static cudaError_t launch_gen_t(const GenArgs &g, cudaStream_t s, int n_sm) {
    if constexpr (DIMS == 2 && !std::is_same<T, double>::value) {
        // family 0: shared-memory tiles; family 1: the per-point kernels
        if (g_step_variant != 1) {
            constexpr int BX = 128, BY = 32, NT = 256;
            typedef GenTile2dShape<MODEL, R, T, BX, BY> Sh;
            auto kern = gen_tile2d_kernel<MODEL, R, T, BX, BY, NT>;
            static const bool attr = [&] {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
                return true;
            }();
            (void)attr;
            kern<<<dim3((g.a.nx + BX - 1) / BX, (g.a.ny + BY - 1) / BY), NT, Sh::smem_bytes, s>>>(g);
            return cudaGetLastError();
        }
    }
    const int segs = (g.a.nx + 255) / 256;
    const long long units = (long long)g.a.ny * g.a.nz * segs;
    const unsigned blocks = (unsigned)std::min<long long>(units, (long long)n_sm * 8);
    if constexpr (MODEL == CH) gen_mu_kernel<R, DIMS, T><<<blocks, 256, 0, s>>>(g, segs);
    gen_step_kernel<MODEL, R, DIMS, T><<<blocks, 256, 0, s>>>(g, segs);
    return cudaGetLastError();
}

template <int MODEL, typename T>
static cudaError_t launch_gen_r(int r, int dims, const GenArgs &g, cudaStream_t s, int n_sm) {
#define SP_GEN(RR)                                                                            \
    case RR:                                                                                  \
        return dims == 2 ? launch_gen_t<MODEL, RR, 2, T>(g, s, n_sm) : launch_gen_t<MODEL, RR, 3, T>(g, s, n_sm);
    switch (r) {
        SP_GEN(1) SP_GEN(2) SP_GEN(3) SP_GEN(4)
    }
#undef SP_GEN
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t launch_gen_m(int model, int r, int dims, const GenArgs &g, cudaStream_t s, int n_sm) {
    switch (model) {
    case AC: return launch_gen_r<AC, T>(r, dims, g, s, n_sm);
    case CH: return launch_gen_r<CH, T>(r, dims, g, s, n_sm);
    case GS: return launch_gen_r<GS, T>(r, dims, g, s, n_sm);
    case MC: return launch_gen_r<MC, T>(r, dims, g, s, n_sm);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_generated(int model, int dtype, int order, int dims, const double *wk, const StepArgs &a, void *mu,
                             cudaStream_t s, int n_sm) {
    GenArgs g;
    g.a = a;
    g.mu = mu;
    const int r = order / 2;
    for (int j = 0; j <= kMaxGenRadius; ++j) {
        g.W.w[j] = j <= r ? wk[j] : 0.0;
        g.W.wf[j] = (float)g.W.w[j];
    }
    switch (dtype) {
    case SP_F64: return launch_gen_m<double>(model, r, dims, g, s, n_sm);
    case SP_F32: return launch_gen_m<float>(model, r, dims, g, s, n_sm);
    default: return launch_gen_m<bf16>(model, r, dims, g, s, n_sm);
    }
}

}  // namespace sp

extern "C" int sp_stencil_weights(int order, int dims, double *w, double *lambda_max) {
    if (!w) return SP_EINVAL;
    return sp::generated_weights(order, dims, w, lambda_max);
}

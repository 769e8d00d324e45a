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

// Stencil sums of a block of 4 columns x RY rows (columns j .. j+3, j a
// multiple of 4; rows i0 .. i0+RY-1) of the field read by L(i, jc, dst), which
// loads the 4 values of row i at columns jc .. jc+3 (jc a multiple of 4; the
// caller's L clamps rows outside its region, whose sums are then not used).
// The block's columns are read once over rows i0-R .. i0+RY-1+R (the y taps),
// and each output row once more 4 columns to the left and to the right (the x
// taps): 16-byte reads, about 1.25 per cell for RY = 4.  Each sum is gen_sum's,
// with the same taps in the same order, evaluated two cells per instruction.
template <int R, int RY, typename Ld>
__device__ __forceinline__ void gen_block_sums(const Ld &L, int i0, int j, const GenW &W, float (&S)[RY][4],
                                               float (&ctr)[RY][4]) {
    static_assert(R <= 4, "the x taps reach at most 4 columns beyond the block");
    float col[RY + 2 * R][4];
#pragma unroll
    for (int a = 0; a < RY + 2 * R; ++a) L(i0 - R + a, j, col[a]);
#pragma unroll
    for (int b = 0; b < RY; ++b) {
        float row[12];
        L(i0 + b, j - 4, row);
#pragma unroll
        for (int c = 0; c < 4; ++c) row[4 + c] = col[b + R][c];
        L(i0 + b, j + 4, row + 8);
        // two cells per instruction (each lane rounds as the scalar operation):
        // y pairs always, x pairs where the shifted cells form a register pair
#pragma unroll
        for (int c = 0; c < 4; c += 2) {
            const int x = 4 + c;
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int jj = R; jj >= 1; --jj) {
                float2 xp;
                if (jj % 2 == 0) xp = add2(make_float2(row[x + jj], row[x + 1 + jj]), make_float2(row[x - jj], row[x + 1 - jj]));
                else xp = make_float2(row[x + jj] + row[x - jj], row[x + 1 + jj] + row[x + 1 - jj]);
                const float2 yp = add2(make_float2(col[b + R + jj][c], col[b + R + jj][c + 1]),
                                       make_float2(col[b + R - jj][c], col[b + R - jj][c + 1]));
                const float2 pj = add2(xp, yp);
                const float2 w = splat2(W.wf[jj]);
                acc = (jj == R) ? mul2(w, pj) : fma2(w, pj, acc);
            }
            const float2 s2 = fma2(splat2(W.wf[0]), make_float2(row[x], row[x + 1]), acc);
            S[b][c] = s2.x;
            S[b][c + 1] = s2.y;
            ctr[b][c] = row[x];
            ctr[b][c + 1] = row[x + 1];
        }
    }
}

// 2D tiles (FP32 / BF16 storage): one BX x BY output tile per CTA; the tile and
// its halo (2R rows for Cahn-Hilliard, whose mu is evaluated on the tile grown
// by R, else R; 8 or 4 columns, so that every 4-column block can read 4 columns
// beyond itself) are fetched once into shared memory, and mu stays in shared
// memory (columns -4 .. BX+3), so the step is one pass over HBM.  Each thread
// takes blocks of 4 columns x 4 rows (gen_block_sums); consecutive threads take
// consecutive column blocks.  The same expressions as the per-point kernels, so
// the results are identical.
template <int MODEL, int R, typename T, int BX, int BY>
struct GenTile2dShape {
    typedef typename Cmp<T>::type C;
    static constexpr int RIN = (MODEL == CH) ? 2 * R : R;
    static constexpr int CK = 16 / sizeof(T);
    static constexpr int XH = (MODEL == CH) ? 8 : 4;  // halo columns in shared memory
    static constexpr int HC = (XH + CK - 1) / CK;
    static constexpr int NCK = BX / CK + 2 * HC;
    static constexpr int SW = NCK * CK, X0 = HC * CK;
    static constexpr int HIN = BY + 2 * RIN;
    static constexpr int NF = num_fields<MODEL>();
    static constexpr int RY = 4;   // rows per block of the output stage
    static constexpr int RYM = 5;  // rows per block of the mu stage (Cahn-Hilliard)
    static constexpr int WMU = (MODEL == CH) ? BX + 8 : 0, HMU = (MODEL == CH) ? BY + 2 * R : 0;
    static constexpr size_t bytes_in = sizeof(T) * (size_t)NF * HIN * SW;
    static constexpr size_t smem_bytes = bytes_in + sizeof(C) * (size_t)WMU * HMU;
    static_assert(bytes_in % 16 == 0 && BX % 4 == 0 && BY % RY == 0, "aligned rows and whole blocks");
};

// three CTAs per SM where the registers allow it without spills (one-field models)
template <int MODEL, int R, typename T, int BX, int BY, int NT>
__global__ void __launch_bounds__(NT, (MODEL == GS || MODEL == MC) ? 2 : 3) gen_tile2d_kernel(GenArgs g) {
    typedef GenTile2dShape<MODEL, R, T, BX, BY> Sh;
    typedef typename Sh::C C;
    constexpr int RIN = Sh::RIN, CK = Sh::CK, NCK = Sh::NCK, SW = Sh::SW, X0 = Sh::X0, HIN = Sh::HIN;
    constexpr int NF = Sh::NF, WMU = Sh::WMU, RY = Sh::RY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_in = reinterpret_cast<T *>(smem_raw);                 // [NF][HIN][SW]
    C *s_mu = reinterpret_cast<C *>(smem_raw + Sh::bytes_in);  // [HMU][WMU], columns -4 .. BX+3
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

    // 4 values of field f at tile row i (clamped to the fetched rows), columns jc .. jc+3
    auto ld_phi = [&](int f, int i, int jc, float *dst) {
        i = min(max(i, -RIN), BY + RIN - 1);
        const T *src = s_in + ((size_t)f * HIN + i + RIN) * SW + jc + X0;
        if constexpr (sizeof(T) == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(src);
            dst[0] = v.x, dst[1] = v.y, dst[2] = v.z, dst[3] = v.w;
        } else {
            union { uint2 w; T t[4]; } u;
            u.w = *reinterpret_cast<const uint2 *>(src);
#pragma unroll
            for (int c = 0; c < 4; ++c) dst[c] = to_c(u.t[c]);
        }
    };
    auto L0 = [&](int i, int jc, float *dst) { ld_phi(0, i, jc, dst); };
    auto L1 = [&](int i, int jc, float *dst) {
        if constexpr (MODEL == MC) {  // the density's chemical potential at every tap
            float p[4], q[4];
            ld_phi(0, i, jc, p);
            ld_phi(NF - 1, i, jc, q);
#pragma unroll
            for (int c = 0; c < 4; ++c) dst[c] = mc_mu<C>(p[c], q[c], k);
        } else {
            ld_phi(NF - 1, i, jc, dst);
        }
    };
    if constexpr (MODEL == CH) {
        constexpr int RYM = Sh::RYM;
        constexpr int NBM = (BY + 2 * R + RYM - 1) / RYM, NGM = WMU / 4;  // mu row blocks and column blocks
        for (int q = t; q < NBM * NGM; q += NT) {
            const int b = q / NGM, gc = q - b * NGM;
            const int i0 = b * RYM - R, j = gc * 4 - 4;
            float S[RYM][4], p[RYM][4];
            gen_block_sums<R, RYM>(L0, i0, j, g.W, S, p);
#pragma unroll
            for (int bb = 0; bb < RYM; ++bb)
                if (i0 + bb < BY + R)
                    *reinterpret_cast<float4 *>(s_mu + (size_t)(i0 + bb + R) * WMU + (j + 4)) =
                        make_float4(ch_mu<C>(p[bb][0], S[bb][0], k), ch_mu<C>(p[bb][1], S[bb][1], k),
                                    ch_mu<C>(p[bb][2], S[bb][2], k), ch_mu<C>(p[bb][3], S[bb][3], k));
        }
        __syncthreads();
    }
    constexpr int NBO = BY / RY, NGO = BX / 4;
    for (int q = t; q < NBO * NGO; q += NT) {
        const int b = q / NGO, gc = q - b * NGO;
        const int i0 = b * RY, j = gc * 4;
        float o0[RY][4], o1[RY][4];
        if constexpr (MODEL == CH) {
            auto Lmu = [&](int i, int jc, float *dst) {
                i = min(max(i, -R), BY + R - 1);
                const float4 v = *reinterpret_cast<const float4 *>(s_mu + (size_t)(i + R) * WMU + jc + 4);
                dst[0] = v.x, dst[1] = v.y, dst[2] = v.z, dst[3] = v.w;
            };
            float S[RY][4], dummy[RY][4];
            gen_block_sums<R, RY>(Lmu, i0, j, g.W, S, dummy);
#pragma unroll
            for (int bb = 0; bb < RY; ++bb) {
                float p[4];
                ld_phi(0, i0 + bb, j, p);
#pragma unroll
                for (int c = 0; c < 4; ++c) o0[bb][c] = ch_update<C>(p[c], S[bb][c], k);
            }
        } else {
            float S0[RY][4], p0[RY][4];
            gen_block_sums<R, RY>(L0, i0, j, g.W, S0, p0);
            if constexpr (MODEL == AC) {
#pragma unroll
                for (int bb = 0; bb < RY; ++bb)
#pragma unroll
                    for (int c = 0; c < 4; ++c) o0[bb][c] = ac_update<C>(p0[bb][c], S0[bb][c], k);
            } else {
                float S1[RY][4], p1[RY][4];
                gen_block_sums<R, RY>(L1, i0, j, g.W, S1, p1);
#pragma unroll
                for (int bb = 0; bb < RY; ++bb) {
                    float r1[4];
                    ld_phi(NF - 1, i0 + bb, j, r1);  // rho or v itself at the centre
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        two_field_update<MODEL, C>(p0[bb][c], r1[c], S0[bb][c], S1[bb][c], k, o0[bb][c], o1[bb][c]);
                }
            }
        }
        const int x = x0 + j;
#pragma unroll
        for (int bb = 0; bb < RY; ++bb) {
            const int y = y0 + i0 + bb;
            if (y >= ny) continue;
            const size_t o = (size_t)y * (size_t)nx + x;
            if (vec_ok && x + 4 <= nx) {
                store_vec<T, 4>(out[0] + o, o0[bb]);
                if constexpr (NF == 2) store_vec<T, 4>(out[NF - 1] + o, o1[bb]);
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (x + c < nx) {
                        out[0][o + c] = from_c<T>(o0[bb][c]);
                        if constexpr (NF == 2) out[NF - 1][o + c] = from_c<T>(o1[bb][c]);
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
            // Cahn-Hilliard: 288 threads take the (BY + 2R) / 5 x (BX + 8) / 4 mu blocks
            // (up to 272) in one round and the 8 x 32 output blocks; 256 otherwise
            constexpr int BX = 128, BY = 32, NT = MODEL == CH ? 288 : 256;
            typedef GenTile2dShape<MODEL, R, T, BX, BY> Sh;
            auto kern = gen_tile2d_kernel<MODEL, R, T, BX, BY, NT>;
            static const bool attr = [&] {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem_bytes);
                // several tiles per SM overlap one tile's loads with another's arithmetic
                cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
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

// sp_spectral.cu -- semi-implicit Fourier spectral step (the paper's spectral
// solver scheme, Sec. "Construction of Semi-Implicit Fourier Spectral Scheme";
// the paper runs it on the host only), with this file's own FFTs.
//
// Linear terms are integrated implicitly in Fourier space with the continuous
// symbol -|k|^2, the cubic term explicitly in real space:
//   Allen-Cahn     L(k) = c1 - |k|^2,            N^ = (-c2 phi^3)^
//   Cahn-Hilliard  L(k) = |k|^2 (c1 - kappa |k|^2), N^ = -|k|^2 (c2 phi^3)^
//   phi^' = (phi^ + dt N^) / (1 - dt L(k)),   k = 2 pi m / (n h) per axis.
//
// Transforms.  The real-to-complex transform runs along x (the contiguous
// axis), then complex transforms along y (and z): the order of numpy's
// rfftn, whose inverse irfftn runs the complex axes first and takes the real
// part of the zero and Nyquist bins along x.  Every 1D transform is a
// mixed-radix Stockham FFT (radices 8, 4, 2, 3, 5, 7) of one line held in
// shared memory: at each stage every thread reads its butterflies' inputs into
// registers, applies the twiddles exp(-+2 pi i t / n) (a table computed once
// on the host in extended precision), takes the radix-R DFT and, after a
// barrier, writes the outputs to their sorted positions.  Two real rows are
// transformed as one complex row (real part and imaginary part) and separated
// afterwards.  Sides need prime factors 2, 3, 5, 7 and at most 4096 (FP64) or
// 8192 (FP32) points when all are powers of two, half that otherwise (a line is
// transformed by one CTA in shared memory).
//
// Layout.  The half spectrum (nx/2+1 modes along x) is stored transposed,
// x-mode slowest: Z[kx][z][y] (y fastest), so that the y transforms read
// contiguous lines and the z transforms groups of adjacent lines.  The
// resident spectrum phi^ has the same layout.
//
// One step (2D; 3D adds a forward y pass before and an inverse y pass after the
// z pass, which then holds the update):
//   rows:  phi -> cube -> forward x transforms -> Z       (first step of a call)
//   lines: Z -> forward y -> phi^ update (resident) -> scale 1/N -> inverse y -> Z
//   rows:  Z -> inverse x transforms -> phi, and, when another step follows,
//          cube -> forward x transforms -> Z for it.
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "sp_internal.h"

namespace sp {

constexpr int kFftMaxN = 8192;
constexpr int kFftMaxStages = 16;

struct FftLen {
    int n, nst;
    int rad[kFftMaxStages];
    int tw_off;  // offset (complex entries) of exp(-2 pi i t / n), t < n, in the plan's table
    // powers of two: log2 n, and the two-level table w(t) = lo[t mod 2^ls] * hi[t >> ls]
    // (lo[t] = exp(-2 pi i t / n), hi[u] = exp(-2 pi i u 2^ls / n)) at lo_off / hi_off
    int log2n, ls, lo_off, hi_off;
};

template <typename R> struct Cplx;
template <> struct Cplx<double> { typedef double2 type; };
template <> struct Cplx<float> { typedef float2 type; };

struct SpectralPlan {
    int dtype, dims, nx, ny, nz, nxh;
    size_t N, Nc;                 // real points, half-spectrum modes
    FftLen lx, ly, lz;
    void *uh, *z;                 // resident spectrum and the transform buffer (Nc complex each)
    void *tw;                     // twiddles of every axis length, then the roots of 3, 5, 7
    int roots_off;
    bool pow2;                    // every side a power of two (radices 8, 4, 2 only)
    bool nh_valid;                // z holds the transformed cubic term of the current phi
};

static std::string g_fft_err;
const char *spectral_last_error() { return g_fft_err.c_str(); }

// ------------------------------------------------------- complex helpers --

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return double2{__fma_rn(a.x, b.x, -(a.y * b.y)), __fma_rn(a.x, b.y, a.y * b.x)};
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return float2{__fmaf_rn(a.x, b.x, -(a.y * b.y)), __fmaf_rn(a.x, b.y, a.y * b.x)};
}
// multiply by -i (forward, DIR = -1) or +i (inverse)
template <int DIR, typename C> __device__ __forceinline__ C rot(C a) {
    return DIR < 0 ? C{a.y, -a.x} : C{-a.y, a.x};
}

// ------------------------------------------------------ radix-R DFTs --

template <int DIR, typename C> __device__ __forceinline__ void dft2(C &a, C &b) {
    const C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int DIR, typename C> __device__ __forceinline__ void dft4(C &u0, C &u1, C &u2, C &u3) {
    const C t0 = cadd(u0, u2), t1 = csub(u0, u2), t2 = cadd(u1, u3), t3 = rot<DIR>(csub(u1, u3));
    u0 = cadd(t0, t2);
    u2 = csub(t0, t2);
    u1 = cadd(t1, t3);
    u3 = csub(t1, t3);
}

template <int DIR, typename C> __device__ __forceinline__ void dft8(C (&u)[8]) {
    typedef decltype(u[0].x) R;
    C e0 = u[0], e1 = u[2], e2 = u[4], e3 = u[6], o0 = u[1], o1 = u[3], o2 = u[5], o3 = u[7];
    dft4<DIR>(e0, e1, e2, e3);
    dft4<DIR>(o0, o1, o2, o3);
    // o_k *= exp(DIR 2 pi i k / 8)
    const R h = (R)0.70710678118654752440;  // sqrt(1/2)
    o1 = C{h * (o1.x - DIR * o1.y), h * (o1.y + DIR * o1.x)};
    o2 = rot<DIR>(o2);
    o3 = C{h * (-o3.x - DIR * o3.y), h * (-o3.y + DIR * o3.x)};
    u[0] = cadd(e0, o0);
    u[4] = csub(e0, o0);
    u[1] = cadd(e1, o1);
    u[5] = csub(e1, o1);
    u[2] = cadd(e2, o2);
    u[6] = csub(e2, o2);
    u[3] = cadd(e3, o3);
    u[7] = csub(e3, o3);
}

// Any radix from its roots w[t] = exp(-2 pi i t / R) (conjugated for the inverse).
template <int R_, int DIR, typename C> __device__ __forceinline__ void dft_generic(C (&u)[R_], const C *w) {
    C out[R_];
#pragma unroll
    for (int m = 0; m < R_; ++m) {
        C acc = u[0];
#pragma unroll
        for (int l = 1; l < R_; ++l) {
            C r = w[(m * l) % R_];
            if (DIR > 0) r.y = -r.y;
            acc = cadd(acc, cmul(u[l], r));
        }
        out[m] = acc;
    }
#pragma unroll
    for (int m = 0; m < R_; ++m) u[m] = out[m];
}

template <int RAD, int DIR, typename C> __device__ __forceinline__ void dft(C (&u)[RAD], const C *roots) {
    if constexpr (RAD == 2) dft2<DIR>(u[0], u[1]);
    else if constexpr (RAD == 4) dft4<DIR>(u[0], u[1], u[2], u[3]);
    else if constexpr (RAD == 8) dft8<DIR>(u);
    else dft_generic<RAD, DIR>(u, roots + (RAD == 3 ? 0 : RAD == 5 ? 3 : 8));
}

// ------------------------------------------------- Stockham in shared memory --

// Shared-memory slot of complex entry i of a CTA's lines: FP32 lines are padded
// with one empty slot after every 16 entries, so that the first radix-8 stage's
// stores (stride 8 entries, 8-way bank conflicts unpadded) and the loads of every
// stage (16 consecutive entries per half-warp) are conflict-free.
template <bool PAD> __device__ __forceinline__ int slot(int i) { return PAD ? i + (i >> 4) : i; }
// entries of shared memory that e padded entries span
template <bool PAD> __host__ __device__ __forceinline__ int padded(int e) { return PAD ? e + (e >> 4) + 1 : e; }


// One radix-RAD stage on G lines of n points from buf into out (line l at
// offset l*n of each, both padded alike; one barrier, after the stores); p is
// the product of the radices of the earlier stages.  Butterfly b of a line
// (b < n/RAD) reads its inputs at stride n/RAD and writes them at stride p
// from ((b - k) * RAD + k), k = b mod p.  Each thread keeps at most QMAX
// butterflies in registers.  POW2 (every length a power of two): index
// arithmetic by shifts.  TWS: twiddles from the two-level table in shared
// memory (lo, hi), one extra complex product each (FP32, where the kernels are
// latency-bound); otherwise from the full table in global memory (FP64, where
// the FP64 pipe is the bound and the table stays in L1/L2).
template <int RAD, int QMAX, int DIR, bool POW2, bool TWS, bool PAD, typename C>
__device__ __forceinline__ void fft_stage(const C *buf, C *out, int n, int G, int p, const C *tw, const C *roots,
                                          const C *lo, const C *hi, int lg_m, int lg_p, int ls) {
    const int m = n / RAD, step = n / (p * RAD), total = G * m;
    C u[QMAX][RAD];
    int ob[QMAX];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
        const int b = threadIdx.x + q * blockDim.x;
        ob[q] = -1;
        if (b < total) {
            int line, i, k;
            if constexpr (POW2) {
                line = b >> lg_m;
                i = b & (m - 1);
                k = i & (p - 1);
            } else {
                line = b / m;
                i = b - line * m;
                k = i % p;
            }
            const int src = line * n + i;
#pragma unroll
            for (int j = 0; j < RAD; ++j) u[q][j] = buf[slot<PAD>(src + j * m)];
            if (p > 1) {
                if constexpr (TWS) {
                    // w^j for j = 1 .. RAD-1 from one table look-up of w = exp(-2 pi i k step / n)
                    // by repeated products (FP32: at most RAD-2 roundings more than a look-up
                    // per power, well inside the FP32 tolerance)
                    const int t = k * step;
                    C w1 = cmul(lo[slot<true>(t & ((1 << ls) - 1))], hi[slot<true>(t >> ls)]);
                    if (DIR > 0) w1.y = -w1.y;
                    C wj = w1;
#pragma unroll
                    for (int j = 1; j < RAD; ++j) {
                        u[q][j] = cmul(u[q][j], wj);
                        if (j + 1 < RAD) wj = cmul(wj, w1);
                    }
                } else {
#pragma unroll
                    for (int j = 1; j < RAD; ++j) {
                        C w = __ldg(tw + j * k * step);
                        if (DIR > 0) w.y = -w.y;
                        u[q][j] = cmul(u[q][j], w);
                    }
                }
            }
            dft<RAD, DIR>(u[q], roots);
            ob[q] = line * n + (i - k) * RAD + k;
        }
    }
    (void)lg_p;
#pragma unroll
    for (int q = 0; q < QMAX; ++q)
        if (ob[q] >= 0) {
#pragma unroll
            for (int j = 0; j < RAD; ++j) out[slot<PAD>(ob[q] + j * p)] = u[q][j];
        }
    __syncthreads();
}

// Work split of the transforms: at most NT threads per CTA (512 FP64, 1024
// FP32: the registers of one CTA fill the SM), VPT values of a line per thread
// (each thread holds at most VPT values of a stage: QMAX = VPT / RAD
// butterflies): 8 for powers of two, 4 for other lengths (every radix); TWS as
// above.  (FP32 with 16 values per thread: two CTAs of 512 threads per SM spilled
// registers, one CTA of 512 threads measured 10 % slower than 1024 threads.)
template <typename R, bool POW2> struct FftCfg {
    static constexpr bool f64 = sizeof(R) == 8;
    static constexpr int NT = f64 ? 512 : 1024, MINB = 1;
    static constexpr int VPT = POW2 ? 8 : 4;
    static constexpr bool TWS = POW2 && !f64;
    static constexpr bool PAD = !f64;  // padded shared-memory lines (slot)
};

// Transform G lines of L.n points (DIR = -1 forward, +1 inverse, unnormalised),
// alternating between the buffers buf and alt stage by stage; returns the one
// that holds the result (the other is scratch).  Call with every thread of the
// CTA (at least G*n/VPT), after a barrier.
template <int DIR, bool POW2, typename R, typename C>
__device__ __forceinline__ C *fft_lines_t(C *buf, C *alt, const FftLen &L, int G, const C *tw_all, const C *roots,
                                          const C *lo, const C *hi) {
    typedef FftCfg<R, POW2> Cf;
    constexpr int V = Cf::VPT;
    constexpr bool T = Cf::TWS, PD = Cf::PAD;
    const C *tw = tw_all + L.tw_off;
    int p = 1, lg_p = 0, lg_m = L.log2n;
    for (int s = 0; s < L.nst; ++s) {
        const int R_ = L.rad[s];
        if constexpr (POW2) {
            if (R_ == 8) fft_stage<8, V / 8, DIR, true, T, PD>(buf, alt, L.n, G, p, tw, roots, lo, hi, lg_m - 3, lg_p, L.ls);
            else if (R_ == 4) fft_stage<4, V / 4, DIR, true, T, PD>(buf, alt, L.n, G, p, tw, roots, lo, hi, lg_m - 2, lg_p, L.ls);
            else fft_stage<2, V / 2, DIR, true, T, PD>(buf, alt, L.n, G, p, tw, roots, lo, hi, lg_m - 1, lg_p, L.ls);
            lg_p += R_ == 8 ? 3 : R_ == 4 ? 2 : 1;
        } else {
            switch (R_) {
            case 8: fft_stage<8, 1, DIR, false, false, PD>(buf, alt, L.n, G, p, tw, roots, lo, hi, 0, 0, 0); break;
            case 4: fft_stage<4, 1, DIR, false, false, PD>(buf, alt, L.n, G, p, tw, roots, lo, hi, 0, 0, 0); break;
            case 2: fft_stage<2, 2, DIR, false, false, PD>(buf, alt, L.n, G, p, tw, roots, lo, hi, 0, 0, 0); break;
            case 3: fft_stage<3, 2, DIR, false, false, PD>(buf, alt, L.n, G, p, tw, roots, lo, hi, 0, 0, 0); break;
            case 5: fft_stage<5, 1, DIR, false, false, PD>(buf, alt, L.n, G, p, tw, roots, lo, hi, 0, 0, 0); break;
            default: fft_stage<7, 1, DIR, false, false, PD>(buf, alt, L.n, G, p, tw, roots, lo, hi, 0, 0, 0); break;
            }
        }
        p *= R_;
        C *t = buf;
        buf = alt;
        alt = t;
    }
    return buf;
}

template <int DIR, bool POW2, typename C>
__device__ __forceinline__ C *fft_lines(C *buf, C *alt, const FftLen &L, int G, const C *tw_all, const C *roots,
                                        const C *lo, const C *hi) {
    typedef decltype(C{}.x) R;
    return fft_lines_t<DIR, POW2, R>(buf, alt, L, G, tw_all, roots, lo, hi);
}

// Copy the two-level twiddle table of L into shared memory at dst (when the
// transforms use it); returns the (lo, hi) pointers.  The caller's next barrier
// publishes it.
// Both tables are stored padded (slot), like the lines: a stage reads lo at
// strides of up to 16 entries.
template <bool TWS, typename C>
__device__ __forceinline__ void load_twiddles(const FftLen &L, const C *tw_all, C *dst, const C **lo, const C **hi) {
    if constexpr (TWS) {
        const int nlo = 1 << L.ls, nhi = L.n >> L.ls;
        C *h = dst + padded<true>(nlo);
        for (int t = threadIdx.x; t < nlo + nhi; t += blockDim.x) {
            if (t < nlo) dst[slot<true>(t)] = tw_all[L.lo_off + t];
            else h[slot<true>(t - nlo)] = tw_all[L.hi_off + (t - nlo)];
        }
        *lo = dst;
        *hi = h;
    } else {
        *lo = *hi = nullptr;
    }
}

// complex entries of shared memory the two-level table of a length needs
__host__ __device__ __forceinline__ int twiddle_smem(const FftLen &L, bool tws) {
    return tws ? padded<true>(1 << L.ls) + padded<true>(L.n >> L.ls) : 0;
}

// ------------------------------------------------------------ row passes --

// Forward x transforms of rows 2c and 2c+1 (the second may not exist) of a real
// field f (cubed and scaled by coef when CUBE), written to Z[kx][row].
template <typename R, bool CUBE, bool POW2>
__device__ void rows_forward_body(typename Cplx<R>::type *buf, typename Cplx<R>::type *alt, const R *f,
                                  typename Cplx<R>::type *Z, int nx,
                                  int nrows, int ra, R coef, const FftLen &L, const typename Cplx<R>::type *tw,
                                  const typename Cplx<R>::type *roots, const typename Cplx<R>::type *lo,
                                  const typename Cplx<R>::type *hi, bool load) {
    typedef typename Cplx<R>::type C;
    constexpr bool PD = FftCfg<R, POW2>::PAD;
    const int rb = ra + 1;
    const bool has_b = rb < nrows;
    if (load) {
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            R a = f[(size_t)ra * nx + i], b = has_b ? f[(size_t)rb * nx + i] : R(0);
            if (CUBE) {
                a = coef * ((a * a) * a);
                b = coef * ((b * b) * b);
            }
            buf[slot<PD>(i)] = C{a, b};
        }
    }
    __syncthreads();
    const C *res = fft_lines<-1, POW2>(buf, alt, L, 1, tw, roots, lo, hi);
    const int nxh = nx / 2 + 1;
    for (int k = threadIdx.x; k < nxh; k += blockDim.x) {
        const C zk = res[slot<PD>(k)], zc = res[slot<PD>(k == 0 ? 0 : nx - k)];
        // A = (z_k + conj z_{n-k}) / 2, B = -i (z_k - conj z_{n-k}) / 2
        const C A{R(0.5) * (zk.x + zc.x), R(0.5) * (zk.y - zc.y)};
        const C B{R(0.5) * (zk.y + zc.y), R(0.5) * (zc.x - zk.x)};
        Z[(size_t)k * nrows + ra] = A;
        if (has_b) Z[(size_t)k * nrows + rb] = B;
    }
}

template <typename R, bool CUBE, bool POW2>
__global__ void __launch_bounds__(FftCfg<R, POW2>::NT, FftCfg<R, POW2>::MINB)
    rows_forward_kernel(const R *f, typename Cplx<R>::type *Z, int nx, int nrows, R coef, FftLen L,
                        const typename Cplx<R>::type *tw, const typename Cplx<R>::type *roots) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typedef typename Cplx<R>::type C;
    C *buf = reinterpret_cast<C *>(smem_raw);
    C *alt = buf + padded<FftCfg<R, POW2>::PAD>(nx);
    const C *lo, *hi;
    load_twiddles<FftCfg<R, POW2>::TWS>(L, tw, alt + padded<FftCfg<R, POW2>::PAD>(nx), &lo, &hi);
    rows_forward_body<R, CUBE, POW2>(buf, alt, f, Z, nx, nrows, 2 * blockIdx.x, coef, L, tw, roots, lo, hi, true);
}

// Inverse x transforms of rows 2c, 2c+1 from Z into phi; with NEXT, the cubic
// term of the new rows is transformed forward into Z for the next step.
template <typename R, bool NEXT, bool POW2>
__global__ void __launch_bounds__(FftCfg<R, POW2>::NT, FftCfg<R, POW2>::MINB) rows_inverse_kernel(typename Cplx<R>::type *Z, R *phi, int nx, int nrows, R coef, FftLen L,
                                    const typename Cplx<R>::type *tw, const typename Cplx<R>::type *roots) {
    typedef typename Cplx<R>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool PD = FftCfg<R, POW2>::PAD;
    C *buf = reinterpret_cast<C *>(smem_raw);
    C *alt = buf + padded<PD>(nx);
    const C *lo, *hi;
    load_twiddles<FftCfg<R, POW2>::TWS>(L, tw, alt + padded<PD>(nx), &lo, &hi);
    const int ra = 2 * blockIdx.x, rb = ra + 1;
    const bool has_b = rb < nrows;
    const int half = nx / 2;
    for (int k = threadIdx.x; k < nx; k += blockDim.x) {
        // Hermitian extension of both half spectra; the zero and Nyquist bins are real
        const bool lower = k <= half;
        const int kk = lower ? k : nx - k;
        C A = Z[(size_t)kk * nrows + ra], B = has_b ? Z[(size_t)kk * nrows + rb] : C{R(0), R(0)};
        if (k == 0 || 2 * k == nx) {
            A.y = R(0);
            B.y = R(0);
        }
        if (!lower) {
            A.y = -A.y;
            B.y = -B.y;
        }
        buf[slot<PD>(k)] = C{A.x - B.y, A.y + B.x};  // A + i B
    }
    __syncthreads();
    C *res = fft_lines<1, POW2>(buf, alt, L, 1, tw, roots, lo, hi);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const C v = res[slot<PD>(i)];
        phi[(size_t)ra * nx + i] = v.x;
        if (has_b) phi[(size_t)rb * nx + i] = v.y;
        if (NEXT) res[slot<PD>(i)] = C{coef * ((v.x * v.x) * v.x), has_b ? coef * ((v.y * v.y) * v.y) : R(0)};
    }
    if (NEXT) rows_forward_body<R, false, POW2>(res, res == buf ? alt : buf, nullptr, Z, nx, nrows, ra, coef, L, tw, roots, lo, hi, false);
}

// ----------------------------------------------------------- line passes --

enum LineMode { kLineForward = 0, kLineInverse = 1, kLineUpdate = 2 };

// Geometry of the lines of one pass over Z[kx][z][y] (y fastest).
struct LineGeom {
    int n;            // points per line
    int estride;      // elements between consecutive points of a line
    int lstride;      // elements between adjacent lines of a group
    int G;            // lines per CTA
    int groups_per_kx, lines_per_kx;
    int axis;         // 1 = y lines, 2 = z lines
    int ny, nz, nxh;
};

// frequency index of bin m of an n-point transform (numpy fftfreq order)
__device__ __forceinline__ int freq_of(int m, int n) { return (m < (n + 1) / 2) ? m : m - n; }

template <typename R, int MODEL>
__device__ __forceinline__ typename Cplx<R>::type update_mode(typename Cplx<R>::type *uh, typename Cplx<R>::type nh,
                                                              int kx, int ky, int kz, R tx, R ty, R tz, R c1, R kappa,
                                                              R dt, R inv_n) {
    typedef typename Cplx<R>::type C;
    const R fx = tx * (R)kx, fy = ty * (R)ky, fz = tz * (R)kz;
    const R k2 = (fz * fz + fy * fy) + fx * fx;  // slowest axis first
    const R L = (MODEL == AC) ? c1 - k2 : k2 * (c1 - kappa * k2);
    const R w = (MODEL == AC) ? R(1) : -k2;
    const R denom = R(1) - dt * L;
    const C a = *uh;
    C v;
    if constexpr (sizeof(R) == 8) {
        v.x = (a.x + dt * (w * nh.x)) / denom;
        v.y = (a.y + dt * (w * nh.y)) / denom;
    } else {  // FP32: one correctly rounded reciprocal for both parts (within an ulp of the quotients)
        const R rd = __frcp_rn(denom);
        v.x = (a.x + dt * (w * nh.x)) * rd;
        v.y = (a.y + dt * (w * nh.y)) * rd;
    }
    *uh = v;
    return C{v.x * inv_n, v.y * inv_n};
}

template <typename R, int MODE, int MODEL, bool POW2>
__global__ void __launch_bounds__(FftCfg<R, POW2>::NT, FftCfg<R, POW2>::MINB) lines_kernel(typename Cplx<R>::type *Z, typename Cplx<R>::type *uh, LineGeom g, FftLen L,
                             const typename Cplx<R>::type *tw, const typename Cplx<R>::type *roots, R tx, R ty, R tz,
                             R c1, R kappa, R dt, R inv_n) {
    typedef typename Cplx<R>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool PD = FftCfg<R, POW2>::PAD;
    C *buf = reinterpret_cast<C *>(smem_raw);
    C *alt = buf + padded<PD>(g.G * g.n);
    const C *lo, *hi;
    load_twiddles<FftCfg<R, POW2>::TWS>(L, tw, alt + padded<PD>(g.G * g.n), &lo, &hi);
    const int n = g.n;
    // first line of this CTA's group and its line count
    const int gi = blockIdx.x;
    int nl, line0, kx;
    size_t base;
    if (g.axis == 1) {  // y lines, contiguous: line index = kx * nz + z
        line0 = gi * g.G;
        nl = min(g.G, g.nxh * g.nz - line0);
        base = (size_t)line0 * n;
        kx = 0;
    } else {            // z lines: adjacent y within one kx
        kx = gi / g.groups_per_kx;
        line0 = (gi - kx * g.groups_per_kx) * g.G;  // first y
        nl = min(g.G, g.ny - line0);
        base = (size_t)kx * g.nz * g.ny + line0;
    }
    for (int e = threadIdx.x; e < nl * n; e += blockDim.x) {
        int l, i;
        if (g.estride == 1) {
            if (POW2) { l = e >> L.log2n; i = e & (n - 1); }
            else { l = e / n; i = e - l * n; }
        }
        else { i = e / nl; l = e - i * nl; }   // adjacent lines first: coalesced
        buf[slot<PD>(l * n + i)] = Z[base + (size_t)l * g.lstride + (size_t)i * g.estride];
    }
    __syncthreads();
    C *res = (MODE == kLineInverse) ? fft_lines<1, POW2>(buf, alt, L, nl, tw, roots, lo, hi)
                                    : fft_lines<-1, POW2>(buf, alt, L, nl, tw, roots, lo, hi);
    if (MODE == kLineUpdate) {
        for (int e = threadIdx.x; e < nl * n; e += blockDim.x) {
            int l, i;
            if (g.estride == 1) {
            if (POW2) { l = e >> L.log2n; i = e & (n - 1); }
            else { l = e / n; i = e - l * n; }
        }
            else { i = e / nl; l = e - i * nl; }
            const size_t at = base + (size_t)l * g.lstride + (size_t)i * g.estride;
            int mx, my, mz;
            if (g.axis == 1) {  // 2D: the y pass holds the update (nz == 1)
                mx = line0 + l;
                my = freq_of(i, g.ny);
                mz = 0;
            } else {
                mx = kx;
                my = freq_of(line0 + l, g.ny);
                mz = freq_of(i, g.nz);
            }
            res[slot<PD>(l * n + i)] = update_mode<R, MODEL>(uh + at, res[slot<PD>(l * n + i)], mx, my, mz, tx, ty, tz, c1, kappa, dt,
                                                   inv_n);
        }
        __syncthreads();
        res = fft_lines<1, POW2>(res, res == buf ? alt : buf, L, nl, tw, roots, lo, hi);
    }
    for (int e = threadIdx.x; e < nl * n; e += blockDim.x) {
        int l, i;
        if (g.estride == 1) {
            if (POW2) { l = e >> L.log2n; i = e & (n - 1); }
            else { l = e / n; i = e - l * n; }
        }
        else { i = e / nl; l = e - i * nl; }
        Z[base + (size_t)l * g.lstride + (size_t)i * g.estride] = res[slot<PD>(l * n + i)];
    }
}

// ----------------------------------------------------------------- host --

static bool factor_len(int n, FftLen *L) {
    L->n = n;
    L->nst = 0;
    int m = n;
    for (int r : {8, 4, 2, 3, 5, 7})
        while (m % r == 0) {
            if (L->nst == kFftMaxStages) return false;
            L->rad[L->nst++] = r;
            m /= r;
        }
    return m == 1;
}

static bool is_pow2(int n) { return (n & (n - 1)) == 0; }

// threads for G lines of n points: G*n/VPT (so that no thread holds more
// butterflies than a stage's QMAX), whole warps
template <typename R> static int fft_threads(int n, int G, bool pow2) {
    const int vpt = pow2 ? FftCfg<R, true>::VPT : FftCfg<R, false>::VPT;
    const int t = (G * n + vpt - 1) / vpt;
    return std::max(32, (t + 31) / 32 * 32);
}

template <typename R> static size_t csize() { return 2 * sizeof(R); }

// lines per CTA for a pass of n-point lines: within the thread limit of the
// launch and 64 KB of shared memory (at least one line)
template <typename R> static int lines_per_cta(int n, bool pow2, int cap) {
    const int vpt = pow2 ? FftCfg<R, true>::VPT : FftCfg<R, false>::VPT;
    const int by_threads = (pow2 ? FftCfg<R, true>::NT : FftCfg<R, false>::NT) * vpt / n;
    const int by_smem = (int)(64 * 1024 / (csize<R>() * (size_t)n));
    return std::max(1, std::min(std::min(by_threads, by_smem), cap));
}

template <typename R> static bool fits(int n, bool pow2) {
    return n <= kFftMaxN && fft_threads<R>(n, 1, pow2) <= (pow2 ? FftCfg<R, true>::NT : FftCfg<R, false>::NT);
}

int spectral_create(int dtype, int dims, int nx, int ny, int nz, SpectralPlan **out) {
    *out = nullptr;
    SpectralPlan *P = new (std::nothrow) SpectralPlan();
    if (!P) return SP_ENOMEM;
    P->dtype = dtype;
    P->dims = dims;
    P->nx = nx;
    P->ny = ny;
    P->nz = nz;
    P->nxh = nx / 2 + 1;
    P->N = (size_t)nx * ny * nz;
    P->Nc = (size_t)P->nxh * ny * nz;
    P->pow2 = is_pow2(nx) && is_pow2(ny) && is_pow2(nz);
    const int sides[3] = {nx, ny, nz};
    FftLen *ls[3] = {&P->lx, &P->ly, &P->lz};
    const bool f64 = dtype == SP_F64;
    for (int a = 0; a < 3; ++a) {
        const bool ok = factor_len(sides[a], ls[a]) &&
                        (f64 ? fits<double>(sides[a], P->pow2) : fits<float>(sides[a], P->pow2));
        if (!ok) {
            g_fft_err = std::string("the spectral scheme needs sides with prime factors 2, 3, 5, 7 of at most ") +
                        (f64 ? "4096 (FP64, powers of two; 2048 otherwise)" : "8192 (FP32, powers of two; 4096 otherwise)") +
                        " points (got " + std::to_string(sides[a]) + ")";
            delete P;
            return SP_EINVAL;
        }
    }
    // twiddles exp(-2 pi i t / n) of each distinct side, then the roots of 3, 5 and 7,
    // in long double on the host, rounded once to the working precision
    std::vector<long double> re, im;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    int offs[3];
    for (int a = 0; a < 3; ++a) {
        int prev = -1;
        for (int b = 0; b < a; ++b)
            if (sides[b] == sides[a]) prev = b;
        if (prev >= 0) {
            offs[a] = offs[prev];
            continue;
        }
        offs[a] = (int)re.size();
        for (int t = 0; t < sides[a]; ++t) {
            const long double ang = two_pi * (long double)t / (long double)sides[a];
            re.push_back(cosl(ang));
            im.push_back(-sinl(ang));
        }
    }
    P->lx.tw_off = offs[0];
    P->ly.tw_off = offs[1];
    P->lz.tw_off = offs[2];
    // two-level tables of the power-of-two lengths: lo[t] = w^t (t < 2^ls), hi[u] = w^(u 2^ls)
    for (int a = 0; a < 3; ++a) {
        FftLen &L = *ls[a];
        int lg = 0;
        while ((1 << lg) < L.n) ++lg;
        L.log2n = lg;
        L.ls = (lg + 1) / 2;
        L.lo_off = L.hi_off = 0;
        if (!P->pow2) continue;
        L.lo_off = (int)re.size();
        for (int t = 0; t < (1 << L.ls); ++t) {
            const long double ang = two_pi * (long double)t / (long double)L.n;
            re.push_back(cosl(ang));
            im.push_back(-sinl(ang));
        }
        L.hi_off = (int)re.size();
        for (int u = 0; u < (L.n >> L.ls); ++u) {
            const long double ang = two_pi * (long double)u * (long double)(1 << L.ls) / (long double)L.n;
            re.push_back(cosl(ang));
            im.push_back(-sinl(ang));
        }
    }
    P->roots_off = (int)re.size();
    for (int R_ : {3, 5, 7})
        for (int t = 0; t < R_; ++t) {
            const long double ang = two_pi * (long double)t / (long double)R_;
            re.push_back(cosl(ang));
            im.push_back(-sinl(ang));
        }
    const size_t cb = f64 ? sizeof(double2) : sizeof(float2);
    std::vector<unsigned char> host(re.size() * cb);
    for (size_t i = 0; i < re.size(); ++i) {
        if (f64) reinterpret_cast<double2 *>(host.data())[i] = double2{(double)re[i], (double)im[i]};
        else reinterpret_cast<float2 *>(host.data())[i] = float2{(float)re[i], (float)im[i]};
    }
    if (cudaMalloc(&P->uh, P->Nc * cb) != cudaSuccess || cudaMalloc(&P->z, P->Nc * cb) != cudaSuccess ||
        cudaMalloc(&P->tw, host.size()) != cudaSuccess ||
        cudaMemcpy(P->tw, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        spectral_destroy(P);
        g_fft_err = "device allocation for the spectral plan failed";
        return SP_ENOMEM;
    }
    *out = P;
    return SP_OK;
}

void spectral_destroy(SpectralPlan *P) {
    if (!P) return;
    if (P->uh) cudaFree(P->uh);
    if (P->z) cudaFree(P->z);
    if (P->tw) cudaFree(P->tw);
    delete P;
}

size_t spectral_bytes(const SpectralPlan *P) {
    return 2 * P->Nc * (P->dtype == SP_F64 ? sizeof(double2) : sizeof(float2));
}

// opt in to more than 48 KB of dynamic shared memory where needed
template <typename K> static cudaError_t prepare(K kern, size_t bytes) {
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

template <typename R> static LineGeom line_geom(const SpectralPlan *P, int axis) {
    LineGeom g{};
    g.ny = P->ny;
    g.nz = P->nz;
    g.nxh = P->nxh;
    g.axis = axis;
    if (axis == 1) {
        g.n = P->ny;
        g.estride = 1;
        g.lstride = P->ny;
        g.G = lines_per_cta<R>(g.n, P->pow2, P->nxh * P->nz);
        g.lines_per_kx = P->nz;
        g.groups_per_kx = 0;
    } else {
        g.n = P->nz;
        g.estride = P->ny;
        g.lstride = 1;
        g.G = lines_per_cta<R>(g.n, P->pow2, P->ny);
        g.lines_per_kx = P->ny;
        g.groups_per_kx = (P->ny + g.G - 1) / g.G;
    }
    return g;
}

template <typename R, int MODE, int MODEL, bool POW2>
static cudaError_t run_lines_t(SpectralPlan *P, int axis, cudaStream_t s, R tx, R ty, R tz, R c1, R kappa, R dt,
                               R inv_n, typename Cplx<R>::type *Z) {
    typedef typename Cplx<R>::type C;
    const LineGeom g = line_geom<R>(P, axis);
    const FftLen &L = axis == 1 ? P->ly : P->lz;
    const unsigned blocks = axis == 1 ? (unsigned)((P->nxh * P->nz + g.G - 1) / g.G)
                                      : (unsigned)(P->nxh * g.groups_per_kx);
    const size_t smem =
        ((size_t)2 * padded<FftCfg<R, POW2>::PAD>(g.G * g.n) + twiddle_smem(L, FftCfg<R, POW2>::TWS)) * csize<R>();
    auto kern = lines_kernel<R, MODE, MODEL, POW2>;
    cudaError_t e = prepare(kern, smem);
    if (e != cudaSuccess) return e;
    const C *tw = static_cast<const C *>(P->tw);
    kern<<<blocks, fft_threads<R>(g.n, g.G, POW2), smem, s>>>(Z, static_cast<C *>(P->uh), g, L, tw, tw + P->roots_off,
                                                           tx, ty, tz, c1, kappa, dt, inv_n);
    return cudaGetLastError();
}

template <typename R, int MODE, int MODEL>
static cudaError_t run_lines(SpectralPlan *P, int axis, cudaStream_t s, R tx, R ty, R tz, R c1, R kappa, R dt,
                             R inv_n, typename Cplx<R>::type *Z) {
    if (P->pow2) return run_lines_t<R, MODE, MODEL, true>(P, axis, s, tx, ty, tz, c1, kappa, dt, inv_n, Z);
    return run_lines_t<R, MODE, MODEL, false>(P, axis, s, tx, ty, tz, c1, kappa, dt, inv_n, Z);
}

template <typename R, bool CUBE, bool POW2>
static cudaError_t run_rows_forward_t(SpectralPlan *P, const R *f, typename Cplx<R>::type *Z, R coef, cudaStream_t s) {
    typedef typename Cplx<R>::type C;
    const int nrows = P->ny * P->nz;
    const size_t smem =
        ((size_t)2 * padded<FftCfg<R, POW2>::PAD>(P->nx) + twiddle_smem(P->lx, FftCfg<R, POW2>::TWS)) * csize<R>();
    auto kern = rows_forward_kernel<R, CUBE, POW2>;
    cudaError_t e = prepare(kern, smem);
    if (e != cudaSuccess) return e;
    const C *tw = static_cast<const C *>(P->tw);
    kern<<<(unsigned)((nrows + 1) / 2), fft_threads<R>(P->nx, 1, POW2), smem, s>>>(f, Z, P->nx, nrows, coef, P->lx, tw,
                                                                                tw + P->roots_off);
    return cudaGetLastError();
}

template <typename R, bool CUBE>
static cudaError_t run_rows_forward(SpectralPlan *P, const R *f, typename Cplx<R>::type *Z, R coef, cudaStream_t s) {
    if (P->pow2) return run_rows_forward_t<R, CUBE, true>(P, f, Z, coef, s);
    return run_rows_forward_t<R, CUBE, false>(P, f, Z, coef, s);
}

template <typename R, bool NEXT, bool POW2>
static cudaError_t run_rows_inverse_t(SpectralPlan *P, R *phi, R coef, cudaStream_t s) {
    typedef typename Cplx<R>::type C;
    const int nrows = P->ny * P->nz;
    const size_t smem =
        ((size_t)2 * padded<FftCfg<R, POW2>::PAD>(P->nx) + twiddle_smem(P->lx, FftCfg<R, POW2>::TWS)) * csize<R>();
    auto kern = rows_inverse_kernel<R, NEXT, POW2>;
    cudaError_t e = prepare(kern, smem);
    if (e != cudaSuccess) return e;
    const C *tw = static_cast<const C *>(P->tw);
    kern<<<(unsigned)((nrows + 1) / 2), fft_threads<R>(P->nx, 1, POW2), smem, s>>>(
        static_cast<C *>(P->z), phi, P->nx, nrows, coef, P->lx, tw, tw + P->roots_off);
    return cudaGetLastError();
}

template <typename R, bool NEXT>
static cudaError_t run_rows_inverse(SpectralPlan *P, R *phi, R coef, cudaStream_t s) {
    if (P->pow2) return run_rows_inverse_t<R, NEXT, true>(P, phi, coef, s);
    return run_rows_inverse_t<R, NEXT, false>(P, phi, coef, s);
}

// phi^ = forward transform of phi (after the initial condition or a write)
template <typename R> static int spectral_load_t(SpectralPlan *P, const R *phi, cudaStream_t s) {
    typedef typename Cplx<R>::type C;
    C *uh = static_cast<C *>(P->uh);
    cudaError_t e = run_rows_forward<R, false>(P, phi, uh, R(1), s);
    if (e == cudaSuccess && P->ny > 1) e = run_lines<R, kLineForward, AC>(P, 1, s, 0, 0, 0, 0, 0, 0, 0, uh);
    if (e == cudaSuccess && P->nz > 1) e = run_lines<R, kLineForward, AC>(P, 2, s, 0, 0, 0, 0, 0, 0, 0, uh);
    P->nh_valid = false;
    if (e != cudaSuccess) {
        g_fft_err = std::string("forward transform: ") + cudaGetErrorString(e);
        return SP_ECUDA;
    }
    return SP_OK;
}

int spectral_load(SpectralPlan *P, const void *phi, cudaStream_t s) {
    if (P->dtype == SP_F64) return spectral_load_t<double>(P, static_cast<const double *>(phi), s);
    return spectral_load_t<float>(P, static_cast<const float *>(phi), s);
}

template <typename R, int MODEL>
static cudaError_t spectral_step_t(SpectralPlan *P, R *phi, double h, double dt, double c1, double c2, double kappa,
                                   bool more, cudaStream_t s) {
    typedef typename Cplx<R>::type C;
    C *Z = static_cast<C *>(P->z);
    const R coef = (R)(MODEL == AC ? -c2 : c2);
    cudaError_t e = cudaSuccess;
    if (!P->nh_valid) e = run_rows_forward<R, true>(P, phi, Z, coef, s);
    const double two_pi = 6.283185307179586476925286766559;
    const R tx = (R)(two_pi / ((double)P->nx * h)), ty = (R)(two_pi / ((double)P->ny * h)),
            tz = (R)(two_pi / ((double)P->nz * h));
    const R inv_n = (R)(1.0 / (double)P->N);
    if (P->dims == 2) {
        if (e == cudaSuccess)
            e = run_lines<R, kLineUpdate, MODEL>(P, 1, s, tx, ty, tz, (R)c1, (R)kappa, (R)dt, inv_n, Z);
    } else {
        if (e == cudaSuccess) e = run_lines<R, kLineForward, MODEL>(P, 1, s, tx, ty, tz, 0, 0, 0, 0, Z);
        if (e == cudaSuccess)
            e = run_lines<R, kLineUpdate, MODEL>(P, 2, s, tx, ty, tz, (R)c1, (R)kappa, (R)dt, inv_n, Z);
        if (e == cudaSuccess) e = run_lines<R, kLineInverse, MODEL>(P, 1, s, tx, ty, tz, 0, 0, 0, 0, Z);
    }
    if (e == cudaSuccess)
        e = more ? run_rows_inverse<R, true>(P, phi, coef, s) : run_rows_inverse<R, false>(P, phi, coef, s);
    P->nh_valid = more && e == cudaSuccess;
    return e;
}

int spectral_step(SpectralPlan *P, int model, void *phi, void *nbuf, double h, double dt, double c1, double c2,
                  double kappa, cudaStream_t s, int n_sm, bool more) {
    (void)nbuf;
    (void)n_sm;
    cudaError_t e;
    if (P->dtype == SP_F64)
        e = model == AC ? spectral_step_t<double, AC>(P, (double *)phi, h, dt, c1, c2, kappa, more, s)
                        : spectral_step_t<double, CH>(P, (double *)phi, h, dt, c1, c2, kappa, more, s);
    else
        e = model == AC ? spectral_step_t<float, AC>(P, (float *)phi, h, dt, c1, c2, kappa, more, s)
                        : spectral_step_t<float, CH>(P, (float *)phi, h, dt, c1, c2, kappa, more, s);
    if (e != cudaSuccess) {
        g_fft_err = std::string("spectral step: ") + cudaGetErrorString(e);
        return SP_ECUDA;
    }
    return SP_OK;
}

}  // namespace sp

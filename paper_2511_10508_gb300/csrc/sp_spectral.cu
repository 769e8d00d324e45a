// sp_spectral.cu -- semi-implicit Fourier spectral step (the paper's spectral
// solver scheme, Sec. "Construction of Semi-Implicit Fourier Spectral Scheme";
// the paper runs it on the host only).
//
// Linear terms are integrated implicitly in Fourier space with the continuous
// symbol -|k|^2, the cubic term explicitly in real space:
//   Allen-Cahn     L(k) = c1 - |k|^2,            N^ = (-c2 phi^3)^
//   Cahn-Hilliard  L(k) = |k|^2 (c1 - kappa |k|^2), N^ = -|k|^2 (c2 phi^3)^
//   phi^' = (phi^ + dt N^) / (1 - dt L(k)),   k = 2 pi m / (n h) per axis.
// The spectrum phi^ stays resident between steps, so one step is: the cubic
// term in real space (phi -> n), the forward transform of n, the update of
// phi^ (which also writes the normalised copy the inverse transform consumes,
// because an out-of-place complex-to-real transform may overwrite its input),
// and the inverse transform back to phi.  The transforms are cuFFT's; the
// cubic-term and update kernels are this file's.
#include <cufft.h>
#include <dlfcn.h>

#include <mutex>
#include <string>

#include "sp_internal.h"

namespace sp {

// cuFFT is loaded on first use, so programs that never use the spectral scheme
// neither need nor load it.  The table holds its public entry points.
struct CufftApi {
    decltype(&cufftPlan2d) plan2d;
    decltype(&cufftPlan3d) plan3d;
    decltype(&cufftDestroy) destroy;
    decltype(&cufftSetStream) set_stream;
    decltype(&cufftExecD2Z) d2z;
    decltype(&cufftExecZ2D) z2d;
    decltype(&cufftExecR2C) r2c;
    decltype(&cufftExecC2R) c2r;
};
static CufftApi g_fft;
static bool g_fft_ok = false;
static std::once_flag g_fft_once;

static bool load_cufft() {
    std::call_once(g_fft_once, [] {
        void *h = dlopen("libcufft.so.12", RTLD_NOW | RTLD_LOCAL);
        if (!h) h = dlopen("libcufft.so", RTLD_NOW | RTLD_LOCAL);
        if (!h) return;
        bool ok = true;
        auto sym = [&](auto &fn, const char *name) {
            fn = reinterpret_cast<std::remove_reference_t<decltype(fn)>>(dlsym(h, name));
            ok = ok && fn != nullptr;
        };
        sym(g_fft.plan2d, "cufftPlan2d");
        sym(g_fft.plan3d, "cufftPlan3d");
        sym(g_fft.destroy, "cufftDestroy");
        sym(g_fft.set_stream, "cufftSetStream");
        sym(g_fft.d2z, "cufftExecD2Z");
        sym(g_fft.z2d, "cufftExecZ2D");
        sym(g_fft.r2c, "cufftExecR2C");
        sym(g_fft.c2r, "cufftExecC2R");
        g_fft_ok = ok;
    });
    return g_fft_ok;
}

struct SpectralPlan {
    int dtype, dims, nx, ny, nz;
    size_t N, Nc;              // real points, half-spectrum modes
    cufftHandle r2c, c2r;
    void *uh, *scratch;        // resident spectrum, inverse-transform input (Nc complex each)
};

template <typename R> struct Cplx;
template <> struct Cplx<double> { typedef double2 type; };
template <> struct Cplx<float> { typedef float2 type; };

// n = coef * (phi * phi) * phi   (coef = -c2 for Allen-Cahn, c2 for Cahn-Hilliard)
template <typename R>
__global__ void spectral_cubic_kernel(const R *__restrict__ phi, R *__restrict__ n, size_t N, R coef) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const R p = phi[i];
        n[i] = coef * ((p * p) * p);
    }
}

// frequency index of FFT bin m of an n-point transform (numpy fftfreq order)
__device__ __forceinline__ int freq_of(int m, int n) { return (m < (n + 1) / 2) ? m : m - n; }

// nh and out may be the same array (each mode is read before it is written).
template <typename R, int MODEL>
__global__ void spectral_update_kernel(typename Cplx<R>::type *__restrict__ uh, const typename Cplx<R>::type *nh,
                                       typename Cplx<R>::type *out, int nx, int ny, int nz, R tx, R ty, R tz, R c1,
                                       R kappa, R dt, R inv_n) {
    const int nxh = nx / 2 + 1;
    const size_t Nc = (size_t)nxh * ny * nz;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < Nc; i += (size_t)gridDim.x * blockDim.x) {
        const int mx = (int)(i % nxh);
        const size_t r = i / nxh;
        const int my = (int)(r % ny), mz = (int)(r / ny);
        const R kx = tx * (R)mx, ky = ty * (R)freq_of(my, ny), kz = tz * (R)freq_of(mz, nz);
        const R k2 = (kz * kz + ky * ky) + kx * kx;  // slowest axis first
        const R L = (MODEL == AC) ? c1 - k2 : k2 * (c1 - kappa * k2);
        const R w = (MODEL == AC) ? R(1) : -k2;
        const R denom = R(1) - dt * L;
        const typename Cplx<R>::type a = uh[i], b = nh[i];
        typename Cplx<R>::type v;
        v.x = (a.x + dt * (w * b.x)) / denom;
        v.y = (a.y + dt * (w * b.y)) / denom;
        uh[i] = v;
        v.x = v.x * inv_n;
        v.y = v.y * inv_n;
        out[i] = v;
    }
}

static std::string g_cufft_err;
static int cufft_fail(cufftResult r, const char *what) {
    g_cufft_err = std::string(what) + ": cuFFT error " + std::to_string((int)r);
    return SP_ECUDA;
}
const char *spectral_last_error() { return g_cufft_err.c_str(); }

int spectral_create(int dtype, int dims, int nx, int ny, int nz, SpectralPlan **out) {
    *out = nullptr;
    if (!load_cufft()) {
        g_cufft_err = "cuFFT (libcufft.so.12) could not be loaded";
        return SP_ECUDA;
    }
    SpectralPlan *P = new (std::nothrow) SpectralPlan();
    if (!P) return SP_ENOMEM;
    P->dtype = dtype;
    P->dims = dims;
    P->nx = nx;
    P->ny = ny;
    P->nz = nz;
    P->N = (size_t)nx * ny * nz;
    P->Nc = (size_t)(nx / 2 + 1) * ny * nz;
    P->r2c = P->c2r = 0;
    const bool f64 = dtype == SP_F64;
    const cufftType tf = f64 ? CUFFT_D2Z : CUFFT_R2C, tb = f64 ? CUFFT_Z2D : CUFFT_C2R;
    cufftResult r;
    if (dims == 2) {
        r = g_fft.plan2d(&P->r2c, ny, nx, tf);
        if (r == CUFFT_SUCCESS) r = g_fft.plan2d(&P->c2r, ny, nx, tb);
    } else {
        r = g_fft.plan3d(&P->r2c, nz, ny, nx, tf);
        if (r == CUFFT_SUCCESS) r = g_fft.plan3d(&P->c2r, nz, ny, nx, tb);
    }
    if (r != CUFFT_SUCCESS) {
        spectral_destroy(P);
        return cufft_fail(r, "plan");
    }
    const size_t cbytes = P->Nc * (f64 ? sizeof(double2) : sizeof(float2));
    if (cudaMalloc(&P->uh, cbytes) != cudaSuccess || cudaMalloc(&P->scratch, cbytes) != cudaSuccess) {
        spectral_destroy(P);
        return SP_ENOMEM;
    }
    *out = P;
    return SP_OK;
}

void spectral_destroy(SpectralPlan *P) {
    if (!P) return;
    if (P->r2c) g_fft.destroy(P->r2c);
    if (P->c2r) g_fft.destroy(P->c2r);
    if (P->uh) cudaFree(P->uh);
    if (P->scratch) cudaFree(P->scratch);
    delete P;
}

size_t spectral_bytes(const SpectralPlan *P) {
    return 2 * P->Nc * (P->dtype == SP_F64 ? sizeof(double2) : sizeof(float2));
}

// phi^ = forward transform of phi (after the initial condition or a write)
int spectral_load(SpectralPlan *P, const void *phi, cudaStream_t s) {
    cufftResult r = g_fft.set_stream(P->r2c, s);
    if (r == CUFFT_SUCCESS) {
        if (P->dtype == SP_F64)
            r = g_fft.d2z(P->r2c, (cufftDoubleReal *)phi, (cufftDoubleComplex *)P->uh);
        else
            r = g_fft.r2c(P->r2c, (cufftReal *)phi, (cufftComplex *)P->uh);
    }
    return r == CUFFT_SUCCESS ? SP_OK : cufft_fail(r, "forward transform");
}

template <typename R>
static int spectral_step_t(SpectralPlan *P, int model, R *phi, R *nbuf, double h, double dt, double c1, double c2,
                           double kappa, cudaStream_t s, int n_sm) {
    typedef typename Cplx<R>::type Z;
    const unsigned blocks_r = (unsigned)std::min<size_t>((P->N + 255) / 256, (size_t)n_sm * 16);
    const unsigned blocks_c = (unsigned)std::min<size_t>((P->Nc + 255) / 256, (size_t)n_sm * 16);
    spectral_cubic_kernel<R><<<blocks_r, 256, 0, s>>>(phi, nbuf, P->N, (R)(model == AC ? -c2 : c2));
    if (cudaGetLastError() != cudaSuccess) return SP_ECUDA;
    cufftResult r = g_fft.set_stream(P->r2c, s);
    if (r == CUFFT_SUCCESS) {
        if constexpr (sizeof(R) == 8) r = g_fft.d2z(P->r2c, (cufftDoubleReal *)nbuf, (cufftDoubleComplex *)P->scratch);
        else r = g_fft.r2c(P->r2c, (cufftReal *)nbuf, (cufftComplex *)P->scratch);
    }
    if (r != CUFFT_SUCCESS) return cufft_fail(r, "forward transform");
    const double two_pi = 6.283185307179586476925286766559;
    const R tx = (R)(two_pi / ((double)P->nx * h)), ty = (R)(two_pi / ((double)P->ny * h)),
            tz = (R)(two_pi / ((double)P->nz * h));
    const R inv_n = (R)(1.0 / (double)P->N);
    if (model == AC)
        spectral_update_kernel<R, AC><<<blocks_c, 256, 0, s>>>((Z *)P->uh, (const Z *)P->scratch, (Z *)P->scratch, P->nx,
                                                               P->ny, P->nz, tx, ty, tz, (R)c1, (R)kappa, (R)dt, inv_n);
    else
        spectral_update_kernel<R, CH><<<blocks_c, 256, 0, s>>>((Z *)P->uh, (const Z *)P->scratch, (Z *)P->scratch, P->nx,
                                                               P->ny, P->nz, tx, ty, tz, (R)c1, (R)kappa, (R)dt, inv_n);
    if (cudaGetLastError() != cudaSuccess) return SP_ECUDA;
    r = g_fft.set_stream(P->c2r, s);
    if (r == CUFFT_SUCCESS) {
        if constexpr (sizeof(R) == 8) r = g_fft.z2d(P->c2r, (cufftDoubleComplex *)P->scratch, (cufftDoubleReal *)phi);
        else r = g_fft.c2r(P->c2r, (cufftComplex *)P->scratch, (cufftReal *)phi);
    }
    return r == CUFFT_SUCCESS ? SP_OK : cufft_fail(r, "inverse transform");
}

int spectral_step(SpectralPlan *P, int model, void *phi, void *nbuf, double h, double dt, double c1, double c2,
                  double kappa, cudaStream_t s, int n_sm) {
    if (P->dtype == SP_F64)
        return spectral_step_t<double>(P, model, (double *)phi, (double *)nbuf, h, dt, c1, c2, kappa, s, n_sm);
    return spectral_step_t<float>(P, model, (float *)phi, (float *)nbuf, h, dt, c1, c2, kappa, s, n_sm);
}

}  // namespace sp

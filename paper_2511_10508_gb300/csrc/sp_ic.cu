// sp_ic.cu -- seeded initial conditions written directly on the device.
//
// The paper starts every benchmark from "uniformly distributed random noise"
// (Sec. "Benchmarks").  The noise comes from a counter-based generator: the
// n-th output of SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) seeded with
// `seed`, i.e. the finaliser applied to seed + (n+1)*0x9E3779B97F4A7C15.  The
// top 53 bits give U in [0, 1), and a value is base + amp*(2U - 1) (FP64, then
// rounded to the storage type).  Stream layout with N points:
//   field 0 noise: n = i;  field 1 noise: n = N + i;
//   Gray-Scott patch p, axis a (x, y, z): n = 2N + 3p + a, centre = output mod n_a,
//   lower corner = centre - patch/2 (periodic); inside: u = 0.5, v = 0.25.
#include "sp_internal.h"

namespace sp {

__device__ __forceinline__ uint64_t splitmix64_nth(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double noise(uint64_t seed, uint64_t n, double base, double amp) {
    const double U = (double)(splitmix64_nth(seed, n) >> 11) * 0x1.0p-53;
    return base + amp * (2.0 * U - 1.0);
}

// Round an FP64 value once, to nearest, into the storage type.
template <typename T> __device__ __forceinline__ T round_store(double x);
template <> __device__ __forceinline__ double round_store<double>(double x) { return x; }
template <> __device__ __forceinline__ float round_store<float>(double x) { return __double2float_rn(x); }
template <> __device__ __forceinline__ bf16 round_store<bf16>(double x) { return __double2bfloat16(x); }

template <typename T>
__global__ void ic_kernel(T *u, T *v, int model, int dims, int nx, int ny, int nz, uint64_t seed,
                          int ic_kind, double mean, double amp, int patches, int patch) {
    __shared__ int lo[kMaxPatches][3];
    const uint64_t N = (uint64_t)nx * ny * nz;
    const bool gs = (model == GS);
    const int np = (gs && ic_kind == SP_IC_NOISE) ? patches : 0;  // host guarantees np <= kMaxPatches
    for (int q = threadIdx.x; q < np * 3; q += blockDim.x) {
        const int p = q / 3, ax = q % 3;
        const int n_a = ax == 0 ? nx : (ax == 1 ? ny : nz);
        const int c = (int)(splitmix64_nth(seed, 2 * N + 3ull * p + ax) % (uint64_t)n_a);
        int l = (c - patch / 2) % n_a;
        if (l < 0) l += n_a;
        lo[p][ax] = l;
    }
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        if (!gs) {
            u[i] = round_store<T>(ic_kind == SP_IC_NOISE ? noise(seed, i, mean, amp) : mean);
            // Model C: rho from the second stream
            if (model == MC) v[i] = round_store<T>(ic_kind == SP_IC_NOISE ? noise(seed, N + i, mean, amp) : mean);
            continue;
        }
        if (ic_kind != SP_IC_NOISE) {
            u[i] = round_store<T>(mean);
            v[i] = round_store<T>(0.0);
            continue;
        }
        const int x = (int)(i % (uint64_t)nx);
        const int y = (int)((i / (uint64_t)nx) % (uint64_t)ny);
        const int z = (int)(i / ((uint64_t)nx * ny));
        bool in = false;
        for (int p = 0; p < np && !in; ++p) {
            int ox = x - lo[p][0]; if (ox < 0) ox += nx;
            int oy = y - lo[p][1]; if (oy < 0) oy += ny;
            int oz = 0;
            if (dims == 3) { oz = z - lo[p][2]; if (oz < 0) oz += nz; }
            in = (ox < patch) && (oy < patch) && (oz < (dims == 3 ? patch : 1));
        }
        u[i] = round_store<T>(noise(seed, i, in ? 0.5 : 1.0, amp));
        v[i] = round_store<T>(noise(seed, N + i, in ? 0.25 : 0.0, amp));
    }
}

cudaError_t launch_ic(int dtype, void *u, void *v, int model, int dims, int nx, int ny, int nz,
                      uint64_t seed, int ic_kind, double mean, double amp, int patches, int patch,
                      cudaStream_t s, int n_sm) {
    const int threads = 256;
    const uint64_t N = (uint64_t)nx * ny * nz;
    const uint64_t want = (N + threads - 1) / threads;
    const int blocks = (int)(want < (uint64_t)n_sm * 16 ? (want ? want : 1) : (uint64_t)n_sm * 16);
    switch (dtype) {
    case 0: ic_kernel<double><<<blocks, threads, 0, s>>>((double *)u, (double *)v, model, dims, nx, ny, nz, seed, ic_kind, mean, amp, patches, patch); break;
    case 1: ic_kernel<float><<<blocks, threads, 0, s>>>((float *)u, (float *)v, model, dims, nx, ny, nz, seed, ic_kind, mean, amp, patches, patch); break;
    default: ic_kernel<bf16><<<blocks, threads, 0, s>>>((bf16 *)u, (bf16 *)v, model, dims, nx, ny, nz, seed, ic_kind, mean, amp, patches, patch); break;
    }
    return cudaGetLastError();
}

}  // namespace sp

namespace sp {

// Model H currents: component a of j at point i is amp (2U - 1) from stream
// n = (a+1) N + i (mean 0).
template <typename T>
__global__ void ic_currents_kernel(T *j0, T *j1, T *j2, int dims, uint64_t N, uint64_t seed, double amp,
                                   int constant) {
    T *jc[3] = {j0, j1, j2};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        for (int a = 0; a < dims; ++a)
            jc[a][i] = round_store<T>(constant ? 0.0 : noise(seed, (uint64_t)(a + 1) * N + i, 0.0, amp));
}

cudaError_t launch_ic_currents(int dtype, void *const j[3], int dims, uint64_t N, uint64_t seed, int ic_kind, double amp,
                               cudaStream_t s, int n_sm) {
    const unsigned blocks = (unsigned)std::min<uint64_t>((N + 255) / 256, (uint64_t)n_sm * 8);
    const int constant = ic_kind != SP_IC_NOISE;
    switch (dtype) {
    case SP_F64: ic_currents_kernel<double><<<blocks, 256, 0, s>>>((double *)j[0], (double *)j[1], (double *)j[2], dims, N, seed, amp, constant); break;
    case SP_F32: ic_currents_kernel<float><<<blocks, 256, 0, s>>>((float *)j[0], (float *)j[1], (float *)j[2], dims, N, seed, amp, constant); break;
    default: ic_currents_kernel<bf16><<<blocks, 256, 0, s>>>((bf16 *)j[0], (bf16 *)j[1], (bf16 *)j[2], dims, N, seed, amp, constant); break;
    }
    return cudaGetLastError();
}

}  // namespace sp

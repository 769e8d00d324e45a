// sp_noalloc.cu -- a reduction entry point that allocates nothing.
//
// sp_reduce() works on a simulation handle, whose creation allocates the
// fields and a small device scratch for the block partials of the reduction.
// Some callers cannot allocate device memory at the moment they need a mass or
// free-energy value: an application whose memory pool already owns nearly all
// of HBM (cudaMalloc would fail), a latency-critical loop in which cudaMalloc /
// cudaFree would stall or synchronise the device, or a program that keeps its
// fields in its own allocator and only wants diagnostics of them.  For those
// callers sp_reduce_field_noalloc() runs the same two reduction kernels on a
// field the caller owns, with the block partials in a fixed-size array that
// this file reserves in device memory.
//
// Contract:
//  - The scratch is g_reduce_scratch below: room for kNoAllocMaxPartials block
//    partials (two doubles each) plus one result slot, 8 KiB + 8 bytes.  Every
//    GPU that loads the library holds it until the process exits.
//  - A call needs as many partials as sp_reduce() would use for the same grid
//    on the same device (min(ceil(N/256), 2 x SMs)); a call needing more than
//    kNoAllocMaxPartials is rejected with SP_ETOOLARGE before any launch.
//  - Every call shares the array and leaves its contents behind.  Nothing in it
//    has to start at zero: each call's first kernel writes every partial slot it
//    later reads, and the second kernel writes the result slot.  Calls that
//    overlap on the GPU (different streams, or different host threads without
//    ordering) race on the array.
//  - The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (the host-side symbol is only a stand-in and must
//    never be passed to a kernel); make that first call before any stream
//    capture begins.
//  - No cudaMalloc, cudaFree or other allocating routine is called, and no
//    error message is formatted (that could allocate host memory): the status
//    code alone reports a failure, and sp_last_error() is left untouched.
#include <cmath>
#include <mutex>

#include "sp_internal.h"

namespace {

constexpr int kNoAllocMaxPartials = 512;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_reduce_scratch[2 * kNoAllocMaxPartials + 1];

std::mutex g_setup_mu;
double *g_scratch_dev[kMaxDevices];  // device address of g_reduce_scratch, per device
int g_sm_count[kMaxDevices];

// Once per device, with that device current: resolve the array's device address.
int setup_device(int dev, double **scratch, int *n_sm) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_reduce_scratch) != cudaSuccess) {
            cudaGetLastError();
            return SP_ECUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return SP_ECUDA;
        }
        g_sm_count[dev] = sms;
        g_scratch_dev[dev] = static_cast<double *>(p);
    }
    *scratch = g_scratch_dev[dev];
    *n_sm = g_sm_count[dev];
    return SP_OK;
}

}  // namespace

extern "C" int sp_reduce_field_noalloc(int what, int dtype, const void *field, int dims, const int64_t shape[3],
                                       double h, double c1, double c2, double *out, void *stream) {
    if (!field || !shape || !out) return SP_EINVAL;
    if (what != SP_MASS && what != SP_FREE_ENERGY && what != SP_SUM_U && what != SP_MIN_U && what != SP_MAX_U &&
        what != SP_SUMSQ_U)
        return SP_EINVAL;
    if (dtype < SP_F64 || dtype > SP_BF16_F32) return SP_EINVAL;
    if (dims != 2 && dims != 3) return SP_EINVAL;
    const int64_t nx = shape[0], ny = shape[1], nz = dims == 2 ? 1 : shape[2];
    if (dims == 2 && !(shape[2] == 0 || shape[2] == 1)) return SP_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 0x7fffffff || ny > 0x7fffffff || nz > 0x7fffffff) return SP_EINVAL;
    if (!(std::isfinite(h) && h > 0.0)) return SP_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return SP_EINVAL;
    double *scratch = nullptr;
    int n_sm = 0;
    if (int rc = setup_device(dev, &scratch, &n_sm)) return rc;

    const uint64_t N = (uint64_t)nx * (uint64_t)ny * (uint64_t)nz;
    const int nblocks = sp::reduce_blocks(N, n_sm);
    if (nblocks > kNoAllocMaxPartials) return SP_ETOOLARGE;

    sp::ReduceGeom g;
    g.nx = (int)nx;
    g.ny = (int)ny;
    g.nz = (int)nz;
    g.dims = dims;
    g.h = h;
    g.cell_volume = dims == 3 ? (h * h) * h : h * h;
    g.c1 = c1;
    g.c2 = c2;
    const cudaStream_t st = (cudaStream_t)stream;
    double *result = scratch + 2 * kNoAllocMaxPartials;
    if (sp::launch_reduce(dtype, what, field, g, scratch, nblocks, result, st) != cudaSuccess ||
        cudaMemcpyAsync(out, result, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    return SP_OK;
}

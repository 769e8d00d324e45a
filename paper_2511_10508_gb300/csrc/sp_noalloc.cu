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
//  - The first call in a CUDA context looks up the array's device address
//    with cudaGetSymbolAddress (the host-side symbol is only a stand-in and
//    must never be passed to a kernel) and keeps it for that context, keyed by
//    the context's unique ID: after cudaDeviceReset (or any other re-creation
//    of the context) the module is loaded again, possibly at another address,
//    and the next call looks the address up again.  Make the first call on a
//    device before any stream capture begins; a call on a stream that is being
//    captured is rejected (the result travels back through a host copy and a
//    stream synchronisation, which capture does not allow).
//  - The field pointer must be aligned to its element size, and the grid must
//    satisfy the limits of sp_create (each side < 2^31, a 3D plane nx*ny <
//    2^31); SP_EINVAL otherwise.
//  - No cudaMalloc, cudaFree or other allocating routine is called, and no
//    error message is formatted (that could allocate host memory): the status
//    code alone reports a failure, and sp_last_error() is left untouched.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "sp_internal.h"

namespace {

constexpr int kNoAllocMaxPartials = 512;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_reduce_scratch[2 * kNoAllocMaxPartials + 1];

// Driver calls that identify the current context, resolved once through the
// runtime (the library does not link the driver library directly).
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

struct DeviceState {
    unsigned long long ctx_id;  // context in which `scratch` was looked up
    double *scratch;            // device address of g_reduce_scratch in that context
    int n_sm;
};

std::mutex g_setup_mu;
CtxGetCurrentFn g_ctx_get_current;
CtxGetIdFn g_ctx_get_id;
bool g_entry_points_resolved;
DeviceState g_state[kMaxDevices];

int resolve_entry_points() {
    if (g_entry_points_resolved) return SP_OK;
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    g_entry_points_resolved = true;
    return SP_OK;
}

// ID of the context current on this thread, or 0 when none is current yet.
int current_context_id(unsigned long long *id) {
    void *ctx = nullptr;
    *id = 0;
    if (g_ctx_get_current(&ctx) != 0) return SP_ECUDA;
    if (ctx && g_ctx_get_id(ctx, id) != 0) return SP_ECUDA;
    return SP_OK;
}

// Set-up, once per device and context, with that device current: resolve the
// array's device address in the current context.
int setup_device(int dev, double **scratch, int *n_sm) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (int rc = resolve_entry_points()) return rc;
    unsigned long long id = 0;
    if (int rc = current_context_id(&id)) return rc;
    DeviceState &d = g_state[dev];
    if (!d.scratch || id == 0 || id != d.ctx_id) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_reduce_scratch) != cudaSuccess) {  // makes the primary context current
            cudaGetLastError();
            return SP_ECUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return SP_ECUDA;
        }
        if (int rc = current_context_id(&id)) return rc;
        if (id == 0) return SP_ECUDA;
        d.ctx_id = id;
        d.n_sm = sms;
        d.scratch = static_cast<double *>(p);
    }
    *scratch = d.scratch;
    *n_sm = d.n_sm;
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
    if (dims == 3 && nx * ny > (int64_t)0x7fffffff) return SP_EINVAL;  // as sp_create; N < 2^62
    if (!(std::isfinite(h) && h > 0.0)) return SP_EINVAL;
    const uintptr_t esize = dtype == SP_F64 ? 8 : (dtype == SP_F32 ? 4 : 2);
    if ((uintptr_t)field % esize != 0) return SP_EINVAL;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return SP_EINVAL;

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

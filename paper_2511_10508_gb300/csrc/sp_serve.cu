// sp_serve.cu -- continuous-batching server: many resident grids of differing
// model, dimension, size and precision advance together, admitted against an
// HBM budget as memory and slots free up.
//
// Device side: one batched kernel per (dims, storage type).  It walks a table
// of tiles that spans every resident grid of that kind; each CTA reads its
// tile's grid descriptor (model, stencil, sizes, buffers, coefficients) and
// runs the same tile code as the single-grid kernels (2D: 128 x 32 tiles, 3D:
// 32 x 16 x 8 boxes), so a grid's result does not depend on what else is
// resident.  A scheduling quantum is Q time steps = Q launches per kind,
// captured once into a CUDA graph and replayed while the set of resident grids
// is unchanged; grids that finish inside a quantum skip the remaining steps.
//
// Host side: a scheduler thread admits pending requests by priority, in
// arrival order within a priority (later requests may pass one that does not
// fit yet; sp_admission_order), allocates
// their buffers stream-ordered, writes the seeded initial condition, runs
// quanta, and retires finished grids: FP64 mass, optional FP64 copy of the
// fields to host memory, buffers freed, waiters notified.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sp_internal.h"
#include "sp_step.cuh"

namespace sp {

struct GridDesc {
    void *buf[2][2];        // [level][field]
    int model, stencil, nx, ny, nz;
    int parity;             // level that is current at step 0 of the quantum
    int steps;              // steps this grid takes in the quantum
    StepConsts k;
    StepConstsF kf;
};

struct TileDesc {
    int grid, x0, y0, z0;
};

constexpr int kB2X = 128, kB2Y = 32, kB3X = 32, kB3Y = 16, kB3Z = 8, kBatchNT = 256;

template <typename T> constexpr size_t batch2d_smem() {
    size_t m = 0;
#define SP_M(MO, ST) m = std::max(m, Step2dTileShape<MO, ST, T, kB2X, kB2Y>::smem_bytes);
    SP_M(AC, L5) SP_M(AC, L9BOX) SP_M(AC, L9X4) SP_M(CH, L5) SP_M(CH, L9BOX) SP_M(CH, L9X4)
    SP_M(GS, L5) SP_M(GS, L9BOX) SP_M(GS, L9X4) SP_M(MC, L5) SP_M(MC, L9BOX) SP_M(MC, L9X4)
#undef SP_M
    return m;
}
template <typename T> constexpr size_t batch3d_smem() {
    size_t m = 0;
#define SP_M(MO, ST) m = std::max(m, Step3dBoxShape<MO, ST, T, kB3X, kB3Y, kB3Z>::smem_bytes);
    SP_M(AC, L7) SP_M(AC, L27) SP_M(AC, L13X4) SP_M(CH, L7) SP_M(CH, L27) SP_M(CH, L13X4)
    SP_M(GS, L7) SP_M(GS, L27) SP_M(GS, L13X4) SP_M(MC, L7) SP_M(MC, L27) SP_M(MC, L13X4)
#undef SP_M
    return m;
}

template <typename T>
__global__ void __launch_bounds__(kBatchNT) batch2d_kernel(const GridDesc *__restrict__ grids,
                                                           const TileDesc *__restrict__ tiles, int j) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileDesc td = tiles[blockIdx.x];
    const GridDesc &g = grids[td.grid];
    if (j >= g.steps) return;  // this grid finished earlier in the quantum
    const int cur = g.parity ^ (j & 1);
    const T *i0 = static_cast<const T *>(g.buf[cur][0]), *i1 = static_cast<const T *>(g.buf[cur][1]);
    T *o0 = static_cast<T *>(g.buf[cur ^ 1][0]), *o1 = static_cast<T *>(g.buf[cur ^ 1][1]);
    const ConstsC<typename Cmp<T>::type> k(g.k, g.kf);
#define SP_C(MO, ST)                                                                                  \
    case MO * 8 + ST:                                                                                 \
        tile2d<MO, ST, T, kB2X, kB2Y, kBatchNT>(i0, i1, o0, o1, g.nx, g.ny, k, td.x0, td.y0, smem_raw); \
        break;
    switch (g.model * 8 + g.stencil) {
        SP_C(AC, L5) SP_C(AC, L9BOX) SP_C(AC, L9X4) SP_C(CH, L5) SP_C(CH, L9BOX) SP_C(CH, L9X4)
        SP_C(GS, L5) SP_C(GS, L9BOX) SP_C(GS, L9X4) SP_C(MC, L5) SP_C(MC, L9BOX) SP_C(MC, L9X4)
    }
#undef SP_C
}

template <typename T>
__global__ void __launch_bounds__(kBatchNT) batch3d_kernel(const GridDesc *__restrict__ grids,
                                                           const TileDesc *__restrict__ tiles, int j) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileDesc td = tiles[blockIdx.x];
    const GridDesc &g = grids[td.grid];
    if (j >= g.steps) return;
    const int cur = g.parity ^ (j & 1);
    const T *i0 = static_cast<const T *>(g.buf[cur][0]), *i1 = static_cast<const T *>(g.buf[cur][1]);
    T *o0 = static_cast<T *>(g.buf[cur ^ 1][0]), *o1 = static_cast<T *>(g.buf[cur ^ 1][1]);
    const ConstsC<typename Cmp<T>::type> k(g.k, g.kf);
#define SP_C(MO, ST)                                                                                       \
    case MO * 8 + ST:                                                                                      \
        box3d<MO, ST, T, kB3X, kB3Y, kB3Z, kBatchNT>(i0, i1, o0, o1, g.nx, g.ny, g.nz, k, td.x0, td.y0, td.z0, \
                                                     smem_raw);                                            \
        break;
    switch (g.model * 8 + g.stencil) {
        SP_C(AC, L7) SP_C(AC, L27) SP_C(AC, L13X4) SP_C(CH, L7) SP_C(CH, L27) SP_C(CH, L13X4)
        SP_C(GS, L7) SP_C(GS, L27) SP_C(GS, L13X4) SP_C(MC, L7) SP_C(MC, L27) SP_C(MC, L13X4)
    }
#undef SP_C
}

// kinds: 0 = 2D FP64, 1 = 2D FP32, 2 = 3D FP64, 3 = 3D FP32
static int kind_of(int dims, int dtype) { return (dims == 3 ? 2 : 0) + (dtype == SP_F32 ? 1 : 0); }

static cudaError_t set_batch_attributes() {
    cudaError_t e = cudaFuncSetAttribute(batch2d_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batch2d_smem<double>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch2d_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)batch2d_smem<float>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch3d_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)batch3d_smem<double>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch3d_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)batch3d_smem<float>());
    return e;
}

static cudaError_t launch_batch(int kind, const GridDesc *grids, const TileDesc *tiles, int ntiles, int j,
                                cudaStream_t s) {
    switch (kind) {
    case 0: batch2d_kernel<double><<<ntiles, kBatchNT, batch2d_smem<double>(), s>>>(grids, tiles, j); break;
    case 1: batch2d_kernel<float><<<ntiles, kBatchNT, batch2d_smem<float>(), s>>>(grids, tiles, j); break;
    case 2: batch3d_kernel<double><<<ntiles, kBatchNT, batch3d_smem<double>(), s>>>(grids, tiles, j); break;
    default: batch3d_kernel<float><<<ntiles, kBatchNT, batch3d_smem<float>(), s>>>(grids, tiles, j); break;
    }
    return cudaGetLastError();
}

}  // namespace sp

using namespace sp;

// ------------------------------------------------------------------ host --

namespace {

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Req {
    uint64_t ticket = 0;
    sp_request r{};
    int stencil = 0, nf = 1;
    int nx = 1, ny = 1, nz = 1;
    uint64_t N = 0;
    size_t bytes = 0;
    StepConsts k{};
    void *buf[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int parity = 0;
    int64_t steps_left = 0, steps_done = 0;
    double t_submit = 0, t_admit = -1, t_finish = -1;
    int status = SP_PENDING;
    bool done = false;
    double mass = 0;
    std::vector<double> host;  // FP64 fields, field 0 then field 1
};

}  // namespace

struct sp_server {
    size_t budget = 0, used = 0;
    int max_slots = 0, quantum = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::vector<Req *> resident;
    std::unordered_map<uint64_t, Req *> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread th;
    cudaStream_t stream = nullptr;
    int device = 0, n_sm = 0;
    // device tables
    GridDesc *d_grids = nullptr, *h_grids = nullptr;  // h_grids pinned
    int grids_cap = 0;
    TileDesc *d_tiles = nullptr;
    size_t tiles_cap = 0;
    int kind_off[4] = {0, 0, 0, 0}, kind_n[4] = {0, 0, 0, 0};
    double *d_partials = nullptr, *h_scalar = nullptr;
    int nred = 0;
    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
    cudaEvent_t ev = nullptr;
    // statistics
    uint64_t submitted = 0, admitted = 0, finished = 0, failed = 0, quanta = 0;
    double lups = 0, busy_s = 0;
    std::string err;
};

static size_t esize_of(int dtype) { return dtype == SP_F64 ? 8 : 4; }

static StepConsts consts_of(const sp_request &r, int stencil) {
    static const int q[6] = {1, 6, 12, 1, 30, 12};
    StepConsts k;
    const double q_h2 = ((double)q[stencil] * r.h) * r.h;
    k.c1 = r.params.c1;
    k.c2 = r.params.c2;
    k.sAC = 1.0 / q_h2;
    k.kq = r.params.kappa / q_h2;
    k.dq = r.dt / q_h2;
    k.duq = r.params.Du / q_h2;
    k.dvq = r.params.Dv / q_h2;
    k.F = r.params.F;
    k.Fk = r.params.F + r.params.k;
    k.dt = r.dt;
    k.c3 = r.params.c3;
    k.c3x2 = 2.0 * r.params.c3;
    return k;
}

// Grid descriptor and tile tables for the current resident set.
static cudaError_t rebuild_tables(sp_server *S) {
    const int ng = (int)S->resident.size();
    if (ng > S->grids_cap) {
        if (S->d_grids) cudaFree(S->d_grids);
        if (S->h_grids) cudaFreeHost(S->h_grids);
        S->grids_cap = std::max(ng, 2 * S->grids_cap);
        cudaError_t e = cudaMalloc(&S->d_grids, sizeof(GridDesc) * S->grids_cap);
        if (e == cudaSuccess) e = cudaMallocHost(&S->h_grids, sizeof(GridDesc) * S->grids_cap);
        if (e != cudaSuccess) return e;
    }
    std::vector<TileDesc> tiles[4];
    for (int g = 0; g < ng; ++g) {
        const Req *q = S->resident[g];
        const int kind = kind_of(q->r.dims, q->r.params.dtype);
        if (q->r.dims == 2) {
            for (int y = 0; y < q->ny; y += kB2Y)
                for (int x = 0; x < q->nx; x += kB2X) tiles[kind].push_back({g, x, y, 0});
        } else {
            for (int z = 0; z < q->nz; z += kB3Z)
                for (int y = 0; y < q->ny; y += kB3Y)
                    for (int x = 0; x < q->nx; x += kB3X) tiles[kind].push_back({g, x, y, z});
        }
    }
    size_t total = 0;
    for (int kd = 0; kd < 4; ++kd) {
        S->kind_off[kd] = (int)total;
        S->kind_n[kd] = (int)tiles[kd].size();
        total += tiles[kd].size();
    }
    if (total > S->tiles_cap) {
        if (S->d_tiles) cudaFree(S->d_tiles);
        S->tiles_cap = std::max(total, 2 * S->tiles_cap);
        cudaError_t e = cudaMalloc(&S->d_tiles, sizeof(TileDesc) * S->tiles_cap);
        if (e != cudaSuccess) return e;
    }
    std::vector<TileDesc> flat;
    flat.reserve(total);
    for (int kd = 0; kd < 4; ++kd) flat.insert(flat.end(), tiles[kd].begin(), tiles[kd].end());
    if (total) {
        cudaError_t e = cudaMemcpyAsync(S->d_tiles, flat.data(), sizeof(TileDesc) * total, cudaMemcpyHostToDevice,
                                        S->stream);
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(S->stream);  // `flat` is pageable and goes out of scope
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t upload_descriptors(sp_server *S, int Q) {
    for (size_t g = 0; g < S->resident.size(); ++g) {
        const Req *q = S->resident[g];
        GridDesc &d = S->h_grids[g];
        std::memcpy(d.buf, q->buf, sizeof d.buf);
        d.model = q->r.model;
        d.stencil = q->stencil;
        d.nx = q->nx;
        d.ny = q->ny;
        d.nz = q->nz;
        d.parity = q->parity;
        d.steps = (int)std::min<int64_t>(Q, q->steps_left);
        d.k = q->k;
        d.kf = to_float(q->k);
    }
    if (S->resident.empty()) return cudaSuccess;
    return cudaMemcpyAsync(S->d_grids, S->h_grids, sizeof(GridDesc) * S->resident.size(), cudaMemcpyHostToDevice,
                           S->stream);
}

static cudaError_t run_quantum(sp_server *S, int Q) {
    if (!S->graph_valid) {
        if (S->graph) {
            cudaGraphExecDestroy(S->graph);
            S->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        for (int j = 0; j < Q && e == cudaSuccess; ++j)
            for (int kd = 0; kd < 4 && e == cudaSuccess; ++kd)
                if (S->kind_n[kd] > 0)
                    e = launch_batch(kd, S->d_grids, S->d_tiles + S->kind_off[kd], S->kind_n[kd], j, S->stream);
        cudaError_t e2 = cudaStreamEndCapture(S->stream, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&S->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        S->graph_valid = true;
    }
    return cudaGraphLaunch(S->graph, S->stream);
}

static void finish_locked(sp_server *S, Req *q, int status) {
    q->status = status;
    q->done = true;
    q->t_finish = now_s(S->t0);
    S->finished += status == SP_OK;
    S->failed += status != SP_OK;
    S->cv_done.notify_all();
}

static void free_buffers(sp_server *S, Req *q) {
    for (int l = 0; l < 2; ++l)
        for (int f = 0; f < 2; ++f)
            if (q->buf[l][f]) {
                cudaFreeAsync(q->buf[l][f], S->stream);
                q->buf[l][f] = nullptr;
            }
}

// Retire a grid whose steps are all done: mass, optional FP64 copy, free.
static int retire(sp_server *S, Req *q) {
    const int cur = q->parity;
    ReduceGeom g;
    g.nx = q->nx;
    g.ny = q->ny;
    g.nz = q->nz;
    g.dims = q->r.dims;
    g.h = q->r.h;
    g.cell_volume = q->r.dims == 3 ? (q->r.h * q->r.h) * q->r.h : q->r.h * q->r.h;
    g.c1 = q->r.params.c1;
    g.c2 = q->r.params.c2;
    const int nb = reduce_blocks(q->N, S->n_sm);
    double *d_out = S->d_partials + 2 * (size_t)S->nred;
    // the mass of the conserved field (Model C: rho)
    const int mf = q->r.model == SP_MODEL_C ? 1 : 0;
    cudaError_t e = launch_reduce(q->r.params.dtype, SP_MASS, q->buf[cur][mf], g, S->d_partials, nb, d_out, S->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->h_scalar, d_out, sizeof(double), cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess && q->r.return_fields) {
        q->host.resize((size_t)q->N * q->nf);
        for (int f = 0; f < q->nf && e == cudaSuccess; ++f) {
            double *dst = q->host.data() + (size_t)f * q->N;
            if (q->r.params.dtype == SP_F64) {
                e = cudaMemcpyAsync(dst, q->buf[cur][f], q->N * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
            } else {
                double *tmp = nullptr;  // stream-ordered FP64 staging for the widened copy
                e = cudaMallocAsync(&tmp, q->N * sizeof(double), S->stream);
                if (e == cudaSuccess) e = launch_convert_to_f64(q->r.params.dtype, q->buf[cur][f], tmp, q->N, S->stream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(dst, tmp, q->N * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
                if (tmp) cudaFreeAsync(tmp, S->stream);
            }
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    q->mass = *S->h_scalar;
    free_buffers(S, q);
    return e == cudaSuccess ? SP_OK : SP_ECUDA;
}

static void scheduler(sp_server *S) {
    cudaSetDevice(S->device);
    bool changed = true;
    for (;;) {
        std::vector<Req *> admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty() || !S->resident.empty(); });
            if (S->stop) break;
            // admission by priority, arrival order within a priority; a request that
            // does not fit yet lets later ones pass (sp_admission_order)
            const int np = (int)S->pending.size();
            std::vector<size_t> bytes(np);
            std::vector<int> prio(np), order(np);
            for (int i = 0; i < np; ++i) {
                bytes[i] = S->pending[i]->bytes;
                prio[i] = S->pending[i]->r.priority;
            }
            const int free_slots = std::max(0, S->max_slots - (int)S->resident.size());
            const int na = sp_admission_order(np, bytes.data(), prio.data(), S->budget - S->used, free_slots,
                                              order.data());
            std::vector<bool> taken(np, false);
            for (int a = 0; a < na; ++a) {
                Req *q = S->pending[order[a]];
                S->used += q->bytes;
                admit.push_back(q);
                taken[order[a]] = true;
            }
            std::deque<Req *> rest;
            for (int i = 0; i < np; ++i)
                if (!taken[i]) rest.push_back(S->pending[i]);
            S->pending.swap(rest);
        }
        // allocate and initialise outside the lock
        for (Req *q : admit) {
            int rc = SP_OK;
            if (q->r.fault == 1) rc = SP_ENOMEM;  // injected allocation failure
            for (int l = 0; l < 2 && rc == SP_OK; ++l)
                for (int f = 0; f < q->nf && rc == SP_OK; ++f)
                    if (cudaMallocAsync(&q->buf[l][f], q->N * esize_of(q->r.params.dtype), S->stream) != cudaSuccess) {
                        cudaGetLastError();
                        rc = SP_ENOMEM;
                    }
            if (rc == SP_OK) {
                const sp_params &p = q->r.params;
                if (launch_ic(p.dtype, q->buf[0][0], q->nf > 1 ? q->buf[0][1] : nullptr, q->r.model, q->r.dims, q->nx,
                              q->ny, q->nz, p.seed, p.ic_kind, p.ic_mean, p.ic_amp, p.gs_patches, p.gs_patch,
                              S->stream, S->n_sm) != cudaSuccess)
                    rc = SP_ECUDA;
            }
            std::lock_guard<std::mutex> lk(S->mu);
            if (rc == SP_OK) {
                q->t_admit = now_s(S->t0);
                S->resident.push_back(q);
                S->admitted++;
                changed = true;
            } else {
                free_buffers(S, q);
                S->used -= q->bytes;
                finish_locked(S, q, rc);
            }
        }
        if (S->resident.empty()) continue;
        cudaError_t e = cudaSuccess;
        if (changed) {
            e = rebuild_tables(S);
            S->graph_valid = false;
            changed = false;
        }
        const int Q = S->quantum;
        const auto tq = std::chrono::steady_clock::now();
        if (e == cudaSuccess) e = upload_descriptors(S, Q);
        if (e == cudaSuccess) e = run_quantum(S, Q);
        if (e == cudaSuccess) e = cudaEventRecord(S->ev, S->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(S->ev);
        S->busy_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - tq).count();
        S->quanta++;
        // advance bookkeeping; retire finished grids
        std::vector<Req *> keep, done;
        for (Req *q : S->resident) {
            const int64_t adv = std::min<int64_t>(Q, q->steps_left);
            q->steps_left -= adv;
            q->steps_done += adv;
            q->parity ^= (int)(adv & 1);
            S->lups += (double)q->N * (double)adv;
            if (e != cudaSuccess || q->steps_left == 0) done.push_back(q);
            else keep.push_back(q);
        }
        for (Req *q : done) {
            const int rc = e != cudaSuccess ? SP_ECUDA : retire(S, q);
            std::lock_guard<std::mutex> lk(S->mu);
            S->used -= q->bytes;
            finish_locked(S, q, rc);
        }
        if (!done.empty()) changed = true;
        std::lock_guard<std::mutex> lk(S->mu);
        S->resident.swap(keep);
        if (e != cudaSuccess) {
            S->err = cudaGetErrorString(e);
            cudaGetLastError();
        }
    }
}

extern "C" int sp_admission_order(int n, const size_t bytes[], const int priority[], size_t free_bytes,
                                  int free_slots, int order[]) {
    if (n <= 0) return 0;
    if (!bytes || !priority || !order) return -1;
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return priority[a] > priority[b]; });
    int na = 0;
    for (int i : idx) {
        if (na >= free_slots) break;
        if (bytes[i] <= free_bytes) {
            free_bytes -= bytes[i];
            order[na++] = i;
        }
    }
    return na;
}

extern "C" int sp_server_create(size_t hbm_budget_bytes, int max_slots, int quantum_steps, sp_server **out) {
    if (!out) return SP_EINVAL;
    *out = nullptr;
    if (hbm_budget_bytes == 0 || max_slots < 1 || quantum_steps < 1 || quantum_steps > 100000) return SP_EINVAL;
    sp_server *S = new (std::nothrow) sp_server();
    if (!S) return SP_ENOMEM;
    S->budget = hbm_budget_bytes;
    S->max_slots = max_slots;
    S->quantum = quantum_steps;
    S->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->n_sm, cudaDevAttrMultiProcessorCount, S->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev, cudaEventBlockingSync | cudaEventDisableTiming);
    if (e == cudaSuccess) e = set_batch_attributes();
    if (e == cudaSuccess) {
        S->nred = 2 * S->n_sm * kReduceBlocksPerSM;
        e = cudaMalloc(&S->d_partials, sizeof(double) * (2 * (size_t)S->nred + 1));
    }
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_scalar, sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (S->stream) cudaStreamDestroy(S->stream);
        if (S->ev) cudaEventDestroy(S->ev);
        if (S->d_partials) cudaFree(S->d_partials);
        delete S;
        return SP_ECUDA;
    }
    S->th = std::thread(scheduler, S);
    *out = S;
    return SP_OK;
}

extern "C" int sp_submit(sp_server *S, const sp_request *r, uint64_t *ticket) {
    if (!S || !r || !ticket) return SP_EINVAL;
    *ticket = 0;
    sp_params p = r->params;
    const int dims = r->dims;
    if (dims != 2 && dims != 3) return SP_EINVAL;
    const int st = p.stencil == SP_LAP_DEFAULT ? (dims == 2 ? SP_LAP_5 : SP_LAP_7) : p.stencil;
    p.stencil = st;
    if (p.dtype != SP_F64 && p.dtype != SP_F32) return SP_EINVAL;  // the serving kernels cover FP64 and FP32
    if (p.scheme != SP_SCHEME_FD) return SP_EINVAL;                 // and the finite-difference scheme
    if (r->model == SP_MODEL_H) return SP_EINVAL;                   // of the one- and two-field models
    if (st == SP_LAP_GENERATED) return SP_EINVAL;                  // with the fixed stencils
    double factor = 0;
    if (int rc = sp_check_stability(r->model, dims, r->h, r->dt, &p, &factor)) return rc;
    const int64_t nx = r->shape[0], ny = r->shape[1], nz = dims == 2 ? 1 : r->shape[2];
    if (nx < 1 || ny < 1 || nz < 1 || nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20)) return SP_EINVAL;
    if (dims == 3 && nx * ny * nz > (int64_t)1 << 31) return SP_EINVAL;
    if (r->nsteps < 1) return SP_EINVAL;
    if (r->model == SP_GRAY_SCOTT && p.ic_kind == SP_IC_NOISE &&
        (p.gs_patches < 0 || p.gs_patches > kMaxPatches || p.gs_patch < 0 || p.gs_patch > nx || p.gs_patch > ny ||
         (dims == 3 && p.gs_patch > nz)))
        return SP_EINVAL;
    Req *q = new (std::nothrow) Req();
    if (!q) return SP_ENOMEM;
    q->r = *r;
    q->r.params = p;
    q->stencil = st;
    q->nf = (r->model == SP_GRAY_SCOTT || r->model == SP_MODEL_C) ? 2 : 1;
    q->nx = (int)nx;
    q->ny = (int)ny;
    q->nz = (int)nz;
    q->N = (uint64_t)nx * ny * nz;
    q->bytes = 2 * (size_t)q->nf * q->N * esize_of(p.dtype);
    q->k = consts_of(q->r, st);
    q->steps_left = r->nsteps;
    std::lock_guard<std::mutex> lk(S->mu);
    if (q->bytes > S->budget) {
        delete q;
        return SP_EBUDGET;
    }
    q->ticket = S->next_ticket++;
    q->t_submit = now_s(S->t0);
    S->all[q->ticket] = q;
    S->pending.push_back(q);
    S->submitted++;
    *ticket = q->ticket;
    S->cv_work.notify_all();
    return SP_OK;
}

static void fill_result(const Req *q, sp_result *out) {
    out->status = q->status;
    out->steps_done = q->steps_done;
    out->t_submit = q->t_submit;
    out->t_admit = q->t_admit;
    out->t_finish = q->t_finish;
    out->mass = q->mass;
    out->fields = q->host.empty() ? nullptr : q->host.data();
    out->n_values = q->host.size();
}

extern "C" int sp_poll(sp_server *S, uint64_t ticket, sp_result *out) {
    if (!S || !out) return SP_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return SP_ENOTFOUND;
    fill_result(it->second, out);
    return it->second->done ? it->second->status : SP_PENDING;
}

extern "C" int sp_wait(sp_server *S, uint64_t ticket, double timeout_s, sp_result *out) {
    if (!S || !out || !(timeout_s >= 0)) return SP_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return SP_ENOTFOUND;
    Req *q = it->second;
    const bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return q->done; });
    fill_result(q, out);
    if (!ok) return SP_ETIMEOUT;
    return q->status;
}

extern "C" int sp_release(sp_server *S, uint64_t ticket) {
    if (!S) return SP_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return SP_ENOTFOUND;
    if (!it->second->done) return SP_EBUSY;
    delete it->second;
    S->all.erase(it);
    return SP_OK;
}

extern "C" int sp_server_get_stats(sp_server *S, sp_server_stats *st) {
    if (!S || !st) return SP_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    st->submitted = S->submitted;
    st->admitted = S->admitted;
    st->finished = S->finished;
    st->failed = S->failed;
    st->quanta = S->quanta;
    st->resident = (int64_t)S->resident.size();
    st->pending = (int64_t)S->pending.size();
    st->hbm_in_use = S->used;
    st->lups = S->lups;
    st->busy_s = S->busy_s;
    return SP_OK;
}

extern "C" int sp_server_destroy(sp_server *S) {
    if (!S) return SP_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    cudaStreamSynchronize(S->stream);
    for (Req *q : S->resident) free_buffers(S, q);
    for (auto &kv : S->all) {
        if (!kv.second->done) free_buffers(S, kv.second);
        delete kv.second;
    }
    cudaStreamSynchronize(S->stream);
    if (S->graph) cudaGraphExecDestroy(S->graph);
    if (S->d_grids) cudaFree(S->d_grids);
    if (S->h_grids) cudaFreeHost(S->h_grids);
    if (S->d_tiles) cudaFree(S->d_tiles);
    if (S->d_partials) cudaFree(S->d_partials);
    if (S->h_scalar) cudaFreeHost(S->h_scalar);
    if (S->ev) cudaEventDestroy(S->ev);
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
    return SP_OK;
}

// sp_runtime.cu -- the C ABI of include/sp.h: simulation handles, argument
// validation, the forward-Euler stability check, device buffers, initial
// conditions, stepping, host transfers and reductions.
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "sp_internal.h"

using namespace sp;

namespace sp {
thread_local int g_step_variant = 0;
}

// Polls before the kernels' bounded device waits give up (0: their default);
// sp_set_wait_polls, a test hook.
static std::atomic<long long> g_wait_polls{0};

extern "C" int sp_set_wait_polls(long long polls) {
    g_wait_polls.store(polls < 0 ? -1 : polls, std::memory_order_relaxed);
    return 0;
}

// --------------------------------------------------------------- errors --

static thread_local std::string g_last_error;

static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define SP_CUDA(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return fail(SP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" const char *sp_last_error(void) { return g_last_error.c_str(); }
extern "C" int sp_version(void) { return 100; }

// ---------------------------------------------------- stencil metadata --

static int stencil_dims(int st) { return st >= SP_LAP_7 ? 3 : 2; }  // fixed stencils
static int stencil_radius(int st) { return (st == SP_LAP_9CROSS4 || st == SP_LAP_13CROSS4) ? 2 : 1; }
static int stencil_q(int st) {
    static const int q[7] = {1, 6, 12, 1, 30, 12, 1};
    return q[st];
}
// max over theta of the symbol lambda(theta) (eigenvalue of -h^2 L_h)
static double stencil_lambda_max(int st) {
    static const double lm[6] = {8.0, 16.0 / 3.0, 32.0 / 3.0, 12.0, 92.0 / 15.0, 16.0};
    return lm[st];
}

static int resolve_stencil(int st, int dims) {
    if (st == SP_LAP_DEFAULT) return dims == 2 ? SP_LAP_5 : SP_LAP_7;
    return st;
}

extern "C" void sp_params_default(int model, int dims, sp_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->c1 = 1.0;
    p->c2 = 1.0;
    p->kappa = 1.0;
    p->Du = 0.16;
    p->Dv = 0.08;
    p->F = 0.035;
    p->k = 0.065;
    p->c3 = 0.5;
    p->stencil = dims == 3 ? SP_LAP_7 : SP_LAP_5;
    p->stencil_order = 2;
    p->dtype = SP_F64;
    p->seed = 0;
    p->ic_kind = SP_IC_NOISE;
    p->ic_mean = 0.0;
    p->ic_amp = 0.01;
    p->gs_patches = model == SP_GRAY_SCOTT ? 64 : 0;
    p->gs_patch = model == SP_GRAY_SCOTT ? 20 : 0;
    p->steps_per_launch = 0;
    p->flags = 0;
}

static bool is_finite(double x) { return std::isfinite(x); }

// Largest |sigma| of the linearised update over the stencil's spectrum, where
// sigma is the growth rate of a Fourier mode:
//   Allen-Cahn:    sigma = -lam + a,            a in {c1 - 3 c2 (|phi| = 1), c1 (phi = 0)}
//   Cahn-Hilliard: sigma = -lam (kappa lam + a), a in {3 c2 - c1, -c1}
//   Gray-Scott:    about (u, v) = (1, 0): sigma_u = -Du lam - F, sigma_v = -Dv lam - (F + k)
// with lam in [0, lambda_max / h^2].  Forward Euler is stable when dt*max|sigma| <= 2.
static double max_growth(int model, int st, double h, const sp_params &p, int dims) {
    double lm = 0;
    if (st == SP_LAP_GENERATED) {
        double wk[kMaxGenRadius + 1];
        generated_weights(p.stencil_order, dims, wk, &lm);
    } else {
        lm = stencil_lambda_max(st);
    }
    const double lam = lm / (h * h);
    double m = 0.0;
    if (model == SP_ALLEN_CAHN) {
        const double as[2] = {p.c1 - 3.0 * p.c2, p.c1};
        for (double a : as) m = std::fmax(m, std::fmax(std::fabs(a), std::fabs(-lam + a)));
    } else if (model == SP_CAHN_HILLIARD) {
        const double as[2] = {3.0 * p.c2 - p.c1, -p.c1};
        for (double a : as) {
            m = std::fmax(m, std::fabs(lam * (p.kappa * lam + a)));
            if (p.kappa > 0) {
                const double ls = -a / (2.0 * p.kappa);
                if (ls > 0 && ls < lam) m = std::fmax(m, std::fabs(ls * (p.kappa * ls + a)));
            }
        }
    } else if (model == SP_GRAY_SCOTT) {
        m = std::fmax(std::fabs(p.Du * lam + p.F), std::fabs(p.Dv * lam + p.F + p.k));
    } else if (model == SP_MODEL_H) {
        // Model H: m as Cahn-Hilliard, j diffuses with unit mobility
        const double as[2] = {3.0 * p.c2 - p.c1, -p.c1};
        for (double a : as) {
            m = std::fmax(m, std::fabs(lam * (p.kappa * lam + a)));
            if (p.kappa > 0) {
                const double ls = -a / (2.0 * p.kappa);
                if (ls > 0 && ls < lam) m = std::fmax(m, std::fabs(ls * (p.kappa * ls + a)));
            }
        }
        m = std::fmax(m, lam);
    } else {
        // Model C: phi as Allen-Cahn about rho = 0, rho diffuses with unit mobility
        const double as[2] = {p.c1 - 3.0 * p.c2, p.c1};
        for (double a : as) m = std::fmax(m, std::fmax(std::fabs(a), std::fabs(-lam + a)));
        m = std::fmax(m, lam);
    }
    return m;
}

static int validate_params(int model, int dims, double h, double dt, const sp_params &p, int *st_out) {
    if (model < SP_ALLEN_CAHN || model > SP_MODEL_H) return fail(SP_EINVAL, "unknown model %d", model);
    if (dims != 2 && dims != 3) return fail(SP_EINVAL, "dims must be 2 or 3 (got %d)", dims);
    const int st = resolve_stencil(p.stencil, dims);
    if (st < SP_LAP_5 || st > SP_LAP_GENERATED) return fail(SP_EINVAL, "unknown stencil %d", p.stencil);
    if (st == SP_LAP_GENERATED) {
        double wk[kMaxGenRadius + 1];
        if (generated_weights(p.stencil_order, dims, wk, nullptr) != SP_OK)
            return fail(SP_EINVAL, "stencil_order must be even and in [2, %d] (got %d)", 2 * kMaxGenRadius,
                        p.stencil_order);
        if (model == SP_MODEL_H) return fail(SP_EINVAL, "Model H uses the fixed stencils");
    } else if (stencil_dims(st) != dims) {
        return fail(SP_EINVAL, "stencil %d is %dD but the grid is %dD", st, stencil_dims(st), dims);
    }
    if (!(is_finite(h) && h > 0)) return fail(SP_EINVAL, "h must be finite and > 0");
    if (!(is_finite(dt) && dt > 0)) return fail(SP_EINVAL, "dt must be finite and > 0");
    const double vals[8] = {p.c1, p.c2, p.kappa, p.Du, p.Dv, p.F, p.k, p.c3};
    for (double v : vals)
        if (!is_finite(v)) return fail(SP_EINVAL, "non-finite model coefficient");
    if (p.dtype < SP_F64 || p.dtype > SP_BF16_F32) return fail(SP_EINVAL, "unknown dtype %d", p.dtype);
    if (p.flags & ~(SP_FLAG_AUTOTUNE | SP_FLAG_BF16_NO_BOUND)) return fail(SP_EINVAL, "unknown flags 0x%x", p.flags);
    if (p.dtype == SP_BF16_F32 && !(p.flags & SP_FLAG_BF16_NO_BOUND))
        return fail(SP_EINVAL,
                    "BF16 storage meets no accuracy bound on these models (relative L2 vs FP64 of 0.04 to 1.0 over "
                    "the benchmark runs); use SP_F32, or set SP_FLAG_BF16_NO_BOUND to accept unbounded error");
    if (p.steps_per_launch < 0) return fail(SP_EINVAL, "steps_per_launch must be >= 0");
    if (p.ic_kind != SP_IC_NOISE && p.ic_kind != SP_IC_CONSTANT) return fail(SP_EINVAL, "unknown ic_kind %d", p.ic_kind);
    if (p.scheme != SP_SCHEME_FD && p.scheme != SP_SCHEME_SPECTRAL) return fail(SP_EINVAL, "unknown scheme %d", p.scheme);
    if (p.scheme == SP_SCHEME_SPECTRAL) {
        if (model != SP_ALLEN_CAHN && model != SP_CAHN_HILLIARD)
            return fail(SP_EINVAL, "the spectral scheme covers Allen-Cahn and Cahn-Hilliard");
        if (p.dtype != SP_F64 && p.dtype != SP_F32) return fail(SP_EINVAL, "the spectral scheme runs in FP64 or FP32");
        if (p.steps_per_launch > 1) return fail(SP_EINVAL, "the spectral scheme runs one step per launch");
    }
    if (!is_finite(p.ic_mean) || !is_finite(p.ic_amp)) return fail(SP_EINVAL, "non-finite ic_mean/ic_amp");
    *st_out = st;
    return SP_OK;
}

extern "C" int sp_check_stability(int model, int dims, double h, double dt, const sp_params *p, double *factor) {
    if (!p) return fail(SP_EINVAL, "params is NULL");
    int st;
    if (int rc = validate_params(model, dims, h, dt, *p, &st)) return rc;
    if (p->scheme == SP_SCHEME_SPECTRAL) {
        // the implicit linear part needs 1 - dt L(k) > 0 for every k
        double f = dt * p->c1;
        if (model == SP_CAHN_HILLIARD) {
            if (!(p->kappa > 0)) return fail(SP_EUNSTABLE, "spectral Cahn-Hilliard needs kappa > 0");
            f = dt * p->c1 * p->c1 / (4.0 * p->kappa);
        }
        if (factor) *factor = f;
        if (!(f < 1.0)) return fail(SP_EUNSTABLE, "dt max L(k) = %.6g >= 1: the semi-implicit step is undefined", f);
        return SP_OK;
    }
    const double f = dt * max_growth(model, st, h, *p, dims);
    if (factor) *factor = f;
    if (!(f <= 2.0)) return fail(SP_EUNSTABLE, "dt*max|sigma| = %.6g > 2: forward Euler is unstable", f);
    return SP_OK;
}

// ---------------------------------------------------------- the handle --

struct sp_sim {
    int model, dims, stencil, dtype, nf;
    int nx, ny, nz;
    uint64_t N;
    double h, dt;
    sp_params p;
    size_t esize;
    void *f[2][4];        // [level][field] (Model H: m and up to three components of j)
    int cur;              // current level
    int64_t steps;
    cudaStream_t stream;  // library-owned stream
    double *d_partials;   // reduction scratch: 2 doubles per block, the result, then the wait flag
    int *d_flag;          // set by a kernel whose bounded wait expired (inside d_partials)
    bool waits_used;      // a kernel with bounded waits has run (the flag is checked)
    int nred;
    double *h_out;        // pinned host scalar
    double *d_stage;      // FP64 staging for converted transfers (lazy)
    size_t stage_elems;
    StepConsts k;
    int device, n_sm;
    cudaGraphExec_t graph[2];  // kGraphSteps steps starting from level 0 / level 1
    int spl;                   // steps fused per launch (temporal blocking)
    int variant;               // kernel family (see g_step_variant)
    void *mu_tmp;              // unfused ablation: mu temporary (allocated on first use)
    bool tune_pending;         // autotune on the next long sp_step
    double genw[kMaxGenRadius + 1];  // generated stencil: kernel weights (d w_0, w_1, ..., w_r)
    SpectralPlan *spec;        // semi-implicit spectral scheme (else null)
    bool spec_dirty;           // the resident spectrum must be recomputed from phi
};

// Steps per captured graph.  A graph holds kGraphSteps / spl launches, an even
// number for spl in {1, 2, 4}, so a replay returns to the level it started from.
constexpr int kGraphSteps = 32;

static size_t dtype_size(int dt) { return dt == SP_F64 ? 8 : (dt == SP_F32 ? 4 : 2); }

static StepConsts make_consts(const sp_sim &s) {
    StepConsts k;
    const double q_h2 = ((double)stencil_q(s.stencil) * s.h) * s.h;
    k.c1 = s.p.c1;
    k.c2 = s.p.c2;
    k.sAC = 1.0 / q_h2;
    k.kq = s.p.kappa / q_h2;
    k.dq = s.dt / q_h2;
    k.duq = s.p.Du / q_h2;
    k.dvq = s.p.Dv / q_h2;
    k.F = s.p.F;
    k.Fk = s.p.F + s.p.k;
    k.dt = s.dt;
    k.c3 = s.p.c3;
    k.c3x2 = 2.0 * s.p.c3;
    return k;
}

static void release(sp_sim *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (int l = 0; l < 2; ++l)
        for (int f = 0; f < 4; ++f)
            if (s->f[l][f]) cudaFree(s->f[l][f]);
    if (s->d_partials) cudaFree(s->d_partials);
    if (s->d_stage) cudaFree(s->d_stage);
    if (s->mu_tmp) cudaFree(s->mu_tmp);
    spectral_destroy(s->spec);
    for (int l = 0; l < 2; ++l)
        if (s->graph[l]) cudaGraphExecDestroy(s->graph[l]);
    if (s->h_out) cudaFreeHost(s->h_out);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

extern "C" int sp_create(int model, int dims, const int64_t shape[3], double h, double dt, const sp_params *p,
                         sp_sim **out) {
    if (!out) return fail(SP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!shape) return fail(SP_EINVAL, "shape is NULL");
    sp_params prm;
    if (p) prm = *p;
    else sp_params_default(model, dims, &prm);
    int st;
    if (int rc = validate_params(model, dims, h, dt, prm, &st)) return rc;
    const int64_t nx = shape[0], ny = shape[1], nz = dims == 2 ? 1 : shape[2];
    if (dims == 2 && !(shape[2] == 0 || shape[2] == 1)) return fail(SP_EINVAL, "2D grid needs shape[2] in {0, 1}");
    if (nx < 1 || ny < 1 || nz < 1) return fail(SP_EINVAL, "grid sides must be >= 1");
    if (nx > INT_MAX || ny > INT_MAX || nz > INT_MAX) return fail(SP_EINVAL, "grid side too large");
    if (dims == 3 && nx * ny > (int64_t)INT_MAX) return fail(SP_EINVAL, "3D plane nx*ny must be < 2^31");
    if (model == SP_GRAY_SCOTT && prm.ic_kind == SP_IC_NOISE) {
        if (prm.gs_patches < 0 || prm.gs_patches > kMaxPatches)
            return fail(SP_EINVAL, "gs_patches must be in [0, %d]", kMaxPatches);
        if (prm.gs_patch < 0 || prm.gs_patch > nx || prm.gs_patch > ny || (dims == 3 && prm.gs_patch > nz))
            return fail(SP_EINVAL, "gs_patch must be in [0, min side]");
    }
    double factor = 0;
    if (int rc = sp_check_stability(model, dims, h, dt, &prm, &factor)) return rc;

    sp_sim *s = new (std::nothrow) sp_sim();
    if (!s) return fail(SP_ENOMEM, "host allocation failed");
    std::memset(s, 0, sizeof *s);
    s->model = model;
    s->dims = dims;
    s->stencil = st;
    s->dtype = prm.dtype;
    s->nf = model == SP_MODEL_H ? 1 + dims : ((model == SP_GRAY_SCOTT || model == SP_MODEL_C) ? 2 : 1);
    s->nx = (int)nx;
    s->ny = (int)ny;
    s->nz = (int)nz;
    s->N = (uint64_t)nx * ny * nz;
    s->h = h;
    s->dt = dt;
    s->p = prm;
    s->p.stencil = st;
    s->esize = dtype_size(prm.dtype);
    s->k = make_consts(*s);
    s->spl = st == SP_LAP_GENERATED ? 1
             : dims == 3 && prm.scheme == SP_SCHEME_FD
                 ? steps_per_launch_3d(prm.dtype, model, (int)nx, prm.steps_per_launch)
                 : steps_per_launch(dims, prm.dtype, model, prm.steps_per_launch);
    if (st == SP_LAP_GENERATED) generated_weights(prm.stencil_order, dims, s->genw, nullptr);
    s->variant = 0;
    s->tune_pending = (prm.flags & SP_FLAG_AUTOTUNE) != 0 && prm.steps_per_launch == 0;

    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        release(s);
        return fail(SP_ECUDA, "device setup: %s", cudaGetErrorString(e));
    }
    const size_t bytes = s->N * s->esize;
    for (int l = 0; l < 2; ++l)
        for (int f = 0; f < s->nf; ++f) {
            e = cudaMalloc(&s->f[l][f], bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                release(s);
                return fail(SP_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
            }
        }
    s->nred = reduce_blocks(s->N, s->n_sm);
    e = cudaMalloc(&s->d_partials, sizeof(double) * (2 * (size_t)s->nred + 2));
    if (e == cudaSuccess) {
        s->d_flag = reinterpret_cast<int *>(s->d_partials + 2 * (size_t)s->nred + 1);
        e = cudaMemset(s->d_flag, 0, sizeof(int));
    }
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_out, sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        release(s);
        return fail(SP_ENOMEM, "scratch allocation failed: %s", cudaGetErrorString(e));
    }
    if (model == SP_MODEL_H || (st == SP_LAP_GENERATED && model == SP_CAHN_HILLIARD) ||
        (prm.scheme == SP_SCHEME_FD && (twopass_applies(dims, prm.dtype, st, model) ||
                                        (planes27_applies(dims, prm.dtype, st, model) && model == SP_CAHN_HILLIARD)))) {
        e = cudaMalloc(&s->mu_tmp, s->N * (s->dtype == SP_F64 ? sizeof(double) : sizeof(float)));
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->mu_tmp = nullptr;
            release(s);
            return fail(SP_ENOMEM, "mu buffer: %s", cudaGetErrorString(e));
        }
    }
    e = launch_ic(s->dtype, s->f[0][0], (s->nf > 1 && model != SP_MODEL_H) ? s->f[0][1] : nullptr, model, dims, s->nx,
                  s->ny, s->nz, prm.seed, prm.ic_kind, prm.ic_mean, prm.ic_amp, prm.gs_patches, prm.gs_patch, s->stream,
                  s->n_sm);
    if (e == cudaSuccess && model == SP_MODEL_H) {
        void *j[3] = {s->f[0][1], s->f[0][2], dims == 3 ? s->f[0][3] : nullptr};
        e = launch_ic_currents(s->dtype, j, dims, s->N, prm.seed, prm.ic_kind, prm.ic_amp, s->stream, s->n_sm);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        release(s);
        return fail(SP_ECUDA, "initial condition: %s", cudaGetErrorString(e));
    }
    if (prm.scheme == SP_SCHEME_SPECTRAL) {
        int rc = spectral_create(s->dtype, dims, s->nx, s->ny, s->nz, &s->spec);
        if (rc == SP_OK) rc = spectral_load(s->spec, s->f[0][0], s->stream);
        if (rc == SP_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = SP_ECUDA;
        if (rc != SP_OK) {
            release(s);
            return fail(rc, "spectral set-up: %s", spectral_last_error());
        }
    }
    *out = s;
    return SP_OK;
}

static cudaStream_t pick(sp_sim *s, void *stream) { return stream ? (cudaStream_t)stream : s->stream; }

static cudaError_t launch_one_step_impl(sp_sim *s, cudaStream_t st, int k);

static cudaError_t launch_one_step(sp_sim *s, cudaStream_t st, int k = 1) {
    g_step_variant = s->variant;
    const cudaError_t e = launch_one_step_impl(s, st, k);
    g_step_variant = 0;
    return e;
}

static cudaError_t launch_one_step_impl(sp_sim *s, cudaStream_t st, int k) {
    StepArgs a;
    a.in0 = s->f[s->cur][0];
    a.in1 = s->nf > 1 ? s->f[s->cur][1] : s->f[s->cur][0];
    a.out0 = s->f[1 - s->cur][0];
    a.out1 = s->nf > 1 ? s->f[1 - s->cur][1] : s->f[1 - s->cur][0];
    a.nx = s->nx;
    a.ny = s->ny;
    a.nz = s->nz;
    a.k = s->k;
    a.kf = to_float(s->k);
    a.flag = s->d_flag;
    a.wait_polls = g_wait_polls.load(std::memory_order_relaxed);
    if (s->variant == kTmaFamily) s->waits_used = true;
    if (s->stencil == SP_LAP_GENERATED)
        return launch_generated(s->model, s->dtype, s->p.stencil_order, s->dims, s->genw, a, s->mu_tmp, st, s->n_sm);
    if (s->variant == kUnfusedFamily) return launch_unfused_ch(s->dtype, s->stencil, a, s->mu_tmp, st, s->n_sm);
    if (s->model == SP_MODEL_H) {
        void *in[4] = {nullptr, nullptr, nullptr, nullptr}, *out[4] = {nullptr, nullptr, nullptr, nullptr};
        for (int f = 0; f < s->nf; ++f) {
            in[f] = s->f[s->cur][f];
            out[f] = s->f[1 - s->cur][f];
        }
        const double c3g = s->p.c3 * (stencil_radius(s->stencil) == 1 ? 1.0 / (2.0 * s->h) : 1.0 / (12.0 * s->h));
        return launch_model_h(s->dtype, s->stencil, in, out, s->mu_tmp, s->nx, s->ny, s->nz, s->k, c3g, st, s->n_sm);
    }
    if (twopass_applies(s->dims, s->dtype, s->stencil, s->model)) {
        if (s->variant == 0) return launch_ch_twopass_f64(s->stencil, a, s->mu_tmp, st, s->n_sm);
        g_step_variant = 0;  // kFusedFamily: launch_step_f64's family 0
    }
    if (planes27_applies(s->dims, s->dtype, s->stencil, s->model) && s->variant != 1) {
        if (s->variant == 0) return launch_planes27_f64(s->model, a, s->mu_tmp, st, s->n_sm);
        g_step_variant = 0;  // kZregFamily: the z-streaming kernel is launch_step_f64's family 0
    }
    switch (s->dtype) {
    case SP_F64: return launch_step_f64(s->model, s->stencil, a, st, s->n_sm, k);
    case SP_F32: return launch_step_f32(s->model, s->stencil, a, st, s->n_sm, k);
    default: return launch_step_bf16(s->model, s->stencil, a, st, s->n_sm, k);
    }
}

// ---------------------------------------------------------------- autotune --
//
// Candidates: (steps per launch, kernel family).  Every candidate computes the
// same values bit for bit, so the timed steps are ordinary steps of the run.
// The winner is cached per (model, stencil, dtype, dims, log2 of the grid size).

struct TuneKey {
    int model, stencil, dtype, dims, size_log2;
    bool operator<(const TuneKey &o) const {
        return std::tie(model, stencil, dtype, dims, size_log2) < std::tie(o.model, o.stencil, o.dtype, o.dims, o.size_log2);
    }
};
struct TuneChoice {
    int spl, variant;
};
constexpr int kTuneSteps = 8;  // divisible by every candidate's steps per launch
constexpr int64_t kAutotuneMinSteps = 2 * 4 * kTuneSteps;
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneChoice> g_tune_cache;

// Graphs hold launches of one configuration: drop them when it changes.
static void set_launch_config(sp_sim *s, TuneChoice c) {
    if (c.spl == s->spl && c.variant == s->variant) return;
    for (int l = 0; l < 2; ++l)
        if (s->graph[l]) {
            cudaGraphExecDestroy(s->graph[l]);
            s->graph[l] = nullptr;
        }
    s->spl = c.spl;
    s->variant = c.variant;
}

static TuneKey tune_key(const sp_sim *s) {
    int lg = 0;
    while (lg < 62 && (1ull << (lg + 1)) <= s->N) ++lg;
    return {s->model, s->stencil, s->dtype, s->dims, lg};
}

static std::vector<TuneChoice> tune_candidates(const sp_sim *s) {
    std::vector<TuneChoice> c;
    if (s->spec || s->model == SP_MODEL_H || s->stencil == SP_LAP_GENERATED) return {{1, 0}};
    if (s->dims == 2 && s->dtype != SP_F64) {
        c.push_back({1, 1});
        for (int spl : {1, 2, 4}) c.push_back({spl, 0});
    } else if (s->dims == 2 || s->stencil == SP_LAP_27 || s->dtype != SP_F64) {
        c.push_back({1, 0});
        c.push_back({1, 1});
        if (s->dims == 3 && s->dtype != SP_F64) c.push_back({1, 2});
        if (s->dims == 3 && s->dtype != SP_F64 && s->model != SP_MODEL_C && s->nx % (int)(16 / s->esize) == 0 &&
            tma_available())
            c.push_back({1, kTmaFamily});
        if (planes27_applies(s->dims, s->dtype, s->stencil, s->model)) c.push_back({1, kZregFamily});
        if (s->dims == 3 && steps_per_launch_3d(s->dtype, s->model, s->nx, 2) == 2) {
            c.push_back({2, 0});  // two steps per pass, 8 rows
            c.push_back({2, 1});  // 16 rows
            if (s->model == SP_MODEL_C) {  // one step in the plane rings (else the box kernel)
                c.push_back({1, 4});
                c.push_back({1, 5});
            }
        }
        if (s->dims == 2 && s->dtype == SP_F64) {
            if (s->N <= (size_t)kSmallGrid2d) {  // small grids: steps fused per launch
                c.push_back({2, 0});
                c.push_back({4, 0});
            } else {  // two more strip shapes
                c.push_back({1, 2});
                c.push_back({1, 4});
            }
        }
    } else {
        c.push_back({1, 0});
        if (twopass_applies(s->dims, s->dtype, s->stencil, s->model)) c.push_back({1, kFusedFamily});
    }
    return c;
}

// Run the candidates on stream st (kTuneSteps steps each, timed with events);
// returns the number of steps taken.
static int64_t autotune(sp_sim *s, cudaStream_t st, int *rc) {
    *rc = SP_OK;
    const TuneKey key = tune_key(s);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            set_launch_config(s, it->second);
            return 0;
        }
    }
    const std::vector<TuneChoice> cand = tune_candidates(s);
    if (cand.size() < 2) return 0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        *rc = fail(SP_ECUDA, "autotune: cudaEventCreate failed");
        return 0;
    }
    int64_t taken = 0;
    float best = 1e30f;
    TuneChoice win = {s->spl, s->variant};
    for (int pass = 0; pass < 2; ++pass)  // pass 0 warms every candidate up, pass 1 is timed
        for (const TuneChoice &c : cand) {
            set_launch_config(s, c);
            cudaEventRecord(e0, st);
            for (int i = 0; i < kTuneSteps; i += c.spl) {
                cudaError_t e = launch_one_step(s, st, c.spl);
                if (e != cudaSuccess) {
                    *rc = fail(SP_ECUDA, "autotune launch: %s", cudaGetErrorString(e));
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return taken;
                }
                s->cur ^= 1;
                s->steps += c.spl;
                taken += c.spl;
            }
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (pass == 1 && ms < best) {
                best = ms;
                win = c;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_launch_config(s, win);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = win;
    return taken;
}

// Capture kGraphSteps steps starting from the current level into s->graph[s->cur].
static cudaError_t capture_graph(sp_sim *s) {
    const int start = s->cur;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    // one launch (of spl steps) reads the current level and writes the other one
    for (int i = 0; i < kGraphSteps && e == cudaSuccess; i += s->spl) {
        e = launch_one_step(s, s->stream, s->spl);
        s->cur ^= 1;
    }
    s->cur = start;
    const cudaError_t e2 = cudaStreamEndCapture(s->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->graph[start], g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

// Steps are issued as replays of a captured kGraphSteps-step graph (one per
// starting level) plus eager launches for the remainder.  The first step of a
// handle is always eager, so that the kernels' one-time set-up never runs
// inside a capture.
extern "C" int sp_step(sp_sim *s, int64_t nsteps, void *stream) {
    if (!s) return fail(SP_EINVAL, "sim is NULL");
    if (nsteps < 0) return fail(SP_EINVAL, "nsteps must be >= 0");
    const cudaStream_t st = pick(s, stream);
    if (s->spec) {
        // semi-implicit spectral scheme: phi stays in level 0, the spectrum on the device
        for (int64_t i = 0; i < nsteps; ++i) {
            if (s->spec_dirty) {
                if (int rc = spectral_load(s->spec, s->f[0][0], st)) return fail(rc, "%s", spectral_last_error());
                s->spec_dirty = false;
            }
            if (int rc = spectral_step(s->spec, s->model, s->f[0][0], s->f[1][0], s->h, s->dt, s->p.c1, s->p.c2,
                                       s->p.kappa, st, s->n_sm, i + 1 < nsteps))
                return fail(rc, "spectral step: %s", spectral_last_error());
            s->steps += 1;
        }
        return SP_OK;
    }
    if (s->tune_pending && nsteps >= kAutotuneMinSteps + 1) {
        s->tune_pending = false;
        if (s->steps == 0) {  // the first step takes the eager path
            SP_CUDA(launch_one_step(s, st));
            s->cur ^= 1;
            s->steps += 1;
            nsteps -= 1;
        }
        int rc = SP_OK;
        nsteps -= autotune(s, st, &rc);
        if (rc != SP_OK) return rc;
    }
    while (nsteps > 0) {
        if (nsteps >= kGraphSteps && s->steps >= s->spl + 1) {
            if (!s->graph[s->cur]) SP_CUDA(capture_graph(s));
            SP_CUDA(cudaGraphLaunch(s->graph[s->cur], st));
            s->steps += kGraphSteps;
            nsteps -= kGraphSteps;
        } else if (nsteps >= s->spl && s->spl > 1 && s->steps > 0) {
            SP_CUDA(launch_one_step(s, st, s->spl));
            s->cur ^= 1;  // one launch swaps the levels, however many steps it fuses
            s->steps += s->spl;
            nsteps -= s->spl;
        } else {
            SP_CUDA(launch_one_step(s, st));
            s->cur ^= 1;
            s->steps += 1;
            nsteps -= 1;
        }
    }
    return SP_OK;
}

static int check_field(const sp_sim *s, int field) {
    if (field < 0 || field >= s->nf) return fail(SP_EINVAL, "field %d out of range (model has %d)", field, s->nf);
    return SP_OK;
}

static int ensure_stage(sp_sim *s) {
    if (s->d_stage) return SP_OK;
    const size_t want = s->N < ((size_t)1 << 22) ? (size_t)s->N : ((size_t)1 << 22);  // <= 32 MiB
    cudaError_t e = cudaMalloc(&s->d_stage, want * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->d_stage = nullptr;
        return fail(SP_ENOMEM, "staging allocation failed: %s", cudaGetErrorString(e));
    }
    s->stage_elems = want;
    return SP_OK;
}

// After a synchronisation: SP_ETIMEOUT (and the flag cleared) if a kernel's
// bounded wait expired since the last check.
static int check_wait_flag(sp_sim *s) {
    if (!s->waits_used) return SP_OK;
    int v = 0;
    SP_CUDA(cudaMemcpy(&v, s->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (!v) return SP_OK;
    SP_CUDA(cudaMemset(s->d_flag, 0, sizeof(int)));
    return fail(SP_ETIMEOUT, "a bounded wait in the tensor-map plane ring expired: the fields are not valid");
}

extern "C" int sp_read(sp_sim *s, int field, void *host_dst, size_t bytes, int as_f64, void *stream) {
    if (!s || !host_dst) return fail(SP_EINVAL, "NULL argument");
    if (int rc = check_field(s, field)) return rc;
    const bool conv = as_f64 && s->dtype != SP_F64;
    const size_t want = s->N * (as_f64 ? sizeof(double) : s->esize);
    if (bytes != want) return fail(SP_EINVAL, "bytes = %zu, expected %zu", bytes, want);
    const cudaStream_t st = pick(s, stream);
    const void *src = s->f[s->cur][field];
    if (!conv) {
        SP_CUDA(cudaMemcpyAsync(host_dst, src, bytes, cudaMemcpyDeviceToHost, st));
    } else {
        if (int rc = ensure_stage(s)) return rc;
        for (uint64_t off = 0; off < s->N; off += s->stage_elems) {
            const uint64_t n = (s->N - off) < s->stage_elems ? (s->N - off) : s->stage_elems;
            SP_CUDA(launch_convert_to_f64(s->dtype, (const char *)src + off * s->esize, s->d_stage, n, st));
            SP_CUDA(cudaMemcpyAsync((double *)host_dst + off, s->d_stage, n * sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
        }
    }
    SP_CUDA(cudaStreamSynchronize(st));
    return check_wait_flag(s);
}

extern "C" int sp_write(sp_sim *s, int field, const void *host_src, size_t bytes, int is_f64, void *stream) {
    if (!s || !host_src) return fail(SP_EINVAL, "NULL argument");
    if (int rc = check_field(s, field)) return rc;
    const bool conv = is_f64 && s->dtype != SP_F64;
    const size_t want = s->N * (is_f64 ? sizeof(double) : s->esize);
    if (bytes != want) return fail(SP_EINVAL, "bytes = %zu, expected %zu", bytes, want);
    const cudaStream_t st = pick(s, stream);
    void *dst = s->f[s->cur][field];
    if (!conv) {
        SP_CUDA(cudaMemcpyAsync(dst, host_src, bytes, cudaMemcpyHostToDevice, st));
    } else {
        if (int rc = ensure_stage(s)) return rc;
        for (uint64_t off = 0; off < s->N; off += s->stage_elems) {
            const uint64_t n = (s->N - off) < s->stage_elems ? (s->N - off) : s->stage_elems;
            SP_CUDA(cudaMemcpyAsync(s->d_stage, (const double *)host_src + off, n * sizeof(double),
                                    cudaMemcpyHostToDevice, st));
            SP_CUDA(launch_convert_from_f64(s->dtype, s->d_stage, (char *)dst + off * s->esize, n, st));
        }
    }
    SP_CUDA(cudaStreamSynchronize(st));
    if (s->spec) s->spec_dirty = true;  // the resident spectrum no longer matches phi
    return SP_OK;
}

extern "C" int sp_reduce(sp_sim *s, int what, double *out, void *stream) {
    if (!s || !out) return fail(SP_EINVAL, "NULL argument");
    if (what < SP_MASS || what > SP_SUMSQ_U) return fail(SP_EINVAL, "unknown reduction %d", what);
    if (what == SP_SUM_V && s->nf < 2) return fail(SP_EINVAL, "SP_SUM_V needs a two-field model");
    // Model C: the conserved field is rho (field 1)
    const int field = (what == SP_SUM_V || (what == SP_MASS && s->model == SP_MODEL_C)) ? 1 : 0;
    ReduceGeom g;
    g.nx = s->nx;
    g.ny = s->ny;
    g.nz = s->nz;
    g.dims = s->dims;
    g.h = s->h;
    g.cell_volume = s->dims == 3 ? (s->h * s->h) * s->h : s->h * s->h;
    g.c1 = s->p.c1;
    g.c2 = s->p.c2;
    g.c3 = s->p.c3;
    // Model C free energy adds rho^2/2 - c3 phi^2 rho
    g.rho = (what == SP_FREE_ENERGY && s->model == SP_MODEL_C) ? s->f[s->cur][1] : nullptr;
    if (what == SP_FREE_ENERGY && s->model == SP_MODEL_H) {
        g.nq = s->nf - 1;
        for (int c = 0; c < g.nq; ++c) g.jq[c] = s->f[s->cur][1 + c];
    }
    const cudaStream_t st = pick(s, stream);
    double *d_out = s->d_partials + 2 * (size_t)s->nred;
    SP_CUDA(launch_reduce(s->dtype, what, s->f[s->cur][field], g, s->d_partials, s->nred, d_out, st));
    SP_CUDA(cudaMemcpyAsync(s->h_out, d_out, sizeof(double), cudaMemcpyDeviceToHost, st));
    SP_CUDA(cudaStreamSynchronize(st));
    *out = *s->h_out;
    return check_wait_flag(s);
}

extern "C" int sp_field_devptr(sp_sim *s, int field, void **dptr) {
    if (!s || !dptr) return fail(SP_EINVAL, "NULL argument");
    if (int rc = check_field(s, field)) return rc;
    *dptr = s->f[s->cur][field];
    return SP_OK;
}

extern "C" int sp_autotune(sp_sim *s, void *stream, int64_t *steps_taken) {
    if (!s || !steps_taken) return fail(SP_EINVAL, "NULL argument");
    *steps_taken = 0;
    const cudaStream_t st = pick(s, stream);
    int rc = SP_OK;
    s->tune_pending = false;
    if (s->steps == 0) {  // the first step takes the eager path
        if ((rc = sp_step(s, 1, stream)) != SP_OK) return rc;
        *steps_taken = 1;
    }
    *steps_taken += autotune(s, st, &rc);
    return rc;
}

extern "C" int sp_set_launch_config(sp_sim *s, int steps_per_launch, int variant) {
    if (!s) return fail(SP_EINVAL, "sim is NULL");
    for (const TuneChoice &c : tune_candidates(s))
        if (c.spl == steps_per_launch && c.variant == variant) {
            s->tune_pending = false;
            set_launch_config(s, c);
            return SP_OK;
        }
    // 2D FP64 finite differences: every strip shape and fused-step count runs on
    // any grid (the autotuner tries only the likely winners of the size class)
    const bool fd2d64 = s->dims == 2 && s->dtype == SP_F64 && !s->spec && s->model != SP_MODEL_H &&
                        s->stencil != SP_LAP_GENERATED;
    if (fd2d64 && ((steps_per_launch == 1 && (variant == 2 || variant == 4)) ||
                   ((steps_per_launch == 2 || steps_per_launch == 4) && variant == 0))) {
        s->tune_pending = false;
        set_launch_config(s, {steps_per_launch, variant});
        return SP_OK;
    }
    // generated stencils (2D) and Model H (2D and 3D), FP32 / BF16: the
    // per-point kernels instead of tiles
    if (steps_per_launch == 1 && variant == 1 &&
        ((s->stencil == SP_LAP_GENERATED && s->dims == 2) || s->model == SP_MODEL_H) && s->dtype != SP_F64 &&
        !s->spec) {
        s->tune_pending = false;
        set_launch_config(s, {1, 1});
        return SP_OK;
    }
    if (steps_per_launch == 1 && variant == 0) {  // the default is always available
        s->tune_pending = false;
        set_launch_config(s, {1, 0});
        return SP_OK;
    }
    if (steps_per_launch == 1 && variant == kUnfusedFamily && s->model == SP_CAHN_HILLIARD && !s->spec &&
        s->stencil != SP_LAP_GENERATED) {
        if (!s->mu_tmp) {
            const size_t bytes = s->N * (s->dtype == SP_F64 ? sizeof(double) : sizeof(float));
            const cudaError_t e = cudaMalloc(&s->mu_tmp, bytes);
            if (e != cudaSuccess) {
                s->mu_tmp = nullptr;
                return fail(SP_ENOMEM, "unfused ablation: cudaMalloc of %zu bytes failed: %s", bytes,
                            cudaGetErrorString(e));
            }
        }
        s->tune_pending = false;
        set_launch_config(s, {1, kUnfusedFamily});
        return SP_OK;
    }
    return fail(SP_EINVAL, "launch configuration (%d steps per launch, family %d) is not available for this grid",
                steps_per_launch, variant);
}

extern "C" int sp_launch_config(const sp_sim *s, int *steps_per_launch, int *variant) {
    if (!s || !steps_per_launch || !variant) return fail(SP_EINVAL, "NULL argument");
    *steps_per_launch = s->spl;
    *variant = s->variant;
    return SP_OK;
}

extern "C" int sp_steps_taken(const sp_sim *s, int64_t *steps) {
    if (!s || !steps) return fail(SP_EINVAL, "NULL argument");
    *steps = s->steps;
    return SP_OK;
}

extern "C" int sp_destroy(sp_sim *s) {
    if (!s) return SP_OK;
    release(s);
    return SP_OK;
}

// ---------------------------------------------------- conversion kernels --

namespace sp {

template <typename T>
__global__ void from_f64_kernel(const double *__restrict__ src, T *__restrict__ dst, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if constexpr (sizeof(T) == 4) dst[i] = __double2float_rn(src[i]);
        else dst[i] = __double2bfloat16(src[i]);
    }
}

template <typename T>
__global__ void to_f64_kernel(const T *__restrict__ src, double *__restrict__ dst, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = (double)to_c(src[i]);
}

static int conv_blocks(uint64_t n) {
    const uint64_t b = (n + 255) / 256;
    return (int)(b < 4096 ? (b ? b : 1) : 4096);
}

cudaError_t launch_convert_from_f64(int dtype, const double *src, void *dst, uint64_t n, cudaStream_t s) {
    if (dtype == SP_F32) from_f64_kernel<float><<<conv_blocks(n), 256, 0, s>>>(src, (float *)dst, n);
    else from_f64_kernel<bf16><<<conv_blocks(n), 256, 0, s>>>(src, (bf16 *)dst, n);
    return cudaGetLastError();
}

cudaError_t launch_convert_to_f64(int dtype, const void *src, double *dst, uint64_t n, cudaStream_t s) {
    if (dtype == SP_F32) to_f64_kernel<float><<<conv_blocks(n), 256, 0, s>>>((const float *)src, dst, n);
    else to_f64_kernel<bf16><<<conv_blocks(n), 256, 0, s>>>((const bf16 *)src, dst, n);
    return cudaGetLastError();
}

}  // namespace sp

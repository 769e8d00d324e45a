/*
 * sp.h -- C ABI of the GB300 (sm_103a) explicit finite-difference stepper for
 * phase-field and reaction-diffusion models on periodic regular grids.
 *
 * Method: SymPhas 2.0 (arXiv 2511.10508).  Each time step is one fused pass of
 *   - a finite-difference Laplacian (stencils from polynomial interpolation,
 *     Sec. "Compile-Time Stencil Generation"),
 *   - the pointwise reaction / chemical-potential term of the model
 *     (Model A, Eq. (model-a); Model B, Eq. (model-b); Gray-Scott, which the
 *     paper names in its Introduction, in Pearson's two-field form), and
 *   - the forward-Euler update,
 * on a periodic grid (Sec. "Benchmarks": periodic boundaries, seeded uniform
 * noise start).  Fields stay resident on the device; host transfers happen only
 * on explicit read/write (Sec. "CUDA Implementation").
 *
 * Conventions for every call:
 *  - Return value: SP_OK (0) or one of the sp_status codes; sp_last_error()
 *    gives a message for the calling thread's last failing call.
 *  - Grid shape: shape[0] = nx, shape[1] = ny, shape[2] = nz (nz = 1 in 2D).
 *    Fields are row-major with x fastest: index (z*ny + y)*nx + x.  One field
 *    (phi) for Allen-Cahn / Cahn-Hilliard, two (u = field 0, v = field 1) for
 *    Gray-Scott; structure of arrays.
 *  - Streams: `stream` is a cudaStream_t passed as void*.  NULL selects the
 *    simulation's own stream.  Device work is enqueued asynchronously on that
 *    stream, except where a call says it synchronises.
 *  - Ownership: the library owns every device buffer it allocates and frees it
 *    in sp_destroy / sp_server_destroy.  The caller owns every host buffer.
 *  - Thread safety: one handle must not be used from two threads at once;
 *    different handles are independent.
 */
#ifndef SP_H
#define SP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- enums -- */

typedef enum sp_status {
    SP_OK = 0,
    SP_EINVAL = 1,      /* bad argument: shape, model, stencil/dims mismatch, sizes */
    SP_EUNSTABLE = 2,   /* dt above the forward-Euler stability bound */
    SP_ENOMEM = 3,      /* device or host allocation failed */
    SP_EBUDGET = 4,     /* request larger than the server's HBM budget */
    SP_ECUDA = 5,       /* a CUDA runtime call failed (message in sp_last_error) */
    SP_ETIMEOUT = 6,    /* a bounded device-side wait expired */
    SP_EBUSY = 7,       /* resource busy (e.g. server queue full) */
    SP_PENDING = 8,     /* sp_poll: request not finished yet */
    SP_ENOTFOUND = 9,   /* unknown ticket */
    SP_ETOOLARGE = 10   /* request exceeds a fixed-size limit (see sp_reduce_field_noalloc) */
} sp_status;

typedef enum sp_model {
    SP_ALLEN_CAHN = 0,     /* Model A, Eq. (model-a): dphi/dt = lap phi + c1 phi - c2 phi^3 */
    SP_CAHN_HILLIARD = 1,  /* Model B, Eq. (model-b): dphi/dt = lap(c2 phi^3 - c1 phi - kappa lap phi) */
    SP_GRAY_SCOTT = 2,     /* du/dt = Du lap u - u v^2 + F(1-u); dv/dt = Dv lap v + u v^2 - (F+k) v */
    SP_MODEL_C = 3,        /* Model C (Sec. "Model C"), phi = field 0 (non-conserved), rho = field 1
                              (conserved), signs from the paper's free-energy listing
                              F = Landau(phi) + rho^2/2 - c3 phi^2 rho:
                              dphi/dt = lap phi + c1 phi - c2 phi^3 + 2 c3 phi rho;
                              drho/dt = lap(rho - c3 phi^2) */
    SP_MODEL_H = 4         /* Model H (Sec. "Model H", transverse projector at unity), field 0 = m
                              (conserved), fields 1..dims = the components of j; coupling signs
                              from the paper's listing: mu = -kappa lap m - c1 m + c2 m^3,
                              dm/dt = lap mu - c3 div(m j), dj/dt = lap j - c3 m grad mu, grad/div
                              by central differences of the stencil's order.  Two passes per step
                              (mu through a device buffer, as the paper's one temporary). */
} sp_model;

/* Laplacian stencils (integer weights over a denominator q; L f = sum w f / (q h^2)). */
typedef enum sp_stencil {
    SP_LAP_DEFAULT = -1,   /* 5-point in 2D, 7-point in 3D */
    SP_LAP_5 = 0,          /* 2D, q=1:  centre -4, faces 1 */
    SP_LAP_9BOX = 1,       /* 2D, q=6:  centre -20, faces 4, corners 1 (isotropic) */
    SP_LAP_9CROSS4 = 2,    /* 2D, q=12: centre -60, +-1: 16, +-2: -1 per axis (4th order) */
    SP_LAP_7 = 3,          /* 3D, q=1:  centre -6, faces 1 */
    SP_LAP_27 = 4,         /* 3D, q=30: centre -128, faces 14, edges 3, corners 1 (isotropic) */
    SP_LAP_13CROSS4 = 5,   /* 3D, q=12: centre -90, +-1: 16, +-2: -1 per axis (4th order) */
    SP_LAP_GENERATED = 6   /* 2D or 3D cross stencil of accuracy sp_params.stencil_order (2, 4, 6, 8),
                              weights generated at sp_create (see sp_stencil_weights); q = 1.
                              Allen-Cahn, Cahn-Hilliard, Gray-Scott and Model C; not served. */
} sp_stencil;

/* Storage / arithmetic precision of the fields. */
typedef enum sp_dtype {
    SP_F64 = 0,            /* FP64 storage and arithmetic (bitwise-reproducible order) */
    SP_F32 = 1,            /* FP32 storage and arithmetic */
    SP_BF16_F32 = 2        /* BF16 storage, FP32 arithmetic (convert on load/store) */
} sp_dtype;

typedef enum sp_ic_kind {
    SP_IC_NOISE = 0,       /* AC/CH: mean + amp*(2U-1); GS: u=1,v=0, patches, then noise */
    SP_IC_CONSTANT = 1     /* every field = ic_mean (GS: u = ic_mean, v = 0) */
} sp_ic_kind;

typedef enum sp_reduce_what {
    SP_MASS = 0,           /* h^d * sum of the conserved field (field 1, rho, for Model C;
                              field 0 otherwise), compensated FP64 */
    SP_FREE_ENERGY = 1,    /* h^d sum [1/2 |grad+ phi|^2 - c1/2 phi^2 + c2/4 phi^4] (field 0);
                              Model C adds + rho^2/2 - c3 phi^2 rho, Model H + |j|^2/2 */
    SP_SUM_U = 2,          /* sum of field 0 (no h^d) */
    SP_SUM_V = 3,          /* sum of field 1 (Gray-Scott, Model C) */
    SP_MIN_U = 4,          /* minimum of field 0 */
    SP_MAX_U = 5,          /* maximum of field 0 */
    SP_SUMSQ_U = 6         /* sum of squares of field 0 */
} sp_reduce_what;

/* ----------------------------------------------------------- parameters -- */

/* Time integration.  SP_SCHEME_FD: forward Euler with the finite-difference
 * stencil (every model).  SP_SCHEME_SPECTRAL: the paper's semi-implicit Fourier
 * spectral scheme (Sec. "Construction of Semi-Implicit Fourier Spectral Scheme"),
 * Allen-Cahn and Cahn-Hilliard, FP64 or FP32: linear terms implicit in Fourier
 * space with the continuous symbol -|k|^2 (k = 2 pi m / (n h) per axis), the
 * cubic term explicit; phi^' = (phi^ + dt N^) / (1 - dt L(k)) with
 *   Allen-Cahn     L = c1 - |k|^2,              N = -c2 phi^3
 *   Cahn-Hilliard  L = |k|^2 (c1 - kappa |k|^2), N^ = -|k|^2 (c2 phi^3)^.
 * The stencil is ignored; the step needs 1 - dt L(k) > 0 for all k (dt c1 < 1,
 * resp. kappa > 0 and dt c1^2 / (4 kappa) < 1; SP_EUNSTABLE otherwise).  That
 * keeps the step defined; with the cubic term explicit it is not unconditionally
 * stable (Cahn-Hilliard from +-0.5 noise, h = 1: bounded at dt = 0.5, four times
 * the forward-Euler limit of the 5-point stencil, divergent at dt = 1).  The
 * spectrum stays resident on the device: sp_write refreshes it, a write through
 * sp_field_devptr does not. */
typedef enum sp_scheme { SP_SCHEME_FD = 0, SP_SCHEME_SPECTRAL = 1 } sp_scheme;

typedef struct sp_params {
    double c1, c2, kappa;  /* Allen-Cahn / Cahn-Hilliard coefficients (defaults 1) */
    double Du, Dv, F, k;   /* Gray-Scott coefficients */
    double c3;             /* Model C coupling (default 0.5, the paper's value) */
    int stencil;           /* sp_stencil */
    int dtype;             /* sp_dtype */
    uint64_t seed;         /* initial-condition seed */
    int ic_kind;           /* sp_ic_kind */
    double ic_mean, ic_amp;/* noise mean and half-width */
    int gs_patches;        /* Gray-Scott: number of seeded patches */
    int gs_patch;          /* Gray-Scott: patch side (points) */
    int steps_per_launch;  /* time steps fused per kernel launch (temporal blocking:
                              2D grids 2 or 4; 3D FP32 / BF16 Allen-Cahn and
                              Gray-Scott with nx a multiple of 4: 2); 0 = the
                              library's choice, 1 = none */
    int scheme;            /* sp_scheme (default SP_SCHEME_FD) */
    int stencil_order;     /* accuracy order of SP_LAP_GENERATED (even, 2..8; default 2) */
    int flags;             /* SP_FLAG_* bits; other bits must be 0 */
} sp_params;

/* sp_params.flags: with steps_per_launch = 0, SP_FLAG_AUTOTUNE makes the first
 * sp_step call that asks for at least 66 steps autotune as sp_autotune does
 * (steps per launch and kernel family for 2D FP32/BF16; for 2D FP64 the strip
 * shapes or small tiles, and on grids up to 1024^2 steps fused per launch; the
 * kernel families of 3D FP32/BF16 and of the 3D FP64 27-point stencil),
 * counting the timed steps among the steps asked for. */
#define SP_FLAG_AUTOTUNE 1

/* sp_params.flags: SP_FLAG_BF16_NO_BOUND accepts SP_BF16_F32 storage, which
 * sp_create otherwise rejects (SP_EINVAL).  BF16 storage keeps 8 significant
 * bits per stored value: every per-step increment smaller than half a BF16 ulp
 * of the value is lost, and no benchmark configuration stays within a bound of
 * 1e-2 against the FP64 oracle.  Measured relative L2 against FP64 (GB300):
 *   Allen-Cahn 256^2, +-0.1 noise, dt 0.05:  9.8e-3 after 100 steps, 8.7e-2 after 1000
 *   Cahn-Hilliard 4096^2, +-0.01 noise, dt 0.01, 5-point: 0.78 after 1000 steps,
 *     1.0 after 10000 (the field stalls: increments ~1e-6 against an ulp ~4e-5)
 *   Cahn-Hilliard 128^3, +-0.01 noise, dt 0.005, 7-point: 0.84 after 2000 steps
 *   Gray-Scott 2048^2, dt 1: u 4.1e-2 and v 1.0 after 5000 steps
 *   Model C 512^2 and Model H 256^2 (+-0.1 noise): 0.4 to 1.3 after 1000 steps.
 * FP32 storage meets relative L2 <= 1e-5 on the Allen-Cahn and Cahn-Hilliard
 * configurations (measured 1.8e-7 to 4.1e-6) and <= 2e-4 on Gray-Scott after
 * 5000 steps (u 3.3e-6, v 1.0e-4).  The flag exists for throughput studies of
 * the BF16 kernels; results obtained with it carry no accuracy bound. */
#define SP_FLAG_BF16_NO_BOUND 2

/* Fill *p with the defaults: c1 = c2 = kappa = 1; Du = 0.16, Dv = 0.08, F = 0.035,
 * k = 0.065; default stencil of `dims`; FP64; seed 0; noise IC with mean 0 and
 * amp 0.01 (Gray-Scott: 64 patches of side 20); steps_per_launch 0. */
void sp_params_default(int model, int dims, sp_params *p);

/*
 * Forward-Euler stability check, host only (no device needed).  The growth
 * factor of the linearisation about |phi| = 1 (Gray-Scott: the diffusion part
 * plus the largest reaction rate) must satisfy dt * max|sigma| <= 2.
 * *factor (may be NULL) receives dt * max|sigma|.  Returns SP_OK when stable,
 * SP_EUNSTABLE when not, SP_EINVAL for bad arguments.
 */
int sp_check_stability(int model, int dims, double h, double dt, const sp_params *p, double *factor);

/* ------------------------------------------------------- one simulation -- */

typedef struct sp_sim sp_sim;

/*
 * Create a simulation on the current CUDA device: validates the arguments,
 * checks stability (SP_EUNSTABLE), allocates two device buffers per field (the
 * current and the next time level; 2 f words per point, Table 2 of the paper
 * with f0 = 0 because the chemical potential stays on chip) plus a small
 * reduction scratch, and writes the seeded initial condition on the device.
 * Three cases also hold a chemical-potential buffer of N compute-precision
 * values (the paper's one temporary): Model H, Cahn-Hilliard with a generated
 * stencil, and 3D FP64 Cahn-Hilliard with the 7-, 27- or 13-point stencil
 * (whose default kernels take two passes through it: on this part FP64 is
 * bound by the FP64 pipe, where re-evaluating mu on tile halos costs more than
 * the buffer's traffic).
 * Synchronises before returning.  *out receives the handle.
 */
int sp_create(int model, int dims, const int64_t shape[3], double h, double dt,
              const sp_params *p, sp_sim **out);

/* Advance nsteps forward-Euler steps; asynchronous on `stream`. */
int sp_step(sp_sim *sim, int64_t nsteps, void *stream);

/*
 * Copy field `field` (0 = phi/u, 1 = v) of the current time level to host
 * memory.  as_f64 != 0 converts to FP64 (exact widening for FP32/BF16);
 * otherwise the storage type is copied.  `bytes` must equal N * element size.
 * Synchronises `stream` before returning.  SP_ETIMEOUT (once, after copying) if
 * a bounded device wait of a step since the last check expired (the field is
 * then not a valid time level; see sp_set_wait_polls).
 */
int sp_read(sp_sim *sim, int field, void *host_dst, size_t bytes, int as_f64, void *stream);

/*
 * Overwrite field `field` of the current time level from host memory (FP64
 * when is_f64 != 0, rounded to nearest into the storage type; otherwise the
 * storage type).  Synchronises `stream` before returning.
 */
int sp_write(sp_sim *sim, int field, const void *host_src, size_t bytes, int is_f64, void *stream);

/* Reduce the current time level (sp_reduce_what) into *out (FP64).  Synchronises.
 * SP_ETIMEOUT as for sp_read. */
int sp_reduce(sp_sim *sim, int what, double *out, void *stream);

/*
 * Reduce a field that the caller owns, allocating nothing.  The paper has no
 * counterpart; this exists for callers that cannot allocate device memory when
 * they need a diagnostic: an application whose memory pool already holds
 * nearly all of HBM, a latency-critical loop in which cudaMalloc/cudaFree
 * would stall or synchronise the device, or code that keeps its fields in its
 * own allocator.  Same reductions as sp_reduce (except SP_SUM_V: pass the v
 * field with SP_SUM_U), same kernels and, on the same device, the same result.
 *   what:   SP_MASS, SP_FREE_ENERGY, SP_SUM_U, SP_MIN_U, SP_MAX_U or SP_SUMSQ_U
 *   dtype:  storage type of `field` (sp_dtype)
 *   field:  device pointer, nx*ny*nz elements, x fastest; only read
 *   dims, shape, h: grid as in sp_create; c1, c2 enter SP_FREE_ENERGY only
 *   out:    host pointer receiving the FP64 result
 *   stream: cudaStream_t (NULL = the legacy default stream); the call
 *           synchronises it before returning.
 * Block partials live in a fixed device array of the library (room for 512
 * partials, 8 KiB, held on every GPU that loads the library until exit); a
 * grid needing more partials than that fails with SP_ETOOLARGE.  The array is
 * shared by all calls and keeps the last call's contents; calls that overlap
 * on the GPU race on it.  The first call in a CUDA context looks up the
 * array's device address (again after cudaDeviceReset re-creates the
 * context): make it before any stream capture.  The call cannot be used on a
 * stream that is being captured (SP_EINVAL: it copies the result to the host
 * and synchronises).  SP_EINVAL also for a field not aligned to its element
 * size and for grids beyond sp_create's limits.  No cudaMalloc, cudaFree or
 * allocating routine is called; on failure only the status code is returned
 * and sp_last_error() is not updated.
 */
int sp_reduce_field_noalloc(int what, int dtype, const void *field, int dims, const int64_t shape[3], double h,
                            double c1, double c2, double *out, void *stream);

/* Device pointer of field `field` at the current time level (storage type).
 * Valid until the next sp_step / sp_destroy. */
int sp_field_devptr(sp_sim *sim, int field, void **dptr);

/* Autotune now (no counterpart in the paper, whose kernels have fixed shapes):
 * time each candidate launch configuration for this grid on `stream` (8 steps
 * each, twice; all candidates give bit-identical results, so these are ordinary
 * steps of the run) and keep the fastest.  A choice cached earlier in the
 * process for the same (model, stencil, dtype, dims, grid size class) is taken
 * without timing.  Blocks until the timing events complete.  *steps_taken
 * receives the number of time steps advanced (0 to 65).  Captured graphs of
 * another configuration are dropped. */
int sp_autotune(sp_sim *sim, void *stream, int64_t *steps_taken);

/* Pin a launch configuration (for instance one that sp_autotune chose in an
 * earlier run): steps fused per launch (1, or 2 / 4 for 2D grids) and kernel
 * family (0, or 1 / 2 / 4 where sp_launch_config documents an alternative).  Family 3
 * (Cahn-Hilliard only, one step per launch) is an ablation with no use in
 * production: the unfused two-pass step of the paper's solver, which writes mu to
 * a temporary field in device memory (allocated here, N values of the compute
 * precision; SP_ENOMEM if that fails) and reads it back for the outer Laplacian.
 * Every available configuration gives bit-identical results.  SP_EINVAL if the
 * pair is not available for this grid; cancels a pending SP_FLAG_AUTOTUNE. */
int sp_set_launch_config(sp_sim *sim, int steps_per_launch, int variant);

/* Weights of the generated cross Laplacian (SP_LAP_GENERATED; the paper
 * generates stencils by solving a polynomial-interpolation system, Sec.
 * "Compile-Time Stencil Generation").  The symmetric weights w_0..w_r (r =
 * order/2) of the central second derivative exact on polynomials of degree
 * <= order+1 are found in exact rational arithmetic and rounded once to FP64.
 * Host only.  w receives order/2 + 1 values (dims * w_0, w_1, ..., w_r), the
 * kernels' weights: L_h f = (1/h^2) [dims w_0 f_0 + sum_j w_j P_j], P_j the sum
 * over axes of f(+j e_a) + f(-j e_a); *lambda_max (if not NULL) the largest
 * eigenvalue of -h^2 L_h.  SP_EINVAL for an odd order or one outside 2..8, or
 * dims not 2 or 3. */
int sp_stencil_weights(int order, int dims, double *w, double *lambda_max);

/* Measurement aid (no counterpart in the paper): the sustained FP64 fused
 * multiply-add rate of the current device in Gop/s (one operation per FMA),
 * from a kernel of independent FMA chains on every SM timed with CUDA events on
 * `stream` (about 10 ms; the first launch warms up).  FP64 step kernels are
 * bound by this rate.  Blocks until done; allocates 8 bytes of device memory.
 * SP_EINVAL if gops is NULL, SP_ENOMEM / SP_ECUDA on failure. */
int sp_probe_fp64_rate(void *stream, double *gops);

/* Build check (no counterpart in the paper): the compute capability the
 * library's device code was compiled for, as major*10 + minor of the binary the
 * runtime loaded for the current device (103 for sm_103a, GB300).  Needs a
 * device; SP_EINVAL if version is NULL, SP_ECUDA when no binary in the library
 * runs on the current device. */
int sp_binary_version(int *version);

/* Test hook (no counterpart in the paper): the number of polls after which the
 * kernels' bounded device waits (the mbarrier waits of the tensor-map plane
 * ring, kernel family 6) give up; 0 restores the default (about 4 million polls,
 * far beyond any transfer) and a negative value makes every wait give up at
 * once (the copies in flight still land before the kernel returns).  A wait
 * that gives up leaves the step's output
 * invalid, and the next sp_read or sp_reduce of that simulation returns
 * SP_ETIMEOUT.  Process-wide; launches captured in CUDA graphs keep the value
 * they were captured with.  Always returns SP_OK. */
int sp_set_wait_polls(long long polls);

/* Launch configuration in use: steps fused per launch and kernel family
 * (0 = the default for the grid; alternatives the autotuner may pick: 1 for
 * every grid of the finite-difference scheme except 3D FP64 with the 7- and
 * 13-point stencils; 2 for 3D FP32/BF16, for 3D FP64 27-point Allen-Cahn,
 * Cahn-Hilliard and Gray-Scott (plane sums in registers instead of x-pair sums
 * shared between rows) and for 3D FP64 7- and 13-point Cahn-Hilliard (one fused
 * pass instead of two through the mu buffer); 2 and 4 for 2D FP64, the strip
 * kernel with 64 threads per CTA and with half the rows per batch; 6 for 3D
 * FP32/BF16 Allen-Cahn, Cahn-Hilliard and Gray-Scott with nx a multiple of 4
 * (FP32) or 8 (BF16): the plane ring with tensor-map (TMA) plane loads). */
int sp_launch_config(const sp_sim *sim, int *steps_per_launch, int *variant);

/* Number of time steps taken since creation. */
int sp_steps_taken(const sp_sim *sim, int64_t *steps);

/* Release all device memory of the simulation (synchronises its stream). */
int sp_destroy(sp_sim *sim);

/* --------------------------------------------------------------- serving -- */

/*
 * Continuous-batching server (the paper has no serving layer; it benchmarks
 * one grid at a time, Sec. "Benchmarks").  Requests of any model, dimension,
 * size and precision (FP64 or FP32 storage) arrive at any time; a scheduler
 * thread admits them by priority, in arrival order within a priority, whenever
 * a slot and enough of the HBM budget are free (a request that does not fit yet
 * lets later ones that fit pass; sp_admission_order states the rule),
 * keeps their fields resident, and advances all resident grids together in
 * quanta of `quantum_steps` time steps: one batched launch per (dims, dtype)
 * per step covers the tiles of every resident grid, and the quantum's launches
 * are replayed from a CUDA graph while the resident set is unchanged.  A
 * finished grid's FP64 mass (and optionally its fields, as FP64) are copied to
 * host memory and its device memory is freed.  A grid's result does not depend
 * on the other grids in the mix.
 */
typedef struct sp_server sp_server;

typedef struct sp_request {
    int model, dims;        /* as sp_create */
    int64_t shape[3];       /* nx, ny, nz (nz = 1 in 2D) */
    double h, dt;
    sp_params params;       /* dtype must be SP_F64 or SP_F32 */
    int64_t nsteps;         /* time steps to run (>= 1) */
    int return_fields;      /* nonzero: keep an FP64 host copy of the final fields */
    int fault;              /* fault injection for tests: 0 none, 1 the allocation fails */
    int priority;           /* admission priority: higher first (see sp_admission_order) */
} sp_request;

typedef struct sp_result {
    int status;             /* SP_PENDING, SP_OK or the error of this request */
    int64_t steps_done;
    double t_submit, t_admit, t_finish;  /* seconds since server creation; -1 if not reached */
    double mass;            /* SP_MASS of the grid at the end (FP64, compensated) */
    const double *fields;   /* FP64 fields (field 0, then field 1), or NULL; owned by the
                               server, valid until sp_release(ticket) */
    size_t n_values;        /* number of doubles at `fields` */
} sp_result;

typedef struct sp_server_stats {
    uint64_t submitted, admitted, finished, failed, quanta;
    int64_t resident, pending;
    size_t hbm_in_use;      /* bytes of field buffers of admitted requests */
    double lups;            /* lattice-site updates done (points x steps) */
    double busy_s;          /* seconds the scheduler spent running quanta */
} sp_server_stats;

/* The server's admission rule as a pure host function (no device work; the
 * scheduler calls the same code): n pending requests in arrival order, with
 * their field bytes and priorities, `free_bytes` of the budget and `free_slots`
 * slots free.  Requests are taken by priority (higher first), in arrival order
 * within a priority; each one that fits the remaining bytes and slots is
 * admitted, one that does not lets later ones pass.  The indices of the
 * admitted requests, in admission order, go to order[] (room for n); returns
 * their number, or -1 if an array is NULL while n > 0. */
int sp_admission_order(int n, const size_t bytes[], const int priority[], size_t free_bytes, int free_slots,
                       int order[]);

/* Create a server on the current device with an HBM budget for field buffers,
 * at most max_slots resident grids, and quanta of quantum_steps steps. */
int sp_server_create(size_t hbm_budget_bytes, int max_slots, int quantum_steps, sp_server **out);

/* Queue a request; *ticket identifies it.  SP_EBUDGET if it can never fit,
 * SP_EUNSTABLE / SP_EINVAL as sp_create; served requests use FP64 or FP32 storage
 * and the finite-difference scheme (SP_EINVAL otherwise).  Never blocks on the
 * device. */
int sp_submit(sp_server *srv, const sp_request *req, uint64_t *ticket);

/* Non-blocking status: SP_PENDING until the request is done, then its status;
 * *out is filled in either case.  SP_ENOTFOUND for an unknown ticket. */
int sp_poll(sp_server *srv, uint64_t ticket, sp_result *out);

/* Block until the request is done or timeout_s seconds pass (SP_ETIMEOUT). */
int sp_wait(sp_server *srv, uint64_t ticket, double timeout_s, sp_result *out);

/* Free a finished request's host result (SP_EBUSY while it is pending). */
int sp_release(sp_server *srv, uint64_t ticket);

int sp_server_get_stats(sp_server *srv, sp_server_stats *out);

/* Stop the scheduler, free every device and host buffer of the server. */
int sp_server_destroy(sp_server *srv);

/* Message of the calling thread's last failing call ("" if none). */
const char *sp_last_error(void);

/* Library version, e.g. 100 for 0.1.0. */
int sp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SP_H */

// sp_common.cuh -- device-side building blocks shared by the step, initial-
// condition and reduction kernels: stencil tables, the per-model arithmetic in
// a fixed evaluation order, storage/compute type traits and vector loads.
//
// Method: SymPhas 2.0 (arXiv 2511.10508), Model A Eq. (model-a), Model B
// Eq. (model-b), periodic finite-difference stencils (Sec. "Compile-Time
// Stencil Generation"); Gray-Scott in Pearson's two-field form.
//
// Fixed evaluation order.  The whole library is compiled with --fmad=false, so
// a*b+c is never contracted; every fused multiply-add below is explicit.  The
// FP64 kernels evaluate exactly these expressions, so FP64 results are
// reproducible bit for bit by any implementation that follows the same order:
//   stencil sum S (integer weights w over denominator q):
//     S1  C = (f[-1,0]+f[1,0]) + (f[0,-1]+f[0,1]);           S = fma(-4, f0, C)
//     S2  D = (f[-1,-1]+f[1,-1]) + (f[-1,1]+f[1,1]);          S = fma(-20, f0, fma(4, C, D))
//     S3  F2 = (f[-2,0]+f[2,0]) + (f[0,-2]+f[0,2]);           S = fma(-60, f0, fma(16, C, -F2))
//     S4  F = C0 + (f[0,0,-1]+f[0,0,1]);                       S = fma(-6, f0, F)
//     S5  Cz, Dz = in-plane cross / diagonal sums of plane z;
//         F = C0 + (f[0,0,-1]+f[0,0,1]); E = D0 + (C- + C+); K = D- + D+
//                                                              S = fma(-128, f0, fma(14, F, fma(3, E, K)))
//     S6  F1 = F of S4; F2 = ((f[-2,0,0]+f[2,0,0]) + (f[0,-2,0]+f[0,2,0])) + (f[0,0,-2]+f[0,0,2])
//                                                              S = fma(-90, f0, fma(16, F1, -F2))
//   with q_h2 = (q*h)*h (host):
//     Allen-Cahn:    p' = fma(dt, fma(p, fma(-c2, p*p, c1), (1/q_h2)*S(p)), p)
//     Cahn-Hilliard: mu = fma(p, fma(c2, p*p, -c1), -((kappa/q_h2)*S(p)));  p' = fma(dt/q_h2, S(mu), p)
//     Gray-Scott:    uvv = (u*v)*v
//                    u' = fma(dt, fma(F, 1-u, fma(Du/q_h2, S(u), -uvv)), u)
//                    v' = fma(dt, fma(-(F+k), v, fma(Dv/q_h2, S(v), uvv)), v)
//     Model C:       m = fma(-c3, u*u, v) at every tap; g = fma(-c2, u*u, fma(2 c3, v, c1))
//                    u' = fma(dt, fma(u, g, (1/q_h2)*S(u)), u);  v' = fma(dt/q_h2, S(m), v)
#pragma once

#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace sp {

enum Model : int { AC = 0, CH = 1, GS = 2, MC = 3, MH = 4 };
enum Stencil : int { L5 = 0, L9BOX = 1, L9X4 = 2, L7 = 3, L27 = 4, L13X4 = 5 };

template <int ST> struct StencilInfo;
template <> struct StencilInfo<L5>    { static constexpr int dims = 2, r = 1, q = 1; };
template <> struct StencilInfo<L9BOX> { static constexpr int dims = 2, r = 1, q = 6; };
template <> struct StencilInfo<L9X4>  { static constexpr int dims = 2, r = 2, q = 12; };
template <> struct StencilInfo<L7>    { static constexpr int dims = 3, r = 1, q = 1; };
template <> struct StencilInfo<L27>   { static constexpr int dims = 3, r = 1, q = 30; };
template <> struct StencilInfo<L13X4> { static constexpr int dims = 3, r = 2, q = 12; };

// ------------------------------------------------------------ precision --

typedef __nv_bfloat16 bf16;

template <typename T> struct Cmp { typedef T type; };
template <> struct Cmp<bf16> { typedef float type; };

__device__ __forceinline__ double to_c(double x) { return x; }
__device__ __forceinline__ float to_c(float x) { return x; }
__device__ __forceinline__ float to_c(bf16 x) { return __bfloat162float(x); }

template <typename T> __device__ __forceinline__ T from_c(typename Cmp<T>::type x);
template <> __device__ __forceinline__ double from_c<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_c<float>(float x) { return x; }
template <> __device__ __forceinline__ bf16 from_c<bf16>(float x) { return __float2bfloat16_rn(x); }

__device__ __forceinline__ double FMA(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float FMA(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// ------------------------------------------------------- vector access --

template <int BYTES> struct VecT;
template <> struct VecT<2> { typedef unsigned short type; };
template <> struct VecT<4> { typedef unsigned int type; };
template <> struct VecT<8> { typedef uint2 type; };
template <> struct VecT<16> { typedef uint4 type; };

// Load V consecutive elements (16- or 8-byte aligned) and widen to C.
template <typename T, int V>
__device__ __forceinline__ void load_vec(const T *__restrict__ p, typename Cmp<T>::type (&out)[V]) {
    typedef typename VecT<V * sizeof(T)>::type W;
    union { W w; T t[V]; } u;
    u.w = __ldg(reinterpret_cast<const W *>(p));
#pragma unroll
    for (int i = 0; i < V; ++i) out[i] = to_c(u.t[i]);
}

template <typename T, int V>
__device__ __forceinline__ void store_vec(T *__restrict__ p, const typename Cmp<T>::type (&in)[V]) {
    typedef typename VecT<V * sizeof(T)>::type W;
    union { W w; T t[V]; } u;
#pragma unroll
    for (int i = 0; i < V; ++i) u.t[i] = from_c<T>(in[i]);
    *reinterpret_cast<W *>(p) = u.w;
}

template <typename T>
__device__ __forceinline__ typename Cmp<T>::type load_one(const T *__restrict__ p) { return to_c(__ldg(p)); }

// Asynchronous 16-byte global -> shared copy (both addresses 16-byte aligned),
// committed as one group per call site; completion is awaited by the issuing
// thread with cp_async_wait<N> (at most N groups still pending).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// 8-byte variant (both addresses 8-byte aligned; cached in L1 and L2).
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Periodic wrap of an index that may lie anywhere (small grids: several periods).
__device__ __forceinline__ int wrap_slow(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}
__device__ __forceinline__ int wrap_idx(int i, int n) {
    return ((unsigned)i < (unsigned)n) ? i : wrap_slow(i, n);
}

// ------------------------------------------------------------ stencils --

// Unscaled weighted neighbour sum S in the fixed order.  P(dx, dy, dz) returns
// the neighbour value at that offset (2D stencils use dz = 0 only).
template <int ST, typename C, typename Acc>
__device__ __forceinline__ C stencil_sum(const Acc &P) {
    if constexpr (ST == L5) {
        const C Cs = (P(-1, 0, 0) + P(1, 0, 0)) + (P(0, -1, 0) + P(0, 1, 0));
        return FMA(C(-4), P(0, 0, 0), Cs);
    } else if constexpr (ST == L9BOX) {
        const C Cs = (P(-1, 0, 0) + P(1, 0, 0)) + (P(0, -1, 0) + P(0, 1, 0));
        const C D = (P(-1, -1, 0) + P(1, -1, 0)) + (P(-1, 1, 0) + P(1, 1, 0));
        return FMA(C(-20), P(0, 0, 0), FMA(C(4), Cs, D));
    } else if constexpr (ST == L9X4) {
        const C F1 = (P(-1, 0, 0) + P(1, 0, 0)) + (P(0, -1, 0) + P(0, 1, 0));
        const C F2 = (P(-2, 0, 0) + P(2, 0, 0)) + (P(0, -2, 0) + P(0, 2, 0));
        return FMA(C(-60), P(0, 0, 0), FMA(C(16), F1, -F2));
    } else if constexpr (ST == L7) {
        const C F = ((P(-1, 0, 0) + P(1, 0, 0)) + (P(0, -1, 0) + P(0, 1, 0))) + (P(0, 0, -1) + P(0, 0, 1));
        return FMA(C(-6), P(0, 0, 0), F);
    } else if constexpr (ST == L27) {
        const C Cm = (P(-1, 0, -1) + P(1, 0, -1)) + (P(0, -1, -1) + P(0, 1, -1));
        const C C0 = (P(-1, 0, 0) + P(1, 0, 0)) + (P(0, -1, 0) + P(0, 1, 0));
        const C Cp = (P(-1, 0, 1) + P(1, 0, 1)) + (P(0, -1, 1) + P(0, 1, 1));
        const C Dm = (P(-1, -1, -1) + P(1, -1, -1)) + (P(-1, 1, -1) + P(1, 1, -1));
        const C D0 = (P(-1, -1, 0) + P(1, -1, 0)) + (P(-1, 1, 0) + P(1, 1, 0));
        const C Dp = (P(-1, -1, 1) + P(1, -1, 1)) + (P(-1, 1, 1) + P(1, 1, 1));
        const C F = C0 + (P(0, 0, -1) + P(0, 0, 1));
        const C E = D0 + (Cm + Cp);
        const C K = Dm + Dp;
        return FMA(C(-128), P(0, 0, 0), FMA(C(14), F, FMA(C(3), E, K)));
    } else {  // L13X4
        const C F1 = ((P(-1, 0, 0) + P(1, 0, 0)) + (P(0, -1, 0) + P(0, 1, 0))) + (P(0, 0, -1) + P(0, 0, 1));
        const C F2 = ((P(-2, 0, 0) + P(2, 0, 0)) + (P(0, -2, 0) + P(0, 2, 0))) + (P(0, 0, -2) + P(0, 0, 2));
        return FMA(C(-90), P(0, 0, 0), FMA(C(16), F1, -F2));
    }
}

// ------------------------------------------------------ model constants --

// Host-computed coefficients (see the header comment); narrowed to C on use.
struct StepConsts {
    double c1, c2;   // reaction coefficients
    double sAC;      // 1 / q_h2                (Allen-Cahn Laplacian scale)
    double kq;       // kappa / q_h2            (Cahn-Hilliard inner)
    double dq;       // dt / q_h2               (Cahn-Hilliard outer, folded with dt)
    double duq, dvq; // Du / q_h2, Dv / q_h2    (Gray-Scott)
    double F, Fk;    // F, F + k
    double dt;
    double c3, c3x2; // Model C coupling c3 and 2 c3
};

// The same coefficients rounded once to FP32 on the host, so that FP32/BF16
// kernels contain no FP64 instruction (a double->float conversion runs on the
// FP64 pipe, which the compiler may re-run inside loops).
struct StepConstsF {
    float c1, c2, sAC, kq, dq, duq, dvq, F, Fk, dt, c3, c3x2;
};

// FP32 copies, each rounded once from the FP64 value.
inline StepConstsF to_float(const StepConsts &k) {
    return {(float)k.c1, (float)k.c2, (float)k.sAC, (float)k.kq, (float)k.dq, (float)k.duq,
            (float)k.dvq, (float)k.F,  (float)k.Fk, (float)k.dt, (float)k.c3, (float)k.c3x2};
}

template <typename C> struct ConstsC;
template <> struct ConstsC<double> {
    double c1, c2, sAC, kq, dq, duq, dvq, F, Fk, dt, c3, c3x2;
    __device__ __forceinline__ ConstsC(const StepConsts &k, const StepConstsF &)
        : c1(k.c1), c2(k.c2), sAC(k.sAC), kq(k.kq), dq(k.dq), duq(k.duq), dvq(k.dvq), F(k.F), Fk(k.Fk), dt(k.dt),
          c3(k.c3), c3x2(k.c3x2) {}
};
template <> struct ConstsC<float> {
    float c1, c2, sAC, kq, dq, duq, dvq, F, Fk, dt, c3, c3x2;
    __device__ __forceinline__ ConstsC(const StepConsts &, const StepConstsF &k)
        : c1(k.c1), c2(k.c2), sAC(k.sAC), kq(k.kq), dq(k.dq), duq(k.duq), dvq(k.dvq), F(k.F), Fk(k.Fk), dt(k.dt),
          c3(k.c3), c3x2(k.c3x2) {}
};

// Allen-Cahn update of one point from its value and stencil sum.
template <typename C>
__device__ __forceinline__ C ac_update(C p, C S, const ConstsC<C> &k) {
    const C rhs = FMA(p, FMA(-k.c2, p * p, k.c1), k.sAC * S);
    return FMA(k.dt, rhs, p);
}

// Cahn-Hilliard chemical potential of one point.
template <typename C>
__device__ __forceinline__ C ch_mu(C p, C S, const ConstsC<C> &k) {
    return FMA(p, FMA(k.c2, p * p, -k.c1), -(k.kq * S));
}

// Cahn-Hilliard update from the stencil sum of mu.
template <typename C>
__device__ __forceinline__ C ch_update(C p, C Smu, const ConstsC<C> &k) {
    return FMA(k.dq, Smu, p);
}

// Gray-Scott update of (u, v) from values and stencil sums.
template <typename C>
__device__ __forceinline__ void gs_update(C u, C v, C Su, C Sv, const ConstsC<C> &k, C &un, C &vn) {
    const C uvv = (u * v) * v;
    const C ru = FMA(k.F, C(1) - u, FMA(k.duq, Su, -uvv));
    const C rv = FMA(-k.Fk, v, FMA(k.dvq, Sv, uvv));
    un = FMA(k.dt, ru, u);
    vn = FMA(k.dt, rv, v);
}

// Model C: chemical potential of the conserved density at one point, from its
// phi and rho (evaluated at every stencil tap, so it never needs a buffer).
template <typename C>
__device__ __forceinline__ C mc_mu(C p, C r, const ConstsC<C> &k) {
    return FMA(-k.c3, p * p, r);
}

// Model C update of (phi, rho) from the values, the stencil sum of phi and the
// stencil sum of the density's chemical potential.
template <typename C>
__device__ __forceinline__ void mc_update(C p, C r, C Sp, C Sm, const ConstsC<C> &k, C &pn, C &rn) {
    const C g = FMA(-k.c2, p * p, FMA(k.c3x2, r, k.c1));
    pn = FMA(k.dt, FMA(p, g, k.sAC * Sp), p);
    rn = FMA(k.dq, Sm, r);
}

// Fields per model (Gray-Scott u, v; Model C phi, rho).
template <int MODEL> __host__ __device__ constexpr int num_fields() { return (MODEL == GS || MODEL == MC) ? 2 : 1; }

// Second stencil sum of a two-field model from the accessors of field 0 and
// field 1 at the taps: of field 1 itself (Gray-Scott), or of Model C's density
// chemical potential mc_mu evaluated at every tap.
template <int MODEL, int ST, typename C, typename A0, typename A1>
__device__ __forceinline__ C second_sum(const A0 &P0, const A1 &P1, const ConstsC<C> &k) {
    if constexpr (MODEL == MC) {
        auto Pm = [&](int dx, int dy, int dz) -> C { return mc_mu<C>(P0(dx, dy, dz), P1(dx, dy, dz), k); };
        return stencil_sum<ST, C>(Pm);
    } else {
        return stencil_sum<ST, C>(P1);
    }
}

// Update of a two-field model from centre values and the two stencil sums.
template <int MODEL, typename C>
__device__ __forceinline__ void two_field_update(C p0, C p1, C S0, C S1, const ConstsC<C> &k, C &o0, C &o1) {
    if constexpr (MODEL == MC) mc_update<C>(p0, p1, S0, S1, k, o0, o1);
    else gs_update<C>(p0, p1, S0, S1, k, o0, o1);
}

// --------------------------------------- programmatic dependent launch --
//
// A step kernel launched with programmatic stream serialisation may be launched
// as soon as every CTA of the previous kernel in the stream has exited, before
// that grid has completed and flushed; it waits, before its first global-memory
// access, until its predecessor has completed and its writes are visible
// (griddepcontrol.wait, sm_90 and later).  Without that launch attribute the
// wait is a no-op, so every launch path may use these kernels.  (Triggering the
// dependents at the start of the kernel instead measured slower on GB300: the
// waiting CTAs of the next grid took issue slots and SM space.)
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ------------------------------------------------- packed FP32 pairs --
//
// Two cells per instruction (f32x2 arithmetic of sm_100 and later): each lane
// of __fadd2_rn / __fmul2_rn / __ffma2_rn rounds like the scalar operation, so
// the pair forms below give the scalar helpers' results bit for bit (a negated
// operand is exact, so -(a*b) == (-a)*b and x - y == x + (-y)).  Unlike the
// scalar __fmul_rn / __fadd_rn, a packed product that feeds a packed sum or
// difference may be contracted into one fused multiply-add by the code
// generator (measured on sm_103a, with --fmad=false, both for these
// intrinsics and for the PTX add/sub/mul.rn.f32x2 forms: m1*j1 - m2*j2 on
// pairs differed from the scalar result in the last bit).  So no pair product
// here ever feeds a pair addition or subtraction: products enter only as
// multiplicands or as the addend of an explicit fma2, where nothing can be
// contracted.
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

struct ConstsF2 {
    float2 c1, negc1, c2, negc2, sAC, negkq, dq, duq, dvq, F, negFk, dt, one;
    __device__ __forceinline__ explicit ConstsF2(const ConstsC<float> &k)
        : c1(splat2(k.c1)), negc1(splat2(-k.c1)), c2(splat2(k.c2)), negc2(splat2(-k.c2)), sAC(splat2(k.sAC)),
          negkq(splat2(-k.kq)), dq(splat2(k.dq)), duq(splat2(k.duq)), dvq(splat2(k.dvq)), F(splat2(k.F)),
          negFk(splat2(-k.Fk)), dt(splat2(k.dt)), one(splat2(1.f)) {}
};

// ac_update, ch_mu, ch_update and gs_update on pairs of cells
__device__ __forceinline__ float2 ac_update2(float2 p, float2 S, const ConstsF2 &k) {
    const float2 rhs = fma2(p, fma2(k.negc2, mul2(p, p), k.c1), mul2(k.sAC, S));
    return fma2(k.dt, rhs, p);
}
__device__ __forceinline__ float2 ch_mu2(float2 p, float2 S, const ConstsF2 &k) {
    return fma2(p, fma2(k.c2, mul2(p, p), k.negc1), mul2(k.negkq, S));
}
__device__ __forceinline__ float2 ch_update2(float2 p, float2 Smu, const ConstsF2 &k) { return fma2(k.dq, Smu, p); }
__device__ __forceinline__ void gs_update2(float2 u, float2 v, float2 Su, float2 Sv, const ConstsF2 &k, float2 &un,
                                           float2 &vn) {
    const float2 uvv = mul2(mul2(u, v), v);
    const float2 ru = fma2(k.F, add2(k.one, neg2(u)), fma2(k.duq, Su, neg2(uvv)));
    const float2 rv = fma2(k.negFk, v, fma2(k.dvq, Sv, uvv));
    un = fma2(k.dt, ru, u);
    vn = fma2(k.dt, rv, v);
}

// S of the 2D stencils for the pair of cells (c0, c0 + 1), the fixed order of
// stencil_sum: the x-direction pair sums are formed per cell (the shifted
// neighbours are not register pairs), everything else two cells per
// instruction.  P(dx, dy, c) is the value at offset (dx, dy) of cell c.
template <int ST, typename Acc>
__device__ __forceinline__ float2 stencil_sum2_2d(const Acc &P, int c0) {
    const int c1 = c0 + 1;
    auto pr = [&](int dx, int dy) { return make_float2(P(dx, dy, c0), P(dx, dy, c1)); };
    auto xs = [&](int d, int dy) {
        return make_float2(P(-d, dy, c0) + P(d, dy, c0), P(-d, dy, c1) + P(d, dy, c1));
    };
    if constexpr (ST == L5) {
        return fma2(splat2(-4.f), pr(0, 0), add2(xs(1, 0), add2(pr(0, -1), pr(0, 1))));
    } else if constexpr (ST == L9BOX) {
        const float2 Cs = add2(xs(1, 0), add2(pr(0, -1), pr(0, 1)));
        const float2 D = add2(xs(1, -1), xs(1, 1));
        return fma2(splat2(-20.f), pr(0, 0), fma2(splat2(4.f), Cs, D));
    } else {  // L9X4
        const float2 F1 = add2(xs(1, 0), add2(pr(0, -1), pr(0, 1)));
        const float2 F2 = add2(xs(2, 0), add2(pr(0, -2), pr(0, 2)));
        return fma2(splat2(-60.f), pr(0, 0), fma2(splat2(16.f), F1, neg2(F2)));
    }
}

// ------------------------------------------------------- launch records --

struct StepArgs {
    const void *in0, *in1;   // current level (field 0, field 1)
    void *out0, *out1;       // next level
    int nx, ny, nz;
    StepConsts k;            // FP64 coefficients
    StepConstsF kf;          // the same, rounded to FP32
    int *flag = nullptr;     // set to 1 by a kernel whose bounded wait expired (else untouched)
    long long wait_polls = 0;  // polls before a wait gives up (0: the default; < 0: none, a test hook)
};

// ------------------------------------------------------- tensor-map loads --
//
// Tiles moved by the Tensor Memory Accelerator (cp.async.bulk.tensor) into
// shared memory, completion tracked by an mbarrier with a transaction count.
// The tensor maps describe this GPU's own fields only; no multicast.

struct TmaMaps {
    CUtensorMap m[2];  // field 0, field 1
};

// default bound on mbarrier polls (each may sleep up to about 1 us): a few
// seconds, far beyond any transfer
constexpr long long kDefaultWaitPolls = 1LL << 22;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make barrier initialisation visible to the async proxy (TMA)
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's earlier shared-memory accesses before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// one poll: the thread may sleep up to about 1 us unless the phase completes first
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0;
}
// wait for the phase of the given parity to complete, at most `polls` polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, long long polls) {
    for (long long i = 0; i < polls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// box of a rank-3 tensor map at (x, y, z) (x a multiple of 16 bytes) into dst,
// completing `bar`'s transaction count
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace sp

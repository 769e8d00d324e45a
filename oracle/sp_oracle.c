/*
 * sp_oracle.c -- plain FP64 CPU oracle for the explicit finite-difference time
 * step of phase-field and reaction-diffusion models on periodic regular grids
 * (SymPhas 2.0, arXiv 2511.10508: Model A Eq. (model-a), Model B Eq. (model-b),
 * the periodic benchmark protocol of Sec. "Benchmarks"; Gray-Scott in Pearson's
 * two-field form, which the paper names in its Introduction).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library includes, links or
 * calls this file, and this file uses nothing of the GPU library; the two share
 * no code.  Only the tests, the package smoke check and the benchmark's CPU
 * baseline leg load it.
 *
 * Plain on purpose: every time step is a loop over all grid points that reads
 * its neighbours through a periodic wrap; Cahn-Hilliard stores the chemical
 * potential of every point in a full array before the outer Laplacian.  There
 * is no blocking, no fusion across steps and no reordering beyond the fixed
 * evaluation order written below (which the GPU FP64 path also follows, so
 * FP64 results can be compared bit for bit).
 *
 * Layout: a field is an array of nx*ny*nz doubles, index (z*ny + y)*nx + x,
 * x fastest; 2D grids have nz == 1.
 *
 * Readings of the paper (it prints no stencil coefficients, no integrator and
 * no Gray-Scott equations):
 *  - forward Euler: phi' = phi + dt * RHS;
 *  - Laplacian stencils, written as integer weights over a denominator q,
 *    L_h f = (1/(q h^2)) * sum_s w_s f(x+s):
 *      S1 2D 5-point            q=1  : centre -4, faces 1
 *      S2 2D 9-point isotropic  q=6  : centre -20, faces 4, corners 1
 *      S3 2D 4th-order cross    q=12 : centre -60, +-1: 16, +-2: -1 (per axis)
 *      S4 3D 7-point            q=1  : centre -6, faces 1
 *      S5 3D 27-point isotropic q=30 : centre -128, faces 14, edges 3, corners 1
 *      S6 3D 4th-order cross    q=12 : centre -90, +-1: 16, +-2: -1 (per axis)
 *    (the paper derives stencils from polynomial interpolation, Sec.
 *    "Compile-Time Stencil Generation"; the isotropic S2/S5 choice and the
 *    4th-order cross are readings, pinned by tests against Taylor moments and
 *    exact Fourier symbols);
 *  - Cahn-Hilliard with kappa on the inner Laplacian, both Laplacians by the
 *    same stencil, composed (L_h applied to mu), not a direct biharmonic;
 *  - Gray-Scott, both fields read from the old time level:
 *      du/dt = Du lap u - u v^2 + F (1 - u)
 *      dv/dt = Dv lap v + u v^2 - (F + k) v;
 *  - Model C (Sec. "Model C"), a non-conserved phi (u) coupled to a conserved
 *    density rho (v).  The printed equation and the paper's free-energy listing
 *    F = int [ LANDAU(phi) + rho^2/2 - c3 phi^2 rho ] disagree in two signs;
 *    this oracle follows the listing (phi relaxes by -dF/dphi, rho is conserved
 *    with chemical potential dF/drho):
 *      dphi/dt = lap phi + c1 phi - c2 phi^3 + 2 c3 phi rho
 *      drho/dt = lap (rho - c3 phi^2);
 *  - Model H (Sec. "Model H", transverse projector set to unity as the paper
 *    does), a conserved scalar m and a d-vector j.  The printed j equation and
 *    the paper's EQUATION_OF listing differ in the sign of the coupling; this
 *    oracle follows the listing, with which the two couplings cancel in
 *    dF/dt for F = int [ LANDAU(m) + |j|^2/2 ]:
 *      mu     = -lap m - c1 m + c2 m^3          (kappa = 1 by default)
 *      dm/dt  = lap mu - c3 div(m j)
 *      dj/dt  = lap j  - c3 m grad mu
 *    grad and div by central differences of the Laplacian stencil's order:
 *    D f = f(+1) - f(-1) over 2h (radius-1 stencils), fma(8, f(+1) - f(-1),
 *    -(f(+2) - f(-2))) over 12h (radius 2).
 *
 * Fixed evaluation order (the FP64 parity contract), per point:
 *   class sums of neighbours as written in stencil_sum(), then
 *   S = fma(w_centre, f0, <weighted class sums>);
 *   q_h2 = (q*h)*h;
 *   Allen-Cahn:    rhs = fma(p, fma(-c2, p*p, c1), (1/q_h2)*S);  p' = fma(dt, rhs, p)
 *   Cahn-Hilliard: mu  = fma(p, fma(c2, p*p, -c1), -((kappa/q_h2)*S(p)))
 *                  p'  = fma(dt/q_h2, S(mu), p)
 *   Gray-Scott:    uvv = (u*v)*v
 *                  ru  = fma(F, 1-u, fma(Du/q_h2, S(u), -uvv))
 *                  rv  = fma(-(F+k), v, fma(Dv/q_h2, S(v), uvv))
 *                  u'  = fma(dt, ru, u);  v' = fma(dt, rv, v)
 *   Model H:       mu  = fma(m, fma(c2, m*m, -c1), -((kappa/q_h2)*S(m)))   (every point first)
 *                  div = (D_x(m j_x) + D_y(m j_y)) [+ D_z(m j_z)],  c3g = c3 * g (g = 1/(2h) or 1/(12h))
 *                  m'  = fma(dt, fma(1/q_h2, S(mu), -(c3g * div)), m)
 *                  j_a' = fma(dt, fma(1/q_h2, S(j_a), -(c3g * (m * D_a mu))), j_a)
 *   Model C:       m   = fma(-c3, u*u, v)                 (every point first)
 *                  gr  = fma(-c2, u*u, fma(2*c3, v, c1))
 *                  u'  = fma(dt, fma(u, gr, (1/q_h2)*S(u)), u)
 *                  v'  = fma(dt/q_h2, S(m), v)
 * Compile with -ffp-contract=off so that no other multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_S1 = 0, OR_S2 = 1, OR_S3 = 2, OR_S4 = 3, OR_S5 = 4, OR_S6 = 5 };
enum { OR_AC = 0, OR_CH = 1, OR_GS = 2, OR_MC = 3, OR_MH = 4 };
/* parameter vector: c1, c2, kappa, Du, Dv, F, k */
enum { P_C1 = 0, P_C2, P_KAPPA, P_DU, P_DV, P_F, P_K, P_C3, P_COUNT };

#define OR_MAXR 4
#define OR_GEN 6 /* generated cross stencil (weights held in the grid) */

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int or_stencil_dims(int st) { return (st >= OR_S4) ? 3 : 2; }
int or_stencil_radius(int st) { return (st == OR_S3 || st == OR_S6) ? 2 : 1; }
int or_stencil_q(int st) {
    switch (st) {
    case OR_GEN: return 1;
    case OR_S1: return 1;
    case OR_S2: return 6;
    case OR_S3: return 12;
    case OR_S4: return 1;
    case OR_S5: return 30;
    case OR_S6: return 12;
    }
    return 0;
}

/* Periodic neighbour tables: w[a][(d+R)*n + i] = (i + d) mod n for |d| <= R. */
typedef struct {
    int64_t n[3];
    int64_t *w[3];
    int gen_dims, gen_r;  /* generated cross stencil: dimensions, radius */
    double gen_w[5];      /* its kernel weights (d w_0, w_1, ..., w_r) */
} grid_t;

static int grid_init(grid_t *g, int64_t nx, int64_t ny, int64_t nz) {
    g->n[0] = nx; g->n[1] = ny; g->n[2] = nz;
    g->gen_dims = 0; g->gen_r = 0;
    for (int a = 0; a < 3; a++) {
        int64_t n = g->n[a];
        g->w[a] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * OR_MAXR + 1) * (size_t)n);
        if (!g->w[a]) return -1;
        for (int d = -OR_MAXR; d <= OR_MAXR; d++)
            for (int64_t i = 0; i < n; i++) {
                int64_t r = (i + d) % n;
                if (r < 0) r += n;
                g->w[a][(d + OR_MAXR) * n + i] = r;
            }
    }
    return 0;
}

static void grid_free(grid_t *g) {
    for (int a = 0; a < 3; a++) free(g->w[a]);
}

static inline double at(const double *f, const grid_t *g, int64_t x, int64_t y, int64_t z,
                        int dx, int dy, int dz) {
    int64_t xx = g->w[0][(dx + OR_MAXR) * g->n[0] + x];
    int64_t yy = g->w[1][(dy + OR_MAXR) * g->n[1] + y];
    int64_t zz = g->w[2][(dz + OR_MAXR) * g->n[2] + z];
    return f[(zz * g->n[1] + yy) * g->n[0] + xx];
}

/* Unscaled weighted neighbour sum S = sum_s w_s f(x+s), in the fixed order. */
static double stencil_sum(int st, const double *f, const grid_t *g, int64_t x, int64_t y, int64_t z) {
#define P(dx, dy, dz) at(f, g, x, y, z, dx, dy, dz)
    if (st == OR_GEN) {
        /* P_j = ((x pair) + (y pair)) [+ (z pair)];  S = fma(d w_0, f_0, w_r P_r (+ ...) fused down to w_1 P_1) */
        double acc = 0.0;
        for (int jj = g->gen_r; jj >= 1; jj--) {
            double pj = (P(jj, 0, 0) + P(-jj, 0, 0)) + (P(0, jj, 0) + P(0, -jj, 0));
            if (g->gen_dims == 3) pj = pj + (P(0, 0, jj) + P(0, 0, -jj));
            acc = (jj == g->gen_r) ? g->gen_w[jj] * pj : fma(g->gen_w[jj], pj, acc);
        }
        return fma(g->gen_w[0], P(0, 0, 0), acc);
    }
    switch (st) {
    case OR_S1: {
        double C = (P(-1, 0, 0) + P(1, 0, 0)) + (P(0, -1, 0) + P(0, 1, 0));
        return fma(-4.0, P(0, 0, 0), C);
    }
    case OR_S2: {
        double C = (P(-1, 0, 0) + P(1, 0, 0)) + (P(0, -1, 0) + P(0, 1, 0));
        double D = (P(-1, -1, 0) + P(1, -1, 0)) + (P(-1, 1, 0) + P(1, 1, 0));
        return fma(-20.0, P(0, 0, 0), fma(4.0, C, D));
    }
    case OR_S3: {
        double F1 = (P(-1, 0, 0) + P(1, 0, 0)) + (P(0, -1, 0) + P(0, 1, 0));
        double F2 = (P(-2, 0, 0) + P(2, 0, 0)) + (P(0, -2, 0) + P(0, 2, 0));
        return fma(-60.0, P(0, 0, 0), fma(16.0, F1, -F2));
    }
    case OR_S4: {
        double F = ((P(-1, 0, 0) + P(1, 0, 0)) + (P(0, -1, 0) + P(0, 1, 0))) + (P(0, 0, -1) + P(0, 0, 1));
        return fma(-6.0, P(0, 0, 0), F);
    }
    case OR_S5: {
        /* in-plane cross and diagonal sums of the planes dz = -1, 0, 1 */
        double Cm = (P(-1, 0, -1) + P(1, 0, -1)) + (P(0, -1, -1) + P(0, 1, -1));
        double C0 = (P(-1, 0, 0) + P(1, 0, 0)) + (P(0, -1, 0) + P(0, 1, 0));
        double Cp = (P(-1, 0, 1) + P(1, 0, 1)) + (P(0, -1, 1) + P(0, 1, 1));
        double Dm = (P(-1, -1, -1) + P(1, -1, -1)) + (P(-1, 1, -1) + P(1, 1, -1));
        double D0 = (P(-1, -1, 0) + P(1, -1, 0)) + (P(-1, 1, 0) + P(1, 1, 0));
        double Dp = (P(-1, -1, 1) + P(1, -1, 1)) + (P(-1, 1, 1) + P(1, 1, 1));
        double F = C0 + (P(0, 0, -1) + P(0, 0, 1)); /* 6 faces   */
        double E = D0 + (Cm + Cp);                  /* 12 edges  */
        double K = Dm + Dp;                         /* 8 corners */
        return fma(-128.0, P(0, 0, 0), fma(14.0, F, fma(3.0, E, K)));
    }
    case OR_S6: {
        double F1 = ((P(-1, 0, 0) + P(1, 0, 0)) + (P(0, -1, 0) + P(0, 1, 0))) + (P(0, 0, -1) + P(0, 0, 1));
        double F2 = ((P(-2, 0, 0) + P(2, 0, 0)) + (P(0, -2, 0) + P(0, 2, 0))) + (P(0, 0, -2) + P(0, 0, 2));
        return fma(-90.0, P(0, 0, 0), fma(16.0, F1, -F2));
    }
    }
#undef P
    return NAN;
}

static int check_grid(int st, int64_t nx, int64_t ny, int64_t nz) {
    if (st < OR_S1 || st > OR_S6) return -1;
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    if (or_stencil_dims(st) == 2 && nz != 1) return -1;
    return 0;
}

/* out = S (unscaled weighted sum) at every point. */
int or_stencil_sum(int st, int64_t nx, int64_t ny, int64_t nz, const double *f, double *out) {
    grid_t g;
    if (check_grid(st, nx, ny, nz) || grid_init(&g, nx, ny, nz)) return -1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t z = 0; z < nz; z++)
        for (int64_t y = 0; y < ny; y++)
            for (int64_t x = 0; x < nx; x++)
                out[(z * ny + y) * nx + x] = stencil_sum(st, f, &g, x, y, z);
    grid_free(&g);
    return 0;
}

/* out = L_h f = S / (q h^2) at every point. */
int or_laplacian(int st, int64_t nx, int64_t ny, int64_t nz, double h, const double *f, double *out) {
    if (or_stencil_sum(st, nx, ny, nz, f, out)) return -1;
    const double s = 1.0 / (((double)or_stencil_q(st) * h) * h);
    const int64_t n = nx * ny * nz;
    for (int64_t i = 0; i < n; i++) out[i] = s * out[i];
    return 0;
}

/* Cahn-Hilliard chemical potential mu = c2 p^3 - c1 p - kappa L_h p at every point. */
static void ch_mu(int st, const grid_t *g, const double *p, double *mu, double kq, double c1, double c2) {
    const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t z = 0; z < nz; z++)
        for (int64_t y = 0; y < ny; y++)
            for (int64_t x = 0; x < nx; x++) {
                const int64_t i = (z * ny + y) * nx + x;
                const double pi = p[i];
                const double S = stencil_sum(st, p, g, x, y, z);
                mu[i] = fma(pi, fma(c2, pi * pi, -c1), -(kq * S));
            }
}

int or_chemical_potential(int st, int64_t nx, int64_t ny, int64_t nz, double h, const double *prm,
                          const double *p, double *mu) {
    grid_t g;
    if (check_grid(st, nx, ny, nz) || grid_init(&g, nx, ny, nz)) return -1;
    const double q_h2 = ((double)or_stencil_q(st) * h) * h;
    ch_mu(st, &g, p, mu, prm[P_KAPPA] / q_h2, prm[P_C1], prm[P_C2]);
    grid_free(&g);
    return 0;
}

/*
 * Advance nsteps forward-Euler steps in place.  u is the only field of
 * Allen-Cahn / Cahn-Hilliard; Gray-Scott has u and v, Model C phi = u and
 * rho = v.  prm = {c1, c2, kappa, Du, Dv, F, k, c3}.  Returns 0, or -1 on bad
 * arguments / allocation failure.
 */
static int step_body(int model, int st, grid_t *gp, double h, double dt, const double *prm, double *u, double *v,
                     int64_t nsteps);

int or_step(int model, int st, int64_t nx, int64_t ny, int64_t nz, double h, double dt,
            const double *prm, double *u, double *v, int64_t nsteps) {
    grid_t g;
    if (check_grid(st, nx, ny, nz) || model < OR_AC || model > OR_MC || nsteps < 0) return -1;
    if ((model == OR_GS || model == OR_MC) && !v) return -1;
    if (grid_init(&g, nx, ny, nz)) return -1;
    const int rc = step_body(model, st, &g, h, dt, prm, u, v, nsteps);
    grid_free(&g);
    return rc;
}

/*
 * The same steps with a generated cross stencil of radius r (1..4) in dims
 * dimensions: wk = (d w_0, w_1, ..., w_r), the exact weights of the order-2r
 * central second derivative rounded once to FP64 (oracle/stencil_gen.py); the
 * Laplacian is S / h^2 with S = fma(d w_0, f_0, ...) as in stencil_sum().
 */
int or_step_gen(int model, int dims, int r, const double *wk, int64_t nx, int64_t ny, int64_t nz, double h, double dt,
                const double *prm, double *u, double *v, int64_t nsteps) {
    grid_t g;
    if (model < OR_AC || model > OR_MC || nsteps < 0 || r < 1 || r > OR_MAXR || !wk) return -1;
    if ((dims != 2 && dims != 3) || nx < 1 || ny < 1 || nz < 1 || (dims == 2 && nz != 1)) return -1;
    if ((model == OR_GS || model == OR_MC) && !v) return -1;
    if (grid_init(&g, nx, ny, nz)) return -1;
    g.gen_dims = dims;
    g.gen_r = r;
    for (int j = 0; j <= r; j++) g.gen_w[j] = wk[j];
    const int rc = step_body(model, OR_GEN, &g, h, dt, prm, u, v, nsteps);
    grid_free(&g);
    return rc;
}

static int step_body(int model, int st, grid_t *gp, double h, double dt, const double *prm, double *u, double *v,
                     int64_t nsteps) {
    grid_t g = *gp;
    const int two = (model == OR_GS || model == OR_MC);
    const int64_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int64_t n = nx * ny * nz;
    const double q_h2 = ((double)or_stencil_q(st) * h) * h;
    const double c1 = prm[P_C1], c2 = prm[P_C2];
    double *un = (double *)malloc(sizeof(double) * (size_t)n);
    double *vn = two ? (double *)malloc(sizeof(double) * (size_t)n) : NULL;
    double *mu = (model == OR_CH || model == OR_MC) ? (double *)malloc(sizeof(double) * (size_t)n) : NULL;
    if (!un || (two && !vn) || ((model == OR_CH || model == OR_MC) && !mu)) {
        free(un); free(vn); free(mu);
        return -1;
    }
    double *uc = u, *vc = v;
    for (int64_t s = 0; s < nsteps; s++) {
        if (model == OR_AC) {
            const double sAC = 1.0 / q_h2;
#pragma omp parallel for collapse(2) schedule(static)
            for (int64_t z = 0; z < nz; z++)
                for (int64_t y = 0; y < ny; y++)
                    for (int64_t x = 0; x < nx; x++) {
                        const int64_t i = (z * ny + y) * nx + x;
                        const double p = uc[i];
                        const double S = stencil_sum(st, uc, &g, x, y, z);
                        const double rhs = fma(p, fma(-c2, p * p, c1), sAC * S);
                        un[i] = fma(dt, rhs, p);
                    }
        } else if (model == OR_CH) {
            ch_mu(st, &g, uc, mu, prm[P_KAPPA] / q_h2, c1, c2);
            const double dq = dt / q_h2;
#pragma omp parallel for collapse(2) schedule(static)
            for (int64_t z = 0; z < nz; z++)
                for (int64_t y = 0; y < ny; y++)
                    for (int64_t x = 0; x < nx; x++) {
                        const int64_t i = (z * ny + y) * nx + x;
                        un[i] = fma(dq, stencil_sum(st, mu, &g, x, y, z), uc[i]);
                    }
        } else if (model == OR_MC) {
            /* chemical potential of the conserved density at every point first */
            const double c3 = prm[P_C3], c3x2 = 2.0 * prm[P_C3];
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; i++) mu[i] = fma(-c3, uc[i] * uc[i], vc[i]);
            const double sAC = 1.0 / q_h2, dq = dt / q_h2;
#pragma omp parallel for collapse(2) schedule(static)
            for (int64_t z = 0; z < nz; z++)
                for (int64_t y = 0; y < ny; y++)
                    for (int64_t x = 0; x < nx; x++) {
                        const int64_t i = (z * ny + y) * nx + x;
                        const double p = uc[i], r = vc[i];
                        const double gr = fma(-c2, p * p, fma(c3x2, r, c1));
                        un[i] = fma(dt, fma(p, gr, sAC * stencil_sum(st, uc, &g, x, y, z)), p);
                        vn[i] = fma(dq, stencil_sum(st, mu, &g, x, y, z), r);
                    }
        } else {
            const double duq = prm[P_DU] / q_h2, dvq = prm[P_DV] / q_h2;
            const double F = prm[P_F], Fk = prm[P_F] + prm[P_K];
#pragma omp parallel for collapse(2) schedule(static)
            for (int64_t z = 0; z < nz; z++)
                for (int64_t y = 0; y < ny; y++)
                    for (int64_t x = 0; x < nx; x++) {
                        const int64_t i = (z * ny + y) * nx + x;
                        const double a = uc[i], b = vc[i];
                        const double uvv = (a * b) * b;
                        const double ru = fma(F, 1.0 - a, fma(duq, stencil_sum(st, uc, &g, x, y, z), -uvv));
                        const double rv = fma(-Fk, b, fma(dvq, stencil_sum(st, vc, &g, x, y, z), uvv));
                        un[i] = fma(dt, ru, a);
                        vn[i] = fma(dt, rv, b);
                    }
        }
        /* ping-pong: the new level becomes current */
        double *t = uc; uc = un; un = t;
        if (two) { t = vc; vc = vn; vn = t; }
    }
    if (uc != u) { memcpy(u, uc, sizeof(double) * (size_t)n); un = uc; }
    if (two && vc != v) { memcpy(v, vc, sizeof(double) * (size_t)n); vn = vc; }
    free(un); free(vn); free(mu);
    return 0;
}

/* Central difference along axis a (0 = x) of f at (x, y, z), unscaled: radius 1
 * f(+1) - f(-1); radius 2 fma(8, f(+1) - f(-1), -(f(+2) - f(-2))). */
static double central_diff(int radius, int a, const double *f, const grid_t *g, int64_t x, int64_t y, int64_t z) {
    const int ex = (a == 0), ey = (a == 1), ez = (a == 2);
    const double d1 = at(f, g, x, y, z, ex, ey, ez) - at(f, g, x, y, z, -ex, -ey, -ez);
    if (radius == 1) return d1;
    const double d2 = at(f, g, x, y, z, 2 * ex, 2 * ey, 2 * ez) - at(f, g, x, y, z, -2 * ex, -2 * ey, -2 * ez);
    return fma(8.0, d1, -d2);
}

/*
 * Model H: advance m and j (dims components: j[0] = x, j[1] = y, j[2] = z) by
 * nsteps forward-Euler steps in place.  prm = {c1, c2, kappa, Du, Dv, F, k, c3}
 * (only c1, c2, kappa, c3 enter).  Returns 0, or -1 on bad arguments / memory.
 */
int or_step_h(int st, int64_t nx, int64_t ny, int64_t nz, double h, double dt, const double *prm, double *m,
              double *j0, double *j1, double *j2, int64_t nsteps) {
    grid_t g;
    const int dims = or_stencil_dims(st);
    if (check_grid(st, nx, ny, nz) || nsteps < 0 || !m || !j0 || !j1 || (dims == 3 && !j2)) return -1;
    if (grid_init(&g, nx, ny, nz)) return -1;
    const int64_t n = nx * ny * nz;
    const int radius = or_stencil_radius(st);
    const double q_h2 = ((double)or_stencil_q(st) * h) * h;
    const double sL = 1.0 / q_h2, kq = prm[P_KAPPA] / q_h2;
    const double c3g = prm[P_C3] * (radius == 1 ? 1.0 / (2.0 * h) : 1.0 / (12.0 * h));
    double *jc[3] = {j0, j1, j2};
    double *mn = (double *)malloc(sizeof(double) * (size_t)n);
    double *mu = (double *)malloc(sizeof(double) * (size_t)n);
    double *mj = (double *)malloc(sizeof(double) * (size_t)n * (size_t)dims);
    double *jn[3] = {NULL, NULL, NULL};
    int bad = !mn || !mu || !mj;
    for (int a = 0; a < dims; a++) {
        jn[a] = (double *)malloc(sizeof(double) * (size_t)n);
        bad |= !jn[a];
    }
    if (bad) {
        free(mn); free(mu); free(mj);
        for (int a = 0; a < 3; a++) free(jn[a]);
        grid_free(&g);
        return -1;
    }
    double *mc = m;
    double *jcur[3] = {jc[0], jc[1], dims == 3 ? jc[2] : NULL};
    for (int64_t s = 0; s < nsteps; s++) {
        ch_mu(st, &g, mc, mu, kq, prm[P_C1], prm[P_C2]);
        /* the fluxes m j_a at every point */
        for (int a = 0; a < dims; a++) {
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; i++) mj[(size_t)a * n + i] = mc[i] * jcur[a][i];
        }
#pragma omp parallel for collapse(2) schedule(static)
        for (int64_t z = 0; z < nz; z++)
            for (int64_t y = 0; y < ny; y++)
                for (int64_t x = 0; x < nx; x++) {
                    const int64_t i = (z * ny + y) * nx + x;
                    double div = central_diff(radius, 0, mj, &g, x, y, z) +
                                 central_diff(radius, 1, mj + (size_t)n, &g, x, y, z);
                    if (dims == 3) div = div + central_diff(radius, 2, mj + 2 * (size_t)n, &g, x, y, z);
                    mn[i] = fma(dt, fma(sL, stencil_sum(st, mu, &g, x, y, z), -(c3g * div)), mc[i]);
                    for (int a = 0; a < dims; a++) {
                        const double gm = central_diff(radius, a, mu, &g, x, y, z);
                        jn[a][i] = fma(dt, fma(sL, stencil_sum(st, jcur[a], &g, x, y, z), -(c3g * (mc[i] * gm))),
                                       jcur[a][i]);
                    }
                }
        double *t = mc; mc = mn; mn = t;
        for (int a = 0; a < dims; a++) { t = jcur[a]; jcur[a] = jn[a]; jn[a] = t; }
    }
    if (mc != m) { memcpy(m, mc, sizeof(double) * (size_t)n); mn = mc; }
    for (int a = 0; a < dims; a++)
        if (jcur[a] != jc[a]) { memcpy(jc[a], jcur[a], sizeof(double) * (size_t)n); jn[a] = jcur[a]; }
    free(mn); free(mu); free(mj);
    for (int a = 0; a < dims; a++) free(jn[a]);
    grid_free(&g);
    return 0;
}

/* ---------------------------------------------------------------- IC ---- */

/*
 * n-th output (n = 0, 1, ...) of SplitMix64 seeded with `seed` (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
 * state after n+1 calls is seed + (n+1)*gamma, and the output is the state
 * passed through the 64-bit finaliser below.
 */
uint64_t or_splitmix64_nth(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1u) * UINT64_C(0x9E3779B97F4A7C15);
    z = (z ^ (z >> 30)) * UINT64_C(0xBF58476D1CE4E5B9);
    z = (z ^ (z >> 27)) * UINT64_C(0x94D049BB133111EB);
    return z ^ (z >> 31);
}

/* Uniform double in [0, 1): the top 53 bits of the n-th output. */
double or_u01(uint64_t seed, uint64_t n) {
    return (double)(or_splitmix64_nth(seed, n) >> 11) * 0x1.0p-53;
}

/*
 * Seeded initial condition (the paper starts from "uniformly distributed random
 * noise", Sec. "Benchmarks").  With N = nx*ny*nz points:
 *  - Allen-Cahn / Cahn-Hilliard: u_i = mean + amp*(2 U(i) - 1), U(n) = or_u01(seed, n).
 *  - Gray-Scott: u = 1, v = 0 everywhere, then `patches` square (2D) or cubic (3D)
 *    patches of side `patch` set u = 0.5, v = 0.25.  Patch p has lower corner
 *    c_a - patch/2 on axis a, with c_a = splitmix64_nth(seed, 2N + 3p + a) mod n_a,
 *    and wraps periodically.  Then u_i += amp*(2U(i)-1), v_i += amp*(2U(N+i)-1)
 *    (each written as base + amp*(2U-1)).
 * dims selects 2D (nz must be 1) or 3D.
 */
int or_initial_condition(int model, int dims, int64_t nx, int64_t ny, int64_t nz, uint64_t seed,
                         double mean, double amp, int64_t patches, int64_t patch, double *u, double *v) {
    if (nx < 1 || ny < 1 || nz < 1 || (dims == 2 && nz != 1) || (dims != 2 && dims != 3)) return -1;
    const int64_t N = nx * ny * nz;
    if (model == OR_AC || model == OR_CH) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; i++) u[i] = mean + amp * (2.0 * or_u01(seed, (uint64_t)i) - 1.0);
        return 0;
    }
    if (model == OR_MC) {
        if (!v) return -1;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; i++) {
            u[i] = mean + amp * (2.0 * or_u01(seed, (uint64_t)i) - 1.0);
            v[i] = mean + amp * (2.0 * or_u01(seed, (uint64_t)(N + i)) - 1.0);
        }
        return 0;
    }
    if (model != OR_GS || !v || patches < 0 || patch < 0) return -1;
    if (patch > nx || patch > ny || (dims == 3 && patch > nz)) return -1;
    int64_t *lo = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(patches > 0 ? patches : 1));
    if (!lo) return -1;
    for (int64_t p = 0; p < patches; p++) {
        const int64_t nn[3] = {nx, ny, nz};
        for (int a = 0; a < 3; a++) {
            int64_t c = (int64_t)(or_splitmix64_nth(seed, (uint64_t)(2 * N + 3 * p + a)) % (uint64_t)nn[a]);
            int64_t l = (c - patch / 2) % nn[a];
            if (l < 0) l += nn[a];
            lo[3 * p + a] = l;
        }
    }
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t z = 0; z < nz; z++)
        for (int64_t y = 0; y < ny; y++)
            for (int64_t x = 0; x < nx; x++) {
                const int64_t i = (z * ny + y) * nx + x;
                double bu = 1.0, bv = 0.0;
                for (int64_t p = 0; p < patches; p++) {
                    int64_t ox = (x - lo[3 * p + 0]) % nx; if (ox < 0) ox += nx;
                    int64_t oy = (y - lo[3 * p + 1]) % ny; if (oy < 0) oy += ny;
                    int64_t oz = 0;
                    if (dims == 3) { oz = (z - lo[3 * p + 2]) % nz; if (oz < 0) oz += nz; }
                    if (ox < patch && oy < patch && oz < (dims == 3 ? patch : 1)) { bu = 0.5; bv = 0.25; }
                }
                u[i] = bu + amp * (2.0 * or_u01(seed, (uint64_t)i) - 1.0);
                v[i] = bv + amp * (2.0 * or_u01(seed, (uint64_t)(N + i)) - 1.0);
            }
    free(lo);
    return 0;
}

/*
 * The same initial condition evaluated only on a window of the full grid:
 * out[(k*wy + j)*wx + i] is the value at global point ((x0+i) mod nx,
 * (y0+j) mod ny, (z0+k) mod nz) of or_initial_condition on the nx x ny x nz
 * grid.  Lets tests check sampled windows of grids too large to generate whole.
 */
int or_initial_condition_window(int model, int dims, int64_t nx, int64_t ny, int64_t nz, uint64_t seed,
                                double mean, double amp, int64_t patches, int64_t patch,
                                int64_t x0, int64_t y0, int64_t z0, int64_t wx, int64_t wy, int64_t wz,
                                double *u, double *v) {
    if (nx < 1 || ny < 1 || nz < 1 || (dims == 2 && nz != 1) || (dims != 2 && dims != 3)) return -1;
    if (wx < 1 || wy < 1 || wz < 1) return -1;
    const int64_t N = nx * ny * nz;
    int64_t *lo = NULL;
    if (model == OR_GS) {
        if (!v || patches < 0 || patch < 0 || patch > nx || patch > ny || (dims == 3 && patch > nz)) return -1;
        lo = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(patches > 0 ? patches : 1));
        if (!lo) return -1;
        const int64_t nn[3] = {nx, ny, nz};
        for (int64_t p = 0; p < patches; p++)
            for (int a = 0; a < 3; a++) {
                int64_t c = (int64_t)(or_splitmix64_nth(seed, (uint64_t)(2 * N + 3 * p + a)) % (uint64_t)nn[a]);
                int64_t l = (c - patch / 2) % nn[a];
                if (l < 0) l += nn[a];
                lo[3 * p + a] = l;
            }
    } else if (model == OR_MC) {
        if (!v) return -1;
    } else if (model != OR_AC && model != OR_CH) {
        return -1;
    }
    for (int64_t k = 0; k < wz; k++)
        for (int64_t j = 0; j < wy; j++)
            for (int64_t i = 0; i < wx; i++) {
                int64_t x = (x0 + i) % nx; if (x < 0) x += nx;
                int64_t y = (y0 + j) % ny; if (y < 0) y += ny;
                int64_t z = (z0 + k) % nz; if (z < 0) z += nz;
                const int64_t g = (z * ny + y) * nx + x;
                const int64_t o = (k * wy + j) * wx + i;
                if (model != OR_GS) {
                    u[o] = mean + amp * (2.0 * or_u01(seed, (uint64_t)g) - 1.0);
                    if (model == OR_MC) v[o] = mean + amp * (2.0 * or_u01(seed, (uint64_t)(N + g)) - 1.0);
                    continue;
                }
                double bu = 1.0, bv = 0.0;
                for (int64_t p = 0; p < patches; p++) {
                    int64_t ox = (x - lo[3 * p + 0]) % nx; if (ox < 0) ox += nx;
                    int64_t oy = (y - lo[3 * p + 1]) % ny; if (oy < 0) oy += ny;
                    int64_t oz = 0;
                    if (dims == 3) { oz = (z - lo[3 * p + 2]) % nz; if (oz < 0) oz += nz; }
                    if (ox < patch && oy < patch && oz < (dims == 3 ? patch : 1)) { bu = 0.5; bv = 0.25; }
                }
                u[o] = bu + amp * (2.0 * or_u01(seed, (uint64_t)g) - 1.0);
                v[o] = bv + amp * (2.0 * or_u01(seed, (uint64_t)(N + g)) - 1.0);
            }
    free(lo);
    return 0;
}

/* -------------------------------------------------------- reductions ---- */

/* Neumaier-compensated sum, sequential in index order. */
double or_sum(const double *f, int64_t n) {
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; i++) {
        const double x = f[i];
        const double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    return s + c;
}

static double cell_volume(int dims, double h) { return dims == 3 ? (h * h) * h : h * h; }

/* Mass M = h^d * sum_i phi_i. */
double or_mass(int dims, int64_t nx, int64_t ny, int64_t nz, double h, const double *f) {
    return cell_volume(dims, h) * or_sum(f, nx * ny * nz);
}

/*
 * Discrete Landau free energy (the LANDAU_FE density of Models A/B, whose
 * functional derivative gives Eq. (model-a) and Eq. (model-b)):
 *   F_h = h^d sum_i [ 1/2 sum_axes ((phi_{i+e} - phi_i)/h)^2 - c1/2 phi^2 + c2/4 phi^4 ]
 * with forward differences (a reading: the paper gives no discrete gradient).
 */
double or_free_energy(int dims, int64_t nx, int64_t ny, int64_t nz, double h, double c1, double c2,
                      const double *f) {
    const int64_t n = nx * ny * nz;
    double *e = (double *)malloc(sizeof(double) * (size_t)n);
    if (!e) return NAN;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t z = 0; z < nz; z++)
        for (int64_t y = 0; y < ny; y++)
            for (int64_t x = 0; x < nx; x++) {
                const int64_t i = (z * ny + y) * nx + x;
                const double p = f[i];
                const double gx = (f[(z * ny + y) * nx + (x + 1) % nx] - p) / h;
                const double gy = (f[(z * ny + (y + 1) % ny) * nx + x] - p) / h;
                double g2 = gx * gx + gy * gy;
                if (dims == 3) {
                    const double gz = (f[(((z + 1) % nz) * ny + y) * nx + x] - p) / h;
                    g2 += gz * gz;
                }
                const double p2 = p * p;
                e[i] = 0.5 * g2 - 0.5 * c1 * p2 + 0.25 * c2 * p2 * p2;
            }
    const double r = cell_volume(dims, h) * or_sum(e, n);
    free(e);
    return r;
}

/*
 * Discrete Model C free energy (the paper's listing for Model C): the Landau
 * terms of phi as in or_free_energy plus the density terms rho^2/2 - c3 phi^2 rho:
 *   F_h = h^d sum_i [ 1/2 |D+ phi|^2 - c1/2 phi^2 + c2/4 phi^4 + 1/2 rho^2 - c3 phi^2 rho ].
 */
double or_free_energy_c(int dims, int64_t nx, int64_t ny, int64_t nz, double h, double c1, double c2, double c3,
                        const double *f, const double *rho) {
    const int64_t n = nx * ny * nz;
    double *e = (double *)malloc(sizeof(double) * (size_t)n);
    if (!e) return NAN;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t z = 0; z < nz; z++)
        for (int64_t y = 0; y < ny; y++)
            for (int64_t x = 0; x < nx; x++) {
                const int64_t i = (z * ny + y) * nx + x;
                const double p = f[i], r = rho[i];
                const double gx = (f[(z * ny + y) * nx + (x + 1) % nx] - p) / h;
                const double gy = (f[(z * ny + (y + 1) % ny) * nx + x] - p) / h;
                double g2 = gx * gx + gy * gy;
                if (dims == 3) {
                    const double gz = (f[(((z + 1) % nz) * ny + y) * nx + x] - p) / h;
                    g2 += gz * gz;
                }
                const double p2 = p * p;
                e[i] = 0.5 * g2 - 0.5 * c1 * p2 + 0.25 * c2 * p2 * p2 + 0.5 * r * r - c3 * p2 * r;
            }
    const double res = cell_volume(dims, h) * or_sum(e, n);
    free(e);
    return res;
}

/* Relative L2 distance ||a - b|| / ||b|| (plain, with compensated sums). */
double or_rel_l2(const double *a, const double *b, int64_t n) {
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    if (!d || !r) { free(d); free(r); return NAN; }
    for (int64_t i = 0; i < n; i++) { d[i] = (a[i] - b[i]) * (a[i] - b[i]); r[i] = b[i] * b[i]; }
    const double num = or_sum(d, n), den = or_sum(r, n);
    free(d); free(r);
    return den > 0 ? sqrt(num / den) : sqrt(num);
}

/*
 * Model H initial condition: m_i = mean + amp (2U(i) - 1), j_a,i = amp (2U((a+1)N + i) - 1).
 */
int or_initial_condition_h(int dims, int64_t nx, int64_t ny, int64_t nz, uint64_t seed, double mean, double amp,
                           double *m, double *j0, double *j1, double *j2) {
    if (nx < 1 || ny < 1 || nz < 1 || (dims == 2 && nz != 1) || (dims != 2 && dims != 3)) return -1;
    if (!m || !j0 || !j1 || (dims == 3 && !j2)) return -1;
    const int64_t N = nx * ny * nz;
    double *jc[3] = {j0, j1, j2};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++) {
        m[i] = mean + amp * (2.0 * or_u01(seed, (uint64_t)i) - 1.0);
        for (int a = 0; a < dims; a++) jc[a][i] = amp * (2.0 * or_u01(seed, (uint64_t)((a + 1) * N + i)) - 1.0);
    }
    return 0;
}

/* Model H free energy: the Landau terms of m (as or_free_energy) plus h^d sum |j|^2 / 2. */
double or_free_energy_h(int dims, int64_t nx, int64_t ny, int64_t nz, double h, double c1, double c2,
                        const double *m, const double *j0, const double *j1, const double *j2) {
    const int64_t n = nx * ny * nz;
    const double land = or_free_energy(dims, nx, ny, nz, h, c1, c2, m);
    double *e = (double *)malloc(sizeof(double) * (size_t)n);
    if (!e) return NAN;
    const double *jc[3] = {j0, j1, j2};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double q = j0[i] * j0[i] + j1[i] * j1[i];
        if (dims == 3) q = q + j2[i] * j2[i];
        e[i] = 0.5 * q;
    }
    (void)jc;
    const double r = land + cell_volume(dims, h) * or_sum(e, n);
    free(e);
    return r;
}

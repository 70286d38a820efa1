/*
 * FP64 CPU oracle of the thin-film D2Q9 lattice Boltzmann step of
 * Zitz, Scagliarini, Maddu, Darhuber, Harting, "A lattice Boltzmann method for
 * thin liquid film hydrodynamics" (arXiv:1810.07642), Section II.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  It shares no source, header,
 * table or constant with the CUDA library and must never be called by it.
 *
 * Everything is double precision, evaluated phase by phase over the whole
 * lattice (Jacobi: every stencil sees time-t fields only), in the order the
 * paper gives the method:
 *   moments -> Laplacian of h -> film pressure -> gradient of p -> total force
 *   -> BGK collision with source term -> streaming.
 * Build with -ffp-contract=off so that no multiply-add is fused behind the
 * reader's back.  OpenMP splits rows between threads; the arithmetic of every
 * node is the same whatever the thread count, so results are deterministic.
 *
 * Readings taken where the paper is garbled, ambiguous or silent:
 *  - Eq. (equilibria): the printed denominators c_s^2 and c_s^4 violate the
 *    paper's own momentum constraint (with c_s^2 = 1/3 the first moment comes
 *    out as 3hu).  They are read as e^2 and e^4 with e = dx/dt = 1, the
 *    shallow-water form the paper builds on.  The moment constraints of
 *    Section II are then met exactly.
 *  - Eq. (LBE) source term: w_l (dt/c_s^2) c_l.F = 3 w_l c_l.F with c_s^2=1/3,
 *    no extra prefactor; the velocity in f_eq and in the friction is
 *    u = (sum_l c_l f_l)/h taken before collision (forcing = 0, the
 *    default).  forcing = 1 is a labelled alternative, not the paper's
 *    printed equation: the second-order forcing used by many shallow-water
 *    lattice Boltzmann schemes, with u = (sum_l c_l f_l + F/2)/h (the
 *    friction -nu alpha u is then implicit: u (h + nu alpha/2) =
 *    j + F'/2, F' the force without friction) and the source
 *    (1 - omega/2) w_l [3 (c_l - u) + 9 (c_l.u) c_l].F, whose zeroth moment
 *    is 0 and first moment (1 - omega/2) F, so that momentum again gains
 *    exactly F per step.  It exists to compare the two readings against
 *    the growth rates the paper reports (Sec. III A).
 *  - Eq. (pfilm) sign: the printed p = -gamma (lap h - Pi) makes the precursor
 *    film linearly unstable and gives no contact angle.  The physical reading
 *    p = -gamma (lap h + Pi) is the default (pi_sign = +1); pi_sign = -1
 *    evaluates the printed form.
 *  - Eq. (n_laplace): the printed w_l inside the sums is dropped (with it the
 *    stencil does not annihilate a constant); the stencil used is
 *    (1/6)[4 sum_axis + sum_diag - 20 phi].
 *  - The body force F of Eq. (force) is tangential gravity on the liquid
 *    column, F = h (gx_body, gy_body).
 *  - The friction viscosity is the lattice viscosity nu = (tau - 1/2)/3.
 *  - Initial populations are the equilibria at rest, f_l = f_eq_l(h0, 0).
 *  - Normal gravity g enters only through g h^2/2 in the equilibria.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Parameters of one thin-film simulation.  Field order matters: the Python
 * wrapper mirrors it with ctypes. */
typedef struct {
    int32_t nx, ny;       /* periodic lattice, x fastest                     */
    int32_t n_exp, m_exp; /* exponents (n, m) of Eq. (disjoiningP)           */
    int32_t pi_sign;      /* +1: p = -gamma(lap h + Pi); -1: printed form    */
    int32_t forcing;      /* 0: Eq. (LBE) as printed; 1: second-order forcing */
    double tau;           /* BGK relaxation time, omega = 1/tau              */
    double gamma;         /* surface tension                                 */
    double g;             /* gravity in the equilibria (g < 0: hanging film) */
    double delta;         /* slip length of Eq. (alphafric)                  */
    double hstar;         /* precursor film thickness h_*                    */
    double gx_body;       /* tangential body acceleration: F = h (gx, gy)    */
    double gy_body;
} orc_params;

/* ---------------------------------------------------------------- lattice */

/* Eq. (speeds): l = 0 at rest; odd l on the axes, even l on the diagonals,
 * at angle (l-1) pi/4 with length 1 (odd) or sqrt(2) (even). */
static int CX[9], CY[9];
static double W[9];
static int lattice_ready = 0;

static void lattice_setup(void)
{
    if (lattice_ready) return;
    const double pi = 3.14159265358979323846;
    CX[0] = 0; CY[0] = 0;
    for (int l = 1; l < 9; ++l) {
        double len = (l % 2 == 1) ? 1.0 : sqrt(2.0);
        CX[l] = (int)lround(len * cos((l - 1) * pi / 4.0));
        CY[l] = (int)lround(len * sin((l - 1) * pi / 4.0));
    }
    /* weights, Section II: 4/9 at rest, 1/9 on the axes, 1/36 on diagonals */
    W[0] = 4.0 / 9.0;
    for (int l = 1; l < 9; ++l) W[l] = (l % 2 == 1) ? 1.0 / 9.0 : 1.0 / 36.0;
    lattice_ready = 1;
}

void orc_lattice(int32_t* cx, int32_t* cy, double* w)
{
    lattice_setup();
    for (int l = 0; l < 9; ++l) { cx[l] = CX[l]; cy[l] = CY[l]; w[l] = W[l]; }
}

static inline int64_t wrap(int64_t i, int64_t n)
{
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

/* ------------------------------------------------------------ equilibrium */

/* Eq. (equilibria) with c_s^2 read as e^2 = (dx/dt)^2 = 1 (see header). */
void orc_feq(double g, double h, double ux, double uy, double* feq)
{
    lattice_setup();
    const double e2 = 1.0, e4 = e2 * e2;
    const double usq = ux * ux + uy * uy;
    feq[0] = h - 5.0 * g * h * h / (6.0 * e2) - 2.0 * h * usq / (3.0 * e2);
    for (int l = 1; l < 9; ++l) {
        double cu = CX[l] * ux + CY[l] * uy;
        if (l % 2 == 1)
            feq[l] = g * h * h / (6.0 * e2) + h * cu / (3.0 * e2)
                   + h * cu * cu / (2.0 * e4) - h * usq / (6.0 * e2);
        else
            feq[l] = g * h * h / (24.0 * e2) + h * cu / (12.0 * e2)
                   + h * cu * cu / (8.0 * e4) - h * usq / (24.0 * e2);
    }
}

/* ------------------------------------------------------------ stencils */

/* Eq. (n_laplace), read as (1/6)[4 sum_{odd l} phi(x+c_l)
 *                                + sum_{even l} phi(x+c_l) - 20 phi(x)]. */
void orc_laplacian(int32_t nx, int32_t ny, const double* phi, double* out)
{
    lattice_setup();
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
            double s_axis = 0.0, s_diag = 0.0;
            for (int l = 1; l < 9; ++l) {
                double v = phi[wrap(y + CY[l], ny) * nx + wrap(x + CX[l], nx)];
                if (l % 2 == 1) s_axis += v; else s_diag += v;
            }
            out[y * nx + x] = (4.0 * s_axis + s_diag - 20.0 * phi[y * nx + x]) / 6.0;
        }
}

/* Eq. (derivative): grad phi(x) = 3 sum_l w_l c_l phi(x + c_l). */
void orc_gradient(int32_t nx, int32_t ny, const double* phi, double* gx, double* gy)
{
    lattice_setup();
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
            double sx = 0.0, sy = 0.0;
            for (int l = 0; l < 9; ++l) {
                double v = phi[wrap(y + CY[l], ny) * nx + wrap(x + CX[l], nx)];
                sx += W[l] * CX[l] * v;
                sy += W[l] * CY[l] * v;
            }
            gx[y * nx + x] = 3.0 * sx;
            gy[y * nx + x] = 3.0 * sy;
        }
}

/* ------------------------------------------------------------ forces */

/* kappa of Eq. (disjoiningP): (1 - cos theta)(n-1)(m-1)/((n-m) h_*). */
double orc_kappa(double theta, int32_t n, int32_t m, double hstar)
{
    return (1.0 - cos(theta)) * (double)(n - 1) * (double)(m - 1)
         / ((double)(n - m) * hstar);
}

void orc_kappa_field(const orc_params* P, const double* theta, double* kappa)
{
    int64_t N = (int64_t)P->nx * P->ny;
    for (int64_t i = 0; i < N; ++i)
        kappa[i] = orc_kappa(theta[i], P->n_exp, P->m_exp, P->hstar);
}

/* f(h) of Eq. (disjoiningP): (hstar/h)^n - (hstar/h)^m. */
double orc_fdisj(double h, int32_t n, int32_t m, double hstar)
{
    double r = hstar / h;
    return pow(r, (double)n) - pow(r, (double)m);
}

/* Eq. (alphafric): alpha_delta(h) = 6h / (2h^2 + 6 delta h + 3 delta^2). */
double orc_alpha(double h, double delta)
{
    return 6.0 * h / (2.0 * h * h + 6.0 * delta * h + 3.0 * delta * delta);
}

/* ------------------------------------------------------------ the step */

/* Section II, moments: h = sum_l f_l, h u = sum_l c_l f_l. */
void orc_moments(const orc_params* P, const double* f, double* h, double* ux, double* uy)
{
    lattice_setup();
    const int64_t N = (int64_t)P->nx * P->ny;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double hh = 0.0, jx = 0.0, jy = 0.0;
        for (int l = 0; l < 9; ++l) {
            double v = f[l * N + i];
            hh += v;
            jx += CX[l] * v;
            jy += CY[l] * v;
        }
        h[i] = hh;
        if (ux) ux[i] = jx / hh;
        if (uy) uy[i] = jy / hh;
    }
}

/* Film pressure (Eq. pfilm with Eq. disjoiningP) and total force
 * (Eqs. force, forcefric, alphafric) at time t from the moments h, u.
 * lap, p, gpx, gpy are caller workspace of N doubles each. */
static void pressure_force(const orc_params* P, const double* kappa,
                           const double* h, const double* ux, const double* uy,
                           double* lap, double* p, double* gpx, double* gpy,
                           double* Fx, double* Fy)
{
    const int32_t nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    const double nu = (P->tau - 0.5) / 3.0;          /* nu = c_s^2 (tau - 1/2) */

    orc_laplacian(nx, ny, h, lap);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double Pi = kappa[i] * orc_fdisj(h[i], P->n_exp, P->m_exp, P->hstar);
        p[i] = -P->gamma * (lap[i] + (double)P->pi_sign * Pi);
    }
    orc_gradient(nx, ny, p, gpx, gpy);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double a = orc_alpha(h[i], P->delta);
        /* F_film = -(1/rho_0) h grad p with rho_0 = 1 */
        Fx[i] = -h[i] * gpx[i] - nu * a * ux[i] + h[i] * P->gx_body;
        Fy[i] = -h[i] * gpy[i] - nu * a * uy[i] + h[i] * P->gy_body;
    }
}

/* The labelled second-order-forcing alternative (forcing = 1): the velocity
 * u = (j + F/2)/h with the friction -nu alpha u taken at that velocity,
 * u (h + nu alpha/2) = j + F'/2 (F' the film-pressure and body forces), and
 * the total force F = F' - nu alpha u; overwrites ux, uy, Fx, Fy. */
static void second_order_velocity_force(const orc_params* P, const double* f, const double* h,
                                        const double* gpx, const double* gpy, double* ux, double* uy,
                                        double* Fx, double* Fy)
{
    const int64_t N = (int64_t)P->nx * P->ny;
    const double nu = (P->tau - 0.5) / 3.0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double jx = 0.0, jy = 0.0;
        for (int l = 0; l < 9; ++l) { jx += CX[l] * f[l * N + i]; jy += CY[l] * f[l * N + i]; }
        const double a = orc_alpha(h[i], P->delta);
        const double fpx = -h[i] * gpx[i] + h[i] * P->gx_body;
        const double fpy = -h[i] * gpy[i] + h[i] * P->gy_body;
        ux[i] = (jx + 0.5 * fpx) / (h[i] + 0.5 * nu * a);
        uy[i] = (jy + 0.5 * fpy) / (h[i] + 0.5 * nu * a);
        Fx[i] = fpx - nu * a * ux[i];
        Fy[i] = fpy - nu * a * uy[i];
    }
}

/* Film pressure and total force of the post-streaming state f, for
 * diagnostics (the force of the reading selected by P->forcing).  Any output
 * pointer may be NULL. */
void orc_pressure_force(const orc_params* P, const double* kappa, const double* f,
                        double* p_out, double* Fx_out, double* Fy_out)
{
    const int64_t N = (int64_t)P->nx * P->ny;
    double* buf = malloc(sizeof(double) * 9 * N);
    double *h = buf, *ux = buf + N, *uy = buf + 2 * N, *lap = buf + 3 * N,
           *p = buf + 4 * N, *gpx = buf + 5 * N, *gpy = buf + 6 * N,
           *Fx = buf + 7 * N, *Fy = buf + 8 * N;
    orc_moments(P, f, h, ux, uy);
    pressure_force(P, kappa, h, ux, uy, lap, p, gpx, gpy, Fx, Fy);
    if (P->forcing == 1) second_order_velocity_force(P, f, h, gpx, gpy, ux, uy, Fx, Fy);
    if (p_out) memcpy(p_out, p, sizeof(double) * N);
    if (Fx_out) memcpy(Fx_out, Fx, sizeof(double) * N);
    if (Fy_out) memcpy(Fy_out, Fy, sizeof(double) * N);
    free(buf);
}

/* Initial populations: equilibria at rest, f_l(x, 0) = f_eq_l(h0(x), 0). */
void orc_init(const orc_params* P, const double* h0, double* f)
{
    const int64_t N = (int64_t)P->nx * P->ny;
    double fe[9];
    for (int64_t i = 0; i < N; ++i) {
        orc_feq(P->g, h0[i], 0.0, 0.0, fe);
        for (int l = 0; l < 9; ++l) f[l * N + i] = fe[l];
    }
}

/* nsteps applications of Eq. (LBE).  f holds the post-streaming populations
 * f_l(x, t) as [9][ny][nx] and is overwritten by f_l(x, t + nsteps). */
void orc_step(const orc_params* P, const double* kappa, double* f, int64_t nsteps)
{
    lattice_setup();
    const int32_t nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    const double omega = 1.0 / P->tau;
    double* buf = malloc(sizeof(double) * 18 * N);
    double *h = buf, *ux = buf + N, *uy = buf + 2 * N, *lap = buf + 3 * N,
           *p = buf + 4 * N, *gpx = buf + 5 * N, *gpy = buf + 6 * N,
           *Fx = buf + 7 * N, *Fy = buf + 8 * N, *fpost = buf + 9 * N;

    for (int64_t s = 0; s < nsteps; ++s) {
        /* moments, pressure and force, all from time-t fields */
        orc_moments(P, f, h, ux, uy);
        pressure_force(P, kappa, h, ux, uy, lap, p, gpx, gpy, Fx, Fy);
        if (P->forcing == 1) second_order_velocity_force(P, f, h, gpx, gpy, ux, uy, Fx, Fy);
        /* collision: (1 - omega) f + omega f_eq + source */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            double fe[9];
            orc_feq(P->g, h[i], ux[i], uy[i], fe);
            for (int l = 0; l < 9; ++l) {
                double src;
                if (P->forcing == 1) {
                    /* (1 - omega/2) w_l [3 (c_l - u) + 9 (c_l.u) c_l] . F */
                    const double cu = CX[l] * ux[i] + CY[l] * uy[i];
                    const double cF = CX[l] * Fx[i] + CY[l] * Fy[i];
                    const double uF = ux[i] * Fx[i] + uy[i] * Fy[i];
                    src = (1.0 - 0.5 * omega) * W[l] * (3.0 * (cF - uF) + 9.0 * cu * cF);
                } else {
                    /* w_l (dt / c_s^2) c_l . F of Eq. (LBE) */
                    src = 3.0 * W[l] * (CX[l] * Fx[i] + CY[l] * Fy[i]);
                }
                fpost[l * N + i] = (1.0 - omega) * f[l * N + i] + omega * fe[l] + src;
            }
        }
        /* streaming: f_l(x + c_l, t + 1) = f*_l(x, t), periodic */
#pragma omp parallel for schedule(static)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x)
                for (int l = 0; l < 9; ++l) {
                    int64_t to = wrap(y + CY[l], ny) * nx + wrap(x + CX[l], nx);
                    f[l * N + to] = fpost[l * N + y * nx + x];
                }
    }
    free(buf);
}

/* Total liquid volume sum_x h(x) = sum_x sum_l f_l(x), Neumaier-compensated. */
double orc_mass(const orc_params* P, const double* f)
{
    const int64_t n = 9 * (int64_t)P->nx * P->ny;
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double t = s + f[i];
        if (fabs(s) >= fabs(f[i])) c += (s - t) + f[i];
        else c += (f[i] - t) + s;
        s = t;
    }
    return s + c;
}

int32_t orc_num_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------ adjoint */

/* Reverse-mode derivative of one step.  The state is the post-streaming
 * f(t); one step is f(t+1) = S(C(f(t))), C the collision of Eq. (LBE) with
 * the force of Eq. (force), S the streaming.  Given a_next = dL/df(t+1), this
 * writes a = dL/df(t) = (dS C / df)^T a_next and adds (dS C / dkappa)^T a_next
 * to grad_kappa.  The derivative is taken of the same phases as orc_step:
 *   mu_l(x)   = a_next_l(x + c_l)                    (transpose of streaming)
 *   collision f*_l = (1-w) f_l + w E_l(h, j) + 3 w_l c_l . F, with
 *     E_l written in (h, j): E_0 = h - 5gh^2/6 - 2|j|^2/(3h),
 *     axis: gh^2/6 + c.j/3 + (c.j)^2/(2h) - |j|^2/(6h),
 *     diagonal: gh^2/24 + c.j/12 + (c.j)^2/(8h) - |j|^2/(24h);
 *   F = h (G - grad p) - fr(h) j,  fr = 6 nu / (2h^2 + 6 delta h + 3 delta^2);
 *   p = -gamma (lap h + s kappa ((hstar/h)^n - (hstar/h)^m));
 *   h = sum_l f_l,  j = sum_l c_l f_l.
 * Each line of the derivation is a plain loop over the lattice below. */
void orc_adjoint_step(const orc_params* P, const double* kappa, const double* f,
                      const double* a_next, double* a, double* grad_kappa)
{
    lattice_setup();
    const int32_t nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    const double omega = 1.0 / P->tau, nu = (P->tau - 0.5) / 3.0, g = P->g;
    const double s = (double)P->pi_sign;
    double* buf = malloc(sizeof(double) * 28 * N);
    double *h = buf, *jx = buf + N, *jy = buf + 2 * N, *ux = buf + 3 * N, *uy = buf + 4 * N,
           *lap = buf + 5 * N, *p = buf + 6 * N, *gpx = buf + 7 * N, *gpy = buf + 8 * N,
           *mu = buf + 9 * N, /* 9 fields */
           *aH = buf + 18 * N, *aJx = buf + 19 * N, *aJy = buf + 20 * N, *agx = buf + 21 * N,
           *agy = buf + 22 * N, *ap = buf + 23 * N, *alap = buf + 24 * N, *Fx = buf + 25 * N,
           *Fy = buf + 26 * N;

    /* forward quantities at time t */
    orc_moments(P, f, h, ux, uy);
    /* j as the plain population sums, as the forward defines it */
    for (int64_t i = 0; i < N; ++i) {
        double sx = 0.0, sy = 0.0;
        for (int l = 0; l < 9; ++l) { sx += CX[l] * f[l * N + i]; sy += CY[l] * f[l * N + i]; }
        jx[i] = sx; jy[i] = sy;
    }
    pressure_force(P, kappa, h, ux, uy, lap, p, gpx, gpy, Fx, Fy);

    /* transpose of streaming: mu_l(x) = a_next_l(x + c_l) */
    for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x)
            for (int l = 0; l < 9; ++l)
                mu[l * N + y * nx + x] = a_next[l * N + wrap(y + CY[l], ny) * nx + wrap(x + CX[l], nx)];

    /* collision and force, node by node */
    for (int64_t i = 0; i < N; ++i) {
        const double hh = h[i], Jx = jx[i], Jy = jy[i], j2 = Jx * Jx + Jy * Jy;
        double aFx = 0.0, aFy = 0.0, ah = 0.0, ajx = 0.0, ajy = 0.0;
        for (int l = 0; l < 9; ++l) {
            const double m = mu[l * N + i];
            aFx += 3.0 * W[l] * CX[l] * m;
            aFy += 3.0 * W[l] * CY[l] * m;
            const double am = omega * m;  /* adjoint of E_l */
            const double cj = CX[l] * Jx + CY[l] * Jy;
            double dEdh, dEdjx, dEdjy;
            if (l == 0) {
                dEdh = 1.0 - 5.0 * g * hh / 3.0 + 2.0 * j2 / (3.0 * hh * hh);
                dEdjx = -4.0 * Jx / (3.0 * hh);
                dEdjy = -4.0 * Jy / (3.0 * hh);
            } else if (l % 2 == 1) {
                dEdh = g * hh / 3.0 - cj * cj / (2.0 * hh * hh) + j2 / (6.0 * hh * hh);
                dEdjx = CX[l] / 3.0 + cj * CX[l] / hh - Jx / (3.0 * hh);
                dEdjy = CY[l] / 3.0 + cj * CY[l] / hh - Jy / (3.0 * hh);
            } else {
                dEdh = g * hh / 12.0 - cj * cj / (8.0 * hh * hh) + j2 / (24.0 * hh * hh);
                dEdjx = CX[l] / 12.0 + cj * CX[l] / (4.0 * hh) - Jx / (12.0 * hh);
                dEdjy = CY[l] / 12.0 + cj * CY[l] / (4.0 * hh) - Jy / (12.0 * hh);
            }
            ah += am * dEdh;
            ajx += am * dEdjx;
            ajy += am * dEdjy;
        }
        /* F = h (G - grad p) - fr(h) j */
        const double den = 2.0 * hh * hh + 6.0 * P->delta * hh + 3.0 * P->delta * P->delta;
        const double fr = 6.0 * nu / den;
        const double dfr = -6.0 * nu * (4.0 * hh + 6.0 * P->delta) / (den * den);
        ah += aFx * (P->gx_body - gpx[i]) + aFy * (P->gy_body - gpy[i]) - dfr * (aFx * Jx + aFy * Jy);
        ajx += -fr * aFx;
        ajy += -fr * aFy;
        agx[i] = -hh * aFx;
        agy[i] = -hh * aFy;
        aH[i] = ah;
        aJx[i] = ajx;
        aJy[i] = ajy;
    }
    /* transpose of Eq. (derivative): ap(y) = sum_l 3 w_l c_l . ag(y - c_l) */
    for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
            double sum = 0.0;
            for (int l = 0; l < 9; ++l) {
                const int64_t k = wrap(y - CY[l], ny) * nx + wrap(x - CX[l], nx);
                sum += 3.0 * W[l] * (CX[l] * agx[k] + CY[l] * agy[k]);
            }
            ap[y * nx + x] = sum;
        }
    /* p = -gamma (lap + s Pi): Pi contributes to h and to kappa */
    for (int64_t i = 0; i < N; ++i) {
        alap[i] = -P->gamma * ap[i];
        const double api = -P->gamma * s * ap[i];
        const double r = P->hstar / h[i];
        const double rn = pow(r, (double)P->n_exp), rm = pow(r, (double)P->m_exp);
        grad_kappa[i] += api * (rn - rm);
        aH[i] += api * kappa[i] * (-(double)P->n_exp * rn + (double)P->m_exp * rm) / h[i];
    }
    /* Eq. (n_laplace) is symmetric: its transpose is itself */
    orc_laplacian(nx, ny, alap, p); /* p reused as scratch */
    for (int64_t i = 0; i < N; ++i) aH[i] += p[i];
    /* h = sum_l f_l, j = sum_l c_l f_l, and the (1 - w) f_l term */
    for (int64_t i = 0; i < N; ++i)
        for (int l = 0; l < 9; ++l)
            a[l * N + i] = aH[i] + CX[l] * aJx[i] + CY[l] * aJy[i] + (1.0 - omega) * mu[l * N + i];
    free(buf);
}

/* dL/dh0 from dL/df(0) for f_l(x, 0) = f_eq_l(h0(x), 0). */
void orc_adjoint_init(const orc_params* P, const double* h0, const double* a0, double* grad_h0)
{
    lattice_setup();
    const int64_t N = (int64_t)P->nx * P->ny;
    for (int64_t i = 0; i < N; ++i) {
        const double hh = h0[i];
        double s = a0[i] * (1.0 - 5.0 * P->g * hh / 3.0);
        for (int l = 1; l < 9; ++l) s += a0[l * N + i] * P->g * hh * ((l % 2 == 1) ? 1.0 / 3.0 : 1.0 / 12.0);
        grad_h0[i] = s;
    }
}

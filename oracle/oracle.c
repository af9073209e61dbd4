/*
 * oracle.c -- plain, slow, obviously correct CPU oracle for the ensemble ODE
 * method of Nagy, Plavecz & Hegedus, "Solving large number of non-stiff,
 * low-dimensional ordinary differential equation systems on GPUs and CPUs"
 * (arXiv 2011.01740).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py use it.  It shares no source with the CUDA path.
 *
 * Arithmetic: IEEE double throughout, built with -ffp-contract=off (no fused
 * multiply-add), libm sin/cos/pow/sqrt, one system at a time; OpenMP only
 * distributes independent systems over host threads.  Every function follows
 * the equations in the order the paper (or the cited method) states them, with
 * no blocking, fusion or reordering.
 *
 * Sources:
 *   - RK4 (classic fourth-order Runge-Kutta, fixed step): Sec. 3 (introductory
 *     example), Sec. 4.1 (Lorenz).
 *   - Cash-Karp embedded RK4(5): used by the paper (Sec. 4.2.1, Sec. 4.3.1) but
 *     its tableau is not printed there; taken from Cash & Karp, ACM TOMS 16(3),
 *     1990, Table "Cash-Karp parameters".
 *   - Step-size controller, event location and sticking rule: the paper does
 *     not specify them; the readings implemented here are stated at each
 *     function and collected in the design notes of the repository.
 *   - Right-hand sides: x'=x^2-p (Eq. exemplary_system), Lorenz (Eqs. Lorenz1-3),
 *     dimensionless Keller-Miksis (Eqs. dimensionless_system1-2, numerator,
 *     denominator, coefficients), dimensional Keller-Miksis (Eqs.
 *     keller_miksis_1-4), pressure relief valve (Eqs. pressure_relief_valve_1-3)
 *     and its impact law (Eqs. impact_law_1-3).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <float.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXDIM 4

/* systems */
enum {
    ORC_X2P = 0,      /* x' = x^2 - p                   params: p                 */
    ORC_LORENZ = 1,   /* Lorenz                          params: rho, sigma, b     */
    ORC_KM = 2,       /* dimensionless Keller-Miksis     params: C0..C12           */
    ORC_PRV = 3,      /* pressure relief valve           params: q,kappa,delta,beta,r */
    ORC_LINEAR = 4,   /* y' = lambda*y (test problem)    params: lambda            */
    ORC_TPOW = 5,     /* y' = c*t^k   (test problem)     params: k, c              */
    ORC_BALL = 6,     /* y1'=y2, y2'=-g, y3'=0 (test)    params: g, r              */
    ORC_KM_TAN = 7,   /* Keller-Miksis + tangent vector  params: C0..C12           */
    ORC_FCOS = 8      /* y' = c cos(2 pi t) (test)       params: c                 */
};

/* per-system status bits */
enum {
    ORC_ST_DT_UNDERFLOW = 1,
    ORC_ST_MAX_STEPS = 2,
    ORC_ST_NONFINITE = 4,
    ORC_ST_EVENT_NO_CONVERGE = 8
};

int orc_dim(int sys)
{
    switch (sys) {
    case ORC_X2P: return 1;
    case ORC_LORENZ: return 3;
    case ORC_KM: return 2;
    case ORC_PRV: return 3;
    case ORC_LINEAR: return 1;
    case ORC_TPOW: return 1;
    case ORC_BALL: return 3;
    case ORC_KM_TAN: return 4;
    case ORC_FCOS: return 1;
    default: return 0;
    }
}

int orc_npar(int sys)
{
    switch (sys) {
    case ORC_X2P: return 1;
    case ORC_LORENZ: return 3;
    case ORC_KM: return 13;
    case ORC_PRV: return 5;
    case ORC_LINEAR: return 1;
    case ORC_TPOW: return 2;
    case ORC_BALL: return 2;
    case ORC_KM_TAN: return 13;
    case ORC_FCOS: return 1;
    default: return 0;
    }
}

/* ------------------------------------------------------------------------- */
/* Right-hand sides                                                          */
/* ------------------------------------------------------------------------- */

/* x' = x^2 - p  (Sec. 3, Eq. exemplary_system) */
static void rhs_x2p(const double *p, double t, const double *y, double *dy)
{
    (void)t;
    dy[0] = y[0] * y[0] - p[0];
}

/* Lorenz (Sec. 4.1, Eqs. Lorenz1-3) with the printed constants 10 and 2.666
 * generalised to sigma and b:  x1' = sigma (x2 - x1),
 * x2' = rho x1 - x2 - x1 x3,  x3' = x1 x2 - b x3.                          */
static void rhs_lorenz(const double *p, double t, const double *y, double *dy)
{
    const double rho = p[0], sigma = p[1], b = p[2];
    (void)t;
    dy[0] = sigma * (y[1] - y[0]);
    dy[1] = rho * y[0] - y[1] - y[0] * y[2];
    dy[2] = y[0] * y[1] - b * y[2];
}

/* Dimensionless Keller-Miksis equation (Sec. 4.2, Eqs. dimensionless_system1-2
 * with the numerator N_KM and denominator D_KM exactly as printed):
 *   y1' = y2,   y2' = N_KM / D_KM
 *   N_KM = (C0 + C1 y2) (1/y1)^C10 - C2 (1 + C9 y2) - C3 / y1 - C4 y2 / y1
 *          - (1 - C9 y2 / 3) (3/2) y2^2
 *          - (C5 sin(2 pi tau) + C6 sin(2 pi C11 tau + C12)) (1 + C9 y2)
 *          - y1 (C7 cos(2 pi tau) + C8 cos(2 pi C11 tau + C12))
 *   D_KM = y1 - C9 y1 y2 + C4 C9                                           */
static void rhs_km(const double *C, double tau, const double *y, double *dy)
{
    const double y1 = y[0], y2 = y[1];
    const double pi2 = 2.0 * M_PI;
    double N, D;
    N = (C[0] + C[1] * y2) * pow(1.0 / y1, C[10])
        - C[2] * (1.0 + C[9] * y2)
        - C[3] / y1
        - C[4] * y2 / y1
        - (1.0 - C[9] * y2 / 3.0) * 1.5 * y2 * y2
        - (C[5] * sin(pi2 * tau) + C[6] * sin(pi2 * C[11] * tau + C[12])) * (1.0 + C[9] * y2)
        - y1 * (C[7] * cos(pi2 * tau) + C[8] * cos(pi2 * C[11] * tau + C[12]));
    D = y1 - C[9] * y1 * y2 + C[4] * C[9];
    dy[0] = y2;
    dy[1] = N / D;
}

/* Keller-Miksis with its tangent (variational) equation, for the largest
 * Lyapunov exponent of each system.  y = (y1, y2, v1, v2): (y1, y2) follow
 * rhs_km and v' = J v with J the Jacobian of that right-hand side, derived
 * by hand from N_KM and D_KM (g = N_KM / D_KM, F_s and F_c the two forcing
 * sums, P = (1/y1)^C10):
 *   dN/dy1 = -C10 (C0 + C1 y2) P / y1 + C3 / y1^2 + C4 y2 / y1^2 - F_c
 *   dN/dy2 = C1 P - C2 C9 - C4 / y1 - 3 y2 + (3/2) C9 y2^2 - C9 F_s
 *   dD/dy1 = 1 - C9 y2,   dD/dy2 = -C9 y1
 *   dg/dyk = (dN/dyk - g dD/dyk) / D
 *   v1' = v2,   v2' = dg/dy1 v1 + dg/dy2 v2.                                */
static void rhs_km_tan(const double *C, double tau, const double *y, double *dy)
{
    const double y1 = y[0], y2 = y[1];
    const double pi2 = 2.0 * M_PI;
    const double Fs = C[5] * sin(pi2 * tau) + C[6] * sin(pi2 * C[11] * tau + C[12]);
    const double Fc = C[7] * cos(pi2 * tau) + C[8] * cos(pi2 * C[11] * tau + C[12]);
    const double P = pow(1.0 / y1, C[10]);
    double f[2], dNdy1, dNdy2, dDdy1, dDdy2, D, g;
    rhs_km(C, tau, y, f);
    D = y1 - C[9] * y1 * y2 + C[4] * C[9];
    g = f[1];
    dNdy1 = -C[10] * (C[0] + C[1] * y2) * P / y1 + C[3] / (y1 * y1) + C[4] * y2 / (y1 * y1) - Fc;
    dNdy2 = C[1] * P - C[2] * C[9] - C[4] / y1 - 3.0 * y2 + 1.5 * C[9] * y2 * y2 - C[9] * Fs;
    dDdy1 = 1.0 - C[9] * y2;
    dDdy2 = -C[9] * y1;
    dy[0] = f[0];
    dy[1] = f[1];
    dy[2] = y[3];
    dy[3] = (dNdy1 - g * dDdy1) / D * y[2] + (dNdy2 - g * dDdy2) / D * y[3];
}

/* Pressure relief valve (Sec. 4.3, Eqs. pressure_relief_valve_1-3):
 *   y1' = y2,  y2' = -kappa y2 - (y1 + delta) + y3,  y3' = beta (q - y1 sqrt(y3)).
 * The pressure y3 stays non-negative for q > 0; sqrt is taken of max(y3, 0)
 * so that a rounding excursion below zero cannot produce a NaN.           */
static void rhs_prv(const double *p, double t, const double *y, double *dy)
{
    const double q = p[0], kappa = p[1], delta = p[2], beta = p[3];
    const double y3 = y[2] > 0.0 ? y[2] : 0.0;
    (void)t;
    dy[0] = y[1];
    dy[1] = -kappa * y[1] - (y[0] + delta) + y[2];
    dy[2] = beta * (q - y[0] * sqrt(y3));
}

static void rhs_linear(const double *p, double t, const double *y, double *dy)
{
    (void)t;
    dy[0] = p[0] * y[0];
}

static void rhs_tpow(const double *p, double t, const double *y, double *dy)
{
    (void)y;
    dy[0] = p[1] * pow(t, p[0]);
}

/* Forced test problem of period 1 in t: y' = c cos(2 pi t), whose solution
 * y0 + c sin(2 pi t) / (2 pi) has its extremes at t = 1/4 and 3/4 of every
 * period; it pins the per-phase maximum / minimum rows of phase mode.       */
static void rhs_fcos(const double *p, double t, const double *y, double *dy)
{
    (void)y;
    dy[0] = p[0] * cos(2.0 * M_PI * t);
}

static void rhs_ball(const double *p, double t, const double *y, double *dy)
{
    (void)t;
    dy[0] = y[1];
    dy[1] = -p[0];
    dy[2] = 0.0;
}

static void rhs(int sys, const double *p, double t, const double *y, double *dy)
{
    switch (sys) {
    case ORC_X2P: rhs_x2p(p, t, y, dy); break;
    case ORC_LORENZ: rhs_lorenz(p, t, y, dy); break;
    case ORC_KM: rhs_km(p, t, y, dy); break;
    case ORC_KM_TAN: rhs_km_tan(p, t, y, dy); break;
    case ORC_PRV: rhs_prv(p, t, y, dy); break;
    case ORC_LINEAR: rhs_linear(p, t, y, dy); break;
    case ORC_TPOW: rhs_tpow(p, t, y, dy); break;
    case ORC_BALL: rhs_ball(p, t, y, dy); break;
    case ORC_FCOS: rhs_fcos(p, t, y, dy); break;
    default: break;
    }
}

/* One RHS evaluation for a whole ensemble; params SoA [npar][n], y and dy SoA [dim][n]. */
void orc_rhs(int sys, int64_t n, const double *params, const double *t, const double *y, double *dy)
{
    const int dim = orc_dim(sys), npar = orc_npar(sys);
    for (int64_t i = 0; i < n; ++i) {
        double p[16], yy[ORC_MAXDIM], d[ORC_MAXDIM];
        for (int k = 0; k < npar; ++k) p[k] = params[k * n + i];
        for (int k = 0; k < dim; ++k) yy[k] = y[k * n + i];
        rhs(sys, p, t[i], yy, d);
        for (int k = 0; k < dim; ++k) dy[k * n + i] = d[k];
    }
}

/* ------------------------------------------------------------------------- */
/* Keller-Miksis coefficients C0..C12 (Sec. 4.2, Eq. coefficients)           */
/* ------------------------------------------------------------------------- */

/* Liquid / gas constants: rho_L, c_L, mu_L, sigma, p_V, P_inf, gamma. */
typedef struct {
    double rho, c, mu, sigma, pv, pinf, gamma;
} orc_liquid;

/* C0..C12 for each system, SoA out[13][n].  Inputs are SI: pressure amplitudes
 * in Pa, frequencies in Hz, theta in rad, R_E in m.  C8 uses omega2: the
 * printed C8 carries omega1, but the time derivative of P_A2 sin(omega2 t +
 * theta) in Eq. keller_miksis_1 brings out omega2 (the two agree whenever
 * P_A2 = 0, the case the paper runs).                                       */
void orc_km_coefficients(int64_t n, const double *pA1, const double *f1, const double *pA2,
                         const double *f2, const double *theta, const double *RE,
                         const orc_liquid *L, double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        const double w1 = 2.0 * M_PI * f1[i];
        const double w2 = 2.0 * M_PI * f2[i];
        const double R = RE[i];
        const double s = 2.0 * M_PI / (R * w1);         /* 2 pi / (R_E omega1) */
        const double s2 = s * s;
        const double pg0 = L->pinf - L->pv + 2.0 * L->sigma / R;
        double C[13];
        C[0] = (1.0 / L->rho) * pg0 * s2;
        C[1] = (1.0 - 3.0 * L->gamma) / (L->rho * L->c) * pg0 * s;
        C[2] = (L->pinf - L->pv) / L->rho * s2;
        C[3] = 2.0 * L->sigma / (L->rho * R) * s2;
        C[4] = 4.0 * L->mu / (L->rho * R * R) * (2.0 * M_PI / w1);
        C[5] = pA1[i] / L->rho * s2;
        C[6] = pA2[i] / L->rho * s2;
        C[7] = R * w1 * pA1[i] / (L->rho * L->c) * s2;
        C[8] = R * w2 * pA2[i] / (L->rho * L->c) * s2;
        C[9] = R * w1 / (2.0 * M_PI * L->c);
        C[10] = 3.0 * L->gamma;
        C[11] = w2 / w1;
        C[12] = theta[i];
        for (int k = 0; k < 13; ++k) out[k * n + i] = C[k];
    }
}

/* Second, independent route: the dimensional Keller-Miksis equation
 * (Eqs. keller_miksis_1-4) solved for R'' directly in SI units.
 *   p_L = p_G + p_V - 2 sigma / R - 4 mu R' / R
 *   p_G = (P_inf - p_V + 2 sigma / R_E) (R_E / R)^(3 gamma)
 *   p_inf(t) = P_inf + P_A1 sin(w1 t) + P_A2 sin(w2 t + theta)
 *   (1 - R'/c) R R'' + (1 - R'/(3c)) (3/2) R'^2
 *       = (1 + R'/c) (p_L - p_inf) / rho + R/(rho c) d/dt (p_L - p_inf)
 * d/dt p_L contains R'' through the viscous term; the equation is linear in
 * R'' and is solved for it here.  Output: R'' in m/s^2.                     */
double orc_km_dimensional_rdd(double R, double Rd, double t, double pA1, double f1,
                              double pA2, double f2, double theta, double RE,
                              const orc_liquid *L)
{
    const double w1 = 2.0 * M_PI * f1, w2 = 2.0 * M_PI * f2;
    const double g3 = 3.0 * L->gamma;
    const double pg0 = L->pinf - L->pv + 2.0 * L->sigma / RE;
    const double pG = pg0 * pow(RE / R, g3);
    const double dpG = -g3 * pG * Rd / R;                    /* d pG / dt */
    const double pinf_t = L->pinf + pA1 * sin(w1 * t) + pA2 * sin(w2 * t + theta);
    const double dpinf = pA1 * w1 * cos(w1 * t) + pA2 * w2 * cos(w2 * t + theta);
    /* p_L without the part of its derivative that contains R'' */
    const double pL = pG + L->pv - 2.0 * L->sigma / R - 4.0 * L->mu * Rd / R;
    /* d/dt p_L = dpG + 2 sigma R'/R^2 - 4 mu (R'' / R - R'^2 / R^2)
     *          = [dpG + 2 sigma R'/R^2 + 4 mu R'^2/R^2] - (4 mu / R) R''  */
    const double dpL_known = dpG + 2.0 * L->sigma * Rd / (R * R) + 4.0 * L->mu * Rd * Rd / (R * R);
    const double dpL_coef = -4.0 * L->mu / R;
    /* LHS: a R'' + b ;  RHS: e + (R/(rho c)) (dpL_known + dpL_coef R'' - dpinf) */
    const double a = (1.0 - Rd / L->c) * R;
    const double b = (1.0 - Rd / (3.0 * L->c)) * 1.5 * Rd * Rd;
    const double e = (1.0 + Rd / L->c) * (pL - pinf_t) / L->rho;
    const double k = R / (L->rho * L->c);
    /* a R'' + b = e + k (dpL_known - dpinf) + k dpL_coef R'' */
    return (e + k * (dpL_known - dpinf) - b) / (a - k * dpL_coef);
}

/* ------------------------------------------------------------------------- */
/* Classic RK4 (Sec. 3; Sec. 4.1)                                            */
/* ------------------------------------------------------------------------- */

/* One step: k1 = f(t,y); k2 = f(t+h/2, y+h/2 k1); k3 = f(t+h/2, y+h/2 k2);
 * k4 = f(t+h, y+h k3); y_new = y + h/6 (k1 + 2 k2 + 2 k3 + k4).            */
static void rk4_step(int sys, const double *p, int dim, double t, double h, const double *y,
                     double *out)
{
    double k1[ORC_MAXDIM], k2[ORC_MAXDIM], k3[ORC_MAXDIM], k4[ORC_MAXDIM];
    double ys[ORC_MAXDIM] = {0.0, 0.0, 0.0};
    rhs(sys, p, t, y, k1);
    for (int i = 0; i < dim; ++i) ys[i] = y[i] + (h / 2.0) * k1[i];
    rhs(sys, p, t + h / 2.0, ys, k2);
    for (int i = 0; i < dim; ++i) ys[i] = y[i] + (h / 2.0) * k2[i];
    rhs(sys, p, t + h / 2.0, ys, k3);
    for (int i = 0; i < dim; ++i) ys[i] = y[i] + h * k3[i];
    rhs(sys, p, t + h, ys, k4);
    for (int i = 0; i < dim; ++i)
        out[i] = y[i] + (h / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* single step for the pin tests (one system) */
void orc_rk4_step(int sys, const double *p, double t, double h, const double *y, double *out)
{
    rk4_step(sys, p, orc_dim(sys), t, h, y, out);
}

/* Fixed-step ensemble integration: every system takes nsteps steps of size dt
 * from t0; the time of step j is t0 + j dt.  y is SoA [dim][n], updated in place.
 * status[i] gets ORC_ST_NONFINITE if the final state is not finite.         */
void orc_rk4_solve(int sys, int64_t n, const double *params, double *y, double t0, double dt,
                   int64_t nsteps, int32_t *status, int nthreads)
{
    const int dim = orc_dim(sys), npar = orc_npar(sys);
#ifdef _OPENMP
    /* a per-call thread count that leaves the process-wide default alone */
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
#endif
    for (int64_t i = 0; i < n; ++i) {
        double p[16], yy[ORC_MAXDIM], yn[ORC_MAXDIM];
        int st = 0;
        for (int k = 0; k < npar; ++k) p[k] = params[k * n + i];
        for (int k = 0; k < dim; ++k) yy[k] = y[k * n + i];
        for (int64_t j = 0; j < nsteps; ++j) {
            rk4_step(sys, p, dim, t0 + (double)j * dt, dt, yy, yn);
            for (int k = 0; k < dim; ++k) yy[k] = yn[k];
        }
        for (int k = 0; k < dim; ++k) {
            y[k * n + i] = yy[k];
            if (!isfinite(yy[k])) st |= ORC_ST_NONFINITE;
        }
        if (status) status[i] = st;
    }
}

/* ------------------------------------------------------------------------- */
/* Cash-Karp embedded Runge-Kutta 4(5)                                       */
/* ------------------------------------------------------------------------- */

/* Cash & Karp (1990): nodes c, coupling a, fifth-order weights b (propagated)
 * and fourth-order weights bs (embedded estimate).                           */
static const double CK_c[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0};
static const double CK_a[6][5] = {
    {0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0 / 5.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 40.0, 9.0 / 40.0, 0.0, 0.0, 0.0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0.0, 0.0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0.0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0}};
static const double CK_b[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
static const double CK_bs[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0,
                                277.0 / 14336.0, 1.0 / 4.0};

/* Export of the tableau for the order-condition tests: c[6], a[36] row-major
 * (6x6, strictly lower), b[6], bs[6].                                        */
void orc_cashkarp_tableau(double *c, double *a, double *b, double *bs)
{
    for (int i = 0; i < 6; ++i) {
        c[i] = CK_c[i];
        b[i] = CK_b[i];
        bs[i] = CK_bs[i];
        for (int j = 0; j < 6; ++j) a[i * 6 + j] = (j < 5) ? CK_a[i][j] : 0.0;
    }
}

/* One Cash-Karp trial step from (t, y) with step h.  k1 = f(t, y) is passed in
 * (it does not change when a step is retried).  Stage i: k_i = f(t + c_i h,
 * y + h sum_j a_ij k_j).  y5 = y + h sum b_i k_i, and the error estimate is
 * the difference of the fifth- and fourth-order solutions written, as Cash &
 * Karp do, through the weight differences: err = h sum (b_i - bs_i) k_i
 * (the same quantity as y5 - y4 without the cancellation of forming both).  */
static void ck_step(int sys, const double *p, int dim, double t, double h, const double *y,
                    const double *k1, double *y5, double *err)
{
    double k[6][ORC_MAXDIM], ys[ORC_MAXDIM];
    for (int i = 0; i < dim; ++i) k[0][i] = k1[i];
    for (int s = 1; s < 6; ++s) {
        for (int i = 0; i < dim; ++i) {
            double acc = 0.0;
            for (int j = 0; j < s; ++j) acc = acc + CK_a[s][j] * k[j][i];
            ys[i] = y[i] + h * acc;
        }
        rhs(sys, p, t + CK_c[s] * h, ys, k[s]);
    }
    for (int i = 0; i < dim; ++i) {
        double s5 = 0.0, se = 0.0;
        for (int j = 0; j < 6; ++j) {
            s5 = s5 + CK_b[j] * k[j][i];
            se = se + (CK_b[j] - CK_bs[j]) * k[j][i];
        }
        y5[i] = y[i] + h * s5;
        err[i] = h * se;
    }
}

void orc_cashkarp_step(int sys, const double *p, double t, double h, const double *y, double *y5,
                       double *err)
{
    double k1[ORC_MAXDIM];
    const int dim = orc_dim(sys);
    rhs(sys, p, t, y, k1);
    ck_step(sys, p, dim, t, h, y, k1, y5, err);
}

/* ------------------------------------------------------------------------- */
/* Dormand-Prince embedded Runge-Kutta 5(4), "DOPRI5"                        */
/* ------------------------------------------------------------------------- */

/* Dormand & Prince (1980): seven stages, the seventh at c7 = 1 with coupling
 * row a7j = b_j, so that k7 = f(t + h, y5) ("first same as last": after an
 * accepted step k7 is the next step's k1).  Fifth-order weights b
 * (propagated), fourth-order weights bs (embedded estimate).  The solver of
 * the paper's Julia comparison runs (Sec. 4.2).                              */
static const double DP_c[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
static const double DP_a[7][6] = {
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0 / 5.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 40.0, 9.0 / 40.0, 0.0, 0.0, 0.0, 0.0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0.0, 0.0, 0.0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0.0, 0.0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0.0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
static const double DP_b[7] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0,
                               11.0 / 84.0, 0.0};
static const double DP_bs[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0,
                                -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};

/* Export of the tableau for the order-condition tests: c[7], a[49] row-major
 * (7x7, strictly lower), b[7], bs[7].                                        */
void orc_dopri5_tableau(double *c, double *a, double *b, double *bs)
{
    for (int i = 0; i < 7; ++i) {
        c[i] = DP_c[i];
        b[i] = DP_b[i];
        bs[i] = DP_bs[i];
        for (int j = 0; j < 7; ++j) a[i * 7 + j] = (j < 6) ? DP_a[i][j] : 0.0;
    }
}

/* One Dormand-Prince trial step from (t, y) with step h and k1 = f(t, y).
 * Stages 2..7 as for Cash-Karp; the seventh stage's state is y5 itself (its
 * coupling row is b), so y5 is that state and k7 = f(t + h, y5) is returned
 * for reuse.  err = h sum (b_i - bs_i) k_i over the seven stages.            */
static void dp_step(int sys, const double *p, int dim, double t, double h, const double *y,
                    const double *k1, double *y5, double *err, double *k7)
{
    double k[7][ORC_MAXDIM], ys[ORC_MAXDIM];
    for (int i = 0; i < dim; ++i) k[0][i] = k1[i];
    for (int s = 1; s < 7; ++s) {
        for (int i = 0; i < dim; ++i) {
            double acc = 0.0;
            for (int j = 0; j < s; ++j) acc = acc + DP_a[s][j] * k[j][i];
            ys[i] = y[i] + h * acc;
        }
        rhs(sys, p, t + DP_c[s] * h, ys, k[s]);
    }
    for (int i = 0; i < dim; ++i) {
        double se = 0.0;
        for (int j = 0; j < 7; ++j) se = se + (DP_b[j] - DP_bs[j]) * k[j][i];
        y5[i] = ys[i];
        err[i] = h * se;
        k7[i] = k[6][i];
    }
}

void orc_dopri5_step(int sys, const double *p, double t, double h, const double *y, double *y5,
                     double *err)
{
    double k1[ORC_MAXDIM], k7[ORC_MAXDIM];
    const int dim = orc_dim(sys);
    rhs(sys, p, t, y, k1);
    dp_step(sys, p, dim, t, h, y, k1, y5, err, k7);
}

/* ------------------------------------------------------------------------- */
/* Step-size controller (the paper gives tolerances only, Sec. 4.2.1; this
 * reading is the standard elementary controller for an order-4/5 pair):
 *   sc_i = atol + rtol * max(|y_i|, |y5_i|)
 *   E    = max_i |err_i| / sc_i                (max-norm)
 *   accept iff E <= 1
 *   fac  = 0.9 * E^(-1/5) clamped to [0.2, 5]; E == 0 gives 5; E not a
 *          number (overflowed trial) gives 0.2 and a rejection.             */
/* ------------------------------------------------------------------------- */

typedef struct {
    double rtol, atol;
    double dt0, dt_min, dt_max;
    double event_tol;
    int64_t max_steps;      /* cap on trial steps per system            */
    int32_t n_phases;       /* > 0: phase mode (Keller-Miksis)          */
    double phase_len;       /* phase length in tau                      */
    double t0, t1;          /* time span (event mode) / phase start     */
    double acc_t_start;     /* event mode: y1 minimum recorded for t >= */
    int32_t method;         /* ORC_CASHKARP or ORC_DOPRI5               */
} orc_tol;

enum { ORC_CASHKARP = 0, ORC_DOPRI5 = 1 };

/* One trial of the selected pair.  Returns the number of right-hand-side
 * evaluations it made; *k_next_valid tells whether k_next = f(t + h, y5)
 * (Dormand-Prince only).                                                     */
static int rk45_trial(const orc_tol *tol, int sys, const double *p, int dim, double t, double h,
                      const double *y, const double *k1, double *y5, double *err, double *k_next,
                      int *k_next_valid)
{
    if (tol->method == ORC_DOPRI5) {
        dp_step(sys, p, dim, t, h, y, k1, y5, err, k_next);
        *k_next_valid = 1;
        return 6;
    }
    ck_step(sys, p, dim, t, h, y, k1, y5, err);
    *k_next_valid = 0;
    return 5;
}

static double err_norm(int dim, const double *y, const double *y5, const double *err,
                       const orc_tol *tol)
{
    double E = 0.0;
    for (int i = 0; i < dim; ++i) {
        const double sc = tol->atol + tol->rtol * fmax(fabs(y[i]), fabs(y5[i]));
        const double r = fabs(err[i]) / sc;
        if (isnan(r)) return NAN;
        if (r > E) E = r;
    }
    return E;
}

static double step_factor(double E)
{
    double fac;
    if (isnan(E)) return 0.2;
    if (E == 0.0) return 5.0;
    fac = 0.9 * pow(E, -0.2);
    if (fac < 0.2) fac = 0.2;
    if (fac > 5.0) fac = 5.0;
    return fac;
}

/* Phase mode (Keller-Miksis, Sec. 4.2): n_phases integration phases, each over
 * tau in [t0, t0 + phase_len] with tau reset to t0 at the start of a phase
 * (the forcing is periodic with period 1).  After every accepted step (and at
 * the phase start) the running maximum and minimum of y1 are updated; at the
 * end of phase k, acc[(2k)*n + i] = max y1 and acc[(2k+1)*n + i] = min y1.
 * The step that would pass the phase end is shortened to end exactly on it;
 * when such a shortened step is accepted the step-size proposal dt is left as
 * it was, so the next phase starts from the unshortened proposal.  dt carries
 * over from phase to phase.  For ORC_KM_TAN the tangent vector (v1, v2) is
 * scaled to unit length at the start and at every phase end, and
 * acc[(2 n_phases + k)*n + i] = ln |v| at the end of phase k (its growth over
 * the phase): the mean of these rows over phases, divided by phase_len, is the
 * largest Lyapunov exponent (Benettin's renormalisation between phases, the
 * trajectory manipulation between phases that Sec. 1 describes).            */
static void solve_phased(int sys, const double *p, int dim, double *y, double *dt_io,
                         const orc_tol *tol, int64_t n, int64_t i, double *acc, int32_t *status,
                         int64_t *nacc, int64_t *nrej, int64_t *nrhs)
{
    double dt = *dt_io;
    double k1[ORC_MAXDIM], y5[ORC_MAXDIM], err[ORC_MAXDIM], kn[ORC_MAXDIM];
    int64_t trials = 0, acc_steps = 0, rej_steps = 0, rhs_evals = 0;
    int st = 0;
    const int tangent = sys == ORC_KM_TAN;
    if (tangent) {               /* the tangent vector starts at unit length */
        const double nv = hypot(y[2], y[3]);
        y[2] /= nv;
        y[3] /= nv;
    }
    for (int ph = 0; ph < tol->n_phases; ++ph) {
        const double tau_end = tol->t0 + tol->phase_len;
        double tau = tol->t0;
        double ymax = y[0], ymin = y[0];
        int k1_valid = 0;
        while (tau < tau_end && st == 0) {
            double h = dt, E, fac;
            int clamped = 0;
            if (trials >= tol->max_steps) { st |= ORC_ST_MAX_STEPS; break; }
            if (h >= tau_end - tau) { h = tau_end - tau; clamped = 1; }
            int kn_valid;
            if (!k1_valid) { rhs(sys, p, tau, y, k1); rhs_evals += 1; k1_valid = 1; }
            rhs_evals += rk45_trial(tol, sys, p, dim, tau, h, y, k1, y5, err, kn, &kn_valid);
            trials += 1;
            E = err_norm(dim, y, y5, err, tol);
            fac = step_factor(E);
            if (E <= 1.0) {
                tau = clamped ? tau_end : tau + h;
                for (int d = 0; d < dim; ++d) { y[d] = y5[d]; k1[d] = kn[d]; }
                /* Dormand-Prince: k1 of the next step is f(tau + h, y5); a
                 * phase end (the loop ends) restarts from f(t0, y)          */
                k1_valid = kn_valid;
                acc_steps += 1;
                if (y[0] > ymax) ymax = y[0];
                if (y[0] < ymin) ymin = y[0];
                if (!clamped) {
                    dt = h * fac;
                    if (dt > tol->dt_max) dt = tol->dt_max;
                    if (dt < tol->dt_min) dt = tol->dt_min;
                }
            } else {
                rej_steps += 1;
                dt = h * fac;
                if (dt < tol->dt_min) { st |= ORC_ST_DT_UNDERFLOW; break; }
            }
        }
        if (acc) {
            acc[(int64_t)(2 * ph) * n + i] = ymax;
            acc[(int64_t)(2 * ph + 1) * n + i] = ymin;
        }
        if (tangent) {
            /* renormalisation at the phase end (Benettin's method): the log of
             * the tangent vector's growth over this phase, then unit length */
            const double nv = hypot(y[2], y[3]);
            if (acc) acc[(int64_t)(2 * tol->n_phases + ph) * n + i] = st ? NAN : log(nv);
            y[2] /= nv;
            y[3] /= nv;
        }
        if (st) {
            for (int rest = ph + 1; rest < tol->n_phases && acc; ++rest) {
                acc[(int64_t)(2 * rest) * n + i] = NAN;
                acc[(int64_t)(2 * rest + 1) * n + i] = NAN;
                if (tangent) acc[(int64_t)(2 * tol->n_phases + rest) * n + i] = NAN;
            }
            break;
        }
    }
    *dt_io = dt;
    *status = st;
    *nacc = acc_steps;
    *nrej = rej_steps;
    *nrhs = rhs_evals;
}

/* Event mode (pressure relief valve, Sec. 4.3; also the bouncing-ball test
 * problem).  Two event functions, both falling:
 *   g1 = y1  (impact: the body reaches the seat moving towards it, y2 < 0),
 *   g2 = y2  (local maximum of y1: the Poincare section of Sec. 4.3).
 * Reading of the paper's event handling with a "corrected time step" and an
 * absolute event tolerance tol (Sec. 4.3.1), applied to every trial step that
 * passes the error test, with g0 = g(t) and g1 = g(t+h):
 *   - overshoot: the impact overshoots when g1 < -tol; the maximum overshoots
 *     when g0 > tol and g1 < -tol.  The trial is thrown away and retried with
 *     the step shortened to the earliest overshooting event's estimated
 *     root (one half of the step when the impact starts within the band,
 *     g0 <= tol, e.g. right after a bounce); at most 40 retries in a row.
 *     The root estimate (event_frac) is the root in (0, h) of the quadratic
 *     in s that takes the value g0 with slope g'(t) at s = 0 (g' = y2 for
 *     the impact and y2' for the maximum, both from k1 = f(t, y)) and the
 *     value g1 at s = h.
 *   - location: otherwise the trial is accepted, and at its end point the
 *     maximum is located when g0 > tol and |g1| <= tol, the impact when
 *     |g1| <= tol and y2 < 0.  Maximum: y1 is appended to the ring of the last
 *     32 Poincare points.  Impact (Eqs. impact_law_1-3): y1 <- 0,
 *     y2 <- -r y2, y3 unchanged.
 * Sticking (the paper is silent): a bounce whose apex stays inside the event
 * band cannot be resolved.  After an impact that leaves the upward speed v
 * with v^2 <= 2 a tol, where a = delta - y3 > 0 is the net force pressing the
 * body onto the seat, the body stays on the seat (y1 = y2 = 0) while the
 * pressure rises as y3' = beta q until y3 = delta; that interval is advanced
 * in closed form.
 * Accessories (acc SoA [35][n]): rows 0..31 ring of maxima (slot m mod 32
 * holds maximum number m, NaN if never written), row 32 the minimum of y1
 * over the accepted points with t >= acc_t_start, row 33 the number of maxima,
 * row 34 the number of impacts.                                              */
#define ORC_RING 32
#define ORC_EV_RETRIES 40

/* Fraction of the trial step at the estimated root of a falling event
 * function with g0 > 0 at its start (slope d0) and g1 < 0 at its end.
 * With B = d0 h and A = g1 - g0 - B the model g0 + B x + A x^2 (x = s/h)
 * changes sign once on (0, 1); its root there is 2 g0 / (-B + sqrt(B^2 -
 * 4 A g0)) whatever the sign of A (for A > 0 the smaller of two positive
 * roots, for A < 0 the positive one).  The chord fraction g0 / (g0 - g1)
 * stands in if rounding takes the quadratic's root out of (0, 1).  The
 * quadratic is exact for a constant second derivative, so a retry lands in
 * the band even at a grazing impact, where the chord from the fixed start
 * point of the retried step closes in only linearly.                        */
static double event_frac(double g0, double d0, double g1, double h)
{
    const double B = d0 * h;
    const double A = g1 - g0 - B;
    const double D = B * B - 4.0 * A * g0;
    const double chord = g0 / (g0 - g1);
    if (!(D >= 0.0)) return chord;
    const double den = -B + sqrt(D);
    const double x = 2.0 * g0 / den;
    return (den > 0.0 && x > 0.0 && x < 1.0) ? x : chord;
}
static void solve_events(int sys, const double *p, int dim, double *y, double *t_io,
                         double *dt_io, const orc_tol *tol, int64_t n, int64_t i, double *acc,
                         int32_t *status, int64_t *nacc, int64_t *nrej, int64_t *nrhs)
{
    const double r = p[sys == ORC_BALL ? 1 : 4];
    const double q = (sys == ORC_PRV) ? p[0] : 0.0;
    const double delta = (sys == ORC_PRV) ? p[2] : 0.0;
    const double beta = (sys == ORC_PRV) ? p[3] : 0.0;
    const double etol = tol->event_tol;
    double t = *t_io, dt = *dt_io, h_ev = 0.0;
    double k1[ORC_MAXDIM], y5[ORC_MAXDIM], err[ORC_MAXDIM], yold[ORC_MAXDIM], kn[ORC_MAXDIM];
    double ring[ORC_RING];
    double ymin = INFINITY;
    int64_t trials = 0, acc_steps = 0, rej_steps = 0, rhs_evals = 0, nmax = 0, nimp = 0;
    int st = 0, k1_valid = 0, ev_retries = 0, stuck = 0;
    for (int s = 0; s < ORC_RING; ++s) ring[s] = NAN;
    if (t >= tol->acc_t_start) ymin = y[0];
    while (t < tol->t1 && st == 0) {
        double h, E, fac, best_frac = 2.0;
        int limited = 0, overshoot = 0;
        if (stuck) {
            /* closed-form sticking interval: y1 = y2 = 0, y3' = beta q */
            const double t_lift = t + (delta - y[2]) / (beta * q);
            if (t_lift >= tol->t1) {
                y[2] = y[2] + beta * q * (tol->t1 - t);
                t = tol->t1;
            } else {
                y[2] = delta;
                t = t_lift;
                stuck = 0;
            }
            k1_valid = 0;
            if (t >= tol->acc_t_start && y[0] < ymin) ymin = y[0];
            continue;
        }
        if (trials >= tol->max_steps) { st |= ORC_ST_MAX_STEPS; break; }
        h = dt;
        if (h >= tol->t1 - t) { h = tol->t1 - t; limited = 1; }
        if (h_ev > 0.0 && h_ev < h) { h = h_ev; limited = 2; }
        int kn_valid;
        if (!k1_valid) { rhs(sys, p, t, y, k1); rhs_evals += 1; k1_valid = 1; }
        rhs_evals += rk45_trial(tol, sys, p, dim, t, h, y, k1, y5, err, kn, &kn_valid);
        trials += 1;
        E = err_norm(dim, y, y5, err, tol);
        fac = step_factor(E);
        if (!(E <= 1.0)) {
            rej_steps += 1;
            dt = h * fac;
            h_ev = 0.0;
            if (dt < tol->dt_min) { st |= ORC_ST_DT_UNDERFLOW; break; }
            continue;
        }
        /* overshoot test on the error-accepted trial */
        if (y5[0] < -etol) {                                   /* impact */
            const double frac = (y[0] > etol) ? event_frac(y[0], k1[0], y5[0], h) : 0.5;
            if (frac < best_frac) best_frac = frac;
            overshoot = 1;
        }
        if (y[1] > etol && y5[1] < -etol) {                    /* maximum */
            const double frac = event_frac(y[1], k1[1], y5[1], h);
            if (frac < best_frac) best_frac = frac;
            overshoot = 1;
        }
        if (overshoot) {
            ev_retries += 1;
            if (ev_retries > ORC_EV_RETRIES) { st |= ORC_ST_EVENT_NO_CONVERGE; break; }
            h_ev = h * best_frac;
            continue;
        }
        /* accept */
        for (int d = 0; d < dim; ++d) { yold[d] = y[d]; y[d] = y5[d]; k1[d] = kn[d]; }
        t = (limited == 1) ? tol->t1 : t + h;
        k1_valid = kn_valid;          /* Dormand-Prince: f(t + h, y5); cleared by an impact */
        acc_steps += 1;
        ev_retries = 0;
        h_ev = 0.0;
        if (!limited) {
            dt = h * fac;
            if (dt > tol->dt_max) dt = tol->dt_max;
            if (dt < tol->dt_min) dt = tol->dt_min;
        }
        /* events located at the end point */
        if (yold[1] > etol && fabs(y[1]) <= etol) {
            ring[nmax % ORC_RING] = y[0];
            nmax += 1;
        }
        if (fabs(y[0]) <= etol && y[1] < 0.0) {
            y[0] = 0.0;
            y[1] = -r * y[1];
            k1_valid = 0;
            nimp += 1;
            if (sys == ORC_PRV) {
                const double a = delta - y[2];
                if (a > 0.0 && y[1] * y[1] <= 2.0 * a * etol) {
                    y[1] = 0.0;
                    stuck = 1;
                }
            }
        }
        if (t >= tol->acc_t_start && y[0] < ymin) ymin = y[0];
    }
    if (acc) {
        for (int s = 0; s < ORC_RING; ++s) acc[(int64_t)s * n + i] = ring[s];
        acc[(int64_t)32 * n + i] = ymin;
        acc[(int64_t)33 * n + i] = (double)nmax;
        acc[(int64_t)34 * n + i] = (double)nimp;
    }
    *t_io = t;
    *dt_io = dt;
    *status = st;
    *nacc = acc_steps;
    *nrej = rej_steps;
    *nrhs = rhs_evals;
}

/* Adaptive ensemble solve with the pair tol->method selects (Cash-Karp or
 * Dormand-Prince).  Phase mode when tol->n_phases > 0 (the
 * Keller-Miksis runs), event mode for ORC_PRV / ORC_BALL, otherwise plain
 * integration over [t0, t1] (the same controller, no events).
 * y: SoA [dim][n] in/out.  t_out, dt_out: final time and step proposal per
 * system (may be NULL).  acc: accessories (layout per mode, may be NULL).
 * status / nacc / nrej / nrhs: per-system outputs (may be NULL).            */
void orc_cashkarp_solve(int sys, int64_t n, const double *params, double *y, const orc_tol *tol,
                        double *t_out, double *dt_out, double *acc, int32_t *status,
                        int64_t *nacc, int64_t *nrej, int64_t *nrhs, int nthreads)
{
    const int dim = orc_dim(sys), npar = orc_npar(sys);
#ifdef _OPENMP
    /* a per-call thread count that leaves the process-wide default alone */
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int64_t i = 0; i < n; ++i) {
        double p[16], yy[ORC_MAXDIM];
        double t = tol->t0, dt = tol->dt0;
        int32_t st = 0;
        int64_t a = 0, rj = 0, ev = 0;
        for (int k = 0; k < npar; ++k) p[k] = params[k * n + i];
        for (int k = 0; k < dim; ++k) yy[k] = y[k * n + i];
        if (tol->n_phases > 0) {
            solve_phased(sys, p, dim, yy, &dt, tol, n, i, acc, &st, &a, &rj, &ev);
            t = tol->t0 + tol->phase_len;
        } else if (sys == ORC_PRV || sys == ORC_BALL) {
            solve_events(sys, p, dim, yy, &t, &dt, tol, n, i, acc, &st, &a, &rj, &ev);
        } else {
            /* plain adaptive integration over [t0, t1]: one phase, no reset */
            orc_tol one = *tol;
            one.n_phases = 1;
            one.phase_len = tol->t1 - tol->t0;
            solve_phased(sys, p, dim, yy, &dt, &one, n, i, NULL, &st, &a, &rj, &ev);
            t = tol->t1;
        }
        for (int k = 0; k < dim; ++k) y[k * n + i] = yy[k];
        if (t_out) t_out[i] = t;
        if (dt_out) dt_out[i] = dt;
        if (status) status[i] = st;
        if (nacc) nacc[i] = a;
        if (nrej) nrej[i] = rj;
        if (nrhs) nrhs[i] = ev;
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * slpic_oracle.c -- plain, slow FP64 CPU statement of the speed-limited
 * particle-in-cell (SLPIC) step of Werner, Jenkins, Chap & Cary,
 * "Speeding Up Simulations By Slowing Down Particles" (arXiv 1511.08225).
 *
 * THIS IS TEST INFRASTRUCTURE.  It exists to check the CUDA library against
 * the paper.  Only the test suite, the package smoke check and the CPU-baseline
 * leg of the benchmark may load it; the product library never calls it, and it
 * shares no code, header, table or constant with the CUDA path.
 *
 * Everything here is written for readability, in FP64 (except the quantised
 * deposit rule, which is an FP32 integer-exact rule by definition), with no
 * blocking, fusion or reordering.  Each function cites the passage it follows.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared slpic_oracle.c -lm
 * (-ffp-contract=off is required: the quantised deposit rule fixes the
 * rounding of every FP32 operation, so no multiply-add may be fused.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "slpic_oracle.h"

/* ------------------------------------------------------------------------ */
/* Speed-limiting functions, Sec. II, Eq. (relativisticBeta) and            */
/* Eq. (heavisideBeta).  beta_kind ONE is plain PIC (beta == 1, Sec. II).   */
/* ------------------------------------------------------------------------ */
double orc_beta(int kind, double r, double v0)
{
    switch (kind) {
    case ORC_BETA_ONE:
        return 1.0;
    case ORC_BETA_HEAVISIDE:
        /* Theta(v0-|v|) + (v0/|v|) Theta(|v|-v0); at |v| == v0 both give 1 */
        return (r <= v0) ? 1.0 : v0 / r;
    case ORC_BETA_RELATIVISTIC:
        return v0 / sqrt(r * r + v0 * v0);
    default:
        return NAN;
    }
}

/* |u + a tau| : the particle speed after a velocity change a*tau.  During one
 * push E is frozen at E^n(x^n) (Appendix A, Eq. slpicIntegrationV), so the
 * velocity moves along the straight line u + a*tau, tau = int beta dt. */
static double speed_on_line(const double u[3], const double a[3], double tau)
{
    double x = u[0] + a[0] * tau, y = u[1] + a[1] * tau, z = u[2] + a[2] * tau;
    return sqrt(x * x + y * y + z * z);
}

/* dt/dtau = 1/beta(|u + a tau|) */
static double inv_beta_on_line(int kind, const double u[3], const double a[3],
                               double v0, double tau)
{
    return 1.0 / orc_beta(kind, speed_on_line(u, a, tau), v0);
}

/* ------------------------------------------------------------------------ */
/* Adaptive 5-point Gauss-Legendre quadrature of 1/beta along the line.      */
/* The nodes are the roots of the degree-5 Legendre polynomial.              */
/* ------------------------------------------------------------------------ */
static const double GL5_X[5] = {-0.90617984593866399280, -0.53846931010568309104,
                                0.0, 0.53846931010568309104, 0.90617984593866399280};
static const double GL5_W[5] = {0.23692688505618908751, 0.47862867049936646804,
                                0.56888888888888888889, 0.47862867049936646804,
                                0.23692688505618908751};

typedef struct {
    int kind;
    const double *u, *a;
    double v0;
} line_ctx;

static double gl5(const line_ctx *c, double lo, double hi)
{
    double h = 0.5 * (hi - lo), m = 0.5 * (hi + lo), s = 0.0;
    for (int i = 0; i < 5; ++i)
        s += GL5_W[i] * inv_beta_on_line(c->kind, c->u, c->a, c->v0, m + h * GL5_X[i]);
    return s * h;
}

static double gl5_adapt(const line_ctx *c, double lo, double hi, double whole,
                        double tol, int depth)
{
    double mid = 0.5 * (lo + hi);
    double l = gl5(c, lo, mid), r = gl5(c, mid, hi);
    if (depth >= 48 || fabs(l + r - whole) <= tol)
        return l + r;
    return gl5_adapt(c, lo, mid, l, 0.5 * tol, depth + 1) +
           gl5_adapt(c, mid, hi, r, 0.5 * tol, depth + 1);
}

/* t(tau_hi) - t(tau_lo) = int_{tau_lo}^{tau_hi} dtau / beta, to ~1e-15 relative */
static double time_between(const line_ctx *c, double lo, double hi)
{
    if (hi <= lo)
        return 0.0;
    double whole = gl5(c, lo, hi);
    double tol = 1e-15 * fabs(whole) + 1e-300;
    return gl5_adapt(c, lo, hi, whole, tol, 0);
}

static int cmp_double(const void *p, const void *q)
{
    double x = *(const double *)p, y = *(const double *)q;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------ */
/* The velocity integral of Appendix A, Eq. (slpicIntegrationV):            */
/*   tau* = int_{t^{n-1/2}}^{t^{n+1/2}} beta(|v(t)|) dt,                     */
/* with dv/dt = beta(|v|) a and a = (q/m) E^n(x^n) frozen over the step.    */
/* Because v(t) = u + a tau(t) with dtau/dt = beta(|u + a tau|) and beta>0,  */
/* t(tau) = int_0^tau dtau'/beta(|u + a tau'|) is increasing, and tau* is   */
/* the root of t(tau*) = dt.  t(tau) is evaluated by adaptive quadrature on  */
/* pieces split where 1/beta is not smooth: the Heaviside kinks             */
/* |u + a tau| = v0 and the speed minimum tau = -u.a/|a|^2.                  */
/* ------------------------------------------------------------------------ */
double orc_beta_integral(int kind, const double u[3], const double a[3], double dt,
                         double v0)
{
    double A = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    double C = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (kind == ORC_BETA_ONE)
        return dt;
    if (A == 0.0) /* v constant: tau* = beta(|u|) dt */
        return orc_beta(kind, sqrt(C), v0) * dt;
    double B = u[0] * a[0] + u[1] * a[1] + u[2] * a[2];

    /* tau* <= dt because dt/dtau = 1/beta >= 1 */
    if (kind == ORC_BETA_HEAVISIDE) {
        /* |u + a tau| is convex in tau: if both ends are at or below v0, beta
         * is 1 over the whole step and tau* = dt exactly. */
        double end = speed_on_line(u, a, dt);
        if (sqrt(C) <= v0 && end <= v0)
            return dt;
    }

    double brk[4];
    int nb = 0;
    brk[nb++] = 0.0;
    double tmin = -B / A;
    if (tmin > 0.0 && tmin < dt)
        brk[nb++] = tmin;
    if (kind == ORC_BETA_HEAVISIDE) {
        /* A tau^2 + 2 B tau + (C - v0^2) = 0 */
        double disc = B * B - A * (C - v0 * v0);
        if (disc > 0.0) {
            double sq = sqrt(disc);
            double r1 = (-B - sq) / A, r2 = (-B + sq) / A;
            if (r1 > 0.0 && r1 < dt)
                brk[nb++] = r1;
            if (r2 > 0.0 && r2 < dt)
                brk[nb++] = r2;
        }
    }
    qsort(brk, nb, sizeof(double), cmp_double);

    line_ctx c = {kind, u, a, v0};
    /* walk the pieces [brk[k], brk[k+1]] (the last one ends at dt) */
    double t_acc = 0.0;
    for (int k = 0; k < nb; ++k) {
        double lo = brk[k], hi = (k + 1 < nb) ? brk[k + 1] : dt;
        double t_piece = time_between(&c, lo, hi);
        if (t_acc + t_piece < dt && k + 1 < nb) {
            t_acc += t_piece;
            continue;
        }
        /* the root lies in [lo, hi]: safeguarded Newton on
         * f(tau) = t_acc + int_lo^tau 1/beta - dt, f' = 1/beta >= 1 */
        double target = dt - t_acc;
        double blo = lo, bhi = hi;
        double tau = lo + target; /* f' >= 1 => tau* <= lo + target */
        if (tau > hi)
            tau = hi;
        for (int it = 0; it < 200; ++it) {
            double f = time_between(&c, lo, tau) - target;
            if (f > 0.0)
                bhi = tau;
            else
                blo = tau;
            double step = f / inv_beta_on_line(kind, u, a, v0, tau);
            double nt = tau - step;
            if (!(nt > blo && nt < bhi))
                nt = 0.5 * (blo + bhi);
            if (fabs(nt - tau) <= 1e-16 * (fabs(tau) + dt) || bhi - blo <= 1e-16 * dt) {
                tau = nt;
                break;
            }
            tau = nt;
        }
        return tau;
    }
    return dt; /* not reached */
}

/* ------------------------------------------------------------------------ */
/* The paper's own evaluation of the same integral (Appendix A): the        */
/* modified midpoint method (Numerical Recipes), with the number of          */
/* substeps doubled until two successive values agree within rel_tol        */
/* (1e-2 in the paper).  The state integrated is tau, dtau/dt = beta(|u+a tau|). */
/* ------------------------------------------------------------------------ */
static double mmid_once(int kind, const double u[3], const double a[3], double dt,
                        double v0, long n)
{
    double h = dt / (double)n;
    double z0 = 0.0;
    double z1 = z0 + h * orc_beta(kind, speed_on_line(u, a, z0), v0);
    for (long m = 1; m < n; ++m) {
        double z2 = z0 + 2.0 * h * orc_beta(kind, speed_on_line(u, a, z1), v0);
        z0 = z1;
        z1 = z2;
    }
    return 0.5 * (z1 + z0 + h * orc_beta(kind, speed_on_line(u, a, z1), v0));
}

double orc_beta_integral_mmid(int kind, const double u[3], const double a[3], double dt,
                              double v0, double rel_tol, long *n_used)
{
    long n = 2;
    double prev = mmid_once(kind, u, a, dt, v0, 1);
    double cur = prev;
    for (; n <= (1L << 26); n *= 2) {
        cur = mmid_once(kind, u, a, dt, v0, n);
        if (fabs(cur - prev) <= rel_tol * fabs(cur))
            break;
        prev = cur;
    }
    if (n_used)
        *n_used = n;
    return cur;
}

/* ------------------------------------------------------------------------ */
/* Brute-force check of the same integral: classical RK4 on the equations   */
/* of motion of Sec. II, Eq. (LimPtclDyn), xdot = beta v, vdot = beta a,    */
/* with a fixed, plus Idot = beta for I = int beta dt.  n_sub fixed steps.   */
/* out[0..2] = v(dt), out[3..5] = x(dt) - x(0), out[6] = I(dt).             */
/* ------------------------------------------------------------------------ */
static void lim_rhs(int kind, const double a[3], double v0, const double y[7], double f[7])
{
    double r = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
    double b = orc_beta(kind, r, v0);
    for (int i = 0; i < 3; ++i) {
        f[i] = b * a[i];
        f[3 + i] = b * y[i];
    }
    f[6] = b;
}

void orc_rk4_limited(int kind, const double u[3], const double a[3], double dt, double v0,
                     long n_sub, double out[7])
{
    double y[7] = {u[0], u[1], u[2], 0, 0, 0, 0}, k1[7], k2[7], k3[7], k4[7], t[7];
    double h = dt / (double)n_sub;
    for (long s = 0; s < n_sub; ++s) {
        lim_rhs(kind, a, v0, y, k1);
        for (int i = 0; i < 7; ++i) t[i] = y[i] + 0.5 * h * k1[i];
        lim_rhs(kind, a, v0, t, k2);
        for (int i = 0; i < 7; ++i) t[i] = y[i] + 0.5 * h * k2[i];
        lim_rhs(kind, a, v0, t, k3);
        for (int i = 0; i < 7; ++i) t[i] = y[i] + h * k3[i];
        lim_rhs(kind, a, v0, t, k4);
        for (int i = 0; i < 7; ++i)
            y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    memcpy(out, y, sizeof(y));
}

/* ------------------------------------------------------------------------ */
/* Poisson's equation of Appendix A, Eq. (LimPtclDynAppendixDotE), 1D,      */
/* nodal, second-order stencil:                                              */
/*   -(phi_{j+1} - 2 phi_j + phi_{j-1}) / dx^2 = rho_j / eps0.              */
/* ------------------------------------------------------------------------ */

/* Dirichlet: nodes 0..N, phi_0 = phi_lo, phi_N = phi_hi; textbook Thomas
 * algorithm on the N-1 interior unknowns (Sec. IV: plates at fixed potential). */
void orc_poisson1d_dirichlet(int n_cells, double dx, double eps0, const double *rho,
                             double phi_lo, double phi_hi, double *phi)
{
    int N = n_cells;
    phi[0] = phi_lo;
    phi[N] = phi_hi;
    if (N < 2)
        return;
    int m = N - 1; /* unknowns phi_1..phi_{N-1} */
    double *cp = (double *)malloc(sizeof(double) * m);
    double *dp = (double *)malloc(sizeof(double) * m);
    /* row i (node j = i+1): -phi_{j-1} + 2 phi_j - phi_{j+1} = dx^2 rho_j / eps0 */
    for (int i = 0; i < m; ++i) {
        int j = i + 1;
        double d = dx * dx * rho[j] / eps0;
        if (j == 1)
            d += phi_lo;
        if (j == N - 1)
            d += phi_hi;
        double a = (i == 0) ? 0.0 : -1.0, b = 2.0, c = (i == m - 1) ? 0.0 : -1.0;
        if (i == 0) {
            cp[i] = c / b;
            dp[i] = d / b;
        } else {
            double den = b - a * cp[i - 1];
            cp[i] = c / den;
            dp[i] = (d - a * dp[i - 1]) / den;
        }
    }
    phi[m] = dp[m - 1];
    for (int i = m - 2; i >= 0; --i)
        phi[i + 1] = dp[i] - cp[i] * phi[i + 2];
    free(cp);
    free(dp);
}

/* Periodic: nodes 0..N-1 (node N is node 0).  The equation is solvable only
 * for zero-mean rho, so the mean is removed (a uniform neutralising
 * background); phi is then fixed by phi_0 = 0 and the rows j = 1..N-1,
 * which form the same tridiagonal system as above with zero ends; row 0
 * then holds because all rows sum to zero.  Gauge: mean(phi) = 0. */
void orc_poisson1d_periodic(int n_cells, double dx, double eps0, const double *rho,
                            double *phi)
{
    int N = n_cells;
    double mean = 0.0;
    for (int j = 0; j < N; ++j)
        mean += rho[j];
    mean /= (double)N;
    double *r = (double *)malloc(sizeof(double) * (N + 1));
    double *p = (double *)malloc(sizeof(double) * (N + 1));
    for (int j = 0; j < N; ++j)
        r[j] = rho[j] - mean;
    r[N] = r[0];
    orc_poisson1d_dirichlet(N, dx, eps0, r, 0.0, 0.0, p);
    double pm = 0.0;
    for (int j = 0; j < N; ++j)
        pm += p[j];
    pm /= (double)N;
    for (int j = 0; j < N; ++j)
        phi[j] = p[j] - pm;
    free(r);
    free(p);
}

/* Nodal E = -dphi/dx: centred difference inside (and everywhere on a periodic
 * grid), one-sided at Dirichlet wall nodes. */
void orc_efield1d(int n_cells, int periodic, double dx, const double *phi, double *E)
{
    int N = n_cells;
    if (periodic) {
        for (int j = 0; j < N; ++j) {
            int jp = (j + 1) % N, jm = (j + N - 1) % N;
            E[j] = -(phi[jp] - phi[jm]) / (2.0 * dx);
        }
        return;
    }
    for (int j = 1; j < N; ++j)
        E[j] = -(phi[j + 1] - phi[j - 1]) / (2.0 * dx);
    E[0] = -(phi[1] - phi[0]) / dx;
    E[N] = -(phi[N] - phi[N - 1]) / dx;
}

/* ------------------------------------------------------------------------ */
/* A speed limit that varies in space (Sec. II: beta, and so v0, may depend */
/* on position).  Reading: one factor lam[c] > 0 per cell, shared by the    */
/* species, so that the limit of a particle in cell c is v0 lam[c]; with    */
/* lam NULL the limit is v0 everywhere.  beta(x, v) is evaluated where the  */
/* particle is: the push of a step takes the limit of the cell it starts    */
/* the step in (where E is gathered), the charge assignment the limit of    */
/* the cell it is deposited from.                                           */
/* ------------------------------------------------------------------------ */
static double v0_at(double v0, const double *lam, int c)
{
    return lam ? v0 * lam[c] : v0;
}

/* ------------------------------------------------------------------------ */
/* Charge assignment, Appendix A: rho^{n+1} = sum_p w_p beta(|v^{n+1/2}|)    */
/* S(x - x_p^{n+1}), with linear (cloud-in-cell) S as the PIC scatter of    */
/* Sec. II.  Output: number density n_j += w beta S_j / dx (the caller      */
/* multiplies by the species charge).                                       */
/* ------------------------------------------------------------------------ */
void orc_deposit1d(int n_cells, int periodic, double dx, long n, const double *x,
                   const double *v, const uint8_t *alive, int kind, double v0,
                   const double *lam, double w, double *dens)
{
    int N = n_cells;
    for (long p = 0; p < n; ++p) {
        if (alive && !alive[p])
            continue;
        double xi = x[p] / dx;
        double cf = floor(xi);
        int c = (int)cf;
        double d = xi - cf;
        double r = sqrt(v[3 * p] * v[3 * p] + v[3 * p + 1] * v[3 * p + 1] +
                        v[3 * p + 2] * v[3 * p + 2]);
        double b = orc_beta(kind, r, v0_at(v0, lam, c));
        int c1 = periodic ? (c + 1) % N : c + 1;
        dens[c] += w * b * (1.0 - d) / dx;
        dens[c1] += w * b * d / dx;
    }
}

/* ------------------------------------------------------------------------ */
/* The quantised deposit rule.  The paper fixes no deposit precision; this  */
/* rule fixes one so that any two programs that agree on the FP32 particle  */
/* state (cell c, offset d in [0,1), v) agree on the charge bit for bit:    */
/*   s2 = (vx*vx + vy*vy) + vz*vz          (FP32, round-to-nearest each op) */
/*   beta: ONE 1; HEAVISIDE sqrt(s2) <= v0 ? 1 : v0/sqrt(s2);              */
/*         RELATIVISTIC v0 / sqrt(s2 + v0*v0)   (IEEE sqrt and division)    */
/*   qT = rint(beta * 2^40), qR = rint((beta*d) * 2^40), qL = qT - qR       */
/*   acc[c] += qL, acc[c+1 (mod N if periodic)] += qR   (int64)             */
/* Integer sums are exact and order-free, so sum_j acc_j = sum_p qT_p.       */
/* With a per-cell factor lam (FP32), the limit in cell c is the FP32        */
/* product v0 * lam[c], rounded to nearest.                                  */
/* ------------------------------------------------------------------------ */
float orc_beta_f32(int kind, float vx, float vy, float vz, float v0)
{
    float s2 = (vx * vx + vy * vy) + vz * vz;
    if (kind == ORC_BETA_ONE)
        return 1.0f;
    if (kind == ORC_BETA_HEAVISIDE) {
        float r = sqrtf(s2);
        return (r <= v0) ? 1.0f : v0 / r;
    }
    return v0 / sqrtf(s2 + v0 * v0);
}

void orc_deposit_q40(int n_cells, int periodic, long n, const int32_t *cell,
                     const float *offset, const float *v, int kind, float v0,
                     const float *lam, int64_t *acc)
{
    int N = n_cells;
    const float scale = 1099511627776.0f; /* 2^40 */
    for (long p = 0; p < n; ++p) {
        int c = cell[p];
        if (c < 0)
            continue;
        float v0c = lam ? v0 * lam[c] : v0;
        float b = orc_beta_f32(kind, v[3 * p], v[3 * p + 1], v[3 * p + 2], v0c);
        float bd = b * offset[p];
        int64_t qR = llrintf(bd * scale);
        int64_t qT = llrintf(b * scale);
        int c1 = periodic ? (c + 1) % N : c + 1;
        acc[c] += qT - qR;
        acc[c1] += qR;
    }
}

/* ------------------------------------------------------------------------ */
/* Gather + push + move + walls for one species, Appendix A,                */
/* Eq. (slpicIntegration):                                                   */
/*   v^{n+1/2} = v^{n-1/2} + (q/m) E^n(x^n) tau*,                           */
/*   x^{n+1}   = x^n + beta(|v^{n+1/2}|) v^{n+1/2} dt,                      */
/* with E gathered by linear interpolation of the nodal field (Sec. II).   */
/* Walls (Sec. IV): a particle with x < 0 or x >= L is absorbed; on a      */
/* periodic grid x wraps into [0, L).                                       */
/* alive[p]: in/out.  flux[0] / flux[1] count absorptions at x=0 / x=L.    */
/* lam: per-cell factors of v0 (see v0_at) or NULL; both the integral and   */
/* the move take the limit of the cell the particle starts the step in.     */
/* ------------------------------------------------------------------------ */
void orc_push1d(int n_cells, int periodic, double dx, double dt, const double *E, long n,
                double *x, double *v, uint8_t *alive, double qm, int kind, double v0,
                const double *lam, long *flux)
{
    int N = n_cells;
    double L = dx * N;
    for (long p = 0; p < n; ++p) {
        if (!alive[p])
            continue;
        double xi = x[p] / dx;
        double cf = floor(xi);
        int c = (int)cf;
        double d = xi - cf;
        int c1 = periodic ? (c + 1) % N : c + 1;
        double Ep = (1.0 - d) * E[c] + d * E[c1];
        double a[3] = {qm * Ep, 0.0, 0.0};
        double *vp = v + 3 * p;
        double v0p = v0_at(v0, lam, c);
        double tau = orc_beta_integral(kind, vp, a, dt, v0p);
        for (int i = 0; i < 3; ++i)
            vp[i] += a[i] * tau;
        double r = sqrt(vp[0] * vp[0] + vp[1] * vp[1] + vp[2] * vp[2]);
        double b = orc_beta(kind, r, v0p);
        double xn = x[p] + b * vp[0] * dt;
        if (periodic) {
            xn -= L * floor(xn / L);
            if (xn >= L)
                xn -= L;
        } else if (xn < 0.0) {
            alive[p] = 0;
            flux[0] += 1;
        } else if (xn >= L) {
            alive[p] = 0;
            flux[1] += 1;
        }
        x[p] = xn;
    }
}

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; the generator behind       */
/* java.util.SplittableRandom), used counter-style: the i-th output of the  */
/* generator seeded with `key`.  Used for source injection.                 */
/* ------------------------------------------------------------------------ */
static uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64_at(uint64_t key, uint64_t i)
{
    return sm64_mix(key + (i + 1) * 0x9E3779B97F4A7C15ULL);
}

/* stream key for (seed, step, species) */
uint64_t orc_stream_key(uint64_t seed, uint64_t step, uint32_t species)
{
    return sm64_mix(seed ^ sm64_mix(step * 16ULL + species + 1ULL));
}

/* uniform on (0, 1], 24 bits, exactly representable in FP32 */
float orc_u24(uint64_t z) { return (float)((z >> 40) + 1ULL) * (1.0f / 16777216.0f); }

/* ------------------------------------------------------------------------ */
/* Volume source (Sec. IV injects "as if from a stationary plasma"; the     */
/* configured reading is a central source band).  Macroparticle k of this   */
/* step and species takes uniforms u_j = u24(SplitMix64(key, 8k + j)):      */
/*   position (cell units, FP32): xc = lo + u_0 * len                       */
/*   velocity: Box-Muller pairs (u_1,u_2) -> (vx,vy), (u_3,u_4) -> vz,      */
/*   scaled by sqrt(T/m): a physical (f) Maxwellian, because with the       */
/*   approximation of Eq. (ConservSpeedLimApprox) a source term of the f    */
/*   equation enters the g equation unchanged.                              */
/* Writes x (FP64, = xc*dx) and v (FP64) of n_new particles.                */
/* ------------------------------------------------------------------------ */
void orc_inject(uint64_t seed, uint64_t step, uint32_t species, long n_new,
                float src_lo_cells, float src_len_cells, double dx, double vth,
                double *x, double *v)
{
    const double two_pi = 6.283185307179586476925286766559;
    uint64_t key = orc_stream_key(seed, step, species);
    for (long k = 0; k < n_new; ++k) {
        float u0 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 0));
        double u1 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 1));
        double u2 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 2));
        double u3 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 3));
        double u4 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 4));
        float xc = src_lo_cells + u0 * src_len_cells;
        x[k] = (double)xc * dx;
        double r1 = sqrt(-2.0 * log(u1)), r2 = sqrt(-2.0 * log(u3));
        v[3 * k + 0] = vth * r1 * cos(two_pi * u2);
        v[3 * k + 1] = vth * r1 * sin(two_pi * u2);
        v[3 * k + 2] = vth * r2 * cos(two_pi * u4);
    }
}

/* ------------------------------------------------------------------------ */
/* Closed-form time along the line, used only to pin orc_beta_integral.     */
/* With w the velocity component along a (w = u.a/|a| + |a| tau) and       */
/* D = |u|^2 - (u.a)^2/|a|^2, the speed is sqrt(w^2 + D) and                */
/*   t(tau) = [H(w(tau)) - H(w(0))] / |a|,   H(w) = int_0^w dw'/beta,       */
/* with int sqrt(w^2+D) dw = (w sqrt(w^2+D) + D asinh(w/sqrt(D)))/2.        */
/* ------------------------------------------------------------------------ */
static double F_sqrt(double w, double D)
{
    if (D <= 0.0)
        return 0.5 * w * fabs(w);
    return 0.5 * (w * sqrt(w * w + D) + D * asinh(w / sqrt(D)));
}

static double H_closed(int kind, double w, double D, double v0)
{
    double s = (w < 0.0) ? -1.0 : 1.0, aw = fabs(w);
    if (kind == ORC_BETA_ONE)
        return w;
    if (kind == ORC_BETA_RELATIVISTIC)
        return F_sqrt(w, D + v0 * v0) / v0;
    /* Heaviside */
    if (D < v0 * v0) {
        double W0 = sqrt(v0 * v0 - D);
        if (aw <= W0)
            return w;
        return s * (W0 + (F_sqrt(aw, D) - F_sqrt(W0, D)) / v0);
    }
    return F_sqrt(w, D) / v0;
}

double orc_time_closed(int kind, const double u[3], const double a[3], double v0,
                       double tau)
{
    double A = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    double C = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (A == 0.0)
        return tau / orc_beta(kind, sqrt(C), v0);
    double w0 = (u[0] * a[0] + u[1] * a[1] + u[2] * a[2]) / A;
    double D = C - w0 * w0;
    if (D < 0.0)
        D = 0.0;
    return (H_closed(kind, w0 + A * tau, D, v0) - H_closed(kind, w0, D, v0)) / A;
}

/* bisection on the closed form: an independent route to tau* */
double orc_beta_integral_closed(int kind, const double u[3], const double a[3], double dt,
                                double v0)
{
    double lo = 0.0, hi = dt;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (orc_time_closed(kind, u, a, v0, mid) < dt)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ======================================================================== */
/* 2D electrostatic SLPIC (2D3V), the same method on a rectangular grid:    */
/* periodic in x, absorbing plates at fixed potential in y (Sec. IV walls). */
/* Nodes (i, j), i = 0..nx-1 (node nx is node 0), j = 0..ny; node (i, j) is */
/* entry j*nx + i.  Cell size dx in both directions.                        */
/* ======================================================================== */

/* Poisson, Appendix A Eq. (LimPtclDynAppendixDotE) with the 5-point        */
/* stencil: -(sum of the 4 neighbours - 4 phi_ij)/dx^2 = rho_ij/eps0 on     */
/* rows j = 1..ny-1; phi_{i,0} = phi_lo, phi_{i,ny} = phi_hi.               */
/* Direct solve, written for checking rather than speed: a plain DFT in x   */
/* turns the system into one tridiagonal system in y per Fourier mode k,    */
/*   -P_{j-1} + (2 + lambda_k) P_j - P_{j+1} = dx^2 R_j / eps0,            */
/*   lambda_k = 4 sin^2(pi k / nx),                                         */
/* each solved by the Thomas algorithm; then the inverse DFT.               */
static void thomas_const(int m, double diag, const double *d, double *x)
{
    /* -x_{i-1} + diag x_i - x_{i+1} = d_i, i = 0..m-1, x_{-1} = x_m = 0 */
    if (m <= 0)
        return;
    double *cp = (double *)malloc(sizeof(double) * m);
    double *dp = (double *)malloc(sizeof(double) * m);
    for (int i = 0; i < m; ++i) {
        double den = (i == 0) ? diag : diag + cp[i - 1];
        cp[i] = -1.0 / den;
        dp[i] = (i == 0) ? d[i] / den : (d[i] + dp[i - 1]) / den;
    }
    x[m - 1] = dp[m - 1];
    for (int i = m - 2; i >= 0; --i)
        x[i] = dp[i] - cp[i] * x[i + 1];
    free(cp);
    free(dp);
}

void orc_poisson2d_direct(int nx, int ny, double dx, double eps0, const double *rho,
                          double phi_lo, double phi_hi, double *phi)
{
    const double two_pi = 6.283185307179586476925286766559;
    int m = ny - 1; /* unknown rows j = 1..ny-1 */
    double *cs = (double *)malloc(sizeof(double) * nx);
    double *sn = (double *)malloc(sizeof(double) * nx);
    for (int t = 0; t < nx; ++t) {
        cs[t] = cos(two_pi * t / nx);
        sn[t] = sin(two_pi * t / nx);
    }
    /* cosine and sine transforms of the right-hand side, per mode k and row */
    double *ra = (double *)calloc((size_t)nx * m, sizeof(double));
    double *rb = (double *)calloc((size_t)nx * m, sizeof(double));
    for (int r = 0; r < m; ++r) {
        int j = r + 1;
        for (int k = 0; k < nx; ++k) {
            double a = 0.0, b = 0.0;
            for (int i = 0; i < nx; ++i) {
                double f = dx * dx * rho[(size_t)j * nx + i] / eps0;
                int t = (int)(((long)k * i) % nx);
                a += f * cs[t];
                b += f * sn[t];
            }
            /* boundary rows: constant in x, so only mode 0 sees them */
            if (k == 0) {
                if (j == 1)
                    a += nx * phi_lo;
                if (j == ny - 1)
                    a += nx * phi_hi;
            }
            ra[(size_t)k * m + r] = a;
            rb[(size_t)k * m + r] = b;
        }
    }
    double *pa = (double *)malloc(sizeof(double) * (size_t)nx * m);
    double *pb = (double *)malloc(sizeof(double) * (size_t)nx * m);
    for (int k = 0; k < nx; ++k) {
        double s = sin(0.5 * two_pi * k / nx);
        double diag = 2.0 + 4.0 * s * s;
        thomas_const(m, diag, ra + (size_t)k * m, pa + (size_t)k * m);
        thomas_const(m, diag, rb + (size_t)k * m, pb + (size_t)k * m);
    }
    for (int i = 0; i < nx; ++i) {
        phi[i] = phi_lo;
        phi[(size_t)ny * nx + i] = phi_hi;
    }
    for (int r = 0; r < m; ++r) {
        int j = r + 1;
        for (int i = 0; i < nx; ++i) {
            double f = 0.0;
            for (int k = 0; k < nx; ++k) {
                int t = (int)(((long)k * i) % nx);
                f += pa[(size_t)k * m + r] * cs[t] + pb[(size_t)k * m + r] * sn[t];
            }
            phi[(size_t)j * nx + i] = f / nx;
        }
    }
    free(cs);
    free(sn);
    free(ra);
    free(rb);
    free(pa);
    free(pb);
}

/* The same system solved by conjugate gradients with the Jacobi (diagonal) */
/* preconditioner, FP64, from the initial guess in phi (its rows 1..ny-1),  */
/* until ||b - A phi||_2 <= rtol ||b||_2 or maxit iterations.  A is the    */
/* stencil scaled by dx^2 (diagonal 4), b = dx^2 rho/eps0 plus the plates'  */
/* potentials on rows 1 and ny-1.  Returns the iterations used (-1 if not  */
/* converged); *rel_res gets the final relative residual.  The paper names */
/* no 2D solver; this is the textbook preconditioned CG.                   */
static void apply_A(int nx, int ny, const double *u, double *out)
{
    /* u, out: rows 1..ny-1 stored as r = j-1; rows 0 and ny are zero */
    int m = ny - 1;
    for (int r = 0; r < m; ++r)
        for (int i = 0; i < nx; ++i) {
            int ip = (i + 1) % nx, im = (i + nx - 1) % nx;
            double s = u[(size_t)r * nx + ip] + u[(size_t)r * nx + im];
            if (r > 0)
                s += u[(size_t)(r - 1) * nx + i];
            if (r < m - 1)
                s += u[(size_t)(r + 1) * nx + i];
            out[(size_t)r * nx + i] = 4.0 * u[(size_t)r * nx + i] - s;
        }
}

static double dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i)
        s += a[i] * b[i];
    return s;
}

int orc_poisson2d_cg(int nx, int ny, double dx, double eps0, const double *rho,
                     double phi_lo, double phi_hi, double rtol, int maxit, double *phi,
                     double *rel_res)
{
    int m = ny - 1;
    long n = (long)nx * m;
    double *b = (double *)malloc(sizeof(double) * n);
    double *x = (double *)malloc(sizeof(double) * n);
    double *r = (double *)malloc(sizeof(double) * n);
    double *z = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *q = (double *)malloc(sizeof(double) * n);
    for (int rr = 0; rr < m; ++rr)
        for (int i = 0; i < nx; ++i) {
            int j = rr + 1;
            double v = dx * dx * rho[(size_t)j * nx + i] / eps0;
            if (j == 1)
                v += phi_lo;
            if (j == ny - 1)
                v += phi_hi;
            b[(size_t)rr * nx + i] = v;
            x[(size_t)rr * nx + i] = phi[(size_t)j * nx + i];
        }
    apply_A(nx, ny, x, q);
    for (long k = 0; k < n; ++k)
        r[k] = b[k] - q[k];
    double bn = sqrt(dot(n, b, b));
    if (bn == 0.0)
        bn = 1.0;
    int it = 0, done = 0;
    double res = sqrt(dot(n, r, r)) / bn;
    if (res <= rtol)
        done = 1;
    for (long k = 0; k < n; ++k) {
        z[k] = r[k] / 4.0; /* Jacobi: the diagonal of A is 4 */
        p[k] = z[k];
    }
    double rz = dot(n, r, z);
    while (!done && it < maxit) {
        apply_A(nx, ny, p, q);
        double alpha = rz / dot(n, p, q);
        for (long k = 0; k < n; ++k) {
            x[k] += alpha * p[k];
            r[k] -= alpha * q[k];
        }
        ++it;
        res = sqrt(dot(n, r, r)) / bn;
        if (res <= rtol) {
            done = 1;
            break;
        }
        for (long k = 0; k < n; ++k)
            z[k] = r[k] / 4.0;
        double rz1 = dot(n, r, z);
        double beta = rz1 / rz;
        rz = rz1;
        for (long k = 0; k < n; ++k)
            p[k] = z[k] + beta * p[k];
    }
    for (int i = 0; i < nx; ++i) {
        phi[i] = phi_lo;
        phi[(size_t)ny * nx + i] = phi_hi;
    }
    for (int rr = 0; rr < m; ++rr)
        for (int i = 0; i < nx; ++i)
            phi[(size_t)(rr + 1) * nx + i] = x[(size_t)rr * nx + i];
    if (rel_res)
        *rel_res = res;
    free(b);
    free(x);
    free(r);
    free(z);
    free(p);
    free(q);
    return done ? it : -1;
}

/* Nodal E = -grad phi: centred differences (periodic in x), one-sided at   */
/* the plates in y.                                                          */
void orc_efield2d(int nx, int ny, double dx, const double *phi, double *Ex, double *Ey)
{
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = (size_t)j * nx + i;
            int ip = (i + 1) % nx, im = (i + nx - 1) % nx;
            Ex[k] = -(phi[(size_t)j * nx + ip] - phi[(size_t)j * nx + im]) / (2.0 * dx);
            if (j == 0)
                Ey[k] = -(phi[k + nx] - phi[k]) / dx;
            else if (j == ny)
                Ey[k] = -(phi[k] - phi[k - nx]) / dx;
            else
                Ey[k] = -(phi[k + nx] - phi[k - nx]) / (2.0 * dx);
        }
}

/* Bilinear (area) charge assignment, the 2D form of the Appendix A deposit: */
/* number density w beta S / dx^2 on the 4 nodes of the particle's cell.    */
void orc_deposit2d(int nx, int ny, double dx, long n, const double *x, const double *y,
                   const double *v, const uint8_t *alive, int kind, double v0, double w,
                   double *dens)
{
    (void)ny;
    for (long p = 0; p < n; ++p) {
        if (alive && !alive[p])
            continue;
        double xi = x[p] / dx, yi = y[p] / dx;
        int cx = (int)floor(xi), cy = (int)floor(yi);
        double fx = xi - cx, fy = yi - cy;
        double r = sqrt(v[3 * p] * v[3 * p] + v[3 * p + 1] * v[3 * p + 1] +
                        v[3 * p + 2] * v[3 * p + 2]);
        double q = w * orc_beta(kind, r, v0) / (dx * dx);
        int cx1 = (cx + 1) % nx;
        dens[(size_t)cy * nx + cx] += q * (1.0 - fx) * (1.0 - fy);
        dens[(size_t)cy * nx + cx1] += q * fx * (1.0 - fy);
        dens[(size_t)(cy + 1) * nx + cx] += q * (1.0 - fx) * fy;
        dens[(size_t)(cy + 1) * nx + cx1] += q * fx * fy;
    }
}

/* The quantised deposit rule in 2D: with beta as in orc_beta_f32 and FP32   */
/* offsets (dx_, dy_) in [0,1), round-to-nearest each FP32 operation:        */
/*   qT = rint(beta 2^40), qX = rint((beta dx_) 2^40), qY = rint((beta dy_) 2^40), */
/*   qXY = rint(((beta dx_) dy_) 2^40);                                      */
/*   node (c+1, c+1) += qXY, (c+1, c) += qX - qXY, (c, c+1) += qY - qXY,    */
/*   (c, c) += qT - qX - qY + qXY          (int64; the four sum to qT).     */
/* cell = cy*nx + cx; offsets interleaved (dx_, dy_) per particle.           */
void orc_deposit2d_q40(int nx, int ny, long n, const int32_t *cell, const float *offset,
                       const float *v, int kind, float v0, int64_t *acc)
{
    (void)ny;
    const float scale = 1099511627776.0f; /* 2^40 */
    for (long p = 0; p < n; ++p) {
        int c = cell[p];
        if (c < 0)
            continue;
        int cx = c % nx, cy = c / nx;
        float b = orc_beta_f32(kind, v[3 * p], v[3 * p + 1], v[3 * p + 2], v0);
        float bx = b * offset[2 * p];
        float by = b * offset[2 * p + 1];
        float bxy = bx * offset[2 * p + 1];
        int64_t qT = llrintf(b * scale), qX = llrintf(bx * scale);
        int64_t qY = llrintf(by * scale), qXY = llrintf(bxy * scale);
        int cx1 = (cx + 1) % nx;
        acc[(size_t)cy * nx + cx] += qT - qX - qY + qXY;
        acc[(size_t)cy * nx + cx1] += qX - qXY;
        acc[(size_t)(cy + 1) * nx + cx] += qY - qXY;
        acc[(size_t)(cy + 1) * nx + cx1] += qXY;
    }
}

/* Gather + push + move + walls, 2D: bilinear E at the particle, then        */
/* Eq. (slpicIntegration) with a = (q/m)(Ex, Ey, 0); x wraps, a particle    */
/* with y < 0 or y >= Ly is absorbed (flux[0] / flux[1]).                   */
void orc_push2d(int nx, int ny, double dx, double dt, const double *Ex, const double *Ey,
                long n, double *x, double *y, double *v, uint8_t *alive, double qm, int kind,
                double v0, long *flux)
{
    double Lx = dx * nx, Ly = dx * ny;
    for (long p = 0; p < n; ++p) {
        if (!alive[p])
            continue;
        double xi = x[p] / dx, yi = y[p] / dx;
        int cx = (int)floor(xi), cy = (int)floor(yi);
        double fx = xi - cx, fy = yi - cy;
        int cx1 = (cx + 1) % nx;
        size_t k00 = (size_t)cy * nx + cx, k10 = (size_t)cy * nx + cx1;
        size_t k01 = (size_t)(cy + 1) * nx + cx, k11 = (size_t)(cy + 1) * nx + cx1;
        double w00 = (1.0 - fx) * (1.0 - fy), w10 = fx * (1.0 - fy);
        double w01 = (1.0 - fx) * fy, w11 = fx * fy;
        double ex = w00 * Ex[k00] + w10 * Ex[k10] + w01 * Ex[k01] + w11 * Ex[k11];
        double ey = w00 * Ey[k00] + w10 * Ey[k10] + w01 * Ey[k01] + w11 * Ey[k11];
        double a[3] = {qm * ex, qm * ey, 0.0};
        double *vp = v + 3 * p;
        double tau = orc_beta_integral(kind, vp, a, dt, v0);
        for (int i = 0; i < 3; ++i)
            vp[i] += a[i] * tau;
        double r = sqrt(vp[0] * vp[0] + vp[1] * vp[1] + vp[2] * vp[2]);
        double b = orc_beta(kind, r, v0);
        double xn = x[p] + b * vp[0] * dt, yn = y[p] + b * vp[1] * dt;
        xn -= Lx * floor(xn / Lx);
        if (xn >= Lx)
            xn -= Lx;
        x[p] = xn;
        y[p] = yn;
        if (yn < 0.0) {
            alive[p] = 0;
            flux[0] += 1;
        } else if (yn >= Ly) {
            alive[p] = 0;
            flux[1] += 1;
        }
    }
}

/* 2D volume source: the 1D source with the band across y and x uniform.   */
/* Macroparticle k takes u_j = u24(SplitMix64(key, 8k + j)): y in cells =  */
/* lo + u_0 len (FP32), x in cells = u_5 nx (FP32), velocity from          */
/* (u_1..u_4) as in orc_inject.                                            */
void orc_inject2d(uint64_t seed, uint64_t step, uint32_t species, long n_new,
                  float src_lo_cells, float src_len_cells, int nx, double dx, double vth,
                  double *x, double *y, double *v)
{
    const double two_pi = 6.283185307179586476925286766559;
    uint64_t key = orc_stream_key(seed, step, species);
    for (long k = 0; k < n_new; ++k) {
        float u0 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 0));
        double u1 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 1));
        double u2 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 2));
        double u3 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 3));
        double u4 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 4));
        float u5 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 5));
        float yc = src_lo_cells + u0 * src_len_cells;
        float xc = u5 * (float)nx;
        if (xc >= (float)nx)
            xc = 0.0f; /* u_5 = 1 is the periodic image of x = 0 */
        x[k] = (double)xc * dx;
        y[k] = (double)yc * dx;
        double r1 = sqrt(-2.0 * log(u1)), r2 = sqrt(-2.0 * log(u3));
        v[3 * k + 0] = vth * r1 * cos(two_pi * u2);
        v[3 * k + 1] = vth * r1 * sin(two_pi * u2);
        v[3 * k + 2] = vth * r2 * cos(two_pi * u4);
    }
}

/* ------------------------------------------------------------------------ */
/* Wall source (Sec. IV: electrons and ions enter from the right plate "as  */
/* if from a stationary plasma").  A Maxwellian of density n and thermal    */
/* speed vth sends n vth / sqrt(2 pi) particles per unit area and time      */
/* through the plane x = L, with the flux-weighted half-Maxwellian:         */
/* |vx| = vth sqrt(-2 ln u_1) towards -x, (vy, vz) Maxwellian from u_2, u_3. */
/* Under Eq. (ConservSpeedLimApprox) a source of f enters g unchanged, and  */
/* g-particles cross the plane at the rate int beta |vx| g = int |vx| f,    */
/* so PIC and SLPIC inject the same count with the same distribution.  A    */
/* particle entered at a uniformly random moment of the step and has moved  */
/* since at its speed-limited velocity: x = L - u_0 beta(|v|) |vx| dt       */
/* (a particle with vx = 0 is placed 2^-20 cells inside).  Macroparticle k  */
/* of this step and species takes u_j = u24(SplitMix64(key, 8k + j)).       */
/* ------------------------------------------------------------------------ */
void orc_inject_wall(uint64_t seed, uint64_t step, uint32_t species, long n_new, int n_cells,
                     double dx, double dt, double vth, int kind, double v0, double *x,
                     double *v)
{
    const double two_pi = 6.283185307179586476925286766559;
    const double L = dx * n_cells;
    uint64_t key = orc_stream_key(seed, step, species);
    for (long k = 0; k < n_new; ++k) {
        double u0 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 0));
        double u1 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 1));
        double u2 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 2));
        double u3 = orc_u24(orc_splitmix64_at(key, 8ULL * k + 3));
        double vxm = vth * sqrt(-2.0 * log(u1));
        double r2 = vth * sqrt(-2.0 * log(u2));
        double vy = r2 * cos(two_pi * u3), vz = r2 * sin(two_pi * u3);
        double b = orc_beta(kind, sqrt(vxm * vxm + vy * vy + vz * vz), v0);
        double xk = L - u0 * b * vxm * dt;
        if (!(xk < L))
            xk = L - dx * (1.0 / 1048576.0);
        x[k] = xk;
        v[3 * k + 0] = -vxm;
        v[3 * k + 1] = vy;
        v[3 * k + 2] = vz;
    }
}

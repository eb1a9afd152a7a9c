/*
 * lbm_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow, single-threaded FP64 CPU implementation of the D2Q9 BGK
 * lattice Boltzmann update with halfway bounce-back on a voxelised body, and of
 * the three force evaluations of Kaushal, Succi & Ansumali, "Flow force
 * calculation in Lattice Boltzmann Method" (arXiv:2210.10377):
 *   - momentum exchange in the operation order "algorithm A" (pre-collision),
 *   - momentum exchange in the order "algorithm B" (post-collision), Eq. (rtt5),
 *   - the discrete Reynolds transport theorem (DRTT), Eq. (rtt7), second form,
 *     following the Appendix algorithm step by step.
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load this file's library.  It shares no code, header, table or helper
 * with the CUDA library: every constant below is written out here from the
 * paper (Table tabD2Q9) and every loop follows the paper's order of steps.
 *
 * Conventions (stated once, used everywhere in this file):
 *   node n = y*nx + x, populations stored as planes f[i*nx*ny + n];
 *   direction order 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1)
 *                   5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1);
 *   f(x,t) is the pre-collision state, ft(x,t) the post-collision state
 *   (the paper's f and f-tilde, Eq. CollideAdv);
 *   relaxation: ft = f + omega (feq - f) with omega = 2 beta = 1/tau, i.e. the
 *   lattice relaxation time tau of the usual LBM convention (nu = (tau-1/2)/3);
 *   y is periodic; in the channel set-up x has an equilibrium inlet at x = 0
 *   and a zero-gradient (copy) outlet at x = nx-1; in the periodic set-up x is
 *   periodic too.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no FMA contraction,
 * so that the NACA mask predicate is evaluated with plain rounded operations).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---- Section II, Table tabD2Q9: D2Q9 velocities and weights, theta0 = 1/3 ---- */
static const int OC_X[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int OC_Y[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int O_OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double O_W[9] = {16.0 / 36.0, 4.0 / 36.0, 4.0 / 36.0, 4.0 / 36.0, 4.0 / 36.0,
                              1.0 / 36.0,  1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

void oracle_lattice(int *cx, int *cy, double *w, int *opp)
{
    for (int i = 0; i < 9; ++i) {
        cx[i] = OC_X[i];
        cy[i] = OC_Y[i];
        w[i] = O_W[i];
        opp[i] = O_OPP[i];
    }
}

/* Section II, second-order equilibrium:
 *   feq_i = w_i rho [1 + (u.c_i)/theta0 + ((u.c_i)^2 - theta0 u^2)/(2 theta0^2)]
 * With theta0 = 1/3 the three coefficients are 3, 9/2 and 3/2. */
void oracle_feq(double rho, double ux, double uy, double *out)
{
    double usq = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double cu = OC_X[i] * ux + OC_Y[i] * uy;
        out[i] = O_W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    }
}

/* Section II: rho = sum f_i, rho u = sum f_i c_i. */
static void moments(const double *fi, double *rho, double *jx, double *jy)
{
    double r = 0.0, mx = 0.0, my = 0.0;
    for (int i = 0; i < 9; ++i) {
        r += fi[i];
        mx += OC_X[i] * fi[i];
        my += OC_Y[i] * fi[i];
    }
    *rho = r;
    *jx = mx;
    *jy = my;
}

/* ---- NACA 4-digit symmetric section (the paper names NACA0012, 12% thickness
 * to chord, but prints no formula; this is the standard closed form):
 *   y_t(s) = 5 t C [0.2969 sqrt(s) - 0.1260 s - 0.3516 s^2 + 0.2843 s^3 - a4 s^4],
 *   s = xi / C, a4 = 0.1015 (open trailing edge) or 0.1036 (closed).
 * Frame: mid-chord at (xc, yc), angle of attack alpha > 0 nose-up:
 *   xi - C/2 = (x - xc) cos(alpha) - (y - yc) sin(alpha)
 *   eta      = (x - xc) sin(alpha) + (y - yc) cos(alpha)
 * Node (x, y) is solid iff 0 <= xi <= C and |eta| <= y_t(xi / C).
 * The expression is evaluated left to right exactly as written below, in
 * double precision with no fused multiply-add. */
/* Half-thickness y_t / C of the section at s = xi / C, same expression as in
 * oracle_naca_mask (exposed so that the thickness law can be checked alone). */
double oracle_naca_thickness(double s, double thickness, int closed_te)
{
    double a4 = closed_te ? 0.1036 : 0.1015;
    double poly =
        0.2969 * sqrt(s) - 0.1260 * s - 0.3516 * s * s + 0.2843 * s * s * s - a4 * s * s * s * s;
    return 5.0 * thickness * poly;
}

int oracle_naca_mask(int nx, int ny, double chord, double thickness, double alpha_deg,
                     double xc, double yc, int closed_te, unsigned char *out)
{
    if (nx <= 0 || ny <= 0 || !(chord > 0.0) || !(thickness > 0.0))
        return -1;
    double a = alpha_deg * M_PI / 180.0;
    double ca = cos(a), sa = sin(a);
    double a4 = closed_te ? 0.1036 : 0.1015;
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double dx = (double)x - xc;
            double dy = (double)y - yc;
            double xi = dx * ca - dy * sa + 0.5 * chord;
            double eta = dx * sa + dy * ca;
            unsigned char solid = 0;
            if (xi >= 0.0 && xi <= chord) {
                double s = xi / chord;
                double poly = 0.2969 * sqrt(s) - 0.1260 * s - 0.3516 * s * s + 0.2843 * s * s * s -
                              a4 * s * s * s * s;
                double yt = 5.0 * thickness * chord * poly;
                solid = fabs(eta) <= yt;
            }
            out[(long)y * nx + x] = solid;
        }
    }
    return 0;
}

/* ---- Circular cylinder (Section VI, flow past a 2-D circular cylinder):
 * node (x, y) is solid iff (x - xc)^2 + (y - yc)^2 <= r^2, r = D/2, evaluated
 * as written (dx*dx + dy*dy compared with r*r) in double precision with no
 * fused multiply-add. */
int oracle_cylinder_mask(int nx, int ny, double xc, double yc, double radius, unsigned char *out)
{
    if (nx <= 0 || ny <= 0 || !(radius > 0.0)) return -1;
    double r2 = radius * radius;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double dx = (double)x - xc;
            double dy = (double)y - yc;
            out[(long)y * nx + x] = dx * dx + dy * dy <= r2;
        }
    return 0;
}

/* Neighbour x + c_i of node (x, y).  y wraps; x wraps only when periodic_x.
 * Returns -1 when the neighbour lies outside the domain in x. */
static long neighbour(int nx, int ny, int periodic_x, int x, int y, int i)
{
    int x2 = x + OC_X[i];
    int y2 = y + OC_Y[i];
    if (y2 < 0) y2 += ny;
    if (y2 >= ny) y2 -= ny;
    if (x2 < 0 || x2 >= nx) {
        if (!periodic_x) return -1;
        x2 = (x2 + nx) % nx;
    }
    return (long)y2 * nx + x2;
}

/* Fluid-solid links (Fig. basicLadd, halfway bounce-back definition): the pair
 * (x_f, i) with x_f fluid and x_f + c_i solid, i = 1..8.  Packed as
 * n*8 + (i-1) and listed in ascending order (row-major nodes, then i).
 * Writes at most cap entries and returns the total count. */
long oracle_links(const unsigned char *mask, int nx, int ny, int periodic_x, int *out, long cap)
{
    long k = 0;
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            long n = (long)y * nx + x;
            if (mask[n]) continue;
            for (int i = 1; i < 9; ++i) {
                long m = neighbour(nx, ny, periodic_x, x, y, i);
                if (m >= 0 && mask[m]) {
                    if (k < cap) out[k] = (int)(n * 8 + (i - 1));
                    ++k;
                }
            }
        }
    }
    return k;
}

/* Default control volume (Appendix: a rectangle around the body): the bounding
 * box of the solid nodes, widened by m = max(4, ceil(w/4)) nodes on each side,
 * w = bounding-box width in x.  In a channel the x-range is then clipped to
 * [1, nx-2], so the inlet and outlet columns stay outside.  In a periodic
 * direction a widened range that would reach the first or last node becomes the
 * whole period instead (a box never straddles a periodic edge).  With no solid
 * node the box is the whole allowed domain.  Inclusive: cv = {x0, x1, y0, y1}. */
void oracle_auto_cv(const unsigned char *mask, int nx, int ny, int periodic_x, int *cv)
{
    int xmin = nx, xmax = -1, ymin = ny, ymax = -1;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            if (mask[(long)y * nx + x]) {
                if (x < xmin) xmin = x;
                if (x > xmax) xmax = x;
                if (y < ymin) ymin = y;
                if (y > ymax) ymax = y;
            }
    if (xmax < 0) {
        cv[0] = periodic_x ? 0 : 1;
        cv[1] = periodic_x ? nx - 1 : nx - 2;
        cv[2] = 0;
        cv[3] = ny - 1;
        return;
    }
    int w = xmax - xmin + 1;
    int m = (w + 3) / 4;
    if (m < 4) m = 4;
    int x0 = xmin - m, x1 = xmax + m, y0 = ymin - m, y1 = ymax + m;
    if (periodic_x) {
        if (x0 < 1 || x1 > nx - 2) { x0 = 0; x1 = nx - 1; }
    } else {
        if (x0 < 1) x0 = 1;
        if (x1 > nx - 2) x1 = nx - 2;
    }
    if (y0 < 1 || y1 > ny - 2) { y0 = 0; y1 = ny - 1; }
    cv[0] = x0;
    cv[1] = x1;
    cv[2] = y0;
    cv[3] = y1;
}

/* ------------------------------- the solver ------------------------------- */

enum { SCHEME_A = 0, SCHEME_B = 1, SCHEME_DRTT = 2, SCHEME_A_RTT = 3, SCHEME_SI = 4, NSCHEME = 5 };

typedef struct oracle_sim {
    int nx, ny, periodic;
    long N;
    double tau, omega, rho0, gx, gy;
    double *u_in;          /* [ny] inlet velocity per row */
    unsigned char *mask;   /* [ny*nx], 1 = solid */
    int cv[4];             /* inclusive control volume box */
    double *f, *ft, *fn;   /* pre-collision, post-collision, next pre-collision */
    int *links;
    long nlinks;
    long t;                /* steps done */
    double *series;        /* [t][NSCHEME][2] */
    long cap;
    double *jseries;       /* [t][6]: J(t), G(t), Lo(t) */
} oracle_sim;

static int in_cv(const oracle_sim *s, long n)
{
    int x = (int)(n % s->nx), y = (int)(n / s->nx);
    return x >= s->cv[0] && x <= s->cv[1] && y >= s->cv[2] && y <= s->cv[3];
}

/* Eq. (rtt1): J(t) = sum over fluid nodes of the control volume of sum_i c_i f_i. */
static void momentum_cv(const oracle_sim *s, const double *f, double *J)
{
    double jx = 0.0, jy = 0.0;
    for (int y = s->cv[2]; y <= s->cv[3]; ++y)
        for (int x = s->cv[0]; x <= s->cv[1]; ++x) {
            long n = (long)y * s->nx + x;
            if (s->mask[n]) continue;
            for (int i = 0; i < 9; ++i) {
                jx += OC_X[i] * f[i * s->N + n];
                jy += OC_Y[i] * f[i * s->N + n];
            }
        }
    J[0] = jx;
    J[1] = jy;
}

void oracle_destroy(oracle_sim *s)
{
    if (!s) return;
    free(s->u_in);
    free(s->mask);
    free(s->f);
    free(s->ft);
    free(s->fn);
    free(s->links);
    free(s->series);
    free(s->jseries);
    free(s);
}

/* bc_kind: 0 = channel (inlet/outlet in x, periodic y), 1 = fully periodic.
 * u_in: n_u_in values (1 or ny).  g: body force (2 values) or NULL.
 * cv: inclusive box or NULL / cv[0] < 0 for the default box.
 * Initial state: feq(rho0, (u_in(y), 0)) on every fluid node, 0 on solid nodes. */
oracle_sim *oracle_create(const unsigned char *mask, int nx, int ny, double tau, const double *u_in,
                          int n_u_in, int bc_kind, double rho0, const double *g, const int *cv)
{
    if (nx < 3 || ny < 3 || !(tau > 0.5) || (n_u_in != 1 && n_u_in != ny))
        return NULL;
    oracle_sim *s = (oracle_sim *)calloc(1, sizeof(oracle_sim));
    if (!s) return NULL;
    s->nx = nx;
    s->ny = ny;
    s->N = (long)nx * ny;
    s->periodic = bc_kind == 1;
    s->tau = tau;
    s->omega = 1.0 / tau;
    s->rho0 = rho0;
    s->gx = g ? g[0] : 0.0;
    s->gy = g ? g[1] : 0.0;
    s->u_in = (double *)malloc(sizeof(double) * ny);
    s->mask = (unsigned char *)malloc(s->N);
    s->f = (double *)calloc(9 * s->N, sizeof(double));
    s->ft = (double *)calloc(9 * s->N, sizeof(double));
    s->fn = (double *)calloc(9 * s->N, sizeof(double));
    if (!s->u_in || !s->mask || !s->f || !s->ft || !s->fn) {
        oracle_destroy(s);
        return NULL;
    }
    for (int y = 0; y < ny; ++y) s->u_in[y] = n_u_in == 1 ? u_in[0] : u_in[y];
    memcpy(s->mask, mask, s->N);
    if (cv && cv[0] >= 0)
        memcpy(s->cv, cv, sizeof(s->cv));
    else
        oracle_auto_cv(mask, nx, ny, s->periodic, s->cv);
    s->nlinks = oracle_links(mask, nx, ny, s->periodic, NULL, 0);
    s->links = (int *)malloc(sizeof(int) * (s->nlinks > 0 ? s->nlinks : 1));
    oracle_links(mask, nx, ny, s->periodic, s->links, s->nlinks);
    for (long n = 0; n < s->N; ++n) {
        if (mask[n]) continue;
        double feq[9];
        oracle_feq(rho0, s->u_in[n / nx], 0.0, feq);
        for (int i = 0; i < 9; ++i) s->f[i * s->N + n] = feq[i];
    }
    return s;
}

long oracle_nlinks(const oracle_sim *s) { return s->nlinks; }
long oracle_steps_done(const oracle_sim *s) { return s->t; }
void oracle_cv(const oracle_sim *s, int *cv) { memcpy(cv, s->cv, sizeof(s->cv)); }

void oracle_get_links(const oracle_sim *s, int *out) { memcpy(out, s->links, sizeof(int) * s->nlinks); }

/* Pre-collision populations f(x, t) as [9][ny][nx]; solid nodes read 0. */
void oracle_get_populations(const oracle_sim *s, double *out)
{
    for (int i = 0; i < 9; ++i)
        for (long n = 0; n < s->N; ++n) out[i * s->N + n] = s->mask[n] ? 0.0 : s->f[i * s->N + n];
}

/* Replace f(x, t) on fluid nodes (solid nodes keep 0). */
void oracle_set_populations(oracle_sim *s, const double *in)
{
    for (int i = 0; i < 9; ++i)
        for (long n = 0; n < s->N; ++n) s->f[i * s->N + n] = s->mask[n] ? 0.0 : in[i * s->N + n];
}

static int grow_series(oracle_sim *s, long need)
{
    if (need <= s->cap) return 0;
    long cap = s->cap ? s->cap : 64;
    while (cap < need) cap *= 2;
    double *a = (double *)realloc(s->series, sizeof(double) * cap * NSCHEME * 2);
    if (!a) return -1;
    s->series = a;
    double *b = (double *)realloc(s->jseries, sizeof(double) * cap * 6);
    if (!b) return -1;
    s->jseries = b;
    s->cap = cap;
    return 0;
}

/* One time step t -> t+1, in the order of the Appendix algorithm. */
static void step_once(oracle_sim *s)
{
    const int nx = s->nx, ny = s->ny;
    const long N = s->N;
    double *f = s->f, *ft = s->ft, *fn = s->fn;
    double *out = s->series + s->t * NSCHEME * 2;
    double *jout = s->jseries + s->t * 6;

    /* (1) J(t) over the control volume, Eq. (rtt1), on the pre-collision state. */
    double Jt[2];
    momentum_cv(s, f, Jt);

    /* (2) Collide over the whole fluid domain, Eq. (CollideAdv):
     *     ft = f + 2 beta (feq(rho, u) - f), 2 beta = 1/tau.
     *     A uniform body force g (used only by test set-ups) adds 3 w_i c_i.g.
     *     Inlet column (channel set-up): ft = feq(rho0, (u_in(y), 0)). */
    /* Nodes are independent: the loop may run on several threads (the values
     * do not depend on how it is split). */
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (s->mask[n]) continue;
        int x = (int)(n % nx), y = (int)(n / nx);
        double feq[9];
        if (!s->periodic && x == 0) {
            oracle_feq(s->rho0, s->u_in[y], 0.0, feq);
            for (int i = 0; i < 9; ++i) ft[i * N + n] = feq[i];
            continue;
        }
        double fi[9], rho, jx, jy;
        for (int i = 0; i < 9; ++i) fi[i] = f[i * N + n];
        moments(fi, &rho, &jx, &jy);
        oracle_feq(rho, jx / rho, jy / rho, feq);
        for (int i = 0; i < 9; ++i) {
            double v = fi[i] + s->omega * (feq[i] - fi[i]);
            if (s->gx != 0.0 || s->gy != 0.0)
                v += 3.0 * O_W[i] * (OC_X[i] * s->gx + OC_Y[i] * s->gy);
            ft[i * N + n] = v;
        }
    }

    /* (3) Momentum exchange over the fluid-solid links, Eq. (MEA):
     *     F = sum_links -[f_opp(x_f) c_opp - f_i(x_f) c_i] = sum c_i (f_i + f_opp).
     *     Algorithm A: both terms on the pre-collision state f(x_f, t).
     *     Algorithm B: with the post-collision state, and halfway bounce-back
     *       returning ft_i as the opposite population, F = 2 sum c_i ft_i(x_f, t)
     *       (the single-boundary simplification after Eq. rtt5).
     *     A' (Eq. rtt4 read literally for algorithm A): lost momentum counted with
     *       f_i(x_f, t), gained momentum with the bounced ft_i(x_f, t). */
    double A[2] = {0.0, 0.0}, B[2] = {0.0, 0.0}, Ap[2] = {0.0, 0.0};
    for (long k = 0; k < s->nlinks; ++k) {
        long n = s->links[k] / 8;
        int i = s->links[k] % 8 + 1;
        int o = O_OPP[i];
        A[0] += OC_X[i] * (f[i * N + n] + f[o * N + n]);
        A[1] += OC_Y[i] * (f[i * N + n] + f[o * N + n]);
        Ap[0] += OC_X[i] * (f[i * N + n] + ft[i * N + n]);
        Ap[1] += OC_Y[i] * (f[i * N + n] + ft[i * N + n]);
        B[0] += 2.0 * OC_X[i] * ft[i * N + n];
        B[1] += 2.0 * OC_Y[i] * ft[i * N + n];
    }

    /* (3b) Stress integration, Eq. (stress_int), on the voxelised surface.  Each
     *      axis link (x_f, i), i = 1..4, is a unit face between the fluid node
     *      x_f and its solid neighbour x_f + c_i; its normal out of the solid is
     *      n = -c_i.  The stress at x_f is T = -p I + sigma, with p = rho theta0
     *      (theta0 = 1/3) and the deviatoric part from the second moment of the
     *      non-equilibrium populations of the pre-collision f(x_f, t):
     *        sigma_ab = -(1 - omega/2) sum_k (f_k - feq_k) c_ka c_kb
     *      (the paper's factor 1 - beta with 2 beta = omega; the sign makes sigma
     *      the viscous stress rho nu (grad u + grad u^T) of Eq. stress_int; the
     *      theta0/D trace term sums to zero because sum_k (f_k - feq_k) = 0).
     *      Force on the body: F_b = sum_faces n_a T_ab = -sum_faces c_ia T_ab. */
    double SI[2] = {0.0, 0.0};
    for (long k = 0; k < s->nlinks; ++k) {
        long n = s->links[k] / 8;
        int i = s->links[k] % 8 + 1;
        if (i > 4) continue;
        double fi[9], feq[9], rho, jx, jy;
        for (int q = 0; q < 9; ++q) fi[q] = f[q * N + n];
        moments(fi, &rho, &jx, &jy);
        oracle_feq(rho, jx / rho, jy / rho, feq);
        double Pxx = 0.0, Pxy = 0.0, Pyy = 0.0;
        for (int q = 0; q < 9; ++q) {
            double d = fi[q] - feq[q];
            Pxx += d * OC_X[q] * OC_X[q];
            Pxy += d * OC_X[q] * OC_Y[q];
            Pyy += d * OC_Y[q] * OC_Y[q];
        }
        double visc = 1.0 - 0.5 * s->omega;
        double p = rho / 3.0;
        double Txx = -p - visc * Pxx, Txy = -visc * Pxy, Tyy = -p - visc * Pyy;
        SI[0] -= OC_X[i] * Txx + OC_Y[i] * Txy;
        SI[1] -= OC_X[i] * Txy + OC_Y[i] * Tyy;
    }

    /* (4) Fluxes of post-collision populations through the control-volume
     *     surface (Eq. rtt7): gained = populations of fluid nodes outside the box
     *     that stream into a fluid node of the box; lost = populations of fluid
     *     nodes of the box that stream to a fluid node outside it. */
    double G[2] = {0.0, 0.0}, Lo[2] = {0.0, 0.0};
    for (long n = 0; n < N; ++n) {
        if (s->mask[n]) continue;
        int x = (int)(n % nx), y = (int)(n / nx);
        int inside = in_cv(s, n);
        for (int i = 1; i < 9; ++i) {
            long m = neighbour(nx, ny, s->periodic, x, y, i);
            if (m < 0 || s->mask[m]) continue;
            int m_inside = in_cv(s, m);
            if (!inside && m_inside) {
                G[0] += OC_X[i] * ft[i * N + n];
                G[1] += OC_Y[i] * ft[i * N + n];
            } else if (inside && !m_inside) {
                Lo[0] += OC_X[i] * ft[i * N + n];
                Lo[1] += OC_Y[i] * ft[i * N + n];
            }
        }
    }

    /* (5) Advection f(x + c_i, t+1) = ft_i(x, t), with halfway bounce-back
     *     f_opp(x_f, t+1) = ft_i(x_f, t) when x_f + c_i is solid. */
    memset(fn, 0, sizeof(double) * 9 * N);
    /* Every target population is written by exactly one source node (a node
     * next to a solid is never the target of a push from it), so the loop may
     * run on several threads. */
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (s->mask[n]) continue;
        int x = (int)(n % nx), y = (int)(n / nx);
        fn[n] = ft[n]; /* rest population stays */
        for (int i = 1; i < 9; ++i) {
            long m = neighbour(nx, ny, s->periodic, x, y, i);
            if (m < 0) continue; /* leaves through the inlet / outlet column */
            if (s->mask[m])
                fn[O_OPP[i] * N + n] = ft[i * N + n];
            else
                fn[i * N + m] = ft[i * N + n];
        }
    }

    /* (6) Inlet / outlet (channel set-up): equilibrium inlet at x = 0,
     *     zero-gradient outlet f(nx-1, y) = f(nx-2, y). */
    if (!s->periodic) {
        for (int y = 0; y < ny; ++y) {
            double feq[9];
            oracle_feq(s->rho0, s->u_in[y], 0.0, feq);
            long n0 = (long)y * nx, n1 = (long)y * nx + nx - 1, n2 = n1 - 1;
            for (int i = 0; i < 9; ++i) {
                fn[i * N + n0] = feq[i];
                fn[i * N + n1] = fn[i * N + n2];
            }
        }
    }

    /* (7) J(t+1) and the DRTT force, Eq. (rtt7) second form:
     *     F(t) = J(t) - J(t+1) + gained - lost. */
    double Jn[2];
    momentum_cv(s, fn, Jn);
    double D[2] = {Jt[0] - Jn[0] + G[0] - Lo[0], Jt[1] - Jn[1] + G[1] - Lo[1]};

    out[SCHEME_A * 2 + 0] = A[0];
    out[SCHEME_A * 2 + 1] = A[1];
    out[SCHEME_B * 2 + 0] = B[0];
    out[SCHEME_B * 2 + 1] = B[1];
    out[SCHEME_DRTT * 2 + 0] = D[0];
    out[SCHEME_DRTT * 2 + 1] = D[1];
    out[SCHEME_A_RTT * 2 + 0] = Ap[0];
    out[SCHEME_A_RTT * 2 + 1] = Ap[1];
    out[SCHEME_SI * 2 + 0] = SI[0];
    out[SCHEME_SI * 2 + 1] = SI[1];
    jout[0] = Jt[0];
    jout[1] = Jt[1];
    jout[2] = G[0];
    jout[3] = G[1];
    jout[4] = Lo[0];
    jout[5] = Lo[1];

    s->f = fn;
    s->fn = f;
    s->t += 1;
}

/* Host threads for the node loops of oracle_step (1 by default); returns the
 * count in use.  The results do not depend on it: the force, flux and momentum
 * sums always run on one thread in their fixed order. */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Advance n steps; returns 0, or -1 on allocation failure. */
int oracle_step(oracle_sim *s, int n)
{
    if (n < 0) return -1;
    if (grow_series(s, s->t + n)) return -1;
    for (int k = 0; k < n; ++k) step_once(s);
    return 0;
}

/* Forces of steps [first, first+count) for one scheme (0 A, 1 B, 2 DRTT, 3 A').
 * Force on the body, F(t) belongs to the transition t -> t+1. */
int oracle_force_series(const oracle_sim *s, int scheme, long first, long count, double *fx,
                        double *fy)
{
    if (scheme < 0 || scheme >= NSCHEME || first < 0 || count < 0 || first + count > s->t)
        return -1;
    for (long k = 0; k < count; ++k) {
        fx[k] = s->series[(first + k) * NSCHEME * 2 + scheme * 2 + 0];
        fy[k] = s->series[(first + k) * NSCHEME * 2 + scheme * 2 + 1];
    }
    return 0;
}

/* DRTT ingredients of step t: J(t) (2), gained (2), lost (2). */
/* Pressure coefficient at the boundary fluid nodes, Section VI:
 *   C_p = (p - p_inf) / q,  p = rho theta0 = rho / 3,
 * on the pre-collision state of the current step.  The boundary fluid nodes
 * are the distinct fluid nodes of the link list, ascending.  nodes and cp
 * receive at most cap entries; *count the number of boundary nodes. */
void oracle_surface_pressure(const oracle_sim *s, double p_inf, double q, int *nodes, double *cp,
                             long cap, long *count)
{
    long m = 0;
    long prev = -1;
    for (long k = 0; k < s->nlinks; ++k) {
        long n = s->links[k] / 8;
        if (n == prev) continue;
        prev = n;
        if (m < cap) {
            double fi[9], rho, jx, jy;
            for (int i = 0; i < 9; ++i) fi[i] = s->f[i * s->N + n];
            moments(fi, &rho, &jx, &jy);
            if (nodes) nodes[m] = (int)n;
            if (cp) cp[m] = (rho / 3.0 - p_inf) / q;
        }
        ++m;
    }
    *count = m;
}

int oracle_drtt_parts(const oracle_sim *s, long t, double *out6)
{
    if (t < 0 || t >= s->t) return -1;
    memcpy(out6, s->jseries + t * 6, sizeof(double) * 6);
    return 0;
}

/* ------------------------------ discrete adjoint ------------------------------
 * Gradient of the window-averaged force of algorithm B,
 *   J = (1/M) sum_{t = T-M}^{T-1} (wx Fx(t) + wy Fy(t)),  F(t) = 2 sum_links c_i ft_i(x_f, t),
 * with respect to the relaxation time tau, the inlet velocity of every row,
 * and the initial pre-collision populations f(x, 0), for the channel set-up.
 * The forward map of one step (collide, stream with halfway bounce-back, inlet,
 * outlet) is differentiated exactly and transposed step by step, backwards in
 * time; states are recomputed from sqrt(T)-spaced checkpoints.
 *
 * One step, with lt = dJ/d(ft(t)) and lam = dJ/d(f(t)):
 *   lt_j(y) = lam'_j(y + c_j)        if y + c_j is a fluid node in the domain,
 *           = lam'_opp(j)(y)         if y + c_j is solid (bounce-back),
 *           + (2/M) (wx c_jx + wy c_jy) on links inside the window,
 *   where lam' is lam(t+1) with the inlet column set to zero (overwritten by the
 *   inlet), the outlet column set to zero and added to column nx-2 (the outlet
 *   copies it);
 *   lam_k(y) = sum_i lt_i(y) d ft_i / d f_k(y)   (collision Jacobian, entry by entry),
 *   dJ/d omega += sum_i lt_i (feq_i - f_i),  omega = 1/tau,
 *   inlet node: dJ/du_in(y) += sum_i lt_i d feq_i(rho0, (u_in(y), 0)) / du, lam = 0.
 * ------------------------------------------------------------------------------ */

/* d ft_i / d f_k of the BGK collision at one node, from feq_i = w_i rho
 * (1 + 3 cu + 4.5 cu^2 - 1.5 u^2), u = j / rho:
 *   d feq_i / d f_k = feq_i / rho + (d feq_i / d u) . (c_k - u) / rho. */
static void collision_jacobian(const double *fi, double omega, double *Jm /* [9][9], Jm[i*9+k] */)
{
    double rho, jx, jy;
    moments(fi, &rho, &jx, &jy);
    double ux = jx / rho, uy = jy / rho;
    double feq[9];
    oracle_feq(rho, ux, uy, feq);
    for (int i = 0; i < 9; ++i) {
        double cu = OC_X[i] * ux + OC_Y[i] * uy;
        double dux = O_W[i] * rho * (3.0 * OC_X[i] + 9.0 * cu * OC_X[i] - 3.0 * ux);
        double duy = O_W[i] * rho * (3.0 * OC_Y[i] + 9.0 * cu * OC_Y[i] - 3.0 * uy);
        for (int k = 0; k < 9; ++k) {
            double dfeq = feq[i] / rho + (dux * (OC_X[k] - ux) + duy * (OC_Y[k] - uy)) / rho;
            Jm[i * 9 + k] = (i == k ? 1.0 - omega : 0.0) + omega * dfeq;
        }
    }
}

/* mask, nx, ny, tau, u_in[ny], f0[9][ny][nx] (fluid nodes used): as oracle_create.
 * Outputs: *J, *dJ_dtau, dJ_du[ny], dJ_df0[9][ny][nx] (NULL allowed).
 * Returns 0, or -1 on bad arguments / allocation failure. */
int oracle_adjoint(const unsigned char *mask, int nx, int ny, double tau, const double *u_in,
                   const double *f0, int steps, int window, double wx, double wy, double *J,
                   double *dJ_dtau, double *dJ_du, double *dJ_df0)
{
    if (steps < 1 || window < 1 || window > steps) return -1;
    oracle_sim *s = oracle_create(mask, nx, ny, tau, u_in, ny, 0, 1.0, NULL, NULL);
    if (!s) return -1;
    const long N = s->N;
    const size_t state = sizeof(double) * 9 * N;
    int K = 1;
    while ((long)K * K < steps) ++K;
    int nck = (steps + K - 1) / K;
    double *ck = (double *)malloc(state * (size_t)nck);      /* checkpoints f(kK) */
    double *seg = (double *)malloc(state * (size_t)(K + 1)); /* f(t) of one segment */
    double *lam = (double *)calloc(9 * N, sizeof(double));
    double *lamp = (double *)calloc(9 * N, sizeof(double));
    double *lt = (double *)calloc(9 * N, sizeof(double));
    if (!ck || !seg || !lam || !lamp || !lt || grow_series(s, steps)) {
        free(ck); free(seg); free(lam); free(lamp); free(lt);
        oracle_destroy(s);
        return -1;
    }
    oracle_set_populations(s, f0);
    /* forward: checkpoints and the force series */
    for (int t = 0; t < steps; ++t) {
        if (t % K == 0) memcpy(ck + (size_t)(t / K) * 9 * N, s->f, state);
        step_once(s);
    }
    double Jv = 0.0;
    for (int t = steps - window; t < steps; ++t)
        Jv += wx * s->series[t * NSCHEME * 2 + SCHEME_B * 2 + 0] +
              wy * s->series[t * NSCHEME * 2 + SCHEME_B * 2 + 1];
    Jv /= window;

    double domega = 0.0;
    double *du = (double *)calloc(ny, sizeof(double));
    const double obj = 2.0 / window;
    /* lam holds dJ/df(t+1); zero at t+1 = T */
    for (int k = nck - 1; k >= 0; --k) {
        int t0 = k * K, t1 = (k + 1) * K < steps ? (k + 1) * K : steps;
        /* recompute f(t0 .. t1-1) (rewriting the same series entries) */
        memcpy(s->f, ck + (size_t)k * 9 * N, state);
        s->t = t0;
        for (int t = t0; t < t1; ++t) {
            memcpy(seg + (size_t)(t - t0) * 9 * N, s->f, state);
            if (t + 1 < t1) step_once(s);
        }
        for (int t = t1 - 1; t >= t0; --t) {
            const double *f = seg + (size_t)(t - t0) * 9 * N;
            /* lam' = lam(t+1) with the inlet and outlet columns folded */
            memcpy(lamp, lam, sizeof(double) * 9 * N);
            for (int y = 0; y < ny; ++y) {
                long n0 = (long)y * nx, n1 = n0 + nx - 1, n2 = n1 - 1;
                for (int i = 0; i < 9; ++i) {
                    lamp[i * N + n2] += lamp[i * N + n1];
                    lamp[i * N + n1] = 0.0;
                    lamp[i * N + n0] = 0.0;
                }
            }
            int in_window = t >= steps - window;
            for (long n = 0; n < N; ++n) {
                if (mask[n]) continue;
                int x = (int)(n % nx), y = (int)(n / nx);
                for (int j = 0; j < 9; ++j) {
                    long m = j == 0 ? n : neighbour(nx, ny, 0, x, y, j);
                    double v = 0.0;
                    if (m >= 0) {
                        if (mask[m]) {
                            v = lamp[O_OPP[j] * N + n];
                            if (in_window) v += obj * (wx * OC_X[j] + wy * OC_Y[j]);
                        } else {
                            v = lamp[j * N + m];
                        }
                    }
                    lt[j * N + n] = v;
                }
            }
            for (long n = 0; n < N; ++n) {
                for (int i = 0; i < 9; ++i) lam[i * N + n] = 0.0;
                if (mask[n]) continue;
                int x = (int)(n % nx), y = (int)(n / nx);
                if (x == 0) {
                    double u = s->u_in[y];
                    for (int i = 0; i < 9; ++i)
                        du[y] += lt[i * N + n] * O_W[i] * 1.0 *
                                 (3.0 * OC_X[i] + 9.0 * OC_X[i] * OC_X[i] * u - 3.0 * u);
                    continue;
                }
                double fi[9], Jm[81], rho, jx, jy, feq[9];
                for (int i = 0; i < 9; ++i) fi[i] = f[i * N + n];
                collision_jacobian(fi, s->omega, Jm);
                moments(fi, &rho, &jx, &jy);
                oracle_feq(rho, jx / rho, jy / rho, feq);
                for (int k2 = 0; k2 < 9; ++k2) {
                    double acc = 0.0;
                    for (int i = 0; i < 9; ++i) acc += lt[i * N + n] * Jm[i * 9 + k2];
                    lam[k2 * N + n] = acc;
                }
                for (int i = 0; i < 9; ++i) domega += lt[i * N + n] * (feq[i] - fi[i]);
            }
        }
    }
    if (J) *J = Jv;
    if (dJ_dtau) *dJ_dtau = -domega / (tau * tau);
    if (dJ_du) memcpy(dJ_du, du, sizeof(double) * ny);
    if (dJ_df0)
        for (int i = 0; i < 9; ++i)
            for (long n = 0; n < N; ++n) dJ_df0[i * N + n] = mask[n] ? 0.0 : lam[i * N + n];
    free(du); free(ck); free(seg); free(lam); free(lamp); free(lt);
    oracle_destroy(s);
    return 0;
}

/*
 * lbm_ace_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct FP64 CPU implementation of the lattice
 * Boltzmann (LB) method of H. Liang, "An accurate lattice Boltzmann method for
 * interface capturing" (arXiv 2203.05230): a D2Q9 BGK equation with a forcing
 * distribution (Eqs. 9-12) that recovers the modified conservative Allen-Cahn
 * equation (Eq. 8), using the regularised signed distance and unit normal of
 * Eq. 13 and the clip of phi described right after it, on a periodic lattice
 * (Section 3), driven by the time-reversed single-vortex field (Eq. 14).
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file. It shares no code, header, table or helper
 * with the CUDA library; the two meet only in the documented state layout.
 *
 * Structure: the paper's own order. Each step computes, at every node and at
 * time t, phi = sum_i f_i (Eq. 12); psi (Eq. 13); the isotropic gradient of
 * psi and the normal (Eq. 13); the sharpening magnitude (Eqs. 6, 11); the
 * explicit-Euler time derivative of phi*u (Section 2.2); the forcing F_i
 * (Eq. 11); the equilibrium f_i^eq (Eq. 10); the BGK update (Eq. 9); and then
 * pushes the post-collision value to x + c_i (left-hand side of Eq. 9).
 *
 * Readings of the paper (it is silent, ambiguous or inconsistent there):
 *  R1  Factor 4 in psi. Eq. 5's middle form and Eqs. 2, 4, 6 imply
 *      psi = (eps_p/4) ln(phi/(1-phi)), while Eqs. 5 (right) and 13 print
 *      psi = eps ln(...). We use eps := eps_p / 4 throughout, so that
 *      psi = eps ln(phi/(1-phi)) as printed in Eq. 13, the equilibrium profile
 *      of Eq. 2 reads phi = 1/2 + 1/2 tanh(s/(2 eps)), and the sharpening
 *      magnitude of Eqs. 6, 8, 11 reads (1/(4 eps)) [1 - tanh^2(psi/(2 eps))],
 *      which equals phi(1-phi)/eps.
 *  R2  The second-order isotropic gradient (cited, not printed):
 *      grad chi(x) = sum_i w_i c_i chi(x + c_i) / c_s^2.
 *  R3  The explicit-Euler time derivative is the backward difference
 *      (phi u)(t) - (phi u)(t-1); it is zero at the first step t = 0.
 *  R4  The velocity is sampled at t = the step index; nodes sit at integer
 *      coordinates x = 0..nx-1, y = 0..ny-1.
 *  R5  Eq. 14 with a sign factor: u = s U0 sin^2(pi x/nx) sin(2 pi y/ny)
 *      cos(pi t/T), v = -s U0 sin^2(pi y/ny) sin(2 pi x/nx) cos(pi t/T);
 *      s = +1 is the paper's sign.
 *  R6  The regulariser of Eq. 13 (the paper's varepsilon, "delta" here) is an
 *      absolute constant used both inside the logarithm and in the normal.
 *  R7  Initial populations are f_i^eq(phi0, u(x, 0)); phi at t = -1 is phi0.
 *  R8  Conservative-ACE ablation (Eq. 1) under R1: the normal is taken from
 *      the isotropic gradient of phi itself and the sharpening magnitude is
 *      phi(1-phi)/eps with the unclipped phi.
 *
 * State layout (shared with the CUDA library only as a documented format):
 * f[i][y][x] (i = 0..8, x fastest) holds f_i(x, t) after streaming, phi_prev
 * [y][x] holds phi(x, t-1). D2Q9 order: c_0 = (0,0); c_1..c_4 = (1,0), (0,1),
 * (-1,0), (0,-1); c_5..c_8 = (1,1), (-1,1), (-1,-1), (1,-1). The paper
 * defers the velocity set to its Ref. [Liang2]; results do not depend on the
 * order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* D2Q9 weights as printed after Eq. 10, and the standard velocity set. */
static const double W[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double CS2 = 1.0 / 3.0; /* c_s^2, after Eq. 10 */
static const double PI = 3.14159265358979323846;

enum { ORACLE_MODIFIED = 0, ORACLE_CONSERVATIVE = 1 };
enum { ORACLE_VORTEX = 0, ORACLE_UNIFORM = 1, ORACLE_FIELD = 2 };

typedef struct {
    int nx, ny;
    int model;    /* ORACLE_MODIFIED (Eq. 8) or ORACLE_CONSERVATIVE (Eq. 1, R8) */
    int vel_kind; /* ORACLE_VORTEX (Eq. 14), ORACLE_UNIFORM, ORACLE_FIELD */
    double tau;   /* BGK relaxation time, Eq. 9 */
    double eps;   /* interface parameter (R1) */
    double delta; /* regulariser of Eq. 13 (R6) */
    double U0, T, sign; /* single vortex (R5) */
    double ux, uy;      /* uniform velocity */
    const double *ufield, *vfield; /* static velocity field [ny][nx] */
} oracle_params;

void oracle_lattice(double *w, int *cx, int *cy)
{
    for (int i = 0; i < 9; ++i) {
        w[i] = W[i];
        cx[i] = CX[i];
        cy[i] = CY[i];
    }
}

static int wrap(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

/* Eq. 2 under R1: equilibrium profile at signed normal coordinate s. */
double oracle_profile(double s, double eps)
{
    return 0.5 + 0.5 * tanh(s / (2.0 * eps));
}

/* Eq. 13 with the clip that follows it: psi = eps ln((phi_c + d)/(1 - phi_c + d)). */
double oracle_psi(double phi, double eps, double delta)
{
    double phic = phi;
    if (phic < 0.0) phic = 0.0;
    if (phic > 1.0) phic = 1.0;
    return eps * log((phic + delta) / (1.0 - phic + delta));
}

/* Sharpening magnitude of Eqs. 6, 8 and 11 under R1, written with tanh as printed. */
double oracle_sharpen(double psi, double eps)
{
    double th = tanh(psi / (2.0 * eps));
    return (1.0 - th * th) / (4.0 * eps);
}

/* Eq. 10: f_i^eq = w_i phi (1 + c_i . u / c_s^2). */
void oracle_feq(double phi, double u, double v, double *out)
{
    for (int i = 0; i < 9; ++i) {
        double cu = CX[i] * u + CY[i] * v;
        out[i] = W[i] * phi * (1.0 + cu / CS2);
    }
}

/* Eq. 11: F_i = w_i c_i . G / c_s^2 with G = d_t(phi u) + c_s^2 S n. */
void oracle_forcing(double gx, double gy, double *out)
{
    for (int i = 0; i < 9; ++i) out[i] = W[i] * (CX[i] * gx + CY[i] * gy) / CS2;
}

/* R2: isotropic gradient at the centre of a 3x3 window, win[(dy+1)*3 + (dx+1)]
 * = chi(x + dx, y + dy). */
static void grad_window(const double *win, double *out)
{
    double gx = 0.0, gy = 0.0;
    for (int i = 1; i < 9; ++i) {
        double c = win[(CY[i] + 1) * 3 + (CX[i] + 1)];
        gx += W[i] * CX[i] * c;
        gy += W[i] * CY[i] * c;
    }
    out[0] = gx / CS2;
    out[1] = gy / CS2;
}

/* R2: isotropic gradient of a periodic [ny][nx] field at node (x, y). */
void oracle_grad(const double *chi, int nx, int ny, int x, int y, double *out)
{
    double win[9];
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx)
            win[(dy + 1) * 3 + (dx + 1)] = chi[(size_t)wrap(y + dy, ny) * nx + wrap(x + dx, nx)];
    grad_window(win, out);
}

/* Prescribed velocity at node (x, y) and time t (Eq. 14 with R4, R5). */
void oracle_velocity(const oracle_params *p, int x, int y, double t, double *u, double *v)
{
    if (p->vel_kind == ORACLE_VORTEX) {
        double sx = sin(PI * x / p->nx), sy = sin(PI * y / p->ny);
        double ct = cos(PI * t / p->T);
        *u = p->sign * p->U0 * sx * sx * sin(2.0 * PI * y / p->ny) * ct;
        *v = -p->sign * p->U0 * sy * sy * sin(2.0 * PI * x / p->nx) * ct;
    } else if (p->vel_kind == ORACLE_UNIFORM) {
        *u = p->ux;
        *v = p->uy;
    } else {
        size_t k = (size_t)y * p->nx + x;
        *u = p->ufield[k];
        *v = p->vfield[k];
    }
}

/* R7: f_i = f_i^eq(phi0, u(x, 0)), phi_prev = phi0. */
void oracle_init(const oracle_params *p, const double *phi0, double *f, double *phi_prev)
{
    size_t n = (size_t)p->nx * p->ny;
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            size_t k = (size_t)y * p->nx + x;
            double u, v, feq[9];
            oracle_velocity(p, x, y, 0.0, &u, &v);
            oracle_feq(phi0[k], u, v, feq);
            for (int i = 0; i < 9; ++i) f[i * n + k] = feq[i];
            phi_prev[k] = phi0[k];
        }
}

/* Eq. 12 at every node. */
void oracle_phi(const oracle_params *p, const double *f, double *phi)
{
    size_t n = (size_t)p->nx * p->ny;
    for (size_t k = 0; k < n; ++k) {
        double s = 0.0;
        for (int i = 0; i < 9; ++i) s += f[i * n + k];
        phi[k] = s;
    }
}

/* Global mass sum_x sum_i f_i, Neumaier-compensated. */
double oracle_mass(const oracle_params *p, const double *f)
{
    size_t n = 9 * (size_t)p->nx * p->ny;
    double s = 0.0, c = 0.0;
    for (size_t k = 0; k < n; ++k) {
        double a = f[k], t = s + a;
        if (fabs(s) >= fabs(a))
            c += (s - t) + a;
        else
            c += (a - t) + s;
        s = t;
    }
    return s + c;
}

/* Post-collision populations at node (x, y) of a state at time t (Eqs. 9-13).
 * phi_c = phi(x, t) (Eq. 12); chiw = the 3x3 window of chi around the node,
 * chi = psi (Eq. 13) for the modified ACE, chi = phi for the R8 ablation. */
static void collide_node(const oracle_params *p, const double *f, const double *phi_prev,
                         double phi_c, const double *chiw, long long t, int x, int y,
                         double *fstar)
{
    size_t n = (size_t)p->nx * p->ny;
    size_t k = (size_t)y * p->nx + x;

    double g[2];
    grad_window(chiw, g);
    double norm = sqrt(g[0] * g[0] + g[1] * g[1]);
    double nxv = g[0] / (norm + p->delta), nyv = g[1] / (norm + p->delta); /* Eq. 13 */

    double S;
    if (p->model == ORACLE_MODIFIED)
        S = oracle_sharpen(chiw[4], p->eps); /* Eqs. 6, 11 under R1 */
    else
        S = phi_c * (1.0 - phi_c) / p->eps; /* Eq. 1 under R1, R8 */

    double u, v, up, vp;
    oracle_velocity(p, x, y, (double)t, &u, &v);
    oracle_velocity(p, x, y, (double)(t - 1), &up, &vp);
    double dx = 0.0, dy = 0.0; /* R3 */
    if (t > 0) {
        dx = phi_c * u - phi_prev[k] * up;
        dy = phi_c * v - phi_prev[k] * vp;
    }
    double gx = dx + CS2 * S * nxv, gy = dy + CS2 * S * nyv; /* bracket of Eq. 11 */

    double feq[9], F[9];
    oracle_feq(phi_c, u, v, feq);
    oracle_forcing(gx, gy, F);
    for (int i = 0; i < 9; ++i) {
        double fi = f[i * n + k];
        fstar[i] = fi - (fi - feq[i]) / p->tau + (1.0 - 1.0 / (2.0 * p->tau)) * F[i]; /* Eq. 9 */
    }
}

static double chi_of(const oracle_params *p, double phi)
{
    return p->model == ORACLE_MODIFIED ? oracle_psi(phi, p->eps, p->delta) : phi;
}

/* Advance the state (f at time t0, phi_prev = phi(t0 - 1)) by nsteps steps,
 * with up to nthreads OpenMP threads over rows. Returns 0, or -1 when scratch
 * memory cannot be had. */
int oracle_step(const oracle_params *p, double *f, double *phi_prev, long long t0,
                long long nsteps, int nthreads)
{
    size_t n = (size_t)p->nx * p->ny;
    double *phi = malloc(n * sizeof(double));
    double *chi = malloc(n * sizeof(double));
    double *fnew = malloc(9 * n * sizeof(double));
    if (!phi || !chi || !fnew) {
        free(phi);
        free(chi);
        free(fnew);
        return -1;
    }
    if (nthreads < 1) nthreads = 1;
    for (long long s = 0; s < nsteps; ++s) {
        long long t = t0 + s;
        oracle_phi(p, f, phi); /* Eq. 12 */
#pragma omp parallel for num_threads(nthreads) schedule(static)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t k = (size_t)y * p->nx + x;
                chi[k] = chi_of(p, phi[k]);
            }
#pragma omp parallel for num_threads(nthreads) schedule(static)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double chiw[9], fstar[9];
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx)
                        chiw[(dy + 1) * 3 + (dx + 1)] =
                            chi[(size_t)wrap(y + dy, p->ny) * p->nx + wrap(x + dx, p->nx)];
                collide_node(p, f, phi_prev, phi[(size_t)y * p->nx + x], chiw, t, x, y, fstar);
                for (int i = 0; i < 9; ++i) { /* streaming, left side of Eq. 9 */
                    size_t dst = (size_t)wrap(y + CY[i], p->ny) * p->nx + wrap(x + CX[i], p->nx);
                    fnew[i * n + dst] = fstar[i];
                }
            }
        memcpy(phi_prev, phi, n * sizeof(double));
        memcpy(f, fnew, 9 * n * sizeof(double));
    }
    free(phi);
    free(chi);
    free(fnew);
    return 0;
}

/* phi at node (x, y) from the populations there (Eq. 12). */
static double phi_at(const oracle_params *p, const double *f, int x, int y)
{
    size_t n = (size_t)p->nx * p->ny;
    size_t k = (size_t)wrap(y, p->ny) * p->nx + wrap(x, p->nx);
    double s = 0.0;
    for (int i = 0; i < 9; ++i) s += f[i * n + k];
    return s;
}

/* One step evaluated only where it is asked for. For each of the ncells nodes
 * (xs[j], ys[j]) of a state at time t0, writes phi(x, t0) and the populations
 * f_i(x, t0 + 1) after streaming, i.e. the post-collision value of node
 * x - c_i. Used to check very large lattices at sampled nodes. Returns -1 on a
 * node outside the lattice. */
int oracle_step_cells(const oracle_params *p, const double *f, const double *phi_prev,
                      long long t0, int ncells, const int *xs, const int *ys,
                      double *fnext /* [ncells][9] */, double *phi_out /* [ncells] */)
{
    for (int j = 0; j < ncells; ++j) {
        int x = xs[j], y = ys[j];
        if (x < 0 || x >= p->nx || y < 0 || y >= p->ny) return -1;
        phi_out[j] = phi_at(p, f, x, y);
        for (int i = 0; i < 9; ++i) {
            int sx = wrap(x - CX[i], p->nx), sy = wrap(y - CY[i], p->ny);
            double chiw[9], fstar[9];
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    chiw[(dy + 1) * 3 + (dx + 1)] = chi_of(p, phi_at(p, f, sx + dx, sy + dy));
            collide_node(p, f, phi_prev, phi_at(p, f, sx, sy), chiw, t0, sx, sy, fstar);
            fnext[(size_t)j * 9 + i] = fstar[i];
        }
    }
    return 0;
}

/*
 * lbm_oracle_d2q7.c -- the paper's own lattice, D2Q7 (triangular), as a plain,
 * slow CPU oracle of the active lattice Boltzmann update of arXiv:1902.00530.
 *
 * TEST INFRASTRUCTURE ONLY, under the same rules as lbm_oracle.c (which it is
 * linked with, for Philox4x32-10, the seeded initial uniforms and the u*
 * closures, all of which are independent of the lattice).  It shares no code
 * with the CUDA path.
 *
 * Lattice (Sec. 2): e_0 = 0 and e_i = (cos((i-1) pi/3), sin((i-1) pi/3)) for
 * i = 1..6, weights w_0 = 1/2, w_i = 1/12, c_s^2 = 1/4, c = dx = dt = 1.  (The
 * printed angle step reads pi/6; only pi/3 gives the triangular lattice the
 * section names, and the explicit gradient stencils of Sec. 3, whose y
 * spacing is dy = sqrt(3)/2 dx, hold for pi/3.)  Opposite pairs 1-4, 2-5, 3-6
 * (App. A.3 item 2).
 *
 * Box: a rectangle of nx x ny sites with periodic boundaries (App. C, "180 x 60
 * node triangular lattice").  Site (x, y) sits at the point
 *     X = x + (y mod 2)/2,   Y = y sqrt(3)/2,
 * i.e. rows are dy = sqrt(3)/2 apart and every odd row is shifted right by
 * half a spacing.  ny must be even so that the wrap in y keeps that pattern.
 * The neighbour r + e_i of a site is found from these positions (X + e_ix,
 * Y + e_iy), not from a stored offset table.
 *
 * Layout: f[i][y][x], i = 0..6, x fastest.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef REAL
#define REAL double
#endif
typedef REAL real;

/* Row loops on several host threads in the -fopenmp build (see lbm_oracle.c:
 * per-site arithmetic and order unchanged, so results are thread-count
 * independent). */
#ifdef _OPENMP
#define ORC_PARALLEL_ROWS _Pragma("omp parallel for schedule(static)")
#define ORC_PARALLEL_PLANES_ROWS _Pragma("omp parallel for collapse(2) schedule(static)")
#else
#define ORC_PARALLEL_ROWS
#define ORC_PARALLEL_PLANES_ROWS
#endif

#define Q7 7

/* shared with lbm_oracle.c (same library) */
typedef struct {
    double tau, sigma, C, rho_star, u_max, A, B;
} orc_params;
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_init_uniforms(uint64_t seed, uint32_t x, uint32_t y, uint32_t id, double u[4]);
void orc_ustar(int model, const orc_params *p, real rho, real ux, real uy, const real g[2], real us[2]);
int orc_observables_from_moments(const double *rho, const double *ux, const double *uy, int nx, int ny,
                                 double B, double out[6]);

enum { ORC_MIPS = 1 };

/* e_i in units of half a spacing along x (2 e_ix) and in rows along y
 * (e_iy / (sqrt(3)/2)): both are integers on this lattice. */
static const int E2X[Q7] = {0, 2, 1, -1, -2, -1, 1};
static const int ERY[Q7] = {0, 0, 1, 1, 0, -1, -1};
static const int OPP7[Q7] = {0, 4, 5, 6, 1, 2, 3};

static real ex7(int i) { return (real)E2X[i] / (real)2; }
static real ey7(int i) { return (real)ERY[i] * (real)sqrt(3.0) / (real)2; }

static real weight7(int i) { return i == 0 ? (real)1 / (real)2 : (real)1 / (real)12; }

static int wrap7(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

/* The site at r + s e_i (s = +1 or -1) of site (x, y): go to the doubled x
 * position 2X = 2x + (y mod 2), add s 2 e_ix, move s e_iy rows, and read the
 * column index back from the new row's offset. */
void orc7_neighbour(int x, int y, int i, int s, int nx, int ny, int *xn, int *yn)
{
    int y2 = y + s * ERY[i];
    int par_y = wrap7(y, 2), par_y2 = wrap7(y2, 2);
    int twice_x = 2 * x + par_y + s * E2X[i];
    int xi = (twice_x - par_y2) / 2; /* exact: twice_x - par_y2 is even */
    *xn = wrap7(xi, nx);
    *yn = wrap7(y2, ny);
}

#define AT7(arr, i, y, x) arr[((size_t)(i) * (size_t)ny + (size_t)(y)) * (size_t)nx + (size_t)(x)]

/* Eq. (fssD2Q7): f^SS_i = w_i rho [1 + 4 e_i.u + 8 (e_i.u)^2 - 2 |u|^2]. */
void orc7_equilibrium(real rho, real ux, real uy, real out[Q7])
{
    real usq = ux * ux + uy * uy;
    for (int i = 0; i < Q7; ++i) {
        real eu = ex7(i) * ux + ey7(i) * uy;
        out[i] = weight7(i) * rho * ((real)1 + (real)4 * eu + (real)8 * eu * eu - (real)2 * usq);
    }
}

/* App. A.3 with the D2Q7 pairs: f_0 < 0 -> 0; for i = 1..6 in index order a
 * negative f_i goes to its reverse direction and f_i becomes 0; then rescale
 * to rho if anything changed. */
int orc7_negative_correction(real f[Q7], real rho)
{
    int changed = 0;
    if (f[0] < 0) {
        f[0] = 0;
        changed = 1;
    }
    for (int i = 1; i < Q7; ++i) {
        if (f[i] < 0) {
            f[OPP7[i]] += -f[i];
            f[i] = 0;
            changed = 1;
        }
    }
    if (changed) {
        real sum = 0;
        for (int i = 0; i < Q7; ++i) sum += f[i];
        for (int i = 0; i < Q7; ++i) f[i] = f[i] * (rho / sum);
    }
    return changed;
}

/* Sec. 3 explicit stencils with rho_i = rho(r + e_i), dx = 1, dy = sqrt(3)/2:
 *   d rho/dx = [2 (rho_1 - rho_4) + (rho_2 + rho_6) - (rho_3 + rho_5)] / (6 dx)
 *   d rho/dy = [(rho_2 + rho_3) - (rho_5 + rho_6)] / (4 dy)                    */
void orc7_gradient(const real *rho, int nx, int ny, int x, int y, real g[2])
{
    real r[Q7];
    for (int i = 1; i < Q7; ++i) {
        int xn, yn;
        orc7_neighbour(x, y, i, +1, nx, ny, &xn, &yn);
        r[i] = rho[(size_t)yn * nx + xn];
    }
    real dx = 1, dy = (real)sqrt(3.0) / (real)2;
    g[0] = ((real)2 * (r[1] - r[4]) + (r[2] + r[6]) - (r[3] + r[5])) / ((real)6 * dx);
    g[1] = ((r[2] + r[3]) - (r[5] + r[6])) / ((real)4 * dy);
}

/* The seven noise variates s_i of a site and step: one Philox call with the
 * collision-noise counter (x, y, t, id | 0 << 24 | 0 << 28), key = seed; the
 * 16-bit halves h_0..h_6 of its output (h_2j = low half of word j) give
 * s_i = (2 h_i + 1 - 2^16) / 2^16, odd multiples of 2^-16 in (-1, 1), exact in
 * FP32 and FP64.  eta~_i = sigma s_i (Sec. 2, uniform on [-sigma, sigma]). */
void orc7_noise_variates(uint64_t seed, uint32_t x, uint32_t y, uint32_t t, uint32_t id, double s[Q7])
{
    uint32_t ctr[4] = {x, y, t, id & 0xFFFFFFu};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    for (int i = 0; i < Q7; ++i) {
        uint32_t h = (i % 2 == 0) ? (w[i / 2] & 0xFFFFu) : (w[i / 2] >> 16);
        s[i] = (2.0 * (double)h + 1.0 - 65536.0) / 65536.0;
    }
}

/* One step t -> t+1 (App. A.2 steps 1-6) on the D2Q7 lattice, as in
 * lbm_oracle.c's orc_step_window: the arrays are an nx x ny window at (x_off,
 * y_off) of a gnx x gny box, which only the noise counters see.  y_off and gny
 * must be even (the brick offsets).  Returns 0, -1 on allocation failure, -2
 * on an odd ny, y_off or gny. */
int orc7_step_window(const real *fin, real *fout, int nx, int ny, int model, const orc_params *p, uint64_t seed,
                     uint32_t t, uint32_t id, int x_off, int y_off, int gnx, int gny)
{
    if (ny % 2 || y_off % 2 || gny % 2) return -2;
    size_t n = (size_t)nx * (size_t)ny;
    real *fs = (real *)malloc(sizeof(real) * Q7 * n);
    real *rho = (real *)malloc(sizeof(real) * n);
    real *ux = (real *)malloc(sizeof(real) * n);
    real *uy = (real *)malloc(sizeof(real) * n);
    if (!fs || !rho || !ux || !uy) {
        free(fs); free(rho); free(ux); free(uy);
        return -1;
    }
    /* 1. streaming: f*_i(r) = f_i(r - e_i) */
    ORC_PARALLEL_PLANES_ROWS
    for (int i = 0; i < Q7; ++i)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int xs, ys;
                orc7_neighbour(x, y, i, -1, nx, ny, &xs, &ys);
                AT7(fs, i, y, x) = AT7(fin, i, ys, xs);
            }
    /* 2. rho and u of f* (Eq. (D2Q7macroscopic_u_disc)) */
    ORC_PARALLEL_ROWS
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            real r = 0, jx = 0, jy = 0;
            for (int i = 0; i < Q7; ++i) {
                real fi = AT7(fs, i, y, x);
                r += fi;
                jx += fi * ex7(i);
                jy += fi * ey7(i);
            }
            size_t c = (size_t)y * nx + x;
            rho[c] = r;
            ux[c] = r > 0 ? jx / r : (real)0;
            uy[c] = r > 0 ? jy / r : (real)0;
        }
    real tau = (real)p->tau, sigma = (real)p->sigma;
    ORC_PARALLEL_ROWS
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            /* 3. u* and f^SS */
            real g[2] = {0, 0};
            if (model == ORC_MIPS) orc7_gradient(rho, nx, ny, x, y, g);
            real us[2];
            orc_ustar(model, p, rho[c], ux[c], uy[c], g, us);
            real feq[Q7];
            orc7_equilibrium(rho[c], us[0], us[1], feq);
            /* 4. redistribution */
            real f[Q7];
            for (int i = 0; i < Q7; ++i) {
                real fi = AT7(fs, i, y, x);
                f[i] = fi - (fi - feq[i]) / tau;
            }
            /* 5. noise, Eq. (noiseDensityConservation) with 1/7 */
            if (sigma > 0) {
                double s[Q7];
                orc7_noise_variates(seed, (uint32_t)wrap7(x + x_off, gnx), (uint32_t)wrap7(y + y_off, gny), t, id,
                                    s);
                real et[Q7], mean = 0;
                for (int i = 0; i < Q7; ++i) {
                    et[i] = sigma * (real)s[i];
                    mean += et[i];
                }
                mean = mean / (real)Q7;
                for (int i = 0; i < Q7; ++i) f[i] += et[i] - mean;
            }
            /* 6. negative correction */
            orc7_negative_correction(f, rho[c]);
            for (int i = 0; i < Q7; ++i) AT7(fout, i, y, x) = f[i];
        }
    free(fs); free(rho); free(ux); free(uy);
    return 0;
}

int orc7_run_window(real *f, int nx, int ny, int model, const orc_params *p, uint64_t seed, uint32_t t0,
                    int64_t nsteps, uint32_t id, int x_off, int y_off, int gnx, int gny)
{
    size_t bytes = sizeof(real) * Q7 * (size_t)nx * (size_t)ny;
    real *tmp = (real *)malloc(bytes);
    if (!tmp) return -1;
    for (int64_t k = 0; k < nsteps; ++k) {
        int rc = orc7_step_window(f, tmp, nx, ny, model, p, seed, t0 + (uint32_t)k, id, x_off, y_off, gnx, gny);
        if (rc != 0) {
            free(tmp);
            return rc;
        }
        memcpy(f, tmp, bytes);
    }
    free(tmp);
    return 0;
}

/* Initial state (App. C.2) on D2Q7: the same seeded rho and u as
 * orc_init_window (same uniforms, same u_kind recipes) with f_i = f^SS_i of
 * Eq. (fssD2Q7), in FP64. */
void orc7_init_window(real *f, int nx, int ny, uint64_t seed, uint32_t id, double rho_mean, double rho_amp,
                      int u_kind, double u_amp, double ux0, double uy0, const orc_params *p, int x_off, int y_off,
                      int gnx, int gny)
{
    const double two_pi = 6.283185307179586476925286766559;
    const double hs3 = sqrt(3.0) / 2.0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double U[4];
            orc_init_uniforms(seed, (uint32_t)wrap7(x + x_off, gnx), (uint32_t)wrap7(y + y_off, gny), id, U);
            double r = rho_mean * (1.0 + rho_amp * (2.0 * U[0] - 1.0));
            double vx, vy;
            if (u_kind == 0) {
                vx = ux0 + u_amp * (2.0 * U[1] - 1.0);
                vy = uy0 + u_amp * (2.0 * U[2] - 1.0);
            } else if (u_kind == 1) {
                vx = ux0 + u_amp * cos(two_pi * U[1]);
                vy = uy0 + u_amp * sin(two_pi * U[1]);
            } else {
                double a_r2 = p->A * r * r;
                double U0 = (p->B >= a_r2) ? p->B - a_r2 : 0.0;
                vx = U0 * cos(two_pi * U[1]);
                vy = U0 * sin(two_pi * U[1]);
            }
            double usq = vx * vx + vy * vy;
            for (int i = 0; i < Q7; ++i) {
                double w = i == 0 ? 0.5 : 1.0 / 12.0;
                double eu = 0.5 * E2X[i] * vx + hs3 * ERY[i] * vy;
                AT7(f, i, y, x) = (real)(w * r * (1.0 + 4.0 * eu + 8.0 * eu * eu - 2.0 * usq));
            }
        }
}

void orc7_from_moments(real *f, int nx, int ny, const double *rho, const double *ux, const double *uy)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            real feq[Q7];
            orc7_equilibrium((real)rho[c], (real)ux[c], (real)uy[c], feq);
            for (int i = 0; i < Q7; ++i) AT7(f, i, y, x) = feq[i];
        }
}

/* rho and u of every site (Eq. (D2Q7macroscopic_u_disc)), in FP64. */
void orc7_moments(const real *f, int nx, int ny, double *rho, double *ux, double *uy)
{
    const double hs3 = sqrt(3.0) / 2.0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double r = 0, jx = 0, jy = 0;
            for (int i = 0; i < Q7; ++i) {
                double fi = (double)AT7(f, i, y, x);
                r += fi;
                jx += fi * 0.5 * E2X[i];
                jy += fi * hs3 * ERY[i];
            }
            size_t c = (size_t)y * nx + x;
            rho[c] = r;
            ux[c] = r > 0 ? jx / r : 0.0;
            uy[c] = r > 0 ? jy / r : 0.0;
        }
}

/* The observables of lbm_oracle.c on a D2Q7 state.  rho_y(x) averages the
 * sites of column index x (App. D's average over y; a column zigzags by half
 * a spacing between rows). */
int orc7_observables(const real *f, int nx, int ny, double B, double out[6])
{
    size_t n = (size_t)nx * (size_t)ny;
    double *rho = (double *)malloc(sizeof(double) * n);
    double *ux = (double *)malloc(sizeof(double) * n);
    double *uy = (double *)malloc(sizeof(double) * n);
    if (!rho || !ux || !uy) {
        free(rho); free(ux); free(uy);
        return -1;
    }
    orc7_moments(f, nx, ny, rho, ux, uy);
    int rc = orc_observables_from_moments(rho, ux, uy, nx, ny, B, out);
    free(rho); free(ux); free(uy);
    return rc;
}

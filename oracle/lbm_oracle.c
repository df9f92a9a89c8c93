/*
 * lbm_oracle.c -- plain, slow, obviously-correct CPU implementation of the
 * active lattice Boltzmann update of Nesbitt, Pruessner & Lee,
 * "Uncovering novel phase transitions in dense dry polar active fluids using a
 * lattice Boltzmann method" (arXiv:1902.00530).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA path is checked
 * against.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant with the
 * CUDA path; the two sides are written independently from the paper.
 *
 * Precision: compiled twice, with REAL=double (the oracle proper) and with
 * REAL=float (used only to measure the intrinsic FP32 divergence of linearly
 * unstable runs).  No blocking, fusion or reordering: every function below is
 * the paper's step written out on a full lattice, in the paper's order.
 *
 * Lattice.  The paper's lattice is D2Q7 (Sec. 2); this oracle lifts every
 * formula to D2Q9 through the lattice weights w_i and the sound speed
 * c_s^2 = 1/3:  f^SS_i = w_i rho [1 + (e.ustar)/c_s^2 + (e.ustar)^2/(2 c_s^4)
 * - |ustar|^2/(2 c_s^2)], which is Eq. (fssD2Q7) when w, c_s^2 are D2Q7's.
 *
 * Layout: structure of arrays f[i][y][x], i = 0..8, x fastest, periodic.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef REAL
#define REAL double
#endif
typedef REAL real;

/* Row loops of the step may run on several host threads (the build with
 * -fopenmp): every site writes only its own outputs and its arithmetic is the
 * same sequence in the same order, so the result does not depend on the
 * thread count.  Without OpenMP the pragma is empty. */
#ifdef _OPENMP
#include <omp.h>
#define ORC_PARALLEL_ROWS _Pragma("omp parallel for schedule(static)")
#define ORC_PARALLEL_PLANES_ROWS _Pragma("omp parallel for collapse(2) schedule(static)")
#else
#define ORC_PARALLEL_ROWS
#define ORC_PARALLEL_PLANES_ROWS
#endif

/* Host threads the step loops use (1 in a build without OpenMP); n > 0 sets
 * the count first. */
int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

#define Q 9

/* D2Q9 velocity set, weights and opposite directions (Sec. 2 lifted to D2Q9;
 * opposite pairs as in App. A.3 item 2). */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

static real weight(int i)
{
    if (i == 0) return (real)4 / (real)9;
    if (i <= 4) return (real)1 / (real)9;
    return (real)1 / (real)36;
}

enum { ORC_PASSIVE = 0, ORC_MIPS = 1, ORC_CIL = 2 };

typedef struct {
    double tau;      /* relaxation time, Eq. (fevolution2)                    */
    double sigma;    /* noise amplitude: eta~ uniform on [-sigma, sigma]      */
    double C;        /* MIPS gradient sensitivity, Eq. (bu_mips)              */
    double rho_star; /* MIPS density ceiling, Eq. (bu_mips)                   */
    double u_max;    /* MIPS speed clamp, Sec. 3                              */
    double A, B;     /* CIL U0 = max(B - A rho^2, 0), Eq. (U0)                */
} orc_params;

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  Written from the published definition: each round
 * multiplies counter words 0 and 2 by the two round multipliers, takes the
 * high and low halves of the 64-bit products, and mixes the high halves with
 * the other counter words and the key; the key is bumped by the two Weyl
 * constants between rounds.
 * ---------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout shared by definition (not by code) with the GPU path:
 *   word 0 = x, word 1 = y, word 2 = t (the step being taken, t -> t+1),
 *   word 3 = lattice id (bits 0..23) | purpose (bits 24..27) | call (28..31).
 * purpose 0 = collision noise, purpose 1 = initial state.
 * key = (seed low 32 bits, seed high 32 bits). */
static void draw(uint64_t seed, uint32_t x, uint32_t y, uint32_t t, uint32_t id,
                 uint32_t purpose, uint32_t call, uint32_t out[4])
{
    uint32_t ctr[4] = {x, y, t, (id & 0xFFFFFFu) | (purpose << 24) | (call << 28)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* The nine noise variates s_i in (-1, 1) of one site and step, from one
 * Philox call (call index 0): each of the four 32-bit words w_j gives two
 * 14-bit integers, its top bits 18..31 (variate 2j) and its bits 4..17
 * (variate 2j+1); variate 8 gathers the words' low bits, bits 0..3 of w_0,
 * w_1, w_2 (in that order from its lowest bit) and bits 0..1 of w_3.
 * s = (2m + 1 - 2^14) / 2^14 for the 14-bit integer m: an odd multiple of
 * 2^-14, exact in FP32 and FP64 and symmetric about 0, so eta~_i = sigma * s_i
 * is uniform on [-sigma, sigma] (Sec. 2, below Eq. (noiseDensityConservation))
 * to 14 bits. */
void orc_noise_variates(uint64_t seed, uint32_t x, uint32_t y, uint32_t t, uint32_t id,
                        double s[Q])
{
    uint32_t w[4];
    draw(seed, x, y, t, id, 0u, 0u, w);
    uint32_t m[Q];
    for (int j = 0; j < 4; ++j) {
        m[2 * j] = w[j] >> 18;
        m[2 * j + 1] = (w[j] >> 4) & 0x3FFFu;
    }
    m[8] = (w[0] & 0xFu) | ((w[1] & 0xFu) << 4) | ((w[2] & 0xFu) << 8) | ((w[3] & 0x3u) << 12);
    for (int i = 0; i < Q; ++i) s[i] = (2.0 * (double)m[i] + 1.0 - 16384.0) / 16384.0;
}

/* Four uniforms U_j in (0, 1) for the initial state of a site:
 * U = (m + 1/2) / 2^24 with m the top 24 bits of a Philox word. */
void orc_init_uniforms(uint64_t seed, uint32_t x, uint32_t y, uint32_t id, double u[4])
{
    uint32_t w[4];
    draw(seed, x, y, 0u, id, 1u, 0u, w);
    for (int j = 0; j < 4; ++j) u[j] = ((double)(w[j] >> 8) + 0.5) / 16777216.0;
}

/* ------------------------------------------------------------------------
 * Steady-state distribution xi_i(rho, u) (Eq. (fssD2Q7) / App. B "xi"),
 * in its D2Q9 form with c_s^2 = 1/3:  w_i rho [1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u^2].
 * ---------------------------------------------------------------------- */
void orc_equilibrium(real rho, real ux, real uy, real out[Q])
{
    real usq = ux * ux + uy * uy;
    for (int i = 0; i < Q; ++i) {
        real eu = (real)EX[i] * ux + (real)EY[i] * uy;
        out[i] = weight(i) * rho *
                 ((real)1 + (real)3 * eu + (real)4.5 * eu * eu - (real)1.5 * usq);
    }
}

/* Negative correction, App. A.3: f_0 < 0 -> 0; for i = 1..8 in index order,
 * f_i < 0 -> add |f_i| to the opposite population and zero f_i; then, if
 * anything changed, rescale all f_i by rho / sum f. */
int orc_negative_correction(real f[Q], real rho)
{
    int changed = 0;
    if (f[0] < 0) {
        f[0] = 0;
        changed = 1;
    }
    for (int i = 1; i < Q; ++i) {
        if (f[i] < 0) {
            f[OPP[i]] += -f[i];
            f[i] = 0;
            changed = 1;
        }
    }
    if (changed) {
        real sum = 0;
        for (int i = 0; i < Q; ++i) sum += f[i];
        for (int i = 0; i < Q; ++i) f[i] = f[i] * (rho / sum);
    }
    return changed;
}

static int wrap(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

#define AT(arr, i, y, x) arr[((size_t)(i) * (size_t)ny + (size_t)(y)) * (size_t)nx + (size_t)(x)]

/* Isotropic finite-difference gradient of a scalar field (Sec. 3, the
 * stencil "grad rho = a sum (rho_i - rho_{i+3}) e_i", a = 1/(3 dx)), written
 * in its lattice-general form (1/c_s^2) sum_i w_i rho(r + e_i) e_i, which is
 * the paper's stencil on D2Q7 and 3 sum_i w_i rho(r + e_i) e_i on D2Q9. */
void orc_gradient(const real *rho, int nx, int ny, int x, int y, real g[2])
{
    real gx = 0, gy = 0;
    for (int i = 1; i < Q; ++i) {
        real r = rho[(size_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx)];
        gx += weight(i) * r * (real)EX[i];
        gy += weight(i) * r * (real)EY[i];
    }
    g[0] = (real)3 * gx;
    g[1] = (real)3 * gy;
}

/* Steady-state velocity u* of one site (Sec. 2 "u* a function of rho and u"):
 *   PASSIVE  u* = u (standard LBM, App. A.1);
 *   MIPS     u* = C (1 - rho/rho*) grad rho if rho < rho*, else 0, then
 *            |u*| -> min(|u*|, U_max) keeping the direction (Eq. (bu_mips));
 *   CIL      u* = U0(rho) u/|u|, U0 = B - A rho^2 if B >= A rho^2 else 0
 *            (Eqs. (bu_CIL), (U0)); u* = 0 where |u| = 0. */
void orc_ustar(int model, const orc_params *p, real rho, real ux, real uy, const real g[2],
               real us[2])
{
    if (model == ORC_PASSIVE) {
        us[0] = ux;
        us[1] = uy;
    } else if (model == ORC_MIPS) {
        real rs = (real)p->rho_star;
        if (rho < rs) {
            real c = (real)p->C * ((real)1 - rho / rs);
            us[0] = c * g[0];
            us[1] = c * g[1];
        } else {
            us[0] = 0;
            us[1] = 0;
        }
        real mag = sqrt(us[0] * us[0] + us[1] * us[1]);
        if (mag > (real)p->u_max) {
            us[0] = us[0] * ((real)p->u_max / mag);
            us[1] = us[1] * ((real)p->u_max / mag);
        }
    } else {
        real a_rho2 = (real)p->A * rho * rho;
        real U0 = ((real)p->B >= a_rho2) ? (real)p->B - a_rho2 : (real)0;
        real mag = sqrt(ux * ux + uy * uy);
        if (mag > 0) {
            us[0] = U0 * (ux / mag);
            us[1] = U0 * (uy / mag);
        } else {
            us[0] = 0;
            us[1] = 0;
        }
    }
}

/* One time step t -> t+1 of the whole lattice, App. A.2 steps 1-6:
 *  1 stream (pull form of f*_i(r + e_i) = f_i(r), periodic),
 *  2 rho, u from f*, 3 u* and f^SS, 4 BGK redistribution,
 *  5 zero-sum noise (Eq. (noiseDensityConservation)), 6 negative correction.
 * fin and fout are distinct [9][ny][nx] arrays.  Returns 0, or -1 on
 * allocation failure.
 *
 * Window form: the array is the nx x ny window at offset (x_off, y_off) of a
 * larger gnx x gny periodic lattice; only the noise counter sees the global
 * coordinates.  The window itself wraps periodically, so after k steps only
 * sites farther than k (2k for MIPS, whose gradient reads one more ring) from
 * the window edge equal the large lattice's values. */
int orc_step_window(const real *fin, real *fout, int nx, int ny, int model, const orc_params *p,
                    uint64_t seed, uint32_t t, uint32_t id, int x_off, int y_off, int gnx, int gny)
{
    size_t n = (size_t)nx * (size_t)ny;
    real *fs = (real *)malloc(sizeof(real) * Q * n);
    real *rho = (real *)malloc(sizeof(real) * n);
    real *ux = (real *)malloc(sizeof(real) * n);
    real *uy = (real *)malloc(sizeof(real) * n);
    if (!fs || !rho || !ux || !uy) {
        free(fs); free(rho); free(ux); free(uy);
        return -1;
    }
    /* 1. streaming */
    ORC_PARALLEL_PLANES_ROWS
    for (int i = 0; i < Q; ++i)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                AT(fs, i, y, x) = AT(fin, i, wrap(y - EY[i], ny), wrap(x - EX[i], nx));
    /* 2. moments of f* */
    ORC_PARALLEL_ROWS
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            real r = 0, jx = 0, jy = 0;
            for (int i = 0; i < Q; ++i) {
                real fi = AT(fs, i, y, x);
                r += fi;
                jx += fi * (real)EX[i];
                jy += fi * (real)EY[i];
            }
            size_t c = (size_t)y * nx + x;
            rho[c] = r;
            ux[c] = r > 0 ? jx / r : (real)0;
            uy[c] = r > 0 ? jy / r : (real)0;
        }
    real tau = (real)p->tau;
    real sigma = (real)p->sigma;
    ORC_PARALLEL_ROWS
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            /* 3. u* and f^SS */
            real g[2] = {0, 0};
            if (model == ORC_MIPS) orc_gradient(rho, nx, ny, x, y, g);
            real us[2];
            orc_ustar(model, p, rho[c], ux[c], uy[c], g, us);
            real feq[Q];
            orc_equilibrium(rho[c], us[0], us[1], feq);
            /* 4. redistribution f = f* - (f* - f^SS)/tau */
            real f[Q];
            for (int i = 0; i < Q; ++i) {
                real fi = AT(fs, i, y, x);
                f[i] = fi - (fi - feq[i]) / tau;
            }
            /* 5. noise: eta_i = eta~_i - (1/Q) sum_j eta~_j */
            if (sigma > 0) {
                double s[Q];
                orc_noise_variates(seed, (uint32_t)wrap(x + x_off, gnx), (uint32_t)wrap(y + y_off, gny),
                                   t, id, s);
                real et[Q], mean = 0;
                for (int i = 0; i < Q; ++i) {
                    et[i] = sigma * (real)s[i];
                    mean += et[i];
                }
                mean = mean / (real)Q;
                for (int i = 0; i < Q; ++i) f[i] += et[i] - mean;
            }
            /* 6. negative correction */
            orc_negative_correction(f, rho[c]);
            for (int i = 0; i < Q; ++i) AT(fout, i, y, x) = f[i];
        }
    free(fs); free(rho); free(ux); free(uy);
    return 0;
}

/* The whole periodic lattice: a window with no offset. */
int orc_step(const real *fin, real *fout, int nx, int ny, int model, const orc_params *p,
             uint64_t seed, uint32_t t, uint32_t id)
{
    return orc_step_window(fin, fout, nx, ny, model, p, seed, t, id, 0, 0, nx, ny);
}

/* n steps from t0, ping-ponging between f and a scratch copy; the result is
 * left in f.  Returns 0, or -1 on allocation failure. */
int orc_run_window(real *f, int nx, int ny, int model, const orc_params *p, uint64_t seed,
                   uint32_t t0, int64_t nsteps, uint32_t id, int x_off, int y_off, int gnx, int gny)
{
    size_t bytes = sizeof(real) * Q * (size_t)nx * (size_t)ny;
    real *tmp = (real *)malloc(bytes);
    if (!tmp) return -1;
    for (int64_t k = 0; k < nsteps; ++k) {
        if (orc_step_window(f, tmp, nx, ny, model, p, seed, t0 + (uint32_t)k, id, x_off, y_off, gnx,
                            gny) != 0) {
            free(tmp);
            return -1;
        }
        memcpy(f, tmp, bytes);
    }
    free(tmp);
    return 0;
}

int orc_run(real *f, int nx, int ny, int model, const orc_params *p, uint64_t seed,
            uint32_t t0, int64_t nsteps, uint32_t id)
{
    return orc_run_window(f, nx, ny, model, p, seed, t0, nsteps, id, 0, 0, nx, ny);
}

/* Initial state (App. C.2): per site draw uniforms, form rho and u, and set
 * f_i = xi_i(rho, u) = f^SS.  u_kind:
 *   0  u = (ux0, uy0) + u_amp (2U1 - 1, 2U2 - 1)       (componentwise noise)
 *   1  u = (ux0, uy0) + u_amp (cos 2 pi U1, sin 2 pi U1)  (random direction)
 *   2  u = U0(rho) (cos 2 pi U1, sin 2 pi U1)          (paper CIL init)
 * rho = rho_mean (1 + rho_amp (2U0 - 1)). */
void orc_init_window(real *f, int nx, int ny, uint64_t seed, uint32_t id, double rho_mean,
                     double rho_amp, int u_kind, double u_amp, double ux0, double uy0,
                     const orc_params *p, int x_off, int y_off, int gnx, int gny)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double U[4];
            orc_init_uniforms(seed, (uint32_t)wrap(x + x_off, gnx), (uint32_t)wrap(y + y_off, gny), id,
                              U);
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
            for (int i = 0; i < Q; ++i) {
                double w = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
                double eu = EX[i] * vx + EY[i] * vy;
                AT(f, i, y, x) = (real)(w * r * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq));
            }
        }
}

void orc_init(real *f, int nx, int ny, uint64_t seed, uint32_t id, double rho_mean,
              double rho_amp, int u_kind, double u_amp, double ux0, double uy0,
              const orc_params *p)
{
    orc_init_window(f, nx, ny, seed, id, rho_mean, rho_amp, u_kind, u_amp, ux0, uy0, p, 0, 0, nx,
                    ny);
}

/* Populations from given moment fields: f_i = xi_i(rho, u) per site. */
void orc_from_moments(real *f, int nx, int ny, const double *rho, const double *ux,
                      const double *uy)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            real feq[Q];
            orc_equilibrium((real)rho[c], (real)ux[c], (real)uy[c], feq);
            for (int i = 0; i < Q; ++i) AT(f, i, y, x) = feq[i];
        }
}

/* Density and velocity of every site (Eq. (D2Q7macroscopic) on D2Q9). */
void orc_moments(const real *f, int nx, int ny, double *rho, double *ux, double *uy)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double r = 0, jx = 0, jy = 0;
            for (int i = 0; i < Q; ++i) {
                double fi = (double)AT(f, i, y, x);
                r += fi;
                jx += fi * EX[i];
                jy += fi * EY[i];
            }
            size_t c = (size_t)y * nx + x;
            rho[c] = r;
            ux[c] = r > 0 ? jx / r : 0.0;
            uy[c] = r > 0 ? jy / r : 0.0;
        }
}

/* Observables of a stored state, accumulated in FP64:
 *  out[0] mass       = sum rho
 *  out[1] phi        = |sum rho u| / sum rho                (Eq. (phi))
 *  out[2] drho_y     = population std over x of rho_y(x) = (1/Ny) sum_y rho
 *                                                            (App. D)
 *  out[3] drho_x     = the same with the axes swapped
 *  out[4] var_rho    = population variance of rho over all sites
 *  out[5] zeta       = sum rho (B - |u|) / sum rho          (App. D)       */
int orc_observables_from_moments(const double *rho, const double *ux, const double *uy, int nx, int ny,
                                 double B, double out[6])
{
    size_t n = (size_t)nx * (size_t)ny;
    double *col = (double *)calloc((size_t)nx, sizeof(double));
    double *row = (double *)calloc((size_t)ny, sizeof(double));
    if (!col || !row) {
        free(col); free(row);
        return -1;
    }
    double m = 0, px = 0, py = 0, z = 0;
    for (size_t c = 0; c < n; ++c) {
        m += rho[c];
        px += rho[c] * ux[c];
        py += rho[c] * uy[c];
        z += rho[c] * (B - sqrt(ux[c] * ux[c] + uy[c] * uy[c]));
    }
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            col[x] += rho[(size_t)y * nx + x];
            row[y] += rho[(size_t)y * nx + x];
        }
    double mean = m / (double)n;
    double v = 0;
    for (size_t c = 0; c < n; ++c) v += (rho[c] - mean) * (rho[c] - mean);
    double sy = 0, sx = 0;
    for (int x = 0; x < nx; ++x) {
        double d = col[x] / ny - mean;
        sy += d * d;
    }
    for (int y = 0; y < ny; ++y) {
        double d = row[y] / nx - mean;
        sx += d * d;
    }
    out[0] = m;
    out[1] = sqrt(px * px + py * py) / m;
    out[2] = sqrt(sy / nx);
    out[3] = sqrt(sx / ny);
    out[4] = v / (double)n;
    out[5] = z / m;
    free(col); free(row);
    return 0;
}

int orc_observables(const real *f, int nx, int ny, double B, double out[6])
{
    size_t n = (size_t)nx * (size_t)ny;
    double *rho = (double *)malloc(sizeof(double) * n);
    double *ux = (double *)malloc(sizeof(double) * n);
    double *uy = (double *)malloc(sizeof(double) * n);
    if (!rho || !ux || !uy) {
        free(rho); free(ux); free(uy);
        return -1;
    }
    orc_moments(f, nx, ny, rho, ux, uy);
    int rc = orc_observables_from_moments(rho, ux, uy, nx, ny, B, out);
    free(rho); free(ux); free(uy);
    return rc;
}

/* Precision tag, so a loader can tell the two builds apart. */
int orc_real_bytes(void) { return (int)sizeof(real); }

// lbm_step.cuh -- the fused pull stream-collide kernel (one time step).
//
// Work decomposition: a lattice is cut into warp strips, 32*VEC columns wide
// and `rows` rows tall.  Lane l of a warp owns the VEC adjacent sites
// x0 = strip_x + l*VEC .. x0+VEC-1 of every row of its strip and walks the
// rows top to bottom.  For each row and population it issues one aligned
// vector load of VEC values; populations that stream along x (e_x = +-1) take
// the missing neighbour value from the adjacent lane with a warp shuffle, and
// only the strip's first / last lane issues one scalar load across the strip
// edge (with the periodic wrap).  Every population element is therefore read
// from HBM once per step and written once: 72 B per site update in FP32.
//
// MIPS needs grad rho of the post-stream density at the eight neighbours
// (Sec. 3 stencil, App. A.2 steps 2-3).  The warp keeps the post-stream
// density of rows y-1, y, y+1 in registers (a 3-row window that slides with
// the row loop, the populations of row y+1 pulled one row ahead) and obtains
// the x-neighbours by shuffles; only the two strip-edge sites of each row are
// recomputed by scalar pulls.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Pull row `y` of population I for this lane's VEC sites:
//   out[j] = f_I((x0 + j - e_x) mod nx, (y - e_y) mod ny).
template <int ST, int VEC, int I>
__device__ __forceinline__ void pull_pop(const typename Store<ST>::T *plane, int y, int ny,
                                         int nx, int pitch, int x0, bool valid, bool last,
                                         int lane, float shift, float out[VEC])
{
    const int r = wrap_once(y - vy(I), ny);
    const typename Store<ST>::T *row = plane + (size_t)r * pitch;
    float a[VEC];
    if (valid) {
        load_vec<ST, VEC>(row + x0, shift, a);
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) a[j] = 0.f;
    }
    if constexpr (vx(I) == 0) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) out[j] = a[j];
    } else if constexpr (vx(I) == 1) {  // from x - 1
        float left = __shfl_up_sync(FULL, a[VEC - 1], 1);
        if (lane == 0 && valid) left = load_one<ST>(row + (x0 == 0 ? nx - 1 : x0 - 1), shift);
        out[0] = left;
#pragma unroll
        for (int j = 1; j < VEC; ++j) out[j] = a[j - 1];
    } else {  // from x + 1
        float right = __shfl_down_sync(FULL, a[0], 1);
        if (last && valid) right = load_one<ST>(row + (x0 + VEC >= nx ? 0 : x0 + VEC), shift);
#pragma unroll
        for (int j = 0; j < VEC - 1; ++j) out[j] = a[j + 1];
        out[VEC - 1] = right;
    }
}

template <int ST, int VEC>
__device__ __forceinline__ void pull_row(const typename Store<ST>::T *base, size_t plane, int y,
                                         int ny, int nx, int pitch, int x0, bool valid, bool last,
                                         int lane, float rho0, float f[9][VEC])
{
    pull_pop<ST, VEC, 0>(base + 0 * plane, y, ny, nx, pitch, x0, valid, last, lane, wq(0) * rho0, f[0]);
    pull_pop<ST, VEC, 1>(base + 1 * plane, y, ny, nx, pitch, x0, valid, last, lane, wq(1) * rho0, f[1]);
    pull_pop<ST, VEC, 2>(base + 2 * plane, y, ny, nx, pitch, x0, valid, last, lane, wq(2) * rho0, f[2]);
    pull_pop<ST, VEC, 3>(base + 3 * plane, y, ny, nx, pitch, x0, valid, last, lane, wq(3) * rho0, f[3]);
    pull_pop<ST, VEC, 4>(base + 4 * plane, y, ny, nx, pitch, x0, valid, last, lane, wq(4) * rho0, f[4]);
    pull_pop<ST, VEC, 5>(base + 5 * plane, y, ny, nx, pitch, x0, valid, last, lane, wq(5) * rho0, f[5]);
    pull_pop<ST, VEC, 6>(base + 6 * plane, y, ny, nx, pitch, x0, valid, last, lane, wq(6) * rho0, f[6]);
    pull_pop<ST, VEC, 7>(base + 7 * plane, y, ny, nx, pitch, x0, valid, last, lane, wq(7) * rho0, f[7]);
    pull_pop<ST, VEC, 8>(base + 8 * plane, y, ny, nx, pitch, x0, valid, last, lane, wq(8) * rho0, f[8]);
}

template <int VEC>
__device__ __forceinline__ float density(const float f[9][VEC], int j)
{
    return ((f[0][j] + f[1][j]) + (f[2][j] + f[3][j])) + ((f[4][j] + f[5][j]) + (f[6][j] + f[7][j])) +
           f[8][j];
}

// Post-stream density of one site by nine scalar pulls (strip-edge halo),
// summed in the same order as density() so the result does not depend on
// where the strip edges fall.
template <int ST>
__device__ __forceinline__ float pulled_density(const typename Store<ST>::T *base, size_t plane,
                                                int x, int y, int nx, int ny, int pitch, float rho0)
{
    float v[9][1];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int xs = wrap_once(x - vx(i), nx), ys = wrap_once(y - vy(i), ny);
        v[i][0] = load_one<ST>(base + i * plane + (size_t)ys * pitch + xs, wq(i) * rho0);
    }
    return density<1>(v, 0);
}

// Density of this lane's VEC sites plus the two x-neighbours, for one row.
template <int ST, int VEC>
__device__ __forceinline__ void density_window(const float f[9][VEC], const typename Store<ST>::T *base,
                                               size_t plane, int y, int nx, int ny, int pitch, int x0,
                                               bool valid, bool last, int lane, float rho0,
                                               float r[VEC + 2])
{
#pragma unroll
    for (int j = 0; j < VEC; ++j) r[j + 1] = density<VEC>(f, j);
    float left = __shfl_up_sync(FULL, r[VEC], 1);
    float right = __shfl_down_sync(FULL, r[1], 1);
    if (lane == 0 && valid)
        left = pulled_density<ST>(base, plane, x0 == 0 ? nx - 1 : x0 - 1, y, nx, ny, pitch, rho0);
    if (last && valid)
        right = pulled_density<ST>(base, plane, x0 + VEC >= nx ? 0 : x0 + VEC, y, nx, ny, pitch, rho0);
    r[0] = left;
    r[VEC + 1] = right;
}

// Model parameters of one lattice, held in registers.
struct SiteParams {
    float omega, sigma_q, C, inv_rho_star, rho_star, u_max, u_max2, A, B;
};

__device__ __forceinline__ SiteParams load_params(const LatDesc *dp)
{
    SiteParams p;
    p.omega = dp->omega;
    p.sigma_q = dp->sigma_q;
    p.C = dp->C;
    p.inv_rho_star = dp->inv_rho_star;
    p.rho_star = dp->rho_star;
    p.u_max = dp->u_max;
    p.u_max2 = dp->u_max2;
    p.A = dp->A;
    p.B = dp->B;
    return p;
}

// The per-site update after streaming (App. A.2 steps 2-6).  f holds f* on
// entry and the new populations on exit.  (gx, gy) is the isotropic gradient
// of the post-stream density (MIPS only).  eta is the zero-sum noise.
template <int MODEL>
__device__ __forceinline__ void collide_site(float f[9], float gx, float gy, const SiteParams &d,
                                             bool noise, const float eta[9])
{
    // step 2: moments of f*
    const float rho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const float jx = (f[1] + f[5] + f[8]) - (f[3] + f[6] + f[7]);
    const float jy = (f[2] + f[5] + f[6]) - (f[4] + f[7] + f[8]);
    float ux = 0.f, uy = 0.f;
    if (rho > 0.f) {
        const float inv = __frcp_rn(rho);
        ux = jx * inv;
        uy = jy * inv;
    }
    // step 3: u* of the model
    float sx, sy;
    if constexpr (MODEL == MODEL_PASSIVE) {
        sx = ux;
        sy = uy;
    } else if constexpr (MODEL == MODEL_MIPS) {
        // Eq. (bu_mips): C (1 - rho/rho*) grad rho below rho*, then |u*| <= U_max
        const float c = rho < d.rho_star ? d.C * (1.f - rho * d.inv_rho_star) : 0.f;
        sx = c * gx;
        sy = c * gy;
        const float m2 = sx * sx + sy * sy;
        if (m2 > d.u_max2) {
            const float sc = d.u_max * rsqrtf(m2);
            sx *= sc;
            sy *= sc;
        }
    } else {
        // Eqs. (bu_CIL), (U0): U0(rho) u/|u|, U0 = max(B - A rho^2, 0)
        const float ar2 = d.A * rho * rho;
        const float U0 = d.B >= ar2 ? d.B - ar2 : 0.f;
        const float m2 = ux * ux + uy * uy;
        if (m2 > 0.f) {
            const float sc = U0 * rsqrtf(m2);
            sx = ux * sc;
            sy = uy * sc;
        } else {
            sx = 0.f;
            sy = 0.f;
        }
    }
    // step 3 (cont.): f^SS = w rho [1 + 3 e.u* + 9/2 (e.u*)^2 - 3/2 |u*|^2]
    // The rest population takes rho minus the moving ones: identical to
    // w_0 rho [1 - 3/2 |u*|^2] in exact arithmetic, but the FP32 weights sum
    // to 1 + 7.5e-9, which would otherwise change the mass by that much at
    // every collision.
    const float base = 1.f - 1.5f * (sx * sx + sy * sy);
    const float r1 = wq(1) * rho, r5 = wq(5) * rho;
    float eq[9];
    {
        const float tx = fmaf(4.5f * sx, sx, base), ty = fmaf(4.5f * sy, sy, base);
        eq[1] = r1 * fmaf(3.f, sx, tx);
        eq[3] = r1 * fmaf(-3.f, sx, tx);
        eq[2] = r1 * fmaf(3.f, sy, ty);
        eq[4] = r1 * fmaf(-3.f, sy, ty);
        const float p = sx + sy, m = sy - sx;
        const float tp = fmaf(4.5f * p, p, base), tm = fmaf(4.5f * m, m, base);
        eq[5] = r5 * fmaf(3.f, p, tp);
        eq[7] = r5 * fmaf(-3.f, p, tp);
        eq[6] = r5 * fmaf(3.f, m, tm);
        eq[8] = r5 * fmaf(-3.f, m, tm);
        eq[0] = rho - (((eq[1] + eq[3]) + (eq[2] + eq[4])) + ((eq[5] + eq[7]) + (eq[6] + eq[8])));
    }
    // step 4: BGK redistribution f = f* - (f* - f^SS)/tau
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = fmaf(d.omega, eq[i] - f[i], f[i]);
    // step 5: zero-sum noise eta_i = eta~_i - mean(eta~)
    if (noise) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] += eta[i];
    }
    // step 6: negative correction (App. A.3); a set sign bit flags a candidate
    const unsigned sg = (__float_as_uint(f[0]) | __float_as_uint(f[1]) | __float_as_uint(f[2])) |
                        (__float_as_uint(f[3]) | __float_as_uint(f[4]) | __float_as_uint(f[5])) |
                        (__float_as_uint(f[6]) | __float_as_uint(f[7]) | __float_as_uint(f[8]));
    if ((sg & 0x80000000u) &&
        fminf(fminf(fminf(f[0], f[1]), fminf(f[2], f[3])), fminf(fminf(f[4], f[5]), fminf(fminf(f[6], f[7]), f[8]))) <
            0.f) {
        if (f[0] < 0.f) f[0] = 0.f;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (f[i] < 0.f) {
                f[reverse_of(i)] += -f[i];
                f[i] = 0.f;
            }
        }
        const float s = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
        const float sc = rho * __frcp_rn(s);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] *= sc;
    }
}

// Observable sums of one stored row (sites x0..x0+VEC-1): per-thread FP64
// accumulators for the strip's column sums and five scalar sums, and the
// row's density total reduced over the warp.
template <int VEC>
__device__ __forceinline__ void observe_row(const float g[9][VEC], bool valid, double col[VEC],
                                            double acc[5], double *row_out, int lane)
{
    float rs = 0.f, js = 0.f, jxs = 0.f, jys = 0.f, r2s = 0.f;
    if (valid) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            const float r = density<VEC>(g, j);
            const float jx = (g[1][j] + g[5][j] + g[8][j]) - (g[3][j] + g[6][j] + g[7][j]);
            const float jy = (g[2][j] + g[5][j] + g[6][j]) - (g[4][j] + g[7][j] + g[8][j]);
            col[j] += (double)r;
            rs += r;
            jxs += jx;
            jys += jy;
            r2s += r * r;
            js += sqrtf(jx * jx + jy * jy);
        }
    }
    acc[0] += (double)rs;
    acc[1] += (double)jxs;
    acc[2] += (double)jys;
    acc[3] += (double)r2s;
    acc[4] += (double)js;
    double t = (double)rs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    if (lane == 0) *row_out = t;
}

template <int VEC>
__device__ __forceinline__ void observe_flush(double *colp, double *scal, int nx, int s, int sy, int x0,
                                              bool valid, const double col[VEC], double acc[5],
                                              int lane)
{
    if (valid) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) colp[(size_t)sy * nx + x0 + j] = col[j];
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(FULL, acc[q], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) scal[(size_t)s * 5 + q] = acc[q];
    }
}

__device__ __forceinline__ int find_lattice(const LatDesc *desc, int nlat, int block)
{
    int lo = 0, hi = nlat - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (desc[mid].block_begin <= block) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int MODEL, int ST, int VEC, bool SAMPLE>
__global__ void __launch_bounds__(256) step_kernel(const StepArgs a)
{
    using T = typename Store<ST>::T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const LatDesc *dp = a.desc + find_lattice(a.desc, a.nlat, blockIdx.x);
    const int nsx = dp->nsx, nsy = dp->nsy;
    const int s = (blockIdx.x - dp->block_begin) * (blockDim.x >> 5) + warp;
    if (s >= nsx * nsy) return;  // whole warp leaves together
    const int nx = dp->nx, ny = dp->ny, pitch = dp->pitch, rows = dp->rows;
    const SiteParams d = load_params(dp);
    const int sx = s % nsx, sy = s / nsx;
    const int x0 = sx * 32 * VEC + lane * VEC;
    const bool valid = x0 < nx;
    const bool last = (lane == 31) || (x0 + VEC >= nx);
    const int y_begin = sy * rows, y_end = min(y_begin + rows, ny);
    const size_t plane = (size_t)ny * pitch;
    const T *src = reinterpret_cast<const T *>(dp->f[a.src]);
    T *dst = reinterpret_cast<T *>(dp->f[a.src ^ 1]);
    const float rho0 = dp->rho0;
    const uint32_t id = (uint32_t)dp->id;
    const uint32_t t = *a.t_ptr + a.k;
    const bool noise = d.sigma_q > 0.f;

    double col[VEC], acc[5];
    if constexpr (SAMPLE) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) col[j] = 0.0;
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[q] = 0.0;
    }

    float fc[9][VEC];
    float rm[VEC + 2], rc[VEC + 2], rn[VEC + 2];
    if constexpr (MODEL == MODEL_MIPS) {
        float tmp[9][VEC];
        const int yp = wrap_once(y_begin - 1, ny);
        pull_row<ST, VEC>(src, plane, yp, ny, nx, pitch, x0, valid, last, lane, rho0, tmp);
        density_window<ST, VEC>(tmp, src, plane, yp, nx, ny, pitch, x0, valid, last, lane, rho0, rm);
        pull_row<ST, VEC>(src, plane, y_begin, ny, nx, pitch, x0, valid, last, lane, rho0, fc);
        density_window<ST, VEC>(fc, src, plane, y_begin, nx, ny, pitch, x0, valid, last, lane, rho0, rc);
    }

    for (int y = y_begin; y < y_end; ++y) {
        float fn[9][VEC];
        if constexpr (MODEL == MODEL_MIPS) {
            const int yn = wrap_once(y + 1, ny);
            pull_row<ST, VEC>(src, plane, yn, ny, nx, pitch, x0, valid, last, lane, rho0, fn);
            density_window<ST, VEC>(fn, src, plane, yn, nx, ny, pitch, x0, valid, last, lane, rho0, rn);
        } else {
            pull_row<ST, VEC>(src, plane, y, ny, nx, pitch, x0, valid, last, lane, rho0, fc);
        }
        float out[9][VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            float f[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = fc[i][j];
            float gx = 0.f, gy = 0.f;
            if constexpr (MODEL == MODEL_MIPS) {
                // 3 sum_i w_i rho(r + e_i) e_i (Sec. 3 isotropic stencil, D2Q9 form)
                const float e = rc[j + 2], w = rc[j];
                const float ne = rn[j + 2], nw = rn[j], se = rm[j + 2], sw = rm[j];
                gx = (1.f / 3.f) * (e - w) + (1.f / 12.f) * ((ne + se) - (nw + sw));
                gy = (1.f / 3.f) * (rn[j + 1] - rm[j + 1]) + (1.f / 12.f) * ((ne + nw) - (se + sw));
            }
            float eta[9];
            if (noise) noise_eta((uint32_t)(x0 + j), (uint32_t)y, t, id, a.rk, d.sigma_q, eta);
            collide_site<MODEL>(f, gx, gy, d, noise, eta);
#pragma unroll
            for (int i = 0; i < 9; ++i) out[i][j] = f[i];
        }
        if (valid) {
#pragma unroll
            for (int i = 0; i < 9; ++i)
                store_vec<ST, VEC>(dst + i * plane + (size_t)y * pitch + x0, wq(i) * rho0, out[i]);
        }
        if constexpr (SAMPLE) {
            // observables of the stored (rounded) state
            float g[9][VEC];
#pragma unroll
            for (int i = 0; i < 9; ++i)
#pragma unroll
                for (int j = 0; j < VEC; ++j)
                    g[i][j] = Store<ST>::get(Store<ST>::put(out[i][j], wq(i) * rho0), wq(i) * rho0);
            observe_row<VEC>(g, valid, col, acc, dp->rowp + (size_t)sx * ny + y, lane);
        }
        if constexpr (MODEL == MODEL_MIPS) {
#pragma unroll
            for (int i = 0; i < 9; ++i)
#pragma unroll
                for (int j = 0; j < VEC; ++j) fc[i][j] = fn[i][j];
#pragma unroll
            for (int j = 0; j < VEC + 2; ++j) {
                rm[j] = rc[j];
                rc[j] = rn[j];
            }
        }
    }
    if constexpr (SAMPLE) observe_flush<VEC>(dp->colp, dp->scal, nx, s, sy, x0, valid, col, acc, lane);
}

// Observable partials of the stored state without stepping (same strip
// layout and arithmetic as the sample steps).
template <int ST, int VEC>
__global__ void __launch_bounds__(256) observe_kernel(const StepArgs a)
{
    using T = typename Store<ST>::T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const LatDesc *dp = a.desc + find_lattice(a.desc, a.nlat, blockIdx.x);
    const int nsx = dp->nsx, nsy = dp->nsy;
    const int s = (blockIdx.x - dp->block_begin) * (blockDim.x >> 5) + warp;
    if (s >= nsx * nsy) return;
    const int nx = dp->nx, ny = dp->ny, pitch = dp->pitch, rows = dp->rows;
    const float rho0 = dp->rho0;
    const int sx = s % nsx, sy = s / nsx;
    const int x0 = sx * 32 * VEC + lane * VEC;
    const bool valid = x0 < nx;
    const int y_begin = sy * rows, y_end = min(y_begin + rows, ny);
    const size_t plane = (size_t)ny * pitch;
    const T *src = reinterpret_cast<const T *>(dp->f[a.src]);
    double col[VEC], acc[5];
#pragma unroll
    for (int j = 0; j < VEC; ++j) col[j] = 0.0;
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = 0.0;
    for (int y = y_begin; y < y_end; ++y) {
        float g[9][VEC];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (valid) {
                load_vec<ST, VEC>(src + i * plane + (size_t)y * pitch + x0, wq(i) * rho0, g[i]);
            } else {
#pragma unroll
                for (int j = 0; j < VEC; ++j) g[i][j] = 0.f;
            }
        }
        observe_row<VEC>(g, valid, col, acc, dp->rowp + (size_t)sx * ny + y, lane);
    }
    observe_flush<VEC>(dp->colp, dp->scal, nx, s, sy, x0, valid, col, acc, lane);
}

}  // namespace lbm



// lbm_step_q7.cuh -- the fused pull stream-collide step on the paper's own
// lattice, D2Q7 (Sec. 2): e_0 = 0, e_i = (cos((i-1) pi/3), sin((i-1) pi/3)),
// w_0 = 1/2, w_i = 1/12, f^SS_i = w_i rho [1 + 4 e.u* + 8 (e.u*)^2 - 2 |u*|^2]
// (Eq. (fssD2Q7)), the Sec. 3 explicit gradient stencils, and the App. A.3
// correction with the pairs 1-4, 2-5, 3-6.
//
// Box: nx x ny sites, periodic; site (x, y) sits at (x + (y mod 2)/2,
// y sqrt(3)/2), so every odd row is shifted right by half a spacing and ny is
// even.  In storage the seven populations are planes [7][ny][pitch] (28 B per
// site in FP32, 14 B in 16-bit), so a step moves 56 B (28 B) per site.
//
// Decomposition as in lbm_step.cuh: warp strips 32*VEC columns wide and
// `rows` (even) rows tall, lanes owning VEC adjacent sites, rows walked in
// (even, odd) pairs.  Streaming from the rows above and below shifts by half
// a spacing, which on this layout is a column offset of -1 or 0 from an even
// row and 0 or +1 from an odd one: with the row parity a template argument,
// every pull is a vector load plus at most one neighbour shuffle, as on D2Q9.
#pragma once

#include "lbm_step_persistent.cuh"

namespace lbm {

// Row of the source of population i relative to the destination row y:
// f*_i(r) = f_i(r - e_i) comes from row y - e_iy / (sqrt(3)/2).
__host__ __device__ constexpr int q7_src_dy(int i)
{
    return (i == 2 || i == 3) ? -1 : ((i == 5 || i == 6) ? 1 : 0);
}

// Column offset of that source for a destination row of parity P: the point
// r - e_i has x-coordinate X - e_ix with X = x + P/2, and the source row's
// sites sit at column + (1 - P)/2 (other rows) or column + P/2 (same row).
__host__ __device__ constexpr int q7_src_dx(int i, int P)
{
    return i == 1 ? -1 : i == 4 ? 1 : (i == 2 || i == 6) ? (P ? 0 : -1) : (i == 3 || i == 5) ? (P ? 1 : 0) : 0;
}

// Pull row y (parity P) of population I for this lane's VEC sites.
template <int ST, int VEC, int I, int P>
__device__ __forceinline__ void pull_pop7(const typename Store<ST>::T *plane, int y, int ny, int nx, int pitch,
                                          int x0, bool valid, bool last, int lane, float shift, float out[VEC])
{
    const int r = wrap_once(y + q7_src_dy(I), ny);
    const typename Store<ST>::T *row = plane + (size_t)r * pitch;
    float a[VEC];
    if (valid) {
        load_vec<ST, VEC>(row + x0, shift, a);
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) a[j] = 0.f;
    }
    constexpr int DX = q7_src_dx(I, P);
    if constexpr (DX == 0) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) out[j] = a[j];
    } else if constexpr (DX == -1) {
        float left = __shfl_up_sync(FULL, a[VEC - 1], 1);
        if (lane == 0 && valid) left = load_one<ST>(row + (x0 == 0 ? nx - 1 : x0 - 1), shift);
        out[0] = left;
#pragma unroll
        for (int j = 1; j < VEC; ++j) out[j] = a[j - 1];
    } else {
        float right = __shfl_down_sync(FULL, a[0], 1);
        if (last && valid) right = load_one<ST>(row + (x0 + VEC >= nx ? 0 : x0 + VEC), shift);
#pragma unroll
        for (int j = 0; j < VEC - 1; ++j) out[j] = a[j + 1];
        out[VEC - 1] = right;
    }
}

template <int ST, int VEC, int P>
__device__ __forceinline__ void pull_row7(const typename Store<ST>::T *base, size_t plane, int y, int ny, int nx,
                                          int pitch, int x0, bool valid, bool last, int lane, const Shift3 &sh,
                                          float f[7][VEC])
{
    pull_pop7<ST, VEC, 0, P>(base + 0 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q7(0), f[0]);
    pull_pop7<ST, VEC, 1, P>(base + 1 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q7(1), f[1]);
    pull_pop7<ST, VEC, 2, P>(base + 2 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q7(2), f[2]);
    pull_pop7<ST, VEC, 3, P>(base + 3 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q7(3), f[3]);
    pull_pop7<ST, VEC, 4, P>(base + 4 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q7(4), f[4]);
    pull_pop7<ST, VEC, 5, P>(base + 5 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q7(5), f[5]);
    pull_pop7<ST, VEC, 6, P>(base + 6 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q7(6), f[6]);
}

__device__ __forceinline__ float density7(const float f[7])
{
    return __fadd_rn(__fadd_rn(__fadd_rn(f[0], f[1]), __fadd_rn(f[2], f[3])),
                     __fadd_rn(__fadd_rn(f[4], f[5]), f[6]));
}

template <int VEC>
__device__ __forceinline__ float density7_at(const float f[7][VEC], int j)
{
    const float v[7] = {f[0][j], f[1][j], f[2][j], f[3][j], f[4][j], f[5][j], f[6][j]};
    return density7(v);
}

template <int ST, int VEC, int P>
__device__ __forceinline__ void density_window7(const float f[7][VEC], const typename Store<ST>::T *base,
                                                size_t plane, int y, int nx, int ny, int pitch, int x0, bool valid,
                                                bool last, int lane, const Shift3 &sh, float r[VEC + 2])
{
#pragma unroll
    for (int j = 0; j < VEC; ++j) r[j + 1] = density7_at<VEC>(f, j);
    float left = __shfl_up_sync(FULL, r[VEC], 1);
    float right = __shfl_down_sync(FULL, r[1], 1);
    // the sites just outside the strip: lanes 0..6 (left) and 16..22 (right)
    // pull one population each, summed by a shuffle tree in density7's order
    const int xs = x0 - lane * VEC, xe = min(xs + 32 * VEC, nx);
    const int i = lane & 15;
    float v = 0.f;
    if (i < 7) {
        const int xh = lane >= 16 ? (xe >= nx ? 0 : xe) : (xs == 0 ? nx - 1 : xs - 1);
        const int xsrc = wrap_once(xh + q7_src_dx(i, P), nx), ysrc = wrap_once(y + q7_src_dy(i), ny);
        v = load_one<ST>(base + i * plane + (size_t)ysrc * pitch + xsrc, sh.q7(i));
    }
    const float n1 = __shfl_down_sync(FULL, v, 1);
    const float s01 = i == 6 ? v : __fadd_rn(v, n1);                 // lanes 0, 2, 4: pairs; lane 6: f6
    const float s03 = __fadd_rn(s01, __shfl_down_sync(FULL, s01, 2)); // lanes 0, 4
    const float s06 = __fadd_rn(s03, __shfl_down_sync(FULL, s03, 4)); // lane 0
    const float halo_left = __shfl_sync(FULL, s06, 0), halo_right = __shfl_sync(FULL, s06, 16);
    if (lane == 0) left = halo_left;
    if (last) right = halo_right;
    r[0] = left;
    r[VEC + 1] = right;
}

// The Sec. 3 stencils at the lane's sites of a row of parity P, from the
// post-stream density windows of rows y-1 (rm), y (rc), y+1 (rn) (index j+1 is
// site j):  d/dx = [2 (rho_1 - rho_4) + (rho_2 + rho_6) - (rho_3 + rho_5)] / 6,
// d/dy = [(rho_2 + rho_3) - (rho_5 + rho_6)] / (4 sqrt(3)/2), rho_i = rho(r + e_i).
// The neighbours r + e_2, r + e_6 sit at column x + P, r + e_3, r + e_5 at
// column x + P - 1.
template <int VEC, int P>
__device__ __forceinline__ void mips_gradients7(const float rm[VEC + 2], const float rc[VEC + 2],
                                                const float rn[VEC + 2], float gx[VEC], float gy[VEC])
{
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        const float r1 = rc[j + 2], r4 = rc[j];
        const float r2 = rn[j + 1 + P], r3 = rn[j + P], r5 = rm[j + P], r6 = rm[j + 1 + P];
        gx[j] = __fmaf_rn(1.f / 3.f, __fsub_rn(r1, r4),
                          __fmul_rn(1.f / 6.f, __fsub_rn(__fadd_rn(r2, r6), __fadd_rn(r3, r5))));
        gy[j] = __fmul_rn(0.28867513459481287f, __fsub_rn(__fadd_rn(r2, r3), __fadd_rn(r5, r6)));
    }
}

constexpr float Q7_HALF_SQRT3 = 0.86602540378443865f;

// Steps 2-5 on one D2Q7 site; returns rho.  Same conventions as collide_v:
// explicit round-to-nearest operations; with noise, 1/tau and the noise shift
// folded into the equilibrium constants and each moving population updated
// as (1 - 1/tau) f* + (f^SS/tau + c + 2 sigma u_i); the rest population set to
// rho minus the new moving ones (the weights 1/12 are inexact in FP32).  u[i]
// are the site's noise uniforms (noise_u7), read only when noise is on.
template <int MODEL>
__device__ __forceinline__ float collide7(float f[7], float gx, float gy, const SiteParams &d, bool noise,
                                          const float u[7], const float *rho_known)
{
    const float rho = rho_known ? *rho_known : density7(f);
    const float jx = __fmaf_rn(0.5f, __fsub_rn(__fadd_rn(f[2], f[6]), __fadd_rn(f[3], f[5])), __fsub_rn(f[1], f[4]));
    const float jy = __fmul_rn(Q7_HALF_SQRT3, __fsub_rn(__fadd_rn(f[2], f[3]), __fadd_rn(f[5], f[6])));
    float sx, sy;
    ustar_v<MODEL, float>(rho, jx, jy, gx, gy, d, sx, sy);
    // e_1.u* = sx, e_2.u* = sx/2 + (sqrt3/2) sy, e_3.u* = (sqrt3/2) sy - sx/2;
    // e_4..e_6 are their negatives.  With r = R/12 folded into the constants,
    // each opposite pair is t = r (1 - 2|u*|^2) + c + 8 r (e.u*)^2 and
    // t +- 4 r e.u*, one multiply and three fused multiply-adds; R = rho and
    // c = 0 without noise, R = rho/tau and c = -2 sigma (sum_j u_j)/7 with it
    const float om = d.omega;
    const float base = __fmaf_rn(-2.f, __fmaf_rn(sx, sx, __fmul_rn(sy, sy)), 1.f);
    const float r12 = __fmul_rn(1.f / 12.f, noise ? __fmul_rn(om, rho) : rho);
    const float hy = __fmul_rn(Q7_HALF_SQRT3, sy), hx = __fmul_rn(0.5f, sx);
    const float a1 = sx, a2 = __fadd_rn(hy, hx), a3 = __fsub_rn(hy, hx);
    const float b = noise ? __fmaf_rn(r12, base, __fmul_rn(density7(u), -d.sigma_q * (1.f / 7.f)))
                          : __fmul_rn(r12, base);
    const float q = __fmul_rn(8.f, r12), k = __fmul_rn(4.f, r12);
    const float t1 = __fmaf_rn(__fmul_rn(q, a1), a1, b), t2 = __fmaf_rn(__fmul_rn(q, a2), a2, b),
                t3 = __fmaf_rn(__fmul_rn(q, a3), a3, b);
    float eq[7];
    eq[1] = __fmaf_rn(k, a1, t1);
    eq[4] = __fmaf_rn(-k, a1, t1);
    eq[2] = __fmaf_rn(k, a2, t2);
    eq[5] = __fmaf_rn(-k, a2, t2);
    eq[3] = __fmaf_rn(k, a3, t3);
    eq[6] = __fmaf_rn(-k, a3, t3);
    if (noise) {
#pragma unroll
        for (int i = 1; i < 7; ++i) f[i] = __fmaf_rn(d.omc, f[i], __fmaf_rn(d.sigma_q, u[i], eq[i]));
    } else {
#pragma unroll
        for (int i = 1; i < 7; ++i) f[i] = __fmaf_rn(om, __fsub_rn(eq[i], f[i]), f[i]);
    }
    // the rest population from the mass, as on D2Q9 (collide_v)
    f[0] = __fsub_rn(rho, __fadd_rn(__fadd_rn(__fadd_rn(f[1], f[4]), __fadd_rn(f[2], f[5])), __fadd_rn(f[3], f[6])));
    return rho;
}

// App. A.3 on D2Q7 (pairs disjoint, each settled lower index first).
__device__ __forceinline__ void negative_correction7(float f[7], float rho)
{
    const unsigned sg = (__float_as_uint(f[0]) | __float_as_uint(f[1]) | __float_as_uint(f[2])) |
                        (__float_as_uint(f[3]) | __float_as_uint(f[4]) | __float_as_uint(f[5])) |
                        __float_as_uint(f[6]);
    if (!(sg & 0x80000000u)) return;
    f[0] = fmaxf(f[0], 0.f);
    settle_pair(f[1], f[4]);
    settle_pair(f[2], f[5]);
    settle_pair(f[3], f[6]);
    const float sc = __fmul_rn(rho, __frcp_rn(density7(f)));
#pragma unroll
    for (int i = 0; i < 7; ++i) f[i] = __fmul_rn(f[i], sc);
}

// D2Q7 noise: one Philox call, the 16-bit halves h_0..h_6 as variates
// s_i = (2 h_i + 1 - 2^16) 2^-16 = 2 u_i - 3 with u_i = 1 + (h_i + 1/2) 2^-16
// built as FP32 bits; collide7 turns them into eta_i = 2 sigma (u_i - mean u)
// (their sum is exact there: seven multiples of 2^-17 below 2).
__device__ __forceinline__ void noise_u7(uint32_t x, uint32_t y, uint32_t t, uint32_t id, const uint32_t *rk,
                                         float u[7])
{
    const uint4 a = philox4x32_10_rk(make_uint4(x, y, t, id & 0xFFFFFFu), rk);
    const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        const uint32_t h7 = (i & 1) ? ((w[i >> 1] >> 9) & 0x007FFF80u) : ((w[i >> 1] << 7) & 0x007FFF80u);
        u[i] = __uint_as_float(0x3F800040u | h7);
    }
}

template <int VEC>
__device__ __forceinline__ void observe_row7(const float g[7][VEC], bool valid, double col[VEC], double acc[5],
                                             double *row_out, int lane)
{
    float rv[VEC], jxv[VEC], jyv[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        rv[j] = density7_at<VEC>(g, j);
        jxv[j] = (g[1][j] - g[4][j]) + 0.5f * ((g[2][j] + g[6][j]) - (g[3][j] + g[5][j]));
        jyv[j] = Q7_HALF_SQRT3 * ((g[2][j] + g[3][j]) - (g[5][j] + g[6][j]));
    }
    observe_moments<VEC>(rv, jxv, jyv, valid, col, acc, row_out, lane);
}

// Per-warp state of the row walk.
template <int VEC>
struct Q7Walk {
    float fc[7][VEC];                     // populations of the current row (MIPS: pulled one row ahead)
    float rm[VEC + 2], rc[VEC + 2], rn[VEC + 2];
    double col[VEC], acc[5];
};

template <int MODEL, int ST, int VEC, bool SAMPLE, int P>
__device__ __forceinline__ void q7_row(Q7Walk<VEC> &w, int y, const typename Store<ST>::T *src,
                                       typename Store<ST>::T *dst, size_t plane, int nx, int ny, int pitch, int x0,
                                       bool valid, bool last, int lane, const Shift3 &sh, const SiteParams &d, bool noise,
                                       uint32_t t, uint32_t id, const uint32_t *rk, double *rowp)
{
    float fn[7][VEC];
    if constexpr (MODEL == MODEL_MIPS) {
        const int yn = wrap_once(y + 1, ny);
        pull_row7<ST, VEC, 1 - P>(src, plane, yn, ny, nx, pitch, x0, valid, last, lane, sh, fn);
        density_window7<ST, VEC, 1 - P>(fn, src, plane, yn, nx, ny, pitch, x0, valid, last, lane, sh, w.rn);
    } else {
        pull_row7<ST, VEC, P>(src, plane, y, ny, nx, pitch, x0, valid, last, lane, sh, w.fc);
    }
    float gx[VEC], gy[VEC];
    if constexpr (MODEL == MODEL_MIPS) {
        mips_gradients7<VEC, P>(w.rm, w.rc, w.rn, gx, gy);
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) gx[j] = gy[j] = 0.f;
    }
    float out[7][VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        float g[7], u[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) g[i] = w.fc[i][j];
        if (noise) noise_u7((uint32_t)(x0 + j), (uint32_t)y, t, id, rk, u);
        const float rho = collide7<MODEL>(g, gx[j], gy[j], d, noise, u, MODEL == MODEL_MIPS ? &w.rc[j + 1] : nullptr);
        negative_correction7(g, rho);
#pragma unroll
        for (int i = 0; i < 7; ++i) out[i][j] = g[i];
    }
    if (valid) {
#pragma unroll
        for (int i = 0; i < 7; ++i) store_vec<ST, VEC>(dst + i * plane + (size_t)y * pitch + x0, sh.q7(i), out[i]);
    }
    if constexpr (SAMPLE) {
        float g[7][VEC];
#pragma unroll
        for (int i = 0; i < 7; ++i)
#pragma unroll
            for (int j = 0; j < VEC; ++j)
                g[i][j] = Store<ST>::get(Store<ST>::put(out[i][j], sh.q7(i)), sh.q7(i));
        observe_row7<VEC>(g, valid, w.col, w.acc, rowp + y, lane);
    }
    if constexpr (MODEL == MODEL_MIPS) {
#pragma unroll
        for (int i = 0; i < 7; ++i)
#pragma unroll
            for (int j = 0; j < VEC; ++j) w.fc[i][j] = fn[i][j];
#pragma unroll
        for (int j = 0; j < VEC + 2; ++j) {
            w.rm[j] = w.rc[j];
            w.rc[j] = w.rn[j];
        }
    }
}

// One warp's strip s (< nsx nsy) of D2Q7 lattice dp for the step at time t,
// read from buffer `src` and written to the other: the body of the direct
// D2Q7 kernel, shared by the per-step launch and the persistent launch.
template <int MODEL, int ST, int VEC, bool SAMPLE, int NOISE>
__device__ __forceinline__ void direct_strip_q7(const StepArgs &a, const LatDesc *dp, int s, int src_buf, uint32_t t)
{
    using T = typename Store<ST>::T;
    const int lane = threadIdx.x & 31;
    const int nsx = dp->nsx;
    const int nx = dp->nx, ny = dp->ny, pitch = dp->pitch, rows = dp->rows;
    const SiteParams d = load_params(dp);
    const int sx = s % nsx, sy = s / nsx;
    const int x0 = sx * 32 * VEC + lane * VEC;
    const bool valid = x0 < nx;
    const bool last = (lane == 31) || (x0 + VEC >= nx);
    // rows and ny are even, so every strip starts on an even row and holds whole (even, odd) pairs
    const int y_begin = sy * rows, y_end = min(y_begin + rows, ny);
    const size_t plane = (size_t)ny * pitch;
    const T *src = reinterpret_cast<const T *>(dp->f[src_buf]);
    T *dst = reinterpret_cast<T *>(dp->f[src_buf ^ 1]);
    const Shift3 sh = load_shift(dp);
    const uint32_t id = (uint32_t)dp->id;
    const bool noise = NOISE == 2 ? d.sigma_q > 0.f : NOISE == 1;  // as in step_kernel
    double *rowp = dp->rowp + (size_t)sx * ny;

    Q7Walk<VEC> w;
    if constexpr (SAMPLE) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) w.col[j] = 0.0;
#pragma unroll
        for (int q = 0; q < 5; ++q) w.acc[q] = 0.0;
    }
    if constexpr (MODEL == MODEL_MIPS) {
        float tmp[7][VEC];
        const int yp = wrap_once(y_begin - 1, ny);  // odd
        pull_row7<ST, VEC, 1>(src, plane, yp, ny, nx, pitch, x0, valid, last, lane, sh, tmp);
        density_window7<ST, VEC, 1>(tmp, src, plane, yp, nx, ny, pitch, x0, valid, last, lane, sh, w.rm);
        pull_row7<ST, VEC, 0>(src, plane, y_begin, ny, nx, pitch, x0, valid, last, lane, sh, w.fc);
        density_window7<ST, VEC, 0>(w.fc, src, plane, y_begin, nx, ny, pitch, x0, valid, last, lane, sh, w.rc);
    }
    for (int y = y_begin; y < y_end; y += 2) {
        q7_row<MODEL, ST, VEC, SAMPLE, 0>(w, y, src, dst, plane, nx, ny, pitch, x0, valid, last, lane, sh, d, noise,
                                          t, id, a.rk, rowp);
        q7_row<MODEL, ST, VEC, SAMPLE, 1>(w, y + 1, src, dst, plane, nx, ny, pitch, x0, valid, last, lane, sh, d,
                                          noise, t, id, a.rk, rowp);
    }
    if constexpr (SAMPLE) observe_flush<VEC>(dp->colp, dp->scal, nx, s, sy, x0, valid, w.col, w.acc, lane);
}

template <int MODEL, int ST, int VEC, bool SAMPLE, int NOISE>
__global__ void __launch_bounds__(256) step_kernel_q7(const StepArgs a)
{
    const LatDesc *dp = a.desc + find_lattice(a.desc, a.nlat, blockIdx.x);
    const int s = (blockIdx.x - dp->block_begin) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= dp->nsx * dp->nsy) return;  // whole warp leaves together
    direct_strip_q7<MODEL, ST, VEC, SAMPLE, NOISE>(a, dp, s, a.src, *a.t_ptr + a.k);
}

// The D2Q7 strip update of the persistent launch (lbm_step_persistent.cuh).
template <> struct PersistStrip<7> {
    template <int MODEL, int ST, int VEC, int NOISE>
    static __device__ __forceinline__ void run(const StepArgs &a, const LatDesc *dp, int s, int src, uint32_t t)
    {
        direct_strip_q7<MODEL, ST, VEC, false, NOISE>(a, dp, s, src, t);
    }
};

template <int ST, int VEC>
__global__ void __launch_bounds__(256) observe_kernel_q7(const StepArgs a)
{
    using T = typename Store<ST>::T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    const LatDesc *dp = a.desc + find_lattice(a.desc, a.nlat, blockIdx.x);
    const int nsx = dp->nsx, nsy = dp->nsy;
    const int bl = blockIdx.x - dp->block_begin;
    int sx, sy;
    if (a.stages > 0) {  // a staged group's blocks hold `warps` adjacent strips of one strip row
        const int ncx = (nsx + warps - 1) / warps;
        sx = (bl % ncx) * warps + warp;
        sy = bl / ncx;
        if (sx >= nsx) return;
    } else {
        const int s0 = bl * warps + warp;
        if (s0 >= nsx * nsy) return;
        sx = s0 % nsx;
        sy = s0 / nsx;
    }
    const int s = sy * nsx + sx;
    const int nx = dp->nx, ny = dp->ny, pitch = dp->pitch, rows = dp->rows;
    const Shift3 sh = load_shift(dp);
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
        float g[7][VEC];
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            if (valid) {
                load_vec<ST, VEC>(src + i * plane + (size_t)y * pitch + x0, sh.q7(i), g[i]);
            } else {
#pragma unroll
                for (int j = 0; j < VEC; ++j) g[i][j] = 0.f;
            }
        }
        observe_row7<VEC>(g, valid, col, acc, dp->rowp + (size_t)sx * ny + y, lane);
    }
    observe_flush<VEC>(dp->colp, dp->scal, nx, s, sy, x0, valid, col, acc, lane);
}

}  // namespace lbm

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
// the row loop; row y+1 is pulled one row ahead for its densities, and pulled
// again from cache when it is updated) and obtains the x-neighbours by
// shuffles; the two sites just outside the strip are pulled by 18 lanes at
// once, one population each.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Pull row `y` of population I for this lane's VEC sites:
//   out[j] = f_I((x0 + j - e_x) mod nx, (y - e_y) mod ny).
// Elements are addressed by their unsigned 32-bit index from the state base
// (i plane + row pitch + x): one wide multiply-add per address.  The host
// launches these kernels only on lattices whose q ny pitch elements fit.
template <int ST, int VEC, int I>
__device__ __forceinline__ void pull_pop(const typename Store<ST>::T *base, uint32_t plane, int y, int ny,
                                         int nx, int pitch, int x0, bool valid, bool last,
                                         int lane, float shift, float out[VEC])
{
    const uint32_t row = (uint32_t)I * plane + (uint32_t)wrap_once(y - vy(I), ny) * (uint32_t)pitch;
    float a[VEC];
    if (valid) {
        load_vec<ST, VEC>(base + (row + (uint32_t)x0), shift, a);
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) a[j] = 0.f;
    }
    if constexpr (vx(I) == 0) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) out[j] = a[j];
    } else if constexpr (vx(I) == 1) {  // from x - 1
        float left = __shfl_up_sync(FULL, a[VEC - 1], 1);
        if (lane == 0 && valid) left = load_one<ST>(base + (row + (uint32_t)(x0 == 0 ? nx - 1 : x0 - 1)), shift);
        out[0] = left;
#pragma unroll
        for (int j = 1; j < VEC; ++j) out[j] = a[j - 1];
    } else {  // from x + 1
        float right = __shfl_down_sync(FULL, a[0], 1);
        if (last && valid) right = load_one<ST>(base + (row + (uint32_t)(x0 + VEC >= nx ? 0 : x0 + VEC)), shift);
#pragma unroll
        for (int j = 0; j < VEC - 1; ++j) out[j] = a[j + 1];
        out[VEC - 1] = right;
    }
}

// All nine populations of row y.
template <int ST, int VEC>
__device__ __forceinline__ void pull_row(const typename Store<ST>::T *base, uint32_t plane, int y,
                                         int ny, int nx, int pitch, int x0, bool valid, bool last,
                                         int lane, const Shift3 &sh, float f[9][VEC])
{
    pull_pop<ST, VEC, 0>(base, plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(0), f[0]);
    pull_pop<ST, VEC, 1>(base, plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(1), f[1]);
    pull_pop<ST, VEC, 2>(base, plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(2), f[2]);
    pull_pop<ST, VEC, 3>(base, plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(3), f[3]);
    pull_pop<ST, VEC, 4>(base, plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(4), f[4]);
    pull_pop<ST, VEC, 5>(base, plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(5), f[5]);
    pull_pop<ST, VEC, 6>(base, plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(6), f[6]);
    pull_pop<ST, VEC, 7>(base, plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(7), f[7]);
    pull_pop<ST, VEC, 8>(base, plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(8), f[8]);
}

// The same with 64-bit pointer steps from a per-population plane pointer:
// the copy-bound noise-free kernels, where the 32-bit form costs registers.
template <int ST, int VEC, int I>
__device__ __forceinline__ void pull_pop_wide(const typename Store<ST>::T *plane, int y, int ny,
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
__device__ __forceinline__ void pull_row_wide(const typename Store<ST>::T *base, size_t plane, int y,
                                              int ny, int nx, int pitch, int x0, bool valid, bool last,
                                              int lane, const Shift3 &sh, float f[9][VEC])
{
    pull_pop_wide<ST, VEC, 0>(base + 0 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(0), f[0]);
    pull_pop_wide<ST, VEC, 1>(base + 1 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(1), f[1]);
    pull_pop_wide<ST, VEC, 2>(base + 2 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(2), f[2]);
    pull_pop_wide<ST, VEC, 3>(base + 3 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(3), f[3]);
    pull_pop_wide<ST, VEC, 4>(base + 4 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(4), f[4]);
    pull_pop_wide<ST, VEC, 5>(base + 5 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(5), f[5]);
    pull_pop_wide<ST, VEC, 6>(base + 6 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(6), f[6]);
    pull_pop_wide<ST, VEC, 7>(base + 7 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(7), f[7]);
    pull_pop_wide<ST, VEC, 8>(base + 8 * plane, y, ny, nx, pitch, x0, valid, last, lane, sh.q9(8), f[8]);
}

template <int VEC>
__device__ __forceinline__ float density(const float f[9][VEC], int j)
{
    return __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(f[0][j], f[1][j]), __fadd_rn(f[2][j], f[3][j])),
                               __fadd_rn(__fadd_rn(f[4][j], f[5][j]), __fadd_rn(f[6][j], f[7][j]))),
                     f[8][j]);
}

// Density of this lane's VEC sites plus the two x-neighbours, for one row.
// Inside the strip the neighbours come by shuffle.  The two sites just outside
// it (left of lane 0, right of the last lane) are pulled cooperatively: lanes
// 0..8 load one population each of the left site and lanes 16..24 of the right
// one, and a shuffle tree adds them in density()'s order (((f0+f1)+(f2+f3)) +
// ((f4+f5)+(f6+f7))) + f8, so the sums are bitwise those of a single-lane
// pull without its nine serial loads.
template <int ST, int VEC>
__device__ __forceinline__ void density_window(const float f[9][VEC], const typename Store<ST>::T *base,
                                               uint32_t plane, int y, int nx, int ny, int pitch, int x0,
                                               bool valid, bool last, int lane, const Shift3 &sh,
                                               float r[VEC + 2])
{
#pragma unroll
    for (int j = 0; j < VEC; ++j) r[j + 1] = density<VEC>(f, j);
    float left = __shfl_up_sync(FULL, r[VEC], 1);
    float right = __shfl_down_sync(FULL, r[1], 1);
    const int xs = x0 - lane * VEC, xe = min(xs + 32 * VEC, nx);  // the strip's columns
    const int i = lane & 15;
    float v = 0.f;
    if (i < 9) {
        const int xh = lane >= 16 ? (xe >= nx ? 0 : xe) : (xs == 0 ? nx - 1 : xs - 1);
        const int xsrc = wrap_once(xh - vx(i), nx), ysrc = wrap_once(y - vy(i), ny);
        v = load_one<ST>(base + ((uint32_t)i * plane + (uint32_t)ysrc * (uint32_t)pitch + (uint32_t)xsrc),
                         sh.q9(i));
    }
    const float s01 = __fadd_rn(v, __shfl_down_sync(FULL, v, 1));         // lanes 0, 2, 4, 6
    const float s03 = __fadd_rn(s01, __shfl_down_sync(FULL, s01, 2));     // lanes 0, 4
    const float s07 = __fadd_rn(s03, __shfl_down_sync(FULL, s03, 4));     // lane 0
    const float s08 = __fadd_rn(s07, __shfl_down_sync(FULL, v, 8));       // + f8
    const float halo_left = __shfl_sync(FULL, s08, 0), halo_right = __shfl_sync(FULL, s08, 16);
    if (lane == 0) left = halo_left;
    if (last) right = halo_right;
    r[0] = left;
    r[VEC + 1] = right;
}

// Model parameters of one lattice, held in registers.
struct SiteParams {
    float omega, omc, sigma_q, C, inv_rho_star, rho_star, u_max, u_max2, A, B;  // omc = 1 - omega
};

__device__ __forceinline__ SiteParams load_params(const LatDesc *dp)
{
    SiteParams p;
    p.omega = dp->omega;
    p.omc = __fsub_rn(1.f, dp->omega);  // exact: the host picks omega so
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

// ---------------------------------------------------------------------------
// The per-site update after streaming (App. A.2 steps 2-6).  Every arithmetic
// step is an explicit round-to-nearest operation (no compiler contraction),
// so a site's result does not depend on the launch shape that computed it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }

template <typename V> __device__ __forceinline__ V splat(float s);
template <> __device__ __forceinline__ float splat<float>(float s) { return s; }

// apply a scalar function (comparisons, selects, reciprocals)
template <typename F> __device__ __forceinline__ float vmap(float a, F fn) { return fn(a); }
template <typename F> __device__ __forceinline__ float vmap2(float a, float b, F fn) { return fn(a, b); }

// The same operations on two sites at once (V = float2): the paired FP32
// instructions of sm_100-class GPUs round each element exactly as the scalar
// instruction does (round to nearest; a - b is formed as a + (-b), which is
// the same number), so a site's result does not depend on whether it was
// computed alone or paired with a neighbour.
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __fadd2_rn(a, vneg(b)); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
template <> __device__ __forceinline__ float2 splat<float2>(float s) { return make_float2(s, s); }
template <typename F> __device__ __forceinline__ float2 vmap(float2 a, F fn) { return make_float2(fn(a.x), fn(a.y)); }
template <typename F> __device__ __forceinline__ float2 vmap2(float2 a, float2 b, F fn)
{
    return make_float2(fn(a.x, b.x), fn(a.y, b.y));
}

template <typename V>
__device__ __forceinline__ V vdensity(const V f[9])
{
    return vadd(vadd(vadd(vadd(f[0], f[1]), vadd(f[2], f[3])), vadd(vadd(f[4], f[5]), vadd(f[6], f[7]))), f[8]);
}

// Step 3: the steady-state velocity u* of the model from rho, the momentum
// j = rho u and (MIPS) grad rho; independent of the lattice.  Only the passive
// model needs u = j/rho itself: the MIPS u* does not depend on u, and the CIL
// u* only on its direction u/|u| = j/|j|.
template <int MODEL, typename V>
__device__ __forceinline__ void ustar_v(V rho, V jx, V jy, V gx, V gy, const SiteParams &d, V &sx, V &sy)
{
    if constexpr (MODEL == MODEL_PASSIVE) {
        const V inv = vmap(rho, [](float r) { return r > 0.f ? __frcp_rn(r) : 0.f; });  // u = 0 where rho <= 0
        sx = vmul(jx, inv);
        sy = vmul(jy, inv);
    } else if constexpr (MODEL == MODEL_MIPS) {
        // Eq. (bu_mips): C (1 - rho/rho*) grad rho below rho*, then |u*| <= U_max
        const V c0 = vmul(splat<V>(d.C), vfma(vsub(splat<V>(0.f), rho), splat<V>(d.inv_rho_star), splat<V>(1.f)));
        const float rs = d.rho_star;
        const V c = vmap2(c0, rho, [rs](float cc, float r) { return r < rs ? cc : 0.f; });
        sx = vmul(c, gx);
        sy = vmul(c, gy);
        const V m2 = vfma(sx, sx, vmul(sy, sy));
        const float um = d.u_max, um2 = d.u_max2;
        const V sc = vmap(m2, [um, um2](float q) { return q > um2 ? __fmul_rn(um, rsqrtf(q)) : 1.f; });
        sx = vmul(sx, sc);
        sy = vmul(sy, sc);
    } else {
        // Eqs. (bu_CIL), (U0): U0(rho) j/|j|, U0 = max(B - A rho^2, 0); u* = 0
        // where u = 0 (j = 0, or rho <= 0)
        const V ar2 = vmul(vmul(splat<V>(d.A), rho), rho);
        const float B = d.B;
        const V U0 = vmap2(ar2, rho, [B](float q, float r) { return (B >= q && r > 0.f) ? __fsub_rn(B, q) : 0.f; });
        const V m2 = vfma(jx, jx, vmul(jy, jy));
        const V sc = vmap2(U0, m2, [](float u0, float q) { return q > 0.f ? __fmul_rn(u0, rsqrtf(q)) : 0.f; });
        sx = vmul(jx, sc);
        sy = vmul(jy, sc);
    }
}

// Post-stream densities of a lane's VEC sites (out[j] = density of site j),
// two sites per paired instruction when PAIRED: the same sums in the same
// order as density().
template <int VEC, bool PAIRED>
__device__ __forceinline__ void densities(const float f[9][VEC], float *out)
{
    if constexpr (PAIRED) {
#pragma unroll
        for (int p = 0; p < VEC / 2; ++p) {
            float2 g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = make_float2(f[i][2 * p], f[i][2 * p + 1]);
            const float2 r = vdensity(g);
            out[2 * p] = r.x;
            out[2 * p + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) out[j] = density<VEC>(f, j);
    }
}

// Steps 2-5: moments of f*, u*, f^SS, BGK, noise.  Returns rho (for step 6).
// u[i] are the site's noise uniforms (noise_u), read only when noise is on.
template <int MODEL, typename V>
__device__ __forceinline__ V collide_v(V f[9], V gx, V gy, const SiteParams &d, bool noise, const V u[9],
                                       const V *rho_known = nullptr)
{
    // step 2: moments of f* (rho may come precomputed, bitwise equal: the MIPS
    // density window sums the same nine values in the same order)
    const V rho = rho_known ? *rho_known : vdensity(f);
    const V jx = vsub(vadd(vadd(f[1], f[5]), f[8]), vadd(vadd(f[3], f[6]), f[7]));
    const V jy = vsub(vadd(vadd(f[2], f[5]), f[6]), vadd(vadd(f[4], f[7]), f[8]));
    // step 3: u* of the model
    V sx, sy;
    ustar_v<MODEL, V>(rho, jx, jy, gx, gy, d, sx, sy);
    // step 3 (cont.): f^SS = w rho [1 + 3 e.u* + 9/2 (e.u*)^2 - 3/2 |u*|^2].  With
    // r = w R folded into the constants, each opposite pair (e.u* = +-a) is
    // t = r (1 - 3/2 |u*|^2) + c + (9/2) r a^2 and t +- 3 r a: one multiply and
    // three fused multiply-adds (r = R/9 on the axes, R/36 on the diagonals).
    // Without noise R = rho and c = 0, giving f^SS.  With noise R = rho/tau and c
    // is the shift of the zero-sum noise, eta_i = 2 sigma u_i + c with c = -2
    // sigma (sum_j u_j)/9 (the sum is exact: nine multiples of 2^-15 below 2),
    // giving f^SS/tau + c.  The rest population's f^SS_0 is not formed
    // (see below).
    const V om = splat<V>(d.omega);
    const V base = vfma(splat<V>(-1.5f), vfma(sx, sx, vmul(sy, sy)), splat<V>(1.f));
    const V R = noise ? vmul(om, rho) : rho;
    V b1, b5;
    if (noise) {
        const V c = vmul(vdensity(u), splat<V>(-d.sigma_q * (1.f / 9.f)));
        b1 = vfma(vmul(splat<V>(wq(1)), R), base, c);
        b5 = vfma(vmul(splat<V>(wq(5)), R), base, c);
    } else {
        b1 = vmul(vmul(splat<V>(wq(1)), R), base);
        b5 = vmul(vmul(splat<V>(wq(5)), R), base);
    }
    const V q1 = vmul(splat<V>(0.5f), R), q5 = vmul(splat<V>(0.125f), R);
    const V k1 = vmul(splat<V>(1.f / 3.f), R), k5 = vmul(splat<V>(1.f / 12.f), R);
    V eq[9];
    {
        const V p = vadd(sx, sy), m = vsub(sy, sx);
        const V tx = vfma(vmul(q1, sx), sx, b1), ty = vfma(vmul(q1, sy), sy, b1);
        const V tp = vfma(vmul(q5, p), p, b5), tm = vfma(vmul(q5, m), m, b5);
        eq[1] = vfma(k1, sx, tx);
        eq[3] = vfma(vneg(k1), sx, tx);
        eq[2] = vfma(k1, sy, ty);
        eq[4] = vfma(vneg(k1), sy, ty);
        eq[5] = vfma(k5, p, tp);
        eq[7] = vfma(vneg(k5), p, tp);
        eq[6] = vfma(k5, m, tm);
        eq[8] = vfma(vneg(k5), m, tm);
    }
    // step 4: BGK redistribution f = f* - (f* - f^SS)/tau, and step 5: the
    // zero-sum noise, for the eight moving populations.  With noise, as
    // (1 - 1/tau) f* + (f^SS/tau + c + 2 sigma u_i): two fused multiply-adds (the
    // mass is closed by the rest population below, so the form need not conserve
    // it); without, as f* + (f^SS - f*)/tau, which stays accurate near
    // equilibrium.
    if (noise) {
        const V omc = splat<V>(d.omc), ts = splat<V>(d.sigma_q);
#pragma unroll
        for (int i = 1; i < 9; ++i) f[i] = vfma(omc, f[i], vfma(ts, u[i], eq[i]));
    } else {
#pragma unroll
        for (int i = 1; i < 9; ++i) f[i] = vfma(om, vsub(eq[i], f[i]), f[i]);
    }
    // The rest population is rho minus the new moving ones.  Since sum_i f^SS_i
    // = rho and sum_i eta_i = 0, this equals f*_0 + eta_0 + (f^SS_0 - f*_0)/tau in
    // exact arithmetic; in FP32 it conserves the mass to one rounding (the
    // rounded weights w_i sum to 1 + 7.5e-9, so a separately formed f^SS_0 would
    // not), and the rest population, with e_0 = 0, takes the noise sum.  The
    // shift c enters the two members of an opposite pair through the same t,
    // so its rounding cancels in their difference and gives no momentum kick.
    f[0] = vsub(rho, vadd(vadd(vadd(f[1], f[3]), vadd(f[2], f[4])), vadd(vadd(f[5], f[7]), vadd(f[6], f[8]))));
    return rho;
}

// Step 6, the negative correction of App. A.3, for one site: f_0 < 0 -> 0;
// for i = 1..8 in index order, f_i < 0 moves |f_i| to the opposite population
// and zeroes f_i; if anything changed, rescale to rho.  The opposite pairs are
// disjoint, so each pair (i, j), i < j, is settled in closed form: the lower
// index first, then the upper.
__device__ __forceinline__ void settle_pair(float &a, float &b)
{
    const float na = fminf(a, 0.f);
    a = __fsub_rn(a, na);
    b = __fsub_rn(b, na);
    const float nb = fminf(b, 0.f);
    b = __fsub_rn(b, nb);
    a = __fsub_rn(a, nb);
}

// A population with its sign bit set is negative: round-to-nearest never
// produces -0 from the non-zero or +0 operands this update works with, so the
// sign bits decide "anything changed" exactly.
__device__ __forceinline__ void negative_correction(float f[9], float rho)
{
    const unsigned sg = (__float_as_uint(f[0]) | __float_as_uint(f[1]) | __float_as_uint(f[2])) |
                        (__float_as_uint(f[3]) | __float_as_uint(f[4]) | __float_as_uint(f[5])) |
                        (__float_as_uint(f[6]) | __float_as_uint(f[7]) | __float_as_uint(f[8]));
    if (!(sg & 0x80000000u)) return;
    f[0] = fmaxf(f[0], 0.f);
    settle_pair(f[1], f[3]);
    settle_pair(f[2], f[4]);
    settle_pair(f[5], f[7]);
    settle_pair(f[6], f[8]);
    const float s = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(f[0], f[1]), __fadd_rn(f[2], f[3])),
                                        __fadd_rn(__fadd_rn(f[4], f[5]), __fadd_rn(f[6], f[7]))),
                              f[8]);
    const float sc = __fmul_rn(rho, __frcp_rn(s));  // correctly rounded: an approximate one biases the mass
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = __fmul_rn(f[i], sc);
}

// The same for two sites at once.  A site with nothing negative must come out
// unchanged, as in the single-site form's early return: its settle steps
// subtract zeros (exact) and its rescale factor is exactly 1.
__device__ __forceinline__ void negative_correction2(float2 f[9], float2 rho)
{
    unsigned sa = 0u, sb = 0u;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        sa |= __float_as_uint(f[i].x);
        sb |= __float_as_uint(f[i].y);
    }
    if (!((sa | sb) & 0x80000000u)) return;
    f[0] = make_float2(fmaxf(f[0].x, 0.f), fmaxf(f[0].y, 0.f));
    auto settle2 = [](float2 &a, float2 &b) {
        const float2 na = make_float2(fminf(a.x, 0.f), fminf(a.y, 0.f));
        a = vsub(a, na);
        b = vsub(b, na);
        const float2 nb = make_float2(fminf(b.x, 0.f), fminf(b.y, 0.f));
        b = vsub(b, nb);
        a = vsub(a, nb);
    };
    settle2(f[1], f[3]);
    settle2(f[2], f[4]);
    settle2(f[5], f[7]);
    settle2(f[6], f[8]);
    const float2 s = vdensity(f);
    const float2 sc = make_float2((sa & 0x80000000u) ? __fmul_rn(rho.x, __frcp_rn(s.x)) : 1.f,
                                  (sb & 0x80000000u) ? __fmul_rn(rho.y, __frcp_rn(s.y)) : 1.f);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = vmul(f[i], sc);
}

// The noise uniforms of one site, u_i = 1 + (m_i + 1/2) 2^-14 (the variates
// are s_i = 2 u_i - 3); collide_v turns them into the zero-sum noise eta_i =
// 2 sigma (u_i - mean u).
__device__ __forceinline__ void noise_u(uint32_t x, uint32_t y, uint32_t t, uint32_t id, const uint32_t *rk,
                                        float u[9])
{
    const uint4 a = philox4x32_10_rk(make_uint4(x, y, t, id & 0xFFFFFFu), rk);
    const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        u[2 * j] = u_from_bits((w[j] >> 9) & 0x007FFE00u);      // bits 18..31
        u[2 * j + 1] = u_from_bits((w[j] << 5) & 0x007FFE00u);  // bits 4..17
    }
    const uint32_t m8 = (w[0] & 0xFu) | ((w[1] & 0xFu) << 4) | ((w[2] & 0xFu) << 8) | ((w[3] & 0x3u) << 12);
    u[8] = u_from_bits(m8 << 9);
}

// The update of a lane's VEC sites.  f[i][j] holds f*_i of site j on entry
// and the new f_i on exit; g*[j] are the MIPS gradients (ignored otherwise).
// With PAIRED (an even VEC) the sites go two at a time through paired FP32
// instructions (V = float2: half the arithmetic instructions, each element
// rounded as the single-site form rounds it), otherwise one at a time: every
// launch shape gives the same bits.  Measured at 8192^2 MIPS: the 16-bit
// storage kernels gain 5 % from pairing; the FP32 kernels lose 2-4 % (the
// paired temporaries spill at the register cap that their occupancy needs),
// so FP32 keeps single sites.
#ifndef LBM_PAIRED_F32
#define LBM_PAIRED_F32 0
#endif
#ifndef LBM_PAIRED_16
#define LBM_PAIRED_16 1
#endif
template <int ST, int VEC> __host__ __device__ constexpr bool paired_sites()
{
    return VEC % 2 == 0 && (ST == ST_F32 ? LBM_PAIRED_F32 != 0 : LBM_PAIRED_16 != 0);
}

template <int MODEL, int VEC, bool PAIRED>
__device__ __forceinline__ void collide_sites(float f[9][VEC], const float gxs[VEC], const float gys[VEC],
                                              const SiteParams &d, bool noise, uint32_t x0, uint32_t y, uint32_t t,
                                              uint32_t id, const uint32_t *rk, const float *rho_row = nullptr)
{
    if constexpr (PAIRED) {
#pragma unroll
        for (int p = 0; p < VEC / 2; ++p) {
            const int j0 = 2 * p, j1 = 2 * p + 1;
            float2 g[9], u[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = make_float2(f[i][j0], f[i][j1]);
            if (noise) {
                float ua[9], ub[9];
                noise_u(x0 + j0, y, t, id, rk, ua);
                noise_u(x0 + j1, y, t, id, rk, ub);
#pragma unroll
                for (int i = 0; i < 9; ++i) u[i] = make_float2(ua[i], ub[i]);
            }
            float2 rk2;
            if (rho_row) rk2 = make_float2(rho_row[j0], rho_row[j1]);
            const float2 rho = collide_v<MODEL, float2>(g, make_float2(gxs[j0], gxs[j1]), make_float2(gys[j0], gys[j1]),
                                                        d, noise, u, rho_row ? &rk2 : nullptr);
            negative_correction2(g, rho);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                f[i][j0] = g[i].x;
                f[i][j1] = g[i].y;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            float g[9], u[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = f[i][j];
            if (noise) noise_u(x0 + j, y, t, id, rk, u);
            const float rho = collide_v<MODEL, float>(g, gxs[j], gys[j], d, noise, u, rho_row ? rho_row + j : nullptr);
            negative_correction(g, rho);
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i][j] = g[i];
        }
    }
}

// The MIPS gradient 3 sum_i w_i rho(r + e_i) e_i at the lane's VEC sites from
// the density windows of rows y-1 (rm), y (rc), y+1 (rn): index j+1 is site j.
template <int VEC>
__device__ __forceinline__ void mips_gradients(const float rm[VEC + 2], const float rc[VEC + 2],
                                               const float rn[VEC + 2], float gx[VEC], float gy[VEC])
{
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        const float e = rc[j + 2], w = rc[j];
        const float ne = rn[j + 2], nw = rn[j], se = rm[j + 2], sw = rm[j];
        gx[j] = __fmaf_rn(1.f / 3.f, __fsub_rn(e, w),
                          __fmul_rn(1.f / 12.f, __fsub_rn(__fadd_rn(ne, se), __fadd_rn(nw, sw))));
        gy[j] = __fmaf_rn(1.f / 3.f, __fsub_rn(rn[j + 1], rm[j + 1]),
                          __fmul_rn(1.f / 12.f, __fsub_rn(__fadd_rn(ne, nw), __fadd_rn(se, sw))));
    }
}

// Observable sums of one stored row (sites x0..x0+VEC-1) from its moments
// rho and j = rho u: per-thread FP64 accumulators for the strip's column sums
// and five scalar sums, and the row's density total reduced over the warp.
// The sums that cancel (rho and rho^2 in the variance, j in the polar order of
// a nearly disordered state) are formed in FP64 from the lane's first site on
// (rho^2 exactly: a product of two FP32 values fits FP64), so they do not
// depend on how the launch shape groups sites into lanes beyond FP64 rounding;
// |j|, a sum of magnitudes, is summed in FP32 over the lane's sites.
// Lattice-independent.
template <int VEC>
__device__ __forceinline__ void observe_moments(const float rv[VEC], const float jxv[VEC], const float jyv[VEC],
                                                bool valid, double col[VEC], double acc[5], double *row_out,
                                                int lane)
{
    double rs = 0.0, jxs = 0.0, jys = 0.0, r2s = 0.0;
    float js = 0.f;
    if (valid) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            const float jx = jxv[j], jy = jyv[j];
            const double r = (double)rv[j];
            col[j] += r;
            rs += r;
            jxs += (double)jx;
            jys += (double)jy;
            r2s = __fma_rn(r, r, r2s);
            js += sqrtf(jx * jx + jy * jy);
        }
    }
    acc[0] += rs;
    acc[1] += jxs;
    acc[2] += jys;
    acc[3] += r2s;
    acc[4] += (double)js;
    double t = rs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    if (lane == 0) *row_out = t;
}

// The same for a stored D2Q9 row.
template <int VEC>
__device__ __forceinline__ void observe_row(const float g[9][VEC], bool valid, double col[VEC],
                                            double acc[5], double *row_out, int lane)
{
    float rv[VEC], jxv[VEC], jyv[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        rv[j] = density<VEC>(g, j);
        jxv[j] = (g[1][j] + g[5][j] + g[8][j]) - (g[3][j] + g[6][j] + g[7][j]);
        jyv[j] = (g[2][j] + g[5][j] + g[6][j]) - (g[4][j] + g[7][j] + g[8][j]);
    }
    observe_moments<VEC>(rv, jxv, jyv, valid, col, acc, row_out, lane);
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

// NOISE: 0 = no noise in any lattice of the launch, 1 = noise in all of them
// (both decided at compile time, so the per-site code has no branch around
// the generator), 2 = decided per lattice from sigma at run time.
// Minimum resident 256-thread blocks per SM the compiler must allow for,
// which caps registers per thread at 65536 / (256 * blocks): 128 for MIPS
// (its density window needs them), 85 for the other closures, where the
// extra occupancy hides more load latency (measured at 8192^2 FP32).  No cap
// where one would spill: sample steps (observables), 16-bit vec 8.
template <int MODEL, int ST, int VEC, bool SAMPLE> constexpr int direct_min_blocks()
{
    if (SAMPLE) return 1;
    if (ST != ST_F32 && VEC == 8) return 1;
    return MODEL == MODEL_MIPS ? 2 : 3;
}

// One warp's strip s (< nsx nsy) of lattice dp for the step at time t, read
// from buffer `src` and written to the other: the body of the direct kernel,
// shared by the per-step launch and the persistent launch.
template <int MODEL, int ST, int VEC, bool SAMPLE, int NOISE>
__device__ __forceinline__ void direct_strip(const StepArgs &a, const LatDesc *dp, int s, int src_buf, uint32_t t)
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
    const int y_begin = sy * rows, y_end = min(y_begin + rows, ny);
    const size_t plane = (size_t)ny * pitch;
    const uint32_t plane32 = (uint32_t)plane;  // q ny pitch <= 2^32 (host check) where used
    // 64-bit pointer steps only in the copy-bound noise-free kernels (see pull_pop_wide)
    constexpr bool WIDE = MODEL != MODEL_MIPS && NOISE == 0 && !SAMPLE;
    const T *src = reinterpret_cast<const T *>(dp->f[src_buf]);
    T *dst = reinterpret_cast<T *>(dp->f[src_buf ^ 1]);
    const Shift3 sh = load_shift(dp);
    const uint32_t id = (uint32_t)dp->id;
    const bool noise = NOISE == 2 ? d.sigma_q > 0.f : NOISE == 1;

    double col[VEC], acc[5];
    if constexpr (SAMPLE) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) col[j] = 0.0;
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[q] = 0.0;
    }

    // MIPS: the densities of rows y-1 and y slide along in registers; the
    // populations of row y are pulled again when row y is updated (they were
    // pulled one row earlier for its densities, so the loads hit L1 / L2)
    // rather than held across the collide of the row before: fewer registers,
    // more resident warps.
    float rm[VEC + 2], rc[VEC + 2], rn[VEC + 2];
    if constexpr (MODEL == MODEL_MIPS) {
        float tmp[9][VEC];
        const int yp = wrap_once(y_begin - 1, ny);
        pull_row<ST, VEC>(src, plane32, yp, ny, nx, pitch, x0, valid, last, lane, sh, tmp);
        density_window<ST, VEC>(tmp, src, plane32, yp, nx, ny, pitch, x0, valid, last, lane, sh, rm);
        pull_row<ST, VEC>(src, plane32, y_begin, ny, nx, pitch, x0, valid, last, lane, sh, tmp);
        density_window<ST, VEC>(tmp, src, plane32, y_begin, nx, ny, pitch, x0, valid, last, lane, sh, rc);
    }

    for (int y = y_begin; y < y_end; ++y) {
        // MIPS: prefetch into L2 the nine source-row segments of row y+2, which
        // the next iteration pulls first (one instruction per population, no
        // registers; the row's work covers the DRAM latency).  The lighter
        // closures run at the copy bandwidth, where the extra requests cost.
        if (MODEL == MODEL_MIPS && valid) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const T *pp = src + ((uint32_t)i * plane32 +
                                     (uint32_t)wrap_once(wrap_once(y + 2, ny) - vy(i), ny) * (uint32_t)pitch + (uint32_t)x0);
                asm volatile("prefetch.global.L2 [%0];" ::"l"(pp));
            }
        }
        float fc[9][VEC];
        if constexpr (MODEL == MODEL_MIPS) {
            float fn[9][VEC];
            const int yn = wrap_once(y + 1, ny);
            pull_row<ST, VEC>(src, plane32, yn, ny, nx, pitch, x0, valid, last, lane, sh, fn);
            density_window<ST, VEC>(fn, src, plane32, yn, nx, ny, pitch, x0, valid, last, lane, sh, rn);
        }
        if constexpr (WIDE)
            pull_row_wide<ST, VEC>(src, plane, y, ny, nx, pitch, x0, valid, last, lane, sh, fc);
        else
            pull_row<ST, VEC>(src, plane32, y, ny, nx, pitch, x0, valid, last, lane, sh, fc);
        float gx[VEC], gy[VEC];
        if constexpr (MODEL == MODEL_MIPS) {
            mips_gradients<VEC>(rm, rc, rn, gx, gy);
        } else {
#pragma unroll
            for (int j = 0; j < VEC; ++j) gx[j] = gy[j] = 0.f;
        }
        float out[9][VEC];
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int j = 0; j < VEC; ++j) out[i][j] = fc[i][j];
        collide_sites<MODEL, VEC, paired_sites<ST, VEC>()>(out, gx, gy, d, noise, (uint32_t)x0, (uint32_t)y, t, id, a.rk,
                                  MODEL == MODEL_MIPS ? rc + 1 : nullptr);
        if (valid) {
#pragma unroll
            for (int i = 0; i < 9; ++i)
                if constexpr (WIDE)
                    store_vec<ST, VEC>(dst + i * plane + (size_t)y * pitch + x0, sh.q9(i), out[i]);
                else
                    store_vec<ST, VEC>(dst + ((uint32_t)i * plane32 + (uint32_t)y * (uint32_t)pitch + (uint32_t)x0),
                                       sh.q9(i), out[i]);
        }
        if constexpr (SAMPLE) {
            // observables of the stored (rounded) state
            float g[9][VEC];
#pragma unroll
            for (int i = 0; i < 9; ++i)
#pragma unroll
                for (int j = 0; j < VEC; ++j)
                    g[i][j] = Store<ST>::get(Store<ST>::put(out[i][j], sh.q9(i)), sh.q9(i));
            observe_row<VEC>(g, valid, col, acc, dp->rowp + (size_t)sx * ny + y, lane);
        }
        if constexpr (MODEL == MODEL_MIPS) {
#pragma unroll
            for (int j = 0; j < VEC + 2; ++j) {
                rm[j] = rc[j];
                rc[j] = rn[j];
            }
        }
    }
    if constexpr (SAMPLE) observe_flush<VEC>(dp->colp, dp->scal, nx, s, sy, x0, valid, col, acc, lane);
}

template <int MODEL, int ST, int VEC, bool SAMPLE, int NOISE>
__global__ void __launch_bounds__(256, direct_min_blocks<MODEL, ST, VEC, SAMPLE>()) step_kernel(const StepArgs a)
{
    const LatDesc *dp = a.desc + find_lattice(a.desc, a.nlat, blockIdx.x);
    const int s = (blockIdx.x - dp->block_begin) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= dp->nsx * dp->nsy) return;  // whole warp leaves together
    direct_strip<MODEL, ST, VEC, SAMPLE, NOISE>(a, dp, s, a.src, *a.t_ptr + a.k);
}

// Observable partials of the stored state without stepping (same strip
// layout and arithmetic as the sample steps).
template <int ST, int VEC>
__global__ void __launch_bounds__(256) observe_kernel(const StepArgs a)
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
        float g[9][VEC];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (valid) {
                load_vec<ST, VEC>(src + i * plane + (size_t)y * pitch + x0, sh.q9(i), g[i]);
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



// lbm_step_q7_staged.cuh -- the D2Q7 step with bulk-copied population rows.
//
// The data movement of step_staged_kernel (lbm_step_staged.cuh) applied to the
// paper's triangular lattice: each warp owns a ring of `stages` shared-memory
// buffers; buffer q holds, for destination row r(q), the seven source-row
// segments it pulls from (row r + q7_src_dy(i) of population i), each covering
// the warp's 32*VEC columns plus 16 bytes of periodic halo on both sides, and
// arrives by cp.async.bulk copies completing on the buffer's mbarrier, issued
// rows ahead of use.  The half-site column offsets of the brick layout (-1/0
// from an even row, 0/+1 from an odd one) become shared-memory index offsets;
// rows are walked in (even, odd) pairs so the parity is a template argument.
// The per-site arithmetic is collide7 / negative_correction7 / noise_u7 of
// lbm_step_q7.cuh, so states are bitwise those of step_kernel_q7.
//
// Requirements (checked on the host): nx a multiple of the 16-byte halo width
// and at least that wide; rows even.  Every wait is bounded as in the D2Q9
// staged kernel (DEVERR_TIMEOUT, bounded drain, return).
#pragma once

#include <type_traits>

#include "lbm_step_q7.cuh"
#include "lbm_step_staged.cuh"

namespace lbm {

template <int ST, int VEC> struct StageGeom7 {
    using T = typename Store<ST>::T;
    static constexpr int HALO = 16 / (int)sizeof(T);
    static constexpr int W = 32 * VEC;
    static constexpr int SEG = W + 2 * HALO;
    static constexpr int STAGE_BYTES = 7 * SEG * (int)sizeof(T);
};

// Issue the segment copies of destination row y and arm the barrier: one copy
// per population (lanes 0..6) for a strip whose halos lie inside the row,
// else three (lanes 0..20: left halo, strip, right halo), as in issue_row.
template <int ST, int VEC>
__device__ __forceinline__ void issue_row7(typename Store<ST>::T *buf, uint64_t *bar, const typename Store<ST>::T *src,
                                           size_t plane, int pitch, int nx, int ny, int xs, int xe, int y, int lane)
{
    using G = StageGeom7<ST, VEC>;
    using T = typename Store<ST>::T;
    const uint32_t main_bytes = (uint32_t)(xe - xs) * (uint32_t)sizeof(T);
    __syncwarp();  // every lane has finished reading this buffer's previous row
    if (lane == 0) mbar_arrive_expect_tx(bar, 7u * (main_bytes + 32u));
    __syncwarp();
    if (xs >= G::HALO && xe + G::HALO <= nx) {
        if (lane < 7) {
            fence_proxy_async_smem();
            const int i = lane;
            const int r = wrap_once(y + ((i == 2 || i == 3) ? -1 : ((i == 5 || i == 6) ? 1 : 0)), ny);
            const T *row = src + (size_t)i * plane + (size_t)r * pitch;
            bulk_copy_g2s(buf + i * G::SEG, row + (xs - G::HALO), main_bytes + 32u, bar);
        }
    } else if (lane < 21) {
        fence_proxy_async_smem();
        const int i = lane / 3, part = lane % 3;
        const int r = wrap_once(y + ((i == 2 || i == 3) ? -1 : ((i == 5 || i == 6) ? 1 : 0)), ny);
        const T *row = src + (size_t)i * plane + (size_t)r * pitch;
        T *seg = buf + i * G::SEG;
        if (part == 0) {
            const int c = xs == 0 ? nx - G::HALO : xs - G::HALO;
            bulk_copy_g2s(seg, row + c, 16u, bar);
        } else if (part == 1) {
            bulk_copy_g2s(seg + G::HALO, row + xs, main_bytes, bar);
        } else {
            const int c = xe >= nx ? 0 : xe;
            bulk_copy_g2s(seg + G::HALO + (xe - xs), row + c, 16u, bar);
        }
    }
}

// Pulled values of population I at the lane's sites of a row of parity P:
// f_I at column x0 + j + q7_src_dx(I, P), shared index b + j + dx.
template <int ST, int VEC, int I, int P>
__device__ __forceinline__ void stage_pop7(const typename Store<ST>::T *seg, int b, float shift, float out[VEC])
{
    float a[VEC];
    load_vec_plain<ST, VEC>(seg + b, shift, a);
    constexpr int DX = q7_src_dx(I, P);
    if constexpr (DX == 0) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) out[j] = a[j];
    } else if constexpr (DX == -1) {
        out[0] = Store<ST>::get(seg[b - 1], shift);
#pragma unroll
        for (int j = 1; j < VEC; ++j) out[j] = a[j - 1];
    } else {
#pragma unroll
        for (int j = 0; j < VEC - 1; ++j) out[j] = a[j + 1];
        out[VEC - 1] = Store<ST>::get(seg[b + VEC], shift);
    }
}

template <int ST, int VEC, int P>
__device__ __forceinline__ void stage_row7(const typename Store<ST>::T *buf, int b, const Shift3 &sh, float f[7][VEC])
{
    using G = StageGeom7<ST, VEC>;
    stage_pop7<ST, VEC, 0, P>(buf + 0 * G::SEG, b, sh.q7(0), f[0]);
    stage_pop7<ST, VEC, 1, P>(buf + 1 * G::SEG, b, sh.q7(1), f[1]);
    stage_pop7<ST, VEC, 2, P>(buf + 2 * G::SEG, b, sh.q7(2), f[2]);
    stage_pop7<ST, VEC, 3, P>(buf + 3 * G::SEG, b, sh.q7(3), f[3]);
    stage_pop7<ST, VEC, 4, P>(buf + 4 * G::SEG, b, sh.q7(4), f[4]);
    stage_pop7<ST, VEC, 5, P>(buf + 5 * G::SEG, b, sh.q7(5), f[5]);
    stage_pop7<ST, VEC, 6, P>(buf + 6 * G::SEG, b, sh.q7(6), f[6]);
}

// Post-stream density at shared index c of a staged row of parity P.
template <int ST, int VEC, int P>
__device__ __forceinline__ float stage_density_at7(const typename Store<ST>::T *buf, int c, const Shift3 &sh)
{
    using G = StageGeom7<ST, VEC>;
    float v[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) v[i] = Store<ST>::get(buf[i * G::SEG + c + q7_src_dx(i, P)], sh.q7(i));
    return density7(v);
}

template <int ST, int VEC, int P>
__device__ __forceinline__ void stage_density_window7(const typename Store<ST>::T *buf, int b, const Shift3 &sh, int lane,
                                                      float r[VEC + 2])
{
    float f[7][VEC];
    stage_row7<ST, VEC, P>(buf, b, sh, f);
#pragma unroll
    for (int j = 0; j < VEC; ++j) r[j + 1] = density7_at<VEC>(f, j);
    const float right = stage_density_at7<ST, VEC, P>(buf, b + VEC, sh);
    float left = __shfl_up_sync(FULL, r[VEC], 1);
    if (lane == 0) left = stage_density_at7<ST, VEC, P>(buf, b - 1, sh);
    r[0] = left;
    r[VEC + 1] = right;
}

template <int VEC> constexpr int staged7_min_blocks()
{
    return VEC == 1 ? 6 : (VEC == 2 ? 5 : 4);
}

template <int MODEL, int ST, int VEC, bool SAMPLE, int NOISE>
__global__ void __launch_bounds__(128, staged7_min_blocks<VEC>()) step_staged_kernel_q7(const StepArgs a)
{
    using T = typename Store<ST>::T;
    using G = StageGeom7<ST, VEC>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int S = a.stages;
    T *ring = reinterpret_cast<T *>(smem_raw + (size_t)warp * S * G::STAGE_BYTES);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + (size_t)(blockDim.x >> 5) * S * G::STAGE_BYTES) +
                     warp * S;

    const LatDesc *dp = a.desc + find_lattice(a.desc, a.nlat, blockIdx.x);
    const int nsx = dp->nsx, nsy = dp->nsy;
    const int s = (blockIdx.x - dp->block_begin) * (blockDim.x >> 5) + warp;
    if (s >= nsx * nsy) return;
    const int nx = dp->nx, ny = dp->ny, pitch = dp->pitch, rows = dp->rows;
    const SiteParams d = load_params(dp);
    const int sx = s % nsx, sy = s / nsx;
    const int xs = sx * G::W, xe = min(xs + G::W, nx);
    const int x0 = xs + lane * VEC;
    const bool valid = x0 < nx;
    const int b = G::HALO + lane * VEC;
    const int y_begin = sy * rows, y_end = min(y_begin + rows, ny);  // even, even
    const size_t plane = (size_t)ny * pitch;
    const T *src = reinterpret_cast<const T *>(dp->f[a.src]);
    T *dst = reinterpret_cast<T *>(dp->f[a.src ^ 1]);
    const Shift3 sh = load_shift(dp);
    const uint32_t id = (uint32_t)dp->id;
    const uint32_t t = *a.t_ptr + a.k;
    const bool noise = NOISE == 2 ? d.sigma_q > 0.f : NOISE == 1;

    if (lane == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[k], 1);
        mbar_init_fence();
    }
    __syncwarp();

    constexpr bool MIPS = (MODEL == MODEL_MIPS);
    const int q_first_row = MIPS ? y_begin - 1 : y_begin;
    const int nq = (y_end - y_begin) + (MIPS ? 2 : 0);
    int issued = 0;
    auto issue_next = [&]() {
        if (issued < nq) {
            const int k = issued % S;
            issue_row7<ST, VEC>(ring + (size_t)k * (G::STAGE_BYTES / sizeof(T)), &bars[k], src, plane, pitch, nx, ny,
                                xs, xe, wrap_once(q_first_row + issued, ny), lane);
            ++issued;
        }
    };
    for (int k = 0; k < S; ++k) issue_next();

    auto stage_ptr = [&](int q) { return ring + (size_t)(q % S) * (G::STAGE_BYTES / sizeof(T)); };
    bool ok = true;
    auto wait_q = [&](int q) {
        if (ok && !stage_wait(&bars[q % S], (uint32_t)((q / S) & 1))) {
            ok = false;
            if (lane == 0) atomicOr(a.err, (unsigned)DEVERR_TIMEOUT);
        }
        return ok;
    };

    double col[VEC], acc[5];
    if constexpr (SAMPLE) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) col[j] = 0.0;
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[q] = 0.0;
    }
    double *rowp = dp->rowp + (size_t)sx * ny;

    float rm[VEC + 2], rc[VEC + 2], rn[VEC + 2];
    int q = 0;
    if constexpr (MIPS) {
        if (wait_q(0)) stage_density_window7<ST, VEC, 1>(stage_ptr(0), b, sh, lane, rm);  // row y_begin-1: odd
        issue_next();
        q = 1;
        if (wait_q(1)) stage_density_window7<ST, VEC, 0>(stage_ptr(1), b, sh, lane, rc);
    }

    // one row of parity P; returns false if a wait gave up
    auto do_row = [&](auto parity, int y) -> bool {
        constexpr int P = decltype(parity)::value;
        const int qc = q;
        float f[7][VEC];
        if constexpr (MIPS) {
            if (!wait_q(qc + 1)) return false;
            stage_density_window7<ST, VEC, 1 - P>(stage_ptr(qc + 1), b, sh, lane, rn);
        } else {
            if (!wait_q(qc)) return false;
        }
        stage_row7<ST, VEC, P>(stage_ptr(qc), b, sh, f);
        issue_next();
        q = qc + 1;
        float gx[VEC], gy[VEC];
        if constexpr (MIPS) {
            mips_gradients7<VEC, P>(rm, rc, rn, gx, gy);
        } else {
#pragma unroll
            for (int j = 0; j < VEC; ++j) gx[j] = gy[j] = 0.f;
        }
        float out[7][VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            float g[7], u[7];
#pragma unroll
            for (int i = 0; i < 7; ++i) g[i] = f[i][j];
            if (noise) noise_u7((uint32_t)(x0 + j), (uint32_t)y, t, id, a.rk, u);
            const float rho = collide7<MODEL>(g, gx[j], gy[j], d, noise, u, MIPS ? &rc[j + 1] : nullptr);
            negative_correction7(g, rho);
#pragma unroll
            for (int i = 0; i < 7; ++i) out[i][j] = g[i];
        }
        if (valid) {
#pragma unroll
            for (int i = 0; i < 7; ++i)
                store_vec<ST, VEC>(dst + i * plane + (size_t)y * pitch + x0, sh.q7(i), out[i]);
        }
        if constexpr (SAMPLE) {
            float g[7][VEC];
#pragma unroll
            for (int i = 0; i < 7; ++i)
#pragma unroll
                for (int j = 0; j < VEC; ++j)
                    g[i][j] = Store<ST>::get(Store<ST>::put(out[i][j], sh.q7(i)), sh.q7(i));
            observe_row7<VEC>(g, valid, col, acc, rowp + y, lane);
        }
        if constexpr (MIPS) {
#pragma unroll
            for (int j = 0; j < VEC + 2; ++j) {
                rm[j] = rc[j];
                rc[j] = rn[j];
            }
        }
        return true;
    };

    for (int y = y_begin; y < y_end && ok; y += 2) {
        if (!do_row(std::integral_constant<int, 0>{}, y)) break;
        if (!do_row(std::integral_constant<int, 1>{}, y + 1)) break;
    }
    if (!ok) {
        for (int qq = q; qq < issued; ++qq) (void)stage_wait(&bars[qq % S], (uint32_t)((qq / S) & 1));
        return;
    }
    for (int qq = q + (MIPS ? 1 : 0); qq < issued; ++qq) (void)stage_wait(&bars[qq % S], (uint32_t)((qq / S) & 1));
    if constexpr (SAMPLE) observe_flush<VEC>(dp->colp, dp->scal, nx, s, sy, x0, valid, col, acc, lane);
}

template <int MODEL, int ST, int VEC, bool SAMPLE, int NOISE>
static cudaError_t launch_one_staged7(const StepArgs &a, int blocks, int warps, cudaStream_t stream)
{
    const size_t bytes = (size_t)warps * a.stages * (StageGeom7<ST, VEC>::STAGE_BYTES + sizeof(uint64_t));
    auto kern = step_staged_kernel_q7<MODEL, ST, VEC, SAMPLE, NOISE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    kern<<<blocks, warps * 32, bytes, stream>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launchers (instantiated once per storage type by LBM_INSTANTIATE_Q7).
// ---------------------------------------------------------------------------
template <int MODEL, int ST, int VEC, bool SAMPLE, int NOISE>
static cudaError_t launch_one_q7(int kind, const StepArgs &a, int blocks, int warps, cudaStream_t stream)
{
    if (kind == 1) return launch_one_staged7<MODEL, ST, VEC, SAMPLE, NOISE>(a, blocks, warps, stream);
    step_kernel_q7<MODEL, ST, VEC, SAMPLE, NOISE><<<blocks, warps * 32, 0, stream>>>(a);
    return cudaGetLastError();
}

template <int MODEL, int ST, int VEC>
static cudaError_t launch_q7_mv(int kind, bool sample, int noise, const StepArgs &a, int blocks, int warps,
                                cudaStream_t stream)
{
    if (sample) return launch_one_q7<MODEL, ST, VEC, true, 2>(kind, a, blocks, warps, stream);
    if (noise == 0) return launch_one_q7<MODEL, ST, VEC, false, 0>(kind, a, blocks, warps, stream);
    if (noise == 1) return launch_one_q7<MODEL, ST, VEC, false, 1>(kind, a, blocks, warps, stream);
    return launch_one_q7<MODEL, ST, VEC, false, 2>(kind, a, blocks, warps, stream);
}

template <int MODEL, int ST>
static cudaError_t launch_q7_m(int kind, int vec, bool sample, int noise, const StepArgs &a, int blocks, int warps,
                               cudaStream_t stream)
{
    switch (vec) {
    case 1: return launch_q7_mv<MODEL, ST, 1>(kind, sample, noise, a, blocks, warps, stream);
    case 2: return launch_q7_mv<MODEL, ST, 2>(kind, sample, noise, a, blocks, warps, stream);
    case 4: return launch_q7_mv<MODEL, ST, 4>(kind, sample, noise, a, blocks, warps, stream);
    case 8:
        if constexpr (ST != ST_F32) return launch_q7_mv<MODEL, ST, 8>(kind, sample, noise, a, blocks, warps, stream);
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <int ST>
static cudaError_t launch_step_q7_storage(int model, int kind, int vec, bool sample, int noise, const StepArgs &a,
                                         int blocks, int warps, cudaStream_t stream)
{
    switch (model) {
    case MODEL_PASSIVE: return launch_q7_m<MODEL_PASSIVE, ST>(kind, vec, sample, noise, a, blocks, warps, stream);
    case MODEL_MIPS: return launch_q7_m<MODEL_MIPS, ST>(kind, vec, sample, noise, a, blocks, warps, stream);
    case MODEL_CIL: return launch_q7_m<MODEL_CIL, ST>(kind, vec, sample, noise, a, blocks, warps, stream);
    default: return cudaErrorInvalidValue;
    }
}

template <int ST>
static cudaError_t launch_observe_q7_storage(int vec, const StepArgs &a, int blocks, int warps, cudaStream_t stream)
{
    switch (vec) {
    case 1: observe_kernel_q7<ST, 1><<<blocks, warps * 32, 0, stream>>>(a); break;
    case 2: observe_kernel_q7<ST, 2><<<blocks, warps * 32, 0, stream>>>(a); break;
    case 4: observe_kernel_q7<ST, 4><<<blocks, warps * 32, 0, stream>>>(a); break;
    case 8:
        if constexpr (ST != ST_F32) {
            observe_kernel_q7<ST, 8><<<blocks, warps * 32, 0, stream>>>(a);
            break;
        }
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbm

#define LBM_INSTANTIATE_Q7(ST, SUFFIX)                                                                        \
    namespace lbm {                                                                                          \
    cudaError_t launch_step_q7_##SUFFIX(int model, int kind, int vec, bool sample, int noise, const StepArgs &a, \
                                        int blocks, int warps, cudaStream_t stream)                          \
    {                                                                                                        \
        return launch_step_q7_storage<ST>(model, kind, vec, sample, noise, a, blocks, warps, stream);         \
    }                                                                                                        \
    cudaError_t launch_observe_q7_##SUFFIX(int vec, const StepArgs &a, int blocks, int warps,                 \
                                           cudaStream_t stream)                                              \
    {                                                                                                        \
        return launch_observe_q7_storage<ST>(vec, a, blocks, warps, stream);                                  \
    }                                                                                                        \
    }

// lbm_step_q7_staged.cuh -- the D2Q7 step with bulk-copied population rows.
//
// The data movement of step_staged_kernel (lbm_step_staged.cuh) applied to the
// paper's triangular lattice: a block of W warps owns W adjacent warp strips
// of one strip row and a ring of `stages` shared-memory buffers; buffer q
// holds, for destination row r(q), the seven source-row segments it pulls from
// (row r + q7_src_dy(i) of population i), each covering the block's columns
// plus 16 bytes of periodic halo on both sides, and arrives by cp.async.bulk
// copies completing on the buffer's "full" mbarrier, issued by warp 0 rows
// ahead of use once every warp has released the buffer ("empty" mbarrier).
// The half-site column offsets of the brick layout (-1/0 from an even row, 0/+1
// from an odd one) become shared-memory index offsets; rows are walked in
// (even, odd) pairs so the parity is a template argument.  As on D2Q9, the
// MIPS kernel with 16-bit storage converts each staged row once into two FP32
// rows per warp.  The per-site arithmetic is collide7 / negative_correction7 /
// noise_u7 of lbm_step_q7.cuh, so states are bitwise those of step_kernel_q7.
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
    // elements per population segment of a block of `warps` warps (16-byte multiple)
    __host__ __device__ static constexpr int seg(int warps) { return warps * W + 2 * HALO; }
};
static_assert(staged_smem_bytes(7, 4, 4, 8, 4) == 4 * (7 * StageGeom7<ST_F32, 4>::seg(8) * 4 + 2 * sizeof(uint64_t)), "");
static_assert(staged_smem_bytes(7, 2, 4, 8, 2, true) ==
                  2 * (7 * StageGeom7<ST_BF16, 4>::seg(8) * 2 + 2 * sizeof(uint64_t)) + 2 * 8 * 7 * StageGeom7<ST_BF16, 4>::W * 4,
              "");

// Issue the segment copies of destination row y into buffer `buf` (seg
// elements per population) and arm its barrier, for the block's columns xs ..
// xe-1: one copy per population (lanes 0..6) where the halos lie inside the
// row, else three (lanes 0..20: left halo, columns, right halo), as issue_row.
template <int ST, int VEC>
__device__ __forceinline__ void issue_row7(typename Store<ST>::T *buf, int seg_elems, uint64_t *bar,
                                           const typename Store<ST>::T *src, size_t plane, int pitch, int nx, int ny,
                                           int xs, int xe, int y, int lane)
{
    using G = StageGeom7<ST, VEC>;
    using T = typename Store<ST>::T;
    const uint32_t main_bytes = (uint32_t)(xe - xs) * (uint32_t)sizeof(T);
    if (lane == 0) mbar_arrive_expect_tx(bar, 7u * (main_bytes + 32u));
    __syncwarp();
    if (xs >= G::HALO && xe + G::HALO <= nx) {
        if (lane < 7) {
            fence_proxy_async_smem();
            const int i = lane;
            const int r = wrap_once(y + ((i == 2 || i == 3) ? -1 : ((i == 5 || i == 6) ? 1 : 0)), ny);
            const T *row = src + (size_t)i * plane + (size_t)r * pitch;
            bulk_copy_g2s(buf + i * seg_elems, row + (xs - G::HALO), main_bytes + 32u, bar);
        }
    } else if (lane < 21) {
        fence_proxy_async_smem();
        const int i = lane / 3, part = lane % 3;
        const int r = wrap_once(y + ((i == 2 || i == 3) ? -1 : ((i == 5 || i == 6) ? 1 : 0)), ny);
        const T *row = src + (size_t)i * plane + (size_t)r * pitch;
        T *seg = buf + i * seg_elems;
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
__device__ __forceinline__ void stage_row7(const typename Store<ST>::T *buf, int sg, int b, const Shift3 &sh,
                                           float f[7][VEC])
{
    stage_pop7<ST, VEC, 0, P>(buf + 0 * sg, b, sh.q7(0), f[0]);
    stage_pop7<ST, VEC, 1, P>(buf + 1 * sg, b, sh.q7(1), f[1]);
    stage_pop7<ST, VEC, 2, P>(buf + 2 * sg, b, sh.q7(2), f[2]);
    stage_pop7<ST, VEC, 3, P>(buf + 3 * sg, b, sh.q7(3), f[3]);
    stage_pop7<ST, VEC, 4, P>(buf + 4 * sg, b, sh.q7(4), f[4]);
    stage_pop7<ST, VEC, 5, P>(buf + 5 * sg, b, sh.q7(5), f[5]);
    stage_pop7<ST, VEC, 6, P>(buf + 6 * sg, b, sh.q7(6), f[6]);
}

// Post-stream density at shared index c of a staged row of parity P.
template <int ST, int VEC, int P>
__device__ __forceinline__ float stage_density_at7(const typename Store<ST>::T *buf, int sg, int c, const Shift3 &sh)
{
    float v[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) v[i] = Store<ST>::get(buf[i * sg + c + q7_src_dx(i, P)], sh.q7(i));
    return density7(v);
}

// Density window of a staged row (r[0] at x0-1, r[1..VEC] the lane's sites,
// r[VEC+1] at x0+VEC): neighbours by shuffle, the two sites outside the warp's
// columns summed from shared memory in one pass (lane 0 the left one, every
// other lane the right one, which lane 31 keeps).  With a converted row `cv`
// the pulled FP32 values are also left there (population i at cv + i * cs).
template <int ST, int VEC, int P>
__device__ __forceinline__ void stage_density_window7(const typename Store<ST>::T *buf, int sg, int b,
                                                      const Shift3 &sh, int lane, float r[VEC + 2],
                                                      float *cv = nullptr, int cs = 0)
{
    float f[7][VEC];
    stage_row7<ST, VEC, P>(buf, sg, b, sh, f);
    if (cv) {
#pragma unroll
        for (int i = 0; i < 7; ++i) put_f32<VEC>(cv + i * cs, f[i]);
    }
#pragma unroll
    for (int j = 0; j < VEC; ++j) r[j + 1] = density7_at<VEC>(f, j);
    const float edge = stage_density_at7<ST, VEC, P>(buf, sg, lane == 0 ? b - 1 : b + VEC, sh);
    float left = __shfl_up_sync(FULL, r[VEC], 1);
    float right = __shfl_down_sync(FULL, r[1], 1);
    if (lane == 0) left = edge;
    if (lane == 31) right = edge;
    r[0] = left;
    r[VEC + 1] = right;
}

template <int MODEL, int ST, int VEC, bool SAMPLE, int NOISE>
__global__ void __maxnreg__(staged_max_regs<VEC>()) step_staged_kernel_q7(const StepArgs a)
{
    using T = typename Store<ST>::T;
    using G = StageGeom7<ST, VEC>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    const int S = a.stages;
    const int sg = G::seg(warps);
    const int stage_elems = 7 * sg;
    // carve-out: S stage buffers, then S "full" and S "empty" barriers
    // carve-out: S stage buffers, S "full" and S "empty" barriers, then (CONV,
    // as in step_staged_kernel) two converted rows per warp
    constexpr bool CONV = staged_conv_rows(MODEL, ST);
    T *ring = reinterpret_cast<T *>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + (size_t)S * stage_elems * sizeof(T));
    uint64_t *empty = full + S;
    float *const cv0 = reinterpret_cast<float *>(empty + S) + (size_t)warp * 7 * G::W + (threadIdx.x & 31) * VEC;
    auto cv = [&](int q) { return cv0 + (size_t)(q & 1) * warps * 7 * G::W; };

    const StagedBlock blk = staged_block(a, warps);
    const LatDesc *dp = blk.dp;
    const int nsx = dp->nsx;
    const int nx = dp->nx, ny = dp->ny, pitch = dp->pitch, rows = dp->rows;
    const SiteParams d = load_params(dp);
    const int sx = blk.sx0 + warp, sy = blk.sy;
    const int s = sy * nsx + sx;
    const int xs = blk.sx0 * G::W, xe = min(xs + blk.nact * G::W, nx);  // the block's columns
    const int x0 = sx * G::W + lane * VEC;
    const bool valid = x0 < nx;
    const int b = G::HALO + warp * G::W + lane * VEC;
    const int y_begin = sy * rows, y_end = min(y_begin + rows, ny);  // even, even
    const size_t plane = (size_t)ny * pitch;
    const T *src = reinterpret_cast<const T *>(dp->f[a.src]);
    T *dst = reinterpret_cast<T *>(dp->f[a.src ^ 1]);
    const Shift3 sh = load_shift(dp);
    const uint32_t id = (uint32_t)dp->id;
    const uint32_t t = *a.t_ptr + a.k;
    const bool noise = NOISE == 2 ? d.sigma_q > 0.f : NOISE == 1;
    const bool leader = warp == 0;

    if (threadIdx.x == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], (uint32_t)blk.nact);
        }
        mbar_init_fence();
    }
    __syncthreads();
    if (warp >= blk.nact) return;  // a strip past the lattice's last column

    constexpr bool MIPS = (MODEL == MODEL_MIPS);
    const int q_first_row = MIPS ? y_begin - 1 : y_begin;
    const int nq = (y_end - y_begin) + (MIPS ? 2 : 0);
    auto stage_ptr = [&](int q) { return ring + (size_t)(q % S) * stage_elems; };
    bool ok = true;
    auto fail = [&]() {
        ok = false;
        if (lane == 0) atomicOr(a.err, (unsigned)DEVERR_TIMEOUT);
    };
    int issued = 0;  // rows issued (warp 0)
    auto issue = [&]() {
        const int k = issued % S;
        issue_row7<ST, VEC>(ring + (size_t)k * stage_elems, sg, &full[k], src, plane, pitch, nx, ny, xs, xe,
                            wrap_once(q_first_row + issued, ny), lane);
        ++issued;
    };
    if (leader)
        while (issued < S && issued < nq) issue();

    // Row q is consumed by this warp; warp 0 refills its buffer with row q + S
    // once every warp has (a single warp needs no barrier for that).
    auto release = [&](int q) {
        __syncwarp();
        if (blk.nact == 1) {
            if (ok && issued < nq) issue();
            return;
        }
        if (lane == 0) mbar_arrive(&empty[q % S]);
        if (leader && ok && issued < nq) {
            if (!stage_wait(&empty[q % S], (uint32_t)((q / S) & 1))) fail();
            else issue();
        }
    };
    auto wait_q = [&](int q) {
        if (ok && !stage_wait(&full[q % S], (uint32_t)((q / S) & 1))) fail();
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
        if (wait_q(0)) {
            stage_density_window7<ST, VEC, 1>(stage_ptr(0), sg, b, sh, lane, rm);  // row y_begin-1: odd
            release(0);
        }
        q = 1;
        if (wait_q(1)) {
            stage_density_window7<ST, VEC, 0>(stage_ptr(1), sg, b, sh, lane, rc, CONV ? cv(1) : nullptr, G::W);
            if constexpr (CONV) release(1);
        }
    }

    // one row of parity P; returns false if a wait gave up
    auto do_row = [&](auto parity, int y) -> bool {
        constexpr int P = decltype(parity)::value;
        const int qc = q;
        float f[7][VEC];
        if constexpr (CONV) {
            if (!wait_q(qc + 1)) return false;
            stage_density_window7<ST, VEC, 1 - P>(stage_ptr(qc + 1), sg, b, sh, lane, rn, cv(qc + 1), G::W);
            release(qc + 1);
#pragma unroll
            for (int i = 0; i < 7; ++i) get_f32<VEC>(cv(qc) + i * G::W, f[i]);
        } else if constexpr (MIPS) {
            if (!wait_q(qc + 1)) return false;
            stage_density_window7<ST, VEC, 1 - P>(stage_ptr(qc + 1), sg, b, sh, lane, rn);
            stage_row7<ST, VEC, P>(stage_ptr(qc), sg, b, sh, f);
            release(qc);
        } else {
            if (!wait_q(qc)) return false;
            stage_row7<ST, VEC, P>(stage_ptr(qc), sg, b, sh, f);
            release(qc);
        }
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
    if (leader) {
        // the copies warp 0 issued must land before the block's shared memory is
        // released: wait for the rows it has not waited for itself (bounded)
        for (int qq = q + (MIPS ? 1 : 0); qq < issued; ++qq)
            (void)stage_wait(&full[qq % S], (uint32_t)((qq / S) & 1));
    }
    if (!ok) return;
    if constexpr (SAMPLE) observe_flush<VEC>(dp->colp, dp->scal, nx, s, sy, x0, valid, col, acc, lane);
}

template <int MODEL, int ST, int VEC, bool SAMPLE, int NOISE>
static cudaError_t launch_one_staged7(const StepArgs &a, int blocks, int warps, cudaStream_t stream)
{
    const size_t bytes =
        staged_smem_bytes(7, (int)sizeof(typename Store<ST>::T), VEC, warps, a.stages, staged_conv_rows(MODEL, ST));
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

// lbm_step_staged.cuh -- the fused step with TMA-staged population rows.
//
// Same per-site arithmetic as step_kernel (lbm_step.cuh), different data
// movement.  A block of W warps owns W horizontally adjacent warp strips of one
// strip row (W * 32 * VEC columns, `rows` rows) and a ring of `stages`
// shared-memory buffers.  Buffer q holds, for destination row r(q), the nine
// source-row segments it pulls from (row r - e_y of population i), each
// covering the block's columns plus 16 bytes of halo on both sides (the
// periodic wrap is resolved by copying the halo from the other end of the
// row).  The segments arrive by bulk copies (cp.async.bulk, global -> shared)
// that complete on the buffer's "full" mbarrier; warp 0 issues them for the
// whole block, `stages - 1` (MIPS: `stages - 2`) rows ahead of use, once every
// warp has released the buffer's previous row on its "empty" mbarrier.  So a
// row costs nine copies per block rather than per warp, and the memory
// latency is hidden without holding rows in registers.  Lanes read their
// pulled values straight from shared memory, halo included: no shuffles and no
// lane-divergent edge loads.  The MIPS kernel with 16-bit storage converts
// each staged row once, in its density pass, into two FP32 rows per warp that
// the update then reads; its staged rows are released a row earlier, so it
// fetches `stages - 1` rows ahead as well.
//
// Requirements (checked on the host): nx a multiple of the 16-byte halo width
// (4 FP32 / 8 16-bit values) and at least that wide.  Every wait is bounded:
// on expiry the warp raises DEVERR_TIMEOUT in the error word and leaves its
// loop; warp 0 then drains the copies in flight (again bounded) before the
// block exits.
#pragma once

#include "lbm_step.cuh"

namespace lbm {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Test a phase of the barrier; while it is incomplete the thread may be
// suspended in hardware for up to WAIT_SUSPEND_NS (so a waiting warp takes no
// issue slots from the others) before the test returns.
constexpr uint32_t WAIT_SUSPEND_NS = 1000000u;

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(WAIT_SUSPEND_NS)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ~1 s at the GB300 clock; a healthy copy completes in microseconds.
constexpr long long WAIT_LIMIT_CYCLES = 2000000000LL;

// Warp-uniform bounded wait for one phase of a stage barrier.
__device__ __forceinline__ bool stage_wait(uint64_t *bar, uint32_t parity)
{
    if (__all_sync(FULL, mbar_try_wait(bar, parity))) return true;  // the usual case: no clock read
    const long long t0 = clock64();
    while (true) {
        const bool ok = mbar_try_wait(bar, parity);
        if (__all_sync(FULL, ok)) return true;
        if (clock64() - t0 > WAIT_LIMIT_CYCLES) return false;
    }
}

template <int ST, int VEC> struct StageGeom {
    using T = typename Store<ST>::T;
    static constexpr int HALO = 16 / (int)sizeof(T);        // halo width in elements (16 bytes)
    static constexpr int W = 32 * VEC;                       // strip width of one warp
    // elements per population segment of a block of `warps` warps (a multiple
    // of 16 bytes, so every segment starts 16-byte aligned)
    __host__ __device__ static constexpr int seg(int warps) { return warps * W + 2 * HALO; }
};
// the launcher's shared-memory size is the kernel's carve-out (ring, barriers,
// then the converted row)
static_assert(staged_smem_bytes(9, 4, 4, 4, 3) == 3 * (9 * StageGeom<ST_F32, 4>::seg(4) * 4 + 2 * sizeof(uint64_t)), "");
static_assert(staged_smem_bytes(9, 2, 8, 8, 5, true) == 5 * (9 * StageGeom<ST_F16, 8>::seg(8) * 2 + 2 * sizeof(uint64_t)) +
                                                            2 * 8 * 9 * StageGeom<ST_F16, 8>::W * 4,
              "");

// Issue the segment copies of destination row y into stage buffer `buf` (seg
// elements per population) and arm its barrier (lane 0 arms); executed by one
// warp for the block, whose columns are xs .. xe-1.  Where the halos lie inside
// the row (xs >= HALO, xe + HALO <= nx) each population takes one copy, lanes
// 0..8: the left halo, the block's columns and the right halo are contiguous in
// the row and in the segment.  At the periodic edge each takes three, lanes
// 0..26.  Each copy is issued by one elected lane at a time.
template <int ST, int VEC>
__device__ __forceinline__ void issue_row(typename Store<ST>::T *buf, int seg_elems, uint64_t *bar,
                                          const typename Store<ST>::T *src, size_t plane, int pitch,
                                          int nx, int ny, int xs, int xe, int y, int lane)
{
    using G = StageGeom<ST, VEC>;
    using T = typename Store<ST>::T;
    const uint32_t main_bytes = (uint32_t)(xe - xs) * (uint32_t)sizeof(T);
    if (lane == 0) mbar_arrive_expect_tx(bar, 9u * (main_bytes + 32u));
    __syncwarp();
    if (xs >= G::HALO && xe + G::HALO <= nx) {
        if (lane < 9) {
            fence_proxy_async_smem();  // order the buffer's earlier reads before the copy's writes
            const int i = lane;
            const int dy = (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
            const int r = wrap_once(y - dy, ny);
            const T *row = src + (size_t)i * plane + (size_t)r * pitch;
            bulk_copy_g2s(buf + i * seg_elems, row + (xs - G::HALO), main_bytes + 32u, bar);
        }
    } else if (lane < 27) {
        fence_proxy_async_smem();  // order the buffer's earlier reads before the copy's writes
        const int i = lane / 3, part = lane % 3;
        const int dy = (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
        const int r = wrap_once(y - dy, ny);
        const T *row = src + (size_t)i * plane + (size_t)r * pitch;
        T *seg = buf + i * seg_elems;
        if (part == 0) {  // left halo: columns xs-HALO .. xs-1 (periodic)
            const int c = xs == 0 ? nx - G::HALO : xs - G::HALO;
            bulk_copy_g2s(seg, row + c, 16u, bar);
        } else if (part == 1) {  // the block's columns
            bulk_copy_g2s(seg + G::HALO, row + xs, main_bytes, bar);
        } else {  // right halo: columns xe .. xe+HALO-1 (periodic)
            const int c = xe >= nx ? 0 : xe;
            bulk_copy_g2s(seg + G::HALO + (xe - xs), row + c, 16u, bar);
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Pulled values of population I for this lane's VEC sites, from the stage:
// f_I(x0 + j - e_x), read at shared index b + j - e_x.
template <int ST, int VEC, int I>
__device__ __forceinline__ void stage_pop(const typename Store<ST>::T *seg, int b, float shift, float out[VEC])
{
    float a[VEC];
    load_vec_plain<ST, VEC>(seg + b, shift, a);
    if constexpr (vx(I) == 0) {
#pragma unroll
        for (int j = 0; j < VEC; ++j) out[j] = a[j];
    } else if constexpr (vx(I) == 1) {
        out[0] = Store<ST>::get(seg[b - 1], shift);
#pragma unroll
        for (int j = 1; j < VEC; ++j) out[j] = a[j - 1];
    } else {
#pragma unroll
        for (int j = 0; j < VEC - 1; ++j) out[j] = a[j + 1];
        out[VEC - 1] = Store<ST>::get(seg[b + VEC], shift);
    }
}

template <int ST, int VEC>
__device__ __forceinline__ void stage_row(const typename Store<ST>::T *buf, int sg, int b, const Shift3 &sh,
                                          float f[9][VEC])
{
    stage_pop<ST, VEC, 0>(buf + 0 * sg, b, sh.q9(0), f[0]);
    stage_pop<ST, VEC, 1>(buf + 1 * sg, b, sh.q9(1), f[1]);
    stage_pop<ST, VEC, 2>(buf + 2 * sg, b, sh.q9(2), f[2]);
    stage_pop<ST, VEC, 3>(buf + 3 * sg, b, sh.q9(3), f[3]);
    stage_pop<ST, VEC, 4>(buf + 4 * sg, b, sh.q9(4), f[4]);
    stage_pop<ST, VEC, 5>(buf + 5 * sg, b, sh.q9(5), f[5]);
    stage_pop<ST, VEC, 6>(buf + 6 * sg, b, sh.q9(6), f[6]);
    stage_pop<ST, VEC, 7>(buf + 7 * sg, b, sh.q9(7), f[7]);
    stage_pop<ST, VEC, 8>(buf + 8 * sg, b, sh.q9(8), f[8]);
}

// Post-stream density at shared index c (one site) of a staged row.
template <int ST, int VEC>
__device__ __forceinline__ float stage_density_at(const typename Store<ST>::T *buf, int sg, int c, const Shift3 &sh)
{
    float v[9][1];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i][0] = Store<ST>::get(buf[i * sg + c - vx(i)], sh.q9(i));
    return density<1>(v, 0);
}

// The lane's VEC FP32 values at p (16-byte aligned for VEC >= 4).
template <int VEC> __device__ __forceinline__ void put_f32(float *p, const float v[VEC])
{
    if constexpr (VEC % 4 == 0) {
#pragma unroll
        for (int k = 0; k < VEC / 4; ++k)
            reinterpret_cast<float4 *>(p)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    } else if constexpr (VEC == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
        p[0] = v[0];
    }
}
template <int VEC> __device__ __forceinline__ void get_f32(const float *p, float v[VEC])
{
    if constexpr (VEC % 4 == 0) {
#pragma unroll
        for (int k = 0; k < VEC / 4; ++k) {
            const float4 w = reinterpret_cast<const float4 *>(p)[k];
            v[4 * k] = w.x;
            v[4 * k + 1] = w.y;
            v[4 * k + 2] = w.z;
            v[4 * k + 3] = w.w;
        }
    } else if constexpr (VEC == 2) {
        const float2 w = *reinterpret_cast<const float2 *>(p);
        v[0] = w.x;
        v[1] = w.y;
    } else {
        v[0] = p[0];
    }
}

// Density window of a staged row: r[0] at x0-1, r[1..VEC] the lane's sites,
// r[VEC+1] at x0+VEC.  Neighbours come by shuffle (a lane past a ragged strip
// end sums the right halo's site, which its segment index reaches); the two
// sites outside the warp's columns, lane 0's left and lane 31's right, are
// summed from shared memory in one pass, each lane summing the site its role
// needs (the same values and order as its neighbour's own sum).  With a
// converted row `cv` (population i of the lane's sites at cv + i * cs), the
// pulled FP32 values are also left there for the row's update.
template <int ST, int VEC>
__device__ __forceinline__ void stage_density_window(const typename Store<ST>::T *buf, int sg, int b,
                                                     const Shift3 &sh, int lane, float r[VEC + 2],
                                                     float *cv = nullptr, int cs = 0)
{
    float f[9][VEC];
    stage_row<ST, VEC>(buf, sg, b, sh, f);
    if (cv) {
#pragma unroll
        for (int i = 0; i < 9; ++i) put_f32<VEC>(cv + i * cs, f[i]);
    }
    densities<VEC, paired_sites<ST, VEC>()>(f, r + 1);
    const float edge = stage_density_at<ST, VEC>(buf, sg, lane == 0 ? b - 1 : b + VEC, sh);
    float left = __shfl_up_sync(FULL, r[VEC], 1);
    float right = __shfl_down_sync(FULL, r[1], 1);
    if (lane == 0) left = edge;
    if (lane == 31) right = edge;
    r[0] = left;
    r[VEC + 1] = right;
}

// Register cap per thread of the staged kernels per VEC (80, 96, 128, 128):
// measured per VEC, these caps cost FP32 nothing and speed 16-bit storage up.
// Blocks have up to 8 warps (256 threads).
#ifndef LBM_STAGED_REGS_1
#define LBM_STAGED_REGS_1 80
#endif
#ifndef LBM_STAGED_REGS_2
#define LBM_STAGED_REGS_2 96
#endif
#ifndef LBM_STAGED_REGS_4
#define LBM_STAGED_REGS_4 128
#endif
#ifndef LBM_STAGED_REGS_8
#define LBM_STAGED_REGS_8 128
#endif
template <int VEC> constexpr int staged_max_regs()
{
    return VEC == 1 ? LBM_STAGED_REGS_1 : (VEC == 2 ? LBM_STAGED_REGS_2 : (VEC == 4 ? LBM_STAGED_REGS_4 : LBM_STAGED_REGS_8));
}

// The block's place in its lattice: strip row sy, first strip column sx0, and
// the number of its warps whose strips lie inside the lattice (at least 1).
struct StagedBlock {
    const LatDesc *dp;
    int sx0, sy, nact;
};

__device__ __forceinline__ StagedBlock staged_block(const StepArgs &a, int warps)
{
    StagedBlock g;
    g.dp = a.desc + find_lattice(a.desc, a.nlat, blockIdx.x);
    const int ncx = (g.dp->nsx + warps - 1) / warps;
    const int bl = blockIdx.x - g.dp->block_begin;
    g.sx0 = (bl % ncx) * warps;
    g.sy = bl / ncx;
    g.nact = min(warps, g.dp->nsx - g.sx0);
    return g;
}

template <int MODEL, int ST, int VEC, bool SAMPLE, int NOISE>
__global__ void __maxnreg__(staged_max_regs<VEC>()) step_staged_kernel(const StepArgs a)
{
    using T = typename Store<ST>::T;
    using G = StageGeom<ST, VEC>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    const int S = a.stages;
    const int sg = G::seg(warps);  // elements per population segment
    const int stage_elems = 9 * sg;
    // carve-out: S stage buffers, then S "full" and S "empty" barriers, then
    // (CONV) two converted rows per warp, row q in cv(q): population i of the
    // warp's sites at i * W
    constexpr bool CONV = staged_conv_rows(MODEL, ST);
    T *ring = reinterpret_cast<T *>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + (size_t)S * stage_elems * sizeof(T));
    uint64_t *empty = full + S;
    float *const cv0 = reinterpret_cast<float *>(empty + S) + (size_t)warp * 9 * G::W + (threadIdx.x & 31) * VEC;
    auto cv = [&](int q) { return cv0 + (size_t)(q & 1) * warps * 9 * G::W; };

    const StagedBlock blk = staged_block(a, warps);
    const LatDesc *dp = blk.dp;
    const int nsx = dp->nsx;
    const int nx = dp->nx, ny = dp->ny, pitch = dp->pitch, rows = dp->rows;
    const int sx = blk.sx0 + warp, sy = blk.sy;
    const int s = sy * nsx + sx;  // this warp's strip (observable partials)
    const int xs = blk.sx0 * G::W, xe = min(xs + blk.nact * G::W, nx);  // the block's columns
    const int x0 = sx * G::W + lane * VEC;
    const bool valid = x0 < nx;
    const int b = G::HALO + warp * G::W + lane * VEC;  // shared index of x0 within a segment
    const int y_begin = sy * rows, y_end = min(y_begin + rows, ny);
    const size_t plane = (size_t)ny * pitch;
    const T *src = reinterpret_cast<const T *>(dp->f[a.src]);
    T *dst = reinterpret_cast<T *>(dp->f[a.src ^ 1]);
    const Shift3 sh = load_shift(dp);
    const uint32_t id = (uint32_t)dp->id;
    const uint32_t t = *a.t_ptr + a.k;
    const SiteParams d = load_params(dp);
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
    if (warp >= blk.nact) return;  // a strip past the lattice's last column: no work, no arrivals

    // rows in order of use: MIPS also needs y_begin-1 and y_end (density halo)
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
        issue_row<ST, VEC>(ring + (size_t)k * stage_elems, sg, &full[k], src, plane, pitch, nx, ny, xs, xe,
                           wrap_once(q_first_row + issued, ny), lane);
        ++issued;
    };
    if (leader)
        while (issued < S && issued < nq) issue();

    // Row q is consumed: every lane of the warp has finished its reads, and the
    // warp tells warp 0, which refills the buffer with row q + S once all warps
    // have done so.
    auto release = [&](int q) {
        __syncwarp();
        if (blk.nact == 1) {  // a single warp: its own reads are all there is to wait for
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

    // MIPS: row q+1's densities are taken one row ahead of its update.  With
    // CONV its pulled populations are converted then too, into converted row
    // cv(q+1), so the update reads them from there and the staged row is
    // released one row earlier.
    float rm[VEC + 2], rc[VEC + 2], rn[VEC + 2];
    int q = 0;  // next stage to consume
    if constexpr (MIPS) {
        if (wait_q(0)) {
            stage_density_window<ST, VEC>(stage_ptr(0), sg, b, sh, lane, rm);
            release(0);
        }
        q = 1;
        if (wait_q(1)) {
            stage_density_window<ST, VEC>(stage_ptr(1), sg, b, sh, lane, rc, CONV ? cv(1) : nullptr, G::W);
            if constexpr (CONV) release(1);
        }
    }

    for (int y = y_begin; y < y_end && ok; ++y) {
        const int qc = q;  // stage of row y
        float f[9][VEC];
        if constexpr (CONV) {
            if (!wait_q(qc + 1)) break;
            stage_density_window<ST, VEC>(stage_ptr(qc + 1), sg, b, sh, lane, rn, cv(qc + 1), G::W);
            release(qc + 1);
#pragma unroll
            for (int i = 0; i < 9; ++i) get_f32<VEC>(cv(qc) + i * G::W, f[i]);
        } else if constexpr (MIPS) {
            if (!wait_q(qc + 1)) break;
            stage_density_window<ST, VEC>(stage_ptr(qc + 1), sg, b, sh, lane, rn);
            stage_row<ST, VEC>(stage_ptr(qc), sg, b, sh, f);
            release(qc);
        } else {
            if (!wait_q(qc)) break;
            stage_row<ST, VEC>(stage_ptr(qc), sg, b, sh, f);
            release(qc);
        }
        q = qc + 1;

        float gx[VEC], gy[VEC];
        if constexpr (MIPS) {
            mips_gradients<VEC>(rm, rc, rn, gx, gy);
        } else {
#pragma unroll
            for (int j = 0; j < VEC; ++j) gx[j] = gy[j] = 0.f;
        }
        float out[9][VEC];
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int j = 0; j < VEC; ++j) out[i][j] = f[i][j];
        collide_sites<MODEL, VEC, paired_sites<ST, VEC>()>(out, gx, gy, d, noise, (uint32_t)x0, (uint32_t)y, t, id,
                                                           a.rk, MIPS ? rc + 1 : nullptr);
        if (valid) {
#pragma unroll
            for (int i = 0; i < 9; ++i)
                store_vec<ST, VEC>(dst + i * plane + (size_t)y * pitch + x0, sh.q9(i), out[i]);
        }
        if constexpr (SAMPLE) {
            float g[9][VEC];
#pragma unroll
            for (int i = 0; i < 9; ++i)
#pragma unroll
                for (int j = 0; j < VEC; ++j)
                    g[i][j] = Store<ST>::get(Store<ST>::put(out[i][j], sh.q9(i)), sh.q9(i));
            observe_row<VEC>(g, valid, col, acc, dp->rowp + (size_t)sx * ny + y, lane);
        }
        if constexpr (MIPS) {
#pragma unroll
            for (int j = 0; j < VEC + 2; ++j) {
                rm[j] = rc[j];
                rc[j] = rn[j];
            }
        }
    }
    if (leader) {
        // every copy warp 0 issued must land before the block's shared memory
        // is released: wait for the rows it has not waited for itself (the
        // latest phase of each of their buffers; bounded)
        for (int qq = q + (MIPS ? 1 : 0); qq < issued; ++qq)
            (void)stage_wait(&full[qq % S], (uint32_t)((qq / S) & 1));
    }
    if (!ok) return;
    if constexpr (SAMPLE) observe_flush<VEC>(dp->colp, dp->scal, nx, s, sy, x0, valid, col, acc, lane);
}


}  // namespace lbm

// ---------------------------------------------------------------------------
// Launchers (instantiated once per storage type by LBM_INSTANTIATE_STORAGE).
// ---------------------------------------------------------------------------
namespace lbm {

template <int MODEL, int ST, int VEC, bool SAMPLE, int NOISE>
static cudaError_t launch_one_staged(const StepArgs &a, int blocks, int warps, cudaStream_t stream)
{
    const size_t bytes =
        staged_smem_bytes(9, (int)sizeof(typename Store<ST>::T), VEC, warps, a.stages, staged_conv_rows(MODEL, ST));
    auto kern = step_staged_kernel<MODEL, ST, VEC, SAMPLE, NOISE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    kern<<<blocks, warps * 32, bytes, stream>>>(a);
    return cudaGetLastError();
}

template <int MODEL, int ST, int VEC, bool SAMPLE, int NOISE>
static cudaError_t launch_one(int kind, const StepArgs &a, int blocks, int warps, cudaStream_t stream)
{
    if (kind == 1) return launch_one_staged<MODEL, ST, VEC, SAMPLE, NOISE>(a, blocks, warps, stream);
    step_kernel<MODEL, ST, VEC, SAMPLE, NOISE><<<blocks, warps * 32, 0, stream>>>(a);
    return cudaGetLastError();
}

// Sample steps (one in sample_every) decide the noise at run time; the other
// steps take the compile-time forms when the launch group is uniform.
template <int MODEL, int ST, int VEC>
static cudaError_t launch_mv(int kind, bool sample, int noise, const StepArgs &a, int blocks, int warps,
                             cudaStream_t stream)
{
    if (sample) return launch_one<MODEL, ST, VEC, true, 2>(kind, a, blocks, warps, stream);
    if (noise == 0) return launch_one<MODEL, ST, VEC, false, 0>(kind, a, blocks, warps, stream);
    if (noise == 1) return launch_one<MODEL, ST, VEC, false, 1>(kind, a, blocks, warps, stream);
    return launch_one<MODEL, ST, VEC, false, 2>(kind, a, blocks, warps, stream);
}

template <int MODEL, int ST>
static cudaError_t launch_m(int kind, int vec, bool sample, int noise, const StepArgs &a, int blocks, int warps,
                            cudaStream_t stream)
{
    switch (vec) {
    case 1: return launch_mv<MODEL, ST, 1>(kind, sample, noise, a, blocks, warps, stream);
    case 2: return launch_mv<MODEL, ST, 2>(kind, sample, noise, a, blocks, warps, stream);
    case 4: return launch_mv<MODEL, ST, 4>(kind, sample, noise, a, blocks, warps, stream);
    case 8:
        if constexpr (ST != ST_F32) return launch_mv<MODEL, ST, 8>(kind, sample, noise, a, blocks, warps, stream);
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <int ST>
static cudaError_t launch_step_storage(int model, int kind, int vec, bool sample, int noise, const StepArgs &a,
                                       int blocks, int warps, cudaStream_t stream)
{
    switch (model) {
    case MODEL_PASSIVE: return launch_m<MODEL_PASSIVE, ST>(kind, vec, sample, noise, a, blocks, warps, stream);
    case MODEL_MIPS: return launch_m<MODEL_MIPS, ST>(kind, vec, sample, noise, a, blocks, warps, stream);
    case MODEL_CIL: return launch_m<MODEL_CIL, ST>(kind, vec, sample, noise, a, blocks, warps, stream);
    default: return cudaErrorInvalidValue;
    }
}

template <int ST>
static cudaError_t launch_observe_storage(int vec, const StepArgs &a, int blocks, int warps, cudaStream_t stream)
{
    switch (vec) {
    case 1: observe_kernel<ST, 1><<<blocks, warps * 32, 0, stream>>>(a); break;
    case 2: observe_kernel<ST, 2><<<blocks, warps * 32, 0, stream>>>(a); break;
    case 4: observe_kernel<ST, 4><<<blocks, warps * 32, 0, stream>>>(a); break;
    case 8:
        if constexpr (ST != ST_F32) {
            observe_kernel<ST, 8><<<blocks, warps * 32, 0, stream>>>(a);
            break;
        }
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbm

#define LBM_INSTANTIATE_STORAGE(ST, SUFFIX)                                                                  \
    namespace lbm {                                                                                          \
    cudaError_t launch_step_##SUFFIX(int model, int kind, int vec, bool sample, int noise, const StepArgs &a,  \
                                     int blocks, int warps, cudaStream_t stream)                             \
    {                                                                                                        \
        return launch_step_storage<ST>(model, kind, vec, sample, noise, a, blocks, warps, stream);            \
    }                                                                                                        \
    cudaError_t launch_observe_##SUFFIX(int vec, const StepArgs &a, int blocks, int warps,                    \
                                        cudaStream_t stream)                                                 \
    {                                                                                                        \
        return launch_observe_storage<ST>(vec, a, blocks, warps, stream);                                     \
    }                                                                                                        \
    }

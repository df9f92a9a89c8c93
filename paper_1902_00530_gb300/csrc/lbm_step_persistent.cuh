// lbm_step_persistent.cuh -- many steps of a launch group in one launch.
//
// The paper advances many independent lattices per parameter point (App.
// C.3-C.4); each of their steps is the App. A.2 update, here the body of the
// direct kernel (direct_strip, lbm_step.cuh) unchanged.  One persistent launch
// runs `nsteps` consecutive steps, none of them a sample step, of every
// lattice of a launch group.
//
// Work items are the blocks of the per-step grid, one per step: item (j, b) is
// block b of step j.  Blocks take items from a counter in a fixed order:
// lattice group by lattice group (groups of consecutive lattices whose
// population buffers together fit the L2 budget the host sets), and inside a
// group step by step.  An item of step j >= 1 waits until every strip of the
// strip rows it reads -- its own and the ones above and below, periodically --
// has finished step j - 1.  Those strip rows are also all the readers of the
// buffer it writes, so that one condition orders its reads after their writes
// and its writes after their reads.  A strip publishes its completion by a
// release increment of its strip row's counter after a fence; the waiting
// warp polls with acquire loads and the block passes a barrier before reading.
//
// No deadlock, whatever the number of resident blocks: an item depends only on
// items with smaller indices, taken earlier by blocks that are already
// running, so the smallest unfinished item can always proceed.  Each wait is
// still bounded (about 1 s): on expiry the block raises DEVERR_TIMEOUT, and
// every block leaves at its next item or wait once the error word is set.
//
// A lattice group's populations stay in L2 for its nsteps steps, so HBM sees
// them about once on the way in and once on the way out, and consecutive steps
// of a group overlap: a block starts on step j + 1 of a strip row as soon as
// that row's neighbourhood has finished step j, with no launch boundary or
// grid-wide barrier between steps.
#pragma once

#include <algorithm>

#include "lbm_step.cuh"

namespace lbm {

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_gpu_add(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// ~1 s at the GB300 clock; a healthy neighbourhood finishes in microseconds.
constexpr long long PERSIST_WAIT_CYCLES = 2000000000LL;

// The lattice group of item w: the last g with nsteps * pg[g] <= w.
__device__ __forceinline__ int persist_group(const PersistArgs &p, unsigned w)
{
    int lo = 0, hi = p.npg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((unsigned)p.nsteps * (unsigned)p.pg[mid] <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int MODEL, int ST, int VEC, int NOISE>
__global__ void __launch_bounds__(256, direct_min_blocks<MODEL, ST, VEC, false>())
    step_persistent_kernel(const StepArgs a, const PersistArgs p)
{
    __shared__ unsigned item_s;
    __shared__ int abort_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    const uint32_t t0 = *a.t_ptr + a.k;
    const unsigned total = (unsigned)p.nsteps * (unsigned)p.pg[p.npg];
    volatile unsigned *err = a.err;
    while (true) {
        if (threadIdx.x == 0) {
            item_s = *err ? total : atomicAdd(p.work, 1u);
            abort_s = 0;
        }
        __syncthreads();
        const unsigned w = item_s;
        if (w >= total) return;  // block-uniform
        const int g = persist_group(p, w);
        const unsigned lo = (unsigned)p.pg[g], nb = (unsigned)p.pg[g + 1] - lo;
        const unsigned r = w - (unsigned)p.nsteps * lo;
        const int j = (int)(r / nb);
        const int b = (int)(lo + r % nb);
        const LatDesc *dp = a.desc + find_lattice(a.desc, a.nlat, b);
        const int nsx = dp->nsx, nsy = dp->nsy;
        const int s0 = (b - dp->block_begin) * warps;  // the block's strips s0 .. s1-1 (as step_kernel)
        const int s1 = min(s0 + warps, nsx * nsy);
        if (j > 0 && warp == 0) {
            // strip rows sy_lo-1 .. sy_hi+1 (periodic) must have finished step j-1
            const int sy_lo = s0 / nsx, sy_hi = (s1 - 1) / nsx;
            const int nrow = min(nsy, sy_hi - sy_lo + 3);
            const unsigned need = (unsigned)j * (unsigned)nsx;
            bool ok = true;
            if (lane < nrow) {
                int row = sy_lo - 1 + lane;
                row = row < 0 ? row + nsy : (row >= nsy ? row - nsy : row);
                const unsigned *ctr = p.prog + dp->prog_off + row;
                if (ld_acquire_gpu(ctr) < need) {
                    const long long c0 = clock64();
                    while (ld_acquire_gpu(ctr) < need) {
                        if (*err) {
                            ok = false;
                            break;
                        }
                        if (clock64() - c0 > PERSIST_WAIT_CYCLES) {
                            atomicOr(a.err, (unsigned)DEVERR_TIMEOUT);
                            ok = false;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
            }
            if (!__all_sync(FULL, ok) && lane == 0) abort_s = 1;
        }
        __syncthreads();
        if (abort_s) return;  // block-uniform
        fence_acq_rel_gpu();  // this thread's reads come after the neighbourhood's writes
        const int s = s0 + warp;
        if (s < s1) {
            direct_strip<MODEL, ST, VEC, false, NOISE>(a, dp, s, a.src ^ (j & 1), t0 + (uint32_t)j);
            __threadfence();  // the strip's stores, before its completion is published
            __syncwarp();
            if (lane == 0) red_release_gpu_add(p.prog + dp->prog_off + s / nsx, 1u);
        }
        __syncthreads();  // item_s and abort_s are rewritten for the next item
    }
}

// Launch with as many blocks as fit on the GPU at once (fewer if there are
// fewer items); blocks that start later take items as they come.
// step_blocks: blocks of the per-step grid (pg[npg]).
template <int MODEL, int ST, int VEC, int NOISE>
static cudaError_t launch_persistent_one(const StepArgs &a, const PersistArgs &p, int step_blocks, int warps,
                                         cudaStream_t stream)
{
    auto kern = step_persistent_kernel<MODEL, ST, VEC, NOISE>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, 0);
    if (e != cudaSuccess) return e;
    const long long items = (long long)p.nsteps * step_blocks;
    const int grid = (int)std::min<long long>(items, (long long)std::max(1, per_sm) * sms);
    kern<<<grid, warps * 32, 0, stream>>>(a, p);
    return cudaGetLastError();
}

template <int MODEL, int ST, int VEC>
static cudaError_t launch_persistent_mv(int noise, const StepArgs &a, const PersistArgs &p, int step_blocks,
                                        int warps, cudaStream_t stream)
{
    if (noise == 0) return launch_persistent_one<MODEL, ST, VEC, 0>(a, p, step_blocks, warps, stream);
    if (noise == 1) return launch_persistent_one<MODEL, ST, VEC, 1>(a, p, step_blocks, warps, stream);
    return launch_persistent_one<MODEL, ST, VEC, 2>(a, p, step_blocks, warps, stream);
}

template <int MODEL, int ST>
static cudaError_t launch_persistent_m(int vec, int noise, const StepArgs &a, const PersistArgs &p, int step_blocks,
                                       int warps, cudaStream_t stream)
{
    switch (vec) {
    case 1: return launch_persistent_mv<MODEL, ST, 1>(noise, a, p, step_blocks, warps, stream);
    case 2: return launch_persistent_mv<MODEL, ST, 2>(noise, a, p, step_blocks, warps, stream);
    case 4: return launch_persistent_mv<MODEL, ST, 4>(noise, a, p, step_blocks, warps, stream);
    case 8:
        if constexpr (ST != ST_F32) return launch_persistent_mv<MODEL, ST, 8>(noise, a, p, step_blocks, warps, stream);
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <int ST>
static cudaError_t launch_persistent_storage(int model, int vec, int noise, const StepArgs &a, const PersistArgs &p,
                                             int step_blocks, int warps, cudaStream_t stream)
{
    switch (model) {
    case MODEL_PASSIVE: return launch_persistent_m<MODEL_PASSIVE, ST>(vec, noise, a, p, step_blocks, warps, stream);
    case MODEL_MIPS: return launch_persistent_m<MODEL_MIPS, ST>(vec, noise, a, p, step_blocks, warps, stream);
    case MODEL_CIL: return launch_persistent_m<MODEL_CIL, ST>(vec, noise, a, p, step_blocks, warps, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm

#define LBM_INSTANTIATE_PERSISTENT(ST, SUFFIX)                                                              \
    namespace lbm {                                                                                         \
    cudaError_t launch_persistent_##SUFFIX(int model, int vec, int noise, const StepArgs &a,                 \
                                           const PersistArgs &p, int step_blocks, int warps,                 \
                                           cudaStream_t stream)                                              \
    {                                                                                                       \
        return launch_persistent_storage<ST>(model, vec, noise, a, p, step_blocks, warps, stream);           \
    }                                                                                                       \
    }

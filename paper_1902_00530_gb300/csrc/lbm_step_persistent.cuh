// lbm_step_persistent.cuh -- many steps of a launch group in one launch.
//
// The paper advances many independent lattices per parameter point (App.
// C.3-C.4); each of their steps is the App. A.2 update, here the body of the
// direct kernel of the group's lattice unchanged (direct_strip, lbm_step.cuh,
// for D2Q9; direct_strip_q7, lbm_step_q7.cuh, for D2Q7).  One persistent
// launch runs `nsteps` consecutive steps, none of them a sample step, of every
// lattice of a launch group.
//
// Work items are the blocks of the per-step grid, one per step: item (j, b) is
// block b of step j.  Blocks take items from a counter in a fixed order:
// lattice group by lattice group (groups of consecutive lattices whose
// population buffers together fit a budget the host sets; by default one
// group), and inside a group step by step.  An item of step j >= 1 waits until
// every strip of the strip rows it reads -- its own and the ones above and
// below, periodically -- has finished step j - 1.  Those strip rows are also
// all the readers of the buffer it writes, so that one condition orders its
// reads after their writes and its writes after their reads.  A block
// publishes its finished strips per strip row (a barrier, one fence, then a
// relaxed increment per strip row it covers); the waiting warp polls with
// acquire loads, and the block passes a barrier before reading.
//
// No deadlock, whatever the number of resident blocks: an item depends only on
// items with smaller indices, taken earlier by blocks that are already
// running, so the smallest unfinished item can always proceed.  Each wait is
// still bounded (about 1 s): on expiry the block raises DEVERR_TIMEOUT, and
// every block leaves at its next item or wait once the error word is set.
//
// Consecutive steps overlap: a block starts on step j + 1 of a strip row as
// soon as that row's neighbourhood has finished step j, with no launch
// boundary or grid-wide barrier between steps, so no step waits for the last
// blocks of the one before.  With small lattice groups a group's populations
// could stay in L2 across its steps, but the strips of a periodic lattice all
// become ready together, so a group has one step in flight, and a group that
// fits L2 (about 20 lattices of 256^2 in FP32) gives a few hundred items per
// step where a GB300 holds about 900 blocks: measured 11-61 GLUPS against 81
// per step.  One lattice group for the whole launch group is the default.
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

__device__ __forceinline__ void red_relaxed_gpu_add(unsigned *p, unsigned v)
{
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// The block's current item, set up by thread 0 (kept in shared memory, so
// that none of it stays in registers across the strip's update).
struct PersistItem {
    int lat;     // lattice index in the launch group's table; -1: no more items
    int s0, s1;  // the block's strips s0 .. s1-1 (as in step_kernel)
    int j;       // step of the launch
    int abort;   // a wait gave up or the error word is set
};

// Thread 0: turn item w into the block's work (or the end of the launch).
__device__ __forceinline__ void persist_setup(const StepArgs &a, const PersistArgs &p, unsigned w, unsigned total,
                                              int warps, PersistItem &it)
{
    it.abort = 0;
    if (w >= total || *(volatile unsigned *)a.err) {
        it.lat = -1;
        return;
    }
    const int g = persist_group(p, w);
    const unsigned lo = (unsigned)p.pg[g], nb = (unsigned)p.pg[g + 1] - lo;
    const unsigned r = w - (unsigned)p.nsteps * lo;
    const int b = (int)(lo + r % nb);
    const int lat = find_lattice(a.desc, a.nlat, b);
    const LatDesc *dp = a.desc + lat;
    it.lat = lat;
    it.j = (int)(r / nb);
    it.s0 = (b - dp->block_begin) * warps;
    it.s1 = min(it.s0 + warps, dp->nsx * dp->nsy);
}

// Register cap per thread (blocks are at most 256 threads).  The loop around
// the strip's update keeps more values live than one launch per step does, so
// the per-step kernel's cap of 80 spills here; measured on the 256-lattice CIL
// batch (FP32, 16-row strips): 81.8 GLUPS at 80, 85.9 at 96, 80.2 at 128.
#ifndef LBM_PERSIST_REGS
#define LBM_PERSIST_REGS 96
#endif
template <int MODEL> constexpr int persist_max_regs() { return MODEL == MODEL_MIPS ? 128 : LBM_PERSIST_REGS; }

// The strip update of lattice Q (9: D2Q9, 7: D2Q7); the D2Q7 form is defined
// beside its direct kernel.
template <int Q> struct PersistStrip;
template <> struct PersistStrip<9> {
    template <int MODEL, int ST, int VEC, int NOISE>
    static __device__ __forceinline__ void run(const StepArgs &a, const LatDesc *dp, int s, int src, uint32_t t)
    {
        direct_strip<MODEL, ST, VEC, false, NOISE>(a, dp, s, src, t);
    }
};

template <int Q, int MODEL, int ST, int VEC, int NOISE>
__global__ void __maxnreg__(persist_max_regs<MODEL>()) step_persistent_kernel(const StepArgs a, const PersistArgs p)
{
    __shared__ PersistItem it;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned total = (unsigned)p.nsteps * (unsigned)p.pg[p.npg];
    // Thread 0 takes the block's next item while it sets up the current one,
    // so that the counter's round trip overlaps the item's work.  Still no
    // deadlock: a block's current item is smaller than the one it holds next,
    // so the smallest unfinished item is always one a block is working on.
    unsigned next = 0;
    if (threadIdx.x == 0) next = atomicAdd(p.work, 1u);
    while (true) {
        if (threadIdx.x == 0) {
            const unsigned w = next;
            if (w < total) next = atomicAdd(p.work, 1u);
            persist_setup(a, p, w, total, blockDim.x >> 5, it);
        }
        __syncthreads();
        if (it.lat < 0) return;  // block-uniform
        const LatDesc *dp = a.desc + it.lat;
        if (it.j > 0 && warp == 0) {
            // strip rows sy_lo-1 .. sy_hi+1 (periodic) must have finished step j-1
            const int nsx = dp->nsx, nsy = dp->nsy;
            const int sy_lo = it.s0 / nsx, sy_hi = (it.s1 - 1) / nsx;
            const int nrow = min(nsy, sy_hi - sy_lo + 3);
            const unsigned need = (unsigned)it.j * (unsigned)nsx;
            bool ok = true;
            if (lane < nrow) {
                int row = sy_lo - 1 + lane;
                row = row < 0 ? row + nsy : (row >= nsy ? row - nsy : row);
                const unsigned *ctr = p.prog + dp->prog_off + row;
                if (ld_acquire_gpu(ctr) < need) {
                    const long long c0 = clock64();
                    while (ld_acquire_gpu(ctr) < need) {
                        if (*(volatile unsigned *)a.err) {
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
            if (!__all_sync(FULL, ok) && lane == 0) it.abort = 1;
        }
        // The barrier orders every thread's reads after warp 0's acquire loads,
        // and so after the neighbourhood's writes (causality through the CTA
        // barrier; the acquire also keeps the SM's L1 from serving stale lines).
        __syncthreads();
        if (it.abort) return;  // block-uniform
        const int s = it.s0 + warp;
        const int jj = p.retime ? 0 : it.j;  // the timing form repeats step 0: same reads, same values written
        if (s < it.s1)
            PersistStrip<Q>::template run<MODEL, ST, VEC, NOISE>(a, dp, s, a.src ^ (jj & 1), *a.t_ptr + a.k + (uint32_t)jj);
        __syncthreads();  // every strip of the block is stored
        if (threadIdx.x == 0) {
            // publish the block's strips per strip row: one fence orders the
            // whole block's stores (ordered before it by the barrier), then
            // relaxed increments
            const LatDesc *dq = a.desc + it.lat;
            const int nsx = dq->nsx, sy_lo = it.s0 / nsx, sy_hi = (it.s1 - 1) / nsx;
            fence_acq_rel_gpu();
            for (int row = sy_lo; row <= sy_hi; ++row) {
                const int n = min(it.s1, (row + 1) * nsx) - max(it.s0, row * nsx);
                red_relaxed_gpu_add(p.prog + dq->prog_off + row, (unsigned)n);
            }
        }
    }
}

// Launch with as many blocks as fit on the GPU at once (fewer if there are
// fewer items); blocks that start later take items as they come.
// step_blocks: blocks of the per-step grid (pg[npg]).
template <int Q, int MODEL, int ST, int VEC, int NOISE>
static cudaError_t launch_persistent_one(const StepArgs &a, const PersistArgs &p, int step_blocks, int warps,
                                         cudaStream_t stream)
{
    auto kern = step_persistent_kernel<Q, MODEL, ST, VEC, NOISE>;
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

template <int Q, int MODEL, int ST, int VEC>
static cudaError_t launch_persistent_mv(int noise, const StepArgs &a, const PersistArgs &p, int step_blocks,
                                        int warps, cudaStream_t stream)
{
    if (noise == 0) return launch_persistent_one<Q, MODEL, ST, VEC, 0>(a, p, step_blocks, warps, stream);
    if (noise == 1) return launch_persistent_one<Q, MODEL, ST, VEC, 1>(a, p, step_blocks, warps, stream);
    return launch_persistent_one<Q, MODEL, ST, VEC, 2>(a, p, step_blocks, warps, stream);
}

template <int Q, int MODEL, int ST>
static cudaError_t launch_persistent_m(int vec, int noise, const StepArgs &a, const PersistArgs &p, int step_blocks,
                                       int warps, cudaStream_t stream)
{
    switch (vec) {
    case 1: return launch_persistent_mv<Q, MODEL, ST, 1>(noise, a, p, step_blocks, warps, stream);
    case 2: return launch_persistent_mv<Q, MODEL, ST, 2>(noise, a, p, step_blocks, warps, stream);
    case 4: return launch_persistent_mv<Q, MODEL, ST, 4>(noise, a, p, step_blocks, warps, stream);
    case 8:
        if constexpr (ST != ST_F32) return launch_persistent_mv<Q, MODEL, ST, 8>(noise, a, p, step_blocks, warps, stream);
        return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <int Q, int ST>
static cudaError_t launch_persistent_storage(int model, int vec, int noise, const StepArgs &a, const PersistArgs &p,
                                             int step_blocks, int warps, cudaStream_t stream)
{
    switch (model) {
    case MODEL_PASSIVE: return launch_persistent_m<Q, MODEL_PASSIVE, ST>(vec, noise, a, p, step_blocks, warps, stream);
    case MODEL_MIPS: return launch_persistent_m<Q, MODEL_MIPS, ST>(vec, noise, a, p, step_blocks, warps, stream);
    case MODEL_CIL: return launch_persistent_m<Q, MODEL_CIL, ST>(vec, noise, a, p, step_blocks, warps, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm

#define LBM_INSTANTIATE_PERSISTENT(Q, ST, SUFFIX)                                                           \
    namespace lbm {                                                                                         \
    cudaError_t launch_persistent_##SUFFIX(int model, int vec, int noise, const StepArgs &a,                 \
                                           const PersistArgs &p, int step_blocks, int warps,                 \
                                           cudaStream_t stream)                                              \
    {                                                                                                       \
        return launch_persistent_storage<Q, ST>(model, vec, noise, a, p, step_blocks, warps, stream);        \
    }                                                                                                       \
    }

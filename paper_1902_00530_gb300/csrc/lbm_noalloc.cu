// lbm_noalloc.cu -- observables of a population field without any allocation.
//
// For callers that cannot allocate device memory -- code running inside a
// memory pool that forbids new allocations, an embedding whose device memory
// footprint is fixed, or a host whose allocator is owned by another runtime
// -- this entry point reduces a dense
// FP32 population field to the observables of lbm_observables using a fixed
// scratch array compiled into the library instead of caller-provided scratch.
//
// The scratch is one file-scope __device__ array (LBM_NOALLOC_SCRATCH_BYTES,
// about 1.1 MB), resident on every GPU that loads the library until the
// process exits.  Host code cannot use the array's name as a device address;
// the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it.  Every call
// shares the array: calls whose work overlaps on the GPU (two streams, or two
// host threads) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int NA_BLOCKS = 32;        // row-interleaved blocks of the partial pass
constexpr int NA_THREADS = 256;
constexpr int NA_MAX_SIDE = LBM_NOALLOC_MAX_SIDE;
constexpr int NA_MAX_DEVICES = 64;
// layout (doubles): [NA_BLOCKS][5] scalars | [NA_BLOCKS][NA_MAX_SIDE] column sums |
//                   [NA_MAX_SIDE] row sums | [8] record
constexpr size_t NA_SCAL = 0;
constexpr size_t NA_COL = NA_SCAL + (size_t)NA_BLOCKS * 5;
constexpr size_t NA_ROW = NA_COL + (size_t)NA_BLOCKS * NA_MAX_SIDE;
constexpr size_t NA_REC = NA_ROW + (size_t)NA_MAX_SIDE;
constexpr size_t NA_DOUBLES = NA_REC + 8;
static_assert(NA_DOUBLES * sizeof(double) <= LBM_NOALLOC_SCRATCH_BYTES, "scratch size");

static __device__ __align__(256) double na_scratch[LBM_NOALLOC_SCRATCH_BYTES / sizeof(double)];

std::mutex na_mutex;
void *na_ptr[NA_MAX_DEVICES] = {};

__device__ double na_block_sum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NA_THREADS / 32; ++w) t += sh[w];
    __syncthreads();
    return t;  // valid in thread 0
}

// Pass 1: block b takes rows b, b + NA_BLOCKS, ...; thread k the columns
// k, k + NA_THREADS, ...  Per-site density and momentum in FP32 (the same sums
// as the library's other reductions), accumulated in FP64.
__global__ void __launch_bounds__(NA_THREADS) na_partials(const float *f, int nx, int ny, double *scratch)
{
    __shared__ double sh[NA_THREADS / 32];
    const size_t plane = (size_t)nx * ny;
    double s_rho = 0, s_jx = 0, s_jy = 0, s_r2 = 0, s_j = 0;
    double *col = scratch + NA_COL + (size_t)blockIdx.x * NA_MAX_SIDE;
    for (int x = threadIdx.x; x < nx; x += NA_THREADS) col[x] = 0.0;
    for (int y = blockIdx.x; y < ny; y += NA_BLOCKS) {
        double row = 0.0;
        for (int x = threadIdx.x; x < nx; x += NA_THREADS) {
            const size_t c = (size_t)y * nx + x;
            float g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = f[i * plane + c];
            const float r = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
            const float jx = (g[1] + g[5] + g[8]) - (g[3] + g[6] + g[7]);
            const float jy = (g[2] + g[5] + g[6]) - (g[4] + g[7] + g[8]);
            s_rho += r;
            s_jx += jx;
            s_jy += jy;
            s_r2 += (double)(r * r);
            s_j += (double)sqrtf(jx * jx + jy * jy);
            row += r;
            col[x] += r;
        }
        const double t = na_block_sum(row, sh);
        if (threadIdx.x == 0) scratch[NA_ROW + y] = t;
    }
    const double v[5] = {s_rho, s_jx, s_jy, s_r2, s_j};
    for (int q = 0; q < 5; ++q) {
        const double t = na_block_sum(v[q], sh);
        if (threadIdx.x == 0) scratch[NA_SCAL + (size_t)blockIdx.x * 5 + q] = t;
    }
}

// Pass 2 (one block): combine the partials in a fixed order into a record.
__global__ void __launch_bounds__(NA_THREADS) na_finish(int nx, int ny, double B, double *scratch)
{
    __shared__ double sh[NA_THREADS / 32];
    double cs = 0, cs2 = 0, rs = 0, rs2 = 0;
    for (int x = threadIdx.x; x < nx; x += NA_THREADS) {
        double c = 0;
        for (int b = 0; b < NA_BLOCKS; ++b) c += scratch[NA_COL + (size_t)b * NA_MAX_SIDE + x];
        cs += c;
        cs2 += c * c;
    }
    for (int y = threadIdx.x; y < ny; y += NA_THREADS) {
        const double r = scratch[NA_ROW + y];
        rs += r;
        rs2 += r * r;
    }
    const double t_cs = na_block_sum(cs, sh), t_cs2 = na_block_sum(cs2, sh);
    const double t_rs = na_block_sum(rs, sh), t_rs2 = na_block_sum(rs2, sh);
    if (threadIdx.x != 0) return;
    double S[5] = {0, 0, 0, 0, 0};
    for (int b = 0; b < NA_BLOCKS; ++b)
        for (int q = 0; q < 5; ++q) S[q] += scratch[NA_SCAL + (size_t)b * 5 + q];
    const double n = (double)nx * ny, mass = S[0], mean = mass / n;
    const double mc = t_cs / ((double)ny * nx), vyv = t_cs2 / ((double)ny * ny * nx) - mc * mc;
    const double mr = t_rs / ((double)nx * ny), vxv = t_rs2 / ((double)nx * nx * ny) - mr * mr;
    double *rec = scratch + NA_REC;
    rec[0] = 0.0;
    rec[1] = mass;
    rec[2] = sqrt(S[1] * S[1] + S[2] * S[2]) / mass;
    rec[3] = sqrt(fmax(vyv, 0.0));
    rec[4] = sqrt(fmax(vxv, 0.0));
    rec[5] = fmax(S[3] / n - mean * mean, 0.0);
    rec[6] = B - S[4] / mass;
    rec[7] = 0.0;
}

}  // namespace

extern "C" lbm_status lbm_observables_noalloc(const float *f_dev, int32_t nx, int32_t ny, double B, lbm_obs *out,
                                              void *cuda_stream)
{
    if (!f_dev || !out || nx < 1 || ny < 1 || nx > NA_MAX_SIDE || ny > NA_MAX_SIDE || !std::isfinite(B))
        return LBM_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return LBM_ERR_CUDA;
    void *ptr;
    {
        std::lock_guard<std::mutex> lock(na_mutex);
        if (!na_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, na_scratch) != cudaSuccess || !p) return LBM_ERR_CUDA;
            na_ptr[dev] = p;
        }
        ptr = na_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double *scratch = static_cast<double *>(ptr);
    na_partials<<<NA_BLOCKS, NA_THREADS, 0, s>>>(f_dev, nx, ny, scratch);
    na_finish<<<1, NA_THREADS, 0, s>>>(nx, ny, B, scratch);
    double rec[8];
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaMemcpyAsync(rec, scratch + NA_REC, sizeof(rec), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_ERR_CUDA;
    out->t = 0;
    out->mass = rec[1];
    out->phi = rec[2];
    out->drho_y = rec[3];
    out->drho_x = rec[4];
    out->var_rho = rec[5];
    out->zeta = rec[6];
    if (!(std::isfinite(rec[1]) && std::isfinite(rec[2]) && std::isfinite(rec[6]))) return LBM_ERR_NUMERIC;
    return LBM_OK;
}

// lbm_aux.cu -- initialisation, moment output, state exchange and the
// observable finaliser.  Small kernels around the fused step.
#include "lbm_internal.h"
#include "lbm_step_staged.cuh"  // the bounded barrier wait of the staged kernels

namespace lbm {

// ---------------------------------------------------------------------------
// Initial state (App. C.2): per site two Philox words give rho and the
// direction of u; populations are f^SS(rho, u) evaluated in FP64 and rounded
// once to the storage type.  Counter purpose 1, t = 0, call 0.
// ---------------------------------------------------------------------------
struct InitSpecDev {
    double rho_mean, rho_amp, u_amp, ux0, uy0, A, B;
    int u_kind, pad;
};

template <int ST>
__global__ void init_kernel(const LatDesc *desc, const InitSpecDev *specs, int dst,
                            uint32_t key0, uint32_t key1)
{
    using T = typename Store<ST>::T;
    const LatDesc d = desc[blockIdx.y];
    const Shift3 shf = load_shift(&d);
    const InitSpecDev sp = specs[blockIdx.y];
    const long long n = (long long)d.nx * d.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % d.nx), y = (int)(c / d.nx);
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)x, (uint32_t)y, 0u, ((uint32_t)d.id & 0xFFFFFFu) | (1u << 24)), key0, key1);
        const double U0v = ((double)(w.x >> 8) + 0.5) * (1.0 / 16777216.0);
        const double U1v = ((double)(w.y >> 8) + 0.5) * (1.0 / 16777216.0);
        const double U2v = ((double)(w.z >> 8) + 0.5) * (1.0 / 16777216.0);
        const double rho = sp.rho_mean * (1.0 + sp.rho_amp * (2.0 * U0v - 1.0));
        double ux, uy;
        if (sp.u_kind == 0) {
            ux = sp.ux0 + sp.u_amp * (2.0 * U1v - 1.0);
            uy = sp.uy0 + sp.u_amp * (2.0 * U2v - 1.0);
        } else {
            double sn, cs;
            sincospi(2.0 * U1v, &sn, &cs);
            double mag = sp.u_amp;
            if (sp.u_kind == 2) {
                const double ar2 = sp.A * rho * rho;
                mag = sp.B >= ar2 ? sp.B - ar2 : 0.0;
                ux = mag * cs;
                uy = mag * sn;
            } else {
                ux = sp.ux0 + mag * cs;
                uy = sp.uy0 + mag * sn;
            }
        }
        const double usq = ux * ux + uy * uy;
        T *base = reinterpret_cast<T *>(d.f[dst]);
        const size_t plane = (size_t)d.ny * d.pitch;
        auto put = [&](int i, double feq, float shift) {
            T v;
            if constexpr (ST == ST_F32) v = (float)feq;
            else if constexpr (ST == ST_F16) v = __double2half(feq - (double)shift);
            else v = __double2bfloat16(feq - (double)shift);
            base[i * plane + (size_t)y * d.pitch + x] = v;
        };
        if (d.q == 7) {
            // Eq. (fssD2Q7): w_i rho [1 + 4 e.u + 8 (e.u)^2 - 2 u^2], e_i at (i-1) pi/3
            const double hs3 = 0.86602540378443864676;
            const double ex[7] = {0.0, 1.0, 0.5, -0.5, -1.0, -0.5, 0.5};
            const double ey[7] = {0.0, 0.0, hs3, hs3, 0.0, -hs3, -hs3};
#pragma unroll
            for (int i = 0; i < 7; ++i) {
                const double eu = ex[i] * ux + ey[i] * uy;
                put(i, wq7_d(i) * rho * (1.0 + 4.0 * eu + 8.0 * eu * eu - 2.0 * usq), shf.q7(i));
            }
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const double eu = vx(i) * ux + vy(i) * uy;
                put(i, wq_d(i) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq), shf.q9(i));
            }
        }
    }
}

// Stored state -> dense FP32 moments (rho, ux, uy) [ny][nx].
template <int ST>
__global__ void moments_kernel(const LatDesc *desc, int lat, int src, float *rho, float *ux, float *uy)
{
    using T = typename Store<ST>::T;
    const LatDesc d = desc[lat];
    const Shift3 shf = load_shift(&d);
    const T *base = reinterpret_cast<const T *>(d.f[src]);
    const size_t plane = (size_t)d.ny * d.pitch;
    const long long n = (long long)d.nx * d.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % d.nx), y = (int)(c / d.nx);
        float f[9];
        float r, jx, jy;
        if (d.q == 7) {
#pragma unroll
            for (int i = 0; i < 7; ++i)
                f[i] = load_one<ST>(base + i * plane + (size_t)y * d.pitch + x, shf.q7(i));
            r = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + f[6]);
            jx = (f[1] - f[4]) + 0.5f * ((f[2] + f[6]) - (f[3] + f[5]));
            jy = 0.86602540378443865f * ((f[2] + f[3]) - (f[5] + f[6]));
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i)
                f[i] = load_one<ST>(base + i * plane + (size_t)y * d.pitch + x, shf.q9(i));
            r = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
            jx = (f[1] + f[5] + f[8]) - (f[3] + f[6] + f[7]);
            jy = (f[2] + f[5] + f[6]) - (f[4] + f[7] + f[8]);
        }
        rho[c] = r;
        ux[c] = r > 0.f ? jx / r : 0.f;
        uy[c] = r > 0.f ? jy / r : 0.f;
    }
}

// Stored state <-> dense FP32 populations [q][ny][nx].
template <int ST>
__global__ void export_kernel(const LatDesc *desc, int lat, int src, float *out)
{
    using T = typename Store<ST>::T;
    const LatDesc d = desc[lat];
    const Shift3 shf = load_shift(&d);
    const T *base = reinterpret_cast<const T *>(d.f[src]);
    const size_t plane = (size_t)d.ny * d.pitch;
    const long long n = (long long)d.nx * d.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < (long long)d.q * n;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c / n);
        const long long r = c % n;
        const int x = (int)(r % d.nx), y = (int)(r / d.nx);
        out[c] = Store<ST>::get(base[i * plane + (size_t)y * d.pitch + x], shf.of(d.q, i));
    }
}

template <int ST>
__global__ void import_kernel(const LatDesc *desc, int lat, int dst, const float *in)
{
    using T = typename Store<ST>::T;
    const LatDesc d = desc[lat];
    const Shift3 shf = load_shift(&d);
    T *base = reinterpret_cast<T *>(d.f[dst]);
    const size_t plane = (size_t)d.ny * d.pitch;
    const long long n = (long long)d.nx * d.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < (long long)d.q * n;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c / n);
        const long long r = c % n;
        const int x = (int)(r % d.nx), y = (int)(r / d.nx);
        base[i * plane + (size_t)y * d.pitch + x] = Store<ST>::put(in[c], shf.of(d.q, i));
    }
}

// Add a constant to every population of one lattice (App. C.2 density step).
template <int ST>
__global__ void add_density_kernel(const LatDesc *desc, int lat, int buf, float per_population)
{
    using T = typename Store<ST>::T;
    const LatDesc d = desc[lat];
    const Shift3 shf = load_shift(&d);
    T *base = reinterpret_cast<T *>(d.f[buf]);
    const size_t plane = (size_t)d.ny * d.pitch;
    const long long n = (long long)d.nx * d.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < (long long)d.q * n;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c / n);
        const long long r = c % n;
        const int x = (int)(r % d.nx), y = (int)(r / d.nx);
        T *p = base + i * plane + (size_t)y * d.pitch + x;
        const float shift = shf.of(d.q, i);
        *p = Store<ST>::put(__fadd_rn(Store<ST>::get(*p, shift), per_population), shift);
    }
}

// ---------------------------------------------------------------------------
// Observable finaliser.  Grid (nchunk, nlat): block (c, l) sums, in a fixed
// order, chunk c of lattice l's column partials (over strip rows), row
// partials (over strip columns) and per-strip scalars, and writes nine chunk
// sums.  The last block to arrive for a lattice combines the chunks in chunk
// order and writes one record: deterministic whatever the arrival order.
// ---------------------------------------------------------------------------
constexpr int FIN_THREADS = 256;

__device__ double block_sum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(FIN_THREADS) finalize_kernel(const LatDesc *desc, int nlat,
                                                               const uint32_t *t_ptr, uint32_t k,
                                                               int to_ring, unsigned *err)
{
    __shared__ double sh[FIN_THREADS / 32];
    __shared__ bool am_last;
    const int l = blockIdx.y;
    if (l >= nlat) return;
    const LatDesc d = desc[l];
    const int c = blockIdx.x;
    if (c >= d.nchunk) return;
    const int nstrip = d.nsx * d.nsy;
    // this chunk's share of columns, rows and strips
    const int cx0 = (int)((long long)d.nx * c / d.nchunk), cx1 = (int)((long long)d.nx * (c + 1) / d.nchunk);
    const int cy0 = (int)((long long)d.ny * c / d.nchunk), cy1 = (int)((long long)d.ny * (c + 1) / d.nchunk);
    const int cs0 = (int)((long long)nstrip * c / d.nchunk), cs1 = (int)((long long)nstrip * (c + 1) / d.nchunk);
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int s = cs0 + threadIdx.x; s < cs1; s += blockDim.x)
        for (int q = 0; q < 5; ++q) v[q] += d.scal[(size_t)s * 5 + q];
    for (int x = cx0 + threadIdx.x; x < cx1; x += blockDim.x) {
        double cs = 0.0;
        for (int sy = 0; sy < d.nsy; ++sy) cs += d.colp[(size_t)sy * d.nx + x];
        v[5] += cs;
        v[6] += cs * cs;
    }
    for (int y = cy0 + threadIdx.x; y < cy1; y += blockDim.x) {
        double rs = 0.0;
        for (int sx = 0; sx < d.nsx; ++sx) rs += d.rowp[(size_t)sx * d.ny + y];
        v[7] += rs;
        v[8] += rs * rs;
    }
    for (int q = 0; q < 9; ++q) {
        const double t = block_sum(v[q], sh);
        if (threadIdx.x == 0) d.finp[(size_t)c * 9 + q] = t;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(&d.counters[1], 1u);
        am_last = (ticket == (unsigned)d.nchunk - 1);
    }
    __syncthreads();
    if (!am_last || threadIdx.x != 0) return;
    __threadfence();
    double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int cc = 0; cc < d.nchunk; ++cc)
        for (int q = 0; q < 9; ++q) S[q] += ((volatile double *)d.finp)[(size_t)cc * 9 + q];
    const double n = (double)d.nx * (double)d.ny;
    const double mass = S[0];
    const double mean = mass / n;
    const double phi = sqrt(S[1] * S[1] + S[2] * S[2]) / mass;
    // column means rho_y(x) = colsum / ny; population std over x
    const double mcol = S[5] / ((double)d.ny * d.nx);
    const double vy = S[6] / ((double)d.ny * d.ny * d.nx) - mcol * mcol;
    const double mrow = S[7] / ((double)d.nx * d.ny);
    const double vxr = S[8] / ((double)d.nx * d.nx * d.ny) - mrow * mrow;
    const double var = S[3] / n - mean * mean;
    const double zeta = (double)d.B - S[4] / mass;
    double rec[8];
    const uint32_t tt = *t_ptr + k + (to_ring ? 1u : 0u);
    rec[0] = __longlong_as_double((long long)tt);
    rec[1] = mass;
    rec[2] = phi;
    rec[3] = sqrt(fmax(vy, 0.0));
    rec[4] = sqrt(fmax(vxr, 0.0));
    rec[5] = fmax(var, 0.0);
    rec[6] = zeta;
    rec[7] = 0.0;
    bool finite = isfinite(mass) && isfinite(phi) && isfinite(vy) && isfinite(vxr) && isfinite(zeta);
    if (!finite) atomicOr(err, (unsigned)DEVERR_NUMERIC);
    double *out;
    if (to_ring) {
        const unsigned idx = d.counters[0];
        out = d.ring + (size_t)(idx % (unsigned)d.ring_cap) * 8;
        d.counters[0] = idx + 1;
    } else {
        out = d.now;
    }
    for (int q = 0; q < 8; ++q) out[q] = rec[q];
    d.counters[1] = 0;
    __threadfence();
}

__global__ void advance_time_kernel(uint32_t *t_ptr, uint32_t n) { *t_ptr += n; }

__global__ void set_time_kernel(uint32_t *t_ptr, uint32_t t) { *t_ptr = t; }

// The failure path of the staged kernels' waits, exercised on purpose: one
// warp waits, with the same bounded wait, on a barrier phase that nothing
// completes; the wait gives up after its limit (about 1 s) and the warp raises
// the timeout flag, as a step kernel does when a staged row never arrives.
__global__ void wait_timeout_kernel(unsigned *err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncwarp();
    if (!stage_wait(&bar, 0u) && threadIdx.x == 0) atomicOr(err, (unsigned)DEVERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int grid_for(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    if (b > 152LL * 64) b = 152LL * 64;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_init(int storage, const LatDesc *desc, const void *specs, int nlat, long long max_cells,
                        int dst, uint64_t seed, cudaStream_t s)
{
    dim3 g(grid_for(max_cells, 256), nlat);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const InitSpecDev *sp = reinterpret_cast<const InitSpecDev *>(specs);
    if (storage == ST_F32) init_kernel<ST_F32><<<g, 256, 0, s>>>(desc, sp, dst, k0, k1);
    else if (storage == ST_F16) init_kernel<ST_F16><<<g, 256, 0, s>>>(desc, sp, dst, k0, k1);
    else init_kernel<ST_BF16><<<g, 256, 0, s>>>(desc, sp, dst, k0, k1);
    return cudaGetLastError();
}

size_t init_spec_bytes() { return sizeof(InitSpecDev); }

void pack_init_spec(void *dst, double rho_mean, double rho_amp, int u_kind, double u_amp, double ux0,
                    double uy0, double A, double B)
{
    InitSpecDev s;
    s.rho_mean = rho_mean;
    s.rho_amp = rho_amp;
    s.u_amp = u_amp;
    s.ux0 = ux0;
    s.uy0 = uy0;
    s.A = A;
    s.B = B;
    s.u_kind = u_kind;
    s.pad = 0;
    *reinterpret_cast<InitSpecDev *>(dst) = s;
}

cudaError_t launch_moments(int storage, const LatDesc *desc, int lat, long long cells, int src, float *rho,
                           float *ux, float *uy, cudaStream_t s)
{
    const int g = grid_for(cells, 256);
    if (storage == ST_F32) moments_kernel<ST_F32><<<g, 256, 0, s>>>(desc, lat, src, rho, ux, uy);
    else if (storage == ST_F16) moments_kernel<ST_F16><<<g, 256, 0, s>>>(desc, lat, src, rho, ux, uy);
    else moments_kernel<ST_BF16><<<g, 256, 0, s>>>(desc, lat, src, rho, ux, uy);
    return cudaGetLastError();
}

cudaError_t launch_export(int storage, const LatDesc *desc, int lat, long long cells, int src, float *out,
                          cudaStream_t s)
{
    const int g = grid_for(9 * cells, 256);  // enough for q <= 9
    if (storage == ST_F32) export_kernel<ST_F32><<<g, 256, 0, s>>>(desc, lat, src, out);
    else if (storage == ST_F16) export_kernel<ST_F16><<<g, 256, 0, s>>>(desc, lat, src, out);
    else export_kernel<ST_BF16><<<g, 256, 0, s>>>(desc, lat, src, out);
    return cudaGetLastError();
}

cudaError_t launch_import(int storage, const LatDesc *desc, int lat, long long cells, int dst, const float *in,
                          cudaStream_t s)
{
    const int g = grid_for(9 * cells, 256);  // enough for q <= 9
    if (storage == ST_F32) import_kernel<ST_F32><<<g, 256, 0, s>>>(desc, lat, dst, in);
    else if (storage == ST_F16) import_kernel<ST_F16><<<g, 256, 0, s>>>(desc, lat, dst, in);
    else import_kernel<ST_BF16><<<g, 256, 0, s>>>(desc, lat, dst, in);
    return cudaGetLastError();
}

cudaError_t launch_add_density(int storage, const LatDesc *desc, int lat, long long cells, int buf, float per_pop,
                               cudaStream_t s)
{
    const int g = grid_for(9 * cells, 256);  // enough for q <= 9
    if (storage == ST_F32) add_density_kernel<ST_F32><<<g, 256, 0, s>>>(desc, lat, buf, per_pop);
    else if (storage == ST_F16) add_density_kernel<ST_F16><<<g, 256, 0, s>>>(desc, lat, buf, per_pop);
    else add_density_kernel<ST_BF16><<<g, 256, 0, s>>>(desc, lat, buf, per_pop);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const LatDesc *desc, int nlat, int max_chunk, const uint32_t *t_ptr, uint32_t k,
                            int to_ring, unsigned *err, cudaStream_t s)
{
    dim3 g(max_chunk, nlat);
    finalize_kernel<<<g, FIN_THREADS, 0, s>>>(desc, nlat, t_ptr, k, to_ring, err);
    return cudaGetLastError();
}

cudaError_t launch_advance_time(uint32_t *t_ptr, uint32_t n, cudaStream_t s)
{
    advance_time_kernel<<<1, 1, 0, s>>>(t_ptr, n);
    return cudaGetLastError();
}

cudaError_t launch_wait_timeout(unsigned *err, cudaStream_t s)
{
    wait_timeout_kernel<<<1, 32, 0, s>>>(err);
    return cudaGetLastError();
}

cudaError_t launch_set_time(uint32_t *t_ptr, uint32_t t, cudaStream_t s)
{
    set_time_kernel<<<1, 1, 0, s>>>(t_ptr, t);
    return cudaGetLastError();
}

}  // namespace lbm

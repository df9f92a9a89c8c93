// lbm_device.cuh -- device-side pieces of the fused active-LBM step for sm_103a.
//
// The step (App. A.2 of arXiv:1902.00530) per site: pull-stream the nine
// populations, form rho and u, the steady-state velocity u* of the model,
// f^SS = xi(rho, u*) (Eq. (fssD2Q7) in D2Q9 form), BGK relaxation, zero-sum
// uniform noise (Eq. (noiseDensityConservation)) and the negative correction
// (App. A.3), all in registers, in one pass over HBM.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr unsigned FULL = 0xffffffffu;

// D2Q9 velocity set: 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+x,+y), 6 (-x,+y),
// 7 (-x,-y), 8 (+x,-y).
__host__ __device__ constexpr int vx(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int vy(int i)
{
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int reverse_of(int i)
{
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}
__host__ __device__ constexpr float wq(int i)
{
    return i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr double wq_d(int i)
{
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}
static_assert(reverse_of(1) == 3 && reverse_of(2) == 4 && reverse_of(3) == 1 &&
                  reverse_of(4) == 2 && reverse_of(5) == 7 && reverse_of(6) == 8 &&
                  reverse_of(7) == 5 && reverse_of(8) == 6,
              "D2Q9 reverse directions");

// D2Q7 weights (Sec. 2): 1/2 for the rest population, 1/12 for the six moving
// ones; velocities e_i = (cos((i-1) pi/3), sin((i-1) pi/3)).
__host__ __device__ constexpr float wq7(int i) { return i == 0 ? 0.5f : 1.0f / 12.0f; }
__host__ __device__ constexpr double wq7_d(int i) { return i == 0 ? 0.5 : 1.0 / 12.0; }


enum { MODEL_PASSIVE = 0, MODEL_MIPS = 1, MODEL_CIL = 2 };
enum { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };
enum { DEVERR_NUMERIC = 1u, DEVERR_TIMEOUT = 2u };

// Per-lattice descriptor, resident in device memory for the whole run.
struct LatDesc {
    void *f[2];          // the two population buffers, [q][ny][pitch] of the storage type
    double *scal;        // [nstrips][5] per-strip sums: rho, jx, jy, rho^2, |j|
    double *colp;        // [nsy][nx] per-strip-row column sums of rho
    double *rowp;        // [nsx][ny] per-strip-column row sums of rho
    double *finp;        // [nchunk][9] finaliser chunk partials
    double *ring;        // [ring_cap][8] observable records
    double *now;         // [8] on-demand observable record
    unsigned *counters;  // [2]: samples written, finaliser arrivals
    int nx, ny, pitch, id;
    int nsx, nsy, rows, block_begin;
    int ring_cap, nchunk;
    int q;               // populations per site: 9 (D2Q9) or 7 (D2Q7)
    int prog_off;        // persistent launch: index of this lattice's first strip-row progress counter
    float omega;         // 1/tau
    float sigma_q;       // 2 sigma: noise scale of u in [1, 2) (0 = no noise)
    float C, inv_rho_star, rho_star, u_max, u_max2, A, B;
    float rho0;          // reference density of the storage shift
    float sh[3];         // storage shifts per weight class (see Shift3)
};

// The shift of 16-bit storage, s_i = f_i - shift_i with shift_i = w_i rho0,
// per weight class: rest, axis (D2Q7: every moving population), diagonal.
// The host rounds each shift to a value the storage type holds exactly
// (storage_shift), so that a population the negative correction set to zero,
// or one equal to its shift, is stored exactly: with a shift the format rounds
// (1/9 and 1/36 are not dyadic), every such store would err the same way, a
// systematic drift of mass and momentum.  FP32 storage ignores the shift.
struct Shift3 {
    float c[3];
    __host__ __device__ __forceinline__ float q9(int i) const { return i == 0 ? c[0] : (i <= 4 ? c[1] : c[2]); }
    __host__ __device__ __forceinline__ float q7(int i) const { return i == 0 ? c[0] : c[1]; }
    __host__ __device__ __forceinline__ float of(int q, int i) const { return q == 7 ? q7(i) : q9(i); }
};

__host__ __device__ __forceinline__ Shift3 load_shift(const LatDesc *d)
{
    Shift3 s;
    s.c[0] = d->sh[0];
    s.c[1] = d->sh[1];
    s.c[2] = d->sh[2];
    return s;
}

// w rho0 in FP32, rounded to the nearest value of the storage type.
inline float storage_shift(int storage, double w, float rho0)
{
    const float s = (float)(w * (double)rho0);
    if (storage == ST_F16) return __half2float(__float2half_rn(s));
    if (storage == ST_BF16) return __bfloat162float(__float2bfloat16_rn(s));
    return s;
}

// Dynamic shared memory of a staged block: `stages` row buffers of q
// population segments, each the block's 32 vec warps columns plus a 16-byte
// halo on both sides, and a "full" and an "empty" barrier per buffer; with
// `conv`, also two FP32 rows of the q pulled populations of the block's sites
// (the converted rows the MIPS update of 16-bit storage reads).
__host__ __device__ constexpr size_t staged_smem_bytes(int q, int elem_bytes, int vec, int warps, int stages,
                                                       bool conv = false)
{
    return (size_t)stages * ((size_t)q * (size_t)(warps * 32 * vec + 2 * (16 / elem_bytes)) * (size_t)elem_bytes + 16) +
           (conv ? 2 * (size_t)q * (size_t)(warps * 32 * vec) * 4 : 0);
}

// Whether a staged MIPS kernel keeps the converted row (above): 16-bit
// storage, where it saves converting each staged value a second time.
#ifndef LBM_CONV_ROWS_F32
#define LBM_CONV_ROWS_F32 0
#endif
__host__ __device__ constexpr bool staged_conv_rows(int model, int storage)
{
    return model == MODEL_MIPS && (storage != ST_F32 || LBM_CONV_ROWS_F32 != 0);
}
// The most dynamic shared memory one block can have on sm_103a (227 KB).
constexpr size_t STAGED_SMEM_MAX = 232448;

struct StepArgs {
    const LatDesc *desc;  // lattices of this launch group
    int nlat;
    int src;              // index of the buffer holding the current state
    const uint32_t *t_ptr;
    uint32_t k;           // step offset of this launch from *t_ptr
    uint32_t key0, key1;  // Philox key = seed
    int stages;           // staged kernel: shared-memory row buffers per warp
    unsigned *err;        // device error word (bounded waits report here)
    uint32_t rk[20];      // Philox round keys: (key0 + r W0, key1 + r W1), r = 0..9
};

// The persistent launch's work list (lbm_step_persistent.cuh): items are the
// blocks of the per-step grid, one per step, taken in order by a counter.
struct PersistArgs {
    unsigned *work;  // item counter, zero at launch
    unsigned *prog;  // strips finished per strip row (summed over the launch), zero at launch
    const int *pg;   // first block of each lattice group; pg[npg] = blocks of the step grid
    int npg;         // lattice groups
    int nsteps;      // steps of the launch: items = nsteps * pg[npg] < 2^31 (host check)
    int retime;      // timing form (the tuner): every item recomputes the first step, from the
                     // current buffer into the spare one, so the state is left as it was
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// -> 64-bit products of counter words 0 and 2, whose high halves are XORed
// with the other counter words and the round key; the key advances by the
// Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53u;
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57u;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same with the ten round keys precomputed (rk[2r], rk[2r+1]).
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t *rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53u;
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57u;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1],
                       (uint32_t)p0);
    }
    return c;
}

// Noise counter: (x, y, t, id | purpose << 24 | call << 28), purpose 0 and
// call 0 for the collision noise.  One Philox call gives four 32-bit words
// w_j: each gives two 14-bit integers, m_2j = bits 18..31 and m_2j+1 = bits
// 4..17, and m_8 gathers bits 0..3 of w_0, w_1, w_2 and bits 0..1 of w_3 (w_0's
// lowest first).  The variate s_i = (2 m_i + 1 - 2^14) 2^-14 is built without
// an integer conversion: u_i = 1 + (m_i + 1/2) 2^-14 is assembled directly as
// FP32 bits (exponent of 1, m_i in the top 14 mantissa bits, then a 1), and
// s_i = 2 u_i - 3 exactly.  The zero-sum noise is then eta_i = sigma (s_i -
// mean s) = 2 sigma (u_i - mean u).
__device__ __forceinline__ float u_from_bits(uint32_t mantissa14_at_bit9)
{
    return __uint_as_float(0x3F800100u | mantissa14_at_bit9);
}

// ---------------------------------------------------------------------------
// Storage: FP32, or 16-bit values of s = f - w_i rho0 (FP16 / BF16, RN).
// ---------------------------------------------------------------------------
template <int ST> struct Store;
template <> struct Store<ST_F32> {
    using T = float;
    __device__ static __forceinline__ float get(T v, float) { return v; }
    __device__ static __forceinline__ T put(float f, float) { return f; }
};
// The 16-bit forms also convert two values at a time (packed conversions and
// a paired shift, the same round-to-nearest per element): put2 packs (a, b)
// into one word, a in the low half, and get2 unpacks it.
template <> struct Store<ST_F16> {
    using T = __half;
    __device__ static __forceinline__ float get(T v, float shift) { return __half2float(v) + shift; }
    __device__ static __forceinline__ T put(float f, float shift) { return __float2half_rn(f - shift); }
    __device__ static __forceinline__ uint32_t put2(float a, float b, float shift)
    {
        const float2 s = __fadd2_rn(make_float2(a, b), make_float2(-shift, -shift));
        const __half2 h = __floats2half2_rn(s.x, s.y);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    __device__ static __forceinline__ void get2(uint32_t w, float shift, float &a, float &b)
    {
        const float2 v = __fadd2_rn(__half22float2(*reinterpret_cast<const __half2 *>(&w)), make_float2(shift, shift));
        a = v.x;
        b = v.y;
    }
};
template <> struct Store<ST_BF16> {
    using T = __nv_bfloat16;
    __device__ static __forceinline__ float get(T v, float shift)
    {
        return __bfloat162float(v) + shift;
    }
    __device__ static __forceinline__ T put(float f, float shift)
    {
        return __float2bfloat16_rn(f - shift);
    }
    __device__ static __forceinline__ uint32_t put2(float a, float b, float shift)
    {
        const float2 s = __fadd2_rn(make_float2(a, b), make_float2(-shift, -shift));
        const __nv_bfloat162 h = __floats2bfloat162_rn(s.x, s.y);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    __device__ static __forceinline__ void get2(uint32_t w, float shift, float &a, float &b)
    {
        const float2 v =
            __fadd2_rn(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w)), make_float2(shift, shift));
        a = v.x;
        b = v.y;
    }
};

// Expand / pack the 32-bit words of a vector of VEC 16-bit values (VEC even).
template <int ST, int VEC>
__device__ __forceinline__ void unpack_words(const uint32_t *w, float shift, float out[VEC])
{
#pragma unroll
    for (int k = 0; k < VEC / 2; ++k) Store<ST>::get2(w[k], shift, out[2 * k], out[2 * k + 1]);
}
template <int ST, int VEC>
__device__ __forceinline__ void pack_words(const float in[VEC], float shift, uint32_t *w)
{
#pragma unroll
    for (int k = 0; k < VEC / 2; ++k) w[k] = Store<ST>::put2(in[2 * k], in[2 * k + 1], shift);
}

template <int BYTES> struct VecWord;
template <> struct VecWord<2> { using T = unsigned short; };
template <> struct VecWord<4> { using T = unsigned int; };
template <> struct VecWord<8> { using T = uint2; };
template <> struct VecWord<16> { using T = uint4; };
template <> struct VecWord<32> { using T = uint4; };  // two 16-byte words

// Load VEC consecutive values (aligned to VEC elements) and expand to FP32.
template <int ST, int VEC>
__device__ __forceinline__ void load_vec(const typename Store<ST>::T *p, float shift, float out[VEC])
{
    using T = typename Store<ST>::T;
    constexpr int BYTES = (int)sizeof(T) * VEC;
    if constexpr (BYTES <= 16) {
        using W = typename VecWord<BYTES>::T;
        W w = __ldg(reinterpret_cast<const W *>(p));
        if constexpr (sizeof(T) == 2 && VEC % 2 == 0) {
            unpack_words<ST, VEC>(reinterpret_cast<const uint32_t *>(&w), shift, out);
        } else {
            const T *e = reinterpret_cast<const T *>(&w);
#pragma unroll
            for (int j = 0; j < VEC; ++j) out[j] = Store<ST>::get(e[j], shift);
        }
    } else {
        const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
        for (int h = 0; h < BYTES / 16; ++h) {
            uint4 w = __ldg(q + h);
            constexpr int PER = 16 / (int)sizeof(T);
            if constexpr (sizeof(T) == 2) {
                unpack_words<ST, PER>(reinterpret_cast<const uint32_t *>(&w), shift, out + h * PER);
            } else {
                const T *e = reinterpret_cast<const T *>(&w);
#pragma unroll
                for (int j = 0; j < PER; ++j) out[h * PER + j] = Store<ST>::get(e[j], shift);
            }
        }
    }
}

// The same from any address space (shared memory): a plain vector load.
template <int ST, int VEC>
__device__ __forceinline__ void load_vec_plain(const typename Store<ST>::T *p, float shift, float out[VEC])
{
    using T = typename Store<ST>::T;
    constexpr int BYTES = (int)sizeof(T) * VEC;
    static_assert(BYTES <= 16, "vector wider than 16 bytes");
    using W = typename VecWord<BYTES>::T;
    const W w = *reinterpret_cast<const W *>(p);
    if constexpr (sizeof(T) == 2 && VEC % 2 == 0) {
        unpack_words<ST, VEC>(reinterpret_cast<const uint32_t *>(&w), shift, out);
    } else {
        const T *e = reinterpret_cast<const T *>(&w);
#pragma unroll
        for (int j = 0; j < VEC; ++j) out[j] = Store<ST>::get(e[j], shift);
    }
}

template <int ST, int VEC>
__device__ __forceinline__ void store_vec(typename Store<ST>::T *p, float shift, const float in[VEC])
{
    using T = typename Store<ST>::T;
    constexpr int BYTES = (int)sizeof(T) * VEC;
    if constexpr (BYTES <= 16) {
        using W = typename VecWord<BYTES>::T;
        W w;
        if constexpr (sizeof(T) == 2 && VEC % 2 == 0) {
            pack_words<ST, VEC>(in, shift, reinterpret_cast<uint32_t *>(&w));
        } else {
            T *e = reinterpret_cast<T *>(&w);
#pragma unroll
            for (int j = 0; j < VEC; ++j) e[j] = Store<ST>::put(in[j], shift);
        }
        *reinterpret_cast<W *>(p) = w;
    } else {
        uint4 *q = reinterpret_cast<uint4 *>(p);
#pragma unroll
        for (int h = 0; h < BYTES / 16; ++h) {
            uint4 w;
            constexpr int PER = 16 / (int)sizeof(T);
            if constexpr (sizeof(T) == 2) {
                pack_words<ST, PER>(in + h * PER, shift, reinterpret_cast<uint32_t *>(&w));
            } else {
                T *e = reinterpret_cast<T *>(&w);
#pragma unroll
                for (int j = 0; j < PER; ++j) e[j] = Store<ST>::put(in[h * PER + j], shift);
            }
            q[h] = w;
        }
    }
}

template <int ST>
__device__ __forceinline__ float load_one(const typename Store<ST>::T *p, float shift)
{
    return Store<ST>::get(p[0], shift);
}

__device__ __forceinline__ int wrap_once(int a, int n)
{
    a = a < 0 ? a + n : a;
    return a >= n ? a - n : a;
}

}  // namespace lbm

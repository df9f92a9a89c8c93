// lbm_api.cu -- host side of the C ABI declared in include/lbm.h.
//
// The context holds host descriptors only; all device memory (population
// buffers and scratch) belongs to the caller.  Scratch layout (256-byte
// aligned regions): control words (step counter t, error flag), per-lattice
// counters, descriptor tables (all lattices, then one table per launch group),
// per launch group the persistent launch's work counter, strip-row progress
// counters and lattice-group table, initial-state specs, and per lattice the
// reduction partials, the finaliser partials, the observable ring and the
// on-demand record.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

constexpr int ROWS_MIN = 8;        // smallest strip height; scratch is sized for it
constexpr int CHUNK_COLS = 256;    // columns / rows / strips per finaliser block
constexpr int NCHUNK_MAX = 1024;
constexpr int GRAPH_CHUNK_MAX = 256;
constexpr int PERSIST_STEPS_MAX = 4096;  // steps of one persistent launch
constexpr int TUNE_STEPS = 3;            // steps the tuner times per candidate (per-step launches)
constexpr int TUNE_STEPS_PERSIST = 12;   // ... and as one persistent launch (longer: its fill and drain)
constexpr float TUNE_MIN_MS = 0.25f;     // shorter timings are repeated over more steps (event resolution, noise)
constexpr int TUNE_STEPS_MAX = 256;
// Mode 2 considers persistent launches only for groups with at least this
// many sites per step.  Below it a step's items cannot fill the GPU in either
// form and the persistent launch's dependency waits cost more than a launch
// boundary; measured, 32 lattices of 180 x 60 (0.35 M sites): 26.6 GLUPS
// persistent against 29.0 per step, while the tuner's timing form preferred
// it; 256 of 128^2 (4.2 M): 82.6 against 64.2.
constexpr long long PERSIST_AUTO_MIN_SITES = 1LL << 20;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

size_t elem_bytes(int storage) { return storage == LBM_F32 ? 4 : 2; }

struct LatHost {
    lbm_lattice lat;
    int q = 9;  // populations per site (9 for D2Q9, 7 for D2Q7)
    int model;
    lbm_params p;
    float rho0 = 1.f;
    size_t pitch = 0, buf_bytes = 0, state_off = 0;
    size_t scal_off = 0, colp_off = 0, rowp_off = 0, finp_off = 0, ring_off = 0, now_off = 0, ctr_off = 0;
    int nsx = 0, nsy = 0, nchunk = 1, nchunk_max = 1;
    int group = 0, block_begin = 0;
    int prog_off = 0;  // first strip-row progress counter in its group's persistent region
    int64_t consumed = 0;
};

struct GroupHost {
    int model = 0, storage = 0, q = 9;
    std::vector<int> members;
    int vec = 1, rows = 32, warps = 4, blocks = 0;
    int stages = 0;  // 0: direct-load kernel; >= 2: TMA-staged kernel with that many row buffers
    size_t desc_off = 0;
    // persistent launch: work counter, then progress counters (persist_bytes
    // in all, zeroed before each launch); lattice-group table at pg_off
    size_t persist_off = 0, persist_bytes = 0, pg_off = 0;
    int npg = 0;
    bool persist = false;  // mode 2: the tuner chose persistent launches for this group
};

struct GraphKey {
    int64_t n, phase;
    int parity;
    bool operator<(const GraphKey &o) const
    {
        return std::tie(n, phase, parity) < std::tie(o.n, o.phase, o.parity);
    }
};

}  // namespace

struct lbm_ctx {
    std::vector<LatHost> lats;
    std::vector<GroupHost> groups;
    int32_t sample_every = 0, ring_cap = 0;
    char *state = nullptr, *scratch = nullptr;
    cudaStream_t stream = nullptr;
    bool bound = false, initialized = false;
    uint64_t seed = 0;
    int64_t t = 0;
    int parity = 0;
    std::string err;
    size_t state_bytes = 0, scratch_bytes = 0;
    size_t all_desc_off = 0, spec_off = 0;
    int max_chunk = 1;
    int tune_mode = 0, fixed_vec = 0, fixed_rows = 0;
    bool tuned = false, use_graphs = true;
    std::map<GraphKey, std::pair<cudaGraphExec_t, int64_t>> graphs;  // graph and its kernel launches
    int64_t last_launches = 0;
    // kernel timing (lbm_set_profiling)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    struct ProfMark {
        int ev;         // first event of the pair
        bool step;      // a fused step kernel
        int64_t steps;  // steps it ran (a persistent launch runs several)
    };
    std::vector<ProfMark> ev_marks;
    // persistent launches (lbm_set_persistent): mode 0 off, 1 on, 2 chosen by the tuner
    int persist_mode = 2;
    int persist_l2_mib = 0;  // 0: every lattice of a launch group in one lattice group
    size_t ev_used = 0;
    // launch groups after the first run on their own streams, forked from and
    // joined back into the bound stream (parallel branches of the step graph)
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> aux_ev;  // [0]: fork, [1 + i]: join of aux[i]
};

namespace {

lbm_status fail(lbm_ctx *c, lbm_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

bool finite_all(const lbm_params &p)
{
    const double v[] = {p.tau, p.sigma, p.C, p.rho_star, p.u_max, p.A, p.B, p.rho0};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

std::string validate(const lbm_lattice &l, int model, const lbm_params &p)
{
    if (l.nx < 1 || l.ny < 1 || l.nx > 65536 || l.ny > 65536) return "nx, ny must be in [1, 65536]";
    if (l.storage < LBM_F32 || l.storage > LBM_BF16_SHIFTED) return "unknown storage type";
    if (l.id < 0 || l.id >= (1 << 24)) return "lattice id must be in [0, 2^24)";
    if (l.velocity_set != LBM_D2Q9 && l.velocity_set != LBM_D2Q7) return "unknown velocity set";
    if (l.velocity_set == LBM_D2Q7 && l.ny % 2) return "a periodic D2Q7 box needs an even ny (odd rows are offset)";
    if (model < LBM_PASSIVE || model > LBM_CIL) return "unknown model";
    if (!finite_all(p)) return "parameters must be finite";
    if (!(p.tau > 0.5)) return "tau must exceed 1/2";
    if (p.sigma < 0) return "sigma must be >= 0";
    if (p.rho0 < 0) return "rho0 must be >= 0";
    if (model == LBM_MIPS && !(p.rho_star > 0)) return "MIPS needs rho_star > 0";
    if (model == LBM_MIPS && p.u_max < 0) return "MIPS needs u_max >= 0";
    return "";
}

// The staged kernels copy 16-byte halos: nx must be a multiple of that width.
bool staged_fits(const lbm_lattice &l)
{
    const int halo = l.storage == LBM_F32 ? 4 : 8;
    return l.nx % halo == 0 && l.nx >= halo;
}

// Whether the group's staged kernel keeps converted FP32 rows (MIPS with
// 16-bit storage), and the fewest row buffers its ring needs: MIPS holds two
// rows in use (one with the converted rows) plus one in flight.
bool conv_rows(const GroupHost &g) { return staged_conv_rows(g.model, g.storage); }
int min_stages(const GroupHost &g) { return g.model == LBM_MIPS ? (conv_rows(g) ? 2 : 3) : 2; }

bool staged_ok(const lbm_ctx *c, const GroupHost &g)
{
    for (int m : g.members)
        if (!staged_fits(c->lats[m].lat)) return false;
    return true;
}

// Row pitch in elements: nx rounded up to 128 bytes.
size_t row_pitch(const lbm_lattice &l)
{
    const size_t align_elems = 128 / elem_bytes(l.storage);
    return ((size_t)l.nx + align_elems - 1) / align_elems * align_elems;
}

// The direct D2Q9 kernel addresses a state buffer by unsigned 32-bit element
// index (i plane + row pitch + x): its q ny pitch elements must not exceed 2^32.
bool index32_fits(const lbm_lattice &l, int q)
{
    return q != 9 || (size_t)q * (size_t)l.ny * row_pitch(l) <= ((size_t)1 << 32);
}

bool direct_ok(const lbm_ctx *c, const GroupHost &g)
{
    for (int m : g.members)
        if (!index32_fits(c->lats[m].lat, g.q)) return false;
    return true;
}

int allowed_vec(int storage, int v)
{
    if (storage == LBM_F32) return v == 1 || v == 2 || v == 4;
    return v == 1 || v == 2 || v == 4 || v == 8;
}

int default_vec(const lbm_ctx *c, const GroupHost &g)
{
    const int cands_f32[] = {4, 2, 1};
    const int cands_16[] = {8, 4, 2, 1};
    const int *cands = g.storage == LBM_F32 ? cands_f32 : cands_16;
    const int nc = g.storage == LBM_F32 ? 3 : 4;
    for (int k = 0; k < nc; ++k) {
        bool ok = true;
        for (int m : g.members) ok = ok && (c->lats[m].lat.nx % cands[k] == 0);
        if (ok) return cands[k];
    }
    return 1;
}

// Scratch / state layout; depends only on the lattices and sampling settings.
void layout(lbm_ctx *c)
{
    size_t so = 0;
    for (auto &L : c->lats) {
        const size_t eb = elem_bytes(L.lat.storage);
        L.pitch = row_pitch(L.lat);
        L.buf_bytes = align256((size_t)L.q * L.lat.ny * L.pitch * eb);
        L.state_off = so;
        so += 2 * L.buf_bytes;
    }
    c->state_bytes = so;
    const int nl = (int)c->lats.size();
    size_t o = 256;  // [0]: t (uint32), [4]: error flag (uint32)
    for (auto &L : c->lats) {
        L.ctr_off = o;
        o += 16;
    }
    o = align256(o);
    c->all_desc_off = o;
    o = align256(o + nl * sizeof(LatDesc));
    for (auto &g : c->groups) {
        g.desc_off = o;
        o = align256(o + g.members.size() * sizeof(LatDesc));
    }
    for (auto &g : c->groups) {
        // the work counter in a slot of its own, then the progress counters of
        // every strip row at the smallest strip height
        g.persist_off = o;
        size_t nctr = 0;
        for (int m : g.members) {
            c->lats[m].prog_off = (int)nctr;
            nctr += (size_t)ceil_div(c->lats[m].lat.ny, ROWS_MIN);
        }
        g.persist_bytes = 256 + nctr * sizeof(unsigned);
        o = align256(o + g.persist_bytes);
        g.pg_off = o;
        o = align256(o + (g.members.size() + 1) * sizeof(int));
    }
    c->spec_off = o;
    o = align256(o + nl * init_spec_bytes());
    for (auto &L : c->lats) {
        const int nsx_max = ceil_div(L.lat.nx, 32);
        const int nsy_max = ceil_div(L.lat.ny, ROWS_MIN);
        const long long nstrip_max = (long long)nsx_max * nsy_max;
        L.nchunk_max = std::min(NCHUNK_MAX,
                                std::max(1, ceil_div(std::max<long long>({L.lat.nx, L.lat.ny, nstrip_max}), CHUNK_COLS)));
        L.scal_off = o;
        o = align256(o + nstrip_max * 5 * sizeof(double));
        L.colp_off = o;
        o = align256(o + (size_t)nsy_max * L.lat.nx * sizeof(double));
        L.rowp_off = o;
        o = align256(o + (size_t)nsx_max * L.lat.ny * sizeof(double));
        L.finp_off = o;
        o = align256(o + (size_t)L.nchunk_max * 9 * sizeof(double));
        L.ring_off = o;
        o = align256(o + (size_t)std::max(c->ring_cap, 1) * 8 * sizeof(double));
        L.now_off = o;
        o = align256(o + 8 * sizeof(double));
    }
    c->scratch_bytes = o;
}

// The storage shifts of a lattice (rest, axis, diagonal; D2Q7: rest, moving),
// each exactly representable in its storage type.
Shift3 host_shift(const LatHost &L)
{
    Shift3 s;
    const int st = L.lat.storage == LBM_F16_SHIFTED ? ST_F16 : (L.lat.storage == LBM_BF16_SHIFTED ? ST_BF16 : ST_F32);
    s.c[0] = storage_shift(st, L.q == 7 ? wq7_d(0) : wq_d(0), L.rho0);
    s.c[1] = storage_shift(st, L.q == 7 ? wq7_d(1) : wq_d(1), L.rho0);
    s.c[2] = storage_shift(st, L.q == 7 ? wq7_d(1) : wq_d(5), L.rho0);
    return s;
}

LatDesc make_desc(const lbm_ctx *c, const LatHost &L, int block_begin, const GroupHost &g)
{
    LatDesc d;
    std::memset(&d, 0, sizeof(d));
    char *sb = c->state + L.state_off;
    d.f[0] = sb;
    d.f[1] = sb + L.buf_bytes;
    d.scal = reinterpret_cast<double *>(c->scratch + L.scal_off);
    d.colp = reinterpret_cast<double *>(c->scratch + L.colp_off);
    d.rowp = reinterpret_cast<double *>(c->scratch + L.rowp_off);
    d.finp = reinterpret_cast<double *>(c->scratch + L.finp_off);
    d.ring = reinterpret_cast<double *>(c->scratch + L.ring_off);
    d.now = reinterpret_cast<double *>(c->scratch + L.now_off);
    d.counters = reinterpret_cast<unsigned *>(c->scratch + L.ctr_off);
    d.nx = L.lat.nx;
    d.ny = L.lat.ny;
    d.pitch = (int)L.pitch;
    d.id = L.lat.id;
    d.nsx = ceil_div(L.lat.nx, 32 * g.vec);
    d.nsy = ceil_div(L.lat.ny, g.rows);
    d.rows = g.rows;
    d.block_begin = block_begin;
    d.ring_cap = std::max(c->ring_cap, 1);
    d.q = L.q;
    d.prog_off = L.prog_off;
    const long long nstrip = (long long)d.nsx * d.nsy;
    d.nchunk = std::min(L.nchunk_max, std::max(1, ceil_div(std::max<long long>({L.lat.nx, L.lat.ny, nstrip}), CHUNK_COLS)));
    // 1/tau in FP32 such that 1 - 1/tau is exact too (the noisy update weighs f*
    // by 1 - 1/tau and f^SS by 1/tau): automatic for 1/tau in [1/2, 2]
    // (Sterbenz); below 1/2 the value is rounded to a multiple of 2^-24.
    double om = 1.0 / L.p.tau;
    if (om < 0.5) om = std::nearbyint(om * 16777216.0) / 16777216.0;
    d.omega = (float)om;
    d.sigma_q = (float)(2.0 * L.p.sigma);
    d.C = (float)L.p.C;
    d.rho_star = (float)L.p.rho_star;
    d.inv_rho_star = L.p.rho_star > 0 ? (float)(1.0 / L.p.rho_star) : 0.f;
    d.u_max = (float)L.p.u_max;
    d.u_max2 = (float)(L.p.u_max * L.p.u_max);
    d.A = (float)L.p.A;
    d.B = (float)L.p.B;
    d.rho0 = L.rho0;
    const Shift3 sh = host_shift(L);
    for (int k = 0; k < 3; ++k) d.sh[k] = sh.c[k];
    return d;
}

// Recompute strip geometry from the group shapes and upload all descriptor
// tables.  Syncs.
lbm_status upload_descs(lbm_ctx *c)
{
    std::vector<LatDesc> all(c->lats.size());
    c->max_chunk = 1;
    for (size_t gi = 0; gi < c->groups.size(); ++gi) {
        GroupHost &g = c->groups[gi];
        std::vector<LatDesc> gd;
        int blocks = 0;
        for (int m : g.members) {
            LatHost &L = c->lats[m];
            LatDesc d = make_desc(c, L, blocks, g);
            L.nsx = d.nsx;
            L.nsy = d.nsy;
            L.nchunk = d.nchunk;
            L.block_begin = blocks;
            // a staged kernel gives a block `warps` adjacent strips of one strip
            // row; the direct kernels take `warps` consecutive strips
            if (g.stages > 0)
                blocks += ceil_div(d.nsx, g.warps) * d.nsy;
            else
                blocks += ceil_div((long long)d.nsx * d.nsy, g.warps);
            gd.push_back(d);
            all[m] = d;
            c->max_chunk = std::max(c->max_chunk, d.nchunk);
        }
        g.blocks = blocks;
        CK(cudaMemcpyAsync(c->scratch + g.desc_off, gd.data(), gd.size() * sizeof(LatDesc),
                           cudaMemcpyHostToDevice, c->stream),
           "upload group descriptors");
        // lattice groups of the persistent launch: consecutive members whose
        // two population buffers each fit the L2 budget together (at least one
        // lattice per group); entry i is the group's first block of the step grid
        std::vector<int> pg;
        const size_t budget = c->persist_l2_mib > 0 ? (size_t)c->persist_l2_mib << 20 : SIZE_MAX;
        size_t bytes = 0;
        for (int m : g.members) {
            const LatHost &L = c->lats[m];
            if (pg.empty() || bytes + 2 * L.buf_bytes > budget) {
                pg.push_back(L.block_begin);
                bytes = 0;
            }
            bytes += 2 * L.buf_bytes;
        }
        g.npg = (int)pg.size();
        pg.push_back(blocks);
        CK(cudaMemcpyAsync(c->scratch + g.pg_off, pg.data(), pg.size() * sizeof(int), cudaMemcpyHostToDevice,
                           c->stream),
           "upload lattice groups");
    }
    CK(cudaMemcpyAsync(c->scratch + c->all_desc_off, all.data(), all.size() * sizeof(LatDesc),
                       cudaMemcpyHostToDevice, c->stream),
       "upload descriptors");
    CK(cudaStreamSynchronize(c->stream), "synchronise after descriptor upload");
    return LBM_OK;
}

const LatDesc *all_desc(const lbm_ctx *c)
{
    return reinterpret_cast<const LatDesc *>(c->scratch + c->all_desc_off);
}
uint32_t *t_dev(const lbm_ctx *c) { return reinterpret_cast<uint32_t *>(c->scratch); }
unsigned *err_dev(const lbm_ctx *c) { return reinterpret_cast<unsigned *>(c->scratch + 4); }

StepArgs step_args(const lbm_ctx *c, const GroupHost &g, int src, uint32_t k)
{
    StepArgs a;
    a.desc = reinterpret_cast<const LatDesc *>(c->scratch + g.desc_off);
    a.nlat = (int)g.members.size();
    a.src = src;
    a.t_ptr = t_dev(c);
    a.k = k;
    a.key0 = (uint32_t)c->seed;
    a.key1 = (uint32_t)(c->seed >> 32);
    a.stages = g.stages;
    a.err = err_dev(c);
    for (int r = 0; r < 10; ++r) {  // Philox round keys (Weyl increments, Salmon et al. 2011)
        a.rk[2 * r] = a.key0 + (uint32_t)r * 0x9E3779B9u;
        a.rk[2 * r + 1] = a.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    return a;
}

// Noise form of a group's launches: compile-time when the group is uniform in
// sigma (0: none, 1: all), else decided per lattice (2).
int group_noise(const lbm_ctx *c, const GroupHost &g)
{
    int with = 0;
    for (int m : g.members) with += (float)(2.0 * c->lats[m].p.sigma) > 0.f ? 1 : 0;  // as the kernel sees sigma_q
    return with == 0 ? 0 : (with == (int)g.members.size() ? 1 : 2);
}

cudaError_t launch_group_step(const lbm_ctx *c, const GroupHost &g, int src, uint32_t k, bool sample,
                              cudaStream_t stream)
{
    const StepArgs a = step_args(c, g, src, k);
    const int noise = group_noise(c, g);
    const int kind = g.stages > 0 ? 1 : 0;
    if (g.q == 7) {
        if (g.storage == LBM_F32)
            return launch_step_q7_f32(g.model, kind, g.vec, sample, noise, a, g.blocks, g.warps, stream);
        if (g.storage == LBM_F16_SHIFTED)
            return launch_step_q7_f16(g.model, kind, g.vec, sample, noise, a, g.blocks, g.warps, stream);
        return launch_step_q7_bf16(g.model, kind, g.vec, sample, noise, a, g.blocks, g.warps, stream);
    }
    if (g.storage == LBM_F32)
        return launch_step_f32(g.model, kind, g.vec, sample, noise, a, g.blocks, g.warps, stream);
    if (g.storage == LBM_F16_SHIFTED)
        return launch_step_f16(g.model, kind, g.vec, sample, noise, a, g.blocks, g.warps, stream);
    return launch_step_bf16(g.model, kind, g.vec, sample, noise, a, g.blocks, g.warps, stream);
}

// Groups the persistent launch can take: those on a direct kernel (D2Q9 or D2Q7).
bool persist_eligible(const GroupHost &g) { return g.stages == 0; }
// Whether a group runs its plain steps as persistent launches: always in mode
// 1, where the tuner chose to in mode 2.
bool persistent_ok(const lbm_ctx *c, const GroupHost &g)
{
    return persist_eligible(g) && (c->persist_mode == 1 || (c->persist_mode == 2 && g.persist));
}

// Most steps one persistent launch of the group may run (its items stay below 2^31).
int64_t persist_steps_max(const GroupHost &g)
{
    return std::max<int64_t>(1, std::min<int64_t>(PERSIST_STEPS_MAX, ((int64_t(1) << 31) - 1) / std::max(1, g.blocks)));
}

// m steps k .. k+m-1 of group g in one persistent launch: clear its counters,
// then launch.
cudaError_t launch_group_persistent(const lbm_ctx *c, const GroupHost &g, int src, uint32_t k, int64_t m,
                                    cudaStream_t stream, bool retime = false)
{
    const StepArgs a = step_args(c, g, src, k);
    PersistArgs p;
    p.work = reinterpret_cast<unsigned *>(c->scratch + g.persist_off);
    p.prog = p.work + 256 / sizeof(unsigned);
    p.pg = reinterpret_cast<const int *>(c->scratch + g.pg_off);
    p.npg = g.npg;
    p.nsteps = (int)m;
    p.retime = retime ? 1 : 0;
    cudaError_t e = cudaMemsetAsync(c->scratch + g.persist_off, 0, g.persist_bytes, stream);
    if (e != cudaSuccess) return e;
    const int noise = group_noise(c, g);
    if (g.q == 7) {
        if (g.storage == LBM_F32)
            return launch_persistent_q7_f32(g.model, g.vec, noise, a, p, g.blocks, g.warps, stream);
        if (g.storage == LBM_F16_SHIFTED)
            return launch_persistent_q7_f16(g.model, g.vec, noise, a, p, g.blocks, g.warps, stream);
        return launch_persistent_q7_bf16(g.model, g.vec, noise, a, p, g.blocks, g.warps, stream);
    }
    if (g.storage == LBM_F32) return launch_persistent_f32(g.model, g.vec, noise, a, p, g.blocks, g.warps, stream);
    if (g.storage == LBM_F16_SHIFTED)
        return launch_persistent_f16(g.model, g.vec, noise, a, p, g.blocks, g.warps, stream);
    return launch_persistent_bf16(g.model, g.vec, noise, a, p, g.blocks, g.warps, stream);
}

// The tuner's measure of a group: `steps` recomputations of the current step
// into the spare buffer (the state is left as it was), as one persistent launch
// in its timing form or as that many per-step launches.
cudaError_t launch_group_timed(const lbm_ctx *c, const GroupHost &g, int steps, cudaStream_t stream)
{
    if (persistent_ok(c, g)) return launch_group_persistent(c, g, c->parity, 0, steps, stream, true);
    for (int q = 0; q < steps; ++q) {
        const cudaError_t e = launch_group_step(c, g, c->parity, 0, false, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_group_observe(const lbm_ctx *c, const GroupHost &g, int src)
{
    StepArgs a;
    a.desc = reinterpret_cast<const LatDesc *>(c->scratch + g.desc_off);
    a.nlat = (int)g.members.size();
    a.src = src;
    a.t_ptr = t_dev(c);
    a.k = 0;
    a.key0 = a.key1 = 0;
    a.stages = g.stages;  // the strip-to-block mapping follows the group's step kernel
    a.err = err_dev(c);
    for (int r = 0; r < 20; ++r) a.rk[r] = 0;
    if (g.q == 7) {
        if (g.storage == LBM_F32) return launch_observe_q7_f32(g.vec, a, g.blocks, g.warps, c->stream);
        if (g.storage == LBM_F16_SHIFTED) return launch_observe_q7_f16(g.vec, a, g.blocks, g.warps, c->stream);
        return launch_observe_q7_bf16(g.vec, a, g.blocks, g.warps, c->stream);
    }
    if (g.storage == LBM_F32) return launch_observe_f32(g.vec, a, g.blocks, g.warps, c->stream);
    if (g.storage == LBM_F16_SHIFTED) return launch_observe_f16(g.vec, a, g.blocks, g.warps, c->stream);
    return launch_observe_bf16(g.vec, a, g.blocks, g.warps, c->stream);
}

// Kernel timing: an event pair around a launch when profiling is on.
cudaError_t prof_begin(lbm_ctx *c, bool is_step, int64_t steps = 1)
{
    if (!c->profiling) return cudaSuccess;
    while (c->ev_pool.size() < c->ev_used + 2) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        c->ev_pool.push_back(e);
    }
    c->ev_marks.push_back({(int)c->ev_used, is_step, steps});
    cudaError_t err = cudaEventRecord(c->ev_pool[c->ev_used], c->stream);
    c->ev_used += 2;
    return err;
}

cudaError_t prof_end(lbm_ctx *c)
{
    if (!c->profiling) return cudaSuccess;
    return cudaEventRecord(c->ev_pool[c->ev_marks.back().ev + 1], c->stream);
}

// Enqueue n steps starting at host time t0 from buffer parity p0.
// Streams and events for running the launch groups side by side (created
// once, outside any capture; destroyed with the context).
lbm_status ensure_aux(lbm_ctx *c)
{
    const size_t need = c->groups.size() - 1;
    if (c->aux_ev.empty()) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "create event");
        c->aux_ev.push_back(e);
    }
    while (c->aux.size() < need) {
        cudaStream_t s;
        CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "create stream");
        c->aux.push_back(s);
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "create event");
        c->aux_ev.push_back(e);
    }
    return LBM_OK;
}

// The groups hold disjoint lattices, so their step launches are independent:
// with several groups (and no per-launch timing) group i > 0 runs on aux[i-1],
// forked from the bound stream, and the branches join before each finaliser
// (which reads every lattice's partials) and at the end.  In a captured graph
// these are parallel branches, so one group's launch fills the other's tail.
cudaError_t fork_groups(lbm_ctx *c)
{
    cudaError_t e = cudaEventRecord(c->aux_ev[0], c->stream);
    for (size_t i = 0; e == cudaSuccess && i + 1 < c->groups.size(); ++i)
        e = cudaStreamWaitEvent(c->aux[i], c->aux_ev[0], 0);
    return e;
}

cudaError_t join_groups(lbm_ctx *c)
{
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; e == cudaSuccess && i + 1 < c->groups.size(); ++i) {
        e = cudaEventRecord(c->aux_ev[1 + i], c->aux[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->aux_ev[1 + i], 0);
    }
    return e;
}

// Enqueue n steps starting at host time t0 from buffer parity p0.  The steps
// fall into runs without a sample step, each followed by its sample step (if
// it lies within the n).  Per run, every group steps on its own stream (see
// fork_groups): a group the persistent launch takes runs as few launches as its
// step limit allows, any other launches once per step.  Then the sample step
// of every group, the join, and the finaliser.
lbm_status enqueue_steps(lbm_ctx *c, int64_t n, int64_t t0, int p0, int64_t *launches)
{
    const bool par = c->groups.size() > 1 && !c->profiling && c->aux.size() + 1 >= c->groups.size();
    bool forked = false;
    auto fork = [&]() -> cudaError_t {
        const cudaError_t e = fork_groups(c);
        forked = e == cudaSuccess;
        return e;
    };
    auto join = [&]() -> cudaError_t {
        forked = false;
        return join_groups(c);
    };
    auto stream_of = [&](size_t gi) { return par && gi > 0 ? c->aux[gi - 1] : c->stream; };
    int64_t k = 0;
    while (k < n) {
        // steps k .. e-1 have no sample step; step e is one (if e < n)
        int64_t e = n;
        if (c->sample_every > 0) {
            const int64_t r = (t0 + k + 1) % c->sample_every;
            e = std::min(n, k + (r == 0 ? 0 : c->sample_every - r));
        }
        if (par && !forked) CK(fork(), "fork launch groups");
        for (size_t gi = 0; gi < c->groups.size(); ++gi) {
            const GroupHost &g = c->groups[gi];
            const int64_t mmax = persistent_ok(c, g) ? persist_steps_max(g) : 1;
            for (int64_t kk = k; kk < e;) {
                const int64_t m = std::min(e - kk, mmax);
                CK(prof_begin(c, true, m), "record event");
                if (m >= 2)
                    CK(launch_group_persistent(c, g, (int)((p0 + kk) & 1), (uint32_t)kk, m, stream_of(gi)),
                       "launch persistent step kernel");
                else
                    CK(launch_group_step(c, g, (int)((p0 + kk) & 1), (uint32_t)kk, false, stream_of(gi)),
                       "launch step kernel");
                CK(prof_end(c), "record event");
                ++*launches;
                kk += m;
            }
        }
        if (e < n) {
            for (size_t gi = 0; gi < c->groups.size(); ++gi) {
                CK(prof_begin(c, true), "record event");
                CK(launch_group_step(c, c->groups[gi], (int)((p0 + e) & 1), (uint32_t)e, true, stream_of(gi)),
                   "launch step kernel");
                CK(prof_end(c), "record event");
                ++*launches;
            }
            if (par) CK(join(), "join launch groups");
            CK(prof_begin(c, false), "record event");
            CK(launch_finalize(all_desc(c), (int)c->lats.size(), c->max_chunk, t_dev(c), (uint32_t)e, 1,
                               err_dev(c), c->stream),
               "launch finaliser");
            CK(prof_end(c), "record event");
            ++*launches;
        }
        k = e + 1;
    }
    if (forked) CK(join(), "join launch groups");
    CK(prof_begin(c, false), "record event");
    CK(launch_advance_time(t_dev(c), (uint32_t)n, c->stream), "launch time advance");
    CK(prof_end(c), "record event");
    ++*launches;
    return LBM_OK;
}

void drop_graphs(lbm_ctx *c)
{
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second.first);
    c->graphs.clear();
}

lbm_status read_error_flag(lbm_ctx *c)
{
    unsigned flag = 0;
    CK(cudaMemcpyAsync(&flag, err_dev(c), sizeof(flag), cudaMemcpyDeviceToHost, c->stream), "read error flag");
    CK(cudaStreamSynchronize(c->stream), "synchronise");
    if (flag) {
        const unsigned zero = 0;
        CK(cudaMemcpyAsync(err_dev(c), &zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream), "clear error flag");
        CK(cudaStreamSynchronize(c->stream), "synchronise");
        if (flag & DEVERR_TIMEOUT) return fail(c, LBM_ERR_TIMEOUT, "a device-side wait timed out");
        return fail(c, LBM_ERR_NUMERIC, "non-finite observable sums");
    }
    return LBM_OK;
}

lbm_status require_ready(lbm_ctx *c, bool need_init)
{
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!c->bound) return fail(c, LBM_ERR_UNBOUND, "buffers are not bound (lbm_bind)");
    if (need_init && !c->initialized) return fail(c, LBM_ERR_UNBOUND, "state is not initialised (lbm_init)");
    return LBM_OK;
}

struct Shape {
    int vec, rows, warps, stages;
};

// A pair of timing events, destroyed on every way out of the tuner.
struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t create()
    {
        cudaError_t e = cudaEventCreate(&e0);
        return e == cudaSuccess ? cudaEventCreate(&e1) : e;
    }
    ~EventPair()
    {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Times the launch-shape candidates of one group on its own and keeps the
// fastest; *alts receives the alternatives for the joint check of a batch's
// groups: the fastest candidate of the other kernel kind (direct or staged),
// if any, and, where the fastest was a persistent launch, the fastest per-step
// form.  With persistent launches on (mode 1) direct candidates are timed as
// persistent launches; in mode 2 both ways, and the faster way is kept with
// the shape.
struct Alt {
    Shape shape;
    bool persist;
};

lbm_status tune_group(lbm_ctx *c, GroupHost &g, std::vector<Alt> *alts)
{
    std::vector<Shape> cands;
    long long max_ny = 1, group_sites = 0;
    for (int m : g.members) {
        max_ny = std::max<long long>(max_ny, c->lats[m].lat.ny);
        group_sites += (long long)c->lats[m].lat.nx * c->lats[m].lat.ny;
    }
    const int all_v[] = {1, 2, 4, 8};
    const bool staged = staged_ok(c, g);
    const bool direct = direct_ok(c, g);
    const int base_stages = g.model == LBM_MIPS ? 4 : 3;
    for (int v : all_v) {
        if (!allowed_vec(g.storage, v)) continue;
        bool ok = true;
        for (int m : g.members) ok = ok && (c->lats[m].lat.nx % v == 0);
        if (!ok) continue;
        for (int r : {8, 16, 32, 64, 128}) {
            if (r > 16 && r > 2 * max_ny) continue;
            if (direct)
                for (int w : {4, 8}) cands.push_back({v, r, w, 0});
            if (staged && v >= 2) {
                // MIPS also tries the least its ring needs (less shared memory, more
                // warps); with the converted row a ring of 2 fetches as far ahead
                // as one of 3 without it
                const bool mips = g.model == LBM_MIPS;
                const int sts[3] = {conv_rows(g) ? 3 : base_stages, conv_rows(g) ? 4 : base_stages + 2,
                                    min_stages(g)};
                for (int w : {1, 2, 4, 8})
                    for (int k = 0; k < (mips ? 3 : 2); ++k)
                        if (staged_smem_bytes(g.q, (int)elem_bytes(g.storage), v, w, sts[k],
                                              conv_rows(g)) <= STAGED_SMEM_MAX)
                            cands.push_back({v, r, w, sts[k]});
            }
        }
    }
    EventPair ev;
    CK(ev.create(), "create event");
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    float best = 1e30f, best_kind[2] = {1e30f, 1e30f}, best_step = 1e30f;
    Shape bs{g.vec, g.rows, g.warps, g.stages}, bk[2] = {bs, bs}, bstep = bs;
    bool bp = g.persist, bkp[2] = {bp, bp};
    for (const Shape &sh : cands) {
        g.vec = sh.vec;
        g.rows = sh.rows;
        g.warps = sh.warps;
        g.stages = sh.stages;
        lbm_status st = upload_descs(c);
        if (st != LBM_OK) return st;
        // launch forms to time: as lbm_step would launch it (modes 0, 1), or
        // per step and persistent (mode 2, direct shapes, enough sites)
        for (int form = 0; form < 2; ++form) {
            if (form == 1 && !(c->persist_mode == 2 && persist_eligible(g) && group_sites >= PERSIST_AUTO_MIN_SITES))
                break;
            g.persist = form == 1;
            cudaError_t e = launch_group_timed(c, g, 1, c->stream);
            if (e != cudaSuccess) {  // a shape this device cannot launch (e.g. shared memory): skip it
                cudaGetLastError();
                continue;
            }
            int steps = persistent_ok(c, g) ? TUNE_STEPS_PERSIST : TUNE_STEPS;
            float ms = 0.f;
            while (true) {
                CK(cudaEventRecord(e0, c->stream), "record event");
                CK(launch_group_timed(c, g, steps, c->stream), "tuning launch");
                CK(cudaEventRecord(e1, c->stream), "record event");
                CK(cudaEventSynchronize(e1), "synchronise event");
                CK(cudaEventElapsedTime(&ms, e0, e1), "event time");
                if (ms >= TUNE_MIN_MS || steps >= TUNE_STEPS_MAX) break;
                steps = std::min(TUNE_STEPS_MAX, (int)std::ceil(steps * TUNE_MIN_MS / std::max(ms, 1e-3f)) + 1);
            }
            ms *= (float)TUNE_STEPS / (float)steps;  // per TUNE_STEPS steps
            if (ms < best) {
                best = ms;
                bs = sh;
                bp = g.persist;
            }
            const int kind = sh.stages > 0 ? 1 : 0;
            if (ms < best_kind[kind]) {
                best_kind[kind] = ms;
                bk[kind] = sh;
                bkp[kind] = g.persist;
            }
            if (!persistent_ok(c, g) && ms < best_step) {
                best_step = ms;
                bstep = sh;
            }
        }
    }
    const int other = bs.stages > 0 ? 0 : 1;
    alts->clear();
    if (best_kind[other] < 1e29f) alts->push_back({bk[other], bkp[other]});
    // mode 2, a persistent choice: its best per-step direct form too (beside
    // other groups, a persistent launch holds the SMs its grid fills; the best
    // staged form is the alternative above)
    if (bp && best_step < 1e29f && bstep.stages == 0) alts->push_back({bstep, false});
    g.vec = bs.vec;
    g.rows = bs.rows;
    g.warps = bs.warps;
    g.stages = bs.stages;
    g.persist = bp;
    lbm_status st = upload_descs(c);
    if (st != LBM_OK) return st;
    return read_error_flag(c);
}

void set_shape(GroupHost &g, const Shape &sh)
{
    g.vec = sh.vec;
    g.rows = sh.rows;
    g.warps = sh.warps;
    g.stages = sh.stages;
}

// TUNE_STEPS_PERSIST steps of every group as lbm_step runs a batch (forked,
// side by side, joined), after a warm-up: their time in ms (timed over more
// steps when that is under TUNE_MIN_MS, and scaled back).  Writes only the
// spare buffers.
lbm_status time_joint_step(lbm_ctx *c, float *ms)
{
    lbm_status st = upload_descs(c);
    if (st != LBM_OK) return st;
    EventPair ev;
    CK(ev.create(), "create event");
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    int steps = TUNE_STEPS_PERSIST;
    while (true) {
        for (int rep = 0; rep < 2; ++rep) {
            if (rep == 1) CK(cudaEventRecord(e0, c->stream), "record event");  // the first is a warm-up
            CK(fork_groups(c), "fork launch groups");
            for (size_t gi = 0; gi < c->groups.size(); ++gi)
                CK(launch_group_timed(c, c->groups[gi], steps, gi > 0 ? c->aux[gi - 1] : c->stream), "tuning launch");
            CK(join_groups(c), "join launch groups");
        }
        CK(cudaEventRecord(e1, c->stream), "record event");
        CK(cudaEventSynchronize(e1), "synchronise event");
        CK(cudaEventElapsedTime(ms, e0, e1), "event time");
        if (*ms >= TUNE_MIN_MS || steps >= TUNE_STEPS_MAX) break;
        steps = std::min(TUNE_STEPS_MAX, (int)std::ceil(steps * TUNE_MIN_MS / std::max(*ms, 1e-3f)) + 1);
    }
    *ms *= (float)TUNE_STEPS_PERSIST / (float)steps;
    return LBM_OK;
}

// Each group's shape is chosen on its own, but a batch runs its groups side by
// side, where kernels of the two kinds can slow each other (measured on a
// 64-lattice ragged MIPS/CIL batch: a staged MIPS group beside a direct CIL
// group ran at 71 GLUPS, slower than the same launches one after the other,
// 73; both direct, about 79), and a persistent launch keeps the SMs its grid
// fills from the other groups' launches (the same batch with its CIL group
// persistent: 77 against 79 GLUPS).  So each group's alternatives (its best
// shape of the other kind; its best per-step form where it chose a persistent
// launch) are tried in turn with the whole batch running, and kept where the
// batch step is faster.
lbm_status do_tune(lbm_ctx *c)
{
    const size_t ng = c->groups.size();
    std::vector<std::vector<Alt>> alts(ng);
    for (size_t gi = 0; gi < ng; ++gi) {
        lbm_status st = tune_group(c, c->groups[gi], &alts[gi]);
        if (st != LBM_OK) return st;
    }
    if (ng > 1) {
        lbm_status st = ensure_aux(c);
        if (st != LBM_OK) return st;
        float best = 0.f;
        st = time_joint_step(c, &best);
        if (st != LBM_OK) return st;
        for (size_t gi = 0; gi < ng; ++gi) {
            GroupHost &g = c->groups[gi];
            for (const Alt &al : alts[gi]) {
                const Shape keep{g.vec, g.rows, g.warps, g.stages};
                const bool keep_persist = g.persist;
                set_shape(g, al.shape);
                g.persist = al.persist;
                float ms = 0.f;
                st = time_joint_step(c, &ms);
                if (st != LBM_OK) return st;
                if (ms < best) {
                    best = ms;
                } else {
                    set_shape(g, keep);
                    g.persist = keep_persist;
                }
            }
        }
        st = upload_descs(c);
        if (st != LBM_OK) return st;
        st = read_error_flag(c);
        if (st != LBM_OK) return st;
    }
    drop_graphs(c);
    c->tuned = true;
    return LBM_OK;
}

lbm_status create_common(int32_t n, const lbm_lattice *lats, const lbm_model *models, const lbm_params *ps,
                         lbm_ctx **out)
{
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || !lats || !models || !ps) return LBM_ERR_INVALID_ARG;
    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_INVALID_ARG;
    for (int32_t k = 0; k < n; ++k) {
        const std::string why = validate(lats[k], (int)models[k], ps[k]);
        if (!why.empty()) {
            delete c;
            return LBM_ERR_INVALID_ARG;
        }
        // beyond the direct kernel's 32-bit element index only the staged kernel runs
        const int q = lats[k].velocity_set == LBM_D2Q7 ? 7 : 9;
        if (!index32_fits(lats[k], q) && !staged_fits(lats[k])) {
            delete c;
            return LBM_ERR_UNSUPPORTED;
        }
        LatHost L;
        L.lat = lats[k];
        L.model = (int)models[k];
        L.p = ps[k];
        L.rho0 = ps[k].rho0 > 0 ? (float)ps[k].rho0 : 1.f;
        L.q = lats[k].velocity_set == LBM_D2Q7 ? 7 : 9;
        c->lats.push_back(L);
    }
    // launch groups: one per (model, storage, velocity set)
    for (int32_t k = 0; k < n; ++k) {
        LatHost &L = c->lats[k];
        int gi = -1;
        for (size_t q = 0; q < c->groups.size(); ++q)
            if (c->groups[q].model == L.model && c->groups[q].storage == L.lat.storage && c->groups[q].q == L.q)
                gi = (int)q;
        if (gi < 0) {
            GroupHost g;
            g.model = L.model;
            g.storage = L.lat.storage;
            g.q = L.q;
            c->groups.push_back(g);
            gi = (int)c->groups.size() - 1;
        }
        c->groups[gi].members.push_back(k);
        L.group = gi;
    }
    for (auto &g : c->groups) {
        g.vec = default_vec(c, g);
        g.rows = 32;
        g.warps = 4;
        if (!direct_ok(c, g)) g.stages = g.model == LBM_MIPS ? 4 : 3;
    }
    layout(c);
    *out = c;
    return LBM_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

lbm_status lbm_create(const lbm_lattice *lattice, lbm_model model, const lbm_params *params, lbm_ctx **out)
{
    return create_common(1, lattice, &model, params, out);
}

lbm_status lbm_create_batch(int32_t n, const lbm_lattice *lattices, const lbm_model *models,
                            const lbm_params *params, lbm_ctx **out)
{
    return create_common(n, lattices, models, params, out);
}

lbm_status lbm_set_sampling(lbm_ctx *c, int32_t sample_every, int32_t ring_capacity)
{
    if (!c) return LBM_ERR_INVALID_ARG;
    if (c->bound) return fail(c, LBM_ERR_INVALID_ARG, "set sampling before lbm_bind");
    if (sample_every < 0 || ring_capacity < 0 || ring_capacity > (1 << 24))
        return fail(c, LBM_ERR_INVALID_ARG, "sample_every >= 0 and 0 <= ring_capacity <= 2^24");
    if (sample_every > 0 && ring_capacity < 1)
        return fail(c, LBM_ERR_INVALID_ARG, "sampling needs ring_capacity >= 1");
    c->sample_every = sample_every;
    c->ring_cap = ring_capacity;
    layout(c);
    return LBM_OK;
}

lbm_status lbm_buffer_bytes(const lbm_ctx *c, size_t *state_bytes, size_t *scratch_bytes)
{
    if (!c || !state_bytes || !scratch_bytes) return LBM_ERR_INVALID_ARG;
    *state_bytes = c->state_bytes;
    *scratch_bytes = c->scratch_bytes;
    return LBM_OK;
}

lbm_status lbm_bind(lbm_ctx *c, void *state_dev, void *scratch_dev, void *cuda_stream)
{
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!state_dev || !scratch_dev) return fail(c, LBM_ERR_INVALID_ARG, "null buffer");
    if (((uintptr_t)state_dev & 255) || ((uintptr_t)scratch_dev & 255))
        return fail(c, LBM_ERR_INVALID_ARG, "buffers must be 256-byte aligned");
    drop_graphs(c);
    c->state = static_cast<char *>(state_dev);
    c->scratch = static_cast<char *>(scratch_dev);
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->bound = true;
    c->initialized = false;
    CK(cudaMemsetAsync(c->scratch, 0, c->all_desc_off, c->stream), "clear control words");
    return upload_descs(c);
}

lbm_status lbm_init(lbm_ctx *c, uint64_t seed, const lbm_init_spec *specs)
{
    lbm_status st = require_ready(c, false);
    if (st != LBM_OK) return st;
    if (!specs) return fail(c, LBM_ERR_INVALID_ARG, "null init spec");
    const size_t nl = c->lats.size();
    std::vector<char> packed(nl * init_spec_bytes());
    for (size_t k = 0; k < nl; ++k) {
        const lbm_init_spec &s = specs[k];
        const double v[] = {s.rho_mean, s.rho_amp, s.u_amp, s.ux0, s.uy0};
        for (double x : v)
            if (!std::isfinite(x)) return fail(c, LBM_ERR_INVALID_ARG, "init spec must be finite");
        if (s.u_kind < 0 || s.u_kind > 2) return fail(c, LBM_ERR_INVALID_ARG, "u_kind must be 0, 1 or 2");
        if (!(s.rho_mean > 0)) return fail(c, LBM_ERR_INVALID_ARG, "rho_mean must be > 0");
        LatHost &L = c->lats[k];
        L.rho0 = L.p.rho0 > 0 ? (float)L.p.rho0 : (float)s.rho_mean;
        pack_init_spec(packed.data() + k * init_spec_bytes(), s.rho_mean, s.rho_amp, s.u_kind, s.u_amp, s.ux0,
                       s.uy0, L.p.A, L.p.B);
    }
    st = upload_descs(c);
    if (st != LBM_OK) return st;
    CK(cudaMemcpyAsync(c->scratch + c->spec_off, packed.data(), packed.size(), cudaMemcpyHostToDevice, c->stream),
       "upload init specs");
    c->seed = seed;
    for (size_t k = 0; k < nl; ++k) {
        const LatHost &L = c->lats[k];
        CK(launch_init(L.lat.storage, all_desc(c) + k, c->scratch + c->spec_off + k * init_spec_bytes(), 1,
                       (long long)L.lat.nx * L.lat.ny, 0, seed, c->stream),
           "launch init kernel");
        c->lats[k].consumed = 0;
    }
    CK(cudaMemsetAsync(c->scratch, 0, c->all_desc_off, c->stream), "clear control words");
    CK(cudaStreamSynchronize(c->stream), "synchronise after init");
    c->t = 0;
    c->parity = 0;
    c->initialized = true;
    drop_graphs(c);
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *c, int64_t n)
{
    lbm_status st = require_ready(c, true);
    if (st != LBM_OK) return st;
    if (n < 0) return fail(c, LBM_ERR_INVALID_ARG, "n must be >= 0");
    if (c->t + n >= (int64_t(1) << 32)) return fail(c, LBM_ERR_INVALID_ARG, "t + n must stay below 2^32");
    c->last_launches = 0;
    if (n == 0) return LBM_OK;
    if (!c->tuned && c->tune_mode == 0) {
        st = do_tune(c);
        if (st != LBM_OK) return st;
    }
    const bool graphs = c->use_graphs && c->stream != nullptr && !c->profiling;
    if (c->groups.size() > 1 && !c->profiling) {
        st = ensure_aux(c);
        if (st != LBM_OK) return st;
    }
    int64_t done = 0;
    while (done < n) {
        int64_t chunk = n - done;
        if (graphs) {
            int64_t cap = GRAPH_CHUNK_MAX;
            if (c->sample_every > 0 && c->sample_every <= GRAPH_CHUNK_MAX)
                cap = (GRAPH_CHUNK_MAX / c->sample_every) * c->sample_every;
            chunk = std::min(chunk, cap);
            const GraphKey key{chunk, c->sample_every > 0 ? c->t % c->sample_every : 0, c->parity};
            auto it = c->graphs.find(key);
            if (it == c->graphs.end()) {
                CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
                int64_t captured = 0;
                st = enqueue_steps(c, chunk, c->t, c->parity, &captured);
                cudaGraph_t graph = nullptr;
                cudaError_t ec = cudaStreamEndCapture(c->stream, &graph);
                if (st != LBM_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    return st;
                }
                if (ec != cudaSuccess) return cuda_fail(c, ec, "end capture");
                cudaGraphExec_t exec = nullptr;
                ec = cudaGraphInstantiate(&exec, graph, 0);
                cudaGraphDestroy(graph);
                if (ec != cudaSuccess) return cuda_fail(c, ec, "instantiate graph");
                it = c->graphs.emplace(key, std::make_pair(exec, captured)).first;
            }
            CK(cudaGraphLaunch(it->second.first, c->stream), "launch graph");
            c->last_launches += it->second.second;
        } else {
            st = enqueue_steps(c, chunk, c->t, c->parity, &c->last_launches);
            if (st != LBM_OK) return st;
        }
        c->t += chunk;
        c->parity = (int)((c->parity + chunk) & 1);
        done += chunk;
    }
    return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx *c, int32_t lattice, float *rho, float *ux, float *uy)
{
    lbm_status st = require_ready(c, true);
    if (st != LBM_OK) return st;
    if (lattice < 0 || lattice >= (int32_t)c->lats.size()) return fail(c, LBM_ERR_INVALID_ARG, "bad lattice index");
    if (!rho || !ux || !uy) return fail(c, LBM_ERR_INVALID_ARG, "null output pointer");
    const LatHost &L = c->lats[lattice];
    CK(launch_moments(L.lat.storage, all_desc(c), lattice, (long long)L.lat.nx * L.lat.ny, c->parity, rho, ux,
                      uy, c->stream),
       "launch moments kernel");
    return LBM_OK;
}

lbm_status lbm_observables(lbm_ctx *c, int32_t lattice, lbm_obs *out)
{
    lbm_status st = require_ready(c, true);
    if (st != LBM_OK) return st;
    if (lattice < 0 || lattice >= (int32_t)c->lats.size() || !out)
        return fail(c, LBM_ERR_INVALID_ARG, "bad lattice index or null output");
    for (const GroupHost &g : c->groups) CK(launch_group_observe(c, g, c->parity), "launch observe kernel");
    CK(launch_finalize(all_desc(c), (int)c->lats.size(), c->max_chunk, t_dev(c), 0, 0, err_dev(c), c->stream),
       "launch finaliser");
    double rec[8];
    CK(cudaMemcpyAsync(rec, c->scratch + c->lats[lattice].now_off, sizeof(rec), cudaMemcpyDeviceToHost, c->stream),
       "read observables");
    CK(cudaStreamSynchronize(c->stream), "synchronise");
    long long tt;
    std::memcpy(&tt, &rec[0], sizeof(tt));
    out->t = c->t;
    out->mass = rec[1];
    out->phi = rec[2];
    out->drho_y = rec[3];
    out->drho_x = rec[4];
    out->var_rho = rec[5];
    out->zeta = rec[6];
    return read_error_flag(c);
}

lbm_status lbm_observable_series(lbm_ctx *c, int32_t lattice, lbm_obs *out, int32_t cap, int32_t *n_out)
{
    lbm_status st = require_ready(c, true);
    if (st != LBM_OK) return st;
    if (lattice < 0 || lattice >= (int32_t)c->lats.size() || !n_out || cap < 0 || (cap > 0 && !out))
        return fail(c, LBM_ERR_INVALID_ARG, "bad arguments");
    *n_out = 0;
    LatHost &L = c->lats[lattice];
    unsigned count = 0;
    CK(cudaMemcpyAsync(&count, c->scratch + L.ctr_off, sizeof(count), cudaMemcpyDeviceToHost, c->stream),
       "read sample count");
    CK(cudaStreamSynchronize(c->stream), "synchronise");
    const int64_t rc = std::max(c->ring_cap, 1);
    int64_t first = std::max<int64_t>(L.consumed, (int64_t)count - rc);
    const int64_t avail = (int64_t)count - first;
    const int64_t take = std::min<int64_t>(avail, cap);
    if (take > 0) {
        std::vector<double> ring((size_t)rc * 8);
        CK(cudaMemcpyAsync(ring.data(), c->scratch + L.ring_off, ring.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream),
           "read observable ring");
        CK(cudaStreamSynchronize(c->stream), "synchronise");
        for (int64_t q = 0; q < take; ++q) {
            const double *r = &ring[(size_t)((first + q) % rc) * 8];
            long long tt;
            std::memcpy(&tt, &r[0], sizeof(tt));
            out[q].t = tt;
            out[q].mass = r[1];
            out[q].phi = r[2];
            out[q].drho_y = r[3];
            out[q].drho_x = r[4];
            out[q].var_rho = r[5];
            out[q].zeta = r[6];
        }
    }
    L.consumed = first + take;
    *n_out = (int32_t)take;
    return read_error_flag(c);
}

lbm_status lbm_get_state(lbm_ctx *c, int32_t lattice, float *dst, int32_t dst_is_host)
{
    lbm_status st = require_ready(c, true);
    if (st != LBM_OK) return st;
    if (lattice < 0 || lattice >= (int32_t)c->lats.size() || !dst)
        return fail(c, LBM_ERR_INVALID_ARG, "bad lattice index or null output");
    const LatHost &L = c->lats[lattice];
    const char *src = c->state + L.state_off + (c->parity ? L.buf_bytes : 0);
    const size_t eb = elem_bytes(L.lat.storage);
    const long long cells = (long long)L.lat.nx * L.lat.ny;
    if (L.lat.storage == LBM_F32) {
        CK(cudaMemcpy2DAsync(dst, L.lat.nx * 4, src, L.pitch * 4, L.lat.nx * 4, (size_t)L.q * L.lat.ny,
                             dst_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream),
           "copy populations");
    } else if (!dst_is_host) {
        CK(launch_export(L.lat.storage, all_desc(c), lattice, cells, c->parity, dst, c->stream), "launch export");
    } else {
        std::vector<uint16_t> raw((size_t)L.q * cells);
        CK(cudaMemcpy2DAsync(raw.data(), L.lat.nx * eb, src, L.pitch * eb, L.lat.nx * eb, (size_t)L.q * L.lat.ny,
                             cudaMemcpyDeviceToHost, c->stream),
           "copy populations");
        CK(cudaStreamSynchronize(c->stream), "synchronise");
        for (int i = 0; i < L.q; ++i) {
            const float shift = host_shift(L).of(L.q, i);
            for (long long q = 0; q < cells; ++q) {
                const uint16_t bits = raw[(size_t)i * cells + q];
                float v;
                if (L.lat.storage == LBM_F16_SHIFTED) {
                    __half h;
                    std::memcpy(&h, &bits, 2);
                    v = __half2float(h);
                } else {
                    const uint32_t w = (uint32_t)bits << 16;
                    std::memcpy(&v, &w, 4);
                }
                dst[(size_t)i * cells + q] = v + shift;
            }
        }
    }
    CK(cudaStreamSynchronize(c->stream), "synchronise");
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_ctx *c, int32_t lattice, const float *src, int32_t src_is_host)
{
    lbm_status st = require_ready(c, false);
    if (st != LBM_OK) return st;
    if (lattice < 0 || lattice >= (int32_t)c->lats.size() || !src)
        return fail(c, LBM_ERR_INVALID_ARG, "bad lattice index or null input");
    if (!c->initialized) {  // state set directly: start the clock at 0
        CK(cudaMemsetAsync(c->scratch, 0, c->all_desc_off, c->stream), "clear control words");
        c->t = 0;
        c->parity = 0;
        c->initialized = true;
    }
    const LatHost &L = c->lats[lattice];
    char *dstp = c->state + L.state_off + (c->parity ? L.buf_bytes : 0);
    const size_t eb = elem_bytes(L.lat.storage);
    const long long cells = (long long)L.lat.nx * L.lat.ny;
    if (L.lat.storage == LBM_F32) {
        CK(cudaMemcpy2DAsync(dstp, L.pitch * 4, src, L.lat.nx * 4, L.lat.nx * 4, (size_t)L.q * L.lat.ny,
                             src_is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream),
           "copy populations");
    } else if (!src_is_host) {
        CK(launch_import(L.lat.storage, all_desc(c), lattice, cells, c->parity, src, c->stream), "launch import");
    } else {
        std::vector<uint16_t> raw((size_t)L.q * cells);
        for (int i = 0; i < L.q; ++i) {
            const float shift = host_shift(L).of(L.q, i);
            for (long long q = 0; q < cells; ++q) {
                const float v = src[(size_t)i * cells + q] - shift;
                uint16_t bits;
                if (L.lat.storage == LBM_F16_SHIFTED) {
                    const __half h = __float2half_rn(v);
                    std::memcpy(&bits, &h, 2);
                } else {
                    const __nv_bfloat16 b = __float2bfloat16_rn(v);
                    std::memcpy(&bits, &b, 2);
                }
                raw[(size_t)i * cells + q] = bits;
            }
        }
        CK(cudaMemcpy2DAsync(dstp, L.pitch * eb, raw.data(), L.lat.nx * eb, L.lat.nx * eb, (size_t)L.q * L.lat.ny,
                             cudaMemcpyHostToDevice, c->stream),
           "copy populations");
    }
    CK(cudaStreamSynchronize(c->stream), "synchronise");
    return LBM_OK;
}

lbm_status lbm_add_density(lbm_ctx *c, int32_t lattice, double delta_rho_bar)
{
    lbm_status st = require_ready(c, true);
    if (st != LBM_OK) return st;
    if (lattice < -1 || lattice >= (int32_t)c->lats.size()) return fail(c, LBM_ERR_INVALID_ARG, "bad lattice index");
    if (!std::isfinite(delta_rho_bar)) return fail(c, LBM_ERR_INVALID_ARG, "delta must be finite");
    for (int k = 0; k < (int)c->lats.size(); ++k) {
        if (lattice != -1 && k != lattice) continue;
        const LatHost &L = c->lats[k];
        CK(launch_add_density(L.lat.storage, all_desc(c), k, (long long)L.lat.nx * L.lat.ny, c->parity,
                              (float)(delta_rho_bar / (double)L.q), c->stream),
           "launch density step");
    }
    return LBM_OK;
}

lbm_status lbm_set_params(lbm_ctx *c, int32_t lattice, const lbm_params *params)
{
    if (!c || !params) return LBM_ERR_INVALID_ARG;
    if (lattice < -1 || lattice >= (int32_t)c->lats.size()) return fail(c, LBM_ERR_INVALID_ARG, "bad lattice index");
    for (int k = 0; k < (int)c->lats.size(); ++k) {
        if (lattice != -1 && k != lattice) continue;
        const std::string why = validate(c->lats[k].lat, c->lats[k].model, *params);
        if (!why.empty()) return fail(c, LBM_ERR_INVALID_ARG, why);
    }
    for (int k = 0; k < (int)c->lats.size(); ++k) {
        if (lattice != -1 && k != lattice) continue;
        const double keep_rho0 = c->lats[k].p.rho0;
        c->lats[k].p = *params;
        c->lats[k].p.rho0 = keep_rho0;
    }
    drop_graphs(c);
    if (c->bound) return upload_descs(c);
    return LBM_OK;
}

lbm_status lbm_get_time(const lbm_ctx *c, int64_t *t)
{
    if (!c || !t) return LBM_ERR_INVALID_ARG;
    *t = c->t;
    return LBM_OK;
}

static const char kMagic[8] = {'L', 'B', 'M', 'S', 'T', 'A', 'T', '2'};

lbm_status lbm_save(lbm_ctx *c, const char *path)
{
    lbm_status st = require_ready(c, true);
    if (st != LBM_OK) return st;
    if (!path) return fail(c, LBM_ERR_INVALID_ARG, "null path");
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(c, LBM_ERR_INVALID_ARG, std::string("cannot open ") + path);
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8;
    const int64_t hdr[3] = {(int64_t)c->lats.size(), c->t, (int64_t)c->seed};
    ok = ok && std::fwrite(hdr, sizeof(hdr), 1, f) == 1;
    for (size_t k = 0; ok && k < c->lats.size(); ++k) {
        const LatHost &L = c->lats[k];
        const int32_t meta[6] = {L.lat.nx, L.lat.ny, L.lat.storage, L.model, L.lat.id, L.lat.velocity_set};
        ok = ok && std::fwrite(meta, sizeof(meta), 1, f) == 1;
        ok = ok && std::fwrite(&L.rho0, sizeof(float), 1, f) == 1;
        const size_t eb = elem_bytes(L.lat.storage);
        std::vector<char> raw((size_t)L.q * L.lat.ny * L.lat.nx * eb);
        const char *src = c->state + L.state_off + (c->parity ? L.buf_bytes : 0);
        cudaError_t e = cudaMemcpy2DAsync(raw.data(), L.lat.nx * eb, src, L.pitch * eb, L.lat.nx * eb,
                                          (size_t)L.q * L.lat.ny, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            std::fclose(f);
            return cuda_fail(c, e, "read populations for save");
        }
        ok = ok && std::fwrite(raw.data(), 1, raw.size(), f) == raw.size();
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(c, LBM_ERR_INVALID_ARG, std::string("write failed: ") + path);
    return LBM_OK;
}

lbm_status lbm_load(lbm_ctx *c, const char *path)
{
    lbm_status st = require_ready(c, false);
    if (st != LBM_OK) return st;
    if (!path) return fail(c, LBM_ERR_INVALID_ARG, "null path");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(c, LBM_ERR_INVALID_ARG, std::string("cannot open ") + path);
    char magic[8];
    int64_t hdr[3];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0;
    ok = ok && std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == (int64_t)c->lats.size();
    ok = ok && hdr[1] >= 0 && hdr[1] < (int64_t(1) << 32);
    std::vector<std::vector<char>> raws;
    std::vector<float> rho0s;
    for (size_t k = 0; ok && k < c->lats.size(); ++k) {
        const LatHost &L = c->lats[k];
        int32_t meta[6];
        float r0 = 0.f;
        ok = ok && std::fread(meta, sizeof(meta), 1, f) == 1 && std::fread(&r0, sizeof(float), 1, f) == 1;
        ok = ok && meta[0] == L.lat.nx && meta[1] == L.lat.ny && meta[2] == L.lat.storage && meta[3] == L.model &&
             meta[4] == L.lat.id && meta[5] == L.lat.velocity_set;
        if (!ok) break;
        const size_t eb = elem_bytes(L.lat.storage);
        std::vector<char> raw((size_t)L.q * L.lat.ny * L.lat.nx * eb);
        ok = std::fread(raw.data(), 1, raw.size(), f) == raw.size();
        raws.push_back(std::move(raw));
        rho0s.push_back(r0);
    }
    std::fclose(f);
    if (!ok) return fail(c, LBM_ERR_INVALID_ARG, "state file does not match this context");
    for (size_t k = 0; k < c->lats.size(); ++k) c->lats[k].rho0 = rho0s[k];
    st = upload_descs(c);
    if (st != LBM_OK) return st;
    for (size_t k = 0; k < c->lats.size(); ++k) {
        const LatHost &L = c->lats[k];
        const size_t eb = elem_bytes(L.lat.storage);
        CK(cudaMemcpy2DAsync(c->state + L.state_off, L.pitch * eb, raws[k].data(), L.lat.nx * eb, L.lat.nx * eb,
                             (size_t)L.q * L.lat.ny, cudaMemcpyHostToDevice, c->stream),
           "upload populations");
        c->lats[k].consumed = 0;
    }
    CK(cudaMemsetAsync(c->scratch, 0, c->all_desc_off, c->stream), "clear control words");
    CK(launch_set_time(t_dev(c), (uint32_t)hdr[1], c->stream), "set time");
    CK(cudaStreamSynchronize(c->stream), "synchronise");
    c->t = hdr[1];
    c->seed = (uint64_t)hdr[2];
    c->parity = 0;
    c->initialized = true;
    drop_graphs(c);
    return LBM_OK;
}

lbm_status lbm_set_tuning(lbm_ctx *c, int32_t mode, int32_t vec, int32_t rows, int32_t warps, int32_t stages)
{
    if (!c) return LBM_ERR_INVALID_ARG;
    if (mode == 0) {
        c->tune_mode = 0;
        c->tuned = false;
        return LBM_OK;
    }
    if (mode != 1) return fail(c, LBM_ERR_INVALID_ARG, "mode must be 0 or 1");
    if (rows < ROWS_MIN || rows > 4096) return fail(c, LBM_ERR_INVALID_ARG, "rows must be in [8, 4096]");
    if (warps < 1 || warps > 8) return fail(c, LBM_ERR_INVALID_ARG, "warps must be in [1, 8]");
    if (stages != 0 && (stages < 2 || stages > 8))
        return fail(c, LBM_ERR_INVALID_ARG, "stages must be 0 (direct) or 2..8");
    if (stages != 0)
        for (auto &g : c->groups)
            if (stages < min_stages(g))
                return fail(c, LBM_ERR_INVALID_ARG, "MIPS needs at least 3 stages (2 with 16-bit storage)");
    if (stages != 0)
        for (auto &g : c->groups)
            if (!staged_ok(c, g)) return fail(c, LBM_ERR_INVALID_ARG, "staged kernel needs nx a multiple of 16 bytes");
    if (stages != 0)
        for (auto &g : c->groups)
            if (staged_smem_bytes(g.q, (int)elem_bytes(g.storage), vec, warps, stages,
                                  conv_rows(g)) > STAGED_SMEM_MAX)
                return fail(c, LBM_ERR_INVALID_ARG,
                            "staged shape needs more than the 227 KB of shared memory a block can have");
    if (stages == 0)
        for (auto &g : c->groups)
            if (!direct_ok(c, g))
                return fail(c, LBM_ERR_INVALID_ARG, "direct kernel needs q ny pitch <= 2^32 elements: use stages > 0");
    for (auto &g : c->groups)
        if (g.q == 7 && rows % 2) return fail(c, LBM_ERR_INVALID_ARG, "D2Q7 strips need an even number of rows");
    for (auto &g : c->groups) {
        if (!allowed_vec(g.storage, vec)) return fail(c, LBM_ERR_INVALID_ARG, "vec not available for this storage");
        for (int m : g.members)
            if (c->lats[m].lat.nx % vec) return fail(c, LBM_ERR_INVALID_ARG, "vec must divide nx");
    }
    for (auto &g : c->groups) {
        g.vec = vec;
        g.rows = rows;
        g.warps = warps;
        g.stages = stages;
    }
    c->tune_mode = 1;
    c->tuned = true;
    drop_graphs(c);
    if (c->bound) return upload_descs(c);
    return LBM_OK;
}

lbm_status lbm_tune(lbm_ctx *c)
{
    lbm_status st = require_ready(c, true);
    if (st != LBM_OK) return st;
    return do_tune(c);
}

lbm_status lbm_get_tuning(const lbm_ctx *c, int32_t lattice, int32_t *vec, int32_t *rows, int32_t *warps,
                          int32_t *stages)
{
    if (!c || !vec || !rows || !warps || !stages || lattice < 0 || lattice >= (int32_t)c->lats.size())
        return LBM_ERR_INVALID_ARG;
    const GroupHost &g = c->groups[c->lats[lattice].group];
    *vec = g.vec;
    *rows = g.rows;
    *warps = g.warps;
    *stages = g.stages;
    return LBM_OK;
}

lbm_status lbm_check_wait_timeout(lbm_ctx *c)
{
    lbm_status st = require_ready(c, false);
    if (st != LBM_OK) return st;
    CK(launch_wait_timeout(err_dev(c), c->stream), "launch wait check");
    return read_error_flag(c);
}

lbm_status lbm_set_graphs(lbm_ctx *c, int32_t enabled)
{
    if (!c) return LBM_ERR_INVALID_ARG;
    c->use_graphs = enabled != 0;
    if (!c->use_graphs) drop_graphs(c);
    return LBM_OK;
}

lbm_status lbm_set_persistent(lbm_ctx *c, int32_t mode, int32_t l2_group_mib)
{
    if (!c) return LBM_ERR_INVALID_ARG;
    if (mode < 0 || mode > 2) return fail(c, LBM_ERR_INVALID_ARG, "mode must be 0, 1 or 2");
    if (l2_group_mib < 0 || l2_group_mib > (1 << 20))
        return fail(c, LBM_ERR_INVALID_ARG, "l2_group_mib must be in [0, 2^20]");
    c->persist_mode = mode;
    c->persist_l2_mib = l2_group_mib;
    for (auto &g : c->groups) g.persist = false;
    if (mode == 2 && c->tune_mode == 0) c->tuned = false;  // the next lbm_step tunes, and chooses
    drop_graphs(c);
    if (c->bound) return upload_descs(c);
    return LBM_OK;
}

lbm_status lbm_get_persistent(const lbm_ctx *c, int32_t lattice, int32_t *persistent)
{
    if (!c || !persistent || lattice < 0 || lattice >= (int32_t)c->lats.size()) return LBM_ERR_INVALID_ARG;
    *persistent = persistent_ok(c, c->groups[c->lats[lattice].group]) ? 1 : 0;
    return LBM_OK;
}

lbm_status lbm_last_launch_count(const lbm_ctx *c, int64_t *count)
{
    if (!c || !count) return LBM_ERR_INVALID_ARG;
    *count = c->last_launches;
    return LBM_OK;
}

lbm_status lbm_set_profiling(lbm_ctx *c, int32_t enabled)
{
    if (!c) return LBM_ERR_INVALID_ARG;
    c->profiling = enabled != 0;
    c->ev_marks.clear();
    c->ev_used = 0;
    return LBM_OK;
}

lbm_status lbm_profile_read(lbm_ctx *c, double *step_ms, int64_t *step_launches, double *other_ms)
{
    if (!c || !step_ms || !step_launches || !other_ms) return LBM_ERR_INVALID_ARG;
    *step_ms = 0.0;
    *other_ms = 0.0;
    *step_launches = 0;
    if (!c->ev_marks.empty()) {
        CK(cudaEventSynchronize(c->ev_pool[c->ev_marks.back().ev + 1]), "synchronise event");
        for (const auto &m : c->ev_marks) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->ev_pool[m.ev], c->ev_pool[m.ev + 1]), "event time");
            if (m.step) {
                *step_ms += ms;
                *step_launches += m.steps;
            } else {
                *other_ms += ms;
            }
        }
    }
    c->ev_marks.clear();
    c->ev_used = 0;
    return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *c)
{
    if (!c) return "null context";
    return c->err.c_str();
}

void lbm_destroy(lbm_ctx *c)
{
    if (!c) return;
    drop_graphs(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : c->aux_ev) cudaEventDestroy(e);
    for (cudaStream_t s : c->aux) cudaStreamDestroy(s);
    delete c;
}

}  // extern "C"

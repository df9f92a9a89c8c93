/*
 * lbm.h -- C ABI of the GB300 active lattice Boltzmann library (liblbm.so).
 *
 * The library advances the active lattice Boltzmann model of Nesbitt,
 * Pruessner & Lee (arXiv:1902.00530) on periodic D2Q9 lattices:
 *   f_i(t+1, r + e_i) - f_i(t, r) = -(f_i - f^SS_i)/tau + eta_i
 * (Sec. 2, Eq. (fevolution2)) with f^SS_i = xi_i(rho, u*) (Eq. (fssD2Q7),
 * lifted to D2Q9 with c_s^2 = 1/3), u* given by the MIPS closure (Sec. 3,
 * Eq. (bu_mips) with the U_max clamp), the CIL closure (Sec. 4, Eqs. (bu_CIL),
 * (U0)) or the passive limit u* = u (App. A.1), zero-sum uniform noise
 * (Eq. (noiseDensityConservation)) and the negative correction of App. A.3,
 * in the step order of App. A.2.
 *
 * Conventions for every call:
 *  - Ownership.  The caller owns all device memory and the CUDA stream: it
 *    allocates the state and scratch buffers whose sizes lbm_buffer_bytes
 *    reports and hands them over with lbm_bind.  The context owns only host
 *    descriptors, tuning results, cached CUDA graphs and, for a batch of
 *    several launch groups (lattices differing in model, storage or velocity
 *    set), one auxiliary stream per extra group and their events, created on
 *    the first lbm_step and destroyed by lbm_destroy.  Every call that launches
 *    device work enqueues it on the bound stream or on work forked from it and
 *    joined back into it before the call returns; calls documented as "syncs"
 *    wait for that stream before returning.
 *  - Errors.  Every call returns an lbm_status.  Nothing throws across the ABI
 *    and nothing exits.  lbm_last_error(ctx) describes the last failure.
 *    Device-side conditions (non-finite observables, a barrier that timed out)
 *    are latched in a device flag and reported by the next syncing call.
 *  - Populations.  Device storage is structure-of-arrays per lattice:
 *    f[i][y][pitch] for i = 0..Q-1, x fastest, with the D2Q9 velocities
 *    e = (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
 *    (Q = 9) or the D2Q7 set below (Q = 7).  Calls that exchange populations
 *    with the caller use dense FP32 [Q][ny][nx] arrays regardless of the
 *    storage type.
 *  - Threads.  One context per host thread; contexts are independent.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = 1, /* a bad argument; nothing was changed            */
    LBM_ERR_UNBOUND = 2,     /* buffers not bound (lbm_bind) or not initialised */
    LBM_ERR_CUDA = 3,        /* a CUDA runtime call failed                      */
    LBM_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up              */
    LBM_ERR_NUMERIC = 5,     /* non-finite observables were detected            */
    LBM_ERR_UNSUPPORTED = 6  /* a valid request the library does not provide    */
} lbm_status;

typedef enum {
    LBM_PASSIVE = 0, /* u* = u: standard BGK lattice Boltzmann (App. A.1)          */
    LBM_MIPS = 1,    /* u* = C (1 - rho/rho*) grad rho, clamped to U_max (Sec. 3)  */
    LBM_CIL = 2      /* u* = U0(rho) u/|u|, U0 = max(B - A rho^2, 0) (Sec. 4)      */
} lbm_model;

typedef enum {
    LBM_F32 = 0,          /* populations stored as FP32                              */
    LBM_F16_SHIFTED = 1,  /* stored as FP16 of f_i - w_i rho0, collided in FP32      */
    LBM_BF16_SHIFTED = 2  /* stored as BF16 of f_i - w_i rho0, collided in FP32      */
} lbm_storage;

typedef enum {
    LBM_D2Q9 = 0, /* square lattice, nine velocities (the default)                  */
    LBM_D2Q7 = 1  /* the paper's triangular lattice (Sec. 2), seven velocities       */
} lbm_velocity_set;

/* One periodic rectangular lattice (Sec. 4: "rectangular geometry with
 * periodic boundary conditions").  id keys the lattice's random streams: two
 * lattices with the same seed, id and state evolve identically.
 *
 * D2Q7 (Sec. 2): e_0 = 0, e_i = (cos((i-1) pi/3), sin((i-1) pi/3)), i = 1..6,
 * w_0 = 1/2, w_i = 1/12, c_s^2 = 1/4; f^SS with the printed coefficients 4, 8,
 * -2 (Eq. (fssD2Q7)); grad rho by the explicit Sec. 3 stencils; App. A.3
 * pairs 1-4, 2-5, 3-6.  Site (x, y) sits at (x + (y mod 2)/2, y sqrt(3)/2):
 * rows are sqrt(3)/2 apart and every odd row is shifted right by half a
 * spacing, so ny must be even.  Populations are f[i][y][x], i = 0..6.  The
 * noise of a site uses one Philox call whose 16-bit halves h_0..h_6 give
 * s_i = (2 h_i + 1 - 2^16) / 2^16. */
typedef struct {
    int32_t nx, ny;        /* sites along x and y, each in [1, 65536]; D2Q7: ny even */
    int32_t storage;       /* an lbm_storage value                                   */
    int32_t id;            /* random-stream id, in [0, 2^24)                         */
    int32_t velocity_set;  /* an lbm_velocity_set value (0 = D2Q9)                   */
} lbm_lattice;

/* Model parameters (App. C tables), all in lattice units dx = dt = c = 1. */
typedef struct {
    double tau;      /* relaxation time, > 1/2; the paper uses tau >= 1 (App. A.3) */
    double sigma;    /* noise: eta~_i uniform on [-sigma, sigma] (Sec. 2); >= 0    */
    double C;        /* MIPS gradient sensitivity (Eq. (bu_mips))                  */
    double rho_star; /* MIPS density ceiling rho* > 0                              */
    double u_max;    /* MIPS speed clamp U_max >= 0                                */
    double A, B;     /* CIL U0(rho) = max(B - A rho^2, 0) (Eq. (U0))               */
    double rho0;     /* 16-bit storage shift; 0 = the mean density set by lbm_init */
} lbm_params;

/* Seeded initial state (App. C.2): per site, rho = rho_mean (1 + rho_amp (2U-1))
 * and u by u_kind; populations are set to f^SS(rho, u) computed in FP64.
 *   u_kind 0: u = (ux0, uy0) + u_amp (2U1 - 1, 2U2 - 1)
 *   u_kind 1: u = (ux0, uy0) + u_amp (cos 2 pi U1, sin 2 pi U1)
 *   u_kind 2: u = U0(rho) (cos 2 pi U1, sin 2 pi U1)   (the paper's CIL start) */
typedef struct {
    double rho_mean, rho_amp;
    int32_t u_kind;
    double u_amp, ux0, uy0;
} lbm_init_spec;

/* One observable record of a stored state (after the step's correction):
 * mass = sum rho; phi = |sum rho u| / sum rho (Eq. (phi));
 * drho_y = population std over x of rho_y(x) = mean over y of rho (App. D);
 * drho_x = the same with axes swapped; var_rho = population variance of rho;
 * zeta = sum rho (B - |u|) / sum rho (App. D).  t is the time of the state. */
typedef struct {
    int64_t t;
    double mass, phi, drho_y, drho_x, var_rho, zeta;
} lbm_obs;

typedef struct lbm_ctx lbm_ctx;

/* Create a context for one lattice.  Validates the parameters: tau <= 1/2,
 * sigma < 0, a NaN parameter, nx or ny outside [1, 65536], an unknown model or
 * storage, or a non-positive rho_star (MIPS) returns LBM_ERR_INVALID_ARG and
 * sets *out = NULL.  A D2Q9 lattice of more than 2^32 population elements per
 * buffer (9 ny pitch, pitch = nx rounded up to 128 bytes; about 477 million
 * sites) runs only the shared-memory staged kernel, which needs nx a multiple
 * of 16 bytes of storage: otherwise LBM_ERR_UNSUPPORTED, *out = NULL.  Host
 * only; no CUDA call. */
lbm_status lbm_create(const lbm_lattice *lattice, lbm_model model, const lbm_params *params,
                      lbm_ctx **out);

/* Create a context for n independent lattices advanced together (a batch, as
 * in the paper's sweeps over density and activity, App. C.3-C.4).  Arrays
 * hold n entries.  Lattice k of the batch is addressed by index k below.
 * Same validation and status codes as lbm_create.  Host only. */
lbm_status lbm_create_batch(int32_t n, const lbm_lattice *lattices, const lbm_model *models,
                            const lbm_params *params, lbm_ctx **out);

/* Observable sampling: every sample_every steps (0 = never) the step's
 * stored state is reduced to one lbm_obs record per lattice into a device
 * ring of ring_capacity records per lattice (App. C: samples every t_sample
 * steps).  Must be called before lbm_buffer_bytes/lbm_bind.  Host only. */
lbm_status lbm_set_sampling(lbm_ctx *ctx, int32_t sample_every, int32_t ring_capacity);

/* Device bytes the caller must allocate: state (two population buffers per
 * lattice) and scratch (reduction partials, observable ring, step counter,
 * descriptors, error flag).  Host only. */
lbm_status lbm_buffer_bytes(const lbm_ctx *ctx, size_t *state_bytes, size_t *scratch_bytes);

/* Hand over device buffers (256-byte aligned, at least the sizes above) and
 * the stream (a cudaStream_t; NULL = legacy default stream).  The caller keeps
 * ownership and must keep them alive until lbm_destroy or the next lbm_bind.
 * Uploads descriptors; syncs. */
lbm_status lbm_bind(lbm_ctx *ctx, void *state_dev, void *scratch_dev, void *cuda_stream);

/* Seeded initial state of every lattice (App. C.2); specs holds one entry per
 * lattice.  Sets t = 0, clears the observable ring.  Enqueued; syncs. */
lbm_status lbm_init(lbm_ctx *ctx, uint64_t seed, const lbm_init_spec *specs);

/* Advance every lattice n >= 0 steps (App. A.2 steps 1-6 per step), t += n.
 * Enqueued on the bound stream; returns without waiting.  The first call
 * tunes the launch shape unless lbm_set_tuning disabled it.  Requires
 * t + n < 2^32 (the step index is one 32-bit word of the noise counter). */
lbm_status lbm_step(lbm_ctx *ctx, int64_t n);

/* Density and velocity of every site of lattice `lattice` in its stored
 * state (Eq. (D2Q7macroscopic), on either lattice): rho, ux, uy are DEVICE pointers to
 * dense FP32 [ny][nx] arrays, written asynchronously on the bound stream. */
lbm_status lbm_moments(lbm_ctx *ctx, int32_t lattice, float *rho, float *ux, float *uy);

/* Observables of lattice `lattice` in its current stored state, computed now
 * by the same fused reduction the sample steps use.  Syncs; returns
 * LBM_ERR_NUMERIC if a sum is not finite. */
lbm_status lbm_observables(lbm_ctx *ctx, int32_t lattice, lbm_obs *out);

/* Copy the sampled records of lattice `lattice` (oldest first, at most cap)
 * to host memory and report how many were written; the ring is then empty
 * for that lattice.  Records beyond the ring capacity overwrite the oldest.
 * Syncs. */
lbm_status lbm_observable_series(lbm_ctx *ctx, int32_t lattice, lbm_obs *out, int32_t cap,
                                 int32_t *n_out);

/* Copy lattice `lattice`'s populations out as dense FP32 [Q][ny][nx]; dst is a
 * host pointer if dst_is_host, else a device pointer.  16-bit storage is
 * expanded to f_i = w_i rho0 + s_i.  Syncs. */
lbm_status lbm_get_state(lbm_ctx *ctx, int32_t lattice, float *dst, int32_t dst_is_host);

/* Replace lattice `lattice`'s populations by dense FP32 [Q][ny][nx] from src
 * (host if src_is_host, else device).  16-bit storage stores s_i = f_i -
 * w_i rho0 rounded to nearest.  Does not change t.  Syncs. */
lbm_status lbm_set_state(lbm_ctx *ctx, int32_t lattice, const float *src, int32_t src_is_host);

/* Change the mean density of lattice `lattice` (-1: every lattice) without
 * re-initialising, as in the paper's adiabatic density sweeps (App. C.2:
 * "adding delta rho-bar / 7 to every f_i": delta / Q to each of the Q
 * populations of every site).  For 16-bit storage the shifted stored
 * values are updated and rounded to nearest.  Enqueued on the bound stream. */
lbm_status lbm_add_density(lbm_ctx *ctx, int32_t lattice, double delta_rho_bar);

/* Replace the model parameters of lattice `lattice` (-1: every lattice)
 * between steps (noise sweeps, App. C.1; activity sweeps, App. C.4).  Same
 * validation as lbm_create; rho0 (the 16-bit storage shift) cannot change
 * after lbm_init and is ignored.  Host side plus a descriptor upload (syncs). */
lbm_status lbm_set_params(lbm_ctx *ctx, int32_t lattice, const lbm_params *params);

/* Current time step t (steps taken since lbm_init or loaded with lbm_load). */
lbm_status lbm_get_time(const lbm_ctx *ctx, int64_t *t);

/* Serialise all lattices (raw storage, t, seed) to a file / restore them.
 * The context must have the same lattices, models and storage.  Because the
 * noise is counter-based (keyed by seed, site, t and id), a run resumed from a
 * file continues bit-identically.  Syncs. */
lbm_status lbm_save(lbm_ctx *ctx, const char *path);
lbm_status lbm_load(lbm_ctx *ctx, const char *path);

/* Launch-shape tuning.  mode 0: automatic on the first lbm_step (default);
 * mode 1: off, use the fixed shape given for every lattice: vec = sites per
 * thread along x (1, 2 or 4 for FP32; 1, 2, 4 or 8 for 16-bit storage; must
 * divide nx), rows = rows per warp strip (8..4096), warps = warps per block
 * (1..8), stages = 0 for the kernel that loads populations straight from
 * global memory, or 2..8 (MIPS: 3..8) for the kernel that stages population
 * rows in shared memory with bulk copies, that many rows in flight per block,
 * whose warps share each staged row (needs nx a multiple of 16 bytes of
 * storage; D2Q7 lattices also need rows even; the buffers, stages x Q x
 * (32 vec warps + 2 halo) values, must fit the 227 KB of shared memory a
 * block can have, else LBM_ERR_INVALID_ARG).  stages = 0 is refused (LBM_ERR_INVALID_ARG) while a D2Q9
 * lattice exceeds 2^32 elements per buffer (see lbm_create); such lattices
 * start on a staged shape and the tuner tries only staged shapes for them.
 * Host only; re-uploads descriptors (syncs) when bound. */
lbm_status lbm_set_tuning(lbm_ctx *ctx, int32_t mode, int32_t vec, int32_t rows, int32_t warps,
                          int32_t stages);

/* Run the tuner now (times candidate shapes on the bound buffers without
 * changing the state).  Syncs. */
lbm_status lbm_tune(lbm_ctx *ctx);

/* The launch shape in use for lattice `lattice`: vec, rows, warps per block,
 * stages (0 = direct-load kernel). */
lbm_status lbm_get_tuning(const lbm_ctx *ctx, int32_t lattice, int32_t *vec, int32_t *rows,
                          int32_t *warps, int32_t *stages);

/* CUDA-graph replay of lbm_step: 1 = capture each distinct step sequence once
 * and replay it (default), 0 = launch kernels directly. */
lbm_status lbm_set_graphs(lbm_ctx *ctx, int32_t enabled);

/* Persistent launches (the paper's many independent runs per parameter point,
 * App. C.3-C.4, advanced together; each step is App. A.2's update, unchanged).
 * A launch group that takes them (either lattice, on the direct kernel:
 * stages = 0 in lbm_get_tuning) runs each stretch of two or more consecutive
 * steps without a sample step as ONE kernel launch, of at most 4096 steps
 * (fewer for very large groups, so that steps x blocks stays below 2^31);
 * sample steps and staged groups launch once per step.  Inside the launch, blocks take
 * (step, block) work items from a counter -- lattice group by lattice group,
 * step by step inside a group -- and each item waits only for the strip rows
 * it reads to finish the previous step, so consecutive steps overlap with no
 * launch boundary or grid-wide barrier between them.  A lattice group is a run
 * of consecutive lattices whose two population buffers together fit
 * l2_group_mib MiB (at least one lattice per group); 0 (the default) puts every
 * lattice of a launch group in one.  States, samples and observables are
 * bitwise those of the per-step launches.
 * mode 0: one launch per step.  mode 1: every group that can takes persistent
 * launches; the tuner times its direct shapes that way.  mode 2 (default): for
 * a group of at least 2^20 sites (smaller steps cannot fill the GPU in either
 * form, and there one launch per step measured faster), the tuner times every
 * direct shape both ways (the persistent way over 12 steps,
 * recomputing the current step into the spare buffer) and keeps the faster
 * form with the shape, per group, then checks the choice with the whole batch
 * running; until it has run (and with tuning off, lbm_set_tuning mode 1)
 * groups launch once per step.  Setting mode 2 makes the next lbm_step tune
 * again when tuning is automatic.  Measured on one GB300: the 256-lattice
 * 256^2 CIL batch in FP32 at 85.9 GLUPS persistent (16-row strips) against
 * 81.3 per step; in FP16 storage the per-step launch stays faster (83.5).
 * The waits are bounded (about 1 s, then the error flag is raised and the call
 * that reads it returns LBM_ERR_TIMEOUT).  Each launch first clears its
 * counters in the context's scratch (a memset on the bound stream; a graph
 * node when graphs are on), so launches of one context must not overlap on
 * the GPU, as for every other call.  mode outside 0..2 or l2_group_mib
 * outside [0, 2^20] gives LBM_ERR_INVALID_ARG.  Host only; drops captured
 * graphs and re-uploads descriptors (syncs) when bound. */
lbm_status lbm_set_persistent(lbm_ctx *ctx, int32_t mode, int32_t l2_group_mib);

/* Whether lattice `lattice`'s launch group runs its stretches of plain steps as
 * persistent launches (1) or one launch per step (0) under the current mode,
 * shape and tuning (see lbm_set_persistent).  Host only. */
lbm_status lbm_get_persistent(const lbm_ctx *ctx, int32_t lattice, int32_t *persistent);

/* Number of kernels the last lbm_step call enqueued (graph nodes included). */
lbm_status lbm_last_launch_count(const lbm_ctx *ctx, int64_t *count);

/* Kernel timing on the bound stream.  While enabled, lbm_step launches its
 * kernels directly (no graph replay) with a CUDA event pair around each one;
 * lbm_profile_read syncs and reports the summed device time of the fused step
 * kernels and of all other kernels since profiling was enabled (or last
 * read), and the number of step-kernel launches; reading resets the sums. */
lbm_status lbm_set_profiling(lbm_ctx *ctx, int32_t enabled);
lbm_status lbm_profile_read(lbm_ctx *ctx, double *step_ms, int64_t *step_launches, double *other_ms);

/* Check of the device-side failure path (the bounded waits of the staged
 * kernels, App. A.2's step being the work they wait for): runs one warp that
 * waits on a barrier phase nothing completes.  The wait gives up after its
 * limit (about 1 s) and raises the device error flag, which this call reads and
 * clears, so it returns LBM_ERR_TIMEOUT; the context stays usable.  Syncs the
 * bound stream.  LBM_ERR_UNBOUND before lbm_bind. */
lbm_status lbm_check_wait_timeout(lbm_ctx *ctx);

/* Observables of a population field, allocating nothing.
 *
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory -- code inside a memory pool or allocator owned by
 * another runtime, which may not take device memory of its own, or an
 * embedding that must keep its device memory footprint fixed.  It computes
 * the same record as lbm_observables for a caller-supplied state instead of a
 * context's.
 *
 * f_dev: DEVICE pointer to dense FP32 D2Q9 populations [9][ny][nx] (caller-owned,
 * read only); 1 <= nx, ny <= LBM_NOALLOC_MAX_SIDE.  B: the CIL constant used
 * by zeta.  out: host record (t is set to 0).  cuda_stream: the stream to run
 * on (NULL = legacy default stream).  The call copies the record to a host
 * buffer and synchronises that stream before it returns.
 *
 * Scratch: a fixed array of LBM_NOALLOC_SCRATCH_BYTES compiled into the
 * library, held by every GPU that loads the library until the process exits.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it.  All calls share the array, which keeps the
 * last call's partial sums (each call overwrites what it reads): calls that
 * overlap on the GPU -- from two streams or two host threads -- race and must
 * be serialised by the caller.  No cudaMalloc, cudaFree or allocating library
 * routine is called.
 * Returns LBM_ERR_INVALID_ARG for sizes beyond the maximum or null pointers,
 * LBM_ERR_CUDA if a CUDA call fails, LBM_ERR_NUMERIC for non-finite sums. */
#define LBM_NOALLOC_MAX_SIDE 4096
#define LBM_NOALLOC_SCRATCH_BYTES (1088 * 1024)
lbm_status lbm_observables_noalloc(const float *f_dev, int32_t nx, int32_t ny, double B, lbm_obs *out,
                                   void *cuda_stream);

/* Text of the last error on this context (never NULL; "" if none). */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Release host resources.  NULL is a no-op.  Does not free caller buffers. */
void lbm_destroy(lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */

// lbm_internal.h -- declarations shared by the library's translation units.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// fused step / observe kernels (lbm_step_*.cu, one unit per storage type).
// noise: 0 = sigma = 0 in every lattice of the launch, 1 = sigma > 0 in every
// one, 2 = mixed (decided per lattice in the kernel).
cudaError_t launch_step_f32(int model, int kind, int vec, bool sample, int noise, const StepArgs &a, int blocks,
                            int warps, cudaStream_t stream);
cudaError_t launch_step_f16(int model, int kind, int vec, bool sample, int noise, const StepArgs &a, int blocks,
                            int warps, cudaStream_t stream);
cudaError_t launch_step_bf16(int model, int kind, int vec, bool sample, int noise, const StepArgs &a, int blocks,
                             int warps, cudaStream_t stream);
// the persistent launch of the direct kernels over `p.nsteps` steps
// (lbm_step_persistent.cuh), D2Q9 and D2Q7 (q7_); step_blocks = blocks of
// the per-step grid
cudaError_t launch_persistent_f32(int model, int vec, int noise, const StepArgs &a, const PersistArgs &p,
                                  int step_blocks, int warps, cudaStream_t stream);
cudaError_t launch_persistent_f16(int model, int vec, int noise, const StepArgs &a, const PersistArgs &p,
                                  int step_blocks, int warps, cudaStream_t stream);
cudaError_t launch_persistent_bf16(int model, int vec, int noise, const StepArgs &a, const PersistArgs &p,
                                   int step_blocks, int warps, cudaStream_t stream);
cudaError_t launch_persistent_q7_f32(int model, int vec, int noise, const StepArgs &a, const PersistArgs &p,
                                     int step_blocks, int warps, cudaStream_t stream);
cudaError_t launch_persistent_q7_f16(int model, int vec, int noise, const StepArgs &a, const PersistArgs &p,
                                     int step_blocks, int warps, cudaStream_t stream);
cudaError_t launch_persistent_q7_bf16(int model, int vec, int noise, const StepArgs &a, const PersistArgs &p,
                                      int step_blocks, int warps, cudaStream_t stream);
cudaError_t launch_observe_f32(int vec, const StepArgs &a, int blocks, int warps, cudaStream_t stream);
cudaError_t launch_observe_f16(int vec, const StepArgs &a, int blocks, int warps, cudaStream_t stream);
cudaError_t launch_observe_bf16(int vec, const StepArgs &a, int blocks, int warps, cudaStream_t stream);

// the D2Q7 step / observe kernels (lbm_step_q7_*.cu, one unit per storage
// type); kind 0 = direct loads, 1 = bulk-copy staged rows
cudaError_t launch_step_q7_f32(int model, int kind, int vec, bool sample, int noise, const StepArgs &a, int blocks,
                               int warps, cudaStream_t stream);
cudaError_t launch_step_q7_f16(int model, int kind, int vec, bool sample, int noise, const StepArgs &a, int blocks,
                               int warps, cudaStream_t stream);
cudaError_t launch_step_q7_bf16(int model, int kind, int vec, bool sample, int noise, const StepArgs &a, int blocks,
                                int warps, cudaStream_t stream);
cudaError_t launch_observe_q7_f32(int vec, const StepArgs &a, int blocks, int warps, cudaStream_t stream);
cudaError_t launch_observe_q7_f16(int vec, const StepArgs &a, int blocks, int warps, cudaStream_t stream);
cudaError_t launch_observe_q7_bf16(int vec, const StepArgs &a, int blocks, int warps, cudaStream_t stream);

// auxiliary kernels (lbm_aux.cu); the lattice's q comes from its descriptor,
// so `cells` counts sites and q * cells elements are touched
size_t init_spec_bytes();
void pack_init_spec(void *dst, double rho_mean, double rho_amp, int u_kind, double u_amp, double ux0,
                    double uy0, double A, double B);
cudaError_t launch_init(int storage, const LatDesc *desc, const void *specs, int nlat, long long max_cells,
                        int dst, uint64_t seed, cudaStream_t s);
cudaError_t launch_moments(int storage, const LatDesc *desc, int lat, long long cells, int src, float *rho,
                           float *ux, float *uy, cudaStream_t s);
cudaError_t launch_export(int storage, const LatDesc *desc, int lat, long long cells, int src, float *out,
                          cudaStream_t s);
cudaError_t launch_import(int storage, const LatDesc *desc, int lat, long long cells, int dst,
                          const float *in, cudaStream_t s);
cudaError_t launch_finalize(const LatDesc *desc, int nlat, int max_chunk, const uint32_t *t_ptr, uint32_t k,
                            int to_ring, unsigned *err, cudaStream_t s);
cudaError_t launch_advance_time(uint32_t *t_ptr, uint32_t n, cudaStream_t s);
cudaError_t launch_add_density(int storage, const LatDesc *desc, int lat, long long cells, int buf, float per_pop,
                               cudaStream_t s);
cudaError_t launch_set_time(uint32_t *t_ptr, uint32_t t, cudaStream_t s);
cudaError_t launch_wait_timeout(unsigned *err, cudaStream_t s);

}  // namespace lbm

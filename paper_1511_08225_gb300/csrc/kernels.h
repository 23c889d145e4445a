// kernels.h -- host-side launchers of the SLPIC kernels (kernels.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "slpic_internal.cuh"

namespace slpic {

constexpr int kParticleThreads = 256;
constexpr int kFieldThreads = 1024;        // k_potential (one CTA)
constexpr int kFieldClusterCtas = 8;       // k_field: one cluster of 8 CTAs
constexpr int kFieldClusterCtasWide = 16;  // k_field_wide: 16 (non-portable cluster size)
constexpr int kFieldClusterThreads = 256;

size_t particle_smem_bytes(int nn);         // E + one int64 per node (allocation-free kernel)
size_t particle_kernel_smem_bytes(int nn);  // k_particles_compact: E + split deposit
size_t particle_inplace_smem_bytes(int nn); // k_particles: E + split deposit
constexpr int kCompactEvery = 16;           // one compacting particle step per this many
size_t field_smem_bytes(int nn);
size_t field_cluster_smem_bytes(int nn, int ns, int ctas);
int field_max_nodes();
cudaError_t configure_kernels(int nn);
cudaError_t particle_ctas_per_sm(int nn, int *inplace, int *compacting);

void launch_particles(const StepParams &p, int ctas_per_species, bool compact, cudaStream_t st);
// k_particles_tma: the in-place step with the particle stream staged by TMA bulk
// copies, one CTA of kTmaThreads per SM (kTmaConsumers consumer threads, one
// producer warp), tiles of kTmaTile particles in a ring of `stages` stages.
constexpr int kTmaThreads = 1024;
constexpr int kTmaConsumers = 992;
constexpr int kTmaPer = 2;                         // particles per consumer thread per tile
constexpr int kTmaTile = kTmaConsumers * kTmaPer;  // 1,984 particles: 7,936 B of cells
size_t particle_tma_smem_bytes(int nn, int stages);
// ring stages that fit beside an nn-node grid (at most 4); 0 if fewer than 2 fit
cudaError_t configure_particles_tma(int nn, int *stages);
void launch_particles_tma(const StepParams &p, int ctas, int stages, cudaStream_t st);
void launch_hard(const StepParams &p, int ctas, bool compact, cudaStream_t st);
void launch_field(const StepParams &p, int mode, cudaStream_t st);
// copy of a deposit ([species][nn], ndep words) and of E, for an overlapped read-back
void launch_snapshot(const unsigned long long *dep, unsigned long long *dep_out, size_t ndep,
                     const float *E, float *E_out, int nn, cudaStream_t st);
// rho and phi (p.rho, p.phi) from the deposit dep ([species][nn]) of time level step
void launch_potential(const StepParams &p, const unsigned long long *dep, long long step,
                      cudaStream_t st);
// batched forms over many instances: d_params[m] on the device; the particle
// kernels take one CTA per work item (instance, species, share, shares)
cudaError_t configure_batch_kernels(int max_nn, int *inplace_per_sm, int *compact_per_sm);
void launch_particles_batch(const StepParams *d_params, const int4 *d_work, int n_work,
                            int max_nn, bool compact, cudaStream_t st);
void launch_hard_batch(const StepParams *d_params, int m, int ctas_per_instance, bool compact,
                       cudaStream_t st);
void launch_field_batch(const StepParams *d_params, int m, int max_nn, int max_ns, int mode,
                        cudaStream_t st);
void launch_deposit(const StepParams &p, int ctas_per_species, cudaStream_t st);
void launch_diag(const StepParams &p, double *out, int ctas_per_species, cudaStream_t st);
void launch_validate(const int32_t *cell, const float *off, const float *v, long long n,
                     int n_cells, int *bad, cudaStream_t st);
void launch_pack(const int32_t *cell, const float *off, const float *v, long long n,
                 int32_t *cdst, float4 *pdst, cudaStream_t st);
void launch_unpack(const int32_t *csrc, const float4 *psrc, long long n, int32_t *cell,
                   float *off, float *v, cudaStream_t st);

}  // namespace slpic

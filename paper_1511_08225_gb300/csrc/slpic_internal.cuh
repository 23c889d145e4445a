// slpic_internal.cuh -- device data layout shared by the kernels and the C ABI.
//
// Particle store (per species, ping-pong buffer b = 0/1):
//   cell[b][i]  int32   cell index c (0 <= c < N), or -1 for a hole (a particle
//                       absorbed since the last compacting step)
//   pv[b][i]    float4  {offset in [0,1), vx, vy, vz}
// 20 bytes per macroparticle, structure-of-arrays so that one warp reads 512
// contiguous bytes of float4 and 128 bytes of int32 per access.  The particles
// of time level n sit in slots [0, count) of buffer (n & 1); the particle kernel
// of step n reads buffer (n & 1) and writes buffer ((n+1) & 1).  Most steps write
// every particle back to its own slot and leave a hole where one was absorbed;
// every compaction interval a compacting step packs the survivors.
//
// Charge deposit: int64 fixed point, 2 time levels x species x nodes; the
// deposit of rho^n is acc[(n & 1)][s][j].
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "slpic.h"

namespace slpic {

constexpr int kMaxSpecies = SLPIC_MAX_SPECIES;

// Counters and bookkeeping that live on the device, so that a captured CUDA
// graph can run many steps with no host round trip.
struct DevState {
    long long step;                                // time level n of the current particles
    unsigned long long count[kMaxSpecies][2];      // slots in use per buffer (live + holes)
    unsigned long long absorbed_step[kMaxSpecies][2];  // absorbed this step, per wall
    long long absorbed_total[kMaxSpecies][2];
    long long injected_total[kMaxSpecies];
    long long iterative_total[kMaxSpecies];        // pushed by k_hard (walk + Newton), cumulative
    double src_frac[kMaxSpecies];                  // fractional macroparticles carried over
    unsigned long long holes[kMaxSpecies][2];      // absorbed slots (cell < 0) per buffer
    unsigned long long hard_n[kMaxSpecies];        // particles listed for k_hard this step
    int error;                                     // first SLPIC_ERR_* raised on the device
    int pad;
    // device time of the step's kernels (0 particle, 1 k_hard, 2 k_field): per launch
    // the span from the first CTA's start to the last CTA's end (globaltimer, ns)
    unsigned long long span_t0n[3];       // ~(earliest start) of the running launch; 0 = none
    unsigned long long span_ns[3];        // summed spans
    unsigned long long span_launches[3];  // launches summed
    unsigned int span_done[3];            // CTAs of the running launch that have finished
    unsigned int pad2;
};

// A particle listed for the iterative push, with what the push needs, so that the
// kernel that pushes it reads one record instead of a chain of dependent loads.
struct HardRec {
    int32_t slot;  // its slot in the step's input buffer
    int32_t cell;  // c at time level n
    float ax;      // (q/m) E gathered at the particle
    int32_t pad;
    float4 q;      // {offset, vx, vy, vz} at time level n (v = v^{n-1/2})
};

struct SpeciesDev {
    int32_t *cell[2];
    float4 *pv[2];
    // this step's particles that need the iterative push: entry k < hard_recs is a
    // record in hard[k]; a longer list (rare) continues as slots in hard_slot[k]
    HardRec *hard;
    int32_t *hard_slot;
    long long hard_recs;
    long long capacity;
    float qm;        // q/m
    float v0;        // speed limit
    float vth_src;   // sqrt(T_src/m) of the source Maxwellian (0 = not injected)
    int kind;        // SLPIC_BETA_*
    double qw_dx;    // q * w / dx: charge density of one whole particle's deposit
    double rho_unit; // q * w / dx * 2^-40: charge density of one fixed-point unit
    double w;        // g-weight
    double inv_w;    // 1 / w
    double wall_rate;  // wall source: macroparticles entering per step (0 = none)
};

// Everything a kernel needs, passed by value (fixed at graph capture; the
// time level is read from DevState at run time).
struct StepParams {
    int n_cells;
    int nn;           // nodes: N+1 (Dirichlet) or N (periodic)
    int periodic;
    int ns;
    float dt;
    float dt_dx;      // dt / dx
    double dx;
    double dt64;
    double eps0;
    double phi_lo, phi_hi;
    double inv_n;     // 1 / n_cells
    double inv_dx;    // 1 / dx
    double k2;        // dx^2 / eps0
    // source
    int src_mode;
    int src_ref;
    float src_lo_cells;
    float src_len_cells;
    double src_rate;
    unsigned long long seed;
    SpeciesDev sp[kMaxSpecies];
    // prescribed wave (test-particle mode): phi = phi0(t) sin(k (x - vphi t)),
    // phi0(t) = wave_phi0 min(1, t / wave_ramp); E is -dphi/dx, the charge unused
    int wave_on;
    double wave_phi0, wave_k, wave_vphi, wave_ramp;
    unsigned long long *acc;  // [2][ns][nn]
    float *E;                 // [nn]  FP32 copy gathered by the particle kernel
    double *E64;              // [nn]
    double *phi;              // [nn]
    double *rho;              // [nn]
    DevState *st;
    // speed limit that varies in space: the limit of species s in cell c is
    // sp[s].v0 * lam[c] (FP32 product); nullptr = uniform
    const float *lam;         // [n_cells]
    // longest spin of a pipeline wait in the particle kernel, in SM clock cycles
    // (slpic_set_wait_limit); the wait for the CTA's own copies in flight before it
    // exits keeps kDrainCycles whatever this is
    long long wait_cycles;
};

constexpr long long kWaitCycles = 2000000000LL;   // default wait limit, about a second
constexpr long long kDrainCycles = 2000000000LL;  // limit of the drain of copies in flight

}  // namespace slpic

/*
 * slpic.h -- C ABI of the GB300 speed-limited particle-in-cell library.
 *
 * Speed-limited PIC (SLPIC; Werner, Jenkins, Chap & Cary, arXiv 1511.08225)
 * advances macroparticles that sample g = f / beta along the characteristics
 * of Sec. II, Eq. (LimPtclDyn):  xdot = beta(|v|) v,  vdot = beta(|v|) q E / m,
 * with the leapfrog discretisation of Appendix A, Eq. (slpicIntegration):
 *
 *   v^{n+1/2} = v^{n-1/2} + (q/m) E^n(x^n) int_{t^{n-1/2}}^{t^{n+1/2}} beta dt
 *   x^{n+1}   = x^n + beta(|v^{n+1/2}|) v^{n+1/2} dt
 *   rho^{n+1} = sum_p q w beta(|v^{n+1/2}|) S(x - x^{n+1})
 *   div E^{n+1} = rho^{n+1} / eps0
 *
 * This library runs that loop on one GPU: 1D, 3 velocity components (1D3V,
 * as in the paper's sheath of Sec. IV), electrostatic, linear (CIC) shape,
 * absorbing Dirichlet or periodic boundaries, and a volume source.
 *
 * Units: whatever the caller uses consistently; the test problems use
 * normalised units (omega_pe = lambda_De = v_te = eps0 = e = m_e = 1).
 *
 * General rules for every entry point
 *  - Return value: SLPIC_OK (0) or a negative SLPIC_ERR_* code.  After an
 *    error, slpic_last_error(h) returns a message (valid until the next call).
 *  - Handles are opaque, created by slpic_create and owned by the caller,
 *    who must call slpic_destroy.  A handle is not thread-safe.
 *  - Array arguments belong to the caller.  Host arrays are read or written
 *    during the call only.  *_dev entry points take device pointers and run
 *    on the handle's stream (slpic_set_stream); they retain nothing.
 *  - The handle allocates its device memory (particle store, grid arrays) in
 *    slpic_create and frees it in slpic_destroy.
 *  - Work is asynchronous on the handle's stream; entry points that return
 *    host data synchronise that stream first.  Errors raised by kernels
 *    (capacity overflow, invalid particles) are reported by the next
 *    synchronising call.
 */
#ifndef SLPIC_H
#define SLPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SLPIC_OK 0
#define SLPIC_ERR_INVALID (-1)    /* bad argument or bad particle data        */
#define SLPIC_ERR_CFL (-2)        /* dt * v0 > dx: more than one cell a step  */
#define SLPIC_ERR_OOM (-3)        /* device allocation failed                 */
#define SLPIC_ERR_CAPACITY (-4)   /* particle store full (injection dropped)  */
#define SLPIC_ERR_NOCONVERGE (-5) /* iterative solve did not converge          */
#define SLPIC_ERR_TIMEOUT (-6)    /* a bounded device-side wait ran out        */
#define SLPIC_ERR_CUDA (-7)       /* CUDA runtime error (message has details)  */

/* ---- enumerations -------------------------------------------------------- */
/* beta of Sec. II: ONE = plain PIC; HEAVISIDE = Eq. (heavisideBeta),
 * beta = 1 for |v| <= v0 else v0/|v|; RELATIVISTIC = Eq. (relativisticBeta),
 * beta = v0 / sqrt(|v|^2 + v0^2). */
#define SLPIC_BETA_ONE 0
#define SLPIC_BETA_HEAVISIDE 1
#define SLPIC_BETA_RELATIVISTIC 2

#define SLPIC_BC_DIRICHLET_ABSORB 0 /* phi fixed at both walls; x<0 or x>=L absorbed */
#define SLPIC_BC_PERIODIC 1         /* x wraps; rho mean removed; mean(phi) = 0       */

#define SLPIC_SRC_NONE 0
#define SLPIC_SRC_LOSS_MATCHED 1 /* re-inject the physical count of ref-species losses */
#define SLPIC_SRC_RATE 2         /* inject rate*dt physical pairs per step              */
#define SLPIC_SRC_WALL 3         /* Sec. IV: every species with T_src > 0 enters through
                                    the plate at x = L from a stationary Maxwellian plasma
                                    of density src_rate: the one-sided flux
                                    src_rate sqrt(T_src/m) / sqrt(2 pi) per unit area and
                                    time, with the flux-weighted half-Maxwellian (|vx|
                                    Rayleigh, towards -x; vy, vz Maxwellian), each particle
                                    placed where it has moved since a uniformly random
                                    entry time in the step.  Dirichlet boundaries only. */

#define SLPIC_MAX_SPECIES 4

/* ---- configuration (Sec. IV problem statement) ---------------------------- */
typedef struct {
    double q;         /* charge per real particle                                  */
    double m;         /* mass per real particle                                    */
    double w;         /* g-weight: real particles per macroparticle (per unit area) */
    double v0;        /* speed limit of beta (ignored for SLPIC_BETA_ONE)          */
    double T_src;     /* temperature of the physical source Maxwellian; 0 = none   */
    int64_t capacity; /* maximum macroparticles of this species                    */
    int32_t beta_kind;/* SLPIC_BETA_*                                               */
    int32_t reserved;
} slpic_species;

typedef struct {
    int32_t ndim;          /* must be 1                                              */
    int32_t n_cells;       /* N; nodes are 0..N (Dirichlet) or 0..N-1 (periodic)     */
    double dx;             /* cell size                                              */
    double dt;             /* timestep                                               */
    int32_t bc;            /* SLPIC_BC_*                                             */
    int32_t n_species;     /* 1..SLPIC_MAX_SPECIES                                   */
    double phi_lo, phi_hi; /* wall potentials (Dirichlet)                            */
    double eps0;           /* permittivity (1 in normalised units)                   */
    double max_speed;      /* for SLPIC_BETA_ONE species: the caller's bound on |v|,
                              checked against dx/dt (0 = unchecked)                 */
    uint64_t seed;         /* source random stream                                   */
    int32_t src_mode;      /* SLPIC_SRC_*                                            */
    int32_t src_ref_species; /* LOSS_MATCHED: species whose losses are re-injected   */
    double src_lo_cells;   /* source band start, in cells                            */
    double src_len_cells;  /* source band length, in cells                           */
    double src_rate;       /* RATE: physical pairs per unit time (per unit area);
                              WALL: density of the plasma behind the right plate     */
    slpic_species species[SLPIC_MAX_SPECIES];
} slpic_config;

/* ---- diagnostics ----------------------------------------------------------- */
typedef struct {
    int64_t step;                       /* steps taken                           */
    double time;                        /* step * dt                             */
    int64_t count[SLPIC_MAX_SPECIES];   /* live macroparticles                   */
    double sum_w[SLPIC_MAX_SPECIES];    /* g-weight sum                          */
    double sum_wbeta[SLPIC_MAX_SPECIES];/* physical particle count sum(w beta)   */
    double kinetic[SLPIC_MAX_SPECIES];  /* physical kinetic energy
                                           sum(1/2 m w beta |v|^2) (f = beta g)  */
    double field_energy;                /* 1/2 eps0 dx sum_j E_j^2 (walls x 1/2) */
    int64_t absorbed[SLPIC_MAX_SPECIES][2]; /* macroparticles absorbed at x=0 / x=L,
                                               cumulative                         */
    int64_t injected[SLPIC_MAX_SPECIES];    /* macroparticles injected, cumulative */
    int64_t iterative[SLPIC_MAX_SPECIES];   /* pushes that took the iterative path
                                               (piece walk and Newton), cumulative  */
} slpic_diag;

typedef struct slpic_sim slpic_t;

/* ---- lifetime -------------------------------------------------------------- */

/* Validate *cfg and allocate a simulation on the current CUDA device.
 * Checks (Sec. II, "dt <~ dx/v0"): dt * v0_s <= dx for every speed-limited
 * species, and dt * max_speed <= dx for SLPIC_BETA_ONE species when
 * max_speed > 0; otherwise SLPIC_ERR_CFL.  Allocates 2 x capacity particle
 * slots per species (ping-pong) and the grid arrays; SLPIC_ERR_OOM if that
 * fails.  *out is set only on success. */
int slpic_create(const slpic_config *cfg, slpic_t **out);

/* Free everything the handle owns.  NULL is accepted. */
int slpic_destroy(slpic_t *h);

/* Message for the last error on this handle ("" if none).  Owned by h. */
const char *slpic_last_error(const slpic_t *h);

/* Message for the last slpic_create failure in this thread. */
const char *slpic_create_error(void);

/* A batch of m independent simulations (one per cfgs[i], each validated as by
 * slpic_create, of any size, species and speed limit) advanced together: every
 * slpic_step runs, for all instances at once, one particle launch (CTAs spread
 * over the instances in proportion to their particles), one launch for the
 * particles that need the iterative push, and one field launch (one thread-block
 * cluster per instance), captured in a CUDA graph.  Per-instance calls (loads,
 * fields, diagnostics, read-back) take the instance index.  slpic_save,
 * slpic_restore and the kernel-timing calls are not available on a batch
 * (SLPIC_ERR_INVALID).  On failure nothing is allocated and
 * slpic_create_error() names the instance that failed. */
int slpic_create_batch(const slpic_config *cfgs, int m, slpic_t **out);

/* Run all further work on `stream` (a cudaStream_t; NULL = the legacy default
 * stream).  The handle starts on a private non-blocking stream. */
int slpic_set_stream(slpic_t *h, void *stream);

/* ---- particles ------------------------------------------------------------- */

/* Append n macroparticles of `species` (Appendix A: the state at load is
 * x^0 and v^{-1/2}).  Host arrays: cell[n] (int32, 0 <= cell < N), offset[n]
 * (float32 in [0,1): x = (cell + offset) dx), v[3n] (float32, vx vy vz per
 * particle).  Invalid data (cell out of range, offset outside [0,1), non-finite
 * v) gives SLPIC_ERR_INVALID and loads nothing; more than the free capacity
 * gives SLPIC_ERR_CAPACITY.  After the last load call slpic_prepare (or the
 * first slpic_step) deposits rho^0 with beta(|v^{-1/2}|) and solves E^0.
 * `instance` is 0 for a handle from slpic_create and 0..m-1 for a batch from
 * slpic_create_batch (every per-instance entry point below takes it the same
 * way; SLPIC_ERR_INVALID outside that range). */
int slpic_load_particles(slpic_t *h, int instance, int species, int64_t n,
                         const int32_t *cell, const float *offset, const float *v);

/* Same, from device pointers (e.g. tensors already on the GPU). */
int slpic_load_particles_dev(slpic_t *h, int instance, int species, int64_t n,
                             const int32_t *cell, const float *offset, const float *v);

/* Same, from FP64 host positions x[n] in [0, L) and velocities v[3n]; the
 * library splits x into (cell, offset) and rounds to FP32. */
int slpic_load_particles_f64(slpic_t *h, int instance, int species, int64_t n,
                             const double *x, const double *v);

/* Deposit rho from the current particles (beta of their current velocity,
 * the quantised rule below) and solve phi and E.  Called implicitly by the
 * first slpic_step after a load. */
int slpic_prepare(slpic_t *h);

/* ---- the timestep ---------------------------------------------------------- */

/* Enqueue nsteps timesteps of Appendix A on the handle's stream and return.
 * One step: gather E^n, push v by the exact beta integral, move x by
 * beta(|v^{n+1/2}|) v^{n+1/2} dt, absorb at walls (or wrap), deposit
 * rho^{n+1}; then inject source particles (deposited into rho^{n+1}, first
 * pushed next step) and solve phi^{n+1}, E^{n+1}.  The steps run as a
 * captured CUDA graph with no host synchronisation between them. */
int slpic_step(slpic_t *h, int64_t nsteps);

/* Wait for queued work; report device-side errors raised since the last
 * report (SLPIC_ERR_CAPACITY, ...). */
int slpic_synchronize(slpic_t *h);

/* ---- read-back (host, synchronising) -------------------------------------- */

/* Fields of the latest solve, all nodal, n_nodes = N+1 (Dirichlet) or N
 * (periodic): rho (charge density, the wall nodes carry the half-cell charge
 * divided by dx), phi, E (the FP32 copy the particles gather).  Any pointer
 * may be NULL. */
int slpic_fields(slpic_t *h, int instance, double *rho, double *phi, float *E);
/* The same read-back without waiting: the potential kernel and the three copies
 * are queued on the handle's stream behind the steps already queued, and the
 * arrays are filled when the stream gets there (slpic_synchronize, or a CUDA event
 * on the stream, tells when).  The arrays must stay valid until then; page-locked
 * (pinned) host memory makes the copies overlap the following steps.  Errors of the
 * queued work are reported by the next synchronising call. */
int slpic_fields_async(slpic_t *h, int instance, double *rho, double *phi, float *E);

/* Physical number density sum(w beta S)/dx of one species, nodal. */
int slpic_density(slpic_t *h, int instance, int species, double *n);

/* The raw fixed-point deposit of one species from the latest deposit, int64
 * per node: every particle adds qT = rint(beta 2^40) split into
 * rint(beta*offset*2^40) on node cell+1 and the rest on node cell, with
 * beta = ONE ? 1 : HEAVISIDE ? (|v| <= v0 ? 1 : v0/|v|) : v0/sqrt(|v|^2+v0^2),
 * |v|^2 = (vx*vx + vy*vy) + vz*vz, every FP32 operation rounded to nearest
 * (no fused multiply-add).  Integer sums are exact, so the result does not
 * depend on particle order. */
int slpic_charge_raw(slpic_t *h, int instance, int species, int64_t *acc);

int slpic_particle_count(slpic_t *h, int instance, int species, int64_t *n);

/* Copy up to `cap` particles of a species to host arrays (layout as in
 * slpic_load_particles); *n_out = number copied.  Particle order is not
 * preserved across steps (absorbed particles are compacted out). */
int slpic_get_particles(slpic_t *h, int instance, int species, int64_t cap,
                        int32_t *cell, float *offset, float *v, int64_t *n_out);

/* Counts, energies and wall fluxes (see slpic_diag). */
int slpic_diagnostics(slpic_t *h, int instance, slpic_diag *out);

/* ---- checkpoint ------------------------------------------------------------ */

/* Serialise the complete state (particles, deposit, fields, counters, source
 * remainders, step index) into a host buffer.  With buf == NULL, *size
 * receives the bytes needed.  Restoring into a handle created from the same
 * config continues bit for bit.  Settings changed after creation
 * (slpic_set_speed_limit, slpic_set_speed_limit_profile, slpic_set_timestep,
 * slpic_set_wave) are not part of the checkpoint: set them again on the
 * restored handle. */
int slpic_save(slpic_t *h, void *buf, size_t *size);
int slpic_restore(slpic_t *h, const void *buf, size_t size);

/* ---- timing --------------------------------------------------------------- */

/* From now on slpic_step runs its steps in blocks of `steps_per_graph` (1..4096;
 * 0 turns timing off), each block one graph in which CUDA events bracket the
 * kernels of every step, starting at whatever step the run has reached.  The
 * events are recorded on the handle's stream, the stream the kernels run on; each
 * graph replay re-records them.  The steps of a call beyond a whole number of
 * blocks run untimed.  The event nodes separate the kernels, which adds a few
 * microseconds of launch latency to each bracketed interval. */
int slpic_enable_kernel_timing(slpic_t *h, int64_t steps_per_graph);

/* Mean device time (ms) per step of the streaming particle kernel, of the kernel
 * that pushes the particles needing iteration, and of the field/source kernel,
 * over the steps of the most recent timed graph replay (*steps of them; 0 if none
 * ran); synchronising.  Any pointer may be NULL. */
int slpic_kernel_times(slpic_t *h, double *particle_ms, double *hard_ms, double *field_ms,
                       int64_t *steps);

/* The particle kernel's pipeline waits (for a tile's bulk copy to land, for the
 * consumer warps to free a stage) give up after `cycles` SM clock cycles (default
 * 2e9, about a second; 0 restores the default).  A wait that gives up records
 * SLPIC_ERR_TIMEOUT, which the next synchronising call reports; the kernel then
 * skips its remaining tiles, waits for its own copies still in flight (with the
 * default limit, whatever `cycles` is) and returns, so the GPU context stays
 * usable.  The step it cut short leaves the handle's particles and fields no longer
 * those of the method: destroy the handle (reading it back stays safe).  A limit far
 * below a copy's latency exercises that path.  Below the default the waits poll the
 * barrier without suspending the thread (which costs issue slots), so that a short
 * limit can run out.  Takes effect from the next step (the step graphs are captured
 * again).  SLPIC_ERR_INVALID for cycles < 0 or a batch. */
int slpic_set_wait_limit(slpic_t *h, int64_t cycles);

/* Device time of the step's kernels, always recorded: for kind 0 (the particle
 * kernel, in-place or compacting), 1 (the kernel for the particles that need the
 * iterative push) and 2 (the source and field kernel), ms[kind] is the summed
 * device time of its launches since the handle was created, each launch counted
 * from the start of its first CTA to the end of its last on the GPU's global timer,
 * and launches[kind] the number of launches.  Differences of two calls give the
 * time of the steps between them.  Synchronising; either pointer may be NULL;
 * SLPIC_ERR_INVALID for a batch handle. */
int slpic_kernel_spans(slpic_t *h, double *ms, int64_t *launches);

/* Number of kernels one slpic_step(h, 1) launches. */
int slpic_kernels_per_step(slpic_t *h, int *n);

/* ---- performance settings and the autotuner ----------------------------------
 * None of these changes a result.  The source draws its random numbers by (seed,
 * step, species, particle index), the deposit is an integer sum and the field
 * follows from it, so the same steps give the same particles (as a set: their
 * slots may differ), fields and diagnostics whatever the settings.
 *   compact_every    a compacting particle step (survivors packed, holes
 *                    dropped) every this many steps, 2..1024 (default 16); holes
 *                    of absorbed particles occupy slots until then
 *   particle_kernel  in-place steps: 0 = the TMA-staged kernel when the grid
 *                    leaves room for its ring (default), 1 = the per-warp kernel;
 *                    single simulations only
 *   batch_waves      batches: particle-kernel work items ~ waves x resident CTAs
 *                    of the GPU, 1..16 (default 2)
 *   batch_min_share  batches: fewest particles per work item, 256..2^20
 *                    (default 4096)
 * slpic_set_tuning takes effect from the next step (the step graphs are captured
 * again).  slpic_autotune runs a coordinate search over candidate values (intervals
 * 8/16/32/64; the two kernels; waves 1/2/4/8; shares 1k/4k/16k/64k), each trial a
 * few steps to capture the graphs and then steps_per_trial steps (rounded up to
 * whole intervals) timed with CUDA events on the handle's stream, and keeps the
 * fastest.  The trials are real steps: the simulation advances by all of them.
 * An interval of v steps is tried only if the free slots of every species exceed
 * 4 v (2 r + 64), r the larger of its mean source rate per step since the start and
 * its rate over the tuner's first trial (a loss-matched source can still be growing):
 * eight times the holes and source particles the interval may gather.  A source that
 * later grows past that is truncated and reported (SLPIC_ERR_CAPACITY).
 * *chosen (may be NULL) receives the settings kept, *ms_per_step (may be NULL)
 * their time per step.  Synchronises. */
typedef struct {
    int32_t compact_every;
    int32_t particle_kernel;
    int32_t batch_waves;
    int32_t batch_min_share;
} slpic_tuning;

int slpic_get_tuning(slpic_t *h, slpic_tuning *out);
int slpic_set_tuning(slpic_t *h, const slpic_tuning *t);
int slpic_autotune(slpic_t *h, int32_t steps_per_trial, slpic_tuning *chosen, double *ms_per_step);

/* ---- a speed limit that changes in time or space (Sec. II; the Summary) ----- */

/* Change the speed limit v0 of a speed-limited species from the next step on
 * (the paper notes that v0 may vary in time, e.g. raised mid-run to tighten or
 * verify the approximation).  dt * v0 <= dx must still hold (SLPIC_ERR_CFL:
 * lower the timestep first).  The particles, their g-weights and the current
 * fields are kept; their physical weight w beta follows the new beta from the
 * next deposit on.  SLPIC_ERR_INVALID for a beta == 1 species or v0 <= 0.  On a
 * batch handle, `instance` selects the member. */
int slpic_set_speed_limit(slpic_t *h, int instance, int species, double v0);

/* Test-particle mode (Sec. V): from now on the field is the prescribed wave
 * phi(x, t) = phi0(t) sin(k (x - vphi t)), phi0(t) = phi0 min(1, t / t_ramp)
 * (t = step * dt; t_ramp = 0: no ramp), and E = -dphi/dx is evaluated at the
 * nodes for each time level; the particles' charge is still deposited but no
 * longer enters E.  Periodic grids only; k = 0 returns to the Poisson field from
 * the next step.  E of the current level is recomputed at once.  Not available
 * on a batch handle. */
int slpic_set_wave(slpic_t *h, double phi0, double k, double vphi, double t_ramp);

/* Change the timestep from the next step on, with the CFL checks of
 * slpic_create.  The stored velocities are taken as v^{n+1/2} of the new step
 * (the usual first-order restart of a leapfrog); the wall source's rate per step
 * follows dt.  With a speed-limit profile, dt * v0 * (its largest factor) <= dx.
 * Not available on a batch handle. */
int slpic_set_timestep(slpic_t *h, double dt);

/* A speed limit that varies in space (Sec. II: beta, and so v0, may depend on
 * position, e.g. on a grid whose spacing varies).  lambda: n_cells factors
 * (host, FP64, copied; converted to FP32, each finite and > 0 there), one per
 * cell, shared by the species: a speed-limited species s in cell c has the limit
 * v0_s * lambda_c, the FP32 product of its FP32 v0 and factor rounded to
 * nearest.  The push of a step (the integral of beta and the move) takes the
 * limit of the cell the particle starts the step in, where E is gathered; every
 * deposit (the particle step's, the loaded state's, the source's) takes the limit
 * of the cell the particle is deposited from; the wall source places entering
 * particles with the limit of cell n_cells - 1.  slpic_charge_raw's rule holds
 * with that limit.  lambda == NULL returns to the uniform limit.  Applies from
 * the next step (or prepare); the particles and their g-weights are kept.
 * Errors: SLPIC_ERR_INVALID for a batch handle, n_cells other than the grid's,
 * or a factor that is not finite and > 0; SLPIC_ERR_CFL if dt * v0_s * (largest
 * factor) > dx for a speed-limited species.  Every particle kernel has a
 * variant that reads the profile (compiled apart, so that the uniform limit
 * pays nothing for it); results do not depend on which kernel runs. */
int slpic_set_speed_limit_profile(slpic_t *h, const double *lambda, int n_cells);

/* ---- allocation-free particle step ------------------------------------------ */

/* The paper has no counterpart to this entry point; it exists for callers that
 * must not allocate device memory: code running inside another framework's step
 * loop whose memory pool owns the device, services that reserve all memory at
 * start-up, and loops that cannot afford the device synchronisation that
 * cudaMalloc/cudaFree may cause.  It needs no handle and calls no allocator.
 *
 * One particle step of one species of *cfg (gather, push, move, walls, deposit,
 * compaction: the same per-particle arithmetic as slpic_step's particle kernel),
 * on device arrays owned by the caller, on `stream` (a cudaStream_t; NULL = the
 * legacy default stream):
 *   cell_in[n] (int32), state_in[4n] (float32 {offset, vx, vy, vz} per particle,
 *   16-byte aligned): the particles at time level n;
 *   E[nodes] (float32): the nodal field they gather;
 *   cell_out[n], state_out[4n]: receive the survivors, compacted (order not kept);
 *   charge_out[nodes] (int64, device): receives the fixed-point deposit of the
 *   survivors, the rule of slpic_charge_raw (overwritten, not accumulated);
 *   *n_out (host): survivors; absorbed[2] (host): losses at x=0 and x=L.
 * nodes = n_cells + 1 (Dirichlet) or n_cells (periodic).  The call waits for its
 * work on `stream` to finish before it returns.
 *
 * Every input particle must have 0 <= cell < n_cells and 0 <= offset < 1; one that
 * does not is skipped (neither deposited nor written out) and the call returns
 * SLPIC_ERR_INVALID after completing the step for the others.  The output arrays
 * must not overlap the input arrays (SLPIC_ERR_INVALID): survivors are packed
 * across thread blocks, so an overlap could overwrite particles not yet read.
 *
 * Its only scratch (four counters and the int64 accumulator) is a fixed array in
 * device memory that every GPU loading the library holds until exit; grids of
 * more than 16384 nodes return SLPIC_ERR_CAPACITY.  The first call on a device
 * also looks up that array's device address and sets the kernel's shared-memory
 * limit.  All calls share the array; each call clears what it uses, so calls
 * that overlap on the GPU (concurrent streams or threads) race and must be
 * serialised by the caller.  Returns SLPIC_ERR_INVALID for bad arguments,
 * misaligned or overlapping arrays, or skipped particles, SLPIC_ERR_CFL if
 * dt * v0 > dx, SLPIC_ERR_CUDA on a runtime error. */
int slpic_particle_step_noalloc(const slpic_config *cfg, int species, int64_t n,
                                const int32_t *cell_in, const float *state_in, const float *E,
                                int32_t *cell_out, float *state_out, int64_t *charge_out,
                                int64_t *n_out, int64_t *absorbed, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SLPIC_H */

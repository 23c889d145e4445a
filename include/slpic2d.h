/*
 * slpic2d.h -- C ABI of the 2D (2D3V) speed-limited PIC path.
 *
 * The same method as slpic.h (Appendix A, Eq. (slpicIntegration) of Werner
 * et al., arXiv 1511.08225) on a rectangular grid of nx x ny square cells of
 * side dx: periodic in x, absorbing plates at fixed potential in y (the Sec. IV
 * walls turned into planes), bilinear (2D cloud-in-cell) gather and deposit,
 * and the 5-point Poisson equation of Eq. (LimPtclDynAppendixDotE) solved each
 * step by Jacobi-preconditioned conjugate gradients (the paper names no 2D
 * solver; CG is the reading taken here) to a relative residual
 * ||b - A phi||_2 / ||b||_2 <= cg_rtol, warm-started from the previous step's
 * potential.
 *
 * Grid: nodes (i, j), i = 0..nx-1 (node nx is node 0), j = 0..ny; node (i, j)
 * is entry j*nx + i of every nodal array (rho, phi, Ex, Ey, charge).  The
 * plates are rows j = 0 (phi_lo) and j = ny (phi_hi).
 * Particles: cell = cy*nx + cx (int32), offsets (ox, oy) in [0,1) (FP32),
 * velocity (vx, vy, vz) (FP32); position ((cx + ox) dx, (cy + oy) dx).
 *
 * Deposit precision: int64 fixed point, 2^40 per unit of beta, with the 2D
 * quantised rule (bit-exact across implementations that agree on the FP32
 * particle state; every FP32 operation rounded to nearest, none fused):
 *   beta as in slpic_charge_raw;  bx = beta*ox,  by = beta*oy,  bxy = bx*oy;
 *   qT = rint(beta 2^40), qX = rint(bx 2^40), qY = rint(by 2^40),
 *   qXY = rint(bxy 2^40);
 *   node (cx+1, cy+1) += qXY, (cx+1, cy) += qX - qXY, (cx, cy+1) += qY - qXY,
 *   (cx, cy) += qT - qX - qY + qXY            (the four sum to qT).
 * rho_ij = sum_s q_s w_s / dx^2 * acc_s[ij] * 2^-40.
 *
 * General rules (return codes, handle ownership, host/device arrays,
 * asynchrony) are those stated at the top of slpic.h.
 */
#ifndef SLPIC2D_H
#define SLPIC2D_H

#include "slpic.h"
#include "slpic_unet.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t nx, ny;          /* cells in x (periodic) and in y (between the plates)   */
    double dx;               /* cell side                                             */
    double dt;               /* timestep; dt * v0_s <= dx required (SLPIC_ERR_CFL)     */
    double phi_lo, phi_hi;   /* plate potentials at y = 0 and y = ny dx               */
    double eps0;             /* permittivity                                          */
    double max_speed;        /* SLPIC_BETA_ONE species: caller's bound on |v| (0 = unchecked) */
    uint64_t seed;           /* source random stream                                  */
    int32_t n_species;       /* 1..SLPIC_MAX_SPECIES                                  */
    int32_t src_mode;        /* SLPIC_SRC_*                                           */
    int32_t src_ref_species; /* LOSS_MATCHED: species whose losses are re-injected    */
    int32_t cg_maxit;        /* iteration cap per solve (SLPIC_ERR_NOCONVERGE beyond) */
    double src_lo_cells;     /* source band in y: start, in cells                     */
    double src_len_cells;    /* source band in y: length, in cells (x: whole period)  */
    double src_rate;         /* RATE: physical pairs per unit time                    */
    double cg_rtol;          /* relative residual target of each solve (e.g. 1e-8)    */
    slpic_species species[SLPIC_MAX_SPECIES];
    int32_t solver;          /* SLPIC2D_SOLVER_CG (default) or SLPIC2D_SOLVER_FFT      */
    int32_t reserved;        /* 0                                                     */
} slpic2d_config;

/* Field solvers.  Both solve the same 5-point system exactly as stated above.
 *   SLPIC2D_SOLVER_CG   Jacobi-preconditioned CG to ||b - A phi|| <= cg_rtol ||b||
 *                       (FP32 iterates, FP64 reliable updates), warm-started
 *                       (slpic2d_set_warm_start).
 *   SLPIC2D_SOLVER_FFT  direct: the system is separable (periodic x, Dirichlet y),
 *                       so a discrete Fourier transform along x (radix-2, FP64;
 *                       nx a power of two, 2..8192) turns it into one tridiagonal
 *                       system along y per mode, (4 - 2 cos(2 pi k/nx)) u_j -
 *                       u_{j-1} - u_{j+1} = b^_j, solved by the Thomas algorithm
 *                       (its multipliers depend on the grid only and are tabulated
 *                       at creation), then transformed back.  No iterations; the
 *                       true relative residual (~1e-15) is still formed, reported
 *                       and held to cg_rtol. */
#define SLPIC2D_SOLVER_CG 0
#define SLPIC2D_SOLVER_FFT 1

typedef struct {
    int64_t step;
    double time;
    int64_t count[SLPIC_MAX_SPECIES];       /* live macroparticles                      */
    int64_t absorbed[SLPIC_MAX_SPECIES][2]; /* cumulative, at y = 0 / y = Ly            */
    int64_t injected[SLPIC_MAX_SPECIES];    /* cumulative                               */
    int32_t cg_iterations;                  /* iterations of the last solve             */
    int32_t iterative_last;                 /* pushes of the last step that took the
                                               piece walk (all species)                 */
    int64_t cg_iterations_total;            /* over every solve since creation          */
    double cg_rel_residual;                 /* ||b - A phi|| / ||b|| after the last solve */
} slpic2d_diag;

typedef struct slpic2d_sim slpic2d_t;

/* Validate *cfg (nx >= 2, ny >= 2, dx > 0, dt > 0, 0 < cg_rtol < 1,
 * cg_maxit > 0, species as in slpic_create, CFL as in slpic_create) and
 * allocate on the current device: 2 x capacity particle slots per species
 * (24 bytes each), nodal int64 deposits, and the FP64 CG vectors.
 * *out is set only on success; slpic_create_error() explains a failure. */
int slpic2d_create(const slpic2d_config *cfg, slpic2d_t **out);
int slpic2d_destroy(slpic2d_t *h);
const char *slpic2d_last_error(const slpic2d_t *h);
/* Run subsequent work on this CUDA stream (cudaStream_t cast to void*; NULL =
 * the legacy default stream). */
int slpic2d_set_stream(slpic2d_t *h, void *stream);

/* Append n particles of species s from host arrays: cell[n] (cy*nx + cx),
 * offset[2n] interleaved (ox, oy) in [0,1), v[3n] interleaved (vx, vy, vz),
 * the velocity being v^{-1/2}.  Checks every particle (SLPIC_ERR_INVALID)
 * and the capacity (SLPIC_ERR_CAPACITY) before anything is stored. */
int slpic2d_load_particles(slpic2d_t *h, int s, int64_t n, const int32_t *cell,
                           const float *offset, const float *v);

/* Deposit rho^0 from the loaded particles (beta of v^{-1/2}) and solve for
 * phi^0, E^0.  Required once after loading, before slpic2d_step. */
int slpic2d_prepare(slpic2d_t *h);

/* Advance nsteps steps of Appendix A (per step: gather/push/move/absorb and
 * deposit of rho^{n+1}; source injection; CG solve; E^{n+1}).  Asynchronous;
 * the status of earlier device work is returned. */
int slpic2d_step(slpic2d_t *h, int64_t nsteps);
int slpic2d_synchronize(slpic2d_t *h);

/* Current fields, host arrays of (ny+1)*nx entries; any pointer may be NULL. */
int slpic2d_fields(slpic2d_t *h, double *rho, double *phi, float *Ex, float *Ey);
/* The int64 deposit of species s for the current time level ((ny+1)*nx). */
int slpic2d_charge_raw(slpic2d_t *h, int s, int64_t *acc);
int slpic2d_particle_count(slpic2d_t *h, int s, int64_t *n);
/* Copy out species s (capacity *n on entry, count on return).  Order: by cell
 * after slpic2d_prepare and after every compacting step (every 16th), when the
 * particles are sorted by cell (a counting sort; holes dropped); in between, each
 * particle keeps its slot; within a cell the order is arbitrary. */
int slpic2d_get_particles(slpic2d_t *h, int s, int32_t *cell, float *offset, float *v,
                          int64_t *n);
int slpic2d_diagnostics(slpic2d_t *h, slpic2d_diag *out);

/* Kernel timing: with on != 0, every following step (up to 4096) records CUDA
 * events on the handle's stream around its three kernels; slpic2d_kernel_times
 * synchronises and returns the mean per-step time (ms) of the particle kernel,
 * the source kernel and the CG field kernel over the recorded steps (*steps of
 * them), then starts a new recording. */
int slpic2d_enable_kernel_timing(slpic2d_t *h, int on);
int slpic2d_kernel_times(slpic2d_t *h, double *particle_ms, double *inject_ms, double *field_ms,
                         int64_t *steps);

/* The field solve alone, for a given charge density: rho and phi host arrays
 * of (ny+1)*nx entries (phi's rows 0 and ny are set to the plate potentials,
 * its other rows are the initial guess on entry and the solution on return).
 * Same CG kernel and tolerance as slpic2d_step; *iterations and *rel_residual
 * (may be NULL) report the solve.  Leaves the simulation's own fields alone. */
int slpic2d_solve_poisson(slpic2d_t *h, const double *rho, double *phi, int32_t *iterations,
                          double *rel_residual);

/* Initial guess of the CG in each following slpic2d_step (the answer is the same
 * to cg_rtol whatever the guess; the iterations it takes are not):
 *   SLPIC2D_WARM_PREV  the potential of the previous step (the default);
 *   SLPIC2D_WARM_ZERO  the straight line between the plate potentials;
 *   SLPIC2D_WARM_UNET  that line plus net(rho), rho the step's charge density on
 *                      rows 0..ny-1 (row 0 set to 0) as an (H, W) = (ny, nx)
 *                      FP32 image (slpic_unet.h), net's output taken on the
 *                      interior rows 1..ny-1;
 *   SLPIC2D_WARM_UNET_DELTA  the previous step's potential plus
 *                      net(rho - rho_prev), rho_prev the image of the step
 *                      before, for a network trained on the changes between
 *                      consecutive steps (the first step after this call or
 *                      slpic2d_prepare has no rho_prev and takes the previous
 *                      potential alone).
 * net: required for the two network modes (grid (ny, nx), max_batch >= 1),
 * ignored otherwise.  It is borrowed: it must outlive its use, and is run on this
 * handle's stream, so it must not be used on another stream meanwhile.  The
 * network's time counts in the field time of slpic2d_kernel_times. */
#define SLPIC2D_WARM_PREV 0
#define SLPIC2D_WARM_ZERO 1
#define SLPIC2D_WARM_UNET 2
#define SLPIC2D_WARM_UNET_DELTA 3
int slpic2d_set_warm_start(slpic2d_t *h, int32_t mode, slpic_unet_t *net);

#ifdef __cplusplus
}
#endif

#endif

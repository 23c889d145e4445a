/*
 * slpic_fp64.h -- the plain FP64 form of the 1D speed-limited PIC step.
 *
 * The same method and problem as slpic.h (Appendix A, Eq. (slpicIntegration) of
 * Werner et al., arXiv 1511.08225; configuration by slpic_config), written the
 * plain way: positions x and velocities v in FP64 (32 bytes per macroparticle),
 * the velocity push solved in FP64 (closed-form time along the velocity line,
 * inverted by safeguarded Newton), an FP64 cloud-in-cell deposit with
 * floating-point atomics (order-dependent in the last bits), the Poisson solve
 * in FP64, and the survivors packed every step.  It is the reference point the
 * mixed-precision library is measured against, and shares its problem
 * statement, source rule and random stream (SplitMix64 counters; Box-Muller in
 * FP64), not its arithmetic.
 *
 * Rules for return codes, handles and asynchrony are those of slpic.h.
 */
#ifndef SLPIC_FP64_H
#define SLPIC_FP64_H

#include "slpic.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slpic_fp64_sim slpic_fp64_t;

/* Validate *cfg as slpic_create does and allocate 2 x capacity FP64 particle
 * slots per species. */
int slpic_fp64_create(const slpic_config *cfg, slpic_fp64_t **out);
int slpic_fp64_destroy(slpic_fp64_t *h);
const char *slpic_fp64_last_error(const slpic_fp64_t *h);
int slpic_fp64_set_stream(slpic_fp64_t *h, void *stream);

/* Append n particles of species s: x[n] (0 <= x < L), v[3n] = v^{-1/2}.
 * SLPIC_ERR_INVALID / SLPIC_ERR_CAPACITY as in slpic_load_particles. */
int slpic_fp64_load_particles(slpic_fp64_t *h, int s, int64_t n, const double *x,
                              const double *v);
/* Deposit rho^0 and solve E^0 (after loading). */
int slpic_fp64_prepare(slpic_fp64_t *h);
/* nsteps steps: push/move/walls/deposit, source, field solve.  Asynchronous. */
int slpic_fp64_step(slpic_fp64_t *h, int64_t nsteps);
int slpic_fp64_synchronize(slpic_fp64_t *h);
/* Nodal rho, phi, E (host arrays of N+1 (Dirichlet) or N (periodic) entries;
 * any may be NULL). */
int slpic_fp64_fields(slpic_fp64_t *h, double *rho, double *phi, double *E);
int slpic_fp64_particle_count(slpic_fp64_t *h, int s, int64_t *n);
/* Copy out species s: x[cap], v[3 cap]; *n = count (SLPIC_ERR_CAPACITY if
 * cap is too small). */
int slpic_fp64_get_particles(slpic_fp64_t *h, int s, int64_t cap, double *x, double *v,
                             int64_t *n);

#ifdef __cplusplus
}
#endif

#endif

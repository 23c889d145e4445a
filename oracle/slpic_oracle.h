/*
 * slpic_oracle.h -- declarations of the FP64 CPU oracle (test infrastructure).
 *
 * This header belongs to the oracle alone.  The CUDA library has its own
 * public header and never includes this one; the two implementations share
 * no code.  Citations are to Werner et al., arXiv 1511.08225.
 */
#ifndef SLPIC_ORACLE_H
#define SLPIC_ORACLE_H

#include <stdint.h>

enum { ORC_BETA_ONE = 0, ORC_BETA_HEAVISIDE = 1, ORC_BETA_RELATIVISTIC = 2 };

/* Sec. II, Eqs. (relativisticBeta), (heavisideBeta) */
double orc_beta(int kind, double r, double v0);

/* Appendix A, Eq. (slpicIntegrationV): tau* = int beta(|v(t)|) dt over one step */
double orc_beta_integral(int kind, const double u[3], const double a[3], double dt,
                         double v0);
/* the paper's modified-midpoint evaluation, doubling substeps until rel_tol */
double orc_beta_integral_mmid(int kind, const double u[3], const double a[3], double dt,
                              double v0, double rel_tol, long *n_used);
/* pins: closed-form time along the velocity line, and brute-force RK4 */
double orc_time_closed(int kind, const double u[3], const double a[3], double v0,
                       double tau);
double orc_beta_integral_closed(int kind, const double u[3], const double a[3], double dt,
                                double v0);
void orc_rk4_limited(int kind, const double u[3], const double a[3], double dt, double v0,
                     long n_sub, double out[7]);

/* Appendix A, Eq. (LimPtclDynAppendixDotE), 1D nodal Poisson */
void orc_poisson1d_dirichlet(int n_cells, double dx, double eps0, const double *rho,
                             double phi_lo, double phi_hi, double *phi);
void orc_poisson1d_periodic(int n_cells, double dx, double eps0, const double *rho,
                            double *phi);
void orc_efield1d(int n_cells, int periodic, double dx, const double *phi, double *E);

/* Appendix A charge assignment (FP64) and the quantised FP32 -> int64 rule */
void orc_deposit1d(int n_cells, int periodic, double dx, long n, const double *x,
                   const double *v, const uint8_t *alive, int kind, double v0,
                   const double *lam, double w, double *dens);
float orc_beta_f32(int kind, float vx, float vy, float vz, float v0);
void orc_deposit_q40(int n_cells, int periodic, long n, const int32_t *cell,
                     const float *offset, const float *v, int kind, float v0,
                     const float *lam, int64_t *acc);

/* Appendix A gather/push/move with Sec. IV walls; lam (per-cell factors of  */
/* v0, Sec. II: the limit may vary in space) or NULL in all three            */
void orc_push1d(int n_cells, int periodic, double dx, double dt, const double *E, long n,
                double *x, double *v, uint8_t *alive, double qm, int kind, double v0,
                const double *lam, long *flux);

/* counter-based SplitMix64 and the volume source */
uint64_t orc_splitmix64_at(uint64_t key, uint64_t i);
uint64_t orc_stream_key(uint64_t seed, uint64_t step, uint32_t species);
float orc_u24(uint64_t z);
void orc_inject(uint64_t seed, uint64_t step, uint32_t species, long n_new,
                float src_lo_cells, float src_len_cells, double dx, double vth,
                double *x, double *v);

/* 2D: periodic x, plates in y; node (i, j) at j*nx + i, j = 0..ny */
void orc_poisson2d_direct(int nx, int ny, double dx, double eps0, const double *rho,
                          double phi_lo, double phi_hi, double *phi);
int orc_poisson2d_cg(int nx, int ny, double dx, double eps0, const double *rho,
                     double phi_lo, double phi_hi, double rtol, int maxit, double *phi,
                     double *rel_res);
void orc_efield2d(int nx, int ny, double dx, const double *phi, double *Ex, double *Ey);
void orc_deposit2d(int nx, int ny, double dx, long n, const double *x, const double *y,
                   const double *v, const uint8_t *alive, int kind, double v0, double w,
                   double *dens);
void orc_deposit2d_q40(int nx, int ny, long n, const int32_t *cell, const float *offset,
                       const float *v, int kind, float v0, int64_t *acc);
void orc_push2d(int nx, int ny, double dx, double dt, const double *Ex, const double *Ey,
                long n, double *x, double *y, double *v, uint8_t *alive, double qm, int kind,
                double v0, long *flux);
void orc_inject_wall(uint64_t seed, uint64_t step, uint32_t species, long n_new, int n_cells,
                     double dx, double dt, double vth, int kind, double v0, double *x,
                     double *v);
void orc_inject2d(uint64_t seed, uint64_t step, uint32_t species, long n_new,
                  float src_lo_cells, float src_len_cells, int nx, double dx, double vth,
                  double *x, double *y, double *v);

#endif

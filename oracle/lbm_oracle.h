/*
 * lbm_oracle.h -- plain FP64 CPU oracle of the D2Q9 lattice Boltzmann hot path
 * of Basagaoglu, Harwell, Nguyen & Succi, "Enhanced computational performance
 * of the lattice Boltzmann model for simulating micron- and submicron-size
 * particle flows and non-Newtonian fluid flows" (arXiv:2006.12910).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against the paper.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may build, load or call it.  It shares no source with
 * the CUDA library (no headers, tables or helpers in common).
 *
 * Everything is double precision, written as plain nested loops in the order
 * the paper states the method, one function per equation:
 *   Sec. 2, Eqs. (e.LB1)-(e.LB2): D2Q9 BGK with velocity-shift body force
 *   Sec. 3, Eqs. (MP1)-(MP8):     Ladd moving bounce-back, momentum-exchange
 *                                 force, covered/uncovered nodes, LJ repulsion,
 *                                 Newton-Euler particle update
 *   Sec. 4, Eqs. (NP1)-(NP2), Table 1: fluctuating LB noise on modes 3..8
 *   Sec. 5, Eqs. (nn1)-(nn5):     power-law local relaxation time
 *
 * State convention: the stored populations are the POST-collision values
 * f*(x,t) (the populations about to stream).  One oracle step computes the
 * particle forces at t from f*(t), advances the particle velocities (Eqs.
 * MP5-MP6, with the boundary velocity of the link exchange taken at mid-step,
 * see or_newton_euler), streams with bounce-back (t -> t+1) using that same
 * mid-step boundary velocity in Eqs. MP7-MP8, applies the inlet/outlet
 * columns, collides at t+1 (adding noise) and re-rasterises the particles at
 * their new positions.  Over n steps this is the paper's collide-then-stream
 * sequence shifted by half a step.
 *
 * Population layout of every array crossing this interface: f[q][y][x],
 * x fastest, q = 0..8 in the paper's order (Sec. 2): e0=(0,0), e1..e4 axis
 * vectors (1,0),(0,1),(-1,0),(0,-1), e5..e8 diagonals (1,1),(-1,1),(-1,-1),(1,-1).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t nx, ny;
    int32_t periodic_x, periodic_y, walls_y, inlet_outlet;
    double tau, rho0, gx, gy;
    double rho_in, rho_out;        /* Zou-He density columns when inlet_outlet */
    double kT;                     /* 0 disables the noise of Sec. 4 */
    uint64_t seed;
    uint32_t domain_id;            /* fourth Philox counter word */
    int32_t power_law;             /* 1 enables Sec. 5 */
    double n_pl, xi_pl, tau_min, tau_max;
    double lj_psi, lj_rit;         /* Eq. (MP2) stiffness and threshold */
    double kappa_pl;               /* kappa of Eq. (nn4); 0 means 2^(n-1) */
} or_params;

typedef struct {
    double x, y, R, rho_p, U, V, Omega, theta;
    int32_t fixed;                 /* 1: position and velocity are held */
    int32_t pad_;
} or_particle;

/* Per-particle diagnostics of the most recent step, in this order:
 * F_links(x,y), T_links, F_cu(x,y), T_cu, F_lj(x,y), T_lj,
 * n_covered, n_uncovered, mass_covered, mass_uncovered. */
#define OR_DIAG_N 13

typedef struct or_domain or_domain;

or_domain* or_create(const or_params* p);
void or_destroy(or_domain* d);
int  or_set_solid(or_domain* d, const uint8_t* solid);          /* ny*nx, 1 = solid */
int  or_add_particles(or_domain* d, int n, const or_particle* p);
void or_init_equilibrium(or_domain* d, double rho, double ux, double uy);
int  or_set_populations(or_domain* d, const double* f);         /* [9][ny][nx] */
void or_get_populations(const or_domain* d, double* f);
void or_step(or_domain* d, int64_t nsteps);
int64_t or_step_count(const or_domain* d);
void or_moments(const or_domain* d, double* rho, double* ux, double* uy);
int  or_get_particles(const or_domain* d, or_particle* out, int cap);
void or_particle_diag(const or_domain* d, int p, double* out);  /* OR_DIAG_N values */
void or_checks(const or_domain* d, double* out3);               /* mass, px, py */
void or_exterior_momentum(const or_domain* d, double* out2);    /* sum of j* over fluid outside particles */
int  or_links(const or_domain* d, int p, int32_t* node, int32_t* dir, int cap);
void or_owner(const or_domain* d, int32_t* out);                /* ny*nx, 0 or particle+1 */
void or_set_threads(int n);

/* Building blocks exposed for the pin tests. */
void   or_lattice(int32_t* e, double* w, int32_t* opp);          /* e[9][2], w[9], opp[9] */
void   or_basis(double* chi, double* wk);                        /* chi[9 modes][9 dirs], wk[9] */
void   or_feq(double rho, double ux, double uy, double* out9);
double or_solve_tau(double A, double n, double xi, double tmin, double tmax);
double or_strain_A(const double* f9, double rho, double jx, double jy);
void   or_collide_node(const or_params* p, const double* f9, double* out9,
                       uint32_t node, uint32_t step);
void   or_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out);
void   or_thetas(uint64_t seed, uint32_t node, uint32_t step, uint32_t domain, double* theta6);
void   or_noise(double rho, double kT, double omega, const double* theta6, double* zeta9);
/* Eqs. (MP5)-(MP6) with the mid-step boundary velocity: F = (Fx, Fy, T) the
 * force and torque that do not depend on the particle's motion, Z[6] the upper
 * triangle (xx xy xO yy yO OO) of the link friction matrix; returns the
 * mid-step (U, V, Omega) in xmid[3]. */
void   or_newton_euler(or_particle* p, const double* F, const double* Z,
                       double gx, double gy, double rho0, double* xmid);
void   or_lj_pair_force(double ax, double ay, double bx, double by,
                        double psi, double rit, double* F2);

#ifdef __cplusplus
}
#endif
#endif

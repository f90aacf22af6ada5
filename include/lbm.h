/*
 * lbm.h -- C ABI of the GB300 D2Q9 lattice Boltzmann library.
 *
 * What it computes: the per-timestep hot path of the 2-D lattice Boltzmann
 * model of arXiv:2006.12910 (Basagaoglu, Harwell, Nguyen & Succi):
 *   - D2Q9 single-relaxation BGK with a velocity-shift body force
 *     (Sec. 2, Eqs. e.LB1, e.LB2, rho u = sum f e + tau rho g);
 *   - halfway bounce-back at walls and stationary obstacles (Sec. 3);
 *   - Ladd moving bounce-back on circular particles with the momentum-exchange
 *     force, covered/uncovered-node force, LJ-type repulsion and a Newton-Euler
 *     update (Sec. 3, Eqs. MP1-MP8);
 *   - fluctuating-LB thermal noise on modes 3..8 (Sec. 4, Eqs. NP1-NP2,
 *     Table 1), from a counter-based Philox4x32-10 stream keyed on
 *     (seed, node, step, draw, domain) so that no random state is stored;
 *   - a local power-law relaxation time tau* (Sec. 5, Eqs. nn1-nn5);
 *   - Zou-He density columns at the x ends (an addition: the paper's
 *     benchmark 1 uses periodic ends with a body force).
 * Every step runs in hand-written CUDA kernels for sm_103a; there is no CPU
 * fallback.  All device memory is owned by the context.
 *
 * Conventions for every call:
 *   - Return value: LBM_OK (0) or a negative LBM_E_* code; no exception ever
 *     crosses this interface.  lbm_last_error() gives a one-line reason.
 *   - Host arrays passed in are copied before the call returns; output arrays
 *     are allocated by the caller.
 *   - Field layout on the host: x fastest, rows of nx values, ny rows
 *     (index y*nx + x); populations as [9][ny][nx] with the paper's velocity
 *     order e0=(0,0), e1..e4 = (1,0),(0,1),(-1,0),(0,-1),
 *     e5..e8 = (1,1),(-1,1),(-1,-1),(1,-1) (Sec. 2).
 *   - The stored state is the POST-collision populations f*(t): one step
 *     streams them with bounce-back and collides (the paper's collide-then-
 *     stream sequence shifted by half a step).
 *   - lbm_step enqueues work on the context's stream and returns; errors that
 *     arise on the device (instability, particle overlap, a bounded wait
 *     running out) are reported by the next blocking call.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_E_INVAL (-1)    /* bad argument or parameter */
#define LBM_E_NOMEM (-2)    /* device or pinned allocation failed */
#define LBM_E_CUDA (-3)     /* a CUDA runtime call failed */
#define LBM_E_UNSTABLE (-4) /* NaN / Inf or rho <= 0 seen on the lattice */
#define LBM_E_TIMEOUT (-5)  /* a bounded device-side wait ran out */
#define LBM_E_STATE (-6)    /* call order, particle overlap or list capacity */
#define LBM_E_IO (-7)       /* checkpoint file error */

/* Population storage.  F64 stores f and computes in FP64 (the plain FP64
 * path).  Every other kind computes in FP32 registers: F32 stores f, the
 * shifted kinds store (f_i - omega_i rho0) * store_scale. */
typedef enum {
    LBM_F64 = 0,
    LBM_F32 = 1,
    LBM_F32S = 2,
    LBM_F16S = 3,
    LBM_BF16S = 4
} lbm_store;

/* One lattice domain.  Lattice units, dx = dt = 1 (Sec. 6). */
typedef struct {
    int32_t nx, ny;            /* nodes; nx, ny >= 3 */
    int32_t periodic_x;        /* exactly one of periodic_x / inlet_outlet */
    int32_t periodic_y;        /* exactly one of periodic_y / walls_y */
    int32_t walls_y;           /* halfway walls at y = -1/2 and y = ny - 1/2 */
    int32_t inlet_outlet;      /* Zou-He density columns at x = 0 and x = nx-1 */
    double tau;                /* BGK relaxation time (> 1/2); nu = (tau - 1/2)/3 */
    double rho0;               /* reference density (rest state, particle links) */
    double gx, gy;             /* body-force acceleration g (Sec. 2) */
    double rho_in, rho_out;    /* densities of the open columns */
    double kT;                 /* thermal energy of Eq. NP2; 0 disables noise */
    uint64_t seed;             /* Philox key */
    uint32_t domain_id;        /* fourth Philox counter word */
    int32_t power_law;         /* 1: tau* of Sec. 5 replaces tau */
    double n_pl, xi_pl;        /* power-law index n and consistency xi (Eq. nn1) */
    double tau_min, tau_max;   /* clamp of tau* */
    double lj_psi, lj_rit;     /* Eq. MP2 stiffness psi and threshold |r_it| */
    int32_t store;             /* lbm_store; must be the same for every domain */
    int32_t max_particles;     /* capacity reserved for lbm_add_particles */
    double store_scale;        /* power-of-two scale of the shifted FP16/BF16 store */
    double kappa_pl;           /* kappa of Eq. nn4 (Sec. 5 cites 0.5^(n-1), 1 and 2^(n-1));
                                  0 takes 2^(n-1), the value the paper adopts */
} lbm_params;

/* A rigid circular particle (Sec. 3).  Position in lattice units with node
 * (x, y) at integer coordinates; velocity U, V; angular velocity Omega;
 * orientation theta.  fixed = 1 holds position and velocity. */
typedef struct {
    double x, y, R, rho_p, U, V, Omega, theta;
    int32_t fixed;
    int32_t pad_;
} lbm_particle;

typedef struct lbm_ctx lbm_ctx;

/* Create a context for one domain (Sec. 2 parameters), allocate its device
 * memory and set the state to the rest equilibrium f* = omega_i rho0.
 * cuda_stream: a cudaStream_t the context enqueues on (NULL: the context
 * creates its own).  On success *out owns everything until lbm_destroy. */
int lbm_create(const lbm_params* p, void* cuda_stream, lbm_ctx** out);

/* Create a context holding ndom independent domains of uneven size that
 * advance together (one stream-and-collide launch per step over a work list
 * covering all domains).  per_domain[d] describes domain d; store must agree. */
int lbm_create_ensemble(int ndom, const lbm_params* per_domain, void* cuda_stream, lbm_ctx** out);

/* Stationary solid nodes of domain dom (Sec. 3 "inline obstacles"):
 * solid[y*nx + x] != 0 marks a solid node.  Copied.  Solid nodes hold no
 * populations; their neighbours bounce back halfway.  Must precede
 * lbm_add_particles. */
int lbm_set_geometry(lbm_ctx* ctx, int dom, const uint8_t* solid);

/* Add n particles to domain dom (copied) and rasterise them (Sec. 3, Fig. 1:
 * a node belongs to a particle when strictly inside its disk).  Particles
 * must not overlap each other.  Total per domain <= max_particles. */
int lbm_add_particles(lbm_ctx* ctx, int dom, int n, const lbm_particle* p);

/* Replace the populations f*(t) of domain dom with host FP64 values
 * f[9][ny][nx] (converted to the store type; solid nodes ignored).  It first
 * waits for the queued steps and clears the context's sticky device error
 * word (LBM_E_UNSTABLE, LBM_E_TIMEOUT, LBM_E_STATE of earlier steps, for every
 * domain): the caller starts again from a known state.  Call lbm_sync before
 * it to see such an error. */
int lbm_set_populations(lbm_ctx* ctx, int dom, const double* f);

/* Read the populations f*(t) of domain dom into host FP64 f[9][ny][nx]
 * (solid nodes read as 0).  Blocking. */
int lbm_get_populations(lbm_ctx* ctx, int dom, double* f);

/* Advance every domain by nsteps timesteps (Eqs. e.LB1, MP1-MP8, NP1-NP2,
 * nn5 per step).  Enqueued on the context stream (replayed as CUDA graphs:
 * one graph of exactly nsteps steps when lbm_prepare_steps prepared that
 * count, else one graph per binary digit of nsteps, up to 64 steps each);
 * returns without waiting. */
int lbm_step(lbm_ctx* ctx, int64_t nsteps);

/* Per-step particle trajectories without a host round trip per step (the
 * particle velocity and position series behind the Brownian statistics of
 * Sec. 6; no paper counterpart as an interface).  While a buffer is set,
 * every step writes the state of every particle after it, from the particle
 * force launch directly into host_buf (page-locked host memory mapped into
 * the device address space: cudaHostAlloc, or cudaHostRegister with the
 * mapped flag), as record (t mod capacity) for the step count t it reaches:
 * np_slots x 6 doubles (x, y, U, V, Omega, theta), np_slots the sum of
 * max_particles over the domains, domain d's particles from the sum of
 * max_particles of the domains before it; slots beyond a domain's particle
 * count are not written.  A record is complete once a blocking call
 * (lbm_sync, lbm_particles, ...) issued after the step has returned.  The
 * caller keeps the buffer alive and page-locked while it is set;
 * host_buf = NULL stops recording.  Waits for the queued steps; the step
 * graphs are rebuilt at the next step.  LBM_E_INVAL for memory that is not
 * page-locked and mapped, or capacity < 1. */
int lbm_record_particles(lbm_ctx* ctx, double* host_buf, int64_t capacity);

/* Set-up for a step count the caller repeats (no paper counterpart): build
 * the step graphs of exactly nsteps steps (1 .. LBM_PREPARE_MAX_STEPS) from
 * either state parity now, so that every later lbm_step(nsteps) replays one
 * graph.  The chains of particle and stream-collide launches overlap across
 * the steps of one graph but drain at its end, so one graph per call keeps a
 * call of nsteps steps closest to the steady per-step time.  At most
 * LBM_PREPARE_SLOTS counts stay prepared (the oldest is dropped); changes of
 * geometry, particles or launch configuration rebuild them at the next step.
 * Blocking (capture and upload of the graphs); LBM_E_INVAL for a count out
 * of range. */
#define LBM_PREPARE_MAX_STEPS 256
#define LBM_PREPARE_SLOTS 4
int lbm_prepare_steps(lbm_ctx* ctx, int64_t nsteps);

/* Wait for the context stream and report device-side errors. */
int lbm_sync(lbm_ctx* ctx);

/* Density and physical velocity u = (sum f* e - rho g / 2) / rho of domain dom
 * into caller host arrays of ny*nx doubles (solid nodes: 0).  Blocking. */
int lbm_moments(lbm_ctx* ctx, int dom, double* rho, double* ux, double* uy);

/* Same moments as FP32 into caller DEVICE arrays of ny*nx floats on the
 * context stream (for example torch tensors).  Not blocking. */
int lbm_moments_device(lbm_ctx* ctx, int dom, float* d_rho, float* d_ux, float* d_uy);

/* Start an asynchronous copy of the moments of domain dom to pinned host
 * memory on a side stream (output offloading); lbm_moments_async_wait copies
 * them into the caller's host arrays (FP32, ny*nx each). */
int lbm_moments_async(lbm_ctx* ctx, int dom);
int lbm_moments_async_wait(lbm_ctx* ctx, float* rho, float* ux, float* uy);

/* Particle state of domain dom at the current step (up to cap entries).
 * Returns the particle count (>= 0) or an error. Blocking.  After lbm_step it
 * waits only until the step's particle force launch has written the state
 * (the rest of the step keeps running on the device) and copies it through a
 * side stream; device error bits of that step are then reported by the next
 * call that synchronises the whole context (lbm_sync, lbm_moments,
 * lbm_checks, ...).  Otherwise (after set-up, lbm_load or lbm_profile_steps)
 * it synchronises the context stream and reports its error bits. */
int lbm_particles(lbm_ctx* ctx, int dom, lbm_particle* out, int cap);

/* Force and torque terms of the last step for particle i of domain dom, 13
 * doubles: F_links(x,y), T_links (Eq. MP1), F_cu(x,y), T_cu (covered /
 * uncovered nodes), F_lj(x,y), T_lj (Eq. MP2), n_covered, n_uncovered,
 * mass_covered, mass_uncovered.  Blocking. */
int lbm_particle_forces(lbm_ctx* ctx, int dom, int i, double* out13);

/* FP64 global sums over fluid nodes of domain dom: mass sum f*, momentum
 * sum f* e_x, sum f* e_y (deterministic block order).  Blocking. */
int lbm_checks(lbm_ctx* ctx, int dom, double* out3);

/* Steps completed since creation (or since the loaded checkpoint). */
int64_t lbm_step_count(const lbm_ctx* ctx);

/* Checkpoint: populations, particle state, rasterisation and step counter.
 * Because the noise is counter-based, a resumed run is bit-identical.
 * lbm_load replaces the whole state and, like lbm_set_populations, clears the
 * sticky device error word of earlier steps. */
int lbm_save(lbm_ctx* ctx, const char* path);
int lbm_load(lbm_ctx* ctx, const char* path);

/* Pick the stream-and-collide kernel and launch shape (kernel, threads per
 * block and stages as in lbm_set_launch) by short timed trials on the
 * context's own data, among the register-kernel grids 0, 1, 3 and 4 (kernel 3
 * only without particles; the staged kernel 2 is chosen only through
 * lbm_set_launch).  The trials write only the second population arena,
 * which the next step overwrites, so the state and step count are unchanged. */
int lbm_autotune(lbm_ctx* ctx, int trial_steps);

/* Launch configuration of the stream-and-collide kernel (no paper
 * counterpart; it selects among equivalent implementations of Eqs. e.LB1 /
 * e.LB2, all with the same results).  kernel: 0 register-pipelined with one
 * warp item per warp, 1 the same with a grid-stride grid of 16 CTAs' worth of
 * warps per SM, 2 staged through shared memory with bulk asynchronous copies
 * (`stages` row segments in flight per warp, 1..8; block at most 256
 * threads), 3 register kernel on a grid-stride grid of only the CTAs that fit
 * the SMs at once, 4 the same on half the grid of kernel 1 (8 CTAs' worth of
 * warps per SM).  block: threads per CTA, a multiple of 32, at most
 * 128 for kernels 0, 1, 3 and 4.  LBM_E_INVAL for values out of range
 * or a staged configuration whose shared memory does not fit an SM; the
 * previous configuration then stays.  lbm_get_launch writes {kernel, block,
 * stages, grid} to out4. */
int lbm_set_launch(lbm_ctx* ctx, int32_t kernel, int32_t block, int32_t stages);
int lbm_get_launch(const lbm_ctx* ctx, int64_t* out4);

/* Failure detection (no paper counterpart).  Every wait inside a kernel of
 * this library is bounded: the staged stream-and-collide kernel (kernel 2 of
 * lbm_set_launch) waits for its bulk copies at most `ns` nanoseconds of the
 * GPU's global timer per stage (default 1e9), then records LBM_E_TIMEOUT,
 * waits for its copies still in flight (always with the full second, so no
 * copy lands in shared memory it has left) and ends its work; the next
 * blocking call returns LBM_E_TIMEOUT and the populations of that step are
 * not valid (reload them with lbm_set_populations or lbm_load).  ns = 0 makes
 * every stage wait report expiry at once without waiting, which is how the
 * tests exercise this path.  Takes effect from the next lbm_step.
 * LBM_E_INVAL for ns above 60 s. */
int lbm_set_wait_limit(lbm_ctx* ctx, uint64_t ns);

/* Failure injection on the host (no paper counterpart): the nth device
 * allocation that the library makes from now on (any context; creation,
 * particles, staging buffers) fails as it would on an exhausted device, so
 * that the caller sees LBM_E_NOMEM and the library frees whatever it had
 * allocated for that call.  nth = 0 switches the hook off; it also goes off
 * by itself once it has fired.  LBM_E_INVAL for nth < 0. */
int lbm_debug_fail_alloc(int32_t nth);

/* Measurement: advance nsteps timesteps with plain launches in sequence (no
 * graph, no overlap), enqueued back to back in batches of 32 steps with a
 * CUDA-event pair around every kernel on the context stream and one
 * synchronisation per batch; ms_out[0] receives the summed device time of
 * the particle launch of forces, exchange and Newton-Euler, ms_out[1] that
 * of the particle launches of rasterisation, marks and the Eq. MP2 sums
 * (they run beside the stream-collide pass in lbm_step), ms_out[2] that of the
 * stream-and-collide kernel over every work item, and launches_out (if not
 * NULL) the number of kernels launched.  Blocking.  The state advances
 * exactly as with lbm_step. */
int lbm_profile_steps(lbm_ctx* ctx, int64_t nsteps, double* ms_out3, int64_t* launches_out);

/* Measurement of the stream-and-collide kernel alone: nlaunches passes over
 * every work item (the variant without the moments of nodes that change side
 * under a particle), back to back on the context stream, each from the
 * current state into the other population arena, with one CUDA-event pair
 * around them; *ms_out receives their total device time.  The state does not
 * advance (the next step rewrites what the passes wrote: the same values),
 * so the number is the kernel's sustained time per launch in a busy stream.
 * Blocking.  LBM_E_INVAL for nlaunches < 1 or ms_out NULL. */
int lbm_time_stream(lbm_ctx* ctx, int32_t nlaunches, double* ms_out);

/* Measurement of the device's FP64 rate (no paper counterpart; it sets the
 * arithmetic roofline of the FP64 store, whose collision is bound by FP64
 * issue on this part rather than by HBM).  Eight independent FMA chains in
 * every thread of 8 CTAs x 256 threads per SM, timed with CUDA events on
 * cuda_stream (NULL: the default stream), best of three launches after one
 * warm-up; *gflops_out = 2 x FMAs / second / 1e9.  Blocking; allocates
 * nothing.  LBM_E_INVAL for gflops_out NULL, LBM_E_CUDA on a CUDA error
 * (lbm_last_error(NULL) gives the reason). */
int lbm_fp64_fma_rate(void* cuda_stream, double* gflops_out);

/* Largest row count lbm_checks_noalloc accepts (its static scratch holds one
 * FP64 triple per row). */
#define LBM_NOALLOC_MAX_ROWS 16384

/* The sums of lbm_checks over caller-owned device buffers, allocating nothing.
 * The paper has no counterpart: this entry point exists for callers that must
 * not allocate device memory -- code running while a stream is captured,
 * stepping loops that cannot take the device synchronisation of cudaMalloc /
 * cudaFree, frameworks whose memory pool owns the GPU -- and so cannot create
 * a context.  Inputs: d_populations = device populations of one domain in the
 * library's layout, [9][ny][pitch] elements of the store type (lbm_store;
 * shifted kinds hold (f_i - omega_i rho0) * store_scale), x fastest;
 * d_solid = device bytes [ny][pitch], nonzero = solid (NULL: all fluid).
 * Output: d_out3 = device double[3] receiving mass, sum f e_x, sum f e_y.
 * Enqueued on cuda_stream (NULL: the legacy default stream); not blocking.
 * Scratch is one static device array of LBM_NOALLOC_MAX_ROWS x 3 doubles
 * (384 KiB on every GPU that loads the library, until exit); ny above that
 * maximum is rejected with LBM_E_INVAL, as are bad sizes and a NULL buffer.
 * A CUDA error already pending when the call starts is returned as
 * LBM_E_CUDA and left pending; lbm_last_error(NULL) gives the reason of every
 * LBM_E_INVAL and LBM_E_CUDA.
 * The first call on a device looks up the array's device address (the runtime
 * loads the module if it has not yet), so make that first call before any
 * stream capture.  All calls share the array: calls whose kernels may overlap
 * on the GPU must be ordered by the caller. */
int lbm_checks_noalloc(const void* d_populations, int32_t store, int32_t nx, int32_t ny, int32_t pitch,
                       double rho0, double store_scale, const uint8_t* d_solid, double* d_out3,
                       void* cuda_stream);

/* Last error message of the context (static string when ctx is NULL). */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Release the context and all of its device memory. */
void lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */

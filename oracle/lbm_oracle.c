/*
 * lbm_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see
 * lbm_oracle.h).  Nothing here is tuned: nested loops, one function per
 * equation of arXiv:2006.12910, in the paper's order and notation.
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp -ffp-contract=off (no FMA contraction,
 * so x86 and Arm hosts produce the same bits).
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- Sec. 2: D2Q9 lattice (velocities e_i, weights omega_i, c_s^2 = 1/3) ---- */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WI[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0;

struct or_domain {
    or_params p;
    int64_t n;             /* nx * ny */
    uint8_t* solid;        /* 1 = stationary solid node */
    double* f;             /* post-collision populations f*(t), [9][n] */
    double* fn;            /* populations after streaming, [9][n] */
    int np;
    or_particle* part;
    int32_t* owner;        /* rasterisation at t: 0 or particle index + 1 */
    int32_t* owner_prev;   /* rasterisation at t-1 */
    double* diag;          /* np * OR_DIAG_N */
    double* zlink;         /* np * 6: link friction matrix Z of the step (see or_newton_euler) */
    or_particle* bnd;      /* per particle: r_c(t) with the mid-step velocities of the exchange */
    int64_t step;
    int64_t overlap_count; /* nodes found inside two particles */
};

static inline int64_t IDX(const or_domain* d, int x, int y) { return (int64_t)y * d->p.nx + x; }

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

void or_lattice(int32_t* e, double* w, int32_t* opp) {
    for (int i = 0; i < 9; ++i) {
        e[2 * i] = EX[i];
        e[2 * i + 1] = EY[i];
        w[i] = WI[i];
        opp[i] = OPP[i];
    }
}

/* ---- Table 1: D2Q9 mode basis e_ki and its lengths w_k (Sec. 4) ---- */
static double mode_e(int k, int i) {
    const double ex = EX[i], ey = EY[i], e2 = ex * ex + ey * ey;
    switch (k) {
        case 0: return 1.0;
        case 1: return ex;
        case 2: return ey;
        case 3: return 3.0 * e2 - 2.0;
        case 4: return 2.0 * ex * ex - e2;
        case 5: return ex * ey;
        case 6: return (3.0 * e2 - 4.0) * ex;
        case 7: return (3.0 * e2 - 4.0) * ey;
        default: return 9.0 * e2 * e2 - 15.0 * e2 + 2.0;
    }
}
/* w_k as printed in Table 1. */
static const double WK[9] = {1.0, 1.0 / 3.0, 1.0 / 3.0, 4.0, 4.0 / 9.0, 1.0 / 9.0,
                             2.0 / 3.0, 2.0 / 3.0, 16.0};

void or_basis(double* chi, double* wk) {
    /* chi_ki = e_ki / sqrt(w_k) (Sec. 4, below Eq. NP2) */
    for (int k = 0; k < 9; ++k) {
        wk[k] = WK[k];
        for (int i = 0; i < 9; ++i) chi[k * 9 + i] = mode_e(k, i) / sqrt(WK[k]);
    }
}

/* ---- Eq. (e.LB2): second-order equilibrium ---- */
void or_feq(double rho, double ux, double uy, double* out) {
    const double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        const double eu = EX[i] * ux + EY[i] * uy;
        out[i] = WI[i] * rho * (1.0 + eu / CS2 + (eu * eu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* ---- Sec. 5: local strain from the non-equilibrium momentum flux ----
 * Pi^neq = sum_i e_i e_i f_i - rho c_s^2 I - j j / rho; the Chapman-Enskog
 * strain rate is D = -Pi^neq / (2 rho c_s^2 tau).  Eq. (nn3) gives
 * Pi_D = D_xy^2 - D_xx D_yy = P / (2 rho c_s^2 tau)^2 with
 * P = Pi_xy^2 - Pi_xx Pi_yy, so the shear rate of Eq. (nn2) is
 * 2 sqrt|Pi_D| = A / tau with A = sqrt|P| / (rho c_s^2).  Returns A. */
double or_strain_A(const double* f, double rho, double jx, double jy) {
    double sxx = 0.0, syy = 0.0, sxy = 0.0;
    for (int i = 0; i < 9; ++i) {
        sxx += EX[i] * EX[i] * f[i];
        syy += EY[i] * EY[i] * f[i];
        sxy += EX[i] * EY[i] * f[i];
    }
    const double pxx = sxx - rho * CS2 - jx * jx / rho;
    const double pyy = syy - rho * CS2 - jy * jy / rho;
    const double pxy = sxy - jx * jy / rho;
    const double P = pxy * pxy - pxx * pyy;
    return sqrt(fabs(P)) / (rho * CS2);
}

/* ---- Eqs. (nn1)-(nn4) and the tau* relation of Sec. 5 ----
 * nu* = xi * kappa * |Pi_D|^((n-1)/2) with kappa = 2^(n-1) equals
 * xi * (A/tau)^(n-1); tau* = 1/2 + 3 nu*.  Because Pi_D depends on tau*, tau*
 * is the root of g(t) = t - 1/2 - 3 xi (A/t)^(n-1), clamped to
 * [tmin, tmax].  Safeguarded Newton inside the bracket, to round-off. */
double or_solve_tau(double A, double n, double xi, double tmin, double tmax) {
    if (n == 1.0) {
        double t = 0.5 + 3.0 * xi;
        return t < tmin ? tmin : (t > tmax ? tmax : t);
    }
    if (!(A > 0.0)) return n < 1.0 ? tmax : tmin;
    const double c = 3.0 * xi * pow(A, n - 1.0); /* g(t) = t - 1/2 - c t^(1-n) */
    const double glo = tmin - 0.5 - c * pow(tmin, 1.0 - n);
    if (glo >= 0.0) return tmin;
    const double ghi = tmax - 0.5 - c * pow(tmax, 1.0 - n);
    if (ghi <= 0.0) return tmax;
    double lo = tmin, hi = tmax;
    double t = n < 1.0 ? tmax : tmin;
    for (int it = 0; it < 200; ++it) {
        const double g = t - 0.5 - c * pow(t, 1.0 - n);
        if (g > 0.0) hi = t; else lo = t;
        const double dg = 1.0 - c * (1.0 - n) * pow(t, -n);
        double tn = t - g / dg;
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        if (fabs(tn - t) <= 1e-16 * t || hi - lo <= 1e-16 * hi) { t = tn; break; }
        t = tn;
    }
    return t;
}

/* ---- Sec. 4: Philox4x32-10 counter-based generator (Salmon, Moraes, Dror,
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Written from
 * the published definition: 10 rounds of two 32x32->64 multiplies with a
 * Weyl-sequence key schedule. ---- */
void or_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1) from the top 23 bits: ((x >> 9) + 1/2) / 2^23 is an odd
 * multiple of 2^-24 below 1, exactly representable in FP32 and FP64, so every
 * implementation of the generator draws the identical uniform. */
static double u23(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Six standard normal deviates Theta_3..Theta_8 of Eq. (NP2) for one node and
 * step.  Counter = (node, step, draw, domain), key = (seed_lo, seed_hi); draw 0
 * gives two Box-Muller pairs, draw 1 the third pair. */
void or_thetas(uint64_t seed, uint32_t node, uint32_t step, uint32_t domain, double* th) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[8];
    for (uint32_t draw = 0; draw < 2; ++draw) {
        const uint32_t ctr[4] = {node, step, draw, domain};
        or_philox4x32_10(ctr, key, r + 4 * draw);
    }
    const double two_pi = 6.283185307179586476925286766559;
    for (int pr = 0; pr < 3; ++pr) {
        const double ua = u23(r[2 * pr]), ub = u23(r[2 * pr + 1]);
        const double rad = sqrt(-2.0 * log(ua));
        th[2 * pr] = rad * cos(two_pi * ub);
        th[2 * pr + 1] = rad * sin(two_pi * ub);
    }
}

/* ---- Eq. (NP2): zeta_i = sqrt(rho kT w(2-w) / c_s^2) sum_{k=3..8} omega_i chi_ki Theta_k ---- */
void or_noise(double rho, double kT, double omega, const double* th, double* zeta) {
    const double amp = sqrt(rho * kT * omega * (2.0 - omega) / CS2);
    for (int i = 0; i < 9; ++i) {
        double s = 0.0;
        for (int k = 3; k < 9; ++k) s += WI[i] * (mode_e(k, i) / sqrt(WK[k])) * th[k - 3];
        zeta[i] = amp * s;
    }
}

/* ---- One node: Eq. (e.LB1) right-hand side with Eq. (e.LB2), the force
 * entering through rho u = sum f e + tau rho g (Sec. 2), the local tau* of
 * Eq. (nn5) when the power law is on, then Eq. (NP1) noise. ---- */
void or_collide_node(const or_params* p, const double* f, double* out, uint32_t node, uint32_t step) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        rho += f[i];
        jx += f[i] * EX[i];
        jy += f[i] * EY[i];
    }
    double tau = p->tau;
    if (p->power_law) {
        const double A = or_strain_A(f, rho, jx, jy);
        /* Eq. (nn4) with another kappa: nu* = xi kappa |Pi_D|^((n-1)/2)
         * = (xi kappa / 2^(n-1)) (A/tau)^(n-1), i.e. the solve below with the
         * consistency scaled by kappa / 2^(n-1). */
        double xi = p->xi_pl;
        if (p->kappa_pl > 0.0) xi *= p->kappa_pl / pow(2.0, p->n_pl - 1.0);
        tau = or_solve_tau(A, p->n_pl, xi, p->tau_min, p->tau_max);
    }
    const double ux = (jx + tau * rho * p->gx) / rho;
    const double uy = (jy + tau * rho * p->gy) / rho;
    double feq[9];
    or_feq(rho, ux, uy, feq);
    for (int i = 0; i < 9; ++i) out[i] = f[i] - (f[i] - feq[i]) / tau;
    if (p->kT > 0.0) {
        double th[6], zeta[9];
        or_thetas(p->seed, node, step, p->domain_id, th);
        or_noise(rho, p->kT, 1.0 / tau, th, zeta);
        for (int i = 0; i < 9; ++i) out[i] += zeta[i];
    }
}

/* ---- Eqs. (MP5), (MP6) and the position update of Sec. 3 ----
 * m_p = rho_p pi R^2 and I_p = m_p R^2 / 2 (disk); the fluid density in the
 * buoyancy term is rho0.  The position moves with the OLD velocity U(t).
 *
 * Generalised velocity X = (U, V, Omega).  The force of Eq. (MP1) on a link
 * splits into a part that does not depend on the particle's motion,
 * -2 f'_k e_k, and a part linear in the boundary velocity,
 * -(2 rho0 omega_k / c_s^2)(u_b . e_k) e_k with u_b . e_k = a_k . X,
 * a_k = (e_kx, e_ky, (r_b - r_c) x e_k).  Summed over the links with the torque
 * of Eq. (MP4) this is -Z X, Z = sum_k (2 rho0 omega_k / c_s^2) a_k a_k^T.
 * The link exchange happens half-way through the step (the bounced population
 * meets the boundary node r_b, half-way between the nodes, at t + dt/2), so
 * u_b is taken at mid-step, X_mid = (X(t) + X(t+dt)) / 2, on both sides of the
 * link (force here, Eqs. (MP7)-(MP8) in the stream).  Eqs. (MP5)-(MP6) then read
 *   diag(m, m, I) (X(t+dt) - X(t)) = F + m (1 - rho0/rho_p) g - Z X_mid,
 * F = the motion-independent link force plus the covered/uncovered and
 * Eq. (MP2) forces (F[2] the torque), a 3x3 linear system for X(t+dt).
 * Returns X_mid in xmid (the held velocity for a fixed particle). */
void or_newton_euler(or_particle* q, const double* F, const double* Z, double gx, double gy,
                     double rho0, double* xmid) {
    const double X0[3] = {q->U, q->V, q->Omega};
    if (q->fixed) {
        for (int j = 0; j < 3; ++j) xmid[j] = X0[j];
        return;
    }
    const double pi = 3.14159265358979323846264338327950288;
    const double m = q->rho_p * pi * q->R * q->R;
    const double I = 0.5 * m * q->R * q->R;
    const double Mv[3] = {m, m, I};
    /* Z as a full symmetric matrix from its upper triangle zxx zxy zxO zyy zyO zOO */
    const double Zm[3][3] = {{Z[0], Z[1], Z[2]}, {Z[1], Z[3], Z[4]}, {Z[2], Z[4], Z[5]}};
    const double buoy = (q->rho_p - rho0) / q->rho_p;
    const double G[3] = {F[0] + m * buoy * gx, F[1] + m * buoy * gy, F[2]};
    /* (M + Z/2) X1 = (M - Z/2) X0 + G, by Cramer's rule */
    double A[3][3], b[3];
    for (int r = 0; r < 3; ++r) {
        b[r] = Mv[r] * X0[r] + G[r];
        for (int c = 0; c < 3; ++c) {
            A[r][c] = 0.5 * Zm[r][c] + (r == c ? Mv[r] : 0.0);
            b[r] -= 0.5 * Zm[r][c] * X0[c];
        }
    }
    const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
                     - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
                     + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    double X1[3];
    for (int j = 0; j < 3; ++j) {
        double Aj[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) Aj[r][c] = c == j ? b[r] : A[r][c];
        const double dj = Aj[0][0] * (Aj[1][1] * Aj[2][2] - Aj[1][2] * Aj[2][1])
                        - Aj[0][1] * (Aj[1][0] * Aj[2][2] - Aj[1][2] * Aj[2][0])
                        + Aj[0][2] * (Aj[1][0] * Aj[2][1] - Aj[1][1] * Aj[2][0]);
        X1[j] = dj / det;
    }
    for (int j = 0; j < 3; ++j) xmid[j] = 0.5 * (X0[j] + X1[j]);
    q->U = X1[0];
    q->V = X1[1];
    q->Omega = X1[2];
    q->x += X0[0];
    q->y += X0[1];
    q->theta += X0[2];
}

/* ---- Eq. (MP2): repulsion on the node at a from the node at b ---- */
void or_lj_pair_force(double ax, double ay, double bx, double by, double psi, double rit, double* F) {
    const double rx = ax - bx, ry = ay - by;
    const double d = sqrt(rx * rx + ry * ry);
    const double mag = psi * pow(d / rit, -13.0);
    F[0] = mag * rx / d;
    F[1] = mag * ry / d;
}

/* ------------------------------------------------------------------------ */
/* Domain bookkeeping                                                        */
/* ------------------------------------------------------------------------ */

or_domain* or_create(const or_params* p) {
    if (p->nx < 3 || p->ny < 3 || !(p->tau > 0.5)) return NULL;
    if ((p->periodic_x != 0) == (p->inlet_outlet != 0)) return NULL;
    if ((p->periodic_y != 0) == (p->walls_y != 0)) return NULL;
    or_domain* d = (or_domain*)calloc(1, sizeof(or_domain));
    d->p = *p;
    d->n = (int64_t)p->nx * p->ny;
    d->solid = (uint8_t*)calloc((size_t)d->n, 1);
    d->f = (double*)calloc((size_t)(9 * d->n), sizeof(double));
    d->fn = (double*)calloc((size_t)(9 * d->n), sizeof(double));
    d->owner = (int32_t*)calloc((size_t)d->n, sizeof(int32_t));
    d->owner_prev = (int32_t*)calloc((size_t)d->n, sizeof(int32_t));
    or_init_equilibrium(d, p->rho0, 0.0, 0.0);
    return d;
}

void or_destroy(or_domain* d) {
    if (!d) return;
    free(d->solid); free(d->f); free(d->fn); free(d->part);
    free(d->owner); free(d->owner_prev); free(d->diag); free(d->zlink); free(d->bnd);
    free(d);
}

void or_init_equilibrium(or_domain* d, double rho, double ux, double uy) {
    double feq[9];
    or_feq(rho, ux, uy, feq);
    for (int64_t k = 0; k < d->n; ++k)
        for (int i = 0; i < 9; ++i) {
            d->f[i * d->n + k] = d->solid[k] ? 0.0 : feq[i];
            d->fn[i * d->n + k] = 0.0;
        }
}

int or_set_solid(or_domain* d, const uint8_t* solid) {
    for (int64_t k = 0; k < d->n; ++k) d->solid[k] = solid[k] ? 1 : 0;
    for (int64_t k = 0; k < d->n; ++k)
        if (d->solid[k])
            for (int i = 0; i < 9; ++i) { d->f[i * d->n + k] = 0.0; d->fn[i * d->n + k] = 0.0; }
    return 0;
}

int or_set_populations(or_domain* d, const double* f) {
    for (int i = 0; i < 9; ++i)
        for (int64_t k = 0; k < d->n; ++k)
            d->f[i * d->n + k] = d->solid[k] ? 0.0 : f[i * d->n + k];
    return 0;
}

void or_get_populations(const or_domain* d, double* f) { memcpy(f, d->f, sizeof(double) * 9 * d->n); }
int64_t or_step_count(const or_domain* d) { return d->step; }

/* Minimum-image displacement along a periodic axis. */
static double min_image(double dd, int L, int periodic) {
    if (!periodic) return dd;
    while (dd >= 0.5 * L) dd -= L;
    while (dd < -0.5 * L) dd += L;
    return dd;
}

/* Sec. 3: a lattice node belongs to the particle when strictly inside its disk. */
static int inside(const or_domain* d, const or_particle* q, double x, double y) {
    const double dx = min_image(x - q->x, d->p.nx, d->p.periodic_x);
    const double dy = min_image(y - q->y, d->p.ny, d->p.periodic_y);
    return dx * dx + dy * dy < q->R * q->R;
}

/* Wrap a node coordinate into the domain; returns 0 when it falls outside a
 * non-periodic edge. */
static int wrap_node(const or_domain* d, int* x, int* y) {
    if (*x < 0 || *x >= d->p.nx) {
        if (!d->p.periodic_x) return 0;
        *x = ((*x % d->p.nx) + d->p.nx) % d->p.nx;
    }
    if (*y < 0 || *y >= d->p.ny) {
        if (!d->p.periodic_y) return 0;
        *y = ((*y % d->p.ny) + d->p.ny) % d->p.ny;
    }
    return 1;
}

/* Rasterise every particle (Sec. 3, Fig. 1): owner = particle index + 1 for
 * the nodes inside its disk.  A node claimed twice is counted as an overlap. */
static void rasterise(or_domain* d) {
    memset(d->owner, 0, sizeof(int32_t) * d->n);
    for (int p = 0; p < d->np; ++p) {
        const or_particle* q = &d->part[p];
        const int x0 = (int)floor(q->x - q->R) - 1, x1 = (int)ceil(q->x + q->R) + 1;
        const int y0 = (int)floor(q->y - q->R) - 1, y1 = (int)ceil(q->y + q->R) + 1;
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) {
                int wx = x, wy = y;
                if (!wrap_node(d, &wx, &wy)) continue;
                if (!inside(d, q, wx, wy)) continue;
                int32_t* o = &d->owner[IDX(d, wx, wy)];
                if (*o == 0) *o = p + 1;
                else if (*o != p + 1) d->overlap_count++;
            }
    }
}

int or_add_particles(or_domain* d, int n, const or_particle* p) {
    d->part = (or_particle*)realloc(d->part, sizeof(or_particle) * (size_t)(d->np + n));
    memcpy(d->part + d->np, p, sizeof(or_particle) * (size_t)n);
    d->np += n;
    d->diag = (double*)realloc(d->diag, sizeof(double) * OR_DIAG_N * (size_t)d->np);
    memset(d->diag, 0, sizeof(double) * OR_DIAG_N * (size_t)d->np);
    d->zlink = (double*)realloc(d->zlink, sizeof(double) * 6 * (size_t)d->np);
    memset(d->zlink, 0, sizeof(double) * 6 * (size_t)d->np);
    d->bnd = (or_particle*)realloc(d->bnd, sizeof(or_particle) * (size_t)d->np);
    memcpy(d->bnd, d->part, sizeof(or_particle) * (size_t)d->np);
    rasterise(d);
    memcpy(d->owner_prev, d->owner, sizeof(int32_t) * d->n);
    return (int)d->overlap_count;
}

/* Boundary-node velocity u_b = U_p + Omega_p x (r_b - r_c) (Sec. 3, below MP6). */
static void boundary_velocity(const or_domain* d, const or_particle* q, double bx, double by,
                              double* ubx, double* uby) {
    const double rx = min_image(bx - q->x, d->p.nx, d->p.periodic_x);
    const double ry = min_image(by - q->y, d->p.ny, d->p.periodic_y);
    *ubx = q->U - q->Omega * ry;
    *uby = q->V + q->Omega * rx;
}

/* Node moments of the stored post-collision populations: rho and the
 * physical velocity u = (sum f* e - rho g / 2) / rho. */
static void node_moments(const or_domain* d, int64_t k, double* rho, double* ux, double* uy) {
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        const double fi = d->f[i * d->n + k];
        r += fi;
        jx += fi * EX[i];
        jy += fi * EY[i];
    }
    *rho = r;
    *ux = (jx - 0.5 * r * d->p.gx) / r;
    *uy = (jy - 0.5 * r * d->p.gy) / r;
}

static int is_surface(const or_domain* d, const or_particle* q, int x, int y) {
    if (!inside(d, q, x, y)) return 0;
    for (int i = 1; i < 9; ++i)
        if (!inside(d, q, x + EX[i], y + EY[i])) return 1;
    return 0;
}

/* ---- Eqs. (MP1), (MP3), (MP4) at time t, from the post-collision f*(t) ---- */
static void particle_forces(or_domain* d) {
    const or_params* P = &d->p;
    for (int p = 0; p < d->np; ++p) {
        const or_particle* q = &d->part[p];
        double* dg = &d->diag[p * OR_DIAG_N];
        double* Z = &d->zlink[p * 6];
        memset(dg, 0, sizeof(double) * OR_DIAG_N);
        memset(Z, 0, sizeof(double) * 6);

        /* Eq. (MP1): exterior link r_v -> r_v + e_k with r_v inside p. */
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                const int64_t kv = IDX(d, x, y);
                if (d->owner[kv] != p + 1 || d->solid[kv]) continue;
                for (int k = 1; k < 9; ++k) {
                    int fx = x + EX[k], fy = y + EY[k];
                    if (!wrap_node(d, &fx, &fy)) continue;
                    const int64_t kf = IDX(d, fx, fy);
                    if (d->solid[kf] || d->owner[kf] != 0) continue;
                    const double bx = x + 0.5 * EX[k], by = y + 0.5 * EY[k];
                    const double fprime = d->f[OPP[k] * d->n + kf]; /* population along -e_k at r_v+e_k */
                    /* the part of Eq. (MP1) that does not depend on u_b */
                    const double s = -2.0 * fprime;
                    const double Fx = s * EX[k], Fy = s * EY[k];
                    const double rx = min_image(bx - q->x, P->nx, P->periodic_x);
                    const double ry = min_image(by - q->y, P->ny, P->periodic_y);
                    dg[0] += Fx;
                    dg[1] += Fy;
                    dg[2] += rx * Fy - ry * Fx;
                    /* the part linear in u_b: -c (a . X) a with a = (e_x, e_y, r x e) */
                    const double c = 2.0 * P->rho0 * WI[k] / CS2;
                    const double a[3] = {EX[k], EY[k], rx * EY[k] - ry * EX[k]};
                    Z[0] += c * a[0] * a[0];
                    Z[1] += c * a[0] * a[1];
                    Z[2] += c * a[0] * a[2];
                    Z[3] += c * a[1] * a[1];
                    Z[4] += c * a[1] * a[2];
                    Z[5] += c * a[2] * a[2];
                }
            }

        /* Covered / uncovered nodes between the rasterisations at t-1 and t:
         * F = +rho (u - U_p) when covered, -rho (u - U_p) when uncovered. */
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                const int64_t k = IDX(d, x, y);
                if (d->solid[k]) continue;
                const int now = d->owner[k] == p + 1, before = d->owner_prev[k] == p + 1;
                if (now == before) continue;
                double rho, ux, uy;
                node_moments(d, k, &rho, &ux, &uy);
                const double sgn = now ? 1.0 : -1.0;
                const double Fx = sgn * rho * (ux - q->U), Fy = sgn * rho * (uy - q->V);
                const double rx = min_image(x - q->x, P->nx, P->periodic_x);
                const double ry = min_image(y - q->y, P->ny, P->periodic_y);
                dg[3] += Fx;
                dg[4] += Fy;
                dg[5] += rx * Fy - ry * Fx;
                if (now) { dg[9] += 1.0; dg[11] += rho; }
                else { dg[10] += 1.0; dg[12] += rho; }
            }

        /* Eq. (MP2): surface nodes of p against surface nodes of other
         * particles and against stationary solid / wall nodes within r_it. */
        if (P->lj_psi != 0.0) {
            const int x0 = (int)floor(q->x - q->R) - 1, x1 = (int)ceil(q->x + q->R) + 1;
            const int y0 = (int)floor(q->y - q->R) - 1, y1 = (int)ceil(q->y + q->R) + 1;
            const int reach = (int)floor(P->lj_rit);
            for (int ay = y0; ay <= y1; ++ay)
                for (int ax = x0; ax <= x1; ++ax) {
                    if (!is_surface(d, q, ax, ay)) continue;
                    const double rax = min_image(ax - q->x, P->nx, P->periodic_x);
                    const double ray = min_image(ay - q->y, P->ny, P->periodic_y);
                    /* particle - particle */
                    for (int p2 = 0; p2 < d->np; ++p2) {
                        if (p2 == p) continue;
                        const or_particle* o = &d->part[p2];
                        const int bx0 = (int)floor(o->x - o->R) - 1, bx1 = (int)ceil(o->x + o->R) + 1;
                        const int by0 = (int)floor(o->y - o->R) - 1, by1 = (int)ceil(o->y + o->R) + 1;
                        for (int by = by0; by <= by1; ++by)
                            for (int bx = bx0; bx <= bx1; ++bx) {
                                if (!is_surface(d, o, bx, by)) continue;
                                const double sx = min_image((double)ax - bx, P->nx, P->periodic_x);
                                const double sy = min_image((double)ay - by, P->ny, P->periodic_y);
                                const double dist = sqrt(sx * sx + sy * sy);
                                if (!(dist <= P->lj_rit) || dist == 0.0) continue;
                                double F[2];
                                or_lj_pair_force(sx, sy, 0.0, 0.0, P->lj_psi, P->lj_rit, F);
                                dg[6] += F[0];
                                dg[7] += F[1];
                                dg[8] += rax * F[1] - ray * F[0];
                            }
                    }
                    /* particle - stationary solid (obstacles and the rows beyond the y walls) */
                    for (int oy = -reach; oy <= reach; ++oy)
                        for (int ox = -reach; ox <= reach; ++ox) {
                            if (ox == 0 && oy == 0) continue;
                            const double dist = sqrt((double)(ox * ox + oy * oy));
                            if (!(dist <= P->lj_rit)) continue;
                            int wx = ax + ox, wy = ay + oy;
                            int is_wall = 0;
                            if (P->walls_y && (wy < 0 || wy >= P->ny)) is_wall = 1;
                            else {
                                if (!wrap_node(d, &wx, &wy)) continue;
                                is_wall = d->solid[IDX(d, wx, wy)];
                            }
                            if (!is_wall) continue;
                            double F[2];
                            or_lj_pair_force(0.0, 0.0, ox, oy, P->lj_psi, P->lj_rit, F);
                            dg[6] += F[0];
                            dg[7] += F[1];
                            dg[8] += rax * F[1] - ray * F[0];
                        }
                }
        }
    }
}

/* ---- Eq. (e.LB1) left-hand side: streaming f_i(r + e_i, t+1) = f*_i(r, t),
 * with halfway bounce-back at walls / stationary solids and Eqs. (MP7)-(MP8)
 * on particle links.  Push form, one write per destination slot. ---- */
static void stream(or_domain* d) {
    const or_params* P = &d->p;
    const int64_t n = d->n;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < P->ny; ++y)
        for (int x = 0; x < P->nx; ++x) {
            const int64_t k = IDX(d, x, y);
            if (d->solid[k]) continue;
            for (int i = 0; i < 9; ++i) {
                const double fi = d->f[i * n + k];
                int tx = x + EX[i], ty = y + EY[i];
                if (ty < 0 || ty >= P->ny) {
                    if (P->walls_y) { d->fn[OPP[i] * n + k] = fi; continue; }
                    ty = (ty + P->ny) % P->ny;
                }
                if (tx < 0 || tx >= P->nx) {
                    if (P->periodic_x) tx = (tx + P->nx) % P->nx;
                    else {
                        /* open inlet / outlet column: the population leaves the
                         * domain; wall-corner nodes reflect it instead. */
                        if (P->walls_y && (y == 0 || y == P->ny - 1)) d->fn[OPP[i] * n + k] = fi;
                        continue;
                    }
                }
                const int64_t t = IDX(d, tx, ty);
                if (d->solid[t]) { d->fn[OPP[i] * n + k] = fi; continue; }
                const int32_t ox = d->owner[k], ot = d->owner[t];
                if (ox != ot && (ox == 0 || ot == 0)) {
                    /* r_c(t) and the mid-step velocities (see or_newton_euler) */
                    const or_particle* q = &d->bnd[(ox ? ox : ot) - 1];
                    double ubx, uby;
                    boundary_velocity(d, q, x + 0.5 * EX[i], y + 0.5 * EY[i], &ubx, &uby);
                    const double ube = ubx * EX[i] + uby * EY[i];
                    /* Eq. (MP7) when r is inside, Eq. (MP8) when r is outside */
                    d->fn[OPP[i] * n + k] = fi - 2.0 * P->rho0 * WI[i] * ube / CS2;
                    continue;
                }
                d->fn[i * n + t] = fi;
            }
        }
}

/* Zou & He (Phys. Fluids 9, 1591, 1997) density boundary on the first and last
 * columns: the three populations entering from outside are set from the
 * known ones so that rho = rho_in (rho_out) and u_y = 0. */
static void inlet_outlet(or_domain* d) {
    const or_params* P = &d->p;
    const int64_t n = d->n;
    for (int y = 0; y < P->ny; ++y) {
        if (P->walls_y && (y == 0 || y == P->ny - 1)) continue;
        for (int side = 0; side < 2; ++side) {
            const int x = side == 0 ? 0 : P->nx - 1;
            const int64_t k = IDX(d, x, y);
            if (d->solid[k]) continue;
            double f[9];
            for (int i = 0; i < 9; ++i) f[i] = d->fn[i * n + k];
            if (side == 0) {
                const double r = P->rho_in;
                const double ux = 1.0 - (f[0] + f[2] + f[4] + 2.0 * (f[3] + f[6] + f[7])) / r;
                f[1] = f[3] + (2.0 / 3.0) * r * ux;
                f[5] = f[7] - 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * r * ux;
                f[8] = f[6] + 0.5 * (f[2] - f[4]) + (1.0 / 6.0) * r * ux;
            } else {
                const double r = P->rho_out;
                const double ux = -1.0 + (f[0] + f[2] + f[4] + 2.0 * (f[1] + f[5] + f[8])) / r;
                f[3] = f[1] - (2.0 / 3.0) * r * ux;
                f[7] = f[5] + 0.5 * (f[2] - f[4]) - (1.0 / 6.0) * r * ux;
                f[6] = f[8] - 0.5 * (f[2] - f[4]) - (1.0 / 6.0) * r * ux;
            }
            for (int i = 0; i < 9; ++i) d->fn[i * n + k] = f[i];
        }
    }
}

static void collide_all(or_domain* d) {
    const int64_t n = d->n;
    const uint32_t step = (uint32_t)d->step;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        if (d->solid[k]) continue;
        double f[9], out[9];
        for (int i = 0; i < 9; ++i) f[i] = d->fn[i * n + k];
        or_collide_node(&d->p, f, out, (uint32_t)k, step);
        for (int i = 0; i < 9; ++i) d->f[i * n + k] = out[i];
    }
}

void or_step(or_domain* d, int64_t nsteps) {
    for (int64_t s = 0; s < nsteps; ++s) {
        if (d->np) {
            /* 1. forces on the particles at t (MP1-MP4) */
            particle_forces(d);
            /* 2. Newton-Euler (MP5, MP6) with the mid-step boundary velocity;
             *    the link force reported is the full Eq. (MP1) at that velocity */
            for (int p = 0; p < d->np; ++p) {
                double* dg = &d->diag[p * OR_DIAG_N];
                const double* Z = &d->zlink[p * 6];
                const double F[3] = {dg[0] + dg[3] + dg[6], dg[1] + dg[4] + dg[7], dg[2] + dg[5] + dg[8]};
                or_particle* q = &d->part[p];
                d->bnd[p] = *q;
                double xm[3];
                or_newton_euler(q, F, Z, d->p.gx, d->p.gy, d->p.rho0, xm);
                d->bnd[p].U = xm[0];
                d->bnd[p].V = xm[1];
                d->bnd[p].Omega = xm[2];
                dg[0] -= Z[0] * xm[0] + Z[1] * xm[1] + Z[2] * xm[2];
                dg[1] -= Z[1] * xm[0] + Z[3] * xm[1] + Z[4] * xm[2];
                dg[2] -= Z[2] * xm[0] + Z[4] * xm[1] + Z[5] * xm[2];
            }
        }
        /* 3. stream with bounce-back (e.LB1 LHS, MP7, MP8) */
        stream(d);
        /* 4. open inlet / outlet columns */
        if (d->p.inlet_outlet) inlet_outlet(d);
        /* 5. collide at t+1 with noise (e.LB1 RHS, e.LB2, nn5, NP1) */
        collide_all(d);
        /* 6. particles at their new positions: re-rasterise */
        if (d->np) {
            for (int p = 0; p < d->np; ++p) {
                or_particle* q = &d->part[p];
                if (d->p.periodic_x) q->x = q->x - d->p.nx * floor(q->x / d->p.nx);
                if (d->p.periodic_y) q->y = q->y - d->p.ny * floor(q->y / d->p.ny);
            }
            memcpy(d->owner_prev, d->owner, sizeof(int32_t) * d->n);
            rasterise(d);
        }
        d->step++;
    }
}

void or_moments(const or_domain* d, double* rho, double* ux, double* uy) {
    for (int64_t k = 0; k < d->n; ++k) {
        if (d->solid[k]) { rho[k] = 0.0; ux[k] = 0.0; uy[k] = 0.0; continue; }
        node_moments(d, k, &rho[k], &ux[k], &uy[k]);
    }
}

int or_get_particles(const or_domain* d, or_particle* out, int cap) {
    const int n = d->np < cap ? d->np : cap;
    memcpy(out, d->part, sizeof(or_particle) * (size_t)n);
    return d->np;
}

void or_particle_diag(const or_domain* d, int p, double* out) {
    memcpy(out, &d->diag[p * OR_DIAG_N], sizeof(double) * OR_DIAG_N);
}

/* Kahan-compensated sums of mass and post-collision momentum over fluid nodes. */
static void kahan_add(double* s, double* c, double v) {
    const double y = v - *c;
    const double t = *s + y;
    *c = (t - *s) - y;
    *s = t;
}

void or_checks(const or_domain* d, double* out3) {
    double s[3] = {0, 0, 0}, c[3] = {0, 0, 0};
    for (int64_t k = 0; k < d->n; ++k) {
        if (d->solid[k]) continue;
        for (int i = 0; i < 9; ++i) {
            const double fi = d->f[i * d->n + k];
            kahan_add(&s[0], &c[0], fi);
            kahan_add(&s[1], &c[1], fi * EX[i]);
            kahan_add(&s[2], &c[2], fi * EY[i]);
        }
    }
    out3[0] = s[0]; out3[1] = s[1]; out3[2] = s[2];
}

void or_exterior_momentum(const or_domain* d, double* out2) {
    double s[2] = {0, 0}, c[2] = {0, 0};
    for (int64_t k = 0; k < d->n; ++k) {
        if (d->solid[k] || d->owner[k]) continue;
        for (int i = 0; i < 9; ++i) {
            const double fi = d->f[i * d->n + k];
            kahan_add(&s[0], &c[0], fi * EX[i]);
            kahan_add(&s[1], &c[1], fi * EY[i]);
        }
    }
    out2[0] = s[0]; out2[1] = s[1];
}

int or_links(const or_domain* d, int p, int32_t* node, int32_t* dir, int cap) {
    int m = 0;
    for (int y = 0; y < d->p.ny; ++y)
        for (int x = 0; x < d->p.nx; ++x) {
            const int64_t kv = IDX(d, x, y);
            if (d->owner[kv] != p + 1 || d->solid[kv]) continue;
            for (int k = 1; k < 9; ++k) {
                int fx = x + EX[k], fy = y + EY[k];
                if (!wrap_node(d, &fx, &fy)) continue;
                const int64_t kf = IDX(d, fx, fy);
                if (d->solid[kf] || d->owner[kf] != 0) continue;
                if (m < cap) { node[m] = (int32_t)kv; dir[m] = k; }
                ++m;
            }
        }
    return m;
}

void or_owner(const or_domain* d, int32_t* out) { memcpy(out, d->owner, sizeof(int32_t) * d->n); }

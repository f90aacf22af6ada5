// lbm_dev.cuh -- device building blocks of the GB300 D2Q9 library: lattice
// constants, population storage kinds, the Philox4x32-10 generator and the
// per-node collision (arXiv:2006.12910 Secs. 2, 4, 5).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_types.h"

namespace lbmk {

// ---------------------------------------------------------------------------
// D2Q9 lattice, Sec. 2: e0=(0,0); e1..e4 = (1,0),(0,1),(-1,0),(0,-1);
// e5..e8 = (1,1),(-1,1),(-1,-1),(1,-1); weights 4/9, 1/9, 1/36; c_s^2 = 1/3.
// Written as constexpr functions so fully unrolled loops fold them away.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cx(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int cy(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5); }
__host__ __device__ constexpr double wgt(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }

// Table 1 mode vectors e_ki (k = 3..8) for direction i, with |e_i|^2 = e2.
__host__ __device__ constexpr double mode_vec(int k, int i) {
    return k == 3 ? 3.0 * (cx(i) * cx(i) + cy(i) * cy(i)) - 2.0
         : k == 4 ? 2.0 * cx(i) * cx(i) - (cx(i) * cx(i) + cy(i) * cy(i))
         : k == 5 ? 1.0 * cx(i) * cy(i)
         : k == 6 ? (3.0 * (cx(i) * cx(i) + cy(i) * cy(i)) - 4.0) * cx(i)
         : k == 7 ? (3.0 * (cx(i) * cx(i) + cy(i) * cy(i)) - 4.0) * cy(i)
         : 9.0 * (cx(i) * cx(i) + cy(i) * cy(i)) * (cx(i) * cx(i) + cy(i) * cy(i))
               - 15.0 * (cx(i) * cx(i) + cy(i) * cy(i)) + 2.0;
}
// 1/sqrt(w_k) for the Table 1 lengths w_3..w_8 = 4, 4/9, 1/9, 2/3, 2/3, 16.
__host__ __device__ constexpr double inv_sqrt_wk(int k) {
    return k == 3 ? 0.5 : k == 4 ? 1.5 : k == 5 ? 3.0 : (k == 6 || k == 7) ? 1.2247448713915890491 : 0.25;
}
// Noise weight of mode k in direction i: omega_i chi_ki = omega_i e_ki / sqrt(w_k) (Eq. NP2).
__host__ __device__ constexpr double noise_coef(int i, int k) { return wgt(i) * mode_vec(k, i) * inv_sqrt_wk(k); }

// ---------------------------------------------------------------------------
// Population storage kinds.  V = nodes per 16-byte vector.
// ---------------------------------------------------------------------------
struct StF64 {
    typedef double T; typedef double A;
    static constexpr int V = 2; static constexpr bool SHIFT = false; static constexpr bool SCALED = false;
    static constexpr int KIND = 0;
};
struct StF32 {
    typedef float T; typedef float A;
    static constexpr int V = 4; static constexpr bool SHIFT = false; static constexpr bool SCALED = false;
    static constexpr int KIND = 1;
};
struct StF32S {
    typedef float T; typedef float A;
    static constexpr int V = 4; static constexpr bool SHIFT = true; static constexpr bool SCALED = false;
    static constexpr int KIND = 2;
};
struct StF16S {
    typedef __half T; typedef float A;
    static constexpr int V = 8; static constexpr bool SHIFT = true; static constexpr bool SCALED = true;
    static constexpr int KIND = 3;
};
struct StBF16S {
    typedef __nv_bfloat16 T; typedef float A;
    static constexpr int V = 8; static constexpr bool SHIFT = true; static constexpr bool SCALED = true;
    static constexpr int KIND = 4;
};

__device__ __forceinline__ double to_a(double v, double) { return v; }
__device__ __forceinline__ float to_a(float v, float) { return v; }
__device__ __forceinline__ float to_a(__half v, float inv) { return __half2float(v) * inv; }
__device__ __forceinline__ float to_a(__nv_bfloat16 v, float inv) { return __bfloat162float(v) * inv; }
__device__ __forceinline__ void from_a(double v, double, double& o) { o = v; }
__device__ __forceinline__ void from_a(float v, float, float& o) { o = v; }
__device__ __forceinline__ void from_a(float v, float s, __half& o) { o = __float2half_rn(v * s); }
__device__ __forceinline__ void from_a(float v, float s, __nv_bfloat16& o) { o = __float2bfloat16_rn(v * s); }

// 16-byte vector load (read-only path) and store of V consecutive elements.
template <class S>
__device__ __forceinline__ void load_vec(const typename S::T* p, typename S::A* out, typename S::A inv) {
    union { uint4 u; typename S::T t[S::V]; } r;
    r.u = __ldg(reinterpret_cast<const uint4*>(p));
#pragma unroll
    for (int k = 0; k < S::V; ++k) out[k] = to_a(r.t[k], inv);
}
template <class S>
__device__ __forceinline__ void store_vec(typename S::T* p, const typename S::A* in, typename S::A scale) {
    union { uint4 u; typename S::T t[S::V]; } r;
#pragma unroll
    for (int k = 0; k < S::V; ++k) from_a(in[k], scale, r.t[k]);
    *reinterpret_cast<uint4*>(p) = r.u;
}
template <class S>
__device__ __forceinline__ typename S::A load_one(const typename S::T* p, typename S::A inv) {
    return to_a(__ldg(p), inv);
}
template <>
__device__ __forceinline__ float load_one<StF16S>(const __half* p, float inv) {
    return __half2float(__ldg(p)) * inv;
}
template <>
__device__ __forceinline__ float load_one<StBF16S>(const __nv_bfloat16* p, float inv) {
    return __bfloat162float(__ldg(p)) * inv;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit multiplies, key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Uniform in (0,1) from the top 23 bits; exact in FP32 and FP64.
__device__ __forceinline__ float uni23f(uint32_t x) { return (__uint2float_rn(x >> 9) + 0.5f) * 1.1920928955078125e-07f; }
__device__ __forceinline__ double uni23d(uint32_t x) { return ((double)(x >> 9) + 0.5) * 1.1920928955078125e-07; }

__device__ __forceinline__ void box_muller(float a, float b, float& z0, float& z1) {
    const float r = sqrtf(-2.0f * logf(a));
    float s, c;
    sincospif(2.0f * b, &s, &c);
    z0 = r * c;
    z1 = r * s;
}
__device__ __forceinline__ void box_muller(double a, double b, double& z0, double& z1) {
    const double r = sqrt(-2.0 * log(a));
    double s, c;
    sincospi(2.0 * b, &s, &c);
    z0 = r * c;
    z1 = r * s;
}
template <typename A> __device__ __forceinline__ A uni23(uint32_t x);
template <> __device__ __forceinline__ float uni23<float>(uint32_t x) { return uni23f(x); }
template <> __device__ __forceinline__ double uni23<double>(uint32_t x) { return uni23d(x); }

// Theta_3..Theta_8 of Eq. NP2 for one node: counter (node, step, draw, domain).
template <typename A>
__device__ __forceinline__ void thetas(uint32_t node, uint32_t step, uint32_t dom_id, uint64_t seed, A th[6]) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint4 r0 = philox4x32_10(make_uint4(node, step, 0u, dom_id), k0, k1);
    const uint4 r1 = philox4x32_10(make_uint4(node, step, 1u, dom_id), k0, k1);
    box_muller(uni23<A>(r0.x), uni23<A>(r0.y), th[0], th[1]);
    box_muller(uni23<A>(r0.z), uni23<A>(r0.w), th[2], th[3]);
    box_muller(uni23<A>(r1.x), uni23<A>(r1.y), th[4], th[5]);
}

// ---------------------------------------------------------------------------
// Per-domain parameters in the arithmetic type, loaded once per work item so
// the collision never converts between FP64 and FP32.
// ---------------------------------------------------------------------------
template <typename A>
struct Prm {
    A tau, inv_tau, rho0, gx, gy, kT, n, xi, tmin, tmax, tmin_pow, tmax_pow;
    A rho_in, rho_out, d_in, d_out, scale, inv_scale;
    int n_is_one;
    uint32_t dom_id;
    uint64_t seed;
};
template <typename A> __device__ __forceinline__ Prm<A> load_prm(const DomDev& D);
template <> __device__ __forceinline__ Prm<float> load_prm<float>(const DomDev& D) {
    Prm<float> P;
    P.tau = D.tau_f; P.inv_tau = D.inv_tau_f; P.rho0 = D.rho0_f; P.gx = D.gx_f; P.gy = D.gy_f; P.kT = D.kT_f;
    P.n = D.n_pl_f; P.xi = D.xi_pl_f; P.tmin = D.tau_min_f; P.tmax = D.tau_max_f;
    P.tmin_pow = D.tmin_pow_f; P.tmax_pow = D.tmax_pow_f;
    P.rho_in = D.rho_in_f; P.rho_out = D.rho_out_f; P.d_in = D.drho_in_f; P.d_out = D.drho_out_f;
    P.scale = D.scale_f; P.inv_scale = D.inv_scale_f;
    P.n_is_one = D.n_is_one; P.dom_id = D.domain_id; P.seed = D.seed;
    return P;
}
template <> __device__ __forceinline__ Prm<double> load_prm<double>(const DomDev& D) {
    Prm<double> P;
    P.tau = D.tau; P.inv_tau = D.inv_tau; P.rho0 = D.rho0; P.gx = D.gx; P.gy = D.gy; P.kT = D.kT;
    P.n = D.n_pl; P.xi = D.xi_pl; P.tmin = D.tau_min; P.tmax = D.tau_max;
    P.tmin_pow = D.tmin_pow; P.tmax_pow = D.tmax_pow;
    P.rho_in = D.rho_in; P.rho_out = D.rho_out; P.d_in = D.drho_in; P.d_out = D.drho_out;
    P.scale = D.scale; P.inv_scale = D.inv_scale;
    P.n_is_one = D.n_is_one; P.dom_id = D.domain_id; P.seed = D.seed;
    return P;
}

// ---------------------------------------------------------------------------
// Power-law relaxation time, Sec. 5.  The shear rate of Eq. nn2 with Pi_D of
// Eq. nn3 taken from the Chapman-Enskog strain -Pi_neq / (2 rho c_s^2 tau) is
// A / tau, A = 3 sqrt|Pi_xy^2 - Pi_xx Pi_yy| / rho; nu* = xi (A/tau)^(n-1)
// (nn4, kappa = 2^(n-1)) and tau = 1/2 + 3 nu*.  g(t) = t - 1/2 - c t^(1-n),
// c = 3 xi A^(n-1), is convex for n < 1 and concave for n > 1, so Newton from
// the bracket end where g > 0 (n < 1) or g < 0 (n > 1) converges monotonically.
// ---------------------------------------------------------------------------
template <typename A> __device__ __forceinline__ A powa(A x, A e);
template <> __device__ __forceinline__ float powa<float>(float x, float e) { return exp2f(e * log2f(x)); }
template <> __device__ __forceinline__ double powa<double>(double x, double e) { return exp2(e * log2(x)); }

template <typename A>
__device__ __forceinline__ A solve_tau_pl(A Astr, const Prm<A>& P) {
    const A n = P.n, tmin = P.tmin, tmax = P.tmax;
    if (P.n_is_one) {
        A t = (A)0.5 + (A)3.0 * P.xi;
        return t < tmin ? tmin : (t > tmax ? tmax : t);
    }
    if (!(Astr > (A)0)) return n < (A)1 ? tmax : tmin;
    const A om = (A)1 - n;
    const A c = (A)3.0 * P.xi * powa<A>(Astr, n - (A)1);
    if (tmin - (A)0.5 - c * P.tmin_pow >= (A)0) return tmin;
    if (tmax - (A)0.5 - c * P.tmax_pow <= (A)0) return tmax;
    A t = n < (A)1 ? tmax : tmin;
    const A tol = sizeof(A) == 4 ? (A)2e-7 : (A)1e-15;
#pragma unroll 1
    for (int it = 0; it < 60; ++it) {
        const A p = powa<A>(t, om);
        const A g = t - (A)0.5 - c * p;
        const A dg = (A)1 - c * om * p / t;
        A tn = t - g / dg;
        tn = tn < tmin ? tmin : (tn > tmax ? tmax : tn);
        const A dt = tn - t;
        t = tn;
        if (fabs(dt) <= tol * t) break;
    }
    return t;
}

// ---------------------------------------------------------------------------
// Collision of one node (Eq. e.LB1 right-hand side, Eq. e.LB2 equilibrium,
// rho u = sum f e + tau rho g, optional tau* of Eq. nn5 and noise of NP1-NP2).
// f holds the pre-collision populations, shifted by omega_i rho0 when SHIFT;
// on return it holds the post-collision values in the same units.
// Returns false when rho is not a positive finite number.
// ---------------------------------------------------------------------------
template <typename A, bool SHIFT, bool NOISE, bool PL>
__device__ __forceinline__ bool collide_node(A f[9], const Prm<A>& P, uint32_t node, uint32_t step) {
    A s = f[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) s += f[i];
    const A jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const A jy = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
    const A rho0 = P.rho0;
    const A rho = SHIFT ? rho0 + s : s;
    const A drho = SHIFT ? s : s - rho0;
    const bool ok = (rho > (A)0) && (rho < (A)1e30);
    const A irho = (A)1 / rho;
    A tau = P.tau, itau = P.inv_tau;
    if (PL) {
        const A sxx = (f[1] + f[3]) + (f[5] + f[6]) + (f[7] + f[8]);
        const A syy = (f[2] + f[4]) + (f[5] + f[6]) + (f[7] + f[8]);
        const A sxy = (f[5] - f[6]) + (f[7] - f[8]);
        const A iso = SHIFT ? drho * (A)(1.0 / 3.0) : rho * (A)(1.0 / 3.0);
        const A pxx = sxx - iso - jx * jx * irho;
        const A pyy = syy - iso - jy * jy * irho;
        const A pxy = sxy - jx * jy * irho;
        const A det = pxy * pxy - pxx * pyy;
        const A Astr = (A)3 * sqrt(fabs(det)) * irho;
        tau = solve_tau_pl<A>(Astr, P);
        itau = (A)1 / tau;
    }
    const A ux = (jx + tau * rho * P.gx) * irho;
    const A uy = (jy + tau * rho * P.gy) * irho;
    const A usq = (A)1.5 * (ux * ux + uy * uy);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const A eu = (A)cx(i) * ux + (A)cy(i) * uy;
        const A poly = (A)3 * eu + (A)4.5 * eu * eu - usq;
        const A feq = SHIFT ? (A)wgt(i) * (drho + rho * poly) : (A)wgt(i) * rho * ((A)1 + poly);
        f[i] = f[i] + (feq - f[i]) * itau;
    }
    if (NOISE) {
        if (P.kT > (A)0) {
            A th[6];
            thetas<A>(node, step, P.dom_id, P.seed, th);
            const A amp = sqrt(rho * P.kT * itau * ((A)2 - itau) * (A)3);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                A z = (A)0;
#pragma unroll
                for (int k = 3; k < 9; ++k)
                    if (noise_coef(i, k) != 0.0) z += (A)noise_coef(i, k) * th[k - 3];
                f[i] += amp * z;
            }
        }
    }
    return ok;
}

// Zou-He density column (Zou & He 1997).  side 0: inlet at x = 0, the
// populations 1, 5, 8 enter from outside; side 1: outlet at x = nx-1, the
// populations 3, 6, 7 enter.  rho_b is the prescribed density and d_b its
// excess over the rest density of the stored values (rho_b - rho0 when SHIFT,
// rho_b otherwise); the shifts of the paired populations are equal.
template <typename A>
__device__ __forceinline__ void zou_he(A f[9], int side, A rho_b, A d_b) {
    if (side == 0) {
        const A ru = d_b - (f[0] + f[2] + f[4] + (A)2 * (f[3] + f[6] + f[7]));
        f[1] = f[3] + (A)(2.0 / 3.0) * ru;
        f[5] = f[7] - (A)0.5 * (f[2] - f[4]) + (A)(1.0 / 6.0) * ru;
        f[8] = f[6] + (A)0.5 * (f[2] - f[4]) + (A)(1.0 / 6.0) * ru;
    } else {
        const A ru = (f[0] + f[2] + f[4] + (A)2 * (f[1] + f[5] + f[8])) - d_b;
        f[3] = f[1] - (A)(2.0 / 3.0) * ru;
        f[7] = f[5] + (A)0.5 * (f[2] - f[4]) - (A)(1.0 / 6.0) * ru;
        f[6] = f[8] - (A)0.5 * (f[2] - f[4]) - (A)(1.0 / 6.0) * ru;
    }
    (void)rho_b;
}

}  // namespace lbmk

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
// Population storage kinds.  V = consecutive nodes of one row a lane owns in
// the register stream-collide kernel (one vector load or store of V*sizeof(T)
// = 8 or 16 bytes per plane).  MINB / MINB_EXT: CTAs of 128 threads the
// register kernel asks to keep resident per SM (plain BGK / with noise or
// the power law), which caps its registers per thread.
// ---------------------------------------------------------------------------
struct StF64 {
    typedef double T; typedef double A;
    static constexpr int V = 2; static constexpr bool SHIFT = false; static constexpr bool SCALED = false;
    static constexpr int KIND = 0;
    static constexpr int MINB = 3, MINB_EXT = 3;
};
struct StF32 {
    typedef float T; typedef float A;
    static constexpr int V = 4; static constexpr bool SHIFT = false; static constexpr bool SCALED = false;
    static constexpr int KIND = 1;
    static constexpr int MINB = 5, MINB_EXT = 4;
};
struct StF32S {
    typedef float T; typedef float A;
    static constexpr int V = 4; static constexpr bool SHIFT = true; static constexpr bool SCALED = false;
    static constexpr int KIND = 2;
    static constexpr int MINB = 5, MINB_EXT = 4;
};
// Half-precision kinds take 8-byte vectors (4 nodes per lane): the register
// footprint of an FP32 lane, so five CTAs fit per SM, and chunks near solids
// store 4 rather than 8 nodes one by one.
struct StF16S {
    typedef __half T; typedef float A;
    static constexpr int V = 4; static constexpr bool SHIFT = true; static constexpr bool SCALED = true;
    static constexpr int KIND = 3;
    static constexpr int MINB = 5, MINB_EXT = 4;
};
struct StBF16S {
    typedef __nv_bfloat16 T; typedef float A;
    static constexpr int V = 4; static constexpr bool SHIFT = true; static constexpr bool SCALED = true;
    static constexpr int KIND = 4;
    static constexpr int MINB = 5, MINB_EXT = 4;
};

__device__ __forceinline__ double to_a(double v, double) { return v; }
__device__ __forceinline__ float to_a(float v, float) { return v; }
__device__ __forceinline__ float to_a(__half v, float inv) { return __half2float(v) * inv; }
__device__ __forceinline__ float to_a(__nv_bfloat16 v, float inv) { return __bfloat162float(v) * inv; }
__device__ __forceinline__ void from_a(double v, double, double& o) { o = v; }
__device__ __forceinline__ void from_a(float v, float, float& o) { o = v; }
__device__ __forceinline__ void from_a(float v, float s, __half& o) { o = __float2half_rn(v * s); }
__device__ __forceinline__ void from_a(float v, float s, __nv_bfloat16& o) { o = __float2bfloat16_rn(v * s); }

// Vector load (read-only path) and store of V consecutive elements: one
// 8- or 16-byte access.
template <int B> struct VecOf;
template <> struct VecOf<8> { typedef uint2 type; };
template <> struct VecOf<16> { typedef uint4 type; };
template <class S>
__device__ __forceinline__ void load_vec(const typename S::T* p, typename S::A* out, typename S::A inv) {
    typedef typename VecOf<S::V * sizeof(typename S::T)>::type VT;
    union { VT u; typename S::T t[S::V]; } r;
    r.u = __ldg(reinterpret_cast<const VT*>(p));
#pragma unroll
    for (int k = 0; k < S::V; ++k) out[k] = to_a(r.t[k], inv);
}
template <class S>
__device__ __forceinline__ void store_vec(typename S::T* p, const typename S::A* in, typename S::A scale) {
    typedef typename VecOf<S::V * sizeof(typename S::T)>::type VT;
    union { VT u; typename S::T t[S::V]; } r;
#pragma unroll
    for (int k = 0; k < S::V; ++k) from_a(in[k], scale, r.t[k]);
    *reinterpret_cast<VT*>(p) = r.u;
}
// The register stream-collide kernel keeps the scaled half-precision stores
// in their scaled units through the collision (collide_node<..., SC = true>):
// loads and stores then only convert, two values per instruction where the
// hardware packs them.
template <class S>
__device__ __forceinline__ void load_vec_raw(const typename S::T* p, float* out) {
    static_assert(S::SCALED && S::V == 4, "raw half-precision loads cover 4-node chunks");
    union { uint2 u; typename S::T t[4]; } r;
    r.u = __ldg(reinterpret_cast<const uint2*>(p));
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = to_a(r.t[k], 1.0f);
}
__device__ __forceinline__ uint32_t pack2(float a, float b, __half) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack2(float a, float b, __nv_bfloat16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}
template <class S>
__device__ __forceinline__ void store_vec_raw(typename S::T* p, const float* in) {
    static_assert(S::SCALED && S::V == 4, "raw half-precision stores cover 4-node chunks");
    uint2 u;
    u.x = pack2(in[0], in[1], typename S::T());
    u.y = pack2(in[2], in[3], typename S::T());
    *reinterpret_cast<uint2*>(p) = u;
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
// Noise of Sec. 4: counter-based random numbers, uniforms, normal deviates.
// ---------------------------------------------------------------------------
// Uniform in (0,1) from the top 23 bits, ((x >> 9) + 1/2) / 2^23; exact in FP32
// and FP64.  FP32: the 23 bits as the mantissa of a number in [1, 2), minus 1,
// plus 2^-24 -- both steps exact, so this is the same value with no integer
// to float conversion.
__device__ __forceinline__ float uni23f(uint32_t x) {
    return (__uint_as_float(0x3F800000u | (x >> 9)) - 1.0f) + 5.9604644775390625e-08f;
}
__device__ __forceinline__ double uni23d(uint32_t x) { return ((double)(x >> 9) + 0.5) * 1.1920928955078125e-07; }

// FP32: the angle 2 pi b is taken as pi + 2 pi (b - 1/2) with b - 1/2 exact, so
// the hardware sine / cosine work inside [-pi, pi] (absolute error about 4e-7,
// far inside the noise tolerance); the radius keeps the accurate logarithm,
// whose argument reaches 1 - 2^-24.
__device__ __forceinline__ void box_muller(float a, float b, float& z0, float& z1) {
    const float r = sqrtf(-2.0f * logf(a));
    float s, c;
    __sincosf(6.28318530717958647692f * (b - 0.5f), &s, &c);
    z0 = -r * c;
    z1 = -r * s;
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
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit multiplies, key bumped by the Weyl constants between rounds.
// The two draws of one node (counter words 2 = 0 and 1) run with their rounds
// interleaved, so that they share the key schedule.
__device__ __forceinline__ void philox4x32_10_x2(uint4& a, uint4& b, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t alo0 = 0xD2511F53u * a.x, ahi0 = __umulhi(0xD2511F53u, a.x);
        const uint32_t alo1 = 0xCD9E8D57u * a.z, ahi1 = __umulhi(0xCD9E8D57u, a.z);
        const uint32_t blo0 = 0xD2511F53u * b.x, bhi0 = __umulhi(0xD2511F53u, b.x);
        const uint32_t blo1 = 0xCD9E8D57u * b.z, bhi1 = __umulhi(0xCD9E8D57u, b.z);
        a = make_uint4(ahi1 ^ a.y ^ k0, alo1, ahi0 ^ a.w ^ k1, alo0);
        b = make_uint4(bhi1 ^ b.y ^ k0, blo1, bhi0 ^ b.w ^ k1, blo0);
    }
}

template <typename A>
__device__ __forceinline__ void thetas(uint32_t node, uint32_t step, uint32_t dom_id, uint64_t seed, A th[6]) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint4 r0 = make_uint4(node, step, 0u, dom_id), r1 = make_uint4(node, step, 1u, dom_id);
    philox4x32_10_x2(r0, r1, k0, k1);
    box_muller(uni23<A>(r0.x), uni23<A>(r0.y), th[0], th[1]);
    box_muller(uni23<A>(r0.z), uni23<A>(r0.w), th[2], th[3]);
    box_muller(uni23<A>(r1.x), uni23<A>(r1.y), th[4], th[5]);
}

// ---------------------------------------------------------------------------
// Per-domain parameters in the arithmetic type (no FP64 <-> FP32 conversion in
// the collision).  HotPrm (lbm_types.h) holds what every node needs and is
// read with 16-byte loads; ExtPrm holds what only the power-law, noise or
// Zou-He nodes need and is read only by those variants.
// ---------------------------------------------------------------------------
template <typename A> __device__ __forceinline__ HotPrm<A> load_hot(const DomDev& D);
template <> __device__ __forceinline__ HotPrm<float> load_hot<float>(const DomDev& D) {
    const float4* p = reinterpret_cast<const float4*>(&D.hot_f);
    const float4 a = __ldg(p), b = __ldg(p + 1);
    HotPrm<float> H;
    H.omega = a.x; H.om = a.y; H.tgx = a.z; H.tgy = a.w;
    H.rho0 = b.x; H.scale = b.y; H.inv_scale = b.z; H.pad = b.w;
    return H;
}
// The same from a descriptor held in the launch parameters.
template <typename A> __device__ __forceinline__ HotPrm<A> param_hot(const DomDev& D);
template <> __device__ __forceinline__ HotPrm<float> param_hot<float>(const DomDev& D) { return D.hot_f; }
template <> __device__ __forceinline__ HotPrm<double> param_hot<double>(const DomDev& D) { return D.hot_d; }
template <> __device__ __forceinline__ HotPrm<double> load_hot<double>(const DomDev& D) {
    const double2* p = reinterpret_cast<const double2*>(&D.hot_d);
    const double2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3);
    HotPrm<double> H;
    H.omega = a.x; H.om = a.y; H.tgx = b.x; H.tgy = b.y;
    H.rho0 = c.x; H.scale = c.y; H.inv_scale = d.x; H.pad = d.y;
    return H;
}

template <typename A>
struct ExtPrm {
    A gx, gy, kT, xi, n, tmin, tmax, tmin_pow, tmax_pow;
    int n_is_one;
    uint32_t dom_id;
    uint64_t seed;
};
template <typename A, bool NOISE, bool PL>
__device__ __forceinline__ ExtPrm<A> load_ext(const DomDev& D) {
    ExtPrm<A> X{};
    const bool f = sizeof(A) == 4;
    if (PL) {
        X.gx = (A)(f ? D.gx_f : D.gx); X.gy = (A)(f ? D.gy_f : D.gy);
        X.xi = (A)(f ? D.xi_pl_f : D.xi_pl); X.n = (A)(f ? D.n_pl_f : D.n_pl);
        X.tmin = (A)(f ? D.tau_min_f : D.tau_min); X.tmax = (A)(f ? D.tau_max_f : D.tau_max);
        X.tmin_pow = (A)(f ? D.tmin_pow_f : D.tmin_pow); X.tmax_pow = (A)(f ? D.tmax_pow_f : D.tmax_pow);
        X.n_is_one = D.n_is_one;
    }
    if (NOISE) {
        X.kT = (A)(f ? D.kT_f : D.kT);
        X.dom_id = D.domain_id;
        X.seed = D.seed;
    }
    return X;
}

// Reciprocal of the density: FP32 takes the hardware approximation (relative
// error below 2^-22, far inside the FP32 path's tolerance); FP64 divides.
template <typename A> __device__ __forceinline__ A rcp_rho(A r);
template <> __device__ __forceinline__ float rcp_rho<float>(float r) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r));
    return y;
}
template <> __device__ __forceinline__ double rcp_rho<double>(double r) { return 1.0 / r; }

// ---------------------------------------------------------------------------
// Power-law relaxation time, Sec. 5.  The shear rate of Eq. nn2 with Pi_D of
// Eq. nn3 taken from the Chapman-Enskog strain -Pi_neq / (2 rho c_s^2 tau) is
// A / tau, A = 3 sqrt|Pi_xy^2 - Pi_xx Pi_yy| / rho; nu* = xi (A/tau)^(n-1)
// (nn4, kappa = 2^(n-1)) and tau = 1/2 + 3 nu*.  g(t) = t - 1/2 - c t^(1-n),
// c = 3 xi A^(n-1), is convex for n < 1 and concave for n > 1, so Newton from
// the bracket end where g > 0 (n < 1) or g < 0 (n > 1) converges monotonically.
// ---------------------------------------------------------------------------
// FP32: the hardware base-2 logarithm (x > 0 here: a strain or a relaxation
// time) and a division by the fast reciprocal inside the Newton steps, whose
// fixed point (and so the converged tau*) does not depend on how a step is
// rounded; FP64 keeps the exact operations.
template <typename A> __device__ __forceinline__ A powa(A x, A e);
template <> __device__ __forceinline__ float powa<float>(float x, float e) { return exp2f(e * __log2f(x)); }
template <> __device__ __forceinline__ double powa<double>(double x, double e) { return exp2(e * log2(x)); }
template <typename A> __device__ __forceinline__ A divn(A a, A b);
template <> __device__ __forceinline__ float divn<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double divn<double>(double a, double b) { return a / b; }

template <typename A>
__device__ __forceinline__ A solve_tau_pl(A Astr, const ExtPrm<A>& P) {
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
        const A dg = (A)1 - divn<A>(c * om * p, t);
        A tn = t - divn<A>(g, dg);
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
// Arranged for few operations, with omega = 1/tau and
// p_i = 3 e.u + 9/2 (e.u)^2 - 3/2 u.u; the pair (i, opp(i)) shares
// 9/2 (e.u)^2 - 3/2 u.u and 3 e.u.  Shifted stores (values f - w_i rho0, of
// the size of the non-equilibrium part) relax as
//   f_i' = (1 - omega) f_i + w_i (B + R p_i),  R = omega rho, B = omega (rho - rho0);
// unshifted stores (values ~ w_i) keep the difference form
//   f_i' = f_i + omega (w_i rho (1 + p_i) - f_i),
// whose rounding error stays at the scale of f_i rather than of omega f_i.
// Returns false when rho is not a positive finite number.
// ---------------------------------------------------------------------------
template <typename A, bool SHIFT>
__device__ __forceinline__ void relax_pair(A& fi, A& fo, A e, A w, A usq, A R, A R3, A B, A om, A omega) {
    const A q = (A)4.5 * e * e - usq;
    if (SHIFT) {
        const A h = B + R * q;
        const A k = R3 * e;
        fi = om * fi + w * (h + k);
        fo = om * fo + w * (h - k);
    } else {  // here R = rho, R3 = 3 rho, B = rho
        const A h = B + R * q;
        const A k = R3 * e;
        fi = fi + omega * (w * (h + k) - fi);
        fo = fo + omega * (w * (h - k) - fo);
    }
}

// SC (shifted stores only): f holds (f - w_i rho0) * s in the store's scaled
// units, s = H.scale, and so does the result; the moments are unscaled once
// per node (exact: s is a power of two) instead of every population.
template <typename A, bool SHIFT, bool NOISE, bool PL, bool SC = false>
__device__ __forceinline__ bool collide_node(A f[9], const HotPrm<A>& H, const ExtPrm<A>& X, uint32_t node,
                                             uint32_t step) {
    static_assert(!SC || SHIFT, "scaled units are those of the shifted stores");
    const A a = (f[1] + f[5]) + f[8];  // e_x > 0
    const A b = (f[3] + f[6]) + f[7];  // e_x < 0
    const A c = (f[2] + f[5]) + f[6];  // e_y > 0
    const A d = (f[4] + f[7]) + f[8];  // e_y < 0
    const A s_ = (f[0] + (f[2] + f[4])) + (a + b);
    const A jx_ = a - b, jy_ = c - d;
    // unscaled moments (SC: one multiply each by the power of two 1/s)
    const A s = SC ? s_ * H.inv_scale : s_;
    const A jx = SC ? jx_ * H.inv_scale : jx_, jy = SC ? jy_ * H.inv_scale : jy_;
    const A rho = SHIFT ? H.rho0 + s : s;
    const A drho = SHIFT ? s : s - H.rho0;
    const bool ok = (rho > (A)0) && (rho < (A)1e30);
    const A irho = rcp_rho<A>(rho);
    A omega = H.omega, om = H.om, tgx = H.tgx, tgy = H.tgy;
    if (PL) {
        const A u1 = SC ? H.inv_scale : (A)1;  // unscaled second moments
        const A sxy = ((f[5] + f[7]) - (f[6] + f[8])) * u1;
        const A iso = SHIFT ? drho * (A)(1.0 / 3.0) : rho * (A)(1.0 / 3.0);
        const A pxx = (a + b) * u1 - iso - jx * jx * irho;
        const A pyy = (c + d) * u1 - iso - jy * jy * irho;
        const A pxy = sxy - jx * jy * irho;
        const A det = pxy * pxy - pxx * pyy;
        const A Astr = (A)3 * sqrt(fabs(det)) * irho;
        const A tau = solve_tau_pl<A>(Astr, X);
        omega = (A)1 / tau;
        om = (A)1 - omega;
        tgx = tau * X.gx;
        tgy = tau * X.gy;
    }
    const A ux = (jx + rho * tgx) * irho;
    const A uy = (jy + rho * tgy) * irho;
    const A usq = (A)1.5 * (ux * ux + uy * uy);
    // in the units of f (SC: times s)
    const A R = SHIFT ? (SC ? omega * rho * H.scale : omega * rho) : rho;
    const A B = SHIFT ? omega * (SC ? s_ : drho) : rho;
    const A R3 = (A)3 * R;
    if (SHIFT) f[0] = om * f[0] + (A)wgt(0) * (B - R * usq);
    else f[0] = f[0] + omega * ((A)wgt(0) * (B - R * usq) - f[0]);
    relax_pair<A, SHIFT>(f[1], f[3], ux, (A)wgt(1), usq, R, R3, B, om, omega);
    relax_pair<A, SHIFT>(f[2], f[4], uy, (A)wgt(2), usq, R, R3, B, om, omega);
    relax_pair<A, SHIFT>(f[5], f[7], ux + uy, (A)wgt(5), usq, R, R3, B, om, omega);
    relax_pair<A, SHIFT>(f[6], f[8], uy - ux, (A)wgt(6), usq, R, R3, B, om, omega);
    if (NOISE) {
        if (X.kT > (A)0) {
            A th[6];
            thetas<A>(node, step, X.dom_id, X.seed, th);
            const A amp = SC ? sqrt(rho * X.kT * omega * ((A)2 - omega) * (A)3) * H.scale
                             : sqrt(rho * X.kT * omega * ((A)2 - omega) * (A)3);
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
// populations 3, 6, 7 enter.  d_b is the prescribed density in the units of
// the stored values (rho_b - rho0 when SHIFT, rho_b otherwise); the shifts of
// the paired populations are equal.
template <typename A>
__device__ __forceinline__ A zou_he_excess(const DomDev& D, int side) {
    if (sizeof(A) == 4) return (A)(side == 0 ? D.drho_in_f : D.drho_out_f);
    return (A)(side == 0 ? D.drho_in : D.drho_out);
}
template <typename A>
__device__ __forceinline__ void zou_he(A f[9], int side, A d_b) {
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
}

}  // namespace lbmk

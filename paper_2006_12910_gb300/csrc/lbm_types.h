// lbm_types.h -- plain descriptors shared by the host runtime and the kernels
// of the GB300 D2Q9 library (no CUDA types, no method arithmetic).
#pragma once
#include <stdint.h>

namespace lbmk {

enum : int32_t {
    FLAG_PX = 1,   // periodic in x
    FLAG_PY = 2,   // periodic in y
    FLAG_WY = 4,   // halfway walls at y = -1/2 and y = ny - 1/2
    FLAG_IO = 8,   // Zou-He density columns at x = 0 and x = nx - 1
};

enum : uint32_t {
    ERR_UNSTABLE = 1u,  // rho <= 0 or not finite
    ERR_STATE = 2u,     // particle overlap or list capacity exceeded
    ERR_TIMEOUT = 4u,   // a bounded device wait ran out
};

// Collision parameters read by every stream-collide work item, packed for
// 16-byte loads: omega = 1/tau, om = 1 - omega, tgx/tgy = tau g (the
// velocity shift of the forcing), rho0, and the store scale and its inverse.
template <typename A>
struct alignas(16) HotPrm {
    A omega, om, tgx, tgy, rho0, scale, inv_scale, pad;
};

// One lattice domain as the kernels see it.  Populations of plane i live at
// arena[off + i*plane + y*pitch + x]; with y walls each plane also holds one
// ghost row on each side (y = -1 and y = ny, still addressed as off + i*plane
// + y*pitch + x), whose slots carry the bounced-back populations of the wall
// rows.  Per-node solid bytes, flag words and tags at
// nodes[node_off + y*pitch + x], 0 <= y < ny; the special-chunk bitmask word of
// warp segment s of row y at special[mask_off + y*seg_per_row + s] (bit =
// lane; a chunk is V nodes).
struct alignas(16) DomDev {
    HotPrm<double> hot_d;
    HotPrm<float> hot_f;
    int32_t nx, ny, pitch, flags;
    int64_t off, plane, node_off, mask_off, item_off;
    int32_t seg_per_row, V;
    int32_t p0, np;           // first particle and particle count of this domain
    int32_t n_is_one;
    // work item -> row: y = umulhi(local, spr_magic) when nonzero (exact for
    // every item of the domain), else local / seg_per_row
    uint32_t spr_magic;
    uint64_t seed;
    uint32_t domain_id, pad1;
    double tau, inv_tau, rho0, gx, gy;
    double rho_in, rho_out, drho_in, drho_out;  // open-column densities (and minus rho0)
    double kT;
    double n_pl, xi_pl, tau_min, tau_max, tmin_pow, tmax_pow;  // tmin^(1-n), tmax^(1-n)
    double lj_psi, lj_rit;
    double scale, inv_scale;  // store scale of the shifted FP16/BF16 kinds (1 otherwise)
    // FP32 copies of the collision parameters, so the FP32 path converts nothing
    float tau_f, inv_tau_f, rho0_f, gx_f, gy_f, rho_in_f, rho_out_f, drho_in_f, drho_out_f, kT_f;
    float n_pl_f, xi_pl_f, tau_min_f, tau_max_f, tmin_pow_f, tmax_pow_f, scale_f, inv_scale_f;
};

// Per-node flag words (uint16), written from the geometry on the host.
// Halfway bounce-back uses the slots of solid nodes and wall ghost rows as
// mailboxes: a fluid node whose neighbour x + e_j is solid or a ghost-row
// node carries bit j (1..8), and after its collision it writes its outgoing
// f*_j into slot opp(j) of that neighbour, the slot it pulls direction opp(j)
// from in the next step.  Pulls therefore need no patching, except at the
// wall-corner nodes of open ends (NF_CORNER: the directions whose source lies
// beyond the x range take the node's own opposite slot) and on the Zou-He
// columns.  On a solid node bits 1..8 mark instead which of its slots are
// mailboxes (slot i, when the node x + e_i is fluid); no fluid node ever reads
// the other slots of a solid node, so a chunk may overwrite those with its
// vector stores.  A chunk whose nodes all have zero flags takes the plain
// vector path without reading them.
enum : uint16_t {
    NF_SOLID = 1u << 0,
    NF_ZH_IN = 1u << 9,    // Zou-He inlet node (x = 0)
    NF_ZH_OUT = 1u << 10,  // Zou-He outlet node (x = nx - 1)
    NF_CORNER = 1u << 11,  // wall-corner node of an open end
};

// Particle data on the device (Sec. 3).  State is double precision.
struct PartState {
    double x, y, U, V, Om, th;
};
struct PartStatic {
    double R, rho_p, m, I;
    double inv_m, inv_I, buoy;  // 1/m_p, 1/I_p and (rho_p - rho0)/rho_p (Eq. MP5)
    int32_t dom, fixed;
    int32_t link_cap, flip_cap;
    int64_t link_off, flip_off;
};

// Pair force of Eq. MP2 for one node offset o within the threshold r_it:
// psi (|o|/r_it)^-13 (-o)/|o|, the force on a node from a node at +o.
constexpr int LJ_TAB = 128;
struct LjEntry {
    int32_t ox, oy;
    double fx, fy;
};

constexpr int DIAG_N = 13;  // F_links(2), T_links, F_cu(2), T_cu, F_lj(2), T_lj, n_cov, n_unc, m_cov, m_unc

}  // namespace lbmk

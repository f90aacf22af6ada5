// k_part.cu -- particle kernel of the D2Q9 hot path (arXiv:2006.12910 Sec. 3).
//
// Three launches per timestep, each with CTAs per particle in roles that
// run side by side.  The stored populations are f*(t), post-collision; the
// particle state, the link / flip lists, the node tags of side changes and
// the Eq. MP2 sums are double-buffered by the parity of the step they belong
// to, so a launch reads the copies of one step while it writes those of
// another.
//
//  A. (launch 1 of step t) forces at t: Eq. MP1 over the boundary links of
//     the rasterisation at t (each link's slots belong to this particle
//     alone) and the covered / uncovered-node force of Eq. MP3 from the node
//     moments that the stream-collide pass of the previous step wrote while
//     producing f*(t), plus the Eq. MP2 force at t summed two steps earlier;
//     FP64 totals (Eqs. MP3-MP4) and the Newton-Euler update of Eqs. MP5-MP6.
//     With the forces, Eqs. MP7-MP8 as a pre-stream exchange: for the link
//     r_v -> r_v + e_k the slot that r_v + e_k pulls next receives
//     f*_{-k}(r_v + e_k) + 2 rho0 omega_k (u_b . e_k) / c_s^2 and the slot r_v
//     pulls receives f*_k(r_v) minus the same, so the plain pull stream
//     realises the moving bounce-back on both sides.
// After launch 1 of step t has written the state of t+1, beside the
// stream-collide pass of step t:
//  B, C. (launch 2) for step t+1: re-rasterisation at r_c(t+2) = r_c(t+1) +
//     U_p(t+1), which needs no force of t+1 (new link list and the nodes that
//     change side, tagged for the stream-collide pass of t+1), and the work
//     items near the particle for step t+2;
//  D. (launch 3) Eq. MP2 at t+2, which needs positions only.
// At set-up the same roles run for the current step.
#include "kernels.h"
#include "lbm_dev.cuh"

namespace lbmk {

constexpr int PBLOCK = 256;
constexpr int A_BLOCK = 160;  // role A launched alone: five warps
constexpr int BC_BLOCK = 256;  // roles B + C (rasterisation, near-item marks)
constexpr int MAX_WARPS = (PBLOCK > BC_BLOCK ? PBLOCK : BC_BLOCK) / 32;

__device__ __forceinline__ double min_image(double d, int L, bool periodic) {
    if (!periodic) return d;
    while (d >= 0.5 * L) d -= L;
    while (d < -0.5 * L) d += L;
    return d;
}

// Strictly inside the disk (Sec. 3 rasterisation); no FMA contraction so the
// decision is the same as a plain double evaluation anywhere.
__device__ __forceinline__ bool inside_disk(const DomDev& D, double px, double py, double R, double x, double y) {
    const double dx = min_image(__dsub_rn(x, px), D.nx, D.flags & FLAG_PX);
    const double dy = min_image(__dsub_rn(y, py), D.ny, D.flags & FLAG_PY);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) < __dmul_rn(R, R);
}

__device__ __noinline__ bool is_surface(const DomDev& D, double px, double py, double R, int x, int y) {
    if (!inside_disk(D, px, py, R, x, y)) return false;
#pragma unroll 1
    for (int i = 1; i < 9; ++i)
        if (!inside_disk(D, px, py, R, x + cx(i), y + cy(i))) return true;
    return false;
}

// Wrap a node into the domain; false when it leaves through a non-periodic
// edge.  Nodes handled here lie within R + 8 of the domain, and a particle
// on a periodic axis has 2R + 8 below the period, so one period step (no
// division) brings them in.
__device__ __forceinline__ bool wrap_node(const DomDev& D, int& x, int& y) {
    if (x < 0 || x >= D.nx) {
        if (!(D.flags & FLAG_PX)) return false;
        x += x < 0 ? D.nx : -D.nx;
    }
    if (y < 0 || y >= D.ny) {
        if (!(D.flags & FLAG_PY)) return false;
        y += y < 0 ? D.ny : -D.ny;
    }
    return true;
}

// Box of lattice nodes around a disk, in unwrapped coordinates.
struct Box {
    int x0, y0, w, h;
    __device__ int n() const { return w * h; }
};
__device__ __forceinline__ Box disk_box(double px, double py, double R) {
    Box b;
    b.x0 = (int)floor(px - R) - 1;
    b.y0 = (int)floor(py - R) - 1;
    b.w = (int)ceil(px + R) + 1 - b.x0 + 1;
    b.h = (int)ceil(py + R) + 1 - b.y0 + 1;
    return b;
}

// Inside test of node (xu, yu) (unwrapped, near the disk).  An FP32 distance
// decides when it is clear of the rim by more than its error bound; within
// that margin the exact FP64 evaluation (wrapped coordinates when `wrapped`,
// as the rasterisation uses, unwrapped otherwise) decides, so the answer is
// always that of the plain FP64 test.
struct DiskF {
    double px, py, R;
    int cx, cy;
    float fx, fy, R2, margin;
};
__device__ __noinline__ DiskF make_diskf(double px, double py, double R) {
    DiskF d;
    d.px = px; d.py = py; d.R = R;
    d.cx = (int)floor(px); d.cy = (int)floor(py);
    d.fx = (float)(px - d.cx); d.fy = (float)(py - d.cy);
    d.R2 = (float)(R * R);
    d.margin = 1e-3f * fmaxf(1.0f, d.R2 * 0.01f) + 1e-4f;
    return d;
}
// Integer minimum image, in [-L/2, L/2), of a node offset along a periodic
// axis.  Offsets here (a node within R + 8 of the domain against a centre in
// it, with 2R + 8 below the period) are under 5L/2 in magnitude, so two
// period steps (no division) suffice.
__device__ __forceinline__ int wrap_off(int d, int L, bool periodic) {
    if (!periodic) return d;
    if (2 * d >= L) {
        d -= L;
        if (2 * d >= L) d -= L;
    } else if (2 * d < -L) {
        d += L;
        if (2 * d < -L) d += L;
    }
    return d;
}
// The exact FP64 decision near the rim (out of line: rarely taken, and the
// particle kernel is bound by instruction fetch, so its code is kept small).
__device__ __noinline__ bool inside_exact(const DomDev& D, const DiskF& k, int xu, int yu, bool wrapped) {
    if (wrapped) {
        int x = xu, y = yu;
        if (!wrap_node(D, x, y)) { x = xu; y = yu; }
        return inside_disk(D, k.px, k.py, k.R, x, y);
    }
    return inside_disk(D, k.px, k.py, k.R, xu, yu);
}
__device__ __forceinline__ bool inside_f(const DomDev& D, const DiskF& k, int xu, int yu, bool wrapped) {
    const int dxi = wrap_off(xu - k.cx, D.nx, D.flags & FLAG_PX), dyi = wrap_off(yu - k.cy, D.ny, D.flags & FLAG_PY);
    const float dx = (float)dxi - k.fx, dy = (float)dyi - k.fy;
    const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    if (d2 < k.R2 - k.margin) return true;
    if (d2 > k.R2 + k.margin) return false;
    return inside_exact(D, k, xu, yu, wrapped);
}

template <class S>
__device__ __forceinline__ double full_pop(const typename S::T* base, const DomDev& D, int i, int64_t ni) {
    const double v = (double)to_a(base[(int64_t)i * D.plane + ni], (typename S::A)D.inv_scale);
    return S::SHIFT ? v + wgt(i) * D.rho0 : v;
}

// Exclusive block scan of small non-negative counts; returns the block total.
__device__ __noinline__ int block_scan(int c, int* sh_warp, int& excl) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sh_warp[w] = incl;
    __syncthreads();
    int wbase = 0, total = 0;
    const int nw = (int)(blockDim.x >> 5);
    for (int k = 0; k < nw; ++k) {
        if (k < w) wbase += sh_warp[k];
        total += sh_warp[k];
    }
    excl = wbase + incl - c;
    __syncthreads();
    return total;
}

// Two exclusive block scans at once (the counts packed in one 64-bit word, so
// one pass of shuffles and barriers); returns both block totals.
__device__ __noinline__ void block_scan2(int c0, int c1, long long* sh_warp2, int& excl0, int& excl1, int& total0,
                                         int& total1) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long c = ((long long)c1 << 32) | (unsigned)c0;
    long long incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sh_warp2[w] = incl;
    __syncthreads();
    long long wbase = 0, total = 0;
    const int nw = (int)(blockDim.x >> 5);
    for (int k = 0; k < nw; ++k) {
        if (k < w) wbase += sh_warp2[k];
        total += sh_warp2[k];
    }
    const long long ex = wbase + incl - c;
    excl0 = (int)(unsigned)(ex & 0xffffffffll);
    excl1 = (int)(ex >> 32);
    total0 = (int)(unsigned)(total & 0xffffffffll);
    total1 = (int)(total >> 32);
    __syncthreads();
}

// Warps 5-7 of role A (96 threads) prepare the LJ-type repulsion as one group
// with their own named barrier, so the link and flip warps never wait for them.
constexpr int LJ_W0 = 5, LJ_NT = 96;
__device__ __forceinline__ void lj_sync() { asm volatile("bar.sync 1, 96;" ::: "memory"); }

// Exclusive scan of small counts over the LJ group (gt = thread index in the
// group); returns the group total.  sh holds one int per warp of the group.
__device__ __noinline__ int lj_scan(int c, int gt, int* sh, int& excl) {
    const int lane = gt & 31, w = gt >> 5;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sh[w] = incl;
    lj_sync();
    int wbase = 0, total = 0;
#pragma unroll
    for (int k = 0; k < LJ_NT / 32; ++k) {
        if (k < w) wbase += sh[k];
        total += sh[k];
    }
    excl = wbase + incl - c;
    lj_sync();
    return total;
}

// Fixed-order sum over the lanes of a warp (lane 0 gets the total).
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

constexpr int PB_CAP = 4096;   // nodes of a shared-memory inside bitmap
constexpr int MAXNEAR = 64;     // nearby particles considered per particle


// Inside nodes of one row yu of a disk, as the x range [x, y] (unwrapped; x > y
// when the row misses the disk).  The disk's rows are convex and inside_f gives
// the exact FP64 decision, so an estimate from the circle equation corrected by
// a few inside_f tests at the ends yields exactly the nodes the per-node test
// would accept.
constexpr int RR_MAX = 64;  // rows of a box handled by ranges
__device__ __noinline__ int2 row_range(const DomDev& D, const DiskF& k, int yu, bool wrapped) {
    const int dyi = wrap_off(yu - k.cy, D.ny, D.flags & FLAG_PY);
    const float dy = (float)dyi - k.fy;
    const float s2 = (float)k.R * (float)k.R - dy * dy;
    int xl, xr;
    if (s2 >= 0.0f) {
        const float sx = sqrtf(s2);
        xl = k.cx + (int)ceilf(k.fx - sx);
        xr = k.cx + (int)floorf(k.fx + sx);
    } else {
        xl = 1;
        xr = 0;
    }
    if (xl > xr) {  // the estimate misses: the node nearest the centre decides
        const int xc = k.cx + (k.fx >= 0.5f ? 1 : 0);
        if (!inside_f(D, k, xc, yu, wrapped)) return make_int2(1, 0);
        xl = xr = xc;
    }
#pragma unroll 1
    while (inside_f(D, k, xl - 1, yu, wrapped)) --xl;
#pragma unroll 1
    while (xl <= xr && !inside_f(D, k, xl, yu, wrapped)) ++xl;
#pragma unroll 1
    while (inside_f(D, k, xr + 1, yu, wrapped)) ++xr;
#pragma unroll 1
    while (xr >= xl && !inside_f(D, k, xr, yu, wrapped)) --xr;
    return make_int2(xl, xr);
}

// Surface node of a disk (inside, with an 8-neighbour outside), unwrapped
// coordinates near the disk, using the FP32 test with its exact fallback.
__device__ __noinline__ bool is_surface_f(const DomDev& D, const DiskF& k, int x, int y) {
    if (!inside_f(D, k, x, y, false)) return false;
#pragma unroll 1
    for (int i = 1; i < 9; ++i)
        if (!inside_f(D, k, x + cx(i), y + cy(i), false)) return true;
    return false;
}

// Position at t+1 from the state at t (Sec. 3: r_c(t+1) = r_c(t) + U_p(t)).
// Periodic wrap c - L floor(c / L); inside [0, L(1 - 1e-9)) the floor is 0,
// so the FP64 division (slow here) runs only near or beyond the ends, and
// the result is the same as evaluating the formula everywhere.
__device__ __forceinline__ double wrap_coord(double c, int L) {
    if (c >= 0.0 && c < (double)L * (1.0 - 1e-9)) return c;
    return c - L * floor(c / L);
}
__device__ __forceinline__ void next_position(const DomDev& D, const PartState& q, bool fixed, double& x, double& y) {
    if (fixed) { x = q.x; y = q.y; return; }
    x = q.x + q.U;
    y = q.y + q.V;
    if (D.flags & FLAG_PX) x = wrap_coord(x, D.nx);
    if (D.flags & FLAG_PY) y = wrap_coord(y, D.ny);
}

// Shared memory of one CTA; roles A / D and role B use disjoint parts of a union.
constexpr int NB_MAX = 4, NB_W = 32;  // inside bitmaps of up to 4 nearby disks, boxes up to 32 x 32
constexpr int SURF_CAP = 1024;         // box nodes per LJ chunk, so at most this many surface nodes
struct SmemA {
    double wsum[PBLOCK / 32][DIAG_N];  // per-warp partial sums
    short2 sxy[SURF_CAP];              // surface nodes of one chunk of the box, relative to its corner (LJ group)
    double2 arm[SURF_CAP];             // their torque arms
    int lj_ns;
    int2 rng[RR_MAX];                  // inside range of each row of the box (LJ surface list)
    int nb_h[NB_MAX];                  // half side of each nearby disk's bitmap (0: none)
    float nb_lim[MAXNEAR];             // reach of each nearby disk: R + r_it + 2
    uint8_t nbm[NB_MAX][NB_W * NB_W];  // inside tests of a nearby disk around its centre node
    uint8_t bm[PB_CAP];
    double lj_fx[LJ_TAB], lj_fy[LJ_TAB];
    int lj_ox[LJ_TAB], lj_oy[LJ_TAB];
};
struct SmemB {
    uint8_t bnew[PB_CAP], bold[PB_CAP], node_st[PB_CAP];
    uint16_t res[PB_CAP];  // per box node: link bits 1-8, side change (9), inside the new disk (10)
};

// What the rasterisation of one particle needs to classify a box node.
struct RastCtx {
    const DomDev* D;
    const uint8_t* solid;
    const SmemB* sm;
    const DiskF* near_d;
    int nn;
    Box U;
    bool use_bm, advance;
    double nxp, nyp, qx, qy, R;
};

// Inside the disk at t+1 (newdisk) or at t, by the bitmap or the exact test.
__device__ __noinline__ bool rast_in(const RastCtx& c, bool newdisk, int xu, int yu) {
    if (c.use_bm) {
        const int i = (yu - c.U.y0) * c.U.w + (xu - c.U.x0);
        return (newdisk ? c.sm->bnew[i] : c.sm->bold[i]) != 0;
    }
    int x = xu, y = yu;
    if (!wrap_node(*c.D, x, y)) { x = xu; y = yu; }
    return newdisk ? inside_disk(*c.D, c.nxp, c.nyp, c.R, x, y) : inside_disk(*c.D, c.qx, c.qy, c.R, x, y);
}

// Node i of the box U (lattice order): its links (bit k: r_v + e_k outside
// every disk and not solid), whether it changes side between t and t+1
// (bit 9) and whether it is inside the disk at t+1 (bit 10); node = its
// index in the domain.  ovl is set when it lies inside another disk too.
__device__ __noinline__ uint32_t node_info(const RastCtx& c, int i, int& node, bool& ovl) {
    const DomDev& D = *c.D;
    node = 0;
    const int xu = c.U.x0 + i % c.U.w, yu = c.U.y0 + i / c.U.w;
    int x = xu, y = yu;
    if (!wrap_node(D, x, y)) return 0u;
    node = y * D.pitch + x;
    const bool solid_here = c.use_bm ? c.sm->node_st[i] == 1 : c.solid[D.node_off + node] != 0;
    const bool now = rast_in(c, true, xu, yu);
    uint32_t r = now ? (1u << 10) : 0u;
    if (now) {
#pragma unroll 1
        for (int j = 0; j < c.nn; ++j)
            if (inside_f(D, c.near_d[j], xu, yu, true)) ovl = true;
        if (!solid_here) {
#pragma unroll 1
            for (int k = 1; k < 9; ++k) {
                const int fxu = xu + cx(k), fyu = yu + cy(k);
                if (c.use_bm) {
                    if (c.sm->node_st[(fyu - c.U.y0) * c.U.w + (fxu - c.U.x0)] != 0) continue;
                } else {
                    int fx = fxu, fy = fyu;
                    if (!wrap_node(D, fx, fy)) continue;
                    if (c.solid[D.node_off + (int64_t)fy * D.pitch + fx]) continue;
                }
                bool in_any = rast_in(c, true, fxu, fyu);
#pragma unroll 1
                for (int j = 0; j < c.nn && !in_any; ++j) in_any = inside_f(D, c.near_d[j], fxu, fyu, true);
                if (!in_any) r |= 1u << k;
            }
        }
    }
    if (c.advance && !solid_here && now != rast_in(c, false, xu, yu)) r |= 1u << 9;
    return r;
}
union SmemU {
    SmemA A;
    SmemB B;
};

// LO..HI: the roles an instantiation can run (the code of the others is left
// out, so each launch fetches only its own instructions); role0 >= LO picks
// the first role of the launch.
template <class S, int LO, int HI>
__global__ void __launch_bounds__(LO >= 2 ? BC_BLOCK : PBLOCK) k_particle_step(PartArgs a, int modes, int role0) {
    // A programmatic dependent launch waits here for the kernels before it
    // (completion and memory flush); otherwise this returns at once.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    typedef typename S::A A;
    // 0: forces, exchange and Newton-Euler; 1: Eq. MP2 for the next step;
    // 2: rasterisation; 3: near-item marks
    const int rel = (int)blockIdx.x / a.np;
    const int role = role0 + rel;
    const int p = (int)blockIdx.x - rel * a.np;
    // Independent loads first (step counter, static data, both parities of
    // the state), so the prologue waits for one round trip, then the domain.
    // PL_AHEAD: launched after role A of step t-1 for step t (or t+1), whose
    // state counter is not yet published: t from the word role A stored.
    const int64_t t = (modes & PL_AHEAD) ? *a.pstep : *a.ctr;
    const PartStatic st = a.st[p];
    const PartState q0 = a.state[p], q1 = a.state[(int64_t)a.np + p];
    // role A: the list lengths of both parities in the same round trip
    int nl2[2] = {0, 0}, nf2[2] = {0, 0};
    if (LO == 0 && role == 0) {
        nl2[0] = a.nlinks[p];
        nl2[1] = a.nlinks[(int64_t)a.np + p];
        nf2[0] = a.nflips[p];
        nf2[1] = a.nflips[(int64_t)a.np + p];
    }
    const bool advance = modes & PL_ADVANCE;
    // The near-item list of step t+2 is touched by nobody during this step.
    if (role == 0 && p == 0 && threadIdx.x == 0 && advance) {
        a.near_cnt[(t + 2) % 3] = 0;
        *a.pstep = t + 1;
    }
    const int need = role == 0 ? (PL_FORCES | PL_SWAP) : role == 1 ? PL_LJ : role == 2 ? PL_RASTER : PL_MARK;
    if (!(modes & need)) return;
    if (st.dom < 0) return;
    const DomDev D = a.one_domain ? a.dom0 : a.doms[st.dom];  // one domain: from the launch parameters
    if (p - D.p0 >= D.np) return;
    const int par = (int)(t & 1);
    const PartState* S0 = a.state + (int64_t)par * a.np;
    const PartState q = par ? q1 : q0;
    const double R = st.R;
    const bool px = D.flags & FLAG_PX, py = D.flags & FLAG_PY;
    typename S::T* base = static_cast<typename S::T*>(a.arena) + D.off;

    __shared__ __align__(16) unsigned char smem_raw[sizeof(SmemU)];
    SmemU& sm = *reinterpret_cast<SmemU*>(smem_raw);
    __shared__ double tot[DIAG_N];
    __shared__ int lj_n, nnear;
    __shared__ int sh_warp[MAX_WARPS];
    __shared__ long long sh_warp2[MAX_WARPS];
    __shared__ int near[MAXNEAR];
    __shared__ DiskF near_d[MAXNEAR];
    if (LO == 0 && role == 0) {
        // ------------------------------------------------------------------ role A
        // The boundary velocity of the link exchange is the particle's
        // velocity at mid-step, u_b = U_mid + Omega_mid x (r_b - r_c), on both
        // sides of each link (Eq. MP1 and Eqs. MP7-MP8), so role A runs in three
        // phases:
        //  1. warps 0-3, over the links: the part of Eq. MP1 that does not
        //     depend on u_b, -2 f'_k e_k (with its torque), and the sums that
        //     give the link friction matrix Z = sum c_k a_k a_k^T,
        //     c_k = 2 rho0 omega_k / c_s^2, a_k = (e_kx, e_ky, (r_b - r_c) x e_k);
        //     warp 4: covered / uncovered nodes.  The Eq. MP2 force at t was
        //     summed by role D two steps earlier (or at set-up).
        //  2. thread 0: Eqs. MP5-MP6 with the force -Z X_mid of the moving
        //     boundary, X_mid = (X(t) + X(t+1)) / 2: the SPD system
        //     (M + Z/2) X_mid = M X(t) + G/2 by its adjugate, X(t+1) = 2 X_mid - X(t).
        //  3. warps 0-3: the exchange of Eqs. MP7-MP8 with u_b(X_mid) on each
        //     link's two slots (they belong to this link alone).
        // FP64 issue is scarce on this part, so the per-link work is kept off
        // it.  With r_c = (i + fx, j + fy), i, j integers, the arm of a link
        // is r_b - r_c = (m_x - fx, m_y - fy) with m half-integers, and
        // (r_b - r_c) x e_k = A/2 - B_k, A = 2 (m_x e_ky - m_y e_kx) an integer,
        // B_k = fx e_ky - fy e_kx.  Every entry of Z is then a combination of
        // integer sums over the links (weights W_k = c_k * 6 / rho0 = 4 on axis
        // links, 1 on diagonal ones) with fx, fy applied once per particle, and
        // the torque of the motion-independent force is -sum f' A + 2 fx S_y
        // - 2 fy S_x with S = sum f' e_k: three FP64 additions per link.
        // Each warp sums its own terms by shuffles in a fixed order and the
        // warps are added in a fixed order, so the totals are deterministic.
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        __shared__ double wsa[A_BLOCK / 32][DIAG_N];  // per-warp partial sums
        __shared__ int wsi[4][5];                     // per-warp integer sums Ixx, Ixy, Iyy, J1, J2
        __shared__ long long wsk[4];                  // per-warp integer sum K
        __shared__ double xmid[3];
        const int32_t* links = a.links + (int64_t)par * a.links_total;
        const int32_t* flips = a.flips + (int64_t)par * a.flips_total;
        const int nl = nl2[par], nf = nf2[par];
        // the Eq. MP2 sums of t, loaded now by the threads that add them up
        double ljc = 0.0;
        if (threadIdx.x >= 6 && threadIdx.x < 9 && D.lj_psi != 0.0 && D.lj_rit > 0.0)
            ljc = a.ljf[4 * ((int64_t)par * a.np + p) + (threadIdx.x - 6)];
        const bool forces = modes & PL_FORCES, swap = modes & PL_SWAP;
        double acc[DIAG_N];
#pragma unroll
        for (int c = 0; c < DIAG_N; ++c) acc[c] = 0.0;
        const A scl = (A)D.scale, inv = (A)D.inv_scale;
        // integer node of the centre and the fractional offset
        const double fl_x = floor(q.x), fl_y = floor(q.y);
        const int ix = (int)fl_x, iy = (int)fl_y;
        const double fxd = q.x - fl_x, fyd = q.y - fl_y;
        // one round of four links per thread covers nl <= 512: the slot
        // values then stay in registers from phase 1 to phase 3
        const bool one_round = nl <= 4 * 128;
        A va[4], vb[4];
        if (warp < 4) {
            int Ixx = 0, Ixy = 0, Iyy = 0, J1 = 0, J2 = 0;
            long long K = 0;
            if (forces) {
                // four links per thread at a time: the eight slot loads are in
                // flight before any is used
#pragma unroll 1
                for (int l0 = threadIdx.x; l0 < nl; l0 += 4 * 128) {
                    int kk[4], a2s[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int l = l0 + 128 * u;
                        const int32_t e = l < nl ? links[st.link_off + l] : 0;
                        const int node = e >> 3, k = (e & 7) + 1;
                        const int vy = node / D.pitch, vx = node - vy * D.pitch;
                        int fx = vx + cx(k), fy = vy + cy(k);
                        wrap_node(D, fx, fy);
                        kk[u] = k;
                        const int mx2 = 2 * wrap_off(vx - ix, D.nx, px) + cx(k);
                        const int my2 = 2 * wrap_off(vy - iy, D.ny, py) + cy(k);
                        a2s[u] = mx2 * cy(k) - my2 * cx(k);
                        if (l < nl) {
                            va[u] = to_a(base[(int64_t)k * D.plane + node], inv);
                            vb[u] = to_a(base[(int64_t)opp(k) * D.plane + (int64_t)fy * D.pitch + fx], inv);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (l0 + 128 * u >= nl) break;
                        const int k = kk[u], ex = cx(k), ey = cy(k), a2 = a2s[u];
                        // f'_{-k}(r_v + e_k), the population that r_v pulls across the link
                        const double fo = S::SHIFT ? (double)vb[u] + wgt(opp(k)) * D.rho0 : (double)vb[u];
                        if (ex) acc[0] += ex > 0 ? fo : -fo;
                        if (ey) acc[1] += ey > 0 ? fo : -fo;
                        acc[2] += fo * (double)a2;
                        const int W = k <= 4 ? 4 : 1;
                        Ixx += W * ex * ex;
                        Ixy += W * ex * ey;
                        Iyy += W * ey * ey;
                        J1 += W * ex * a2;
                        J2 += W * ey * a2;
                        K += (long long)(W * a2) * a2;
                    }
                }
            }
            if (forces && __any_sync(0xffffffffu, threadIdx.x < nl)) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double x = warp_sum(acc[c]);
                    if (lane == 0) wsa[warp][c] = x;
                }
                const int r0 = __reduce_add_sync(0xffffffffu, Ixx), r1 = __reduce_add_sync(0xffffffffu, Ixy);
                const int r2 = __reduce_add_sync(0xffffffffu, Iyy), r3 = __reduce_add_sync(0xffffffffu, J1);
                const int r4 = __reduce_add_sync(0xffffffffu, J2);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) K += __shfl_down_sync(0xffffffffu, K, o);
                if (lane == 0) {
                    wsi[warp][0] = r0;
                    wsi[warp][1] = r1;
                    wsi[warp][2] = r2;
                    wsi[warp][3] = r3;
                    wsi[warp][4] = r4;
                    wsk[warp] = K;
                }
            } else if (lane == 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) wsa[warp][c] = 0.0;
#pragma unroll
                for (int c = 0; c < 5; ++c) wsi[warp][c] = 0;
                wsk[warp] = 0;
            }
        } else if (warp == 4) {
            // Covered (+) / uncovered (-) nodes: F = +- rho (u - U_p), with rho and
            // sum f* e of the node at t written by the previous stream-collide pass.
            if (forces) {
#pragma unroll 1
                for (int l = lane; l < nf; l += 32) {
                    const int32_t e = flips[st.flip_off + l];
                    const int node = e >> 1;
                    const bool cov = e & 1;
                    const int y = node / D.pitch, x = node - y * D.pitch;
                    const double* m = a.flipmom + 3 * ((int64_t)par * a.flips_total + st.flip_off + l);
                    const double r = m[0], jx = m[1], jy = m[2];
                    const double ux = (jx - 0.5 * r * D.gx) / r, uy = (jy - 0.5 * r * D.gy) / r;
                    const double sg = cov ? 1.0 : -1.0;
                    const double Fx = sg * r * (ux - q.U), Fy = sg * r * (uy - q.V);
                    const double rx = min_image(x - q.x, D.nx, px), ry = min_image(y - q.y, D.ny, py);
                    acc[3] += Fx;
                    acc[4] += Fy;
                    acc[5] += rx * Fy - ry * Fx;
                    if (cov) { acc[9] += 1.0; acc[11] += r; }
                    else { acc[10] += 1.0; acc[12] += r; }
                }
            }
            const bool any = forces && nf > 0;
#pragma unroll
            for (int c = 3; c < DIAG_N; ++c) {
                if (c >= 6 && c < 9) continue;
                const double x = any ? warp_sum(acc[c]) : 0.0;
                if (lane == 0) wsa[4][c] = x;
            }
        }
        __syncthreads();
        __shared__ long long itot[6];
        if (forces && threadIdx.x < DIAG_N) {
            // component groups: link sums 0-2 (warps 0-3), covered/uncovered 3-5
            // and 9-12 (warp 4), LJ 6-8 (role D, earlier launch); fixed order
            const int c = threadIdx.x;
            double x = 0.0;
            if (c < 3) x = ((wsa[0][c] + wsa[1][c]) + wsa[2][c]) + wsa[3][c];
            else if (c < 6 || c >= 9) x = wsa[4][c];
            else x = ljc;
            tot[c] = x;
            if (c >= 3) a.diag[(int64_t)p * DIAG_N + c] = x;
        } else if (forces && threadIdx.x >= 32 && threadIdx.x < 38) {
            const int c = threadIdx.x - 32;
            itot[c] = c < 5 ? (long long)wsi[0][c] + wsi[1][c] + wsi[2][c] + wsi[3][c]
                            : wsk[0] + wsk[1] + wsk[2] + wsk[3];
        }
        __syncthreads();
        __shared__ double zsh[6], f0sh[3];
        if (threadIdx.x == 0) {
            // Eqs. MP5, MP6 (velocities) with r_c(t+1) = r_c(t) + U_p(t).  One
            // thread, FP64: the dependent chain is kept short (one reciprocal).
            PartState n = q;
            double xm[3] = {q.U, q.V, q.Om};
            double F0x = 0.0, F0y = 0.0, T0 = 0.0, z[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            if (forces) {
                // the motion-independent link force and torque
                F0x = -2.0 * tot[0];
                F0y = -2.0 * tot[1];
                T0 = -tot[2] + 2.0 * fxd * tot[1] - 2.0 * fyd * tot[0];
                // Z = rho0/6 x (integer sums with the fractional offset applied)
                const double Ixx = (double)itot[0], Ixy = (double)itot[1], Iyy = (double)itot[2];
                const double J1 = (double)itot[3], J2 = (double)itot[4], Kd = (double)itot[5];
                const double r6 = D.rho0 / 6.0;
                z[0] = r6 * Ixx;
                z[1] = r6 * Ixy;
                z[2] = r6 * (0.5 * J1 - fxd * Ixy + fyd * Ixx);
                z[3] = r6 * Iyy;
                z[4] = r6 * (0.5 * J2 - fxd * Iyy + fyd * Ixy);
                z[5] = r6 * (0.25 * Kd - (fxd * J2 - fyd * J1) + fxd * fxd * Iyy - 2.0 * fxd * fyd * Ixy +
                             fyd * fyd * Ixx);
            }
            if (advance && !st.fixed) {
                if (forces) {
                    // G = motion-independent force and torque + buoyancy term
                    const double G0 = (F0x + tot[3]) + tot[6] + st.m * st.buoy * D.gx;
                    const double G1 = (F0y + tot[4]) + tot[7] + st.m * st.buoy * D.gy;
                    const double G2 = (T0 + tot[5]) + tot[8];
                    // (M + Z/2) X_mid = M X(t) + G/2, M + Z/2 symmetric positive
                    // definite: X_mid = adj(M + Z/2) r / det(M + Z/2)
                    const double a00 = st.m + 0.5 * z[0], a01 = 0.5 * z[1], a02 = 0.5 * z[2];
                    const double a11 = st.m + 0.5 * z[3], a12 = 0.5 * z[4], a22 = st.I + 0.5 * z[5];
                    const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
                    const double c11 = a00 * a22 - a02 * a02, c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
                    const double inv_det = 1.0 / (a00 * c00 + a01 * c01 + a02 * c02);
                    const double r0 = st.m * q.U + 0.5 * G0, r1 = st.m * q.V + 0.5 * G1, r2 = st.I * q.Om + 0.5 * G2;
                    xm[0] = (c00 * r0 + c01 * r1 + c02 * r2) * inv_det;
                    xm[1] = (c01 * r0 + c11 * r1 + c12 * r2) * inv_det;
                    xm[2] = (c02 * r0 + c12 * r1 + c22 * r2) * inv_det;
                    n.U = 2.0 * xm[0] - q.U;
                    n.V = 2.0 * xm[1] - q.V;
                    n.Om = 2.0 * xm[2] - q.Om;
                }
                next_position(D, q, false, n.x, n.y);
                n.th = q.th + q.Om;
                // A particle faster than a node per step, or a state that is no
                // longer finite (an unstable lattice around it), is an error; the
                // particle then stays where it was, at rest, so that later
                // launches keep rasterising a finite disk inside the domain.
                const bool ok = fabs(n.U) < 1.0 && fabs(n.V) < 1.0 && fabs(n.Om) < 1.0 && isfinite(n.x) &&
                                isfinite(n.y) && isfinite(n.th);
                if (!ok) {
                    atomicOr(a.err, ERR_STATE);
                    n = q;
                    n.U = n.V = n.Om = 0.0;
                    xm[0] = xm[1] = xm[2] = 0.0;
                }
            }
            if (advance) {
                a.state[(int64_t)(par ^ 1) * a.np + p] = n;
                if (a.rec) a.rec[((t + 1) % a.rec_cap) * a.np + p] = n;
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) zsh[c] = z[c];
            f0sh[0] = F0x;
            f0sh[1] = F0y;
            f0sh[2] = T0;
            xmid[0] = xm[0];
            xmid[1] = xm[1];
            xmid[2] = xm[2];
        }
        __syncthreads();
        // the stream-collide pass after this launch may be placed on the SMs
        // now; it waits for this launch's completion before it reads
        asm volatile("griddepcontrol.launch_dependents;");
        if (forces && warp == 4 && lane < 3) {
            // the link force of Eq. MP1 at the mid-step boundary velocity, beside the exchange
            const int c = lane;
            const int i0 = c == 0 ? 0 : (c == 1 ? 1 : 2), i1 = c == 0 ? 1 : (c == 1 ? 3 : 4),
                      i2 = c == 0 ? 2 : (c == 1 ? 4 : 5);
            a.diag[(int64_t)p * DIAG_N + c] = f0sh[c] - (zsh[i0] * xmid[0] + zsh[i1] * xmid[1] + zsh[i2] * xmid[2]);
        }
        if (swap && warp < 4) {
            // Eqs. MP7-MP8 as a pre-stream exchange with u_b at mid-step:
            // u_b . e_k = U e_kx + V e_ky + Omega (A/2 - B_k), in the store's
            // arithmetic type
            const A Um = (A)xmid[0], Vm = (A)xmid[1], Om = (A)xmid[2];
            const A fxa = (A)fxd, fya = (A)fyd, r6a = (A)(6.0 * D.rho0);
#pragma unroll 1
            for (int l0 = threadIdx.x; l0 < nl; l0 += 4 * 128) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int l = l0 + 128 * u;
                    if (l >= nl) break;
                    const int32_t e = links[st.link_off + l];
                    const int node = e >> 3, k = (e & 7) + 1;
                    const int vy = node / D.pitch, vx = node - vy * D.pitch;
                    int fx = vx + cx(k), fy = vy + cy(k);
                    wrap_node(D, fx, fy);
                    typename S::T* sa = base + (int64_t)k * D.plane + node;                          // pulled by r_v + e_k
                    typename S::T* sb = base + (int64_t)opp(k) * D.plane + (int64_t)fy * D.pitch + fx;  // pulled by r_v
                    A xa, xb;
                    if (one_round && forces) {
                        xa = va[u];
                        xb = vb[u];
                    } else {
                        xa = to_a(*sa, inv);
                        xb = to_a(*sb, inv);
                    }
                    const int mx2 = 2 * wrap_off(vx - ix, D.nx, px) + cx(k);
                    const int my2 = 2 * wrap_off(vy - iy, D.ny, py) + cy(k);
                    const A arm = (A)0.5 * (A)(mx2 * cy(k) - my2 * cx(k)) - (fxa * (A)cy(k) - fya * (A)cx(k));
                    const A ube = Um * (A)cx(k) + Vm * (A)cy(k) + Om * arm;
                    const A corr = r6a * (A)wgt(k) * ube;
                    from_a(xb + corr, scl, *sa);
                    from_a(xa - corr, scl, *sb);
                }
            }
        }
        return;
    }

    if (HI < 1) return;
    // Per-particle quantities the whole CTA uses, computed once: FP64 issue
    // is scarce on this part, so no warp repeats another's FP64 work.
    struct Uni {
        double nxp, nyp;
        Box bo, bn;  // boxes of the disk at t and at t+1
        DiskF ko, kn;
    };
    __shared__ Uni uni;
    if (threadIdx.x == 0) {  // the disk at t
        uni.bo = disk_box(q.x, q.y, R);
        uni.ko = make_diskf(q.x, q.y, R);
    } else if (threadIdx.x == 32) {  // the disk at t+1, in another warp so the two FP64 chains overlap
        double x1 = q.x, y1 = q.y;
        if (advance) next_position(D, q, st.fixed, x1, y1);
        uni.nxp = x1;
        uni.nyp = y1;
        uni.bn = disk_box(x1, y1, R);
        uni.kn = make_diskf(x1, y1, R);
    }
    __syncthreads();
    const double nxp = uni.nxp, nyp = uni.nyp;

    if (LO <= 1 && role == 1) {
        // ------------------------------------------------------------------ role D
        // Eq. MP2 on p at the step this launch advances to (t+1, or t
        // without PL_ADVANCE): it needs only positions, and r_c(t+1) =
        // r_c(t) + U_p(t) is known before the forces at t are, so the sum
        // runs off the path of the force and exchange launches.  Warps 5-7
        // prepare (their own named barrier), then all eight warps take the
        // surface nodes; fixed-order sums into ljf[(t+1) & 1].
        if (!(D.lj_psi != 0.0 && D.lj_rit > 0.0)) return;  // no pair within a zero threshold
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const DiskF kd = uni.kn;  // the disk at the target step
        const Box bd = uni.bn;
        const double cxd = nxp, cyd = nyp;
        double acc[DIAG_N];
#pragma unroll
        for (int c = 0; c < DIAG_N; ++c) acc[c] = 0.0;
        int wall_near = 0;
        if (warp >= LJ_W0) {
            // Set-up: the other particles within reach, the pair-force
            // table, the inside bitmap of this disk and those of nearby disks.
            const int gt = (int)threadIdx.x - LJ_W0 * 32;
            {
                // other particles within reach, in index order
                if (gt == 0) nnear = 0;
                lj_sync();
                for (int b0 = 0; b0 < D.np; b0 += LJ_NT) {
                    const int j = b0 + gt, p2 = D.p0 + j;
                    int hit = 0;
                    double ox = 0.0, oy = 0.0;
                    if (j < D.np && p2 != p) {
                        const PartState o = S0[p2];
                        ox = o.x;
                        oy = o.y;
                        if (advance) next_position(D, o, a.st[p2].fixed, ox, oy);
                        float dx = (float)ox - (float)cxd, dy = (float)oy - (float)cyd;
                        if (px) { const float L = (float)D.nx; dx -= L * rintf(dx / L); }
                        if (py) { const float L = (float)D.ny; dy -= L * rintf(dy / L); }
                        const float reach = (float)(R + a.st[p2].R + D.lj_rit + 4.0) + 1.0f;
                        hit = dx * dx + dy * dy <= reach * reach;
                    }
                    int excl;
                    const int tot_hit = lj_scan(hit, gt, sh_warp, excl);
                    if (hit && nnear + excl < MAXNEAR) {
                        near[nnear + excl] = p2;
                        near_d[nnear + excl] = make_diskf(ox, oy, a.st[p2].R);
                    }
                    lj_sync();
                    if (gt == 0) nnear += tot_hit;
                    lj_sync();
                }
            }
        } else {
            // Warps 0-4 meanwhile look at the wall / solid field over the box
            // of the disk: any nonzero value (or a box node beyond an open end,
            // summed on the spot below) means the wall term may not vanish.
            const Box b = bd;
#pragma unroll 1
            for (int i = threadIdx.x; i < b.n(); i += LJ_W0 * 32) {
                const int yr = i / b.w;
                int ax = b.x0 + (i - yr * b.w), ay = b.y0 + yr;
                if (!wrap_node(D, ax, ay)) {
                    if ((ax < 0 || ax >= D.nx) && !(D.flags & FLAG_PX)) wall_near = 1;
                    continue;
                }
                const double2 fw = a.ljwall[D.node_off + (int64_t)ay * D.pitch + ax];
                if (fw.x != 0.0 || fw.y != 0.0) wall_near = 1;
            }
        }
        // An isolated particle -- no other particle within reach, no nonzero
        // wall field around it -- feels no Eq. MP2 force: its sums are exactly
        // zero, so the surface list and the pair loops are skipped.
        if (!__syncthreads_or(wall_near) && nnear == 0) {
            if (threadIdx.x >= 6 && threadIdx.x < 9) {
                const int64_t tn = advance ? t + 1 : t;
                a.ljf[4 * ((int64_t)(tn & 1) * a.np + p) + (threadIdx.x - 6)] = 0.0;
            }
            return;
        }
        if (warp >= LJ_W0) {
            const int gt = (int)threadIdx.x - LJ_W0 * 32;
            {
                const int nn = nnear < MAXNEAR ? nnear : MAXNEAR;
                const Box b = bd;
                const Box e = {b.x0 - 1, b.y0 - 1, b.w + 2, b.h + 2};
                if (gt == 0) lj_n = a.lj_cnt[st.dom];
#pragma unroll 1
                for (int i = gt; i < LJ_TAB; i += LJ_NT) {
                    const LjEntry en = a.lj_tab[(int64_t)st.dom * LJ_TAB + i];
                    sm.A.lj_ox[i] = en.ox;
                    sm.A.lj_oy[i] = en.oy;
                    sm.A.lj_fx[i] = en.fx;
                    sm.A.lj_fy[i] = en.fy;
                }
                if (b.h <= RR_MAX) {
#pragma unroll 1
                    for (int r = gt; r < b.h; r += LJ_NT) sm.A.rng[r] = row_range(D, kd, b.y0 + r, false);
                } else if (e.n() <= PB_CAP) {
                    const DiskF kf = kd;
#pragma unroll 1
                    for (int i = gt; i < e.n(); i += LJ_NT)
                        sm.A.bm[i] = inside_f(D, kf, e.x0 + i % e.w, e.y0 + i / e.w, false) ? 1 : 0;
                }
                // Inside bitmaps of the nearby disks (node offsets -h..h from
                // the centre node, h = ceil(R) + 2, which holds every inside
                // node and its neighbours): a surface test of theirs becomes
                // shared-memory reads of the same FP32 / exact decisions.
                if (gt < nn) sm.A.nb_lim[gt] = (float)(near_d[gt].R + D.lj_rit) + 2.0f;
#pragma unroll 1
                for (int j = 0; j < NB_MAX; ++j) {
                    int h = 0;
                    if (j < nn) {
                        h = (int)ceilf((float)near_d[j].R) + 2;
                        if (2 * h + 1 > NB_W) h = 0;
                    }
                    if (gt == 0) sm.A.nb_h[j] = h;
                    const int side = 2 * h + 1;
#pragma unroll 1
                    for (int c = gt; h > 0 && c < side * side; c += LJ_NT) {
                        const int ly = c / side, lx = c - ly * side;
                        sm.A.nbm[j][ly * NB_W + lx] =
                            inside_f(D, near_d[j], near_d[j].cx + lx - h, near_d[j].cy + ly - h, false) ? 1 : 0;
                    }
                }
            }
        }
        __syncthreads();
        // Eq. MP2 over the surface nodes of p, by all eight warps: the force
        // from static solid and wall nodes within r_it comes per node from the
        // field precomputed with the geometry (the same table sum, taken once),
        // the force from surface nodes of nearby particles pair by pair.
        {
            const int gt = threadIdx.x;
            const int nn = nnear < MAXNEAR ? nnear : MAXNEAR;
            const Box b = bd;
            const Box e = {b.x0 - 1, b.y0 - 1, b.w + 2, b.h + 2};
            const bool use_bm = e.n() <= PB_CAP;
            const int ln = lj_n;
            const float inv_ln = ln > 0 ? 1.0f / (float)ln : 0.0f;
            const bool by_rows = b.h <= RR_MAX;
#pragma unroll 1
            for (int c0 = 0; c0 < b.n(); c0 += (by_rows ? b.n() : SURF_CAP)) {
              int ns;
              if (by_rows) {
                // surface nodes from the row ranges: a node of row y is interior
                // when x-1..x+1 lie inside the ranges of rows y-1, y and y+1
                int cnt = 0, il = 1, ir = 0;
                int2 c = make_int2(1, 0);
                if (gt < b.h) {
                    c = sm.A.rng[gt];
                    if (c.x <= c.y) {
                        const int2 up = gt > 0 ? sm.A.rng[gt - 1] : make_int2(1, 0);
                        const int2 dn = gt + 1 < b.h ? sm.A.rng[gt + 1] : make_int2(1, 0);
                        if (up.x <= up.y && dn.x <= dn.y) {
                            il = max(c.x, max(up.x, dn.x)) + 1;
                            ir = min(c.y, min(up.y, dn.y)) - 1;
                        }
                        cnt = (c.y - c.x + 1) - (ir >= il ? ir - il + 1 : 0);
                    }
                }
                int excl;
                ns = block_scan(cnt, sh_warp, excl);
#pragma unroll 1
                for (int x = c.x; cnt > 0 && x <= c.y; ++x) {
                    if (x >= il && x <= ir) continue;
                    const int xx = x - b.x0;
                    sm.A.sxy[excl] = make_short2((short)xx, (short)gt);
                    sm.A.arm[excl] = make_double2(min_image(x - cxd, D.nx, px), min_image(b.y0 + gt - cyd, D.ny, py));
                    ++excl;
                }
                __syncthreads();
              } else {
                // each thread classifies a contiguous run (lattice order); one
                // scan compacts the chunk's surface nodes with their torque arms
                const int chn = min(SURF_CAP, b.n() - c0);
                const int per = (chn + PBLOCK - 1) / PBLOCK;
                const int i0 = c0 + gt * per, i1 = min(c0 + chn, i0 + per);
                int ry = i0 / b.w, rx = i0 - ry * b.w;
                uint32_t bits = 0;  // surface flags of this thread's run (per <= 4)
#pragma unroll 1
                for (int i = i0, k = 0; i < i1; ++i, ++k) {
                    const int ay = b.y0 + ry, ax = b.x0 + rx;
                    bool surf;
                    if (use_bm) {
                        const int c = (ay - e.y0) * e.w + (ax - e.x0);
                        surf = sm.A.bm[c] != 0;
                        if (surf) {
                            bool all_in = true;
#pragma unroll 1
                            for (int kk = 1; kk < 9; ++kk) all_in &= sm.A.bm[c + cy(kk) * e.w + cx(kk)] != 0;
                            surf = !all_in;
                        }
                    } else {
                        surf = is_surface(D, cxd, cyd, R, ax, ay);
                    }
                    if (surf) bits |= 1u << k;
                    if (++rx == b.w) { rx = 0; ++ry; }
                }
                int excl;
                ns = block_scan(__popc(bits), sh_warp, excl);
                ry = i0 / b.w;
                rx = i0 - ry * b.w;
#pragma unroll 1
                for (int k = 0; bits >> k; ++k) {
                    if ((bits >> k) & 1u) {
                        int yy = ry, xx = rx + k;
                        while (xx >= b.w) { xx -= b.w; ++yy; }
                        sm.A.sxy[excl] = make_short2((short)xx, (short)yy);
                        sm.A.arm[excl] = make_double2(min_image(b.x0 + xx - cxd, D.nx, px),
                                                      min_image(b.y0 + yy - cyd, D.ny, py));
                        ++excl;
                    }
                }
                __syncthreads();
              }
                // static solids and walls: one field value per surface node
#pragma unroll 1
                for (int si = gt; si < ns; si += PBLOCK) {
                    const short2 sp = sm.A.sxy[si];
                    int ax = b.x0 + sp.x, ay = b.y0 + sp.y;
                    double2 fw;
                    if (wrap_node(D, ax, ay)) {
                        fw = a.ljwall[D.node_off + (int64_t)ay * D.pitch + ax];
                    } else {  // beyond an open end: the table sum on the spot
                        fw = make_double2(0.0, 0.0);
                        const int bx0 = b.x0 + sp.x, by0 = b.y0 + sp.y;
#pragma unroll 1
                        for (int j = 0; j < ln; ++j) {
                            int wx = bx0 + sm.A.lj_ox[j], wy = by0 + sm.A.lj_oy[j];
                            const bool wall = ((D.flags & FLAG_WY) && (wy < 0 || wy >= D.ny)) ||
                                              (wrap_node(D, wx, wy) && a.solid[D.node_off + (int64_t)wy * D.pitch + wx] != 0);
                            if (wall) { fw.x += sm.A.lj_fx[j]; fw.y += sm.A.lj_fy[j]; }
                        }
                    }
                    if (fw.x != 0.0 || fw.y != 0.0) {
                        const double rax = sm.A.arm[si].x, ray = sm.A.arm[si].y;
                        acc[6] += fw.x;
                        acc[7] += fw.y;
                        acc[8] += rax * fw.y - ray * fw.x;
                    }
                }
                // surface nodes of the other particles at a + o_w
#pragma unroll 1
                for (int pi = gt; nn > 0 && pi < ns * ln; pi += PBLOCK) {
                    int si = (int)((float)pi * inv_ln);  // pi / ln, corrected below
                    if (si * ln > pi) --si;
                    else if ((si + 1) * ln <= pi) ++si;
                    const int w = pi - si * ln;
                    const short2 sp = sm.A.sxy[si];
                    const int ax = b.x0 + sp.x, ay = b.y0 + sp.y;
                    int hits = 0;
#pragma unroll 1
                    for (int j = 0; j < nn; ++j) {
                        const DiskF& ko = near_d[j];
                        const float ddx = (float)wrap_off(ax - ko.cx, D.nx, px) - ko.fx;
                        const float ddy = (float)wrap_off(ay - ko.cy, D.ny, py) - ko.fy;
                        const float lim = sm.A.nb_lim[j];
                        if (ddx * ddx + ddy * ddy > lim * lim) continue;
                        // node b = a + o expressed in the other particle's own frame
                        const int ox = wrap_off(ax + sm.A.lj_ox[w] - ko.cx, D.nx, px);
                        const int oy = wrap_off(ay + sm.A.lj_oy[w] - ko.cy, D.ny, py);
                        const int h = j < NB_MAX ? sm.A.nb_h[j] : 0;
                        bool surf_b;
                        if (h > 0) {
                            surf_b = false;
                            if (ox > -h && ox < h && oy > -h && oy < h) {
                                const uint8_t* m = sm.A.nbm[j] + (oy + h) * NB_W + (ox + h);
                                if (*m) {
                                    bool all_in = true;
#pragma unroll 1
                                    for (int kk = 1; kk < 9; ++kk) all_in &= m[cy(kk) * NB_W + cx(kk)] != 0;
                                    surf_b = !all_in;
                                }
                            }
                        } else {
                            surf_b = is_surface_f(D, ko, ko.cx + ox, ko.cy + oy);
                        }
                        if (surf_b) ++hits;
                    }
                    if (hits) {
                        const double rax = sm.A.arm[si].x, ray = sm.A.arm[si].y;
                        const double fxw = sm.A.lj_fx[w] * hits, fyw = sm.A.lj_fy[w] * hits;
                        acc[6] += fxw;
                        acc[7] += fyw;
                        acc[8] += rax * fyw - ray * fxw;
                    }
                }
                __syncthreads();
            }
        }
#pragma unroll
        for (int c = 6; c < 9; ++c) {
            const double x = warp_sum(acc[c]);
            if (lane == 0) sm.A.wsum[warp][c] = x;
        }
        __syncthreads();
        if (threadIdx.x >= 6 && threadIdx.x < 9) {
            const int c = threadIdx.x;
            double x = 0.0;
            for (int w = 0; w < PBLOCK / 32; ++w) x += sm.A.wsum[w][c];
            const int64_t tn = advance ? t + 1 : t;
            a.ljf[4 * ((int64_t)(tn & 1) * a.np + p) + (c - 6)] = x;
        }
        return;
    }

    if (HI < 2) return;
    const int64_t t_next = advance ? t + 1 : t;
    const int wpar = (int)(t_next & 1);
    if (HI >= 3 && role == 3) {
        // ------------------------------------------------------------------ role C
        // Work items (row segments) within two nodes of the disk's boxes at t
        // and t+1 are "near": the stream-collide pass of that step runs them
        // after this kernel, and they hold every node that changes side.
        const int mpar = (int)(t_next % 3);  // three-way: the passes of t and t+1 read the other two
        const int lpar = (int)(t_next % 3);
        const Box bo = uni.bo, bn = uni.bn;
        const int x0 = min(bo.x0, bn.x0) - 2, x1 = max(bo.x0 + bo.w, bn.x0 + bn.w) + 1;
        const int y0 = min(bo.y0, bn.y0) - 2, y1 = max(bo.y0 + bo.h, bn.y0 + bn.h) + 1;
        const int seg_w = 32 * D.V;
        const int lane = threadIdx.x & 31;
        // Whole warps iterate together (every row has the same segments), so a
        // warp takes its list slots with one atomic add on the shared counter.
        const int nrows = y1 - y0 + 1;
        for (int r0 = threadIdx.x & ~31; r0 < nrows; r0 += (int)blockDim.x) {
            const int r = r0 + lane;
            int y = y0 + r, xdummy = 0;
            const bool row_ok = r < nrows && wrap_node(D, xdummy, y);
            for (int xx = x0;; xx += seg_w) {
                const int xc = xx < x1 ? xx : x1;
                int x = xc, yd = 0;
                bool need = false;
                int64_t item = 0;
                if (row_ok && wrap_node(D, x, yd)) {
                    item = D.item_off + (int64_t)y * D.seg_per_row + x / seg_w;
                    int32_t* m = a.mark + (int64_t)mpar * a.total_items + item;
                    need = atomicExch(m, (int32_t)t_next) != (int32_t)t_next;
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, need);
                if (bal) {
                    int base = 0;
                    if (lane == __ffs(bal) - 1) base = atomicAdd(a.near_cnt + lpar, __popc(bal));
                    base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
                    if (need)
                        a.near_list[(int64_t)lpar * a.total_items + base + __popc(bal & ((1u << lane) - 1u))] =
                            (int32_t)item;
                }
                if (xc == x1) break;
            }
        }
        return;
    }

    // ---------------------------------------------------------------------- role B

    // Particles whose disks at t+1 may touch this one's: they bound the exterior
    // nodes of the new links and reveal overlaps.  Warp 0 screens the
    // domain's particles 32 at a time (ballots keep index order) and stores
    // their disks at t+1.
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int total = 0;
#pragma unroll 1
        for (int b0 = 0; b0 < D.np; b0 += 32) {
            const int j = b0 + lane, p2 = D.p0 + j;
            bool hit = false;
            PartState o;
            if (j < D.np && p2 != p) {
                o = S0[p2];
                // FP32 centre distance with a one-node margin: a superset of the
                // particles within reach is all that is needed here
                float dx = (float)o.x - (float)q.x, dy = (float)o.y - (float)q.y;
                if (px) { const float L = (float)D.nx; dx -= L * rintf(dx / L); }
                if (py) { const float L = (float)D.ny; dy -= L * rintf(dy / L); }
                const float reach = (float)(R + a.st[p2].R + 6.0) + 1.0f;
                hit = dx * dx + dy * dy <= reach * reach;
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, hit);
            const int slot = total + __popc(bal & ((1u << lane) - 1u));
            if (hit && slot < MAXNEAR) {
                near[slot] = p2;
                double ox = o.x, oy = o.y;
                if (advance) next_position(D, o, a.st[p2].fixed, ox, oy);
                near_d[slot] = make_diskf(ox, oy, a.st[p2].R);
            }
            total += __popc(bal);
        }
        if (lane == 0) nnear = total;
    }
    // Union of the old and new boxes; every neighbour of a node inside either
    // disk lies in it.
    const Box bo = uni.bo, bn = uni.bn;
    Box U;
    U.x0 = min(bo.x0, bn.x0);
    U.y0 = min(bo.y0, bn.y0);
    U.w = max(bo.x0 + bo.w, bn.x0 + bn.w) - U.x0;
    U.h = max(bo.y0 + bo.h, bn.y0 + bn.h) - U.y0;
    const bool use_bm = U.n() <= PB_CAP;
    if (use_bm) {
        // 0 = fluid node in the domain, 1 = solid, 2 = outside the domain;
        // bnew / bold: inside the disk at t+1 / t.  Tiles of 32 columns x
        // 4 nw rows (nw warps), warp w taking rows w, w + nw, w + 2 nw,
        // w + 3 nw: no division, and four solid-byte loads per thread in
        // flight at once.
        const DiskF kn = uni.kn, ko = uni.ko;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
#pragma unroll 1
        for (int cb = 0; cb < U.w; cb += 32) {
#pragma unroll 1
            for (int rb = 0; rb < U.h; rb += 4 * nw) {
                uint8_t stv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = rb + warp + nw * u, cc = cb + lane;
                    stv[u] = 2;
                    if (r < U.h && cc < U.w) {
                        int x = U.x0 + cc, y = U.y0 + r;
                        if (wrap_node(D, x, y)) stv[u] = __ldg(a.solid + D.node_off + (int64_t)y * D.pitch + x) ? 1 : 0;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = rb + warp + nw * u, cc = cb + lane;
                    if (r < U.h && cc < U.w) {
                        const int i = r * U.w + cc, xu = U.x0 + cc, yu = U.y0 + r;
                        sm.B.node_st[i] = stv[u];
                        const bool in_n = inside_f(D, kn, xu, yu, true);
                        sm.B.bnew[i] = in_n ? 1 : 0;
                        sm.B.bold[i] = advance ? (inside_f(D, ko, xu, yu, true) ? 1 : 0) : (in_n ? 1 : 0);
                    }
                }
            }
        }
    }
    __syncthreads();
    const int nn = nnear < MAXNEAR ? nnear : MAXNEAR;
    if (nnear > MAXNEAR && threadIdx.x == 0) atomicOr(a.err, ERR_STATE);
    __syncthreads();
    RastCtx rc;
    rc.D = a.doms + st.dom;
    rc.solid = a.solid;
    rc.sm = &sm.B;
    rc.near_d = near_d;
    rc.nn = nn;
    rc.U = U;
    rc.use_bm = use_bm;
    rc.advance = advance;
    rc.nxp = nxp;
    rc.nyp = nyp;
    rc.qx = q.x;
    rc.qy = q.y;
    rc.R = R;
    int32_t* links = a.links + (int64_t)wpar * a.links_total;
    int32_t* flips = a.flips + (int64_t)wpar * a.flips_total;
    const int64_t stamp = (int64_t)(int32_t)(t + 1) << 32;
    // Each thread takes a contiguous run of the box, so one block scan per
    // list places every entry, in lattice order: classify and count, scan,
    // then write (from the stored classification when the box has a bitmap).
    const int nU = U.n();
    const int per = (nU + (int)blockDim.x - 1) / (int)blockDim.x;
    const int i0 = (int)threadIdx.x * per, i1 = min(nU, i0 + per);
    bool overlap = false;
    int lcount = 0, fcount = 0;
    if (use_bm) {
        // Bitmap path, inline: every test is a shared-memory read.
#pragma unroll 1
        for (int i = i0; i < i1; ++i) {
            const uint8_t st0 = sm.B.node_st[i];
            uint32_t r = 0;
            if (st0 != 2) {
                const bool now = sm.B.bnew[i] != 0;
                if (now) {
                    r = 1u << 10;
                    if (nn > 0) {
                        const int xu = U.x0 + i % U.w, yu = U.y0 + i / U.w;
#pragma unroll 1
                        for (int j = 0; j < nn; ++j)
                            if (inside_f(D, near_d[j], xu, yu, true)) overlap = true;
                    }
                    if (st0 == 0) {
#pragma unroll
                        for (int k = 1; k < 9; ++k) {
                            const int jn = i + cy(k) * U.w + cx(k);
                            if (sm.B.node_st[jn] != 0 || sm.B.bnew[jn] != 0) continue;
                            bool in_any = false;
                            if (nn > 0) {
                                const int fxu = U.x0 + jn % U.w, fyu = U.y0 + jn / U.w;
#pragma unroll 1
                                for (int j = 0; j < nn && !in_any; ++j) in_any = inside_f(D, near_d[j], fxu, fyu, true);
                            }
                            if (!in_any) r |= 1u << k;
                        }
                    }
                }
                if (advance && st0 == 0 && now != (sm.B.bold[i] != 0)) r |= 1u << 9;
            }
            sm.B.res[i] = (uint16_t)r;
            lcount += __popc(r & 0x1FEu);
            fcount += (r >> 9) & 1u;
        }
    } else {
#pragma unroll 1
        for (int i = i0; i < i1; ++i) {
            int node;
            const uint32_t r = node_info(rc, i, node, overlap);
            lcount += __popc(r & 0x1FEu);
            fcount += (r >> 9) & 1u;
        }
    }
    int lex, fex, ltotal, ftotal;
    block_scan2(lcount, fcount, sh_warp2, lex, fex, ltotal, ftotal);
#pragma unroll 1
    for (int i = i0; i < i1 && (lcount | fcount); ++i) {
        int node = 0;
        uint32_t r;
        if (use_bm) {
            r = sm.B.res[i];
            if (r) {
                int x = U.x0 + i % U.w, y = U.y0 + i / U.w;
                wrap_node(D, x, y);
                node = y * D.pitch + x;
            }
        } else {
            bool dummy = false;
            r = node_info(rc, i, node, dummy);
        }
#pragma unroll 1
        for (int k = 1; k < 9; ++k)
            if (r & (1u << k)) {
                if (lex < st.link_cap) links[st.link_off + lex] = (node << 3) | (k - 1);
                ++lex;
            }
        if ((r >> 9) & 1u) {
            if (fex < st.flip_cap) {
                const int64_t idx = st.flip_off + fex;
                flips[idx] = (node << 1) | (int)((r >> 10) & 1u);
                // the stream-collide pass of this step leaves this node's moments in flipmom[slot]
                const int64_t slot = (int64_t)wpar * a.flips_total + idx;
                a.fliptag[(int64_t)((t + 1) & 1) * a.fliptag_stride + D.node_off + node] = stamp | (uint32_t)slot;
            }
            ++fex;
        }
    }
    if (overlap || ltotal > st.link_cap || ftotal > st.flip_cap) atomicOr(a.err, ERR_STATE);
    if (threadIdx.x == 0) {
        a.nlinks[(int64_t)wpar * a.np + p] = ltotal < st.link_cap ? ltotal : st.link_cap;
        a.nflips[(int64_t)wpar * a.np + p] = ftotal < st.flip_cap ? ftotal : st.flip_cap;
    }
}

#define LBM_PDISPATCH(kind, CALL)                     \
    switch (kind) {                                   \
        case 0: { typedef StF64 S; CALL; } break;     \
        case 1: { typedef StF32 S; CALL; } break;     \
        case 2: { typedef StF32S S; CALL; } break;    \
        case 3: { typedef StF16S S; CALL; } break;    \
        case 4: { typedef StBF16S S; CALL; } break;   \
        default: return cudaErrorInvalidValue;        \
    }

template <class S, int LO, int HI>
static cudaError_t launch_part(const PartArgs& a, int modes, int role0, int grid, int block, cudaStream_t s, bool pdl) {
    if (!pdl) {
        k_particle_step<S, LO, HI><<<grid, block, 0, s>>>(a, modes, role0);
        return cudaGetLastError();
    }
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_particle_step<S, LO, HI>, a, modes, role0);
}

cudaError_t launch_particle_step(int kind, const PartArgs& a, int modes, cudaStream_t s, bool pdl) {
    if (a.np <= 0) return cudaSuccess;
    // the contiguous range of roles the modes ask for; roles inside the
    // range that the modes leave out return at once
    const bool on[4] = {(modes & (PL_FORCES | PL_SWAP)) != 0, (modes & PL_LJ) != 0, (modes & PL_RASTER) != 0,
                        (modes & PL_MARK) != 0};
    int r0 = 0, r1 = 3;
    while (r0 < 4 && !on[r0]) ++r0;
    while (r1 >= 0 && !on[r1]) --r1;
    if (r0 > r1) return cudaSuccess;
    const int grid = (r1 - r0 + 1) * a.np;
    // role A alone uses warps 0-4 only (links, covered / uncovered nodes): a
    // smaller CTA finds room sooner beside a running stream-collide pass
    const int block = r1 == 0 ? A_BLOCK : (r0 >= 2 ? BC_BLOCK : PBLOCK);
    cudaError_t e = cudaErrorInvalidValue;  // role A or D together with other roles: no such launch
    if (r1 == 0) LBM_PDISPATCH(kind, (e = launch_part<S, 0, 0>(a, modes, r0, grid, block, s, pdl)))
    else if (r0 == 1 && r1 == 1) LBM_PDISPATCH(kind, (e = launch_part<S, 1, 1>(a, modes, r0, grid, block, s, pdl)))
    else if (r0 >= 2) LBM_PDISPATCH(kind, (e = launch_part<S, 2, 3>(a, modes, r0, grid, block, s, pdl)))
    return e;
}

}  // namespace lbmk

// stream_node.cuh -- per-node and per-chunk pieces shared by the two
// stream-collide kernels (register-pipelined k_stream.cu, staged k_staged.cu):
// domain geometry loads, the scalar ragged-tail node, flag-word loads,
// mailbox bounce-back writes, the moments of nodes that change side, and the
// finish of one pulled V-node chunk (Zou-He and corner patches, collision,
// stores).  arXiv:2006.12910 Sec. 2 Eqs. e.LB1 /
// e.LB2, Sec. 3 (halfway bounce-back, Zou-He), Sec. 4 (noise), Sec. 5 (tau*).
#pragma once
#include <cstddef>

#include "kernels.h"
#include "lbm_dev.cuh"

namespace lbmk {

__device__ __forceinline__ int find_domain(const int64_t* __restrict__ item_off, int ndom, int64_t g) {
    int lo = 0, hi = ndom - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(item_off + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Geometry of one domain for a work item, read with 16-byte loads.
struct Geo {
    int nx, ny, pitch, flags;
    int64_t off, plane, node_off, mask_off, item_off;
    int spr;  // warp segments per row
    uint32_t magic;  // multiply-high reciprocal of spr, or 0
};
static_assert(offsetof(DomDev, ny) == offsetof(DomDev, nx) + 4 && offsetof(DomDev, flags) == offsetof(DomDev, nx) + 12 &&
                  offsetof(DomDev, nx) % 16 == 0, "nx..flags must form one 16-byte block");
static_assert(offsetof(DomDev, plane) == offsetof(DomDev, off) + 8 && offsetof(DomDev, off) % 16 == 0 &&
                  offsetof(DomDev, mask_off) == offsetof(DomDev, node_off) + 8 && offsetof(DomDev, node_off) % 16 == 0 &&
                  offsetof(DomDev, seg_per_row) == offsetof(DomDev, item_off) + 8 && offsetof(DomDev, item_off) % 16 == 0,
              "64-bit offsets must pair into 16-byte blocks");
__device__ __forceinline__ Geo load_geo(const DomDev& D) {
    const int4 a = __ldg(reinterpret_cast<const int4*>(&D.nx));
    const longlong2 b = __ldg(reinterpret_cast<const longlong2*>(&D.off));
    const longlong2 c = __ldg(reinterpret_cast<const longlong2*>(&D.node_off));
    const longlong2 e = __ldg(reinterpret_cast<const longlong2*>(&D.item_off));
    Geo G;
    G.nx = a.x; G.ny = a.y; G.pitch = a.z; G.flags = a.w;
    G.off = b.x; G.plane = b.y; G.node_off = c.x; G.mask_off = c.y; G.item_off = e.x;
    G.spr = (int)(uint32_t)(uint64_t)e.y;
    G.magic = 0u;
    return G;
}
// The same from a descriptor held in the launch parameters (no memory loads).
__device__ __forceinline__ Geo param_geo(const DomDev& D) {
    Geo G;
    G.nx = D.nx; G.ny = D.ny; G.pitch = D.pitch; G.flags = D.flags;
    G.off = D.off; G.plane = D.plane; G.node_off = D.node_off; G.mask_off = D.mask_off; G.item_off = D.item_off;
    G.spr = D.seg_per_row;
    G.magic = D.spr_magic;
    return G;
}
// Row of a domain-local work item.
__device__ __forceinline__ int item_row(const Geo& G, int local) {
    return G.magic ? (int)__umulhi((uint32_t)local, G.magic) : local / G.spr;
}

// Rows that row y pulls from: y -/+ 1, wrapped when periodic in y; with y
// walls the ghost rows y = -1 and y = ny hold the bounced-back populations.
__device__ __forceinline__ void pull_rows(const Geo& G, int y, int& ym, int& yp) {
    ym = y - 1;
    yp = y + 1;
    if (G.flags & FLAG_PY) {
        if (ym < 0) ym = G.ny - 1;
        if (yp >= G.ny) yp = 0;
    }
}

// Halfway bounce-back through mailboxes: a fluid node whose neighbour
// x + e_j is solid or a ghost-row node (flag bit j) writes its post-collision
// f*_j into slot opp(j) of that neighbour, from which it pulls direction
// opp(j) in the next step (x wraps when periodic; with open ends no such
// neighbour lies beyond the x range).
template <class S>
__device__ __forceinline__ void mail_node(const Geo& G, typename S::T* obase, int x, int y, uint32_t bits,
                                          const typename S::A (&f)[9], typename S::A scale) {
#pragma unroll
    for (int j = 1; j < 9; ++j) {
        if (bits & (1u << j)) {
            int tx = x + cx(j), ty = y + cy(j);
            if (tx < 0) tx += G.nx;
            if (tx >= G.nx) tx -= G.nx;
            if (G.flags & FLAG_PY) {
                if (ty < 0) ty += G.ny;
                if (ty >= G.ny) ty -= G.ny;
            }
            from_a(f[j], scale, obase[(int64_t)opp(j) * G.plane + (int64_t)ty * G.pitch + tx]);
        }
    }
}

// Mailbox writes of a node whose neighbours need no wrapping (1 <= x <= nx-2,
// and 1 <= y <= ny-2 when periodic in y): plain offsets from the node's own
// element p = obase + y*pitch + x.
template <class S>
__device__ __forceinline__ void mail_direct(typename S::T* p, int64_t plane, int64_t pitch, uint32_t bits,
                                            const typename S::A (&f)[9], typename S::A scale) {
#pragma unroll
    for (int j = 1; j < 9; ++j)
        if (bits & (1u << j)) from_a(f[j], scale, p[opp(j) * plane + cy(j) * pitch + cx(j)]);
}

// True when the mailbox targets of node (x, y) need no wrapping.
__device__ __forceinline__ bool mail_is_direct(const Geo& G, int x, int y) {
    return x > 0 && x < G.nx - 1 && (!(G.flags & FLAG_PY) || (y > 0 && y < G.ny - 1));
}

// Scalar per-node path for the ragged tail: pull (bounced-back populations
// come from the mailboxes), wall-corner reflection and Zou-He on the open
// columns, collision, store and mailbox writes.
template <class S, bool NOISE, bool PL>
__device__ __noinline__ bool slow_node(const DomDev& D, int x, int y, const typename S::T* __restrict__ base,
                                       typename S::T* __restrict__ obase, const uint16_t* __restrict__ nflags,
                                       uint32_t step) {
    typedef typename S::A A;
    const Geo G = load_geo(D);
    const int64_t ni = (int64_t)y * G.pitch + x;
    const uint32_t fl = __ldg(nflags + G.node_off + ni);
    if (fl & NF_SOLID) return true;  // solid slots are mailboxes, written by their fluid neighbours
    const HotPrm<A> H = load_hot<A>(D);
    const ExtPrm<A> X = load_ext<A, NOISE, PL>(D);
    // scaled half-precision stores stay in their scaled units (see collide_node)
    constexpr bool SC = S::SCALED;
    const A inv = SC ? (A)1 : H.inv_scale, osc = SC ? (A)1 : H.scale;
    A f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sx = x - cx(i), sy = y - cy(i);
        if ((G.flags & FLAG_PY) && (sy < 0 || sy >= G.ny)) sy = sy < 0 ? sy + G.ny : sy - G.ny;
        bool own = false, unknown = false;
        if (sx < 0 || sx >= G.nx) {
            if (G.flags & FLAG_PX) sx = sx < 0 ? sx + G.nx : sx - G.nx;
            else if (fl & NF_CORNER) own = true;
            else unknown = true;  // Zou-He replaces it
        }
        if (own) f[i] = load_one<S>(base + (int64_t)opp(i) * G.plane + ni, inv);
        else if (unknown) f[i] = (A)0;
        else f[i] = load_one<S>(base + (int64_t)i * G.plane + (int64_t)sy * G.pitch + sx, inv);
    }
    const A zsc = SC ? H.scale : (A)1;
    if (fl & NF_ZH_IN) zou_he<A>(f, 0, zou_he_excess<A>(D, 0) * zsc);
    else if (fl & NF_ZH_OUT) zou_he<A>(f, 1, zou_he_excess<A>(D, 1) * zsc);
    const bool ok = collide_node<A, S::SHIFT, NOISE, PL, SC>(f, H, X, (uint32_t)((int64_t)y * G.nx + x), step);
#pragma unroll
    for (int i = 0; i < 9; ++i) from_a(f[i], osc, obase[(int64_t)i * G.plane + ni]);
    if (fl & 0x1FEu) mail_node<S>(G, obase, x, y, fl, f, osc);
    return ok;
}

// V per-node flag words of one chunk (V*2 bytes, aligned).
template <int V>
__device__ __forceinline__ void load_flags(const uint16_t* p, uint16_t (&fl)[V]) {
    if constexpr (V == 2) {
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(p));
        fl[0] = (uint16_t)w; fl[1] = (uint16_t)(w >> 16);
    } else if constexpr (V == 4) {
        const uint2 w = __ldg(reinterpret_cast<const uint2*>(p));
        fl[0] = (uint16_t)w.x; fl[1] = (uint16_t)(w.x >> 16); fl[2] = (uint16_t)w.y; fl[3] = (uint16_t)(w.y >> 16);
    } else {
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(p));
        const uint32_t a[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) { fl[2 * k] = (uint16_t)a[k]; fl[2 * k + 1] = (uint16_t)(a[k] >> 16); }
    }
}

// Moments of a node that changes side this step (tag stamped step + 1): rho
// and sum f* e of the populations just stored, read back in the storage
// format so they equal what a later read of the arena would give.
template <class S>
__device__ __noinline__ void flip_moments(const StreamArgs& a, const DomDev& D, int y, int x,
                                          const typename S::T* obase, int32_t stamp) {
    const int64_t ni = (int64_t)y * D.pitch + x;
    const int64_t tag = a.fliptag[(int64_t)(stamp & 1) * a.fliptag_stride + D.node_off + ni];
    if ((int32_t)(tag >> 32) != stamp) return;
    const uint32_t slot = (uint32_t)tag;
    double r = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        double v = (double)to_a(obase[(int64_t)i * D.plane + ni], (typename S::A)D.inv_scale);
        if (S::SHIFT) v += wgt(i) * D.rho0;
        r += v;
        jx += v * cx(i);
        jy += v * cy(i);
    }
    a.flipmom[3 * (int64_t)slot + 0] = r;
    a.flipmom[3 * (int64_t)slot + 1] = jx;
    a.flipmom[3 * (int64_t)slot + 2] = jy;
}

// Everything after the pull of one V-node chunk.  Special chunks (fl holds
// their flag words): Zou-He and wall-corner patches on the open columns before
// the collision, per-node stores that leave solid slots (mailboxes) alone,
// and the mailbox writes after it.  Then the moments of nodes that change
// side (near items only).
template <class S, bool NOISE, bool PL, bool FLIPS>
__device__ __forceinline__ bool finish_chunk(const StreamArgs& a, const DomDev& D, const Geo& G,
                                             const HotPrm<typename S::A>& H, const ExtPrm<typename S::A>& X,
                                             typename S::A (&f)[9][S::V], bool special, const uint16_t (&fl)[S::V],
                                             int y, int x0, const typename S::T* base, typename S::T* obase,
                                             uint32_t step, bool near_item, int32_t next_stamp) {
    typedef typename S::A A;
    constexpr int V = S::V;
    // scaled half-precision stores: f holds scaled values (see collide_node),
    // so loads and stores here convert without scaling
    constexpr bool SC = S::SCALED;
    const A io_inv = SC ? (A)1 : H.inv_scale, io_scale = SC ? (A)1 : H.scale;
    const int64_t pitch = G.pitch, plane = G.plane;
    bool ok = true;
    // any: OR of the fluid nodes' flags (mailbox writes, open-column patches);
    // mb_planes: planes in which a solid node of the chunk has a mailbox slot
    uint32_t solid_bits = 0, any = 0, mb_planes = 0;
    if (special) {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const bool sol = fl[k] & NF_SOLID;
            solid_bits |= (uint32_t)sol << k;
            if (sol) mb_planes |= fl[k];
            else any |= fl[k];
        }
        if (any & (NF_ZH_IN | NF_ZH_OUT | NF_CORNER)) {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                if (fl[k] & NF_CORNER) {  // sources beyond the x range: the node's own opposite slot
                    const int x = x0 + k;
#pragma unroll
                    for (int i = 1; i < 9; ++i)
                        if ((x == 0 && cx(i) == 1) || (x == G.nx - 1 && cx(i) == -1))
                            f[i][k] = load_one<S>(base + (int64_t)opp(i) * plane + y * pitch + x, io_inv);
                }
                if (fl[k] & (NF_ZH_IN | NF_ZH_OUT)) {
                    A n9[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) n9[i] = f[i][k];
                    const int side = (fl[k] & NF_ZH_IN) ? 0 : 1;
                    zou_he<A>(n9, side, SC ? zou_he_excess<A>(D, side) * H.scale : zou_he_excess<A>(D, side));
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i][k] = n9[i];
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
        A n9[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) n9[i] = f[i][k];
        const bool rok = collide_node<A, S::SHIFT, NOISE, PL, SC>(n9, H, X, (uint32_t)(y * G.nx + x0 + k), step);
        ok &= rok || ((solid_bits >> k) & 1u);  // solid nodes compute on mailbox values and are discarded
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i][k] = n9[i];
    }
    typename S::T* orow = obase + y * pitch + x0;
    // A plane in which no solid node of the chunk has a mailbox slot is stored
    // whole (the solid nodes' slots there are read by nobody); otherwise the
    // fluid nodes are stored one by one.  A chunk of solid nodes only stores
    // nothing.
    if (solid_bits != (1u << V) - 1u) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (!((mb_planes >> i) & 1u)) {
                if constexpr (SC) store_vec_raw<S>(orow + (int64_t)i * plane, f[i]);
                else store_vec<S>(orow + (int64_t)i * plane, f[i], H.scale);
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k)
                    if (!((solid_bits >> k) & 1u)) from_a(f[i][k], io_scale, orow[(int64_t)i * plane + k]);
            }
        }
    }
    if (any & 0x1FEu) {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            if ((fl[k] & 0x1FEu) && !(fl[k] & NF_SOLID)) {
                A n9[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) n9[i] = f[i][k];
                if (mail_is_direct(G, x0 + k, y)) mail_direct<S>(orow + k, plane, pitch, fl[k], n9, io_scale);
                else mail_node<S>(G, obase, x0 + k, y, fl[k], n9, io_scale);
            }
        }
    }
    if (FLIPS && near_item) {
#pragma unroll 1
        for (int k = 0; k < V; ++k) flip_moments<S>(a, D, y, x0 + k, obase, next_stamp);
    }
    return ok;
}

}  // namespace lbmk

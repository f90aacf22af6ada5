// k_part.cu -- particle kernels of the D2Q9 hot path (arXiv:2006.12910 Sec. 3).
//
// One CTA per particle.  The stored populations are f*(t), post-collision.
//  * k_particle_forces: Eq. MP1 over the boundary links of the rasterisation at
//    t, the covered/uncovered-node force of Eq. MP3 for nodes that changed side
//    at the previous re-rasterisation, the LJ-type repulsion of Eq. MP2, the
//    totals of Eqs. MP3-MP4 (FP64, fixed-order block reduction) and the
//    Newton-Euler update of Eqs. MP5-MP6 into the next-state slot.
//  * k_particle_links: Eqs. MP7-MP8 as a pre-stream exchange: for the link
//    r_v -> r_v + e_k the slot that r_v + e_k pulls next step receives
//    f*_{-k}(r_v + e_k) + 2 rho0 omega_k (u_b . e_k) / c_s^2 and the slot r_v
//    pulls receives f*_k(r_v) - the same, so the plain pull stream then
//    realises the moving bounce-back on both sides.  It then commits the new
//    state and re-rasterises: the new link list and the list of nodes that
//    changed side (covered / uncovered), compacted in a fixed order.
#include "kernels.h"
#include "lbm_dev.cuh"

namespace lbmk {

constexpr int PBLOCK = 256;

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

__device__ __forceinline__ bool is_surface(const DomDev& D, double px, double py, double R, int x, int y) {
    if (!inside_disk(D, px, py, R, x, y)) return false;
#pragma unroll
    for (int i = 1; i < 9; ++i)
        if (!inside_disk(D, px, py, R, x + cx(i), y + cy(i))) return true;
    return false;
}

// Wrap a node into the domain; false when it leaves through a non-periodic edge.
__device__ __forceinline__ bool wrap_node(const DomDev& D, int& x, int& y) {
    if (x < 0 || x >= D.nx) {
        if (!(D.flags & FLAG_PX)) return false;
        x = ((x % D.nx) + D.nx) % D.nx;
    }
    if (y < 0 || y >= D.ny) {
        if (!(D.flags & FLAG_PY)) return false;
        y = ((y % D.ny) + D.ny) % D.ny;
    }
    return true;
}

template <class S>
__device__ __forceinline__ double full_pop(const typename S::T* base, const DomDev& D, int i, int64_t ni) {
    const double v = (double)to_a(base[(int64_t)i * D.plane + ni], (typename S::A)D.inv_scale);
    return S::SHIFT ? v + wgt(i) * D.rho0 : v;
}

// Fixed-order block reduction of N doubles (deterministic for a fixed blockDim).
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double (*sh)[PBLOCK]) {
#pragma unroll
    for (int c = 0; c < N; ++c) sh[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int s = PBLOCK / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int c = 0; c < N; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] = sh[c][0];
    __syncthreads();
}

// Exclusive block scan of small non-negative counts; returns the block total.
__device__ __forceinline__ int block_scan(int c, int* sh_warp, int& excl) {
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
    for (int k = 0; k < PBLOCK / 32; ++k) {
        if (k < w) wbase += sh_warp[k];
        total += sh_warp[k];
    }
    excl = wbase + incl - c;
    __syncthreads();
    return total;
}

template <class S>
__global__ void __launch_bounds__(PBLOCK) k_particle_forces(PartArgs a) {
    const int p = blockIdx.x;
    const PartStatic st = a.st[p];
    if (st.dom < 0) return;
    const DomDev& D = a.doms[st.dom];
    if (p - D.p0 >= D.np) return;
    const PartState q = a.cur[p];
    const typename S::T* base = static_cast<const typename S::T*>(a.arena) + D.off;
    const bool px = D.flags & FLAG_PX, py = D.flags & FLAG_PY;
    __shared__ double sh[DIAG_N][PBLOCK];

    double acc[DIAG_N];
#pragma unroll
    for (int c = 0; c < DIAG_N; ++c) acc[c] = 0.0;

    // Eq. MP1: F = -2 [f'_k(r_v + e_k, t*) + rho0 omega_k (u_b . e_k) / c_s^2] e_k
    const int nl = a.nlinks[p];
    for (int l = threadIdx.x; l < nl; l += PBLOCK) {
        const int32_t e = a.links[st.link_off + l];
        const int node = e >> 3, k = (e & 7) + 1;
        const int vy = node / D.pitch, vx = node - vy * D.pitch;
        int fx = vx + cx(k), fy = vy + cy(k);
        wrap_node(D, fx, fy);
        const int ko = opp(k);
        const double fo = full_pop<S>(base, D, ko, (int64_t)fy * D.pitch + fx);
        const double bx = min_image((vx + 0.5 * cx(k)) - q.x, D.nx, px);
        const double by = min_image((vy + 0.5 * cy(k)) - q.y, D.ny, py);
        const double ubx = q.U - q.Om * by, uby = q.V + q.Om * bx;
        const double ube = ubx * cx(k) + uby * cy(k);
        const double s = -2.0 * (fo + D.rho0 * wgt(k) * ube * 3.0);
        const double Fx = s * cx(k), Fy = s * cy(k);
        acc[0] += Fx;
        acc[1] += Fy;
        acc[2] += bx * Fy - by * Fx;
    }

    // Covered (+) / uncovered (-) nodes: F = +- rho (u - U_p), u from f*(t).
    const int nf = a.nflips[p];
    for (int l = threadIdx.x; l < nf; l += PBLOCK) {
        const int32_t e = a.flips[st.flip_off + l];
        const int node = e >> 1;
        const bool cov = e & 1;
        const int y = node / D.pitch, x = node - y * D.pitch;
        double r = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double fi = full_pop<S>(base, D, i, node);
            r += fi;
            jx += fi * cx(i);
            jy += fi * cy(i);
        }
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

    // Eq. MP2 between surface nodes of p and surface nodes of the other
    // particles of the domain, and between surface nodes of p and stationary
    // solid / wall nodes, within the threshold r_it.
    if (D.lj_psi != 0.0) {
        const double R = st.R;
        const int bx0 = (int)floor(q.x - R) - 1, bx1 = (int)ceil(q.x + R) + 1;
        const int by0 = (int)floor(q.y - R) - 1, by1 = (int)ceil(q.y + R) + 1;
        const int bw = bx1 - bx0 + 1, bn = bw * (by1 - by0 + 1);
        const int reach = (int)floor(D.lj_rit);
        for (int t = threadIdx.x; t < bn; t += PBLOCK) {
            const int ay = by0 + t / bw, ax = bx0 + t % bw;
            if (!is_surface(D, q.x, q.y, R, ax, ay)) continue;
            const double rax = min_image(ax - q.x, D.nx, px), ray = min_image(ay - q.y, D.ny, py);
            for (int p2 = D.p0; p2 < D.p0 + D.np; ++p2) {
                if (p2 == p) continue;
                const PartState o = a.cur[p2];
                const double oR = a.st[p2].R;
                const double cdx = min_image(o.x - q.x, D.nx, px), cdy = min_image(o.y - q.y, D.ny, py);
                const double reachc = R + oR + D.lj_rit + 4.0;
                if (cdx * cdx + cdy * cdy > reachc * reachc) continue;
                const int ox0 = (int)floor(o.x - oR) - 1, ox1 = (int)ceil(o.x + oR) + 1;
                const int oy0 = (int)floor(o.y - oR) - 1, oy1 = (int)ceil(o.y + oR) + 1;
                for (int by = oy0; by <= oy1; ++by)
                    for (int bx = ox0; bx <= ox1; ++bx) {
                        if (!is_surface(D, o.x, o.y, oR, bx, by)) continue;
                        const double sx = min_image((double)(ax - bx), D.nx, px);
                        const double sy = min_image((double)(ay - by), D.ny, py);
                        const double dist = sqrt(sx * sx + sy * sy);
                        if (!(dist <= D.lj_rit) || dist == 0.0) continue;
                        const double mag = D.lj_psi * pow(dist / D.lj_rit, -13.0);
                        const double Fx = mag * sx / dist, Fy = mag * sy / dist;
                        acc[6] += Fx;
                        acc[7] += Fy;
                        acc[8] += rax * Fy - ray * Fx;
                    }
            }
            for (int oy = -reach; oy <= reach; ++oy)
                for (int ox = -reach; ox <= reach; ++ox) {
                    if (ox == 0 && oy == 0) continue;
                    const double dist = sqrt((double)(ox * ox + oy * oy));
                    if (!(dist <= D.lj_rit)) continue;
                    int wx = ax + ox, wy = ay + oy;
                    bool wall;
                    if ((D.flags & FLAG_WY) && (wy < 0 || wy >= D.ny)) wall = true;
                    else {
                        if (!wrap_node(D, wx, wy)) continue;
                        wall = a.solid[D.node_off + (int64_t)wy * D.pitch + wx] != 0;
                    }
                    if (!wall) continue;
                    const double mag = D.lj_psi * pow(dist / D.lj_rit, -13.0);
                    const double Fx = -mag * ox / dist, Fy = -mag * oy / dist;
                    acc[6] += Fx;
                    acc[7] += Fy;
                    acc[8] += rax * Fy - ray * Fx;
                }
        }
    }

    block_sum<DIAG_N>(acc, sh);
    if (threadIdx.x == 0) {
        double* dg = a.diag + (int64_t)p * DIAG_N;
        for (int c = 0; c < DIAG_N; ++c) dg[c] = acc[c];
        // Eqs. MP5, MP6; r_c(t+1) = r_c(t) + U_p(t).
        PartState n = q;
        if (!st.fixed) {
            const double Fx = acc[0] + acc[3] + acc[6], Fy = acc[1] + acc[4] + acc[7];
            const double T = acc[2] + acc[5] + acc[8];
            const double buoy = (st.rho_p - D.rho0) / st.rho_p;
            n.U = q.U + Fx / st.m + buoy * D.gx;
            n.V = q.V + Fy / st.m + buoy * D.gy;
            n.Om = q.Om + T / st.I;
            n.x = q.x + q.U;
            n.y = q.y + q.V;
            n.th = q.th + q.Om;
            if (px) n.x = n.x - D.nx * floor(n.x / D.nx);
            if (py) n.y = n.y - D.ny * floor(n.y / D.ny);
        }
        a.next[p] = n;
    }
}

template <class S>
__global__ void __launch_bounds__(PBLOCK) k_particle_links(PartArgs a, int swap, int advance) {
    typedef typename S::A A;
    const int p = blockIdx.x;
    const PartStatic st = a.st[p];
    if (st.dom < 0) return;
    const DomDev& D = a.doms[st.dom];
    if (p - D.p0 >= D.np) return;
    const PartState q = a.cur[p];
    typename S::T* base = static_cast<typename S::T*>(a.arena) + D.off;
    const bool px = D.flags & FLAG_PX, py = D.flags & FLAG_PY;
    __shared__ int sh_warp[PBLOCK / 32];

    // Eqs. MP7-MP8 on the links of the rasterisation at t with u_b(t).
    if (swap) {
        const int nl = a.nlinks[p];
        const A scl = (A)D.scale, inv = (A)D.inv_scale;
        for (int l = threadIdx.x; l < nl; l += PBLOCK) {
            const int32_t e = a.links[st.link_off + l];
            const int node = e >> 3, k = (e & 7) + 1;
            const int vy = node / D.pitch, vx = node - vy * D.pitch;
            int fx = vx + cx(k), fy = vy + cy(k);
            wrap_node(D, fx, fy);
            const double bx = min_image((vx + 0.5 * cx(k)) - q.x, D.nx, px);
            const double by = min_image((vy + 0.5 * cy(k)) - q.y, D.ny, py);
            const double ubx = q.U - q.Om * by, uby = q.V + q.Om * bx;
            const A corr = (A)(2.0 * D.rho0 * wgt(k) * (ubx * cx(k) + uby * cy(k)) * 3.0);
            typename S::T* sa = base + (int64_t)k * D.plane + node;                          // pulled by r_v + e_k
            typename S::T* sb = base + (int64_t)opp(k) * D.plane + (int64_t)fy * D.pitch + fx;  // pulled by r_v
            const A va = to_a(*sa, inv), vb = to_a(*sb, inv);
            from_a(vb + corr, scl, *sa);
            from_a(va - corr, scl, *sb);
        }
        __syncthreads();
    }

    const PartState n = advance ? a.next[p] : q;
    const double R = st.R;
    // New link list at the new position.
    {
        const int bx0 = (int)floor(n.x - R) - 1, bx1 = (int)ceil(n.x + R) + 1;
        const int by0 = (int)floor(n.y - R) - 1, by1 = (int)ceil(n.y + R) + 1;
        const int bw = bx1 - bx0 + 1, bn = bw * (by1 - by0 + 1);
        int total = 0;
        bool overlap = false;
        for (int t0 = 0; t0 < bn; t0 += PBLOCK) {
            const int t = t0 + threadIdx.x;
            uint32_t mask = 0;
            int node = 0;
            if (t < bn) {
                int x = bx0 + t % bw, y = by0 + t / bw;
                if (wrap_node(D, x, y) && inside_disk(D, n.x, n.y, R, x, y)) {
                    node = y * D.pitch + x;
                    for (int p2 = D.p0; p2 < D.p0 + D.np; ++p2) {
                        if (p2 == p) continue;
                        const PartState o = advance ? a.next[p2] : a.cur[p2];
                        if (inside_disk(D, o.x, o.y, a.st[p2].R, x, y)) overlap = true;
                    }
                    if (!a.solid[D.node_off + node]) {
#pragma unroll
                        for (int k = 1; k < 9; ++k) {
                            int fx = x + cx(k), fy = y + cy(k);
                            if (!wrap_node(D, fx, fy)) continue;
                            if (a.solid[D.node_off + (int64_t)fy * D.pitch + fx]) continue;
                            bool in_any = inside_disk(D, n.x, n.y, R, fx, fy);
                            for (int p2 = D.p0; p2 < D.p0 + D.np && !in_any; ++p2) {
                                if (p2 == p) continue;
                                const PartState o = advance ? a.next[p2] : a.cur[p2];
                                in_any = inside_disk(D, o.x, o.y, a.st[p2].R, fx, fy);
                            }
                            if (!in_any) mask |= 1u << k;
                        }
                    }
                }
            }
            int excl;
            const int c = __popc(mask);
            const int tot = block_scan(c, sh_warp, excl);
            int w = total + excl;
            for (int k = 1; k < 9; ++k)
                if (mask & (1u << k)) {
                    if (w < st.link_cap) a.links[st.link_off + w] = (node << 3) | (k - 1);
                    ++w;
                }
            total += tot;
        }
        if (overlap || total > st.link_cap) atomicOr(a.err, ERR_STATE);
        if (threadIdx.x == 0) a.nlinks[p] = total < st.link_cap ? total : st.link_cap;
    }
    // Nodes that change side between the old and the new position.
    {
        const int bx0 = (int)floor(fmin(q.x, n.x) - R) - 1, bx1 = (int)ceil(fmax(q.x, n.x) + R) + 1;
        const int by0 = (int)floor(fmin(q.y, n.y) - R) - 1, by1 = (int)ceil(fmax(q.y, n.y) + R) + 1;
        const int bw = bx1 - bx0 + 1, bn = bw * (by1 - by0 + 1);
        int total = 0;
        for (int t0 = 0; t0 < bn; t0 += PBLOCK) {
            const int t = t0 + threadIdx.x;
            int c = 0, code = 0;
            if (t < bn && advance) {
                int x = bx0 + t % bw, y = by0 + t / bw;
                if (wrap_node(D, x, y)) {
                    // the union box stays far below the domain size, so a
                    // wrapped node is visited once
                    const int node = y * D.pitch + x;
                    const bool was = inside_disk(D, q.x, q.y, R, x, y), now = inside_disk(D, n.x, n.y, R, x, y);
                    if (was != now && !a.solid[D.node_off + node]) { c = 1; code = (node << 1) | (now ? 1 : 0); }
                }
            }
            int excl;
            const int tot = block_scan(c, sh_warp, excl);
            if (c) {
                const int w = total + excl;
                if (w < st.flip_cap) a.flips[st.flip_off + w] = code;
            }
            total += tot;
        }
        if (total > st.flip_cap) atomicOr(a.err, ERR_STATE);
        if (threadIdx.x == 0) {
            a.nflips[p] = total < st.flip_cap ? total : st.flip_cap;
            if (advance) a.cur[p] = n;
        }
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

cudaError_t launch_particle_forces(int kind, const PartArgs& a, cudaStream_t s) {
    if (a.np <= 0) return cudaSuccess;
    LBM_PDISPATCH(kind, (k_particle_forces<S><<<a.np, PBLOCK, 0, s>>>(a)));
    return cudaGetLastError();
}

cudaError_t launch_particle_links(int kind, const PartArgs& a, bool swap, bool advance, cudaStream_t s) {
    if (a.np <= 0) return cudaSuccess;
    LBM_PDISPATCH(kind, (k_particle_links<S><<<a.np, PBLOCK, 0, s>>>(a, swap ? 1 : 0, advance ? 1 : 0)));
    return cudaGetLastError();
}

}  // namespace lbmk

// k_part.cu -- particle kernel of the D2Q9 hot path (arXiv:2006.12910 Sec. 3).
//
// One launch per timestep with two CTAs per particle that run side by side
// (roles A and B below).  The stored populations are f*(t), post-collision;
// the particle state and the link / flip lists are double-buffered by the
// parity of the step, so A reads the lists of t while B writes those of t+1.
// Role A (phases 1-2) and role B (phase 3):
//  1. forces at t: Eq. MP1 over the boundary links of the rasterisation at t
//     (each link's slots belong to this particle alone), the covered /
//     uncovered-node force of Eq. MP3 from the node moments that the
//     stream-collide pass of the previous step wrote while producing f*(t),
//     and the LJ-type repulsion of Eq. MP2; FP64 totals (Eqs. MP3-MP4) and the
//     Newton-Euler update of Eqs. MP5-MP6;
//  2. Eqs. MP7-MP8 as a pre-stream exchange: for the link r_v -> r_v + e_k the
//     slot that r_v + e_k pulls next receives f*_{-k}(r_v + e_k) +
//     2 rho0 omega_k (u_b . e_k) / c_s^2 and the slot r_v pulls receives
//     f*_k(r_v) minus the same, so the plain pull stream realises the moving
//     bounce-back on both sides;
//  3. re-rasterisation at r_c(t+1) = r_c(t) + U_p(t), which needs no force and
//     therefore no other CTA's result: new link list, the nodes that change
//     side (tagged for the next stream-collide pass), and the work items near
//     the particle for the next step.
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
__device__ __forceinline__ DiskF make_diskf(double px, double py, double R) {
    DiskF d;
    d.px = px; d.py = py; d.R = R;
    d.cx = (int)floor(px); d.cy = (int)floor(py);
    d.fx = (float)(px - d.cx); d.fy = (float)(py - d.cy);
    d.R2 = (float)(R * R);
    d.margin = 1e-3f * fmaxf(1.0f, d.R2 * 0.01f) + 1e-4f;
    return d;
}
// Integer minimum image of a node offset along a periodic axis.
__device__ __forceinline__ int wrap_off(int d, int L, bool periodic) {
    if (!periodic) return d;
    d %= L;
    if (d < 0) d += L;
    if (2 * d >= L) d -= L;
    return d;
}
__device__ __forceinline__ bool inside_f(const DomDev& D, const DiskF& k, int xu, int yu, bool wrapped) {
    const int dxi = wrap_off(xu - k.cx, D.nx, D.flags & FLAG_PX), dyi = wrap_off(yu - k.cy, D.ny, D.flags & FLAG_PY);
    const float dx = (float)dxi - k.fx, dy = (float)dyi - k.fy;
    const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    if (d2 < k.R2 - k.margin) return true;
    if (d2 > k.R2 + k.margin) return false;
    if (wrapped) {
        int x = xu, y = yu;
        if (!wrap_node(D, x, y)) { x = xu; y = yu; }
        return inside_disk(D, k.px, k.py, k.R, x, y);
    }
    return inside_disk(D, k.px, k.py, k.R, xu, yu);
}

template <class S>
__device__ __forceinline__ double full_pop(const typename S::T* base, const DomDev& D, int i, int64_t ni) {
    const double v = (double)to_a(base[(int64_t)i * D.plane + ni], (typename S::A)D.inv_scale);
    return S::SHIFT ? v + wgt(i) * D.rho0 : v;
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

constexpr int PB_CAP = 4096;   // nodes of a shared-memory inside bitmap
constexpr int MAXNEAR = 64;     // nearby particles considered per particle

// Exclusive block scan of small non-negative counts; returns the block total.
__device__ __forceinline__ int block_scan(int c, int* sh_warp, int& excl);

// Other particles of the domain whose disks come within `extra` of the disk
// (x, y, R), in index order, with their FP32 test data.  Every thread tests
// its share of the particles; a block scan compacts the list, so the order is
// fixed and no thread walks the particle array alone.
__device__ __forceinline__ void near_list(const PartArgs& a, const DomDev& D, int p, const PartState* states,
                                          double x, double y, double R, double extra, int* list, DiskF* disks,
                                          int* count, int* sh_warp) {
    int total = 0;
    for (int b0 = 0; b0 < D.np; b0 += PBLOCK) {
        const int j = b0 + (int)threadIdx.x;
        const int p2 = D.p0 + j;
        int hit = 0;
        PartState o;
        double r2 = 0.0;
        if (j < D.np && p2 != p) {
            o = states[p2];
            r2 = a.st[p2].R;
            // FP32 centre distance with a one-node margin: a superset of the
            // particles within reach is all that is needed here
            float dx = (float)o.x - (float)x, dy = (float)o.y - (float)y;
            if (D.flags & FLAG_PX) { const float L = (float)D.nx; dx -= L * rintf(dx / L); }
            if (D.flags & FLAG_PY) { const float L = (float)D.ny; dy -= L * rintf(dy / L); }
            const float reach = (float)(R + r2 + extra) + 1.0f;
            hit = dx * dx + dy * dy <= reach * reach;
        }
        int excl;
        const int tot = block_scan(hit, sh_warp, excl);
        if (hit && total + excl < MAXNEAR) {
            list[total + excl] = p2;
            disks[total + excl] = make_diskf(o.x, o.y, r2);
        }
        total += tot;
    }
    if (threadIdx.x == 0) *count = total;
    __syncthreads();
}

// Surface node of a disk (inside, with an 8-neighbour outside), unwrapped
// coordinates near the disk, using the FP32 test with its exact fallback.
__device__ __forceinline__ bool is_surface_f(const DomDev& D, const DiskF& k, int x, int y) {
    if (!inside_f(D, k, x, y, false)) return false;
#pragma unroll
    for (int i = 1; i < 9; ++i)
        if (!inside_f(D, k, x + cx(i), y + cy(i), false)) return true;
    return false;
}

// Position at t+1 from the state at t (Sec. 3: r_c(t+1) = r_c(t) + U_p(t)).
__device__ __forceinline__ void next_position(const DomDev& D, const PartState& q, bool fixed, double& x, double& y) {
    if (fixed) { x = q.x; y = q.y; return; }
    x = q.x + q.U;
    y = q.y + q.V;
    if (D.flags & FLAG_PX) x = x - D.nx * floor(x / D.nx);
    if (D.flags & FLAG_PY) y = y - D.ny * floor(y / D.ny);
}

// Fixed-order block sum of the components [c0, c1) of v (deterministic for a
// fixed blockDim).  FP64 issue rate is low on this part, so the tree first
// halves across warps in shared memory (4, 2, 1 warps active) and only then
// shuffles inside warp 0; the totals land in tot[c].
template <int N>
__device__ __forceinline__ void block_sum_range(double (&v)[N], int c0, int c1, double* buf, double* tot) {
    static_assert(PBLOCK == 256, "tree below assumes 256 threads");
#pragma unroll
    for (int c = 0; c < N; ++c)
        if (c >= c0 && c < c1) buf[c * PBLOCK + threadIdx.x] = v[c];
    __syncthreads();
    for (int h = PBLOCK / 2; h >= 32; h >>= 1) {
        if ((int)threadIdx.x < h) {
#pragma unroll
            for (int c = 0; c < N; ++c)
                if (c >= c0 && c < c1) buf[c * PBLOCK + threadIdx.x] += buf[c * PBLOCK + threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x < 32) {
#pragma unroll
        for (int c = 0; c < N; ++c) {
            if (c < c0 || c >= c1) continue;
            double x = buf[c * PBLOCK + threadIdx.x];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (threadIdx.x == 0) tot[c] = x;
        }
    }
    __syncthreads();
}

// Shared memory of one CTA; role A and role B use disjoint parts of a union.
struct SmemA {
    double red[DIAG_N * PBLOCK];
    uint8_t bm[PB_CAP];
    uint8_t wall_win[PB_CAP];
    double lj_fx[LJ_TAB], lj_fy[LJ_TAB];
    int lj_ox[LJ_TAB], lj_oy[LJ_TAB];
};
struct SmemB {
    uint8_t bnew[PB_CAP], bold[PB_CAP], node_st[PB_CAP];
};
union SmemU {
    SmemA A;
    SmemB B;
};

template <class S>
__global__ void __launch_bounds__(PBLOCK) k_particle_step(PartArgs a, int modes) {
    typedef typename S::A A;
    const bool role_b = (int)blockIdx.x >= a.np;
    const int p = role_b ? blockIdx.x - a.np : blockIdx.x;
    const int64_t t = *a.ctr;
    const bool advance = modes & PL_ADVANCE;
    // The near-item list of step t+2 is touched by nobody during this step.
    if (blockIdx.x == 0 && threadIdx.x == 0 && advance) a.near_cnt[(t + 2) % 3] = 0;
    if (role_b ? !(modes & (PL_RASTER | PL_MARK)) : !(modes & (PL_FORCES | PL_SWAP | PL_ADVANCE))) return;
    const PartStatic st = a.st[p];
    if (st.dom < 0) return;
    const DomDev D = a.doms[st.dom];
    if (p - D.p0 >= D.np) return;
    const int par = (int)(t & 1);
    const PartState* S0 = a.state + (int64_t)par * a.np;
    const PartState q = S0[p];
    const double R = st.R;
    const bool px = D.flags & FLAG_PX, py = D.flags & FLAG_PY;
    typename S::T* base = static_cast<typename S::T*>(a.arena) + D.off;
    double nxp = q.x, nyp = q.y;
    if (advance) next_position(D, q, st.fixed, nxp, nyp);

    __shared__ __align__(16) unsigned char smem_raw[sizeof(SmemU)];
    SmemU& sm = *reinterpret_cast<SmemU*>(smem_raw);
    __shared__ double tot[DIAG_N];
    __shared__ int lj_n, nnear;
    __shared__ int sh_warp[PBLOCK / 32];
    __shared__ int near[MAXNEAR];
    __shared__ DiskF near_d[MAXNEAR];

    if (!role_b) {
        // ------------------------------------------------------------------ role A
        const int32_t* links = a.links + (int64_t)par * a.links_total;
        const int32_t* flips = a.flips + (int64_t)par * a.flips_total;
        const int nl = a.nlinks[(int64_t)par * a.np + p];
        const int nf = a.nflips[(int64_t)par * a.np + p];
        double acc[DIAG_N];
#pragma unroll
        for (int c = 0; c < DIAG_N; ++c) acc[c] = 0.0;
        bool lj_on = false;
        if (modes & PL_FORCES) {
            // Eq. MP1: F = -2 [f'_k(r_v + e_k, t*) + rho0 omega_k (u_b . e_k) / c_s^2] e_k
            for (int l = threadIdx.x; l < nl; l += PBLOCK) {
                const int32_t e = links[st.link_off + l];
                const int node = e >> 3, k = (e & 7) + 1;
                const int vy = node / D.pitch, vx = node - vy * D.pitch;
                int fx = vx + cx(k), fy = vy + cy(k);
                wrap_node(D, fx, fy);
                const double fo = full_pop<S>(base, D, opp(k), (int64_t)fy * D.pitch + fx);
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
            // Covered (+) / uncovered (-) nodes: F = +- rho (u - U_p), with rho and
            // sum f* e of the node at t written by the previous stream-collide pass.
            for (int l = threadIdx.x; l < nf; l += PBLOCK) {
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
            // Eq. MP2 between surface nodes of p and surface nodes of the other
            // particles, and between surface nodes of p and stationary solid /
            // wall nodes, within the threshold r_it.
            if (D.lj_psi != 0.0) {
                near_list(a, D, p, S0, q.x, q.y, R, D.lj_rit + 4.0, near, near_d, &nnear, sh_warp);
                const int nn = nnear < MAXNEAR ? nnear : MAXNEAR;
                const Box b = disk_box(q.x, q.y, R);
                const Box e = {b.x0 - 1, b.y0 - 1, b.w + 2, b.h + 2};
                const int reach = (int)floor(D.lj_rit);
                const bool use_bm = e.n() <= PB_CAP;
                // 1 = wall or solid node within reach of the box, 0 = fluid or beyond an open end
                const Box W = {b.x0 - reach, b.y0 - reach, b.w + 2 * reach, b.h + 2 * reach};
                const bool use_win = W.n() <= PB_CAP;
                int any_wall = 0;
                for (int i = threadIdx.x; i < W.n(); i += PBLOCK) {
                    int wx = W.x0 + i % W.w, wy = W.y0 + i / W.w;
                    uint8_t v = 0;
                    if ((D.flags & FLAG_WY) && (wy < 0 || wy >= D.ny)) v = 1;
                    else if (wrap_node(D, wx, wy)) v = a.solid[D.node_off + (int64_t)wy * D.pitch + wx] != 0;
                    if (use_win) sm.A.wall_win[i] = v;
                    any_wall |= v;
                }
                lj_on = __syncthreads_or(any_wall) || nn > 0 || !use_win;
                if (lj_on) {
                    if (threadIdx.x == 0) lj_n = a.lj_cnt[st.dom];
                    for (int i = threadIdx.x; i < LJ_TAB; i += PBLOCK) {
                        const LjEntry en = a.lj_tab[(int64_t)st.dom * LJ_TAB + i];
                        sm.A.lj_ox[i] = en.ox;
                        sm.A.lj_oy[i] = en.oy;
                        sm.A.lj_fx[i] = en.fx;
                        sm.A.lj_fy[i] = en.fy;
                    }
                    if (use_bm) {
                        const DiskF kf = make_diskf(q.x, q.y, R);
                        for (int i = threadIdx.x; i < e.n(); i += PBLOCK)
                            sm.A.bm[i] = inside_f(D, kf, e.x0 + i % e.w, e.y0 + i / e.w, false) ? 1 : 0;
                    }
                    __syncthreads();
                    for (int i = threadIdx.x; i < b.n(); i += PBLOCK) {
                        const int ay = b.y0 + i / b.w, ax = b.x0 + i % b.w;
                        bool surf;
                        if (use_bm) {
                            const int c = (ay - e.y0) * e.w + (ax - e.x0);
                            surf = sm.A.bm[c] != 0;
                            if (surf) {
                                bool all_in = true;
#pragma unroll
                                for (int k = 1; k < 9; ++k) all_in &= sm.A.bm[c + cy(k) * e.w + cx(k)] != 0;
                                surf = !all_in;
                            }
                        } else {
                            surf = is_surface(D, q.x, q.y, R, ax, ay);
                        }
                        if (!surf) continue;
                        double rax = 0.0, ray = 0.0;
                        bool arm = false;  // torque arm of this surface node, computed on first use
                        for (int j = 0; j < nn; ++j) {
                            const DiskF& ko = near_d[j];
                            const float ddx = (float)wrap_off(ax - ko.cx, D.nx, px) - ko.fx;
                            const float ddy = (float)wrap_off(ay - ko.cy, D.ny, py) - ko.fy;
                            const float lim = (float)(ko.R + D.lj_rit) + 2.0f;
                            if (ddx * ddx + ddy * ddy > lim * lim) continue;
                            for (int w = 0; w < lj_n; ++w) {
                                // node b = a + o expressed in the other particle's own frame
                                const int bx = ko.cx + wrap_off(ax + sm.A.lj_ox[w] - ko.cx, D.nx, px);
                                const int by = ko.cy + wrap_off(ay + sm.A.lj_oy[w] - ko.cy, D.ny, py);
                                if (!is_surface_f(D, ko, bx, by)) continue;
                                if (!arm) { rax = min_image(ax - q.x, D.nx, px); ray = min_image(ay - q.y, D.ny, py); arm = true; }
                                acc[6] += sm.A.lj_fx[w];
                                acc[7] += sm.A.lj_fy[w];
                                acc[8] += rax * sm.A.lj_fy[w] - ray * sm.A.lj_fx[w];
                            }
                        }
#pragma unroll 1
                        for (int j = 0; j < lj_n; ++j) {
                            int wx = ax + sm.A.lj_ox[j], wy = ay + sm.A.lj_oy[j];
                            bool wall;
                            if (use_win) {
                                wall = sm.A.wall_win[(wy - W.y0) * W.w + (wx - W.x0)] != 0;
                            } else if ((D.flags & FLAG_WY) && (wy < 0 || wy >= D.ny)) {
                                wall = true;
                            } else {
                                if (!wrap_node(D, wx, wy)) continue;
                                wall = a.solid[D.node_off + (int64_t)wy * D.pitch + wx] != 0;
                            }
                            if (!wall) continue;
                            if (!arm) { rax = min_image(ax - q.x, D.nx, px); ray = min_image(ay - q.y, D.ny, py); arm = true; }
                            acc[6] += sm.A.lj_fx[j];
                            acc[7] += sm.A.lj_fy[j];
                            acc[8] += rax * sm.A.lj_fy[j] - ray * sm.A.lj_fx[j];
                        }
                    }
                }
            }
            // component groups: links 0-2, covered/uncovered 3-5 and 9-12, LJ 6-8
            if (threadIdx.x < DIAG_N) tot[threadIdx.x] = 0.0;
            __syncthreads();
            if (nl > 0) block_sum_range<DIAG_N>(acc, 0, 3, sm.A.red, tot);
            if (nf > 0) {
                block_sum_range<DIAG_N>(acc, 3, 6, sm.A.red, tot);
                block_sum_range<DIAG_N>(acc, 9, 13, sm.A.red, tot);
            }
            if (lj_on) block_sum_range<DIAG_N>(acc, 6, 9, sm.A.red, tot);
            if (threadIdx.x < DIAG_N) a.diag[(int64_t)p * DIAG_N + threadIdx.x] = tot[threadIdx.x];
        }
        // Eqs. MP7-MP8 on the links of the rasterisation at t with u_b(t); every
        // read of these slots above happened before this barrier.
        __syncthreads();
        if (modes & PL_SWAP) {
            const A scl = (A)D.scale, inv = (A)D.inv_scale;
            for (int l = threadIdx.x; l < nl; l += PBLOCK) {
                const int32_t e = links[st.link_off + l];
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
        }
        if (advance && threadIdx.x == 0) {
            // Eqs. MP5, MP6 (velocities) with r_c(t+1) = r_c(t) + U_p(t).
            PartState n = q;
            if (!st.fixed) {
                if (modes & PL_FORCES) {
                    const double Fx = (tot[0] + tot[3]) + tot[6], Fy = (tot[1] + tot[4]) + tot[7];
                    const double T = (tot[2] + tot[5]) + tot[8];
                    n.U = q.U + Fx * st.inv_m + st.buoy * D.gx;
                    n.V = q.V + Fy * st.inv_m + st.buoy * D.gy;
                    n.Om = q.Om + T * st.inv_I;
                }
                n.x = nxp;
                n.y = nyp;
                n.th = q.th + q.Om;
                if (fabs(q.U) >= 1.0 || fabs(q.V) >= 1.0) atomicOr(a.err, ERR_STATE);  // faster than a node per step
            }
            a.state[(int64_t)(par ^ 1) * a.np + p] = n;
        }
        return;
    }

    // ---------------------------------------------------------------------- role B
    const int64_t t_next = advance ? t + 1 : t;
    const int wpar = (int)(t_next & 1);
    if (modes & PL_MARK) {
        // Work items (row segments) within two nodes of the disk's boxes at t
        // and t+1 are "near": the stream-collide pass of that step runs them
        // after this kernel, and they hold every node that changes side.
        const int mpar = (int)(t_next & 1);
        const int lpar = (int)(t_next % 3);
        const Box bo = disk_box(q.x, q.y, R), bn = disk_box(nxp, nyp, R);
        const int x0 = min(bo.x0, bn.x0) - 2, x1 = max(bo.x0 + bo.w, bn.x0 + bn.w) + 1;
        const int y0 = min(bo.y0, bn.y0) - 2, y1 = max(bo.y0 + bo.h, bn.y0 + bn.h) + 1;
        const int seg_w = 32 * D.V;
        for (int r = threadIdx.x; r <= y1 - y0; r += PBLOCK) {
            int y = y0 + r, xdummy = 0;
            if (!wrap_node(D, xdummy, y)) continue;
            for (int xx = x0;; xx += seg_w) {
                const int xc = xx < x1 ? xx : x1;
                int x = xc, yd = 0;
                if (wrap_node(D, x, yd)) {
                    const int64_t item = D.item_off + (int64_t)y * D.seg_per_row + x / seg_w;
                    int32_t* m = a.mark + (int64_t)mpar * a.total_items + item;
                    if (atomicExch(m, (int32_t)t_next) != (int32_t)t_next) {
                        const int slot = atomicAdd(a.near_cnt + lpar, 1);
                        a.near_list[(int64_t)lpar * a.total_items + slot] = (int32_t)item;
                    }
                }
                if (xc == x1) break;
            }
        }
    }
    if (!(modes & PL_RASTER)) return;

    // Particles whose disks at t+1 may touch this one's: they bound the exterior
    // nodes of the new links and reveal overlaps.
    near_list(a, D, p, S0, q.x, q.y, R, 6.0, near, near_d, &nnear, sh_warp);
    const int nn = nnear < MAXNEAR ? nnear : MAXNEAR;
    if (nnear > MAXNEAR && threadIdx.x == 0) atomicOr(a.err, ERR_STATE);
    if (threadIdx.x < nn) {
        const int p2 = near[threadIdx.x];
        const PartState o = S0[p2];
        double ox = o.x, oy = o.y;
        if (advance) next_position(D, o, a.st[p2].fixed, ox, oy);
        near_d[threadIdx.x] = make_diskf(ox, oy, a.st[p2].R);
    }
    // Union of the old and new boxes; every neighbour of a node inside either
    // disk lies in it.
    const Box bo = disk_box(q.x, q.y, R), bn = disk_box(nxp, nyp, R);
    Box U;
    U.x0 = min(bo.x0, bn.x0);
    U.y0 = min(bo.y0, bn.y0);
    U.w = max(bo.x0 + bo.w, bn.x0 + bn.w) - U.x0;
    U.h = max(bo.y0 + bo.h, bn.y0 + bn.h) - U.y0;
    const bool use_bm = U.n() <= PB_CAP;
    if (use_bm) {
        const DiskF kn = make_diskf(nxp, nyp, R), ko = make_diskf(q.x, q.y, R);
        for (int i = threadIdx.x; i < U.n(); i += PBLOCK) {
            const int xu = U.x0 + i % U.w, yu = U.y0 + i / U.w;
            sm.B.bnew[i] = inside_f(D, kn, xu, yu, true) ? 1 : 0;
            sm.B.bold[i] = advance ? (inside_f(D, ko, xu, yu, true) ? 1 : 0) : sm.B.bnew[i];
            // 0 = fluid node in the domain, 1 = solid, 2 = outside an open end
            int x = xu, y = yu;
            sm.B.node_st[i] = wrap_node(D, x, y) ? (a.solid[D.node_off + (int64_t)y * D.pitch + x] ? 1 : 0) : 2;
        }
    }
    __syncthreads();
    auto in_new = [&](int xu, int yu) -> bool {
        if (use_bm) return sm.B.bnew[(yu - U.y0) * U.w + (xu - U.x0)] != 0;
        int x = xu, y = yu;
        if (!wrap_node(D, x, y)) { x = xu; y = yu; }
        return inside_disk(D, nxp, nyp, R, x, y);
    };
    auto in_old = [&](int xu, int yu) -> bool {
        if (use_bm) return sm.B.bold[(yu - U.y0) * U.w + (xu - U.x0)] != 0;
        int x = xu, y = yu;
        if (!wrap_node(D, x, y)) { x = xu; y = yu; }
        return inside_disk(D, q.x, q.y, R, x, y);
    };
    int32_t* links = a.links + (int64_t)wpar * a.links_total;
    int32_t* flips = a.flips + (int64_t)wpar * a.flips_total;
    const int64_t stamp = (int64_t)(int32_t)(t + 1) << 32;
    int ltotal = 0, ftotal = 0;
    bool overlap = false;
    for (int t0 = 0; t0 < U.n(); t0 += PBLOCK) {
        const int i = t0 + threadIdx.x;
        uint32_t mask = 0;
        int node = 0, fcode = 0, fc = 0;
        if (i < U.n()) {
            const int xu = U.x0 + i % U.w, yu = U.y0 + i / U.w;
            int x = xu, y = yu;
            if (wrap_node(D, x, y)) {
                node = y * D.pitch + x;
                const bool solid_here = use_bm ? sm.B.node_st[i] == 1 : a.solid[D.node_off + node] != 0;
                const bool now = in_new(xu, yu);
                if (now) {
                    for (int j = 0; j < nn; ++j)
                        if (inside_f(D, near_d[j], xu, yu, true)) overlap = true;
                    if (!solid_here) {
#pragma unroll 1
                        for (int k = 1; k < 9; ++k) {
                            const int fxu = xu + cx(k), fyu = yu + cy(k);
                            if (use_bm) {
                                if (sm.B.node_st[(fyu - U.y0) * U.w + (fxu - U.x0)] != 0) continue;
                            } else {
                                int fx = fxu, fy = fyu;
                                if (!wrap_node(D, fx, fy)) continue;
                                if (a.solid[D.node_off + (int64_t)fy * D.pitch + fx]) continue;
                            }
                            bool in_any = in_new(fxu, fyu);
                            for (int j = 0; j < nn && !in_any; ++j) in_any = inside_f(D, near_d[j], fxu, fyu, true);
                            if (!in_any) mask |= 1u << k;
                        }
                    }
                }
                if (advance && !solid_here && now != in_old(xu, yu)) {
                    fc = 1;
                    fcode = (node << 1) | (now ? 1 : 0);
                }
            }
        }
        int excl;
        const int tot_l = block_scan(__popc(mask), sh_warp, excl);
        int w = ltotal + excl;
        for (int k = 1; k < 9; ++k)
            if (mask & (1u << k)) {
                if (w < st.link_cap) links[st.link_off + w] = (node << 3) | (k - 1);
                ++w;
            }
        ltotal += tot_l;
        int fex;
        const int tot_f = block_scan(fc, sh_warp, fex);
        if (fc && ftotal + fex < st.flip_cap) {
            const int64_t idx = st.flip_off + ftotal + fex;
            flips[idx] = fcode;
            // the stream-collide pass of this step leaves this node's moments in flipmom[slot]
            const int64_t slot = (int64_t)wpar * a.flips_total + idx;
            a.fliptag[D.node_off + node] = stamp | (uint32_t)slot;
        }
        ftotal += tot_f;
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

cudaError_t launch_particle_step(int kind, const PartArgs& a, int modes, cudaStream_t s) {
    if (a.np <= 0) return cudaSuccess;
    LBM_PDISPATCH(kind, (k_particle_step<S><<<2 * a.np, PBLOCK, 0, s>>>(a, modes)));
    return cudaGetLastError();
}

}  // namespace lbmk

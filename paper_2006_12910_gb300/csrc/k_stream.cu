// k_stream.cu -- fused pull-stream + collide kernel of the D2Q9 hot path
// (arXiv:2006.12910 Sec. 2 Eq. e.LB1 with the collision of Eq. e.LB2, the
// noise of Sec. 4 and the local tau* of Sec. 5; halfway bounce-back of Sec. 3).
//
// Layout: structure of arrays, plane i of domain d at arena[off + i*plane],
// rows of `pitch` elements, x fastest.  The stored values are the
// post-collision populations f*(t).  Each lane owns V consecutive nodes of
// one row (V*sizeof(T) = 16 bytes), a warp owns 32 such chunks; a work item
// is one (domain, row, warp segment).  For every direction the lane loads the
// 16-byte vector of the source row and, for the two x-shifted families, one
// extra element at the chunk edge (served by L1 from the neighbour lane's
// sector), then collides in registers and writes 16-byte vectors.
//
// Chunks that touch a wall, a solid, an open column or a periodic seam are
// flagged in a per-row bitmask; they read the per-node flag words and patch
// the pulled vectors in registers (bounce-back from the node's own opposite
// slot, Zou-He on the open columns), so they stay on the same vector path.
// Only the ragged last chunk of a row whose width is no multiple of V takes
// a scalar per-node path.
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

// Scalar per-node path for the ragged tail: pull with halfway bounce-back at
// walls / solids, wall-corner reflection and Zou-He on the open columns.
template <class S, bool NOISE, bool PL>
__device__ __noinline__ bool slow_node(const DomDev& D, const Prm<typename S::A>& P, int x, int y,
                                       const typename S::T* __restrict__ base, typename S::T* __restrict__ obase,
                                       const uint8_t* __restrict__ solid, uint32_t step) {
    typedef typename S::A A;
    const int nx = D.nx, ny = D.ny, pitch = D.pitch, flags = D.flags;
    const int64_t ni = (int64_t)y * pitch + x;
    if (__ldg(solid + D.node_off + ni)) return true;  // solid nodes hold no populations
    const A inv = P.inv_scale;
    const bool corner_row = (flags & FLAG_WY) && (y == 0 || y == ny - 1);
    A f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sx = x - cx(i), sy = y - cy(i);
        bool bb = false, unknown = false;
        if (sy < 0 || sy >= ny) {
            if (flags & FLAG_WY) bb = true;
            else sy = sy < 0 ? sy + ny : sy - ny;
        }
        if (!bb && (sx < 0 || sx >= nx)) {
            if (flags & FLAG_PX) sx = sx < 0 ? sx + nx : sx - nx;
            else if (corner_row) bb = true;
            else unknown = true;
        }
        if (!bb && !unknown && __ldg(solid + D.node_off + (int64_t)sy * pitch + sx)) bb = true;
        if (bb) f[i] = load_one<S>(base + (int64_t)opp(i) * D.plane + ni, inv);
        else if (unknown) f[i] = (A)0;
        else f[i] = load_one<S>(base + (int64_t)i * D.plane + (int64_t)sy * pitch + sx, inv);
    }
    if ((flags & FLAG_IO) && !corner_row && (x == 0 || x == nx - 1)) {
        if (x == 0) zou_he<A>(f, 0, P.rho_in, P.d_in);
        else zou_he<A>(f, 1, P.rho_out, P.d_out);
    }
    const bool ok = collide_node<A, S::SHIFT, NOISE, PL>(f, P, (uint32_t)((int64_t)y * nx + x), step);
#pragma unroll
    for (int i = 0; i < 9; ++i) from_a(f[i], P.scale, obase[(int64_t)i * D.plane + ni]);
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
    const int64_t tag = a.fliptag[D.node_off + ni];
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

// Everything after the pull of one V-node chunk: bounce-back and Zou-He
// patches from the per-node flag words (special chunks only), collision,
// 16-byte stores, and the moments of nodes that change side (near items).
template <class S, bool NOISE, bool PL, bool FLIPS>
__device__ __forceinline__ bool finish_chunk(const StreamArgs& a, const DomDev& D, const Prm<typename S::A>& P,
                                             typename S::A (&f)[9][S::V], bool special, int y, int x0,
                                             const typename S::T* base, typename S::T* obase, uint32_t step,
                                             bool near_item, int32_t next_stamp) {
    typedef typename S::A A;
    constexpr int V = S::V;
    const int64_t pitch = D.pitch, plane = D.plane;
    const int nx = D.nx;
    const A inv = P.inv_scale;
    bool ok = true;
    uint32_t solid_bits = 0;
    if (special) {
        uint16_t fl[V];
        load_flags<V>(a.nflags + D.node_off + (int64_t)y * pitch + x0, fl);
        uint32_t any = 0;
#pragma unroll
        for (int k = 0; k < V; ++k) any |= fl[k];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (any & (1u << i)) {  // halfway bounce-back: the node's own opposite slot
                A own[V];
                load_vec<S>(base + (int64_t)opp(i) * plane + y * pitch + x0, own, inv);
#pragma unroll
                for (int k = 0; k < V; ++k)
                    if (fl[k] & (1u << i)) f[i][k] = own[k];
            }
        }
        if (any & (NF_ZH_IN | NF_ZH_OUT)) {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                if (fl[k] & (NF_ZH_IN | NF_ZH_OUT)) {
                    A n9[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) n9[i] = f[i][k];
                    if (fl[k] & NF_ZH_IN) zou_he<A>(n9, 0, P.rho_in, P.d_in);
                    else zou_he<A>(n9, 1, P.rho_out, P.d_out);
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i][k] = n9[i];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < V; ++k)
            if (fl[k] & NF_SOLID) solid_bits |= 1u << k;
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
        A n9[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) n9[i] = f[i][k];
        const bool sol = (solid_bits >> k) & 1u;
        if (!sol) ok &= collide_node<A, S::SHIFT, NOISE, PL>(n9, P, (uint32_t)(y * nx + x0 + k), step);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i][k] = sol ? (A)0 : n9[i];
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) store_vec<S>(obase + (int64_t)i * plane + y * pitch + x0, f[i], P.scale);
    if (FLIPS && near_item) {
#pragma unroll 1
        for (int k = 0; k < V; ++k) flip_moments<S>(a, D, y, x0 + k, obase, next_stamp);
    }
    return ok;
}

template <class S, bool NOISE, bool PL, bool FLIPS>
__global__ void __launch_bounds__(512) k_stream_collide(StreamArgs a) {
    typedef typename S::T T;
    typedef typename S::A A;
    constexpr int V = S::V;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t step64 = *a.ctr_in;
    if (a.mode != STREAM_NEAR && blockIdx.x == 0 && threadIdx.x == 0) *a.ctr_out = step64 + 1;
    const uint32_t step = (uint32_t)step64;
    const int par = (int)(step64 & 1);
    const T* __restrict__ src = static_cast<const T*>(a.src);
    T* __restrict__ dst = static_cast<T*>(a.dst);
    bool ok = true;
    const int lpar = (int)(step64 % 3);
    const int64_t count = a.mode == STREAM_NEAR ? (int64_t)__ldg(a.near_cnt + lpar) : a.total_items;
    const int32_t next_stamp = (int32_t)(step64 + 1);

    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < count; w += nwarps) {
        int64_t g = w;
        int32_t mark = (int32_t)step64;
        if (a.mode == STREAM_NEAR) g = __ldg(a.near_list + (int64_t)lpar * a.total_items + w);
        else mark = __ldg(a.mark + (int64_t)par * a.total_items + w);  // consumed after the descriptor loads
        const int d = a.ndom == 1 ? 0 : find_domain(a.item_off, a.ndom, g);
        const DomDev& D = a.doms[d];
        const int nx = D.nx, ny = D.ny, flags = D.flags;
        const int64_t pitch = D.pitch, plane = D.plane;
        const int local = (int)(g - D.item_off);
        const int y = local / D.seg_per_row;
        const int seg = local - y * D.seg_per_row;
        const int x0 = (seg * 32 + lane) * V;
        const uint32_t word = __ldg(a.special + D.mask_off + (int64_t)y * D.seg_per_row + seg);
        const bool near_item = mark == (int32_t)step64;
        if (a.mode == STREAM_FAR && near_item) continue;
        if (x0 >= nx) continue;
        const Prm<A> P = load_prm<A>(D);
        const T* base = src + D.off;
        T* obase = dst + D.off;
        if (x0 + V > nx) {  // ragged tail chunk
#pragma unroll 1
            for (int k = 0; k < V; ++k)
                if (x0 + k < nx) {
                    ok &= slow_node<S, NOISE, PL>(D, P, x0 + k, y, base, obase, a.solid, step);
                    if (FLIPS && near_item) flip_moments<S>(a, D, y, x0 + k, obase, next_stamp);
                }
            continue;
        }
        const A inv = P.inv_scale;
        int ym = y - 1, yp = y + 1;
        if (ym < 0) ym = (flags & FLAG_PY) ? ny - 1 : y;   // a wall row pulls nothing from row -1
        if (yp >= ny) yp = (flags & FLAG_PY) ? 0 : y;
        int xl = x0 - 1, xr = x0 + V;
        if (xl < 0) xl = (flags & FLAG_PX) ? nx - 1 : 0;  // open ends: placeholder, patched below
        if (xr >= nx) xr = (flags & FLAG_PX) ? xr - nx : nx - 1;
        A f[9][V];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int row = cy(i) == 1 ? ym : (cy(i) == -1 ? yp : y);
            const T* p = base + (int64_t)i * plane + row * pitch;
            A v[V];
            load_vec<S>(p + x0, v, inv);
            if (cx(i) == 0) {
#pragma unroll
                for (int k = 0; k < V; ++k) f[i][k] = v[k];
            } else if (cx(i) == 1) {  // source x-1
                f[i][0] = load_one<S>(p + xl, inv);
#pragma unroll
                for (int k = 1; k < V; ++k) f[i][k] = v[k - 1];
            } else {  // source x+1
#pragma unroll
                for (int k = 0; k < V - 1; ++k) f[i][k] = v[k + 1];
                f[i][V - 1] = load_one<S>(p + xr, inv);
            }
        }
        ok &= finish_chunk<S, NOISE, PL, FLIPS>(a, D, P, f, ((word >> lane) & 1u) != 0, y, x0, base, obase, step,
                                                near_item, next_stamp);
    }
    if (!ok) atomicOr(a.err, ERR_UNSTABLE);
}

template <class S, bool FLIPS>
static cudaError_t launch_kind_f(bool noise, bool pl, const StreamArgs& a, int block, int64_t grid, cudaStream_t s) {
    if (noise && pl) k_stream_collide<S, true, true, FLIPS><<<(unsigned)grid, block, 0, s>>>(a);
    else if (noise) k_stream_collide<S, true, false, FLIPS><<<(unsigned)grid, block, 0, s>>>(a);
    else if (pl) k_stream_collide<S, false, true, FLIPS><<<(unsigned)grid, block, 0, s>>>(a);
    else k_stream_collide<S, false, false, FLIPS><<<(unsigned)grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

// The variant that writes the moments of nodes changing side runs the items
// near particles (mode STREAM_NEAR, or STREAM_ALL when particles exist).
template <class S>
static cudaError_t launch_kind(bool noise, bool pl, const StreamArgs& a, int block, int64_t grid, cudaStream_t s) {
    if (a.flips) return launch_kind_f<S, true>(noise, pl, a, block, grid, s);
    return launch_kind_f<S, false>(noise, pl, a, block, grid, s);
}

cudaError_t launch_stream_collide(int kind, bool noise, bool pl, const StreamArgs& a, int block, int64_t grid,
                                  cudaStream_t s) {
    switch (kind) {
        case 0: return launch_kind<StF64>(noise, pl, a, block, grid, s);
        case 1: return launch_kind<StF32>(noise, pl, a, block, grid, s);
        case 2: return launch_kind<StF32S>(noise, pl, a, block, grid, s);
        case 3: return launch_kind<StF16S>(noise, pl, a, block, grid, s);
        case 4: return launch_kind<StBF16S>(noise, pl, a, block, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int store_vector_width(int kind) {
    switch (kind) {
        case 0: return StF64::V;
        case 1: return StF32::V;
        case 2: return StF32S::V;
        case 3: return StF16S::V;
        case 4: return StBF16S::V;
        default: return 0;
    }
}

}  // namespace lbmk

// k_stream.cu -- fused pull-stream + collide kernel of the D2Q9 hot path
// (arXiv:2006.12910 Sec. 2 Eq. e.LB1 with the collision of Eq. e.LB2, the
// noise of Sec. 4 and the local tau* of Sec. 5; halfway bounce-back of Sec. 3).
//
// Layout: structure of arrays, plane i of domain d at arena[off + i*plane],
// rows of `pitch` elements, x fastest.  The stored values are the
// post-collision populations f*(t).  Each lane owns V consecutive nodes of
// one row (V*sizeof(T) = 8 or 16 bytes), a warp owns 32 such chunks; a work
// item is one (domain, row, warp segment).  For every direction the lane loads
// the vector of the source row and, for the two x-shifted families, one
// extra element at the chunk edge (served by L1 from the neighbour lane's
// sector), then collides in registers and writes 16-byte vectors.
//
// Halfway bounce-back needs no patching of the pull: solid nodes and the
// ghost rows beyond y walls hold, in the slot each fluid neighbour pulls, the
// value that neighbour bounced back (its mailbox write of the previous step).
// Chunks that hold a solid node, a mailbox writer, an open column or a
// wall-corner node are flagged in a per-row bitmask; they read their per-node
// flag words (Zou-He and corner patches, stores that leave solid slots alone,
// mailbox writes) and otherwise stay on the same vector path.  Only the
// ragged last chunk of a row whose width is no multiple of V takes a scalar
// per-node path.
#include "stream_node.cuh"

namespace lbmk {

// At most 128 threads per CTA, and the storage kind's resident CTAs per SM
// (MINB / MINB_EXT): the register cap they imply keeps the common variants
// from spilling while leaving room for as many warps as possible (plain FP32
// and half-precision kinds: 96 registers, 20 warps per SM).
template <class S, bool NOISE, bool PL>
constexpr int k1_min_blocks() { return (!NOISE && !PL) ? S::MINB : S::MINB_EXT; }

template <class S, bool NOISE, bool PL, bool FLIPS>
__global__ void __launch_bounds__(REG_K1_MAX_BLOCK, (k1_min_blocks<S, NOISE, PL>()))
    k_stream_collide(const __grid_constant__ StreamArgs a) {
    // A programmatic dependent launch waits here for the kernels before it
    // (completion and memory flush); otherwise this returns at once.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    typedef typename S::T T;
    typedef typename S::A A;
    constexpr int V = S::V;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t step64 = *a.ctr_in;
    // every pass writes the (same) counter of the next state, so whichever
    // pass a later kernel waits for has published it
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.ctr_out = step64 + 1;
    const uint32_t step = (uint32_t)step64;
    const int par = (int)(step64 % 3);
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
        else if (a.mode == STREAM_FAR || FLIPS) mark = __ldg(a.mark + (int64_t)par * a.total_items + w);
        const bool one = a.ndom == 1;
        const int d = one ? 0 : find_domain(a.item_off, a.ndom, g);
        const DomDev& D = a.doms[d];
        const Geo G = one ? param_geo(a.dom0) : load_geo(D);
        const int nx = G.nx;
        const int64_t pitch = G.pitch, plane = G.plane;
        const int local = (int)(g - G.item_off);
        const int y = item_row(G, local);
        const int seg = local - y * G.spr;
        const int x0 = (seg * 32 + lane) * V;
        const uint32_t word = __ldg(a.special + G.mask_off + (int64_t)y * G.spr + seg);
        const bool near_item = mark == (int32_t)step64;
        if (a.mode == STREAM_FAR && near_item) continue;
        if (x0 >= nx) continue;
        const HotPrm<A> H = one ? param_hot<A>(a.dom0) : load_hot<A>(D);
        const ExtPrm<A> X = load_ext<A, NOISE, PL>(one ? a.dom0 : D);
        const T* base = src + G.off;
        T* obase = dst + G.off;
        if (x0 + V > nx) {  // ragged tail chunk
#pragma unroll 1
            for (int k = 0; k < V; ++k)
                if (x0 + k < nx) {
                    ok &= slow_node<S, NOISE, PL>(D, x0 + k, y, base, obase, a.nflags, step);
                    if (FLIPS && near_item) flip_moments<S>(a, D, y, x0 + k, obase, next_stamp);
                }
            continue;
        }
        const bool special = ((word >> lane) & 1u) != 0;
        uint16_t fl[V];
#pragma unroll
        for (int k = 0; k < V; ++k) fl[k] = 0;
        if (special) load_flags<V>(a.nflags + G.node_off + y * pitch + x0, fl);
        // scaled half-precision stores stay in their scaled units (see collide_node)
        const A inv = S::SCALED ? (A)1 : H.inv_scale;
        int ym, yp;
        pull_rows(G, y, ym, yp);
        // x-1 / x+V across a seam: wrapped when periodic; at open ends any
        // in-range element stands in until the Zou-He or corner patch.
        int xl = x0 - 1, xr = x0 + V;
        if (xl < 0) xl = (G.flags & FLAG_PX) ? nx - 1 : 0;
        if (xr >= nx) xr = (G.flags & FLAG_PX) ? xr - nx : nx - 1;
        A f[9][V];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int row = cy(i) == 1 ? ym : (cy(i) == -1 ? yp : y);
            const T* p = base + (int64_t)i * plane + row * pitch;
            A v[V];
            if constexpr (S::SCALED) load_vec_raw<S>(p + x0, v);
            else load_vec<S>(p + x0, v, inv);
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
        ok &= finish_chunk<S, NOISE, PL, FLIPS>(a, D, G, H, X, f, special, fl, y, x0, base, obase, step, near_item,
                                                next_stamp);
    }
    if (!ok) atomicOr(a.err, ERR_UNSTABLE);
}

template <class S, bool NOISE, bool PL, bool FLIPS>
static cudaError_t launch_one(const StreamArgs& a, int block, int64_t grid, cudaStream_t s, bool pdl) {
    if (!pdl) {
        k_stream_collide<S, NOISE, PL, FLIPS><<<(unsigned)grid, block, 0, s>>>(a);
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
    return cudaLaunchKernelEx(&cfg, k_stream_collide<S, NOISE, PL, FLIPS>, a);
}

template <class S, bool FLIPS>
static cudaError_t launch_kind_f(bool noise, bool pl, const StreamArgs& a, int block, int64_t grid, cudaStream_t s,
                                 bool pdl) {
    if (noise && pl) return launch_one<S, true, true, FLIPS>(a, block, grid, s, pdl);
    if (noise) return launch_one<S, true, false, FLIPS>(a, block, grid, s, pdl);
    if (pl) return launch_one<S, false, true, FLIPS>(a, block, grid, s, pdl);
    return launch_one<S, false, false, FLIPS>(a, block, grid, s, pdl);
}

// The variant that writes the moments of nodes changing side runs the items
// near particles (mode STREAM_NEAR, or STREAM_ALL when particles exist).
template <class S>
static cudaError_t launch_kind(bool noise, bool pl, const StreamArgs& a, int block, int64_t grid, cudaStream_t s,
                               bool pdl) {
    if (a.flips) return launch_kind_f<S, true>(noise, pl, a, block, grid, s, pdl);
    return launch_kind_f<S, false>(noise, pl, a, block, grid, s, pdl);
}

cudaError_t launch_stream_staged(int kind, bool noise, bool pl, const StreamArgs& a, int block, int64_t grid,
                                 int stages, cudaStream_t s);

cudaError_t launch_stream_collide(int kind, bool noise, bool pl, const StreamArgs& a, int block, int64_t grid,
                                  int stages, cudaStream_t s, bool pdl) {
    if (stages > 0 && a.mode != STREAM_NEAR) return launch_stream_staged(kind, noise, pl, a, block, grid, stages, s);
    switch (kind) {
        case 0: return launch_kind<StF64>(noise, pl, a, block, grid, s, pdl);
        case 1: return launch_kind<StF32>(noise, pl, a, block, grid, s, pdl);
        case 2: return launch_kind<StF32S>(noise, pl, a, block, grid, s, pdl);
        case 3: return launch_kind<StF16S>(noise, pl, a, block, grid, s, pdl);
        case 4: return launch_kind<StBF16S>(noise, pl, a, block, grid, s, pdl);
        default: return cudaErrorInvalidValue;
    }
}

template <class S>
static int reg_bps(bool noise, bool pl, int block) {
    int n = 0;
    cudaError_t e;
    if (noise && pl) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stream_collide<S, true, true, false>, block, 0);
    else if (noise) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stream_collide<S, true, false, false>, block, 0);
    else if (pl) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stream_collide<S, false, true, false>, block, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stream_collide<S, false, false, false>, block, 0);
    return e == cudaSuccess ? n : 0;
}

int reg_blocks_per_sm(int kind, bool noise, bool pl, int block) {
    if (block < 32 || block > REG_K1_MAX_BLOCK) return 0;
    switch (kind) {
        case 0: return reg_bps<StF64>(noise, pl, block);
        case 1: return reg_bps<StF32>(noise, pl, block);
        case 2: return reg_bps<StF32S>(noise, pl, block);
        case 3: return reg_bps<StF16S>(noise, pl, block);
        case 4: return reg_bps<StBF16S>(noise, pl, block);
        default: return 0;
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

// k_staged.cu -- fused pull-stream + collide, staged through shared memory
// with bulk asynchronous copies (arXiv:2006.12910 Sec. 2 Eqs. e.LB1 / e.LB2,
// bounce-back and Zou-He of Sec. 3, noise of Sec. 4, local tau* of Sec. 5).
//
// Same work items as k_stream.cu (one item = one domain row segment of
// 32 * V nodes), but nothing of an item passes through registers before it
// is needed.  One lane of the warp issues nine cp.async.bulk copies (one per
// direction plane, from the row that direction pulls from) and, for segments
// with flagged nodes, one copy of the flag words, into a shared-memory stage,
// and arms the stage's mbarrier with the expected byte count; each warp keeps
// `stages` items in flight and computes the oldest while the others stream
// in, so the bytes in flight per SM are set by shared memory, not registers.
//
// A stage holds, per plane, the segment plus one 16-byte halo on each side:
// element j of a plane row is x = xs - E + j (xs the segment's first node,
// E = 16 / sizeof(T)), clipped to [0, pitch) at the row ends.  Lane l then
// takes nodes xs + l + 32 k one at a time: the nine pulled values are plain
// shared-memory reads at x - e_ix, so only one node's populations are live in
// registers, and every store of the warp writes 32 consecutive elements.
// Only nodes at x = 0 or nx - 1 read a wrapped source from global memory
// (periodic x) or take the Zou-He / corner patch (open ends).  Every mbarrier
// wait is bounded (about one second by the global timer); a wait that runs
// out sets ERR_TIMEOUT, waits (bounded again, always by the full second) for
// the warp's copies in flight and ends the warp's work.  The limit of the
// stage waits comes with the launch (StreamArgs::wait_ns).
#include "stream_node.cuh"

namespace lbmk {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Orders this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;  // one second
constexpr uint32_t WAIT_LIMIT_ITERS = 1u << 26;     // backstop if the timer stalls

// Bounded wait for the phase of parity `parity` of one mbarrier, at most
// limit_ns of the global timer.  limit_ns == 0 reports expiry at once without
// looking at the barrier (the context's test setting that makes every stage
// wait run out; the copies it skipped are still drained with the full limit).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    if (limit_ns == 0) return false;
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < WAIT_LIMIT_ITERS; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// A node at x = 0 or nx - 1: sources beyond the x range are read wrapped
// (periodic x) or patched (Zou-He column, wall-corner reflection).
template <class S>
__device__ __noinline__ void seam_node(const DomDev& D, const typename S::T* base, int x, int y, uint32_t fl,
                                       typename S::A* f) {
    typedef typename S::A A;
    const Geo G = load_geo(D);
    // scaled half-precision stores stay in their scaled units (collide_node<..., SC>)
    const A inv = S::SCALED ? (A)1 : (A)(sizeof(A) == 4 ? D.inv_scale_f : D.inv_scale);
    const A sc = S::SCALED ? (A)(sizeof(A) == 4 ? D.scale_f : D.scale) : (A)1;
    int ym, yp;
    pull_rows(G, y, ym, yp);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int sx = x - cx(i);
        if (sx < 0 || sx >= G.nx) {
            const int row = cy(i) == 1 ? ym : (cy(i) == -1 ? yp : y);
            if (G.flags & FLAG_PX)
                f[i] = load_one<S>(base + (int64_t)i * G.plane + (int64_t)row * G.pitch + (sx < 0 ? G.nx - 1 : 0), inv);
            else if (fl & NF_CORNER)
                f[i] = load_one<S>(base + (int64_t)opp(i) * G.plane + (int64_t)y * G.pitch + x, inv);
            else
                f[i] = (A)0;
        }
    }
    if (fl & NF_ZH_IN) zou_he<A>(f, 0, zou_he_excess<A>(D, 0) * sc);
    else if (fl & NF_ZH_OUT) zou_he<A>(f, 1, zou_he_excess<A>(D, 1) * sc);
}

// Mailbox writes of one node (flag bits 1..8), out of line.
template <class S>
__device__ __noinline__ void mail_call(const DomDev& D, typename S::T* obase, int x, int y, uint32_t fl,
                                       const typename S::A* f) {
    typedef typename S::A A;
    const Geo G = load_geo(D);
    A v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = f[i];
    // f is in the store's scaled units when S::SCALED: written without scaling
    mail_node<S>(G, obase, x, y, fl, v, S::SCALED ? (A)1 : (A)(sizeof(A) == 4 ? D.scale_f : D.scale));
}

template <class S>
struct StageGeom {
    typedef typename S::T T;
    static constexpr int V = S::V;
    static constexpr int NW = 32 * V;                   // nodes of a work item (one row segment)
    static constexpr int E = 16 / (int)sizeof(T);      // halo elements per side
    static constexpr int ROWE = NW + 2 * E;             // elements per plane row in a stage
    static constexpr int ROWS_B = 9 * ROWE * (int)sizeof(T);
    static constexpr int FLAGS_B = NW * 2;              // the item's flag words
    static constexpr int STAGE_B = ROWS_B + FLAGS_B;
    static_assert(ROWS_B % 16 == 0 && FLAGS_B % 16 == 0, "stage parts must keep 16-byte alignment");
};

// Per warp and stage, besides the data: the descriptor of the item it holds
// (16 bytes; all descriptors first, so each stays 16-byte aligned) and one
// mbarrier (8 bytes).
constexpr int STAGE_META_B = 8 + 16;

template <class S>
__host__ __device__ constexpr size_t staged_bytes(int warps, int stages) {
    return (size_t)warps * stages * (StageGeom<S>::STAGE_B + STAGE_META_B);
}

template <class S, bool NOISE, bool PL, bool FLIPS>
__global__ void __launch_bounds__(STAGED_MAX_BLOCK) k_stream_staged(StreamArgs a, int stages) {
    typedef typename S::T T;
    typedef typename S::A A;
    typedef StageGeom<S> SG;
    constexpr int V = S::V, NW = SG::NW, E = SG::E, ROWE = SG::ROWE;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    unsigned char* wbuf = smem_raw + (size_t)wib * stages * SG::STAGE_B;
    unsigned char* meta = smem_raw + (size_t)wpb * stages * SG::STAGE_B;  // 16-byte aligned
    int4* info = reinterpret_cast<int4*>(meta) + (size_t)wib * stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(meta + (size_t)wpb * stages * 16) + (size_t)wib * stages;

    const int64_t nwarps = (int64_t)gridDim.x * wpb;
    const int64_t wg = (int64_t)blockIdx.x * wpb + wib;
    const int64_t step64 = *a.ctr_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.ctr_out = step64 + 1;
    const uint32_t step = (uint32_t)step64;
    const int par = (int)(step64 % 3);
    const int32_t next_stamp = (int32_t)(step64 + 1);
    const bool far_only = a.mode == STREAM_FAR;
    const T* __restrict__ src = static_cast<const T*>(a.src);
    T* __restrict__ dst = static_cast<T*>(a.dst);
    const int64_t count = a.total_items;

    if (lane == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(smem_u32(bars + s), 1);
        mbar_init_fence();
    }
    __syncwarp();

    // Candidate items of this warp: g = wg + c * nwarps, c = 0, 1, ...; they
    // are screened 32 at a time (one per lane) for the FAR-mode skip, and the
    // lane that screened a candidate also decodes it (domain, row, segment,
    // whether any node of the segment has flags), spreading the decoding
    // over the lanes.
    int64_t cbase = 0;
    uint32_t keep = 0;
    int c_dn = 0, c_y = 0, c_seg = 0;
    bool batch_left = true;  // candidates from cbase on may exist
    auto load_batch = [&]() {
        const int64_t g = wg + (cbase + lane) * nwarps;
        const bool valid = g < count;
        int near = 0, d = 0, y = 0, seg = 0, spec = 0;
        if (valid) {
            near = __ldg(a.mark + (int64_t)par * a.total_items + g) == (int32_t)step64;
            d = a.ndom == 1 ? 0 : find_domain(a.item_off, a.ndom, g);
            const Geo G = load_geo(a.doms[d]);
            const int local = (int)(g - G.item_off);
            y = local / G.spr;
            seg = local - y * G.spr;
            spec = __ldg(a.special + G.mask_off + (int64_t)y * G.spr + seg) != 0u;
        }
        keep = __ballot_sync(0xffffffffu, valid && !(far_only && near));
        c_dn = d | (near << 31);
        c_y = y;
        c_seg = seg | (spec << 30);
        batch_left = wg + (cbase + 32) * nwarps < count;
    };
    load_batch();

    // Issue the next kept candidate into stage s; false when none is left.
    // Nine row copies (one per direction plane, from the row it pulls from,
    // with a 16-byte halo on each side clipped to the row) and, for segments
    // with flagged nodes, the segment's flag words.
    auto issue = [&](int s) -> bool {
        while (keep == 0) {
            if (!batch_left) return false;
            cbase += 32;
            load_batch();
        }
        const int c = __ffs(keep) - 1;
        keep &= keep - 1;
        const int dn = __shfl_sync(0xffffffffu, c_dn, c);
        const int y = __shfl_sync(0xffffffffu, c_y, c);
        const int sg = __shfl_sync(0xffffffffu, c_seg, c);
        if (lane == 0) {
            const Geo G = load_geo(a.doms[dn & 0x7fffffff]);
            const int64_t pitch = G.pitch;
            const int seg = sg & 0x3fffffff;
            const int64_t xs = (int64_t)seg * NW;
            int ym, yp;
            pull_rows(G, y, ym, yp);
            const int64_t w0 = xs >= E ? xs - E : 0;
            const int64_t w1 = xs + NW + E < pitch ? xs + NW + E : pitch;
            const uint32_t bytes = (uint32_t)((w1 - w0) * (int64_t)sizeof(T));
            const bool spec = (sg >> 30) & 1;
            const int64_t f1 = xs + NW < pitch ? xs + NW : pitch;
            const uint32_t fbytes = spec ? (uint32_t)((f1 - xs) * 2) : 0u;
            info[s] = make_int4(dn, y, sg, 0);
            const uint32_t bar = smem_u32(bars + s);
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, 9u * bytes + fbytes);
            unsigned char* st = wbuf + (size_t)s * SG::STAGE_B;
            const uint32_t dst0 = smem_u32(st) + (uint32_t)((w0 - (xs - E)) * (int64_t)sizeof(T));
            const T* base = src + G.off;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int row = cy(i) == 1 ? ym : (cy(i) == -1 ? yp : y);
                bulk_copy_g2s(dst0 + (uint32_t)(i * ROWE * (int)sizeof(T)), base + i * G.plane + row * pitch + w0,
                              bytes, bar);
            }
            if (spec) bulk_copy_g2s(smem_u32(st + SG::ROWS_B), a.nflags + G.node_off + y * pitch + xs, fbytes, bar);
        }
        __syncwarp();
        return true;
    };

    uint32_t pending = 0, phase = 0;
    for (int s = 0; s < stages; ++s) {
        if (!issue(s)) break;
        pending |= 1u << s;
    }
    bool ok = true, aborted = false;
    int sc = 0;
    while (pending & (1u << sc)) {
        const int4 it = info[sc];
        const int d = it.x & 0x7fffffff;
        const bool near_item = it.x < 0;
        const int y = it.y, seg = it.z & 0x3fffffff;
        const bool spec = (it.z >> 30) & 1;
        const DomDev& D = a.doms[d];
        const Geo G = load_geo(D);
        const int nx = G.nx;
        const int64_t pitch = G.pitch, plane = G.plane;
        const int xs = seg * NW;
        const T* base = src + G.off;
        T* obase = dst + G.off;
        T* orow = obase + y * pitch + xs;
        const HotPrm<A> H = load_hot<A>(D);
        const ExtPrm<A> X = load_ext<A, NOISE, PL>(D);
        // scaled half-precision stores stay in their scaled units, as in the register kernel
        const A inv = S::SCALED ? (A)1 : H.inv_scale;
        const A osc = S::SCALED ? (A)1 : H.scale;
        int ym, yp;
        pull_rows(G, y, ym, yp);
        const bool done = mbar_wait_bounded(smem_u32(bars + sc), (phase >> sc) & 1u, a.wait_ns);
        if (__any_sync(0xffffffffu, !done)) {
            aborted = true;
            break;
        }
        phase ^= 1u << sc;
        pending &= ~(1u << sc);

        const T* sb = reinterpret_cast<const T*>(wbuf + (size_t)sc * SG::STAGE_B);
        const uint16_t* sfl = reinterpret_cast<const uint16_t*>(wbuf + (size_t)sc * SG::STAGE_B + SG::ROWS_B);
        // Lane l takes nodes xs + l + 32 k: every shared-memory read and every
        // global store of the warp covers 32 consecutive elements.
#pragma unroll 2
        for (int k = 0; k < V; ++k) {
            const int j = lane + 32 * k;
            const int x = xs + j;
            if (x >= nx) continue;
            const uint32_t fl = spec ? (uint32_t)sfl[j] : 0u;
            if (fl & NF_SOLID) continue;  // solid slots are mailboxes, written by their fluid neighbours
            A f[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = to_a(sb[i * ROWE + E + j - cx(i)], inv);
            if (x == 0 || x == nx - 1) {  // rare: through a local copy, so f stays in registers
                A t[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) t[i] = f[i];
                seam_node<S>(D, base, x, y, fl, t);
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = t[i];
            }
            ok &= collide_node<A, S::SHIFT, NOISE, PL, S::SCALED>(f, H, X, (uint32_t)(y * nx + x), step);
#pragma unroll
            for (int i = 0; i < 9; ++i) from_a(f[i], osc, orow[(int64_t)i * plane + j]);
            if (fl & 0x1FEu) {
                if (mail_is_direct(G, x, y)) {
                    mail_direct<S>(orow + j, plane, pitch, fl, f, osc);
                } else {  // rare: wrapped targets, out of line through a local copy
                    A t[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) t[i] = f[i];
                    mail_call<S>(D, obase, x, y, fl, t);
                }
            }
            if (FLIPS && near_item) flip_moments<S>(a, D, y, x, obase, next_stamp);
        }
        __syncwarp();
        if (issue(sc)) pending |= 1u << sc;
        sc = sc + 1 == stages ? 0 : sc + 1;
    }
    if (aborted) {
        // Leave no copy in flight into shared memory this CTA gives up.
        if (lane == 0) atomicOr(a.err, ERR_TIMEOUT);
        for (int s = 0; s < stages; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(smem_u32(bars + s), (phase >> s) & 1u, WAIT_LIMIT_NS);
        __syncwarp();
    }
    if (!ok) atomicOr(a.err, ERR_UNSTABLE);
}

template <class S>
const void* staged_kernel(bool noise, bool pl, bool flips) {
    if (flips) {
        if (noise && pl) return (const void*)k_stream_staged<S, true, true, true>;
        if (noise) return (const void*)k_stream_staged<S, true, false, true>;
        if (pl) return (const void*)k_stream_staged<S, false, true, true>;
        return (const void*)k_stream_staged<S, false, false, true>;
    }
    if (noise && pl) return (const void*)k_stream_staged<S, true, true, false>;
    if (noise) return (const void*)k_stream_staged<S, true, false, false>;
    if (pl) return (const void*)k_stream_staged<S, false, true, false>;
    return (const void*)k_stream_staged<S, false, false, false>;
}

const void* staged_kernel_for(int kind, bool noise, bool pl, bool flips) {
    switch (kind) {
        case 0: return staged_kernel<StF64>(noise, pl, flips);
        case 1: return staged_kernel<StF32>(noise, pl, flips);
        case 2: return staged_kernel<StF32S>(noise, pl, flips);
        case 3: return staged_kernel<StF16S>(noise, pl, flips);
        case 4: return staged_kernel<StBF16S>(noise, pl, flips);
        default: return nullptr;
    }
}

bool staged_args_ok(int kind, int block, int stages) {
    return kind >= 0 && kind <= 4 && block >= 32 && block <= STAGED_MAX_BLOCK && block % 32 == 0 && stages >= 1 &&
           stages <= STAGED_MAX_STAGES;
}

// Prefer the largest shared-memory carveout and raise the kernel's dynamic
// shared-memory limit to what this launch needs.
cudaError_t prepare(const void* k, size_t bytes) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    if (fa.preferredShmemCarveout != 100) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
    }
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t staged_smem_bytes(int kind, int block, int stages) {
    if (!staged_args_ok(kind, block, stages)) return 0;
    const int w = block / 32;
    switch (kind) {
        case 0: return staged_bytes<StF64>(w, stages);
        case 1: return staged_bytes<StF32>(w, stages);
        case 2: return staged_bytes<StF32S>(w, stages);
        case 3: return staged_bytes<StF16S>(w, stages);
        default: return staged_bytes<StBF16S>(w, stages);
    }
}

int staged_blocks_per_sm(int kind, bool noise, bool pl, int block, int stages) {
    const size_t bytes = staged_smem_bytes(kind, block, stages);
    if (!bytes) return 0;
    const void* k = staged_kernel_for(kind, noise, pl, false);
    if (prepare(k, bytes) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, bytes) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_stream_staged(int kind, bool noise, bool pl, const StreamArgs& a, int block, int64_t grid,
                                 int stages, cudaStream_t s) {
    if (!staged_args_ok(kind, block, stages) || a.mode == STREAM_NEAR || grid < 1) return cudaErrorInvalidValue;
    if ((uint64_t)a.total_items >= (1ull << 31)) return cudaErrorInvalidValue;  // item ids travel as int32
    const size_t bytes = staged_smem_bytes(kind, block, stages);
    const void* k = staged_kernel_for(kind, noise, pl, a.flips != 0);
    cudaError_t e = prepare(k, bytes);
    if (e != cudaSuccess) return e;
    StreamArgs args = a;
    int st = stages;
    void* params[] = {&args, &st};
    return cudaLaunchKernel(k, dim3((unsigned)grid), dim3((unsigned)block), params, bytes, s);
}

}  // namespace lbmk

// capi.cu -- host runtime and C ABI of the GB300 D2Q9 library (include/lbm.h).
//
// The context owns every device buffer: two population arenas (the state
// f*(t) and the next state), per-node solid bytes, the per-chunk slow-path
// bitmask, the step counters, a sticky error word and the particle arrays.
// lbm_step replays CUDA graphs of 2^j timesteps, j = 0 .. GRAPH_LOG (the
// binary digits of the step count, largest first); a timestep is
//   [particle forces + Newton-Euler] -> [link exchange + re-rasterise]
//   -> [fused pull-stream + collide over every domain]
// where the two particle kernels are skipped when no domain holds particles.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "kernels.h"

using namespace lbmk;

namespace {

// Step graphs hold 1, 2, 4, .. 2^GRAPH_LOG timesteps.  Every graph launch
// ends with the whole chain drained (the particle launches run one and two
// steps ahead of the stream-collide passes inside a graph), so fewer, longer
// graphs keep the overlapped step at its steady rate: lbm_step(n) launches
// one graph per binary digit of n mod 2^GRAPH_LOG plus n >> GRAPH_LOG of the
// largest.
constexpr int GRAPH_LOG = 6;
thread_local std::string g_create_error = "no error";

// Test hook of lbm_debug_fail_alloc: when positive, the device allocation
// that brings it to zero fails as an exhausted device would.
std::atomic<int> g_fail_alloc{0};

// Every device allocation of the library goes through here.
template <class T>
cudaError_t dev_malloc(T** p, size_t bytes) {
    int n = g_fail_alloc.load();
    while (n > 0 && !g_fail_alloc.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

size_t elem_bytes(int kind) { return kind == 0 ? 8 : (kind <= 2 ? 4 : 2); }

}  // namespace

struct lbm_ctx {
    int ndom = 0;
    int kind = 2;
    size_t esz = 4;
    int V = 4;
    std::vector<lbm_params> prm;
    std::vector<DomDev> hd;
    std::vector<std::vector<uint8_t>> hsolid;  // host copy of each domain's mask (ny*nx)
    DomDev* dd = nullptr;
    int64_t* d_item_off = nullptr;
    int64_t total_items = 0;
    void* f[2] = {nullptr, nullptr};
    size_t arena_elems = 0;
    uint8_t* solid = nullptr;
    uint16_t* nflags = nullptr;
    size_t node_bytes = 0;
    uint32_t* special = nullptr;
    size_t special_words = 0;
    int64_t* ctr = nullptr;   // [2]
    int64_t* pstep = nullptr; // [2]: by arena, the step after the last particle force launch from it
    unsigned* err = nullptr;  // sticky
    bool noise = false, pl = false;

    // particles: max_particles slots per domain, contiguous per domain
    int np_slots = 0;
    int np_active = 0;
    std::vector<PartStatic> hst;
    std::vector<PartState> hstate;  // host shadow used while adding
    PartState* pstate = nullptr;          // [2][np_slots], slot (step & 1) is current
    PartStatic* pst = nullptr;
    int32_t* links = nullptr;
    int32_t* nlinks = nullptr;
    int32_t* flips = nullptr;
    int32_t* nflips = nullptr;
    double* diag = nullptr;
    int64_t links_total = 0, flips_total = 0;

    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t side = nullptr;
    cudaStream_t far_stream = nullptr;   // branch running the far stream-collide items
    cudaStream_t rast_stream = nullptr;  // branch running the rasterisation of the next step
    cudaStream_t lj_stream = nullptr;    // branch running the Eq. MP2 sums two steps ahead
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr, ev_join3 = nullptr;
    cudaEvent_t ev_a[2] = {nullptr, nullptr}, ev_rast[2] = {nullptr, nullptr}, ev_lj[2] = {nullptr, nullptr};
    cudaEvent_t ev_far[2] = {nullptr, nullptr}, ev_near[2] = {nullptr, nullptr};  // per-step edges inside a graph
    bool overlap = true;                 // far items run concurrently with the particle kernels
    int32_t* mark = nullptr;             // [3][total_items]
    int32_t* near_list = nullptr;        // [3][total_items]
    int32_t* near_cnt = nullptr;         // [3]
    int64_t* fliptag = nullptr;          // [2][nodes], copy by the parity of the tag's step
    double* ljf = nullptr;               // [2][np_slots][4]: Eq. MP2 force and torque, copy by step parity
    double* flipmom = nullptr;           // [2][flips_total][3]
    int64_t near_grid = 1;
    LjEntry* lj_tab = nullptr;           // [ndom][LJ_TAB]
    double2* ljwall = nullptr;           // per node: Eq. MP2 force from walls / solids (domains with psi > 0)
    int32_t* lj_cnt = nullptr;           // [ndom]
    cudaEvent_t ev_snap = nullptr, ev_copied = nullptr;
    // Recorded inside every step graph right after the last particle force
    // launch (which writes the particle state of the graph's last step).
    // pstate_evt: the latest write of the particle state that was enqueued is
    // that launch, so lbm_particles may wait for this event alone.
    cudaEvent_t ev_pstate = nullptr;
    bool pstate_evt = false;
    // gexec[k][j]: 2^j steps from state k, so that any lbm_step(n) runs as
    // whole multi-step graphs (the cross-step overlap of the particle and
    // stream-collide chains holds inside every graph)
    cudaGraphExec_t gexec[2][GRAPH_LOG + 1] = {};
    // trajectory records (lbm_record_particles): device address of the
    // caller's page-locked buffer and its capacity in steps
    PartState* rec = nullptr;
    int64_t rec_cap = 0;
    // step counts prepared by lbm_prepare_steps and their graphs from state
    // 0 / 1 (index-aligned)
    std::vector<int64_t> prepared;
    std::vector<cudaGraphExec_t> gprep[2];
    bool graph_dirty = true;
    uint64_t wait_ns = 1000000000ull;  // limit of the bounded device waits (lbm_set_wait_limit)

    int cur = 0;
    int64_t steps = 0;
    int block = 128;
    // 0: one warp item per warp; 1: grid-stride over 16 CTAs per SM; 2: staged
    // kernel; 3: grid-stride over the CTAs that fit the SMs at once; 4:
    // grid-stride over 8 CTAs per SM
    int grid_mode = 1;
    int stages = 0;     // row segments in flight per warp of the staged kernel
    int64_t grid = 1;

    double* d_stage = nullptr;
    size_t d_stage_bytes = 0;
    double* d_partial = nullptr;
    double* d_sums = nullptr;
    float* d_mom = nullptr;
    float* h_mom = nullptr;
    unsigned char* h_pin = nullptr;  // pinned: error word at 0, particle states from PIN_HEAD
    size_t h_pin_bytes = 0;
    size_t mom_elems = 0;
    int mom_pending = 0;

    std::string msg = "no error";
};

namespace {

int fail(lbm_ctx* c, int code, const std::string& m) {
    if (c) c->msg = m;
    else g_create_error = m;
    return code;
}

#define CKC(ctx, call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? LBM_E_NOMEM : LBM_E_CUDA,    \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                \
    } while (0)

int validate(const lbm_params& p, int d, lbm_ctx* c) {
    char b[256];
    auto bad = [&](const char* what) {
        snprintf(b, sizeof b, "domain %d: %s", d, what);
        return fail(c, LBM_E_INVAL, b);
    };
    if (p.nx < 3 || p.ny < 3) return bad("nx and ny must be >= 3");
    if ((int64_t)p.nx * p.ny > (int64_t)1 << 28) return bad("domain larger than 2^28 nodes");
    if ((p.periodic_x != 0) == (p.inlet_outlet != 0)) return bad("exactly one of periodic_x / inlet_outlet");
    if ((p.periodic_y != 0) == (p.walls_y != 0)) return bad("exactly one of periodic_y / walls_y");
    if (!(p.tau > 0.5) || !std::isfinite(p.tau)) return bad("tau must be > 1/2");
    if (!(p.rho0 > 0.0)) return bad("rho0 must be > 0");
    if (!(p.kT >= 0.0)) return bad("kT must be >= 0");
    if (p.store < 0 || p.store > 4) return bad("unknown store kind");
    if ((p.store == LBM_F16S || p.store == LBM_BF16S) && !(p.store_scale > 0.0)) return bad("store_scale must be > 0");
    if (p.inlet_outlet && (!(p.rho_in > 0.0) || !(p.rho_out > 0.0))) return bad("rho_in / rho_out must be > 0");
    if (p.power_law) {
        if (!(p.n_pl > 0.0) || !(p.xi_pl > 0.0)) return bad("power law needs n > 0 and xi > 0");
        if (!(p.kappa_pl >= 0.0)) return bad("kappa_pl must be >= 0 (0: 2^(n-1))");
        if (!(p.tau_min > 0.5) || !(p.tau_max > p.tau_min)) return bad("power law needs 1/2 < tau_min < tau_max");
    }
    if (p.max_particles < 0 || p.max_particles > 4096) return bad("max_particles must be in [0, 4096]");
    if (!(p.lj_psi >= 0.0) || !(p.lj_rit >= 0.0)) return bad("lj_psi and lj_rit must be >= 0");
    if (p.lj_psi > 0.0 && !(p.lj_rit < 6.0)) return bad("lj_rit must be < 6 (offset table size)");
    return LBM_OK;
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

void fill_dom(DomDev& D, const lbm_params& p, int kind) {
    memset(&D, 0, sizeof D);
    D.nx = p.nx;
    D.ny = p.ny;
    D.flags = (p.periodic_x ? FLAG_PX : 0) | (p.periodic_y ? FLAG_PY : 0) | (p.walls_y ? FLAG_WY : 0) |
              (p.inlet_outlet ? FLAG_IO : 0);
    D.V = store_vector_width(kind);
    D.pitch = (int32_t)round_up(p.nx, std::max<int64_t>(D.V, 128 / (int64_t)elem_bytes(kind)));
    // y walls: one ghost row on each side of every plane (bounce-back mailboxes)
    D.plane = (int64_t)D.pitch * (p.ny + (p.walls_y ? 2 : 0));
    const int nchunks = (p.nx + D.V - 1) / D.V;
    D.seg_per_row = (nchunks + 31) / 32;
    // Division by the invariant seg_per_row as a multiply-high (Granlund and
    // Montgomery, PLDI 1994): with m = floor(2^32 / d) + 1, floor(n m / 2^32)
    // = floor(n / d) whenever n d < 2^32, here for every item n of the domain.
    {
        const uint64_t d = (uint64_t)D.seg_per_row, items = (uint64_t)p.ny * d;
        D.spr_magic = (d > 1 && items * d < ((uint64_t)1 << 32)) ? (uint32_t)(((uint64_t)1 << 32) / d + 1) : 0u;
    }
    D.seed = p.seed;
    D.domain_id = p.domain_id;
    D.tau = p.tau;
    D.inv_tau = 1.0 / p.tau;
    D.rho0 = p.rho0;
    D.gx = p.gx;
    D.gy = p.gy;
    D.rho_in = p.rho_in;
    D.rho_out = p.rho_out;
    const bool shifted = kind >= 2;
    D.drho_in = shifted ? p.rho_in - p.rho0 : p.rho_in;
    D.drho_out = shifted ? p.rho_out - p.rho0 : p.rho_out;
    D.kT = p.kT;
    D.n_pl = p.power_law ? p.n_pl : 1.0;
    // Eq. nn4, nu* = xi kappa |Pi_D|^((n-1)/2) with gamma-dot = 2 sqrt|Pi_D|, is
    // xi kappa 2^(1-n) gamma-dot^(n-1): the kernels take the consistency times
    // kappa / 2^(n-1) (1 for the paper's kappa = 2^(n-1)).
    D.xi_pl = p.xi_pl;
    if (p.power_law && p.kappa_pl > 0.0) D.xi_pl = p.xi_pl * p.kappa_pl / std::pow(2.0, p.n_pl - 1.0);
    D.tau_min = p.tau_min;
    D.tau_max = p.tau_max;
    D.n_is_one = p.power_law ? (p.n_pl == 1.0) : 1;
    if (p.power_law) {
        D.tmin_pow = std::pow(p.tau_min, 1.0 - p.n_pl);
        D.tmax_pow = std::pow(p.tau_max, 1.0 - p.n_pl);
    }
    D.lj_psi = p.lj_psi;
    D.lj_rit = p.lj_rit;
    const bool scaled = kind == LBM_F16S || kind == LBM_BF16S;
    D.scale = scaled ? p.store_scale : 1.0;
    D.inv_scale = scaled ? 1.0 / p.store_scale : 1.0;
    D.tau_f = (float)D.tau; D.inv_tau_f = (float)D.inv_tau; D.rho0_f = (float)D.rho0;
    D.gx_f = (float)D.gx; D.gy_f = (float)D.gy; D.rho_in_f = (float)D.rho_in; D.rho_out_f = (float)D.rho_out;
    D.drho_in_f = (float)D.drho_in; D.drho_out_f = (float)D.drho_out; D.kT_f = (float)D.kT;
    D.n_pl_f = (float)D.n_pl; D.xi_pl_f = (float)D.xi_pl; D.tau_min_f = (float)D.tau_min;
    D.tau_max_f = (float)D.tau_max; D.tmin_pow_f = (float)D.tmin_pow; D.tmax_pow_f = (float)D.tmax_pow;
    D.scale_f = (float)D.scale; D.inv_scale_f = (float)D.inv_scale;
    D.hot_d.omega = 1.0 / p.tau;
    D.hot_d.om = 1.0 - 1.0 / p.tau;
    D.hot_d.tgx = p.tau * p.gx;
    D.hot_d.tgy = p.tau * p.gy;
    D.hot_d.rho0 = p.rho0;
    D.hot_d.scale = D.scale;
    D.hot_d.inv_scale = D.inv_scale;
    D.hot_d.pad = 0.0;
    D.hot_f.omega = (float)D.hot_d.omega;
    D.hot_f.om = (float)D.hot_d.om;
    D.hot_f.tgx = (float)D.hot_d.tgx;
    D.hot_f.tgy = (float)D.hot_d.tgy;
    D.hot_f.rho0 = (float)p.rho0;
    D.hot_f.scale = (float)D.scale;
    D.hot_f.inv_scale = (float)D.inv_scale;
    D.hot_f.pad = 0.0f;
}

// Per-node flag words and per-chunk bits (mailbox bounce-back).  Flag bit j
// (1..8) marks a fluid node whose neighbour x + e_j is solid or lies in a
// ghost row beyond a y wall (x wrapped when periodic; beyond an open end
// there is no neighbour); the node writes its f*_j into that neighbour's slot
// opp(j) after each collision.  On a solid node bit i marks its slot i as such
// a mailbox (the node x + e_i is fluid); its other slots are read by nobody.  Open columns carry the Zou-He bits, except on
// wall rows, whose end nodes carry NF_CORNER (their sources beyond the x
// range reflect from the node's own opposite slot); solid nodes NF_SOLID.  A
// chunk bit is set when any of its nodes has a nonzero flag word.
void build_flags(const DomDev& D, const uint8_t* solid, std::vector<uint16_t>& fl, std::vector<uint32_t>& words) {
    fl.assign((size_t)D.plane, 0);
    words.assign((size_t)D.ny * D.seg_per_row, 0u);
    const bool px = D.flags & FLAG_PX, wy = D.flags & FLAG_WY, io = D.flags & FLAG_IO;
    static const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    static const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (int y = 0; y < D.ny; ++y)
        for (int x = 0; x < D.nx; ++x) {
            uint16_t f = 0;
            const bool wall_row = wy && (y == 0 || y == D.ny - 1);
            if (solid[(size_t)y * D.nx + x]) {
                // bit i of a solid node: slot i is a mailbox, i.e. the node
                // x + e_i exists (wrapped when periodic) and is fluid, and writes it
                f = NF_SOLID;
                for (int i = 1; i < 9; ++i) {
                    int tx = x + ex[i], ty = y + ey[i];
                    if (ty < 0 || ty >= D.ny) {
                        if (wy) continue;
                        ty = (ty + D.ny) % D.ny;
                    }
                    if (tx < 0 || tx >= D.nx) {
                        if (!px) continue;
                        tx = (tx + D.nx) % D.nx;
                    }
                    if (!solid[(size_t)ty * D.nx + tx]) f |= (uint16_t)(1u << i);
                }
            } else {
                for (int j = 1; j < 9; ++j) {
                    int tx = x + ex[j], ty = y + ey[j];
                    bool ghost = false;
                    if (ty < 0 || ty >= D.ny) {
                        if (wy) ghost = true;
                        else ty = (ty + D.ny) % D.ny;
                    }
                    if (tx < 0 || tx >= D.nx) {
                        if (!px) continue;
                        tx = (tx + D.nx) % D.nx;
                    }
                    if (ghost || solid[(size_t)ty * D.nx + tx]) f |= (uint16_t)(1u << j);
                }
                if (io && (x == 0 || x == D.nx - 1)) {
                    if (wall_row) f |= NF_CORNER;
                    else f |= x == 0 ? NF_ZH_IN : NF_ZH_OUT;
                }
            }
            fl[(size_t)y * D.pitch + x] = f;
            if (f) {
                const int c = x / D.V;
                words[(size_t)y * D.seg_per_row + c / 32] |= 1u << (c % 32);
            }
        }
}

int upload_geometry(lbm_ctx* c, int dom);

// The NEAR pass always runs the register kernel, whose CTAs hold at most
// REG_K1_MAX_BLOCK threads.
int near_block(const lbm_ctx* c) { return std::min(c->block, REG_K1_MAX_BLOCK); }

void set_launch(lbm_ctx* c) {
    const int64_t wpb = c->block / 32;
    int64_t full = (c->total_items + wpb - 1) / wpb;
    if (full < 1) full = 1;
    if (c->grid_mode == 2) {
        // Staged kernel: as many warps as fit, trimmed so that the items
        // split into equal whole shares per warp (less tail imbalance).
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int bps = staged_blocks_per_sm(c->kind, c->noise, c->pl, c->block, c->stages);
        const int64_t max_warps = std::max<int64_t>(1, (int64_t)sms * std::max(bps, 1) * wpb);
        const int64_t share = (c->total_items + max_warps - 1) / max_warps;
        const int64_t warps = (c->total_items + share - 1) / std::max<int64_t>(share, 1);
        c->grid = std::max<int64_t>(1, (warps + wpb - 1) / wpb);
    } else if (c->grid_mode == 1 || c->grid_mode == 3 || c->grid_mode == 4) {
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t per_sm = std::max<int64_t>(1, 2048 / c->block);
        const int64_t resident =
            (int64_t)sms * std::max(1, reg_blocks_per_sm(c->kind, c->noise, c->pl, c->block));
        const int64_t want = c->grid_mode == 1 ? (int64_t)sms * per_sm
                             : c->grid_mode == 4 ? (int64_t)sms * std::max<int64_t>(1, per_sm / 2) : resident;
        c->grid = std::min<int64_t>(full, want);
    } else {
        c->grid = full;
    }
    {
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t nwpb = near_block(c) / 32;
        c->near_grid = std::min<int64_t>((c->total_items + nwpb - 1) / nwpb, 2 * (int64_t)sms);
    }
    c->graph_dirty = true;
}

PartArgs part_args(lbm_ctx* c, int cur) {
    PartArgs a;
    a.doms = c->dd;
    a.one_domain = c->ndom == 1;
    a.dom0 = c->hd[0];
    a.arena = c->f[cur];
    a.solid = c->solid;
    a.state = c->pstate;
    a.flipmom = c->flipmom;
    a.fliptag = c->fliptag;
    a.fliptag_stride = (int64_t)std::max<size_t>(1, c->node_bytes);
    a.ljf = c->ljf;
    a.st = c->pst;
    a.np = c->np_slots;
    a.links = c->links;
    a.nlinks = c->nlinks;
    a.flips = c->flips;
    a.nflips = c->nflips;
    a.links_total = c->links_total;
    a.flips_total = c->flips_total;
    a.diag = c->diag;
    a.err = c->err;
    a.ctr = c->ctr + cur;
    a.pstep = c->pstep + cur;
    a.mark = c->mark;
    a.near_list = c->near_list;
    a.near_cnt = c->near_cnt;
    a.total_items = c->total_items;
    a.ljwall = c->ljwall;
    a.lj_tab = c->lj_tab;
    a.lj_cnt = c->lj_cnt;
    a.rec = c->rec;
    a.rec_cap = c->rec_cap;
    return a;
}

// with_flips = false leaves out the moments of nodes changing side (a pass
// that only times the kernel does not need them).
cudaError_t enqueue_stream_collide(lbm_ctx* c, int cur, cudaStream_t s, int block, int64_t grid,
                                   int mode = STREAM_ALL, bool with_flips = true, bool pdl = false) {
    StreamArgs a;
    a.doms = c->dd;
    a.item_off = c->d_item_off;
    a.ndom = c->ndom;
    a.total_items = c->total_items;
    a.src = c->f[cur];
    a.dst = c->f[cur ^ 1];
    a.solid = c->solid;
    a.nflags = c->nflags;
    a.special = c->special;
    a.ctr_in = c->ctr + cur;
    a.ctr_out = c->ctr + (cur ^ 1);
    a.err = c->err;
    a.wait_ns = c->wait_ns;
    a.mode = mode;
    a.flips = with_flips && c->np_active > 0 && mode != STREAM_FAR;
    a.mark = c->mark;
    a.near_list = c->near_list;
    a.near_cnt = c->near_cnt;
    a.fliptag = c->fliptag;
    a.fliptag_stride = (int64_t)std::max<size_t>(1, c->node_bytes);
    a.flipmom = c->flipmom;
    a.dom0 = c->hd[0];
    return launch_stream_collide(c->kind, c->noise, c->pl, a, block, grid, c->grid_mode == 2 ? c->stages : 0, s, pdl);
}

// One timestep in sequence on one stream: with particles, the particle
// launch of forces, exchange and Newton-Euler; the rasterisation and marks
// for step t+1 and the Eq. MP2 sums for t+2 (they need the state of t+1
// only); then the stream-collide pass over every item.
cudaError_t enqueue_step(lbm_ctx* c, int cur, cudaStream_t s) {
    if (c->np_active == 0) return enqueue_stream_collide(c, cur, s, c->block, c->grid, STREAM_ALL);
    const PartArgs a = part_args(c, cur);
    cudaError_t e;
    if ((e = launch_particle_step(c->kind, a, PL_STEP_A, s)) != cudaSuccess) return e;
    if ((e = launch_particle_step(c->kind, a, PL_STEP_R, s)) != cudaSuccess) return e;
    if ((e = launch_particle_step(c->kind, a, PL_STEP_LJ, s)) != cudaSuccess) return e;
    return enqueue_stream_collide(c, cur, s, c->block, c->grid, STREAM_ALL);
}

// nsteps steps with particles, as four chains.  Main stream: the particle
// launch of forces, exchange and Newton-Euler, and the NEAR pass of every
// step.  Far stream: the FAR passes.  Raster stream: the rasterisation and
// near-item marks for the following step, which need only the state that the
// force launch wrote and so run beside the NEAR pass.  LJ stream: the Eq. MP2
// sums two steps ahead.  Edges:
//  - FAR(t) after NEAR(t-1): the near items of t-1 are the only ones it may
//    read that the far chain did not write itself;
//  - NEAR(t) after FAR(t-1) (it overwrites the arena FAR(t-1) read and reads
//    its output at the seams) and after launch 2 for t (the node tags of
//    side changes of t);
//  - the rasterisation for t+1 after the force launch of t (state of t+1; the
//    lists of t it replaces are read) and after FAR(t-1) (the marks it writes
//    are the three-way copy FAR(t-1) read);
//  - the Eq. MP2 sums for t+2 after the force launch of t (state of t+1; the
//    sums of t they replace are read), and the force launch of t+2 after them.
// The force launch of t+1 needs nothing from FAR(t): it reads and writes
// only slots of items near the particles, which NEAR(t) produced.  What the
// first steps of the graph need from launches of earlier steps ran before it
// (previous graph or set-up).  Each NEAR pass is a programmatic dependent of
// the force launch before it: the force launch signals once the particle
// states are solved, the NEAR CTAs are then placed while its exchange
// completes and wait for its completion (and for the edges from the other
// streams) before they touch memory, which takes the launch latency off the
// particle chain.  (The same for the FAR passes and the force launches
// measured no faster.)
cudaError_t enqueue_graph_chains(lbm_ctx* c, int k, int nsteps, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaEventRecord(c->ev_fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c->far_stream, c->ev_fork, 0)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c->rast_stream, c->ev_fork, 0)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c->lj_stream, c->ev_fork, 0)) != cudaSuccess) return e;
    for (int st = 0; st < nsteps; ++st) {
        const int cur = k ^ (st & 1);
        const PartArgs a = part_args(c, cur);
        if (st > 0 && (e = cudaStreamWaitEvent(c->far_stream, c->ev_near[(st - 1) & 1], 0)) != cudaSuccess) return e;
        if ((e = enqueue_stream_collide(c, cur, c->far_stream, c->block, c->grid, STREAM_FAR)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(c->ev_far[st & 1], c->far_stream)) != cudaSuccess) return e;
        if (st > 1 && (e = cudaStreamWaitEvent(s, c->ev_lj[st & 1], 0)) != cudaSuccess) return e;  // sums of st
        if ((e = launch_particle_step(c->kind, a, PL_STEP_A, s)) != cudaSuccess) return e;
        if (st == nsteps - 1 && (e = cudaEventRecordWithFlags(c->ev_pstate, s, cudaEventRecordExternal)) != cudaSuccess)
            return e;
        if ((e = cudaEventRecord(c->ev_a[st & 1], s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(c->lj_stream, c->ev_a[st & 1], 0)) != cudaSuccess) return e;
        if ((e = launch_particle_step(c->kind, a, PL_STEP_LJ, c->lj_stream)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(c->ev_lj[st & 1], c->lj_stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(c->rast_stream, c->ev_a[st & 1], 0)) != cudaSuccess) return e;
        if (st > 0 && (e = cudaStreamWaitEvent(c->rast_stream, c->ev_far[(st - 1) & 1], 0)) != cudaSuccess) return e;
        if ((e = launch_particle_step(c->kind, a, PL_STEP_R, c->rast_stream)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(c->ev_rast[st & 1], c->rast_stream)) != cudaSuccess) return e;
        if (st > 0 && (e = cudaStreamWaitEvent(s, c->ev_rast[(st - 1) & 1], 0)) != cudaSuccess) return e;
        if (st > 0 && (e = cudaStreamWaitEvent(s, c->ev_far[(st - 1) & 1], 0)) != cudaSuccess) return e;
        if ((e = enqueue_stream_collide(c, cur, s, near_block(c), c->near_grid, STREAM_NEAR, true, true)) != cudaSuccess)
            return e;
        if ((e = cudaEventRecord(c->ev_near[st & 1], s)) != cudaSuccess) return e;
    }
    if ((e = cudaEventRecord(c->ev_join, c->far_stream)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(c->ev_join2, c->rast_stream)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(c->ev_join3, c->lj_stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, c->ev_join, 0)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, c->ev_join2, 0)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(s, c->ev_join3, 0);
}

// Captures nsteps steps starting from state k into one executable graph.
int capture_steps(lbm_ctx* c, int k, int nsteps, cudaGraphExec_t* out) {
    if (*out) { cudaGraphExecDestroy(*out); *out = nullptr; }
    cudaGraph_t g = nullptr;
    CKC(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    if (c->np_active > 0 && c->overlap) e = enqueue_graph_chains(c, k, nsteps, c->cap_stream);
    else
        for (int s = 0; s < nsteps && e == cudaSuccess; ++s) e = enqueue_step(c, k ^ (s & 1), c->cap_stream);
    if (e == cudaSuccess && c->np_active > 0 && !c->overlap)
        e = cudaEventRecordWithFlags(c->ev_pstate, c->cap_stream, cudaEventRecordExternal);
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); CKC(c, e); }
    CKC(c, e2);
    e = cudaGraphInstantiate(out, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    CKC(c, e);
    // Upload the executable graph now: otherwise its first launch does it,
    // inside whatever the caller times (tens of microseconds per graph).
    CKC(c, cudaGraphUpload(*out, c->stream));
    return LBM_OK;
}

int build_graphs(lbm_ctx* c) {
    for (int k = 0; k < 2; ++k) {
        for (int j = 0; j <= GRAPH_LOG; ++j) {
            const int r = capture_steps(c, k, 1 << j, &c->gexec[k][j]);
            if (r) return r;
        }
        c->gprep[k].resize(c->prepared.size(), nullptr);
        for (size_t i = 0; i < c->prepared.size(); ++i) {
            const int r = capture_steps(c, k, (int)c->prepared[i], &c->gprep[k][i]);
            if (r) return r;
        }
    }
    c->graph_dirty = false;
    return LBM_OK;
}

// Pinned host block: the error word in the first PIN_HEAD bytes, then
// `extra` bytes of staging (the particle states).
constexpr size_t PIN_HEAD = 64;
int ensure_pin(lbm_ctx* c, size_t extra) {
    if (c->h_pin_bytes >= PIN_HEAD + extra) return LBM_OK;
    if (c->h_pin) cudaFreeHost(c->h_pin);
    c->h_pin = nullptr;
    c->h_pin_bytes = 0;
    void* p = nullptr;
    CKC(c, cudaMallocHost(&p, PIN_HEAD + extra));
    c->h_pin = static_cast<unsigned char*>(p);
    c->h_pin_bytes = PIN_HEAD + extra;
    return LBM_OK;
}

int err_status(lbm_ctx* c, unsigned h) {
    if (h & ERR_UNSTABLE) return fail(c, LBM_E_UNSTABLE, "non-finite or non-positive density on the lattice");
    if (h & ERR_TIMEOUT) return fail(c, LBM_E_TIMEOUT, "a bounded device wait ran out");
    if (h & ERR_STATE) return fail(c, LBM_E_STATE, "particle overlap or particle list capacity exceeded");
    return LBM_OK;
}

// Error word as of the work queued on stream s: one asynchronous copy into
// pinned memory and one synchronisation.
int check_err_on(lbm_ctx* c, cudaStream_t s) {
    int r = ensure_pin(c, 0);
    if (r) return r;
    CKC(c, cudaMemcpyAsync(c->h_pin, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CKC(c, cudaStreamSynchronize(s));
    return err_status(c, *reinterpret_cast<const volatile unsigned*>(c->h_pin));
}

int check_err(lbm_ctx* c) { return check_err_on(c, c->stream); }

int sync_and_check(lbm_ctx* c) { return check_err_on(c, c->stream); }

int ensure_stage(lbm_ctx* c, size_t bytes) {
    if (c->d_stage_bytes >= bytes) return LBM_OK;
    if (c->d_stage) cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->d_stage_bytes = 0;
    CKC(c, dev_malloc(&c->d_stage, bytes));
    c->d_stage_bytes = bytes;
    return LBM_OK;
}

// Solid bytes, flag words and chunk bits of one domain from its host mask.
int upload_geometry(lbm_ctx* c, int dom) {
    const DomDev& D = c->hd[dom];
    const std::vector<uint8_t>& hs = c->hsolid[dom];
    std::vector<uint8_t> pitched((size_t)D.plane, 0);
    for (int y = 0; y < D.ny; ++y) memcpy(&pitched[(size_t)y * D.pitch], &hs[(size_t)y * D.nx], D.nx);
    std::vector<uint16_t> fl;
    std::vector<uint32_t> words;
    build_flags(D, hs.data(), fl, words);
    CKC(c, cudaMemcpy(c->solid + D.node_off, pitched.data(), pitched.size(), cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(c->nflags + D.node_off, fl.data(), fl.size() * 2, cudaMemcpyHostToDevice));
    if (!words.empty())
        CKC(c, cudaMemcpy(c->special + D.mask_off, words.data(), words.size() * 4, cudaMemcpyHostToDevice));
    if (c->ljwall && c->prm[dom].lj_psi > 0.0) {
        CKC(c, launch_lj_wall(D, c->solid, c->lj_tab, c->lj_cnt, dom, c->ljwall, c->stream));
        CKC(c, cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

int check_dom(lbm_ctx* c, int dom) {
    if (!c) return LBM_E_INVAL;
    if (dom < 0 || dom >= c->ndom) return fail(c, LBM_E_INVAL, "domain index out of range");
    return LBM_OK;
}

void free_particles(lbm_ctx* c) {
    cudaFree(c->pstate); cudaFree(c->pst); cudaFree(c->flipmom);
    cudaFree(c->links); cudaFree(c->nlinks); cudaFree(c->flips); cudaFree(c->nflips); cudaFree(c->diag);
    cudaFree(c->ljf);
    c->pstate = nullptr; c->pst = nullptr; c->flipmom = nullptr;
    c->links = c->nlinks = c->flips = c->nflips = nullptr;
    c->diag = nullptr;
    c->ljf = nullptr;
}

}  // namespace

extern "C" {

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->msg.c_str() : g_create_error.c_str(); }

int lbm_create(const lbm_params* p, void* cuda_stream, lbm_ctx** out) {
    return lbm_create_ensemble(1, p, cuda_stream, out);
}

int lbm_create_ensemble(int ndom, const lbm_params* per_domain, void* cuda_stream, lbm_ctx** out) {
    if (!out || !per_domain || ndom < 1 || ndom > 65536) return fail(nullptr, LBM_E_INVAL, "bad arguments to lbm_create");
    *out = nullptr;
    for (int d = 0; d < ndom; ++d) {
        int r = validate(per_domain[d], d, nullptr);
        if (r) return r;
        if (per_domain[d].store != per_domain[0].store) return fail(nullptr, LBM_E_INVAL, "store kind differs between domains");
    }
    lbm_ctx* c = new lbm_ctx();
    c->ndom = ndom;
    c->kind = per_domain[0].store;
    c->esz = elem_bytes(c->kind);
    c->V = store_vector_width(c->kind);
    c->prm.assign(per_domain, per_domain + ndom);
    c->hd.resize(ndom);
    c->hsolid.resize(ndom);
    std::vector<int64_t> item_off(ndom);
    int64_t off = 0, node_off = 0, mask_off = 0, items = 0;
    int pslot = 0;
    for (int d = 0; d < ndom; ++d) {
        DomDev& D = c->hd[d];
        fill_dom(D, per_domain[d], c->kind);
        D.off = off + (per_domain[d].walls_y ? D.pitch : 0);  // row 0 of plane 0, after the ghost row
        D.node_off = node_off;
        D.mask_off = mask_off;
        D.item_off = items;
        D.p0 = pslot;
        D.np = 0;
        item_off[d] = items;
        off += 9 * D.plane;
        node_off += D.plane;
        mask_off += (int64_t)D.ny * D.seg_per_row;
        items += (int64_t)D.ny * D.seg_per_row;
        pslot += per_domain[d].max_particles;
        c->hsolid[d].assign((size_t)D.nx * D.ny, 0);
        c->noise |= per_domain[d].kT > 0.0;
        c->pl |= per_domain[d].power_law != 0;
    }
    c->arena_elems = (size_t)off;
    c->node_bytes = (size_t)node_off;
    c->special_words = (size_t)mask_off;
    c->total_items = items;
    c->np_slots = pslot;

    auto cleanup = [&](int r) { lbm_destroy(c); return r; };
    int r;
#define CKCR(call)                                                                                       \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            g_create_error = std::string(#call) + ": " + cudaGetErrorString(e_);                          \
            return cleanup(e_ == cudaErrorMemoryAllocation ? LBM_E_NOMEM : LBM_E_CUDA);                  \
        }                                                                                                \
    } while (0)
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        CKCR(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    {
        int lo = 0, hi = 0;
        CKCR(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        // Priorities of the overlapped step's chains: every particle launch
        // highest, the FAR pass lowest.  (The Eq. MP2 sums are needed only two
        // steps later, but below the FAR pass, or with the FAR pass in the
        // middle, they starve once the particles come near obstacles and the
        // sums do real work: 42.6 or 38.2 us per step over 20,000 steps of the
        // porous workload against 36.2 with this order, although they were
        // 1.5 us faster while the particles were still far from everything.)
        CKCR(cudaStreamCreateWithPriority(&c->cap_stream, cudaStreamNonBlocking, hi));
        CKCR(cudaStreamCreateWithPriority(&c->far_stream, cudaStreamNonBlocking, lo));
        CKCR(cudaStreamCreateWithPriority(&c->rast_stream, cudaStreamNonBlocking, hi));
        CKCR(cudaStreamCreateWithPriority(&c->lj_stream, cudaStreamNonBlocking, hi));
    }
    CKCR(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    CKCR(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CKCR(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    CKCR(cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming));
    CKCR(cudaEventCreateWithFlags(&c->ev_join3, cudaEventDisableTiming));
    for (int k = 0; k < 2; ++k) {
        CKCR(cudaEventCreateWithFlags(&c->ev_far[k], cudaEventDisableTiming));
        CKCR(cudaEventCreateWithFlags(&c->ev_near[k], cudaEventDisableTiming));
        CKCR(cudaEventCreateWithFlags(&c->ev_a[k], cudaEventDisableTiming));
        CKCR(cudaEventCreateWithFlags(&c->ev_rast[k], cudaEventDisableTiming));
        CKCR(cudaEventCreateWithFlags(&c->ev_lj[k], cudaEventDisableTiming));
    }
    CKCR(dev_malloc(&c->mark, sizeof(int32_t) * 3 * std::max<int64_t>(1, c->total_items)));
    CKCR(dev_malloc(&c->near_list, sizeof(int32_t) * 3 * std::max<int64_t>(1, c->total_items)));
    CKCR(dev_malloc(&c->near_cnt, sizeof(int32_t) * 3));
    CKCR(cudaMemsetAsync(c->mark, 0xff, sizeof(int32_t) * 3 * std::max<int64_t>(1, c->total_items), c->stream));
    CKCR(cudaMemsetAsync(c->near_cnt, 0, sizeof(int32_t) * 3, c->stream));
    CKCR(dev_malloc(&c->fliptag, sizeof(int64_t) * 2 * std::max<size_t>(1, c->node_bytes)));
    CKCR(cudaMemsetAsync(c->fliptag, 0xff, sizeof(int64_t) * 2 * std::max<size_t>(1, c->node_bytes), c->stream));
    {
        // Eq. MP2 pair force per node offset within r_it, one table per domain
        std::vector<LjEntry> tab((size_t)ndom * LJ_TAB);
        std::vector<int32_t> cnt(ndom, 0);
        for (int d = 0; d < ndom; ++d) {
            const lbm_params& P = per_domain[d];
            if (!(P.lj_psi > 0.0) || !(P.lj_rit > 0.0)) continue;
            const int reach = (int)std::floor(P.lj_rit);
            int m = 0;
            for (int oy = -reach; oy <= reach; ++oy)
                for (int ox = -reach; ox <= reach; ++ox) {
                    if (ox == 0 && oy == 0) continue;
                    const double dist = std::sqrt((double)(ox * ox + oy * oy));
                    if (!(dist <= P.lj_rit) || m >= LJ_TAB) continue;
                    const double mag = P.lj_psi * std::pow(dist / P.lj_rit, -13.0);
                    tab[(size_t)d * LJ_TAB + m] = LjEntry{ox, oy, -mag * ox / dist, -mag * oy / dist};
                    ++m;
                }
            cnt[d] = m;
        }
        CKCR(dev_malloc(&c->lj_tab, sizeof(LjEntry) * tab.size()));
        CKCR(dev_malloc(&c->lj_cnt, sizeof(int32_t) * ndom));
        CKCR(cudaMemcpyAsync(c->lj_tab, tab.data(), sizeof(LjEntry) * tab.size(), cudaMemcpyHostToDevice, c->stream));
        CKCR(cudaMemcpyAsync(c->lj_cnt, cnt.data(), sizeof(int32_t) * ndom, cudaMemcpyHostToDevice, c->stream));
        CKCR(cudaStreamSynchronize(c->stream));
    }
    CKCR(cudaEventCreateWithFlags(&c->ev_snap, cudaEventDisableTiming));
    CKCR(cudaEventCreateWithFlags(&c->ev_pstate, cudaEventDisableTiming));
    CKCR(cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming));
    CKCR(dev_malloc(&c->f[0], c->arena_elems * c->esz));
    CKCR(dev_malloc(&c->f[1], c->arena_elems * c->esz));
    CKCR(dev_malloc(&c->solid, c->node_bytes));
    CKCR(dev_malloc(&c->nflags, c->node_bytes * 2));
    CKCR(dev_malloc(&c->special, std::max<size_t>(1, c->special_words) * 4));
    {
        bool any_lj = false;
        for (int d = 0; d < ndom; ++d) any_lj |= per_domain[d].lj_psi > 0.0 && per_domain[d].lj_rit > 0.0;
        if (any_lj) {
            CKCR(dev_malloc(&c->ljwall, sizeof(double2) * std::max<size_t>(1, c->node_bytes)));
            CKCR(cudaMemsetAsync(c->ljwall, 0, sizeof(double2) * std::max<size_t>(1, c->node_bytes), c->stream));
        }
    }
    CKCR(dev_malloc(&c->dd, sizeof(DomDev) * ndom));
    CKCR(dev_malloc(&c->d_item_off, sizeof(int64_t) * ndom));
    CKCR(dev_malloc(&c->ctr, sizeof(int64_t) * 2));
    CKCR(dev_malloc(&c->pstep, sizeof(int64_t) * 2));
    CKCR(cudaMemsetAsync(c->pstep, 0, sizeof(int64_t) * 2, c->stream));
    CKCR(dev_malloc(&c->err, sizeof(unsigned)));
    CKCR(dev_malloc(&c->d_partial, sizeof(double) * 3 * CHECK_BLOCKS));
    CKCR(dev_malloc(&c->d_sums, sizeof(double) * 3));
    CKCR(cudaMemsetAsync(c->solid, 0, c->node_bytes, c->stream));
    CKCR(cudaMemsetAsync(c->special, 0, std::max<size_t>(1, c->special_words) * 4, c->stream));
    CKCR(cudaMemsetAsync(c->f[1], 0, c->arena_elems * c->esz, c->stream));
    CKCR(cudaMemsetAsync(c->ctr, 0, sizeof(int64_t) * 2, c->stream));
    CKCR(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
    CKCR(cudaMemcpyAsync(c->dd, c->hd.data(), sizeof(DomDev) * ndom, cudaMemcpyHostToDevice, c->stream));
    CKCR(cudaMemcpyAsync(c->d_item_off, item_off.data(), sizeof(int64_t) * ndom, cudaMemcpyHostToDevice, c->stream));
    CKCR(cudaStreamSynchronize(c->stream));
    for (int d = 0; d < ndom; ++d)
        if ((r = upload_geometry(c, d)) != LBM_OK) { g_create_error = c->msg; return cleanup(r); }
    // rest state in arena 0
    CKCR(launch_fill_rest(c->kind, c->dd, ndom, c->hd.data(), c->f[0], c->solid, c->stream));
    for (int d = 0; d < ndom; ++d) CKCR(launch_prime_mail(c->kind, c->hd[d], c->f[0], c->nflags, c->stream));
    if (c->np_slots > 0) {
        c->hst.assign(c->np_slots, PartStatic{});
        for (auto& s : c->hst) s.dom = -1;
        c->hstate.assign(c->np_slots, PartState{});
    }
    CKCR(cudaStreamSynchronize(c->stream));
#undef CKCR
    set_launch(c);
    r = LBM_OK;
    *out = c;
    return r;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& gk : c->gexec)
        for (auto& g : gk)
            if (g) cudaGraphExecDestroy(g);
    for (auto& gk : c->gprep)
        for (auto& g : gk)
            if (g) cudaGraphExecDestroy(g);
    cudaFree(c->f[0]); cudaFree(c->f[1]); cudaFree(c->solid); cudaFree(c->nflags); cudaFree(c->special);
    cudaFree(c->dd); cudaFree(c->d_item_off); cudaFree(c->ctr); cudaFree(c->pstep); cudaFree(c->err);
    cudaFree(c->d_partial); cudaFree(c->d_sums); cudaFree(c->d_stage); cudaFree(c->d_mom);
    if (c->h_mom) cudaFreeHost(c->h_mom);
    if (c->h_pin) cudaFreeHost(c->h_pin);
    free_particles(c);
    cudaFree(c->mark); cudaFree(c->near_list); cudaFree(c->near_cnt); cudaFree(c->lj_tab); cudaFree(c->lj_cnt);
    cudaFree(c->ljwall);
    cudaFree(c->fliptag);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_join2) cudaEventDestroy(c->ev_join2);
    if (c->ev_join3) cudaEventDestroy(c->ev_join3);
    for (int k = 0; k < 2; ++k) {
        if (c->ev_far[k]) cudaEventDestroy(c->ev_far[k]);
        if (c->ev_near[k]) cudaEventDestroy(c->ev_near[k]);
        if (c->ev_a[k]) cudaEventDestroy(c->ev_a[k]);
        if (c->ev_rast[k]) cudaEventDestroy(c->ev_rast[k]);
        if (c->ev_lj[k]) cudaEventDestroy(c->ev_lj[k]);
    }
    if (c->far_stream) cudaStreamDestroy(c->far_stream);
    if (c->rast_stream) cudaStreamDestroy(c->rast_stream);
    if (c->lj_stream) cudaStreamDestroy(c->lj_stream);
    if (c->ev_snap) cudaEventDestroy(c->ev_snap);
    if (c->ev_pstate) cudaEventDestroy(c->ev_pstate);
    if (c->ev_copied) cudaEventDestroy(c->ev_copied);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int lbm_set_geometry(lbm_ctx* c, int dom, const uint8_t* solid) {
    int r = check_dom(c, dom);
    if (r) return r;
    if (!solid) return fail(c, LBM_E_INVAL, "solid mask is NULL");
    if (c->np_active > 0) return fail(c, LBM_E_STATE, "set the geometry before adding particles");
    const DomDev& D = c->hd[dom];
    std::vector<uint8_t>& hs = c->hsolid[dom];
    for (size_t k = 0; k < hs.size(); ++k) hs[k] = solid[k] ? 1 : 0;
    CKC(c, cudaStreamSynchronize(c->stream));
    r = upload_geometry(c, dom);
    if (r) return r;
    // solid nodes hold no populations: re-apply the current state with zeros there
    r = ensure_stage(c, sizeof(double) * 9 * (size_t)D.nx * D.ny);
    if (r) return r;
    CKC(c, launch_export(c->kind, D, c->f[c->cur], c->solid, c->d_stage, c->stream));
    CKC(c, launch_import(c->kind, D, c->d_stage, c->f[c->cur], c->solid, c->stream));
    CKC(c, launch_prime_mail(c->kind, D, c->f[c->cur], c->nflags, c->stream));
    return sync_and_check(c);
}

int lbm_add_particles(lbm_ctx* c, int dom, int n, const lbm_particle* p) {
    int r = check_dom(c, dom);
    if (r) return r;
    c->pstate_evt = false;
    if (n < 0 || (n > 0 && !p)) return fail(c, LBM_E_INVAL, "bad particle array");
    if (n == 0) return LBM_OK;
    DomDev& D = c->hd[dom];
    const lbm_params& P = c->prm[dom];
    if (D.np + n > P.max_particles) return fail(c, LBM_E_INVAL, "more particles than max_particles");
    for (int i = 0; i < n; ++i) {
        const lbm_particle& q = p[i];
        if (!(q.R > 0.5) || !(q.rho_p > 0.0) || !std::isfinite(q.x) || !std::isfinite(q.y))
            return fail(c, LBM_E_INVAL, "particle needs R > 1/2, rho_p > 0 and a finite position");
        if (q.x < 0 || q.x >= D.nx || q.y < 0 || q.y >= D.ny) return fail(c, LBM_E_INVAL, "particle centre outside the domain");
        if ((D.flags & FLAG_PX) && 2 * q.R + 8 >= D.nx) return fail(c, LBM_E_INVAL, "particle too large for the periodic x extent");
        if ((D.flags & FLAG_PY) && 2 * q.R + 8 >= D.ny) return fail(c, LBM_E_INVAL, "particle too large for the periodic y extent");
    }
    CKC(c, cudaStreamSynchronize(c->stream));
    // refresh the host shadow of the existing particle states
    if (c->np_active > 0)
        CKC(c, cudaMemcpy(c->hstate.data(), c->pstate + (c->steps & 1) * c->np_slots, sizeof(PartState) * c->np_slots,
                          cudaMemcpyDeviceToHost));
    const double pi = 3.14159265358979323846264338327950288;
    for (int i = 0; i < n; ++i) {
        const lbm_particle& q = p[i];
        const int s = D.p0 + D.np + i;
        PartStatic& st = c->hst[s];
        st.R = q.R;
        st.rho_p = q.rho_p;
        st.m = q.rho_p * pi * q.R * q.R;
        st.I = 0.5 * st.m * q.R * q.R;
        st.inv_m = 1.0 / st.m;
        st.inv_I = 1.0 / st.I;
        st.buoy = (q.rho_p - P.rho0) / q.rho_p;
        st.dom = dom;
        st.fixed = q.fixed ? 1 : 0;
        const int r_up = (int)std::ceil(q.R);
        st.link_cap = 32 * (2 * r_up + 3);
        st.flip_cap = (2 * r_up + 6) * (2 * r_up + 6);
        c->hstate[s] = PartState{q.x, q.y, q.U, q.V, q.Omega, q.theta};
    }
    D.np += n;
    c->np_active += n;
    // lay out the per-particle lists and (re)allocate them
    int64_t lo = 0, fo = 0;
    for (int s = 0; s < c->np_slots; ++s) {
        PartStatic& st = c->hst[s];
        if (st.dom < 0) continue;
        st.link_off = lo;
        st.flip_off = fo;
        lo += st.link_cap;
        fo += st.flip_cap;
    }
    free_particles(c);
    const size_t ns = c->np_slots;
    CKC(c, dev_malloc(&c->pstate, sizeof(PartState) * 2 * ns));
    CKC(c, dev_malloc(&c->flipmom, sizeof(double) * 2 * 3 * std::max<int64_t>(fo, 1)));
    CKC(c, dev_malloc(&c->pst, sizeof(PartStatic) * ns));
    CKC(c, dev_malloc(&c->links, sizeof(int32_t) * 2 * std::max<int64_t>(lo, 1)));
    CKC(c, dev_malloc(&c->flips, sizeof(int32_t) * 2 * std::max<int64_t>(fo, 1)));
    CKC(c, dev_malloc(&c->nlinks, sizeof(int32_t) * 2 * ns));
    CKC(c, dev_malloc(&c->nflips, sizeof(int32_t) * 2 * ns));
    CKC(c, dev_malloc(&c->diag, sizeof(double) * DIAG_N * ns));
    CKC(c, dev_malloc(&c->ljf, sizeof(double) * 2 * 4 * ns));
    CKC(c, cudaMemset(c->ljf, 0, sizeof(double) * 2 * 4 * ns));
    CKC(c, cudaMemset(c->nlinks, 0, sizeof(int32_t) * 2 * ns));
    CKC(c, cudaMemset(c->nflips, 0, sizeof(int32_t) * 2 * ns));
    CKC(c, cudaMemset(c->diag, 0, sizeof(double) * DIAG_N * ns));
    CKC(c, cudaMemcpy(c->pstate, c->hstate.data(), sizeof(PartState) * ns, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(c->pstate + ns, c->hstate.data(), sizeof(PartState) * ns, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(c->pst, c->hst.data(), sizeof(PartStatic) * ns, cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(c->dd + dom, &D, sizeof(DomDev), cudaMemcpyHostToDevice));
    c->links_total = lo;
    c->flips_total = fo;
    // rasterise every particle at its current position (no link exchange, no
    // flips) and mark the work items near the particles for this step, then
    // what every step expects to find: the rasterisation of the next step
    // with its side changes and marks, and the Eq. MP2 sums of this step
    CKC(c, cudaMemsetAsync(c->mark, 0xff, sizeof(int32_t) * 3 * std::max<int64_t>(1, c->total_items), c->stream));
    CKC(c, cudaMemsetAsync(c->near_cnt, 0, sizeof(int32_t) * 3, c->stream));
    CKC(c, launch_particle_step(c->kind, part_args(c, c->cur), PL_RASTER | PL_MARK, c->stream));
    CKC(c, launch_particle_step(c->kind, part_args(c, c->cur), PL_SETUP_R, c->stream));
    CKC(c, launch_particle_step(c->kind, part_args(c, c->cur), PL_LJ, c->stream));
    CKC(c, launch_particle_step(c->kind, part_args(c, c->cur), PL_LJ | PL_ADVANCE, c->stream));
    c->graph_dirty = true;
    return sync_and_check(c);
}

// Wait for the work queued so far and clear the sticky device error word:
// the caller is about to replace the state those steps produced.
int clear_errors(lbm_ctx* c) {
    CKC(c, cudaStreamSynchronize(c->stream));
    CKC(c, cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
    return LBM_OK;
}

int lbm_set_populations(lbm_ctx* c, int dom, const double* f) {
    int r = check_dom(c, dom);
    if (r) return r;
    if (!f) return fail(c, LBM_E_INVAL, "population array is NULL");
    r = clear_errors(c);
    if (r) return r;
    const DomDev& D = c->hd[dom];
    const size_t bytes = sizeof(double) * 9 * (size_t)D.nx * D.ny;
    r = ensure_stage(c, bytes);
    if (r) return r;
    CKC(c, cudaMemcpyAsync(c->d_stage, f, bytes, cudaMemcpyHostToDevice, c->stream));
    CKC(c, launch_import(c->kind, D, c->d_stage, c->f[c->cur], c->solid, c->stream));
    CKC(c, launch_prime_mail(c->kind, D, c->f[c->cur], c->nflags, c->stream));
    return sync_and_check(c);
}

int lbm_get_populations(lbm_ctx* c, int dom, double* f) {
    int r = check_dom(c, dom);
    if (r) return r;
    if (!f) return fail(c, LBM_E_INVAL, "population array is NULL");
    const DomDev& D = c->hd[dom];
    const size_t bytes = sizeof(double) * 9 * (size_t)D.nx * D.ny;
    r = ensure_stage(c, bytes);
    if (r) return r;
    CKC(c, launch_export(c->kind, D, c->f[c->cur], c->solid, c->d_stage, c->stream));
    CKC(c, cudaMemcpyAsync(f, c->d_stage, bytes, cudaMemcpyDeviceToHost, c->stream));
    return sync_and_check(c);
}

int lbm_step(lbm_ctx* c, int64_t nsteps) {
    if (!c) return LBM_E_INVAL;
    if (nsteps < 0) return fail(c, LBM_E_INVAL, "nsteps must be >= 0");
    if (nsteps == 0) return LBM_OK;
    if (c->graph_dirty) {
        int r = build_graphs(c);
        if (r) return r;
    }
    for (size_t i = 0; i < c->prepared.size(); ++i) {
        if (c->prepared[i] != nsteps || i >= c->gprep[c->cur].size() || !c->gprep[c->cur][i]) continue;
        CKC(c, cudaGraphLaunch(c->gprep[c->cur][i], c->stream));
        c->cur ^= (int)(nsteps & 1);
        c->steps += nsteps;
        c->pstate_evt = c->np_active > 0;
        return LBM_OK;
    }
    for (int64_t n = nsteps >> GRAPH_LOG; n > 0; --n)  // even step counts: the state stays in arena cur
        CKC(c, cudaGraphLaunch(c->gexec[c->cur][GRAPH_LOG], c->stream));
    for (int j = GRAPH_LOG - 1; j >= 0; --j) {
        if (!((nsteps >> j) & 1)) continue;
        CKC(c, cudaGraphLaunch(c->gexec[c->cur][j], c->stream));
        if (j == 0) c->cur ^= 1;
    }
    c->steps += nsteps;
    c->pstate_evt = c->np_active > 0;
    return LBM_OK;
}

int lbm_record_particles(lbm_ctx* c, double* host_buf, int64_t capacity) {
    if (!c) return LBM_E_INVAL;
    PartState* dev = nullptr;
    if (host_buf) {
        if (capacity < 1) return fail(c, LBM_E_INVAL, "capacity must be >= 1 step");
        if (reinterpret_cast<uintptr_t>(host_buf) % alignof(double))
            return fail(c, LBM_E_INVAL, "record buffer must be aligned to 8 bytes");
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, host_buf) != cudaSuccess || at.type != cudaMemoryTypeHost ||
            !at.devicePointer) {
            cudaGetLastError();  // a pageable pointer leaves an error behind on some drivers
            return fail(c, LBM_E_INVAL, "record buffer must be page-locked host memory mapped into the device space");
        }
        dev = static_cast<PartState*>(at.devicePointer);
    }
    // every step of a graph launch writes through the pointer captured with it
    int r = sync_and_check(c);
    if (r) return r;
    c->rec = dev;
    c->rec_cap = dev ? capacity : 0;
    c->graph_dirty = true;
    return LBM_OK;
}

int lbm_prepare_steps(lbm_ctx* c, int64_t nsteps) {
    if (!c) return LBM_E_INVAL;
    if (nsteps < 1 || nsteps > LBM_PREPARE_MAX_STEPS)
        return fail(c, LBM_E_INVAL, "nsteps must be in 1 .. LBM_PREPARE_MAX_STEPS");
    int r = LBM_OK;
    for (int64_t n : c->prepared)
        if (n == nsteps) return c->graph_dirty && (r = build_graphs(c)) ? r : sync_and_check(c);
    if ((int)c->prepared.size() >= LBM_PREPARE_SLOTS) {  // drop the oldest
        for (auto& gk : c->gprep) {
            if (!gk.empty() && gk[0]) cudaGraphExecDestroy(gk[0]);
            if (!gk.empty()) gk.erase(gk.begin());
        }
        c->prepared.erase(c->prepared.begin());
    }
    c->prepared.push_back(nsteps);
    if (c->graph_dirty) {
        r = build_graphs(c);
    } else {
        for (int k = 0; k < 2 && !r; ++k) {
            c->gprep[k].resize(c->prepared.size(), nullptr);
            r = capture_steps(c, k, (int)nsteps, &c->gprep[k].back());
        }
    }
    return r ? r : sync_and_check(c);
}

int lbm_sync(lbm_ctx* c) {
    if (!c) return LBM_E_INVAL;
    return sync_and_check(c);
}

int64_t lbm_step_count(const lbm_ctx* c) { return c ? c->steps : -1; }

int lbm_moments(lbm_ctx* c, int dom, double* rho, double* ux, double* uy) {
    int r = check_dom(c, dom);
    if (r) return r;
    if (!rho || !ux || !uy) return fail(c, LBM_E_INVAL, "moment arrays must not be NULL");
    const DomDev& D = c->hd[dom];
    const size_t n = (size_t)D.nx * D.ny;
    r = ensure_stage(c, sizeof(double) * 3 * n);
    if (r) return r;
    CKC(c, launch_moments(c->kind, D, c->f[c->cur], c->solid, c->d_stage, c->d_stage + n, c->d_stage + 2 * n, false,
                          c->stream));
    CKC(c, cudaMemcpyAsync(rho, c->d_stage, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    CKC(c, cudaMemcpyAsync(ux, c->d_stage + n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    CKC(c, cudaMemcpyAsync(uy, c->d_stage + 2 * n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    return sync_and_check(c);
}

int lbm_moments_device(lbm_ctx* c, int dom, float* d_rho, float* d_ux, float* d_uy) {
    int r = check_dom(c, dom);
    if (r) return r;
    if (!d_rho || !d_ux || !d_uy) return fail(c, LBM_E_INVAL, "moment arrays must not be NULL");
    CKC(c, launch_moments(c->kind, c->hd[dom], c->f[c->cur], c->solid, d_rho, d_ux, d_uy, true, c->stream));
    return LBM_OK;
}

int lbm_moments_async(lbm_ctx* c, int dom) {
    int r = check_dom(c, dom);
    if (r) return r;
    const DomDev& D = c->hd[dom];
    const size_t n = (size_t)D.nx * D.ny;
    if (c->mom_pending) CKC(c, cudaEventSynchronize(c->ev_copied));
    if (c->mom_elems < 3 * n) {
        cudaFree(c->d_mom);
        if (c->h_mom) cudaFreeHost(c->h_mom);
        c->d_mom = nullptr;
        c->h_mom = nullptr;
        c->mom_elems = 0;
        CKC(c, dev_malloc(&c->d_mom, sizeof(float) * 3 * n));
        CKC(c, cudaMallocHost(&c->h_mom, sizeof(float) * 3 * n));
        c->mom_elems = 3 * n;
    }
    // snapshot on the main stream (a read of the state), copy on the side stream
    CKC(c, launch_moments(c->kind, D, c->f[c->cur], c->solid, c->d_mom, c->d_mom + n, c->d_mom + 2 * n, true,
                          c->stream));
    CKC(c, cudaEventRecord(c->ev_snap, c->stream));
    CKC(c, cudaStreamWaitEvent(c->side, c->ev_snap, 0));
    CKC(c, cudaMemcpyAsync(c->h_mom, c->d_mom, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, c->side));
    CKC(c, cudaEventRecord(c->ev_copied, c->side));
    c->mom_pending = (int)n;
    return LBM_OK;
}

int lbm_moments_async_wait(lbm_ctx* c, float* rho, float* ux, float* uy) {
    if (!c) return LBM_E_INVAL;
    if (!c->mom_pending) return fail(c, LBM_E_STATE, "no asynchronous moment copy in flight");
    CKC(c, cudaEventSynchronize(c->ev_copied));
    const size_t n = (size_t)c->mom_pending;
    if (rho) memcpy(rho, c->h_mom, sizeof(float) * n);
    if (ux) memcpy(ux, c->h_mom + n, sizeof(float) * n);
    if (uy) memcpy(uy, c->h_mom + 2 * n, sizeof(float) * n);
    c->mom_pending = 0;
    return check_err_on(c, c->side);
}

int lbm_particles(lbm_ctx* c, int dom, lbm_particle* out, int cap) {
    int r = check_dom(c, dom);
    if (r) return r;
    const DomDev& D = c->hd[dom];
    if (D.np == 0) return 0;
    r = ensure_pin(c, sizeof(PartState) * (size_t)D.np);
    if (r) return r;
    const PartState* s = reinterpret_cast<const PartState*>(c->h_pin + PIN_HEAD);
    const PartState* src = c->pstate + (c->steps & 1) * c->np_slots + D.p0;
    if (c->pstate_evt) {
        // after steps: wait only for the force launch that wrote this state
        CKC(c, cudaStreamWaitEvent(c->side, c->ev_pstate, 0));
        CKC(c, cudaMemcpyAsync(c->h_pin + PIN_HEAD, src, sizeof(PartState) * D.np, cudaMemcpyDeviceToHost, c->side));
        CKC(c, cudaStreamSynchronize(c->side));
    } else {
        CKC(c, cudaMemcpyAsync(c->h_pin + PIN_HEAD, src, sizeof(PartState) * D.np, cudaMemcpyDeviceToHost, c->stream));
        r = sync_and_check(c);
        if (r) return r;
    }
    for (int i = 0; i < D.np && i < cap && out; ++i) {
        const PartStatic& st = c->hst[D.p0 + i];
        out[i] = lbm_particle{s[i].x, s[i].y, st.R, st.rho_p, s[i].U, s[i].V, s[i].Om, s[i].th, st.fixed, 0};
    }
    return D.np;
}

int lbm_particle_forces(lbm_ctx* c, int dom, int i, double* out13) {
    int r = check_dom(c, dom);
    if (r) return r;
    const DomDev& D = c->hd[dom];
    if (i < 0 || i >= D.np || !out13) return fail(c, LBM_E_INVAL, "particle index out of range");
    CKC(c, cudaMemcpyAsync(out13, c->diag + (int64_t)(D.p0 + i) * DIAG_N, sizeof(double) * DIAG_N,
                           cudaMemcpyDeviceToHost, c->stream));
    return sync_and_check(c);
}

int lbm_checks(lbm_ctx* c, int dom, double* out3) {
    int r = check_dom(c, dom);
    if (r) return r;
    if (!out3) return fail(c, LBM_E_INVAL, "output is NULL");
    CKC(c, launch_checks(c->kind, c->hd[dom], c->f[c->cur], c->solid, c->d_partial, CHECK_BLOCKS, c->d_sums, c->stream));
    CKC(c, cudaMemcpyAsync(out3, c->d_sums, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream));
    return sync_and_check(c);
}

// ---- checkpoint ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];
    int32_t version, kind, ndom, np_slots;
    int64_t steps, arena_elems, links_total, flips_total;
};
}  // namespace

int lbm_save(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_E_INVAL;
    int r = sync_and_check(c);
    if (r) return r;
    FILE* fp = fopen(path, "wb");
    if (!fp) return fail(c, LBM_E_IO, std::string("cannot open ") + path);
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "LBMGB300", 8);
    h.version = 2;  // 2: planes carry ghost rows with y walls
    h.kind = c->kind;
    h.ndom = c->ndom;
    h.np_slots = c->np_slots;
    h.steps = c->steps;
    h.arena_elems = (int64_t)c->arena_elems;
    h.links_total = c->links_total;
    h.flips_total = c->flips_total;
    bool ok = fwrite(&h, sizeof h, 1, fp) == 1;
    ok = ok && fwrite(c->prm.data(), sizeof(lbm_params), c->ndom, fp) == (size_t)c->ndom;
    for (int d = 0; d < c->ndom && ok; ++d) ok = fwrite(&c->hd[d].np, sizeof(int32_t), 1, fp) == 1;
    std::vector<char> buf(c->arena_elems * c->esz);
    int64_t ctr = 0;
    if (ok && cudaMemcpy(buf.data(), c->f[c->cur], buf.size(), cudaMemcpyDeviceToHost) != cudaSuccess) ok = false;
    if (ok && cudaMemcpy(&ctr, c->ctr + c->cur, sizeof ctr, cudaMemcpyDeviceToHost) != cudaSuccess) ok = false;
    ok = ok && fwrite(&ctr, sizeof ctr, 1, fp) == 1 && fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
    for (int d = 0; d < c->ndom && ok; ++d)
        ok = fwrite(c->hsolid[d].data(), 1, c->hsolid[d].size(), fp) == c->hsolid[d].size();
    if (ok && c->np_slots > 0 && c->np_active > 0) {
        const size_t ns = c->np_slots;
        std::vector<PartState> s(ns);
        std::vector<int32_t> nl(ns), nf(ns), L(std::max<int64_t>(c->links_total, 1)), F(std::max<int64_t>(c->flips_total, 1));
        std::vector<double> dg(ns * DIAG_N);
        std::vector<double> fm(3 * std::max<int64_t>(c->flips_total, 1));
        const int64_t pr = c->steps & 1;  // the lists of the current step
        ok = cudaMemcpy(s.data(), c->pstate + pr * ns, sizeof(PartState) * ns, cudaMemcpyDeviceToHost) == cudaSuccess &&
             cudaMemcpy(fm.data(), c->flipmom + pr * 3 * c->flips_total, 8 * fm.size(), cudaMemcpyDeviceToHost) == cudaSuccess &&
             cudaMemcpy(nl.data(), c->nlinks + pr * ns, 4 * ns, cudaMemcpyDeviceToHost) == cudaSuccess &&
             cudaMemcpy(nf.data(), c->nflips + pr * ns, 4 * ns, cudaMemcpyDeviceToHost) == cudaSuccess &&
             cudaMemcpy(L.data(), c->links + pr * c->links_total, 4 * L.size(), cudaMemcpyDeviceToHost) == cudaSuccess &&
             cudaMemcpy(F.data(), c->flips + pr * c->flips_total, 4 * F.size(), cudaMemcpyDeviceToHost) == cudaSuccess &&
             cudaMemcpy(dg.data(), c->diag, 8 * dg.size(), cudaMemcpyDeviceToHost) == cudaSuccess;
        ok = ok && fwrite(c->hst.data(), sizeof(PartStatic), ns, fp) == ns && fwrite(s.data(), sizeof(PartState), ns, fp) == ns &&
             fwrite(nl.data(), 4, ns, fp) == ns && fwrite(nf.data(), 4, ns, fp) == ns &&
             fwrite(L.data(), 4, L.size(), fp) == L.size() && fwrite(F.data(), 4, F.size(), fp) == F.size() &&
             fwrite(dg.data(), 8, dg.size(), fp) == dg.size() && fwrite(fm.data(), 8, fm.size(), fp) == fm.size();
    }
    ok = (fclose(fp) == 0) && ok;
    return ok ? LBM_OK : fail(c, LBM_E_IO, std::string("write failed: ") + path);
}

int lbm_load(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_E_INVAL;
    c->pstate_evt = false;
    int r = clear_errors(c);
    if (r) return r;
    FILE* fp = fopen(path, "rb");
    if (!fp) return fail(c, LBM_E_IO, std::string("cannot open ") + path);
    auto bail = [&](const char* m) { fclose(fp); return fail(c, LBM_E_IO, m); };
    CkptHeader h;
    if (fread(&h, sizeof h, 1, fp) != 1 || memcmp(h.magic, "LBMGB300", 8) != 0 || h.version != 2) return bail("not a checkpoint");
    if (h.kind != c->kind || h.ndom != c->ndom || h.np_slots != c->np_slots || h.arena_elems != (int64_t)c->arena_elems)
        return bail("checkpoint does not match this context");
    std::vector<lbm_params> prm(c->ndom);
    if (fread(prm.data(), sizeof(lbm_params), c->ndom, fp) != (size_t)c->ndom) return bail("truncated checkpoint");
    for (int d = 0; d < c->ndom; ++d)
        if (prm[d].nx != c->prm[d].nx || prm[d].ny != c->prm[d].ny) return bail("checkpoint domain sizes differ");
    std::vector<int32_t> dnp(c->ndom);
    for (int d = 0; d < c->ndom; ++d)
        if (fread(&dnp[d], sizeof(int32_t), 1, fp) != 1) return bail("truncated checkpoint");
    int64_t ctr = 0;
    std::vector<char> buf(c->arena_elems * c->esz);
    if (fread(&ctr, sizeof ctr, 1, fp) != 1 || fread(buf.data(), 1, buf.size(), fp) != buf.size()) return bail("truncated checkpoint");
    std::vector<std::vector<uint8_t>> sol(c->ndom);
    for (int d = 0; d < c->ndom; ++d) {
        sol[d].resize(c->hsolid[d].size());
        if (fread(sol[d].data(), 1, sol[d].size(), fp) != sol[d].size()) return bail("truncated checkpoint");
    }
    const int np_total = [&] { int s = 0; for (int v : dnp) s += v; return s; }();
    std::vector<PartStatic> hst;
    std::vector<PartState> s;
    std::vector<int32_t> nl, nf, L, F;
    std::vector<double> dg, fm;
    if (np_total > 0) {
        const size_t ns = c->np_slots;
        hst.resize(ns); s.resize(ns); nl.resize(ns); nf.resize(ns);
        L.resize(std::max<int64_t>(h.links_total, 1));
        F.resize(std::max<int64_t>(h.flips_total, 1));
        dg.resize(ns * DIAG_N);
        fm.resize(3 * std::max<int64_t>(h.flips_total, 1));
        bool ok = fread(hst.data(), sizeof(PartStatic), ns, fp) == ns && fread(s.data(), sizeof(PartState), ns, fp) == ns &&
                  fread(nl.data(), 4, ns, fp) == ns && fread(nf.data(), 4, ns, fp) == ns &&
                  fread(L.data(), 4, L.size(), fp) == L.size() && fread(F.data(), 4, F.size(), fp) == F.size() &&
                  fread(dg.data(), 8, dg.size(), fp) == dg.size() && fread(fm.data(), 8, fm.size(), fp) == fm.size();
        if (!ok) return bail("truncated checkpoint");
    }
    fclose(fp);
    // geometry first (it rewrites solid nodes of the current arena), then the state
    for (int d = 0; d < c->ndom; ++d) {
        c->hd[d].np = 0;
        c->np_active = 0;
        r = lbm_set_geometry(c, d, sol[d].data());
        if (r) return r;
    }
    CKC(c, cudaMemcpy(c->f[c->cur], buf.data(), buf.size(), cudaMemcpyHostToDevice));
    CKC(c, cudaMemcpy(c->ctr + c->cur, &ctr, sizeof ctr, cudaMemcpyHostToDevice));
    if (np_total > 0) {
        const size_t ns = c->np_slots;
        free_particles(c);
        c->hst = hst;
        c->hstate = s;
        CKC(c, dev_malloc(&c->pstate, sizeof(PartState) * 2 * ns));
        CKC(c, dev_malloc(&c->flipmom, 2 * 8 * fm.size()));
        CKC(c, dev_malloc(&c->pst, sizeof(PartStatic) * ns));
        CKC(c, dev_malloc(&c->links, 2 * 4 * L.size()));
        CKC(c, dev_malloc(&c->flips, 2 * 4 * F.size()));
        CKC(c, dev_malloc(&c->nlinks, 2 * 4 * ns));
        CKC(c, dev_malloc(&c->nflips, 2 * 4 * ns));
        const int64_t pr = h.steps & 1;  // the lists of the restored step
        CKC(c, dev_malloc(&c->diag, 8 * ns * DIAG_N));
        CKC(c, dev_malloc(&c->ljf, sizeof(double) * 2 * 4 * ns));
        CKC(c, cudaMemset(c->ljf, 0, sizeof(double) * 2 * 4 * ns));
        CKC(c, cudaMemcpy(c->pstate, s.data(), sizeof(PartState) * ns, cudaMemcpyHostToDevice));
        CKC(c, cudaMemcpy(c->pstate + ns, s.data(), sizeof(PartState) * ns, cudaMemcpyHostToDevice));
        CKC(c, cudaMemcpy(c->flipmom + pr * fm.size(), fm.data(), 8 * fm.size(), cudaMemcpyHostToDevice));
        CKC(c, cudaMemcpy(c->pst, hst.data(), sizeof(PartStatic) * ns, cudaMemcpyHostToDevice));
        CKC(c, cudaMemcpy(c->nlinks + pr * ns, nl.data(), 4 * ns, cudaMemcpyHostToDevice));
        CKC(c, cudaMemcpy(c->nflips + pr * ns, nf.data(), 4 * ns, cudaMemcpyHostToDevice));
        CKC(c, cudaMemcpy(c->links + pr * L.size(), L.data(), 4 * L.size(), cudaMemcpyHostToDevice));
        CKC(c, cudaMemcpy(c->flips + pr * F.size(), F.data(), 4 * F.size(), cudaMemcpyHostToDevice));
        CKC(c, cudaMemcpy(c->diag, dg.data(), 8 * dg.size(), cudaMemcpyHostToDevice));
        c->links_total = h.links_total;
        c->flips_total = h.flips_total;
        for (int d = 0; d < c->ndom; ++d) c->hd[d].np = dnp[d];
        c->np_active = np_total;
        CKC(c, cudaMemcpy(c->dd, c->hd.data(), sizeof(DomDev) * c->ndom, cudaMemcpyHostToDevice));
        CKC(c, cudaMemset(c->mark, 0xff, sizeof(int32_t) * 3 * std::max<int64_t>(1, c->total_items)));
        CKC(c, cudaMemset(c->near_cnt, 0, sizeof(int32_t) * 3));
        CKC(c, launch_particle_step(c->kind, part_args(c, c->cur), PL_MARK, c->stream));
        CKC(c, launch_particle_step(c->kind, part_args(c, c->cur), PL_SETUP_R, c->stream));
        CKC(c, launch_particle_step(c->kind, part_args(c, c->cur), PL_LJ, c->stream));
        CKC(c, launch_particle_step(c->kind, part_args(c, c->cur), PL_LJ | PL_ADVANCE, c->stream));
        CKC(c, cudaStreamSynchronize(c->stream));
    }
    CKC(c, cudaMemcpy(c->dd, c->hd.data(), sizeof(DomDev) * c->ndom, cudaMemcpyHostToDevice));
    c->steps = h.steps;
    c->graph_dirty = true;
    return LBM_OK;
}

int lbm_profile_steps(lbm_ctx* c, int64_t nsteps, double* ms_out3, int64_t* launches_out) {
    if (!c || !ms_out3 || nsteps < 0) return c ? fail(c, LBM_E_INVAL, "bad arguments") : LBM_E_INVAL;
    c->pstate_evt = false;
    int r = sync_and_check(c);
    if (r) return r;
    // Steps are enqueued back to back in batches, an event pair around every
    // kernel and one synchronisation per batch, so that each pair brackets
    // one kernel of a busy stream and no host launch latency.
    const int BATCH = 32, NE = 6 * BATCH;
    std::vector<cudaEvent_t> ev(NE, nullptr);
    for (auto& e : ev) {
        cudaError_t ce = cudaEventCreate(&e);
        if (ce != cudaSuccess) {
            for (auto& x : ev)
                if (x) cudaEventDestroy(x);
            CKC(c, ce);
        }
    }
    auto destroy = [&]() {
        for (auto& x : ev) cudaEventDestroy(x);
    };
    double acc[3] = {0.0, 0.0, 0.0};
    int64_t launches = 0;
    const bool parts = c->np_active > 0;
    for (int64_t s0 = 0; s0 < nsteps; s0 += BATCH) {
        const int nb = (int)std::min<int64_t>(BATCH, nsteps - s0);
        cudaError_t ce = cudaSuccess;
        for (int b = 0; b < nb && ce == cudaSuccess; ++b) {
            cudaEvent_t* e = ev.data() + 6 * b;
            if (parts) {
                const PartArgs a = part_args(c, c->cur);
                if (ce == cudaSuccess) ce = cudaEventRecord(e[0], c->stream);
                if (ce == cudaSuccess) ce = launch_particle_step(c->kind, a, PL_STEP_A, c->stream);
                if (ce == cudaSuccess) ce = cudaEventRecord(e[1], c->stream);
                if (ce == cudaSuccess) ce = launch_particle_step(c->kind, a, PL_STEP_R, c->stream);
                if (ce == cudaSuccess) ce = launch_particle_step(c->kind, a, PL_STEP_LJ, c->stream);
                if (ce == cudaSuccess) ce = cudaEventRecord(e[4], c->stream);
                launches += 3;
            }
            if (ce == cudaSuccess) ce = cudaEventRecord(e[2], c->stream);
            if (ce == cudaSuccess) ce = enqueue_stream_collide(c, c->cur, c->stream, c->block, c->grid);
            if (ce == cudaSuccess) ce = cudaEventRecord(e[3], c->stream);
            launches += 1;
            c->cur ^= 1;
            c->steps += 1;
        }
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
        for (int b = 0; b < nb && ce == cudaSuccess; ++b) {
            cudaEvent_t* e = ev.data() + 6 * b;
            float ms = 0.f;
            if (parts) {
                ce = cudaEventElapsedTime(&ms, e[0], e[1]);
                acc[0] += ms;
                if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e[1], e[4]);
                acc[1] += ms;
            }
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e[2], e[3]);
            acc[2] += ms;
        }
        if (ce != cudaSuccess) {
            destroy();
            CKC(c, ce);
        }
    }
    destroy();
    for (int k = 0; k < 3; ++k) ms_out3[k] = acc[k];
    if (launches_out) *launches_out = launches;
    return check_err(c);
}

int lbm_fp64_fma_rate(void* cuda_stream, double* gflops_out) {
    if (!gflops_out) return fail(nullptr, LBM_E_INVAL, "gflops_out is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    CKC(nullptr, cudaGetDevice(&dev));
    CKC(nullptr, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 8 * sms, iters = 4096;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CKC(nullptr, cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch_fp64_fma(blocks, iters, s);  // warm-up
    float best = 0.f;
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = launch_fp64_fma(blocks, iters, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    CKC(nullptr, e);
    const double fmas = (double)blocks * 256.0 * 8.0 * iters;
    *gflops_out = 2.0 * fmas / (best * 1e-3) / 1e9;
    return LBM_OK;
}

int lbm_time_stream(lbm_ctx* c, int32_t nlaunches, double* ms_out) {
    if (!c) return LBM_E_INVAL;
    if (nlaunches < 1 || !ms_out) return fail(c, LBM_E_INVAL, "nlaunches must be >= 1 and ms_out not NULL");
    int r = sync_and_check(c);
    if (r) return r;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CKC(c, cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
    for (int k = 0; k < nlaunches && e == cudaSuccess; ++k)
        e = enqueue_stream_collide(c, c->cur, c->stream, c->block, c->grid, STREAM_ALL, false);
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    CKC(c, e);
    *ms_out = ms;
    return check_err(c);
}

int lbm_autotune(lbm_ctx* c, int trial_steps) {
    if (!c) return LBM_E_INVAL;
    if (trial_steps < 1) trial_steps = 20;
    int r = sync_and_check(c);
    if (r) return r;
    // Trials write only the scratch arena f[cur^1] and its step counter, both
    // of which the next real step overwrites; the state f[cur] is read-only.
    struct Cand { int mode, block, stages; };
    std::vector<Cand> cands;
    // the register kernel at 128 threads; fewer threads per CTA time faster
    // alone but lose in the overlapped step (more CTAs to place beside the
    // particle kernel)
    // a grid of resident CTAs only (3) holds every SM for the whole pass: in a
    // step with particles the particle launches then wait for the pass to end
    // (measured slower there), so it is tried only without particles
    // The staged bulk-copy kernel (2) is not a candidate: measured on every
    // workload and storage kind it ran slower than the register kernel, so it
    // stays a variant that lbm_set_launch selects explicitly.
    for (int mode : {0, 1, 3, 4})
        if (c->np_active == 0 || mode != 3) cands.push_back({mode, 128, 0});
    cudaEvent_t e0, e1;
    CKC(c, cudaEventCreate(&e0));
    CKC(c, cudaEventCreate(&e1));
    float best = 1e30f;
    Cand keep{c->grid_mode, c->block, c->stages};
    for (const Cand& k : cands) {
        c->grid_mode = k.mode;
        c->block = k.block;
        c->stages = k.stages;
        set_launch(c);
        cudaError_t e = enqueue_stream_collide(c, c->cur, c->stream, c->block, c->grid);
        if (e != cudaSuccess) continue;
        cudaEventRecord(e0, c->stream);
        for (int s = 0; s < trial_steps && e == cudaSuccess; ++s)
            e = enqueue_stream_collide(c, c->cur, c->stream, c->block, c->grid);
        cudaEventRecord(e1, c->stream);
        if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; keep = k; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->grid_mode = keep.mode;
    c->block = keep.block;
    c->stages = keep.stages;
    set_launch(c);
    return sync_and_check(c);
}

int lbm_set_launch(lbm_ctx* c, int32_t kernel, int32_t block, int32_t stages) {
    if (!c) return LBM_E_INVAL;
    if (kernel < 0 || kernel > 4 || block < 32 || block > 512 || block % 32 != 0)
        return fail(c, LBM_E_INVAL, "kernel must be 0..4 and block a multiple of 32 in [32, 512]");
    if (kernel != 2 && block > REG_K1_MAX_BLOCK)
        return fail(c, LBM_E_INVAL, "the register kernel runs at most 128 threads per CTA");
    if (kernel == 2) {
        if (stages < 1 || stages > STAGED_MAX_STAGES || block > STAGED_MAX_BLOCK)
            return fail(c, LBM_E_INVAL, "staged kernel: stages 1..8 and block <= 256");
        if (staged_blocks_per_sm(c->kind, c->noise, c->pl, block, stages) < 1)
            return fail(c, LBM_E_INVAL, "staged kernel: the shared memory of one CTA does not fit an SM");
    }
    c->grid_mode = kernel;
    c->block = block;
    c->stages = kernel == 2 ? stages : 0;
    set_launch(c);
    return LBM_OK;
}

int lbm_set_wait_limit(lbm_ctx* c, uint64_t ns) {
    if (!c) return LBM_E_INVAL;
    if (ns > 60ull * 1000000000ull) return fail(c, LBM_E_INVAL, "wait limit above 60 s");
    c->wait_ns = ns;
    c->graph_dirty = true;  // the limit travels with each launch
    return LBM_OK;
}

int lbm_debug_fail_alloc(int32_t nth) {
    if (nth < 0) return LBM_E_INVAL;
    g_fail_alloc.store(nth);
    return LBM_OK;
}

int lbm_get_launch(const lbm_ctx* c, int64_t* out4) {
    if (!c || !out4) return LBM_E_INVAL;
    out4[0] = c->grid_mode;
    out4[1] = c->block;
    out4[2] = c->stages;
    out4[3] = c->grid;
    return LBM_OK;
}

}  // extern "C"

namespace lbmk {
// The message lbm_last_error(NULL) returns, for entry points that take no
// context (the calling thread's copy, as for lbm_create).
void set_global_error(const char* msg) { g_create_error = msg ? msg : ""; }
}  // namespace lbmk

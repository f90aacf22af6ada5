// kernels.h -- launch interface between the host runtime (capi.cu) and the
// kernel translation units of the GB300 D2Q9 library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_types.h"

namespace lbmk {

struct StreamArgs {
    DomDev dom0;              // copy of doms[0] in the launch parameters (read when ndom == 1)
    const DomDev* doms;
    const int64_t* item_off;  // first work item of each domain (ndom entries)
    int ndom;
    int64_t total_items;      // sum over domains of ny * seg_per_row
    const void* src;          // population arena holding f*(t) (after link swaps)
    void* dst;                // population arena receiving f*(t+1)
    const uint8_t* solid;     // per-node solid bytes (ragged tail path)
    const uint16_t* nflags;   // per-node flag words (NF_* and bounce-back bits)
    const uint32_t* special;  // per-chunk bits: the chunk has a node with nonzero flags
    const int64_t* ctr_in;    // step counter of the source state
    int64_t* ctr_out;         // step counter of the destination state
    unsigned* err;            // sticky device error bits
    // Work selection: STREAM_ALL every item; STREAM_FAR the items not marked
    // near a particle for this step (mark[step % 3][item] != step);
    // STREAM_NEAR the items in near_list[step % 3][0 .. near_cnt[step % 3]).
    int mode;
    int flips;                // 1: also write the moments of tagged nodes (items near particles)
    const int32_t* mark;      // [3][total_items]
    const int32_t* near_list; // [3][total_items]
    const int32_t* near_cnt;  // [3]
    // Nodes that change side this step: a node whose tag carries step + 1
    // gets rho, sum f* e_x, sum f* e_y of its new populations written to
    // flipmom[3 * slot] (only work items near particles are looked at).  The
    // tags of stamp s are in copy (s & 1), fliptag_stride nodes apart.
    const int64_t* fliptag;
    int64_t fliptag_stride;
    double* flipmom;
    // Limit of the staged kernel's stage waits in global-timer nanoseconds
    // (1e9 by default; 0 makes every stage wait report expiry at once).
    uint64_t wait_ns;
};
enum { STREAM_ALL = 0, STREAM_FAR = 1, STREAM_NEAR = 2 };

// stages == 0: the register-pipelined kernel (every mode).  stages >= 1 with
// mode ALL or FAR: the staged kernel, in which each warp keeps `stages` row
// segments in flight through bulk asynchronous copies into shared memory;
// mode NEAR always takes the register kernel.  pdl: launch the register
// kernel as a programmatic dependent of the kernel before it in stream s
// (it is then placed on the SMs while that kernel drains, and waits for its
// completion and memory flush before touching memory); ignored by the
// staged kernel.
cudaError_t launch_stream_collide(int kind, bool noise, bool pl, const StreamArgs& a, int block, int64_t grid,
                                  int stages, cudaStream_t s, bool pdl = false);
int store_vector_width(int kind);
// CTAs of the register kernel (no flip moments) that fit on one SM at `block`
// threads, for the storage kind and collision variant (0 on error).
int reg_blocks_per_sm(int kind, bool noise, bool pl, int block);
// Dynamic shared memory of one CTA of the staged kernel, and how many such
// CTAs fit on one SM (0 when none does or the arguments are out of range).
size_t staged_smem_bytes(int kind, int block, int stages);
int staged_blocks_per_sm(int kind, bool noise, bool pl, int block, int stages);
constexpr int REG_K1_MAX_BLOCK = 128;  // threads per CTA of the register kernel
constexpr int STAGED_MAX_STAGES = 8;
constexpr int STAGED_MAX_BLOCK = 256;

// ---- auxiliary kernels (k_aux.cu) ----
// Rest state f* = omega_i rho0 on every fluid node of every domain.
cudaError_t launch_fill_rest(int kind, const DomDev* doms, int ndom, const DomDev* hdoms, void* arena,
                             const uint8_t* solid, cudaStream_t s);
// Per fluid node of one domain: the sum of the Eq. MP2 table forces of every
// offset within r_it that lands on a solid node or beyond a y wall (node
// offsets wrap on periodic axes; beyond an open end there is no wall).
cudaError_t launch_lj_wall(const DomDev& D, const uint8_t* solid, const LjEntry* tab, const int32_t* cnt, int dom,
                           double2* out, cudaStream_t s);
// Mailbox bounce-back slots of one domain from its stored fluid populations
// (after any write of the populations other than a step).
cudaError_t launch_prime_mail(int kind, const DomDev& D, void* arena, const uint16_t* nflags, cudaStream_t s);
// Host-order FP64 f[9][ny][nx] (device buffer) -> stored populations of one domain.
cudaError_t launch_import(int kind, const DomDev& D, const double* in, void* arena, const uint8_t* solid,
                          cudaStream_t s);
// Stored populations of one domain -> FP64 f[9][ny][nx] (device buffer).
cudaError_t launch_export(int kind, const DomDev& D, const void* arena, const uint8_t* solid, double* out,
                          cudaStream_t s);
// rho and u = (sum f e - rho g / 2)/rho of one domain into three [ny][nx] arrays (FP64 or FP32).
cudaError_t launch_moments(int kind, const DomDev& D, const void* arena, const uint8_t* solid, void* rho,
                           void* ux, void* uy, bool out_f32, cudaStream_t s);
// FP64 mass and momentum sums of one domain, deterministic two-stage reduction into out[3].
cudaError_t launch_checks(int kind, const DomDev& D, const void* arena, const uint8_t* solid, double* partial,
                          int nblocks, double* out, cudaStream_t s);
constexpr int CHECK_BLOCKS = 304;
// `blocks` CTAs of 256 threads, each thread 8 x iters FP64 FMAs (the FP64 rate probe).
cudaError_t launch_fp64_fma(int blocks, int iters, cudaStream_t s);

// ---- particle kernel (k_part.cu) ----
struct PartArgs {
    const DomDev* doms;
    int one_domain;            // 1 when the context has a single domain: its descriptor is dom0
    DomDev dom0;               // copy of doms[0] in the launch parameters (no dependent load)
    void* arena;               // populations holding f*(t) (read for forces, link slots exchanged)
    const uint8_t* solid;
    PartState* state;          // [2][np]: state at step t in slot (t & 1)
    const PartStatic* st;
    int np;
    // link / flip lists, two copies by step parity: copy (t & 1) holds the
    // rasterisation at t, the other receives that of t+1
    int32_t* links;            // [2][links_total]: (node << 3) | (k - 1), node = y*pitch + x of r_v
    int32_t* nlinks;           // [2][np]
    int32_t* flips;            // [2][flips_total]: (node << 1) | covered
    int32_t* nflips;           // [2][np]
    int64_t links_total, flips_total;
    double* flipmom;           // [2][flips_total][3]: rho, sum f* e_x, sum f* e_y at the step of use
    int64_t* fliptag;          // [2][nodes]: (step << 32) | flip slot, copy (step & 1), for the stream-collide pass
    int64_t fliptag_stride;
    double* ljf;               // [2][np][4]: Eq. MP2 force x, y and torque on each particle at step s, copy (s & 1)
    double* diag;              // np * DIAG_N
    unsigned* err;
    const int64_t* ctr;        // step counter of the state in `arena`
    // The force launch of step t from `arena` stores t + 1 here; the launches
    // for later steps that follow it read it instead of a state counter that
    // a concurrent stream-collide pass may already have advanced.  One word
    // per arena: the next force launch from the same arena comes only after
    // those launches have finished.
    int64_t* pstep;
    int32_t* mark;             // [3][total_items]
    int32_t* near_list;        // [3][total_items]
    int32_t* near_cnt;         // [3]
    int64_t total_items;
    const double2* ljwall;     // per node: Eq. MP2 force from static solid / wall nodes within r_it (or null)
    const LjEntry* lj_tab;     // [ndom][LJ_TAB], valid entries first
    const int32_t* lj_cnt;     // [ndom]
    // Trajectory records (or null): the force launch that reaches step t + 1
    // also writes each particle's new state to rec[((t + 1) % rec_cap) * np + p],
    // page-locked host memory mapped into the device address space.
    PartState* rec;
    int64_t rec_cap;
};
// Particle-step modes: forces + Newton-Euler, exchange of the link slots,
// advance to t+1, rebuild of the link / flip lists, marking of the near items,
// the Eq. MP2 sum, and "ahead" (the step is one past the published counter).
enum { PL_FORCES = 1, PL_SWAP = 2, PL_ADVANCE = 4, PL_RASTER = 8, PL_MARK = 16, PL_LJ = 32, PL_AHEAD = 64 };
// Launches of step t: forces, exchange and Newton-Euler (role A); after it,
// the rasterisation and marks for step t+1 (roles B, C) and the Eq. MP2 sum
// for step t+2 (role D), each on its own stream.
constexpr int PL_STEP_A = PL_FORCES | PL_SWAP | PL_ADVANCE;
constexpr int PL_STEP_R = PL_RASTER | PL_MARK | PL_ADVANCE | PL_AHEAD;
constexpr int PL_STEP_LJ = PL_LJ | PL_ADVANCE | PL_AHEAD;
// set-up at the current step t: rasterisation and marks of t, then PL_SETUP_R
// (rasterisation and marks of t+1), PL_LJ (Eq. MP2 at t) and
// PL_LJ | PL_ADVANCE (Eq. MP2 at t+1)
constexpr int PL_SETUP_R = PL_RASTER | PL_MARK | PL_ADVANCE;
// pdl as for launch_stream_collide.  The launch of role A signals its
// programmatic dependents once the particle states are solved, so that the
// stream-collide pass after it is placed while the exchange completes.
cudaError_t launch_particle_step(int kind, const PartArgs& a, int modes, cudaStream_t s, bool pdl = false);

// The thread's message for lbm_last_error(NULL) (capi.cu).
void set_global_error(const char* msg);

}  // namespace lbmk

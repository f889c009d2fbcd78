// Internal declarations shared by the CUDA translation units of the SPH library.
#pragma once

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/sph.h"

namespace sph {

constexpr int kMortonBits = 21;          // bits per axis; 63-bit codes (App. B)
constexpr int kCodeBits = 3 * kMortonBits;
constexpr int kGroup = 32;               // largest neighbour-search group (one warp)
constexpr int kStackDepth = 66;          // tree-walk stack (tree depth <= 63 for distinct 63-bit codes)
constexpr double kPi = 3.14159265358979323846;
constexpr int kGatherBatch = 4;          // state fields reordered per gather pass (scratch: 4 x n_cap doubles)
constexpr int kSortTile = 2048;          // keys per tile of a radix-sort pass (256 threads x 8 keys)
constexpr int kChunkWords = 64;          // stage-2 chunk of 32 candidates: 32 lane masks, 32 candidate ids

// Device error word bits (ctx->d_flags[0]).
enum : uint32_t {
    kErrTimeout = 1u << 0,      // a bounded spin ran out
    kErrCandOverflow = 1u << 1, // stage-1 candidate list overflow (host grows and retries)
    kErrStack = 1u << 2,        // walk stack overflow
    kErrNonFinite = 1u << 3,    // NaN/Inf position or h
    kErrNotConverged = 1u << 4, // Newton iteration hit h_max_iter
    kErrStale = 1u << 5,        // an h was clamped at cache_tol * h^n
    kErrCapacity = 1u << 6,     // a count (leaves, groups, candidate chunks) above its arrays (captured step)
    kErrCacheOverflow = 1u << 7,// the neighbour cache is smaller than the kept pairs (host grows and retries)
    kErrTimeoutS2 = 1u << 8,    // the stage-2 look-back wait ran out
    kErrHalo = 1u << 9,         // a tile of the fused reduction needs more halo (host runs the passes one by one)
};

// A captured step (sph_set_graph) runs every stage without the host in between: a stage whose
// inputs an earlier stage left incomplete returns without writing.  Each mask holds the bits that
// the stages before the kernel set (never a bit the kernel itself sets, so all its blocks agree).
constexpr uint32_t kAbortTree = kErrNonFinite | kErrTimeout | kErrCapacity | kErrHalo;
constexpr uint32_t kAbortStage2 = kAbortTree | kErrCandOverflow | kErrStack;
constexpr uint32_t kAbortDensity = kAbortStage2 | kErrCacheOverflow | kErrTimeoutS2;
constexpr uint32_t kAbortStep = kAbortDensity | kErrStale | kErrNotConverged;

// Error word as an abort source: nullptr outside a captured step.  A plain (L1-cached) load: the
// bits that matter were set by earlier kernels, and every warp of a launch reads the same word, so
// an uncached load per warp would queue hundreds of thousands of requests on one L2 slice.
__device__ __forceinline__ bool aborted(const uint32_t *abort, uint32_t mask) {
    return abort && (*abort & mask);
}

// A data-dependent count (leaves, groups) read on the device.  Arrays indexed by it hold cap
// entries; a count above cap flags kErrCapacity and reads as 0, as does any count in a captured step
// after an earlier stage failed (abort bits).  Outside a captured step the host has sized the arrays
// and the launch from the same count.
struct Count {
    const int64_t *n;
    int64_t cap;
    uint32_t *flags;
    const uint32_t *abort;
};
__device__ __forceinline__ int64_t read_count(const Count &c, uint32_t mask) {
    if (aborted(c.abort, mask)) return 0;
    const int64_t v = __ldg(c.n);   // written by an earlier kernel, read-only here
    if (v > c.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(c.flags, kErrCapacity);
        return 0;
    }
    return v;
}

// One tree node: tight box and largest smoothing length; 64 bytes, two 32-byte sectors.
struct __align__(16) Node {
    double lo[3];
    double hmax;
    double hi[3];
    double pad;
};

// FP32 copy of a node with the box rounded outwards and h_max rounded up (tree walk): 32 bytes.
struct __align__(16) NodeF {
    float lo[3];
    float hmax;
    float hi[3];
    float pad;
};

// Both children of an internal node as the walk tests them (64 bytes): their FP32 boxes, each child's
// node id in its .pad (as int bits), so that a popped node costs one dependent load.
struct __align__(16) WNode {
    NodeF l, r;
};

__device__ __forceinline__ NodeF to_float_outward(const Node &b) {
    NodeF f;
    for (int k = 0; k < 3; k++) {
        f.lo[k] = __double2float_rd(b.lo[k]);
        f.hi[k] = __double2float_ru(b.hi[k]);
    }
    f.hmax = __double2float_ru(b.hmax);
    f.pad = 0.f;
    return f;
}

// Groups of the neighbour search: the largest tree nodes holding at most 32 particles and lying in
// one box, so a group is a Morton cell (spatially compact, a run of consecutive particles); a leaf
// with more than 32 particles is cut into runs of 32.  Group g is particles start[g] .. start[g+1].
struct Groups {
    const int64_t *start;     // [G + 1]
    const uint16_t *box;      // [G] or nullptr (one box)
};
__device__ __forceinline__ int64_t group_first(const Groups &gr, int64_t g) { return gr.start[g]; }
__device__ __forceinline__ int64_t group_end(const Groups &gr, int64_t g) { return gr.start[g + 1]; }
__device__ __forceinline__ int group_box_of(const Groups &gr, int64_t g) { return gr.box ? gr.box[g] : 0; }

// Cache layout: group g of S particles owns rows of 4 S entries from off_g (a multiple of 4); the
// particle in lane l of the group keeps its entries k = 4 r + j at off_g + 4 S r + 4 l + j.  Each
// particle's entries come in aligned 16-byte quads, and one row of a group is contiguous, so a
// warp reads a row with one 16-byte load per lane and stage 2 writes whole quads.
// List head of a particle: off_g + 4 l in the low 58 bits, the stride S above.
constexpr int kNbStrideShift = 58;
__device__ __forceinline__ unsigned long long pack_nb_ptr(int64_t off, int64_t stride) {
    return ((unsigned long long)stride << kNbStrideShift) | (unsigned long long)off;
}
__device__ __forceinline__ const uint32_t *nb_list(const uint32_t *nb_ids, unsigned long long w, uint32_t &stride) {
    stride = (uint32_t)(w >> kNbStrideShift);
    return nb_ids + (int64_t)(w & ((1ULL << kNbStrideShift) - 1));
}
// Entry k of a list; quad r (entries 4r .. 4r+3); pair of entries k, k+1 for even k; the extent of
// a list of cnt entries from its head (for prefetches).
__device__ __forceinline__ uint32_t nb_at(const uint32_t *ids, uint32_t k, uint32_t st) {
    return ids[(int64_t)(k >> 2) * 4 * st + (k & 3)];
}
__device__ __forceinline__ uint4 nb_quad(const uint32_t *ids, uint32_t r, uint32_t st) {
    return *reinterpret_cast<const uint4 *>(ids + (int64_t)r * 4 * st);
}
__device__ __forceinline__ uint2 nb_pair(const uint32_t *ids, uint32_t k, uint32_t st) {
    return *reinterpret_cast<const uint2 *>(ids + (int64_t)(k >> 2) * 4 * st + (k & 3));
}
__device__ __forceinline__ int64_t nb_span(uint32_t cnt, uint32_t st) {
    return cnt ? (int64_t)((cnt - 1) >> 2) * 4 * st + 4 : 0;
}

// Device scalars written by kernels and read back by the host in one copy.
struct DevScalars {
    unsigned long long dt_min_bits;   // CFL min over particles (positive double as bits)
    unsigned long long dv_max_bits;   // max |dv| (positive double as bits)
    int64_t n_leaves;
    int64_t total_slots;              // neighbour-cache entries incl. padding
    int64_t total_chunks;             // 32-candidate chunks of stage 2
    int64_t n_pairs;                  // real pairs
    uint32_t max_iters;
    uint32_t flags;
    uint32_t s2_ticket;               // stage-2 group ticket
    uint32_t pad_;
    unsigned long long pair_evals;    // density: neighbour evaluations summed over Newton passes
    unsigned long long dens_inrange;  // density: evaluations with q < 2
    unsigned long long inrange_pairs; // forces: pairs inside 2 max(h_a, h_b)
    double v2_sum;                    // sum |v|^2 after the corrector
    int64_t n_groups;                 // groups of the last tree build
};
static_assert(sizeof(DevScalars) % 8 == 0, "DevScalars is copied as a whole");

struct Buffer {
    void *p = nullptr;
    size_t bytes = 0;
};

// Block-wide exclusive scan of one value per thread; returns the exclusive prefix and sets total
// to the block sum (same value in every thread).
template <int kThreads>
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t &total) {
    __shared__ int64_t warp_off[kThreads / 32];
    __shared__ int64_t s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_off[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = (lane < kThreads / 32) ? warp_off[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kThreads / 32) warp_off[lane] = wi - w;
        if (lane == kThreads / 32 - 1) s_total = wi;
    }
    __syncthreads();
    const int64_t r = warp_off[warp] + incl - v;
    total = s_total;
    __syncthreads();
    return r;
}

}  // namespace sph

struct sph_ctx {
    sph_params p;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    int64_t n_cap = 0;
    int64_t n = 0;
    std::string last_error;

    // ---- tree ----
    uint64_t *keys[2] = {nullptr, nullptr};
    uint32_t *vals[2] = {nullptr, nullptr};
    uint32_t *digit_hist = nullptr;    // [8][256] global digit counts
    uint32_t *lookback = nullptr;      // [8][tiles][256] decoupled look-back words
    uint32_t *tile_ctr = nullptr;      // [8]
    int64_t sort_tiles = 0;
    uint64_t *mu = nullptr;            // sorted codes (points into keys[x])
    uint32_t *perm = nullptr;          // sort permutation (points into vals[x])
    uint8_t *mask[2] = {nullptr, nullptr};
    int64_t *scan_tmp = nullptr;       // block sums for scans
    int64_t *leaf_first = nullptr;     // [n_cap + 1]
    uint64_t *mu_leaf = nullptr;       // [n_cap]
    int32_t *lchild = nullptr, *rchild = nullptr, *endrange = nullptr;  // [n_cap]
    uint8_t *lflag = nullptr, *rflag = nullptr;
    int32_t *child = nullptr;          // [2 n_cap] absolute node ids of both children
    int32_t *node_parent = nullptr;    // [n_cap] parent of internal node (-1 root)
    int32_t *leaf_parent = nullptr;    // [n_cap] parent of leaf
    uint32_t *visit = nullptr;         // [n_cap]
    sph::Node *nodes = nullptr;        // [2 n_cap]
    sph::NodeF *nodesf = nullptr;      // [2 n_cap] FP32 outward copy for the walk
    sph::WNode *wnodes = nullptr;      // [n_cap] per internal node: both children for the walk
    int64_t n_leaves = 0;
    int64_t l_cap = 0;                 // capacity of the leaf- and node-indexed arrays (ensure_tree)
    bool tree_valid = false;

    // ---- reorder scratch and per-particle derived arrays ----
    double *gather_tmp = nullptr;      // [kGatherBatch][n_cap]
    uint32_t *id_tmp = nullptr;
    uint4 *qpos = nullptr;             // [n_cap] fixed-point positions, .w FP32 h (see QScale)
    double *h_base = nullptr;          // [n_cap] h^n of the cache

    // ---- neighbour cache ----
    int64_t n_groups = 0;              // groups of the current tree (tree_build)
    int64_t g_cap = 0;                 // capacity of the per-group arrays
    sph::NodeF *gboxf = nullptr;       // [groups] FP32 group boxes, rounded outwards
    int64_t *grp_chunks = nullptr;     // [groups + 1] candidate chunks per group -> scan
    int64_t *chunk_off = nullptr;      // [groups + 1]
    uint32_t *masks = nullptr;         // [chunks * kChunkWords] stage-2 hit masks and candidates
    int64_t masks_cap = 0;
    uint2 *cand = nullptr;             // [groups * cand_cap] candidate particle ranges [x, y)
    uint32_t *cand_cnt = nullptr;      // [groups]
    int cand_cap = 0;
    uint32_t *nb_cnt = nullptr;        // [n_cap] per-particle neighbour count
    unsigned long long *nb_ptr = nullptr;  // [n_cap] list start and stride (pack_nb_ptr)
    int64_t *grp_slots = nullptr;      // [groups + 1] stage-2 look-back words
    int64_t *grp_off = nullptr;        // [groups + 1]
    uint32_t *nb_ids = nullptr;        // cache entries in quads: off_g + 4 size_g (k/4) + 4 lane + k%4
    int64_t nb_cap = 0;
    int64_t n_pairs = 0, total_slots = 0;
    bool cache_valid = false;

    // ---- physics scratch ----
    void *frec = nullptr;              // [n_cap] 128-byte FP64 records of the force loop
    float4 *m_v = nullptr;             // [n_cap] mixed: vx, vy, vz, 1/h
    float4 *m_t = nullptr;             // [n_cap] mixed: P/(rho^2 Omega), 1/(rho Omega), c_s, P
    float4 *m_r = nullptr;             // [n_cap] mixed: rho, u
    double *a_new = nullptr;           // [4][n_cap] ax, ay, az, du of the force pass inside sph_step
    double *dhdt = nullptr;            // [n_cap] dh/dt from the last force pass (Morton order of the state)
    bool dhdt_valid = false;
    double *block_part = nullptr;      // per-block partial sums
    double *rerun = nullptr;           // [8][n_cap] v*, u*, a^n, du^n of the step (corrector re-runs)
    double cfl_lambda = 1.0;           // CFL multiplier lambda_CFL (App. G)
    int corr_passes = 0;               // corrector passes of the last step
    bool density_valid = false;
    bool forces_valid = false;

    // ---- host-state staging for sph_step_host ----
    double *hs_fields = nullptr;       // [16][n_cap]
    uint32_t *hs_id = nullptr;

    // ---- boxes (one for sph_create, several for sph_batch_create) and groups ----
    bool batch = false;
    int n_boxes = 1;
    int box_bits = 0;                  // bits of the box index at the top of the key
    int morton_bits = 21;              // bits per axis of the Morton code
    std::vector<int64_t> h_box_off;    // [n_boxes + 1] host copy (batch)
    uint16_t *box_of = nullptr;        // [n_cap] box of each particle position (batch)
    double *box_mass = nullptr;        // [n_boxes] (batch)
    double *box_gamma = nullptr;       // [n_boxes] (batch)
    int32_t *box_root = nullptr;       // [n_boxes] node at the root of each box's subtree
    double *box_dt = nullptr;          // [n_boxes] time step of the current step (one entry for one box)
    unsigned long long *box_dt_next = nullptr;  // [n_boxes] CFL minimum (bits) of the last force pass
    std::vector<double> h_box_dt;      // host copy of the last CFL step per box
    int64_t *gstart = nullptr;         // [groups + 1] first particle of each group
    uint16_t *group_box = nullptr;     // [groups] box of each group (batch)

    // ---- scalars / flags ----
    sph::DevScalars *dscal = nullptr;
    sph::DevScalars *hscal = nullptr;  // pinned host mirror
    double dt_next = -1.0;
    sph_stats stats{};
    sph_launch launch{128, 128, 128, 4, 3};  // launch shapes (sph_set_launch / sph_autotune)
    int64_t launches = 0;              // kernels launched by this context
    bool timing = false;               // per-stage CUDA-event timing (sph_set_timing)
    cudaEvent_t ev[2] = {nullptr, nullptr};

    // ---- captured step (sph_set_graph) ----
    bool graph_on = false;             // replay sph_step as one CUDA graph
    bool capturing = false;            // recording: no host reads, grids from the capacities
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap_stream = nullptr; // private stream the step is captured on
    uint64_t eager_gen = 0;            // gen after the last step that ran (or finished) stage by stage
    uint64_t gen = 1;                  // bumped by every reallocation and setting change
    uint64_t graph_gen = 0;            // gen the graph was captured at
    sph_state graph_state{};           // state the graph was captured for
    bool graph_dhdt = false;           // dh/dt gathered with the state in the captured step
    double *h_dt = nullptr;            // [n_boxes] pinned: time step of the next step, copied to box_dt
    unsigned long long *h_dt_bits = nullptr;  // [n_boxes] pinned: box_dt_next read back (batch)
    int64_t graph_launches = 0;        // kernels in the captured step
    int64_t graph_replays = 0, graph_captures = 0, graph_fallbacks = 0;
};

namespace sph {

// ---------------------------------------------------------------- launch helpers (host)
int fail(sph_ctx *c, int code, const char *fmt, ...);
int cuda_fail(sph_ctx *c, cudaError_t e, const char *where);
inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Opt a kernel into `bytes` of dynamic shared memory (above the 48 KiB default) on the current device.
// The attribute is per device, so it is set once per device and kernel (a process may drive contexts
// on several GPUs).
template <auto Kernel>
cudaError_t smem_opt_in(size_t bytes) {
    constexpr int kDevices = 64;
    static std::mutex mu;
    static size_t done[kDevices] = {};
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    const cudaError_t ge = cudaGetDevice(&dev);
    if (ge != cudaSuccess) return ge;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < kDevices && done[dev] >= bytes) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && dev >= 0 && dev < kDevices) done[dev] = bytes;
    return e;
}

#define SPH_CUDA(ctx, call)                                        \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return sph::cuda_fail((ctx), e_, #call); \
    } while (0)

#define SPH_LAUNCH_CHECK(ctx, name)                                \
    do {                                                           \
        ++(ctx)->launches;                                         \
        cudaError_t e_ = cudaGetLastError();                       \
        if (e_ != cudaSuccess) return sph::cuda_fail((ctx), e_, name); \
    } while (0)

// ---------------------------------------------------------------- stage entry points (host)
int tree_build(sph_ctx *c, sph_state *s, bool gather_outputs);
int tree_boxes(sph_ctx *c, const sph_state *s);   // A6 again with the current h
int neighbours_build(sph_ctx *c, const sph_state *s);
int debug_sort_timeout(sph_ctx *c, uint32_t spins);                          // failure-detection probes
int debug_stage2_timeout(sph_ctx *c, const sph_state *s, uint32_t spins);
int density_run(sph_ctx *c, sph_state *s, int *iters, bool *stale);
int forces_run(sph_ctx *c, sph_state *s, double *ax, double *ay, double *az, double *du);
int integrate_predict(sph_ctx *c, sph_state *s, double dt, const double *dhdt);
int integrate_correct(sph_ctx *c, sph_state *s, double dt);
int integrate_correct_again(sph_ctx *c, sph_state *s, double dt);   // corrector re-run from v*, u*
int integrate_save(sph_ctx *c, sph_state *s);                       // v*, u*, a^n, du^n -> rerun
int switch_run(sph_ctx *c, sph_state *s, double dt);               // shock-switch step of alpha
int read_scalars(sph_ctx *c);
Groups make_groups(const sph_ctx *c);
int ensure_groups(sph_ctx *c, int64_t G);   // grow the per-group arrays to G groups
int ensure_tree(sph_ctx *c, int64_t L);     // grow the leaf- and node-indexed arrays to L leaves
int ensure_force_records(sph_ctx *c);       // force records of the current precision
// Per-stage timing: stage_begin/stage_end bracket the launches of one stage on the context stream;
// with timing on, stage_end waits for the stage and adds its duration to stats.stage_ms[k].
enum Stage { kStPredict = 0, kStTree, kStNeigh, kStDensity, kStForcePrep, kStForces, kStCorrect, kStSwitch,
             kStCount };
int stage_begin(sph_ctx *c, int k);
int stage_end(sph_ctx *c, int k);
int exclusive_scan_i64(sph_ctx *c, const int64_t *in, int64_t *out, int64_t n);  // out[n] = total
// The same over the first min(*dn, cap) elements of in, for a count known only on the device (out
// needs cap + 1 entries; out[count] = total).
int exclusive_scan_i64_dev(sph_ctx *c, const int64_t *in, int64_t *out, const int64_t *dn, int64_t cap);
// Launch extents of the leaf- and group-indexed kernels: the counts, or in a captured step the
// capacities (the kernels read the counts on the device).
inline int64_t launch_leaves(const sph_ctx *c) { return c->capturing ? c->l_cap : c->n_leaves; }
inline int64_t launch_groups(const sph_ctx *c) { return c->capturing ? c->g_cap : c->n_groups; }
inline const uint32_t *abort_word(const sph_ctx *c) { return c->capturing ? &c->dscal->flags : nullptr; }
Count leaf_count(sph_ctx *c);
Count group_count(sph_ctx *c);

// Fixed-point positions (uint4 per particle: x, y, z counts, .w the FP32 bits of h): per axis the
// position as an unsigned 32-bit count of steps from an origin.  Periodic box: steps of L 2^-32 from
// the low corner, the count taken modulo 2^32, so that the int32 difference of two counts is the
// separation of the nearest periodic image.  Open box: steps of L 2^-30 from lo - L/2, so that
// differences of positions inside the box stay below 2^31 steps.  A separation is one integer
// subtraction, one conversion and one product per axis; its error is the conversion's rounding
// (2^-24 relative) plus under one step (2^-32 L or 2^-30 L) of absolute error.
struct QScale {
    double lo[3];   // origin
    double k[3];    // steps per unit length
};

inline QScale qpos_scale(const double *box_lo, const double *box_hi, int periodic) {
    QScale q;
    for (int k = 0; k < 3; k++) {
        const double L = box_hi[k] - box_lo[k];
        q.lo[k] = periodic ? box_lo[k] : box_lo[k] - 0.5 * L;
        q.k[k] = (periodic ? 0x1p32 : 0x1p30) / L;
    }
    return q;
}

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ double min_image(double d, double L, double halfL, int periodic) {
    if (periodic) {
        if (d > halfL) d -= L;
        else if (d < -halfL) d += L;
    }
    return d;
}

__device__ __forceinline__ unsigned long long dbits(double v) {
    return (unsigned long long)__double_as_longlong(v);
}

// Signed-integer key with the order of the double (non-NaN values; -0.0 sorts below +0.0): compares
// and min / max of doubles on the integer pipe (the FP64 pipe is 1/64 of FP32 on this GPU).
__device__ __forceinline__ long long order_key(double v) {
    const long long b = __double_as_longlong(v);
    return b < 0 ? b ^ 0x7fffffffffffffffLL : b;
}
__device__ __forceinline__ double from_order_key(long long k) {
    return __longlong_as_double(k < 0 ? k ^ 0x7fffffffffffffffLL : k);
}
__device__ __forceinline__ bool nan_bits(double v) {
    return ((unsigned long long)__double_as_longlong(v) << 1) > 0xffe0000000000000ULL;
}

// Warp-wide FP32 min / max (all 32 lanes).
__device__ __forceinline__ float warp_min_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace sph

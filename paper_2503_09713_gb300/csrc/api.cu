// C ABI of the SPH library: context, allocation, stage entry points and the time step (App. G).
#include <cstdarg>
#include <cstring>
#include <vector>
#include <algorithm>
#include <initializer_list>

#include "sph_internal.cuh"

namespace sph {

int64_t scan_scratch_elems(int64_t n);

// Grow a set of device arrays to new byte sizes (contents not kept); on failure all are freed.
static int regrow(sph_ctx *c, void **const *ptrs, const size_t *bytes, size_t count, const char *what) {
    ++c->gen;   // a captured step holds the old pointers
    for (size_t k = 0; k < count; k++) {
        if (*ptrs[k]) SPH_CUDA(c, cudaFree(*ptrs[k]));
        *ptrs[k] = nullptr;
    }
    for (size_t k = 0; k < count; k++) {
        if (cudaMalloc(ptrs[k], bytes[k]) != cudaSuccess) {
            cudaGetLastError();
            for (size_t j = 0; j < count; j++) {
                if (*ptrs[j]) cudaFree(*ptrs[j]);
                *ptrs[j] = nullptr;
            }
            return fail(c, SPH_ERR_OOM, "%s", what);
        }
    }
    return SPH_OK;
}

// Arrays indexed by leaf or node (their number L is known only after the compaction of A4).
int ensure_tree(sph_ctx *c, int64_t L) {
    if (L <= c->l_cap) return SPH_OK;
    const int64_t cap = std::min(L + L / 4 + 64, c->n_cap);   // L <= n
    void **ptrs[] = {(void **)&c->lchild, (void **)&c->rchild, (void **)&c->endrange, (void **)&c->lflag,
                     (void **)&c->rflag, (void **)&c->child, (void **)&c->node_parent, (void **)&c->leaf_parent,
                     (void **)&c->visit, (void **)&c->nodes, (void **)&c->nodesf, (void **)&c->wnodes};
    const size_t bytes[] = {(size_t)cap * 4, (size_t)cap * 4, (size_t)cap * 4, (size_t)cap, (size_t)cap,
                            (size_t)cap * 8, (size_t)cap * 4, (size_t)cap * 4, (size_t)cap * 4,
                            (size_t)cap * 2 * sizeof(Node), (size_t)cap * 2 * sizeof(NodeF),
                            (size_t)cap * sizeof(WNode)};
    c->l_cap = 0;
    int r = regrow(c, ptrs, bytes, sizeof(ptrs) / sizeof(ptrs[0]), "tree arrays");
    if (r) return r;
    c->l_cap = cap;
    return SPH_OK;
}

// Per-particle records of the force loop of the current precision, allocated on first use.
int ensure_force_records(sph_ctx *c) {
    const size_t N = (size_t)c->n_cap;
    if (c->p.precision == SPH_MIXED) {
        if (c->m_v) return SPH_OK;
        void **ptrs[] = {(void **)&c->m_v, (void **)&c->m_t, (void **)&c->m_r};
        const size_t bytes[] = {N * 16, N * 16, N * 16};
        return regrow(c, ptrs, bytes, 3, "mixed force records");
    }
    if (c->frec) return SPH_OK;
    void **ptrs[] = {(void **)&c->frec};
    const size_t bytes[] = {N * 176};   // one FP64 force record (FRec) per particle
    return regrow(c, ptrs, bytes, 1, "FP64 force records");
}

int fail(sph_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->last_error = buf;
    }
    return code;
}

int cuda_fail(sph_ctx *c, cudaError_t e, const char *where) {
    return fail(c, SPH_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

int stage_begin(sph_ctx *c, int k) {
    (void)k;
    if (!c->timing) return SPH_OK;
    SPH_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
    return SPH_OK;
}

int stage_end(sph_ctx *c, int k) {
    if (!c->timing) return SPH_OK;
    SPH_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
    SPH_CUDA(c, cudaEventSynchronize(c->ev[1]));
    float ms = 0.f;
    SPH_CUDA(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
    c->stats.stage_ms[k] += ms;
    return SPH_OK;
}

Groups make_groups(const sph_ctx *c) {
    Groups g;
    g.start = c->gstart;
    g.box = c->batch ? c->group_box : nullptr;
    return g;
}

// Per-group arrays for G groups (their number is known only after a tree build); grown with a
// margin, contents not kept.
int ensure_groups(sph_ctx *c, int64_t G) {
    if (G <= c->g_cap) return SPH_OK;
    const int64_t cap = std::min(G + G / 4 + 64, c->n_cap);   // G <= n
    void **ptrs[] = {(void **)&c->gboxf, (void **)&c->grp_chunks, (void **)&c->chunk_off,
                     (void **)&c->cand, (void **)&c->cand_cnt, (void **)&c->grp_slots, (void **)&c->grp_off,
                     (void **)&c->gstart, (void **)&c->group_box};
    const size_t bytes[] = {(size_t)cap * sizeof(NodeF), (size_t)(cap + 1) * 8,
                            (size_t)(cap + 1) * 8, (size_t)cap * c->cand_cap * sizeof(uint2), (size_t)cap * 4,
                            (size_t)(cap + 1) * 8, (size_t)(cap + 1) * 8, (size_t)(cap + 1) * 8,
                            (size_t)cap * 2};
    c->g_cap = 0;
    int r = regrow(c, ptrs, bytes, sizeof(ptrs) / sizeof(ptrs[0]), "per-group arrays");
    if (r) return r;
    c->g_cap = cap;
    return SPH_OK;
}

int read_scalars(sph_ctx *c) {
    SPH_CUDA(c, cudaMemcpyAsync(c->hscal, c->dscal, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    if (c->batch)   // per-box CFL minima of the last force pass, in the same synchronisation
        SPH_CUDA(c, cudaMemcpyAsync(c->h_dt_bits, c->box_dt_next, (size_t)c->n_boxes * 8, cudaMemcpyDeviceToHost,
                                    c->stream));
    SPH_CUDA(c, cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

Count leaf_count(sph_ctx *c) { return Count{&c->dscal->n_leaves, c->l_cap, &c->dscal->flags, abort_word(c)}; }
Count group_count(sph_ctx *c) { return Count{&c->dscal->n_groups, c->g_cap, &c->dscal->flags, abort_word(c)}; }

}  // namespace sph

using namespace sph;

namespace {

template <typename T>
int alloc(sph_ctx *c, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, SPH_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    }
    return SPH_OK;
}

void free_all(sph_ctx *c) {
    void *ptrs[] = {c->keys[0], c->keys[1], c->vals[0], c->vals[1], c->digit_hist, c->lookback, c->tile_ctr,
                    c->mask[0], c->mask[1], c->scan_tmp, c->leaf_first, c->mu_leaf, c->lchild, c->rchild,
                    c->endrange, c->lflag, c->rflag, c->child, c->node_parent, c->leaf_parent, c->visit, c->nodes, c->nodesf, c->wnodes,
                    c->gather_tmp, c->id_tmp, c->qpos, c->h_base, c->gboxf, c->grp_chunks, c->chunk_off, c->masks, c->cand, c->cand_cnt, c->nb_cnt, c->nb_ptr,
                    c->grp_slots, c->grp_off, c->nb_ids, c->frec, c->m_v, c->m_t, c->m_r, c->a_new, c->dhdt, c->block_part, c->rerun,
                    c->hs_fields, c->hs_id, c->dscal, c->box_of, c->box_mass, c->box_gamma, c->box_root,
                    c->box_dt, c->box_dt_next, c->gstart, c->group_box};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->hscal) cudaFreeHost(c->hscal);
    if (c->h_dt) cudaFreeHost(c->h_dt);
    if (c->h_dt_bits) cudaFreeHost(c->h_dt_bits);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
}

int check_params(sph_ctx *c, const sph_params *p) {
    if (!p) return fail(c, SPH_ERR_INVALID_ARG, "params is NULL");
    if (p->kernel < SPH_KERNEL_M4 || p->kernel > SPH_KERNEL_C6) return fail(c, SPH_ERR_INVALID_ARG, "unknown kernel");
    if (p->precision != SPH_FP64 && p->precision != SPH_MIXED)
        return fail(c, SPH_ERR_INVALID_ARG, "precision must be SPH_FP64 or SPH_MIXED");
    if (!(p->hfact > 0) || !(p->gamma > 1) || !(p->h_tol > 0) || !(p->h_clamp > 1) || !(p->cache_tol >= 1) ||
        !(p->c_cour > 0) || !(p->c_force > 0) || p->alpha_av < 0 || p->beta_av < 0 || p->alpha_u < 0)
        return fail(c, SPH_ERR_INVALID_ARG, "parameter out of range");
    if (p->morton_bits < 1 || p->morton_bits > 21) return fail(c, SPH_ERR_INVALID_ARG, "morton_bits outside 1..21");
    if ((p->av_switch != 0 && p->av_switch != 1) || p->max_corr < 1 || !(p->alpha_min >= 0) ||
        !(p->alpha_min <= p->alpha_av) || !(p->sigma_decay >= 0) || !(p->eps_v >= 0) || !(p->lambda_stiff >= 0))
        return fail(c, SPH_ERR_INVALID_ARG, "shock-switch / corrector parameters out of range");
    if (p->h_max_iter < 1 || p->reduction_level < 0 || p->reduction_level > 16 || p->max_outer < 1)
        return fail(c, SPH_ERR_INVALID_ARG, "iteration limits out of range");
    for (int k = 0; k < 3; k++)
        if (!(p->box_hi[k] > p->box_lo[k])) return fail(c, SPH_ERR_INVALID_ARG, "empty box along axis %d", k);
    return SPH_OK;
}

int check_state(sph_ctx *c, const sph_state *s, bool need_vel) {
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!s) return fail(c, SPH_ERR_INVALID_ARG, "state is NULL");
    if (s->n < 1 || s->n > c->n_cap)
        return fail(c, SPH_ERR_INVALID_ARG, "n = %lld outside [1, %lld]", (long long)s->n, (long long)c->n_cap);
    if (!c->batch && !(s->mass > 0)) return fail(c, SPH_ERR_INVALID_ARG, "mass must be positive");
    if (c->batch && s->n != c->n_cap) return fail(c, SPH_ERR_INVALID_ARG, "a batch state holds every box");
    if (!s->x || !s->y || !s->z || !s->h) return fail(c, SPH_ERR_INVALID_ARG, "x, y, z and h are required");
    if (need_vel && (!s->vx || !s->vy || !s->vz || !s->u || !s->ax || !s->ay || !s->az || !s->du || !s->rho ||
                     !s->omega || !s->vsig))
        return fail(c, SPH_ERR_INVALID_ARG, "v, u, a, du, rho, omega and vsig are required");
    if (c->tree_valid && s->n != c->n && need_vel) return fail(c, SPH_ERR_ORDER, "n changed since the tree build");
    if (need_vel && c->p.av_switch && !s->alpha)
        return fail(c, SPH_ERR_INVALID_ARG, "av_switch = 1 needs sph_state.alpha");
    return SPH_OK;
}

// Host side of a finished force pass, from the scalars read back: CFL step (per box in a batch),
// pair count, timeout flag.
int absorb_forces(sph_ctx *c) {
    double dt;
    unsigned long long b = c->hscal->dt_min_bits;
    std::memcpy(&dt, &b, sizeof dt);
    c->dt_next = dt;
    c->stats.dt_next = dt;
    c->stats.force_pairs = (int64_t)c->hscal->inrange_pairs;
    if (c->batch)
        for (int b = 0; b < c->n_boxes; b++) std::memcpy(&c->h_box_dt[(size_t)b], &c->h_dt_bits[b], 8);
    if (c->hscal->flags & (kErrTimeout | kErrTimeoutS2)) return fail(c, SPH_ERR_TIMEOUT, "device wait ran out");
    return SPH_OK;
}

int finish_forces(sph_ctx *c) {
    int r = read_scalars(c);
    if (r) return r;
    return absorb_forces(c);
}

// Density with the outer loop of App. F: while some h leaves cache_tol * h^n, refresh the cell
// h_max and rebuild the cache around the current h, then iterate again.  stale: the first density
// pass has already run (in a captured step) and left some h at the cache limit.
int density_with_restarts(sph_ctx *c, sph_state *s, int *iters, int max_outer, bool stale = false) {
    int passes = 1;
    for (;;) {
        int r;
        if (!stale) {
            if ((r = stage_begin(c, kStDensity)) || (r = density_run(c, s, iters, &stale)) ||
                (r = stage_end(c, kStDensity)))
                return r;
            if (!stale) break;
        }
        stale = false;
        if (passes >= max_outer)
            return fail(c, SPH_ERR_CACHE_STALE, "h left the cache tolerance after %d cache builds", passes);
        if ((r = stage_begin(c, kStNeigh)) || (r = tree_boxes(c, s)) || (r = neighbours_build(c, s)) ||
            (r = stage_end(c, kStNeigh)))
            return r;
        ++passes;
    }
    c->stats.outer_passes = passes;
    return SPH_OK;
}

// ------------------------------------------------------------------------------------ sph_step
// Shock switch, the saves for the corrector re-runs and the first force pass with its corrector:
// the part of a step after the density.
int step_tail(sph_ctx *c, sph_state *s, double dt) {
    int r;
    if (c->p.av_switch &&
        ((r = stage_begin(c, kStSwitch)) || (r = switch_run(c, s, dt)) || (r = stage_end(c, kStSwitch))))
        return r;
    const int64_t st = c->n_cap;
    if (c->p.eps_v > 0.0 && (r = integrate_save(c, s))) return r;   // v*, u*, a^n, du^n for the re-runs
    if ((r = forces_run(c, s, c->a_new, c->a_new + st, c->a_new + 2 * st, c->a_new + 3 * st))) return r;
    if ((r = stage_begin(c, kStCorrect)) || (r = integrate_correct(c, s, dt)) || (r = stage_end(c, kStCorrect)))
        return r;
    return SPH_OK;
}

// A0 predictor, A1-A6 tree, A7 cache, A8 density / h, then step_tail.  Stage by stage: with the host
// checks, the capacity growth and the outer restart of the density.  While capturing: one density
// pass; every check is left to the error word read back after the replay.
int step_body(sph_ctx *c, sph_state *s, double dt) {
    int r;
    if (c->p.eps_v > 0.0 && !c->rerun) {
        ++c->gen;
        if ((r = alloc(c, &c->rerun, (size_t)8 * c->n_cap))) return r;
    }
    if ((r = stage_begin(c, kStPredict)) || (r = integrate_predict(c, s, dt, c->dhdt_valid ? c->dhdt : nullptr)) ||
        (r = stage_end(c, kStPredict)))
        return r;
    // tree (reorders the state; outputs are recomputed below)
    if ((r = stage_begin(c, kStTree)) || (r = tree_build(c, s, false)) || (r = stage_end(c, kStTree))) return r;
    // cache at h^n
    if ((r = stage_begin(c, kStNeigh)) || (r = neighbours_build(c, s)) || (r = stage_end(c, kStNeigh))) return r;
    int iters = 0;
    if (c->capturing) {
        bool stale = false;
        if ((r = density_run(c, s, &iters, &stale))) return r;
    } else if ((r = density_with_restarts(c, s, &iters, c->p.max_outer))) {
        return r;
    }
    return step_tail(c, s, dt);
}

bool graph_matches(const sph_ctx *c, const sph_state *s) {
    return c->gexec && c->graph_gen == c->gen && c->graph_dhdt == c->dhdt_valid &&
           std::memcmp(&c->graph_state, s, sizeof *s) == 0;
}

// Records step_body into an executable graph.  The capture runs on a private stream (a capture
// cannot start on the legacy default stream); nothing executes until the replay.
int graph_capture(sph_ctx *c, sph_state *s, double dt) {
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (!c->cap_stream) SPH_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    const int64_t launches0 = c->launches;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        c->stream = user;
        return cuda_fail(c, e, "cudaStreamBeginCapture");
    }
    c->capturing = true;
    int r = SPH_OK;
    e = cudaMemsetAsync(&c->dscal->flags, 0, sizeof(uint32_t), c->stream);   // the step's error word
    if (e != cudaSuccess) r = cuda_fail(c, e, "cudaMemsetAsync");
    if (!r) r = step_body(c, s, dt);
    c->capturing = false;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->stream, &g);
    c->stream = user;
    c->graph_launches = c->launches - launches0;
    c->launches = launches0;
    if (r || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return r ? r : cuda_fail(c, e, "cudaStreamEndCapture");
    }
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->gexec = nullptr;
        cudaGetLastError();
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    c->graph_gen = c->gen;
    c->graph_state = *s;
    c->graph_dhdt = c->dhdt_valid;
    ++c->graph_captures;
    return SPH_OK;
}

// One replay and the single read-back of the step's scalars.  A failed stage skipped everything
// after it on the device; the host then finishes the step stage by stage: from the tree when a
// count outgrew its arrays (they grow, and the next step captures again), from the cache rebuild
// of the outer density loop when some h reached the cache limit.
int graph_replay(sph_ctx *c, sph_state *s, double dt) {
    SPH_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
    c->launches += c->graph_launches;
    ++c->graph_replays;
    int r = read_scalars(c);
    if (r) return r;
    const DevScalars &h = *c->hscal;
    const uint32_t fl = h.flags;
    if (fl & kErrNonFinite) return fail(c, SPH_ERR_NONFINITE, "non-finite position or h <= 0");
    if (fl & (kErrTimeout | kErrTimeoutS2)) return fail(c, SPH_ERR_TIMEOUT, "device wait ran out");
    if (fl & kErrStack) return fail(c, SPH_ERR_CAPACITY, "tree walk stack overflow");
    if (fl & kErrNotConverged) return fail(c, SPH_ERR_H_NOT_CONVERGED, "h iteration exceeded %d", c->p.h_max_iter);
    int iters = 0;
    if (fl & (kErrCapacity | kErrCandOverflow | kErrCacheOverflow | kErrHalo)) {
        ++c->graph_fallbacks;
        if ((r = tree_build(c, s, false)) || (r = neighbours_build(c, s)) ||
            (r = density_with_restarts(c, s, &iters, c->p.max_outer)) || (r = step_tail(c, s, dt)))
            return r;
        return finish_forces(c);
    }
    // tree and cache as built on the device
    c->n_leaves = h.n_leaves;
    c->n_groups = h.n_groups;
    c->total_slots = h.total_slots;
    c->n_pairs = h.n_pairs;
    c->tree_valid = c->cache_valid = true;
    c->stats.n = s->n;
    c->stats.n_leaves = h.n_leaves;
    c->stats.n_red = c->p.reduction_level;
    c->stats.n_groups = h.n_groups;
    c->stats.n_pairs = h.n_pairs;
    c->stats.cache_slots = h.total_slots;
    c->stats.cand_chunks = h.total_chunks;
    c->stats.density_iters_max = (int)h.max_iters;
    c->stats.density_pair_evals = (int64_t)h.pair_evals;
    c->stats.density_inrange = (int64_t)h.dens_inrange;
    if (fl & kErrStale) {
        ++c->graph_fallbacks;
        if ((r = density_with_restarts(c, s, &iters, c->p.max_outer, true)) || (r = step_tail(c, s, dt))) return r;
        return finish_forces(c);
    }
    c->stats.outer_passes = 1;
    c->density_valid = true;
    return absorb_forces(c);
}

}  // namespace

extern "C" {

void sph_default_params(sph_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->kernel = SPH_KERNEL_M4;
    p->precision = SPH_FP64;
    p->hfact = 1.2;
    p->gamma = 5.0 / 3.0;
    p->alpha_av = 1.0;
    p->beta_av = 2.0;
    p->alpha_u = 1.0;
    p->c_cour = 0.3;
    p->c_force = 0.25;
    p->h_tol = 1e-6;
    p->h_clamp = 1.2;
    p->cache_tol = 1.1;
    p->h_max_iter = 64;
    p->reduction_level = 3;
    p->periodic = 1;
    p->max_outer = 8;
    p->morton_bits = 21;
    p->av_switch = 0;
    p->max_corr = 4;
    p->alpha_min = 0.0;
    p->sigma_decay = 0.1;
    p->eps_v = 0.0;
    p->lambda_stiff = 1.0;
    for (int k = 0; k < 3; k++) {
        p->box_lo[k] = 0.0;
        p->box_hi[k] = 1.0;
    }
}

}  // extern "C"

namespace {

// Context for n_cap particles in n_boxes boxes.
int create_ctx(const sph_params *p, int64_t n_cap, int n_boxes, int64_t neigh_cap,
               void *stream, sph_ctx **out) {
    if (!out) return SPH_ERR_INVALID_ARG;
    *out = nullptr;
    sph_ctx *c = new (std::nothrow) sph_ctx();
    if (!c) return SPH_ERR_OOM;
    int r = check_params(c, p);
    if (r) { delete c; return r; }
    if (n_cap < 1 || n_cap > (int64_t)1 << 30) { delete c; return SPH_ERR_INVALID_ARG; }
    c->p = *p;
    c->launch.reduction_level = p->reduction_level;
    c->morton_bits = p->morton_bits;
    c->stream = (cudaStream_t)stream;
    c->n_cap = n_cap;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return SPH_ERR_CUDA;
    }
    const int64_t N = n_cap;
    const int64_t G = (N + 31) / 32 + n_boxes;   // per-group arrays: first guess, grown by ensure_groups
    const int64_t tiles = (N + kSortTile - 1) / kSortTile;
    const int64_t chunks = (N + 2047) / 2048;
    c->sort_tiles = tiles;
    c->cand_cap = 128;
    c->nb_cap = neigh_cap > 0 ? neigh_cap : 96 * N;
    c->masks_cap = G * 16 * kChunkWords;   // grown by the cache build when the candidate chunks need more
    const int64_t scan_elems = 2 * (chunks + 1) + scan_scratch_elems(chunks) + scan_scratch_elems(G + 1) + 64;
    if ((r = alloc(c, &c->keys[0], N)) || (r = alloc(c, &c->keys[1], N)) || (r = alloc(c, &c->vals[0], N)) ||
        (r = alloc(c, &c->vals[1], N)) || (r = alloc(c, &c->digit_hist, 8 * 256)) ||
        (r = alloc(c, &c->lookback, (size_t)8 * tiles * 256)) || (r = alloc(c, &c->tile_ctr, 8)) ||
        (r = alloc(c, &c->mask[0], N)) || (r = alloc(c, &c->mask[1], N)) || (r = alloc(c, &c->scan_tmp, scan_elems)) ||
        (r = alloc(c, &c->leaf_first, N + 1)) || (r = alloc(c, &c->mu_leaf, N)) ||
        (r = ensure_tree(c, std::max<int64_t>(N / 6, 1))) ||
        (r = alloc(c, &c->gather_tmp, (size_t)kGatherBatch * N)) || (r = alloc(c, &c->id_tmp, N)) ||
        (r = alloc(c, &c->qpos, N)) || (r = alloc(c, &c->h_base, N)) ||
        (r = ensure_groups(c, G)) || (r = alloc(c, &c->masks, (size_t)c->masks_cap)) ||
        (r = alloc(c, &c->nb_cnt, N)) || (r = alloc(c, &c->nb_ptr, N)) || (r = alloc(c, &c->nb_ids, c->nb_cap)) ||
        (r = alloc(c, &c->a_new, (size_t)4 * N)) || (r = alloc(c, &c->dhdt, N)) ||
        (r = alloc(c, &c->block_part, (size_t)(N / 256 + 2))) || (r = alloc(c, &c->dscal, 1)) ||
        (r = alloc(c, &c->box_root, n_boxes)) || (r = alloc(c, &c->box_dt, n_boxes))) {
        free_all(c);
        delete c;
        return r;
    }
    if (cudaMallocHost((void **)&c->hscal, sizeof(DevScalars)) != cudaSuccess ||
        cudaMallocHost((void **)&c->h_dt, (size_t)n_boxes * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void **)&c->h_dt_bits, (size_t)n_boxes * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return SPH_ERR_OOM;
    }
    std::memset(c->hscal, 0, sizeof(DevScalars));
    c->stats.cfl_multiplier = 1.0;
    if (cudaEventCreate(&c->ev[0]) != cudaSuccess || cudaEventCreate(&c->ev[1]) != cudaSuccess) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return SPH_ERR_CUDA;
    }
    if (cudaMemsetAsync(c->dscal, 0, sizeof(DevScalars), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->box_root, 0, (size_t)n_boxes * sizeof(int32_t), c->stream) != cudaSuccess) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return SPH_ERR_CUDA;
    }
    *out = c;
    return SPH_OK;
}

}  // namespace

extern "C" {

int sph_create(const sph_params *p, int64_t n_cap, int64_t neigh_cap, void *stream, sph_ctx **out) {
    return create_ctx(p, n_cap, 1, neigh_cap, stream, out);
}

int sph_batch_create(const sph_params *p, int n_boxes, const int64_t *box_offsets, const double *box_mass,
                     const double *box_gamma, int64_t neigh_cap, void *stream, sph_ctx **out) {
    if (!out) return SPH_ERR_INVALID_ARG;
    *out = nullptr;
    if (!p || n_boxes < 1 || n_boxes > 4096 || !box_offsets || !box_mass) return SPH_ERR_INVALID_ARG;
    if (box_offsets[0] != 0) return SPH_ERR_INVALID_ARG;
    for (int b = 0; b < n_boxes; b++) {
        const int64_t nb = box_offsets[b + 1] - box_offsets[b];
        if (nb < 0 || !(box_mass[b] > 0) || (box_gamma && !(box_gamma[b] > 1))) return SPH_ERR_INVALID_ARG;
    }
    const int64_t total = box_offsets[n_boxes];
    if (total < 1) return SPH_ERR_INVALID_ARG;
    sph_ctx *c = nullptr;
    int r = create_ctx(p, total, n_boxes, neigh_cap, stream, &c);
    if (r) return r;
    c->batch = true;
    c->n_boxes = n_boxes;
    int bits = 0;
    while ((1 << bits) < n_boxes) ++bits;
    c->box_bits = bits;
    c->morton_bits = std::min(p->morton_bits, (63 - bits) / 3);
    c->h_box_off.assign(box_offsets, box_offsets + n_boxes + 1);
    std::vector<uint16_t> box_of((size_t)total);
    std::vector<double> gam((size_t)n_boxes);
    for (int b = 0; b < n_boxes; b++) {
        for (int64_t i = box_offsets[b]; i < box_offsets[b + 1]; i++) box_of[(size_t)i] = (uint16_t)b;
        gam[(size_t)b] = box_gamma ? box_gamma[b] : p->gamma;
    }
    c->h_box_dt.assign((size_t)n_boxes, -1.0);
    auto up = [&](void *dst, const void *src, size_t bytes) -> int {
        SPH_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
        return SPH_OK;
    };
    if ((r = alloc(c, &c->box_of, total)) || (r = alloc(c, &c->box_mass, n_boxes)) ||
        (r = alloc(c, &c->box_gamma, n_boxes)) || (r = alloc(c, &c->box_dt_next, n_boxes)) || (r = up(c->box_of, box_of.data(), box_of.size() * 2)) ||
        (r = up(c->box_mass, box_mass, (size_t)n_boxes * 8)) || (r = up(c->box_gamma, gam.data(), gam.size() * 8))) {
        sph_destroy(c);
        return r;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        sph_destroy(c);
        return SPH_ERR_CUDA;
    }
    *out = c;
    return SPH_OK;
}

int sph_batch_dt(sph_ctx *c, double *dt_per_box) {
    if (!c || !dt_per_box) return SPH_ERR_INVALID_ARG;
    if (!c->batch) return fail(c, SPH_ERR_INVALID_ARG, "not a batch context");
    for (int b = 0; b < c->n_boxes; b++) dt_per_box[b] = c->h_box_dt[(size_t)b];
    return SPH_OK;
}

int sph_destroy(sph_ctx *c) {
    if (!c) return SPH_OK;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return SPH_OK;
}

int sph_set_params(sph_ctx *c, const sph_params *p) {
    if (!c) return SPH_ERR_INVALID_ARG;
    int r = check_params(c, p);
    if (r) return r;
    c->p = *p;
    ++c->gen;   // parameters are baked into a captured step
    c->launch.reduction_level = p->reduction_level;
    c->morton_bits = c->batch ? std::min(p->morton_bits, (63 - c->box_bits) / 3) : p->morton_bits;
    c->tree_valid = c->cache_valid = c->density_valid = c->forces_valid = false;
    c->dhdt_valid = false;
    c->dt_next = -1.0;
    return SPH_OK;
}

int sph_build_tree(sph_ctx *c, sph_state *s) {
    int r = check_state(c, s, false);
    if (r) return r;
    c->n = s->n;
    c->density_valid = c->forces_valid = false;
    return tree_build(c, s, true);
}

int sph_find_neighbours(sph_ctx *c, const sph_state *s, int64_t *n_pairs) {
    int r = check_state(c, s, false);
    if (r) return r;
    if (!c->tree_valid || s->n != c->n) return fail(c, SPH_ERR_ORDER, "sph_find_neighbours needs sph_build_tree");
    r = tree_boxes(c, s);   // h_max of the cells from the current h
    if (r) return r;
    r = neighbours_build(c, s);
    if (r) return r;
    if (n_pairs) *n_pairs = c->n_pairs;
    return SPH_OK;
}

int sph_debug_wait_timeout(sph_ctx *c, const sph_state *s, int which, uint32_t spins) {
    if (!c) return SPH_ERR_INVALID_ARG;
    if (spins < 1 || spins > (1u << 20)) return fail(c, SPH_ERR_INVALID_ARG, "spins outside [1, 2^20]");
    if (c->capturing) return fail(c, SPH_ERR_ORDER, "not inside a captured step");
    if (which == 0) return debug_sort_timeout(c, spins);
    if (which == 1) {
        int r = check_state(c, s, false);
        if (r) return r;
        if (s->n != c->n) return fail(c, SPH_ERR_ORDER, "the probe needs the state of the last cache build");
        return debug_stage2_timeout(c, s, spins);
    }
    return fail(c, SPH_ERR_INVALID_ARG, "which must be 0 (sort) or 1 (stage 2)");
}

int sph_compute_density_h(sph_ctx *c, sph_state *s, int *iters) {
    int r = check_state(c, s, false);
    if (r) return r;
    if (!s->rho || !s->omega) return fail(c, SPH_ERR_INVALID_ARG, "rho and omega are required");
    if (!c->cache_valid || s->n != c->n) return fail(c, SPH_ERR_ORDER, "density needs sph_find_neighbours");
    bool stale = false;
    r = density_run(c, s, iters, &stale);
    if (r) return r;
    if (stale) return fail(c, SPH_ERR_CACHE_STALE, "some h exceeded cache_tol * h^n; rebuild the cache");
    return SPH_OK;
}

int sph_compute_forces(sph_ctx *c, sph_state *s) {
    int r = check_state(c, s, true);
    if (r) return r;
    if (!c->cache_valid || s->n != c->n) return fail(c, SPH_ERR_ORDER, "forces need sph_find_neighbours");
    r = forces_run(c, s, s->ax, s->ay, s->az, s->du);
    if (r) return r;
    r = finish_forces(c);
    if (r) return r;
    c->dt_next *= c->cfl_lambda;   // the CFL multiplier of the running step sequence
    c->stats.dt_next = c->dt_next;
    if (c->batch)
        for (double &v : c->h_box_dt) v *= c->cfl_lambda;
    c->forces_valid = true;
    c->dhdt_valid = true;
    return SPH_OK;
}

int sph_step(sph_ctx *c, sph_state *s, double dt, double *dt_used, double *dt_next) {
    int r = check_state(c, s, true);
    if (r) return r;
    // time step of every box, on the device for the predictor, switch and corrector
    if (c->batch) {
        if (s->n != c->n_cap) return fail(c, SPH_ERR_INVALID_ARG, "a batch state holds every box");
        for (int b = 0; b < c->n_boxes; b++) c->h_dt[b] = dt;
        if (!(dt > 0)) {
            for (int b = 0; b < c->n_boxes; b++) {
                if (!(c->h_box_dt[(size_t)b] > 0) && c->h_box_off[b + 1] > c->h_box_off[b])
                    return fail(c, SPH_ERR_ORDER, "dt <= 0 needs a previous force evaluation");
                c->h_dt[b] = c->h_box_dt[(size_t)b] > 0 ? c->h_box_dt[(size_t)b] : 0.0;
            }
        }
        dt = *std::min_element(c->h_dt, c->h_dt + c->n_boxes);
    } else {
        if (!(dt > 0)) {
            if (!(c->dt_next > 0)) return fail(c, SPH_ERR_ORDER, "dt <= 0 needs a previous force evaluation");
            dt = c->dt_next;
        }
        c->h_dt[0] = dt;
    }
    SPH_CUDA(c, cudaMemcpyAsync(c->box_dt, c->h_dt, (size_t)c->n_boxes * sizeof(double), cudaMemcpyHostToDevice,
                                c->stream));
    c->n = s->n;
    // A0-A10 up to the first corrector pass: replayed as one graph, or stage by stage
    bool replay = false;
    if (c->graph_on && !c->timing) {
        if (!graph_matches(c, s) && c->eager_gen == c->gen && (r = graph_capture(c, s, dt))) return r;
        replay = graph_matches(c, s);
    }
    if (replay) r = graph_replay(c, s, dt);
    else if (!(r = step_body(c, s, dt))) r = finish_forces(c);
    if (r) return r;
    c->eager_gen = c->gen;   // capacities fit the current particle distribution
    // corrector re-runs with v* <- v^{n+1} while Eq. cvleapfrog fails
    const bool check = c->p.eps_v > 0.0;
    auto ratio_now = [&]() {
        double dvm;
        const unsigned long long b = c->hscal->dv_max_bits;
        std::memcpy(&dvm, &b, sizeof dvm);
        const double v2 = c->hscal->v2_sum;
        return v2 > 0 ? dvm / std::sqrt(v2 / (double)s->n) : 0.0;
    };
    c->stats.dv_ratio = ratio_now();
    const bool failed = check && !(c->stats.dv_ratio < c->p.eps_v);
    bool fails = failed;
    int pass = 1;
    while (fails && pass < c->p.max_corr) {
        ++pass;
        const int64_t st = c->n_cap;
        if ((r = forces_run(c, s, c->a_new, c->a_new + st, c->a_new + 2 * st, c->a_new + 3 * st)) ||
            (r = stage_begin(c, kStCorrect)) || (r = integrate_correct_again(c, s, dt)) ||
            (r = stage_end(c, kStCorrect)) || (r = finish_forces(c)))
            return r;
        fails = check && !(ratio_now() < c->p.eps_v);
    }
    c->corr_passes = pass;
    // CFL multiplier: halved in a step whose first pass failed, else relaxed towards 1
    if (check) {
        if (failed) c->cfl_lambda *= 0.5;
        else c->cfl_lambda = (1.0 + c->p.lambda_stiff * c->cfl_lambda) / (1.0 + c->p.lambda_stiff);
    } else {
        c->cfl_lambda = 1.0;
    }
    c->dt_next *= c->cfl_lambda;
    c->stats.dt_next = c->dt_next;
    if (c->batch)
        for (double &v : c->h_box_dt) v *= c->cfl_lambda;
    c->stats.cfl_multiplier = c->cfl_lambda;
    c->stats.corrector_passes = pass;
    c->forces_valid = true;
    c->dhdt_valid = true;
    if (dt_used) *dt_used = dt;
    if (dt_next) *dt_next = c->dt_next;
    return SPH_OK;
}

int sph_set_graph(sph_ctx *c, int enable) {
    if (!c) return SPH_ERR_INVALID_ARG;
    c->graph_on = enable != 0;
    if (!c->graph_on && c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return SPH_OK;
}

int sph_step_host(sph_ctx *c, sph_state *hs, double dt, double *dt_used, double *dt_next) {
    int r = check_state(c, hs, true);
    if (r) return r;
    const int64_t n = hs->n;
    const int64_t N = c->n_cap;
    if (!c->hs_fields) {
        if ((r = alloc(c, &c->hs_fields, (size_t)15 * N))) return r;
        if ((r = alloc(c, &c->hs_id, N))) return r;
    }
    double **hf[15] = {&hs->x, &hs->y, &hs->z, &hs->vx, &hs->vy, &hs->vz, &hs->u, &hs->h,
                       &hs->ax, &hs->ay, &hs->az, &hs->du, &hs->rho, &hs->omega, &hs->vsig};
    sph_state ds = *hs;
    double **df[15] = {&ds.x, &ds.y, &ds.z, &ds.vx, &ds.vy, &ds.vz, &ds.u, &ds.h,
                       &ds.ax, &ds.ay, &ds.az, &ds.du, &ds.rho, &ds.omega, &ds.vsig};
    // inputs of the step: positions, velocities, u, h, a, du
    for (int f = 0; f < 15; f++) {
        *df[f] = c->hs_fields + (size_t)f * N;
        if (f < 12)
            SPH_CUDA(c, cudaMemcpyAsync(*df[f], *hf[f], (size_t)n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    }
    ds.id = hs->id ? c->hs_id : nullptr;
    if (hs->id)
        SPH_CUDA(c, cudaMemcpyAsync(ds.id, hs->id, (size_t)n * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream));
    r = sph_step(c, &ds, dt, dt_used, dt_next);
    if (r) return r;
    for (int f = 0; f < 15; f++)
        SPH_CUDA(c, cudaMemcpyAsync(*hf[f], *df[f], (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (hs->id)
        SPH_CUDA(c, cudaMemcpyAsync(hs->id, ds.id, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    SPH_CUDA(c, cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

int sph_tree_sizes(sph_ctx *c, int64_t *n, int64_t *n_leaves) {
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->tree_valid) return fail(c, SPH_ERR_ORDER, "no tree");
    if (n) *n = c->n;
    if (n_leaves) *n_leaves = c->n_leaves;
    return SPH_OK;
}

int sph_export_tree(sph_ctx *c, sph_tree_view *v) {
    if (!c || !v) return SPH_ERR_INVALID_ARG;
    if (!c->tree_valid) return fail(c, SPH_ERR_ORDER, "no tree");
    const int64_t n = c->n, L = c->n_leaves, nin = L - 1, nodes = 2 * L - 1;
    auto cp = [&](void *dst, const void *src, size_t bytes) -> int {
        if (!dst || bytes == 0) return SPH_OK;
        SPH_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream));
        return SPH_OK;
    };
    int r;
    if ((r = cp(v->mu, c->mu, n * 8)) || (r = cp(v->perm, c->perm, n * 4)) ||
        (r = cp(v->leaf_first, c->leaf_first, (L + 1) * 8)) || (r = cp(v->mu_leaf, c->mu_leaf, L * 8)) ||
        (r = cp(v->lchild, c->lchild, nin * 4)) || (r = cp(v->rchild, c->rchild, nin * 4)) ||
        (r = cp(v->lflag, c->lflag, nin)) || (r = cp(v->rflag, c->rflag, nin)) ||
        (r = cp(v->endrange, c->endrange, nin * 4)) ||
        (r = cp(v->group_start, c->gstart, (c->n_groups + 1) * 8)))
        return r;
    if (v->bmin || v->bmax || v->hmax) {
        std::vector<Node> nd((size_t)nodes);
        SPH_CUDA(c, cudaMemcpyAsync(nd.data(), c->nodes, nodes * sizeof(Node), cudaMemcpyDeviceToHost, c->stream));
        SPH_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int64_t i = 0; i < nodes; i++) {
            for (int k = 0; k < 3; k++) {
                if (v->bmin) v->bmin[3 * i + k] = nd[i].lo[k];
                if (v->bmax) v->bmax[3 * i + k] = nd[i].hi[k];
            }
            if (v->hmax) v->hmax[i] = nd[i].hmax;
        }
    }
    SPH_CUDA(c, cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

int sph_export_neighbours(sph_ctx *c, int64_t *off, uint32_t *ids) {
    if (!c || !off) return SPH_ERR_INVALID_ARG;
    if (!c->cache_valid) return fail(c, SPH_ERR_ORDER, "no neighbour cache");
    const int64_t n = c->n, G = c->n_groups;
    std::vector<uint32_t> cnt((size_t)n);
    std::vector<int64_t> goff((size_t)G + 1), gst((size_t)G + 1);
    std::vector<uint32_t> raw((size_t)std::max<int64_t>(c->total_slots, 1));
    SPH_CUDA(c, cudaMemcpyAsync(cnt.data(), c->nb_cnt, n * 4, cudaMemcpyDeviceToHost, c->stream));
    SPH_CUDA(c, cudaMemcpyAsync(goff.data(), c->grp_off, (G + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
    SPH_CUDA(c, cudaMemcpyAsync(gst.data(), c->gstart, (G + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
    if (c->total_slots > 0)
        SPH_CUDA(c, cudaMemcpyAsync(raw.data(), c->nb_ids, c->total_slots * 4, cudaMemcpyDeviceToHost, c->stream));
    SPH_CUDA(c, cudaStreamSynchronize(c->stream));
    off[0] = 0;
    for (int64_t a = 0; a < n; a++) off[a + 1] = off[a] + cnt[a];
    if (ids) {
        for (int64_t g = 0; g < G; g++) {
            const int64_t first = gst[(size_t)g], end = gst[(size_t)g + 1], size = end - first;
            for (int64_t a = first; a < end; a++) {   // entry k at off_g + 4 size (k/4) + 4 lane + k%4
                const int64_t base = goff[g] + 4 * (a - first);
                for (uint32_t k = 0; k < cnt[a]; k++)
                    ids[off[a] + k] = raw[base + (int64_t)(k >> 2) * 4 * size + (k & 3)];
            }
        }
    }
    return SPH_OK;
}

int sph_get_stats(sph_ctx *c, sph_stats *st) {
    if (!c || !st) return SPH_ERR_INVALID_ARG;
    c->stats.kernel_launches = c->launches;
    c->stats.graph_replays = c->graph_replays;
    c->stats.graph_captures = c->graph_captures;
    c->stats.graph_fallbacks = c->graph_fallbacks;
    *st = c->stats;
    return SPH_OK;
}

int sph_get_launch(sph_ctx *c, sph_launch *out) {
    if (!c || !out) return SPH_ERR_INVALID_ARG;
    *out = c->launch;
    return SPH_OK;
}

int sph_set_launch(sph_ctx *c, const sph_launch *in) {
    if (!c || !in) return SPH_ERR_INVALID_ARG;
    auto blk_ok = [](int b) { return b == 64 || b == 128 || b == 256; };
    if (!blk_ok(in->density_block) || !blk_ok(in->forces_block) || !blk_ok(in->walk_block) ||
        in->stage2_warps < 1 || in->stage2_warps > 8 || in->reduction_level < 0 || in->reduction_level > 16)
        return fail(c, SPH_ERR_INVALID_ARG, "launch shape out of range");
    if (in->reduction_level != c->p.reduction_level) {
        c->p.reduction_level = in->reduction_level;
        c->tree_valid = c->cache_valid = false;
    }
    if (std::memcmp(&c->launch, in, sizeof *in) != 0) ++c->gen;   // shapes are baked into a captured step
    c->launch = *in;
    return SPH_OK;
}

static int autotune(sph_ctx *c, sph_state *s, sph_launch *best, double *ms_best) {
    int r;
    // A1-A9 with launch shapes L, timed with events on the context stream; the faster of two runs
    auto run = [&](const sph_launch &L, double &ms) -> int {
        int rr = sph_set_launch(c, &L);
        if (rr) return rr;
        ms = 1e300;
        for (int rep = 0; rep < 2; rep++) {
            SPH_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
            int iters = 0;
            if ((rr = tree_build(c, s, true)) || (rr = neighbours_build(c, s)) ||
                (rr = density_with_restarts(c, s, &iters, c->p.max_outer)) ||
                (rr = forces_run(c, s, s->ax, s->ay, s->az, s->du)) || (rr = finish_forces(c)))
                return rr;
            SPH_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
            SPH_CUDA(c, cudaEventSynchronize(c->ev[1]));
            float t = 0.f;
            SPH_CUDA(c, cudaEventElapsedTime(&t, c->ev[0], c->ev[1]));
            ms = std::min(ms, (double)t);
        }
        return SPH_OK;
    };
    sph_launch cur = c->launch;
    double cur_ms = 0.0;
    if ((r = run(cur, cur_ms))) return r;
    auto try_values = [&](int sph_launch::*field, std::initializer_list<int> values) -> int {
        for (int v : values) {
            if (cur.*field == v) continue;
            sph_launch cand = cur;
            cand.*field = v;
            double ms = 0.0;
            int rr = run(cand, ms);
            if (rr) return rr;
            if (ms < cur_ms) {
                cur = cand;
                cur_ms = ms;
            }
        }
        return SPH_OK;
    };
    if ((r = try_values(&sph_launch::reduction_level, {1, 2, 3, 4, 5, 6, 7})) ||
        (r = try_values(&sph_launch::stage2_warps, {2, 4, 8})) ||
        (r = try_values(&sph_launch::density_block, {64, 128, 256})) ||
        (r = try_values(&sph_launch::forces_block, {64, 128, 256})) ||
        (r = try_values(&sph_launch::walk_block, {64, 128, 256})))
        return r;
    // leave the context (tree, cache, outputs) in the chosen configuration
    double ms = 0.0;
    if ((r = run(cur, ms))) return r;
    c->forces_valid = true;
    c->dhdt_valid = true;
    if (best) *best = cur;
    if (ms_best) *ms_best = std::min(cur_ms, ms);
    return SPH_OK;
}

int sph_autotune(sph_ctx *c, sph_state *s, sph_launch *best, double *ms_best) {
    int r = check_state(c, s, true);
    if (r) return r;
    c->n = s->n;
    const bool timing = c->timing;   // per-stage timing would add a synchronisation per stage
    c->timing = false;
    r = autotune(c, s, best, ms_best);
    c->timing = timing;
    return r;
}

int sph_set_timing(sph_ctx *c, int enable) {
    if (!c) return SPH_ERR_INVALID_ARG;
    c->timing = enable != 0;
    return SPH_OK;
}

int sph_reset_timing(sph_ctx *c) {
    if (!c) return SPH_ERR_INVALID_ARG;
    for (double &v : c->stats.stage_ms) v = 0.0;
    return SPH_OK;
}

const char *sph_last_error(sph_ctx *c) { return c ? c->last_error.c_str() : "no context"; }

const char *sph_error_string(int s) {
    switch (s) {
        case SPH_OK: return "ok";
        case SPH_ERR_INVALID_ARG: return "invalid argument";
        case SPH_ERR_OOM: return "device out of memory";
        case SPH_ERR_CAPACITY: return "capacity exceeded";
        case SPH_ERR_CACHE_STALE: return "neighbour cache stale: h exceeded cache_tol * h^n";
        case SPH_ERR_H_NOT_CONVERGED: return "smoothing-length iteration did not converge";
        case SPH_ERR_TIMEOUT: return "bounded device wait ran out";
        case SPH_ERR_CUDA: return "CUDA error";
        case SPH_ERR_ORDER: return "call order: a required stage has not run";
        case SPH_ERR_NONFINITE: return "non-finite position or smoothing length";
        default: return "unknown status";
    }
}

}  // extern "C"

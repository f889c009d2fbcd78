/*
 * sph.h -- C ABI of the GB300 (sm_103a) SPH hot path: Morton-code radix tree with per-cell bounding
 * boxes, tree-walk neighbour cache, smoothing-length / density iteration (M4, Newton-Raphson on h)
 * and the pairwise momentum / energy loop with artificial viscosity and conductivity, advanced by a
 * kick-drift-kick leapfrog.  Method: "The Shamrock code: I - Smoothed Particle Hydrodynamics on
 * GPUs" (arXiv 2503.09713), Sect. 2.1 and Apps. B-G.
 *
 * General rules
 *  - Every function returns SPH_OK (0) or a negative sph_status; no exception or abort crosses
 *    the ABI.  sph_last_error(ctx) returns a message for the last failure of that context.
 *  - Pointers in sph_state are DEVICE pointers (except for sph_step_host), owned by the caller;
 *    the library never frees them.  All scratch memory (tree, neighbour cache, flags) belongs to
 *    the context and is freed by sph_destroy.
 *  - All device work is issued on the context's CUDA stream.  Functions that return host scalars
 *    (leaf count, pair count, iteration count, time steps) synchronise that stream.
 *  - Particle arrays are structure-of-arrays, float64, length state->n.  sph_build_tree (and
 *    therefore sph_step) reorders every non-NULL per-particle array of the state into Morton order
 *    in place and applies the same permutation to state->id, so id[i] is the original index of the
 *    particle now stored at i.
 *  - Equal-mass particles (state->mass).  The box [box_lo, box_hi) is periodic when periodic = 1;
 *    positions must lie inside it.  The interaction radius 2*cache_tol*h of every particle must
 *    stay below a quarter of the smallest box side.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_ctx sph_ctx;

typedef enum {
    SPH_OK = 0,
    SPH_ERR_INVALID_ARG = -1,     /* NULL pointer, n out of range, bad parameter */
    SPH_ERR_OOM = -2,             /* device allocation failed */
    SPH_ERR_CAPACITY = -3,        /* a fixed-capacity buffer overflowed and could not grow */
    SPH_ERR_CACHE_STALE = -4,     /* some h exceeded cache_tol * h^n: rebuild the cache (App. F) */
    SPH_ERR_H_NOT_CONVERGED = -5, /* Newton iteration on h hit h_max_iter */
    SPH_ERR_TIMEOUT = -6,         /* a bounded device-side wait ran out (no hang, results invalid) */
    SPH_ERR_CUDA = -7,            /* a CUDA runtime call failed */
    SPH_ERR_ORDER = -8,           /* call made before the stage it depends on */
    SPH_ERR_NONFINITE = -9        /* a NaN/Inf appeared in positions or smoothing lengths */
} sph_status;

/* Smoothing kernels of Sect. 2.1: Schoenberg B-splines M4 (R_kern = 2), M5 (2.5), M6 (3) and the
 * Wendland functions C2, C4, C6 (R_kern = 2), W(r, h) = C_norm f(r/h) / h^3 normalised in 3-D. */
enum { SPH_KERNEL_M4 = 0, SPH_KERNEL_M5 = 1, SPH_KERNEL_M6 = 2, SPH_KERNEL_C2 = 3, SPH_KERNEL_C4 = 4,
       SPH_KERNEL_C6 = 5 };
enum { SPH_FP64 = 0, SPH_MIXED = 1 };

/* Solver parameters (Sect. 2.1, App. F, App. G).  sph_default_params fills the paper's values. */
typedef struct {
    int kernel;           /* SPH_KERNEL_*; M4 by default (the paper's tests use M4 with hfact 1.2
                             and M6 with hfact 1.0) */
    int precision;        /* SPH_FP64: all pair arithmetic in FP64.  SPH_MIXED: FP64 positions, h
                             iteration and integration; FP32 pair sums on separations taken from
                             32-bit fixed-point positions, with Kahan-compensated accumulation */
    double hfact;         /* rho(h) = m (hfact/h)^3 (Eq. rhoh); 1.2 */
    double gamma;         /* P = (gamma-1) rho u; 5/3 */
    double alpha_av;      /* alpha^AV of v_sig; 1 */
    double beta_av;       /* beta of v_sig; 2 */
    double alpha_u;       /* beta_u of Lambda_cond; 1 (0 switches conductivity off) */
    double c_cour;        /* CFL factors (App. G); 0.3 */
    double c_force;       /* 0.25 */
    double h_tol;         /* epsilon_c of App. F; 1e-6 */
    double h_clamp;       /* lambda of App. F; 1.2 */
    double cache_tol;     /* chi of App. F (cache / ghost tolerance); 1.1 */
    int h_max_iter;       /* Newton iterations per particle before SPH_ERR_H_NOT_CONVERGED; 64 */
    int reduction_level;  /* n_red reduction passes of App. C; 3 */
    int periodic;         /* 1: periodic box */
    int max_outer;        /* cache rebuilds inside sph_step before SPH_ERR_CACHE_STALE; 8 */
    double box_lo[3];
    double box_hi[3];
    int morton_bits;      /* bits per axis of the Morton codes (App. B): 21 (63-bit codes, default) down
                             to 1; 10 gives the 30-bit codes of the paper's u32 variant, sorted in 4
                             radix passes instead of 8.  A batch keeps the box index above
                             3 * min(morton_bits, (63 - box bits) / 3) */
    /* Extensions of App. G (off by default: av_switch = 0, eps_v = 0 give the fixed-alpha step):  */
    int av_switch;        /* 1: per-particle alpha_a (sph_state.alpha) evolved by the shock switch,
                             Eq. evolalphaanalytic with its implicit step; alpha_av is alpha_max */
    int max_corr;         /* most corrector passes per step (>= 1); 4 */
    double alpha_min;     /* floor of alpha_loc; 0 */
    double sigma_decay;   /* tau_a = h_a / (sigma_decay c_s,a); 0.1 */
    double eps_v;         /* epsilon_v of Eq. cvleapfrog (the paper uses 1e-2); 0 disables the check,
                             the corrector re-runs and the CFL multiplier */
    double lambda_stiff;  /* lambda_stiff of the CFL multiplier relaxation; 1 */
} sph_params;

/* Particle state.  Arrays: float64[n] (id: uint32[n]).  Inputs/outputs per function below. */
typedef struct {
    int64_t n;
    double mass;
    double *x, *y, *z;        /* positions */
    double *vx, *vy, *vz;     /* velocities */
    double *u;                /* specific internal energy */
    double *h;                /* smoothing length */
    double *ax, *ay, *az;     /* acceleration dv/dt */
    double *du;               /* du/dt */
    double *rho, *omega;      /* density rho(h) and grad-h term Omega (outputs of density) */
    double *vsig;             /* signal speed v_sig^dt (output of forces) */
    uint32_t *id;             /* original particle index (permuted with the particles) */
    double *alpha;            /* per-particle alpha_AV (in/out, permuted with the particles) when
                                 params.av_switch = 1; NULL otherwise */
} sph_state;

/* Host view of the tree for sph_export_tree.  The caller allocates every non-NULL array with the
 * sizes returned by sph_tree_sizes: n particles, L leaves, L-1 internal nodes, 2L-1 nodes.  Node c
 * < L-1 is internal node c; node L-1+j is leaf j (App. C tree traversal numbering). */
typedef struct {
    uint64_t *mu;          /* [n]   sorted Morton codes (63-bit, 21 bits per axis, x most significant) */
    uint32_t *perm;        /* [n]   sort permutation epsilon of the last build (index before the build) */
    int64_t *leaf_first;   /* [L+1] id_i of Fig. mortonlistbuild: first sorted particle of leaf i; [L] = n */
    uint64_t *mu_leaf;     /* [L]   leaf Morton codes */
    int32_t *lchild, *rchild;       /* [L-1] Table arrays_fig_karras */
    uint8_t *lflag, *rflag;         /* [L-1] 1 = child is a leaf */
    int32_t *endrange;              /* [L-1] */
    double *bmin, *bmax;            /* [3*(2L-1)] tight per-node box, node-major (x,y,z) */
    double *hmax;                   /* [2L-1] largest h in the node */
    int64_t *group_start;  /* [G+1] first particle of each neighbour-search group, [G] = n, with
                            * G = sph_stats.n_groups: the largest nodes holding at most 32 particles
                            * of one box (a leaf of more than 32 is cut into runs of 32) */
} sph_tree_view;

/* Per-call statistics (host copy, filled by the library after each stage). */
typedef struct {
    int64_t n, n_leaves, n_groups, n_pairs, cache_slots;
    int64_t cand_chunks;     /* 32-candidate chunks tested by stage 2 of the last cache build */
    int density_iters_max;   /* largest per-particle Newton count in the last density call */
    int outer_passes;        /* cache builds in the last sph_step (1 = no restart) */
    int n_red;
    double dt_next;
    double dv_ratio;         /* max |dv_i| / sqrt(<|v|^2>) of the last corrector (Eq. deltavi) */
    int64_t kernel_launches; /* kernels launched by this context since sph_create */
    int64_t density_pair_evals; /* neighbour evaluations of the last density call (all Newton passes) */
    int64_t density_inrange; /* of those, evaluations with r < 2 h_a */
    int64_t force_pairs;     /* pairs inside 2 max(h_a, h_b) in the last force call */
    double stage_ms[8];      /* with sph_set_timing(ctx, 1): accumulated device time per stage since the
                                last sph_reset_timing: predictor, tree, neighbours, density, force
                                preparation, force loop, corrector, shock switch */
    double cfl_multiplier;   /* lambda_CFL after the last sph_step (1 while eps_v = 0) */
    int corrector_passes;    /* corrector passes of the last sph_step */
    int64_t graph_replays;   /* sph_step calls replayed as a captured graph (sph_set_graph) */
    int64_t graph_captures;  /* graphs captured */
    int64_t graph_fallbacks; /* replays finished stage by stage (a capacity grew or h left the cache) */
} sph_stats;

/* Launch shapes of the pair kernels and the tree reduction level, chosen by sph_autotune or set by
 * the caller (defaults: 128, 128, 128, 4, p->reduction_level).  None of them changes a result: the
 * neighbour lists and every per-particle sum are the same for any choice (the cache build keeps the
 * FP64 set and orders each list by particle index). */
typedef struct {
    int density_block;    /* threads per block of the density kernel: 64, 128 or 256 */
    int forces_block;     /* threads per block of the force kernels: 64, 128 or 256 */
    int walk_block;       /* threads per block of the stage-1 tree walk: 64, 128 or 256 */
    int stage2_warps;     /* warps (groups in flight) per block of the stage-2 kernel: 1 .. 8 */
    int reduction_level;  /* n_red of App. C (copied into the context's parameters) */
} sph_launch;

/* Fill *p with the paper's defaults and a periodic unit box.  Never fails. */
void sph_default_params(sph_params *p);

/* Create a context for up to n_cap particles on the current CUDA device.  neigh_cap: initial
 * capacity of the neighbour cache in entries (0: 96 * n_cap); it grows on demand outside graph
 * capture.  stream: a cudaStream_t (NULL = the legacy default stream).  On success *out owns all
 * scratch memory. Errors: INVALID_ARG, OOM, CUDA. */
int sph_create(const sph_params *p, int64_t n_cap, int64_t neigh_cap, void *stream, sph_ctx **out);

/* Batched ensemble of independent periodic boxes in one context (the ensemble workload of the
 * benchmark; the paper runs one box per patch set, this packs many small ones so that every stage is
 * one launch for all boxes).  Box b owns particles box_offsets[b] .. box_offsets[b+1]-1 of every
 * state array (host int64[n_boxes+1], box_offsets[0] = 0); all boxes share the geometry and solver
 * parameters of *p except the particle mass (host double[n_boxes], equal masses within a box) and
 * the adiabatic index (host double[n_boxes], NULL: p->gamma).  Every entry point then works on all
 * boxes at once: state->n must equal box_offsets[n_boxes] and state->mass is ignored; sph_build_tree
 * reorders particles only inside their box; pairs never cross boxes; sph_step with dt > 0 advances
 * every box by dt, with dt <= 0 each box by its own CFL step (sph_batch_dt), and reports the
 * smallest as dt_used / dt_next.  The Morton codes carry the box index in their top bits and
 * (63 - bits(n_boxes))/3 bits per axis.  Errors: INVALID_ARG (n_boxes outside [1, 4096], offsets not
 * starting at 0 or decreasing, non-positive mass, gamma <= 1), OOM, CUDA. */
int sph_batch_create(const sph_params *p, int n_boxes, const int64_t *box_offsets, const double *box_mass,
                     const double *box_gamma, int64_t neigh_cap, void *stream, sph_ctx **out);

/* CFL time step of each box from the last force evaluation of a batch context (host double[n_boxes]). */
int sph_batch_dt(sph_ctx *ctx, double *dt_per_box);

/* Free every buffer of the context (synchronises its stream).  NULL is accepted. */
int sph_destroy(sph_ctx *ctx);

/* Replace the solver parameters (same capacity).  Invalidates the tree and cache. */
int sph_set_params(sph_ctx *ctx, const sph_params *p);

/* A1-A6 (App. B-C): Morton codes of the positions, stable radix sort by code, reorder of every
 * non-NULL state array (and id) into Morton order, duplicate mask + reduction_level reduction
 * passes (Alg. mortonmask), compaction into leaves, Karras radix tree (Table arrays_fig_karras),
 * bottom-up tight box and h_max of every node.  Input: positions, h.  Output: state reordered;
 * the tree is kept in the context.  Errors: INVALID_ARG (n > n_cap), NONFINITE, TIMEOUT, CUDA. */
int sph_build_tree(sph_ctx *ctx, sph_state *s);

/* A7 (App. C two-stage neighbour cache, App. D criteria): stage 1 walks the tree once per group (the
 * largest tree nodes of at most 32 particles of one box, sph_tree_view.group_start), keeping every
 * cell whose box lies within R_kern*cache_tol*max(h_max) of the group's box; stage 2 keeps, for
 * every particle a, each b != a with |r_ab|^2 < (R_kern*cache_tol*max(h_a,h_b))^2 (nearest periodic
 * image, FP64 decision), R_kern = 2 for M4.  h = state->h is recorded as h^n.  *n_pairs (may be
 * NULL) receives the number of cached pairs.  Requires sph_build_tree.  Errors: ORDER, CAPACITY,
 * OOM, CUDA. */
int sph_find_neighbours(sph_ctx *ctx, const sph_state *s, int64_t *n_pairs);

/* A8 (App. F): per particle, Newton-Raphson on rho_sum(h) - m (hfact/h)^3 over the cached
 * neighbours, step clamped to [h/lambda, h*lambda], until |dh|/h^n < h_tol; then rho = rho(h)
 * (Eq. rhoh) and Omega (Eq. sphomega) at the final h.  Input: positions, h.  Output: h, rho, omega.
 * *iters (may be NULL): largest per-particle iteration count.  If some h would exceed
 * cache_tol*h^n it is clamped there and SPH_ERR_CACHE_STALE is returned: rebuild the cache
 * (sph_find_neighbours, after sph_build_tree or not) and call again.  Errors: ORDER, CACHE_STALE,
 * H_NOT_CONVERGED, CUDA. */
int sph_compute_density_h(sph_ctx *ctx, sph_state *s, int *iters);

/* A9 (Sect. 2.1, Eqs. sphvel, sphuint): accelerations, du/dt (artificial viscosity and
 * conductivity) and v_sig^dt for every particle, from positions, v, u, h, omega.  Also stores the
 * CFL time step (App. G) in the stats.  Requires a neighbour cache built from h values with
 * h <= cache_tol*h^n.  Output: ax, ay, az, du, vsig.  Errors: ORDER, CUDA. */
int sph_compute_forces(sph_ctx *ctx, sph_state *s);

/* A0-A10 (App. G): one global kick-drift-kick step: predictor, tree build, neighbour cache,
 * density/h (rebuilding the cache while h leaves its tolerance, App. F outer loop), forces,
 * corrector, CFL.  The h iteration starts from h + dt dh/dt, with dh/dt = -h/(3 rho Omega) sum_b m
 * v_ab . grad_a W_ab(h_a) from this context's last force evaluation (clamped to a factor h_clamp);
 * without one it starts from h.  dt <= 0 uses the CFL step computed by the previous sph_compute_forces /
 * sph_step.  Requires accelerations and du of the current state (a first sph_compute_density_h +
 * sph_compute_forces on the initial state).  *dt_used / *dt_next may be NULL.  The state is
 * reordered into Morton order (see sph_build_tree).  Errors: ORDER, CACHE_STALE (more than
 * max_outer rebuilds), H_NOT_CONVERGED, CAPACITY, TIMEOUT, CUDA. */
int sph_step(sph_ctx *ctx, sph_state *s, double dt, double *dt_used, double *dt_next);

/* Same as sph_step with every pointer of *host_state in HOST memory (pinned or pageable): copies
 * the state to context-owned device buffers, runs the step, copies it back (Morton order).  Used
 * for end-to-end timing.  Errors: as sph_step. */
int sph_step_host(sph_ctx *ctx, sph_state *host_state, double dt, double *dt_used, double *dt_next);

/* Sizes of the current tree: *n particles, *n_leaves L. */
int sph_tree_sizes(sph_ctx *ctx, int64_t *n, int64_t *n_leaves);

/* Copy the current tree to caller-allocated host arrays (NULL entries are skipped). */
int sph_export_tree(sph_ctx *ctx, sph_tree_view *view);

/* Copy the neighbour cache as CSR to host arrays: off[n+1] (int64) and ids[n_pairs] (indices in
 * the current, Morton, order; each list in increasing index order). */
int sph_export_neighbours(sph_ctx *ctx, int64_t *off, uint32_t *ids);

/* Statistics of the last calls. */
int sph_get_stats(sph_ctx *ctx, sph_stats *st);

/* Launch shapes in use (*out) / to use from the next call on (*in).  Errors: INVALID_ARG for a
 * shape outside the ranges of sph_launch. */
int sph_get_launch(sph_ctx *ctx, sph_launch *out);
int sph_set_launch(sph_ctx *ctx, const sph_launch *in);

/* Autotuner of the launch shapes (no counterpart in the paper; the paper reports the optimum
 * reduction level of its own hardware, App. C: about ten particles per leaf).  Times A1-A9 on *s
 * (device pointers, as sph_step) for each candidate: the reduction levels 1-7, then, one knob at a
 * time, the stage-2 warps per block {2, 4, 8} and the density, force and walk block sizes
 * {64, 128, 256}, two runs each with CUDA events (the faster counts), and keeps the fastest
 * combination in the context.  A1-A9 leave the physical state unchanged: the particles are
 * reordered, h is re-converged (it moves by less than h_tol * h) and a, du, rho, Omega, v_sig are
 * recomputed; velocities, u and positions are untouched.  *s should be converged (a previous
 * density + force call or sph_step).  *best (may be NULL) receives the chosen shapes, *ms_best
 * (may be NULL) the A1-A9 time with them.  Errors: as sph_step. */
int sph_autotune(sph_ctx *ctx, sph_state *s, sph_launch *best, double *ms_best);

/* Enable (1) or disable (0) per-stage CUDA-event timing.  With timing on, every stage waits for its
 * own completion, so stage boundaries serialise with the host; kernel durations are unaffected. */
int sph_set_timing(sph_ctx *ctx, int enable);

/* Zero the accumulated stage times. */
int sph_reset_timing(sph_ctx *ctx);

/* Enable (1) or disable (0) graph replay of sph_step.  When enabled, a step whose context and state
 * are unchanged since the last step that ran stage by stage (same state pointers, n, parameters,
 * launch shapes and array capacities) is recorded once into a CUDA graph (captured on a private
 * stream) and then replayed on the context stream: every stage is one launch with its grid sized by
 * the capacity of the leaf- and group-indexed arrays, the leaf, group, candidate-chunk and cache
 * counts stay on the device, and the host reads the step's scalars back once, at the end.  A stage
 * whose input an earlier stage left incomplete (a count above its capacity, a full candidate list or
 * cache, h at the cache limit) does nothing; the host then finishes that step stage by stage (the
 * arrays grow, the outer density loop runs) and the next step captures again
 * (sph_stats.graph_fallbacks).  Results are bit-identical to the stage-by-stage step.  Ignored while
 * per-stage timing is on.  Errors: INVALID_ARG (ctx NULL). */
int sph_set_graph(sph_ctx *ctx, int enable);

/* Morton codes and stable sort without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc/cudaFree -- an application whose device
 * memory is owned by another allocator (a framework's caching allocator or a fixed arena already
 * holding the free memory, where a fresh cudaMalloc fails or fragments it), or a latency-bound caller
 * that cannot accept the device synchronisation cudaFree implies.
 * Computes the same codes and permutation as sph_build_tree (A1-A2): codes_out[i] = i-th smallest
 * 63-bit Morton code of the positions in [box_lo, box_hi), perm_out[i] = its original index, ties in
 * original order.  x, y, z: DEVICE float64[n]; box_lo, box_hi: HOST double[3]; codes_out (uint64[n])
 * and perm_out (uint32[n]): DEVICE, caller-owned, must not alias the inputs.  Work is issued on
 * `stream` (a cudaStream_t, NULL = legacy default) and the call returns after it has finished.
 * Limit: n <= 262144 (SPH_ERR_CAPACITY beyond); n = 0 returns SPH_OK without touching the outputs;
 * SPH_ERR_INVALID_ARG for n < 0, NULL pointers or an empty box.  An error left pending by an earlier,
 * unrelated CUDA runtime call is cleared on entry, so SPH_ERR_CUDA always means this call failed.
 * Scratch: a fixed 4 MiB device array inside the library, one per GPU, created by the CUDA runtime
 * when the library's device code is loaded on that GPU and held until the process exits; its device
 * address is looked up on the first call made on each device, so make that first call outside any
 * stream capture.  Every call on a device shares that array and leaves its last contents there (the
 * parts that must start at zero are cleared by each call); calls whose work overlaps on the GPU
 * (other streams, other host threads) race on it and must be serialised by the caller.  Errors:
 * CAPACITY, INVALID_ARG, TIMEOUT (a bounded look-back wait ran out), CUDA. */
int sph_sort_morton_noalloc(int64_t n, const double *x, const double *y, const double *z, const double *box_lo,
                            const double *box_hi, uint64_t *codes_out, uint32_t *perm_out, void *stream);

/* Failure-detection probe (no counterpart in the paper; for tests).  Makes one of the library's
 * bounded device-side waits run out on purpose, without a fault or a hang, and reports it the way
 * a real stall would be reported.  which = 0: one radix-sort pass over two tiles of scratch keys
 * (buffers allocated and freed by the call) launched so that the first tile is never processed; the
 * second tile's decoupled look-back waits `spins` rounds for it.  which = 1: stage 2 of the current
 * neighbour cache run again as one warp that starts at the second group, whose look-back waits for
 * the first group; the cache is marked invalid afterwards (call sph_find_neighbours again); s must
 * be the state of the last cache build.  spins: rounds of the wait, 1 .. 2^20 (the library's own
 * limits are 2^22).  Returns SPH_ERR_TIMEOUT when the wait ran out as designed (the expected
 * result), SPH_OK if it did not, SPH_ERR_ORDER without a cache of at least two groups (which = 1)
 * or inside a captured step, SPH_ERR_INVALID_ARG, SPH_ERR_OOM, SPH_ERR_CUDA.  The context stays
 * usable. */
int sph_debug_wait_timeout(sph_ctx *ctx, const sph_state *s, int which, uint32_t spins);

/* Message of the last error of ctx (never NULL; "" when none). */
const char *sph_last_error(sph_ctx *ctx);

/* Static description of a status code. */
const char *sph_error_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* SPH_GB300_H */

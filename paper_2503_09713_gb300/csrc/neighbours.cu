// Neighbour cache (App. C "Two-stages neighbour cache", App. D interaction criteria).
//
// Stage 1: every group of 32 consecutive (Morton-ordered) particles walks the radix tree once with
// the group-group criterion  AABB_g  intersects  AABB_c (+) s*max(h_max,g, h_max,c),  s = R_kern*chi,
// shifting the group box by the periodic images it can reach; the surviving leaves are the group's
// candidates.  Stage 2: one warp per group, lane = particle a, tests every particle of the candidate
// leaves against  |r_ab|^2 < (s*max(h_a,h_b))^2  (App. D object-object criterion with the cache
// tolerance of App. F).  The test runs on FP32 cell-relative offsets with a +-2^-10 relative band;
// pairs inside the band are decided in FP64 exactly as the definition states, so the kept set is
// the FP64 set.  A count pass, a scan over groups and a fill pass write the cache in a
// group-interleaved layout: particle a = 32g + lane owns entries off_g + 32k + lane, k < count_a.
#include "sph_internal.cuh"

namespace sph {

struct Geo {
    double lo[3], L[3], halfL[3];
    float cell[3];   // box side / 1024 in FP32
    int periodic;
};

static Geo make_geo(const sph_params &p) {
    Geo g;
    for (int k = 0; k < 3; k++) {
        g.lo[k] = p.box_lo[k];
        g.L[k] = p.box_hi[k] - p.box_lo[k];
        g.halfL[k] = 0.5 * g.L[k];
        g.cell[k] = (float)(g.L[k] / 1024.0);
    }
    g.periodic = p.periodic;
    return g;
}

// ------------------------------------------------------------------ group boxes (warp per group)
__global__ void k_group_boxes(int64_t n, int64_t G, const double *__restrict__ x, const double *__restrict__ y,
                              const double *__restrict__ z, const double *__restrict__ h, Node *__restrict__ gbox) {
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= G) return;
    const int64_t a = g * 32 + lane;
    const bool va = a < n;
    double lo[3], hi[3];
    const double p[3] = {va ? x[a] : 0.0, va ? y[a] : 0.0, va ? z[a] : 0.0};
    for (int k = 0; k < 3; k++) {
        lo[k] = warp_min_d(va ? p[k] : INFINITY);
        hi[k] = warp_max_d(va ? p[k] : -INFINITY);
    }
    const double hm = warp_max_d(va ? h[a] : 0.0);
    if (lane == 0) {
        Node b;
        for (int k = 0; k < 3; k++) { b.lo[k] = lo[k]; b.hi[k] = hi[k]; }
        b.hmax = hm;
        b.pad = 0.0;
        gbox[g] = b;
    }
}

// ------------------------------------------------------------------ stage 1: tree walk per group
__device__ __forceinline__ void load_node_ro(const Node *nd, Node &o) {
    const double2 *p = reinterpret_cast<const double2 *>(nd);
    double2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3);
    o.lo[0] = a.x; o.lo[1] = a.y; o.lo[2] = b.x; o.hmax = b.y;
    o.hi[0] = c.x; o.hi[1] = c.y; o.hi[2] = d.x; o.pad = d.y;
}

__global__ void __launch_bounds__(128) k_walk(int64_t G, int64_t L, const Node *__restrict__ gbox,
                                             const Node *__restrict__ nodes, const int32_t *__restrict__ child,
                                             double s, Geo geo, uint32_t *__restrict__ cand,
                                             uint32_t *__restrict__ cand_cnt, int cap, uint32_t *flags) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    Node q;
    load_node_ro(&gbox[g], q);
    Node root;
    load_node_ro(&nodes[0], root);
    const double margin = 1.0 + 1e-9;
    const double rmax = s * fmax(q.hmax, root.hmax) * margin;
    // periodic images of the group box that can reach the box
    int nsh[3];
    double sh[3][3];
    for (int k = 0; k < 3; k++) {
        nsh[k] = 1;
        sh[k][0] = 0.0;
        if (geo.periodic) {
            if (q.hi[k] - geo.lo[k] + rmax >= geo.L[k]) sh[k][nsh[k]++] = -geo.L[k];
            if (q.lo[k] - geo.lo[k] - rmax <= 0.0) sh[k][nsh[k]++] = geo.L[k];
        }
    }
    uint32_t *out = cand + (size_t)g * cap;
    int count = 0;
    int32_t stack[kStackDepth];
    const int64_t nin = L - 1;
    for (int ix = 0; ix < nsh[0]; ix++)
        for (int iy = 0; iy < nsh[1]; iy++)
            for (int iz = 0; iz < nsh[2]; iz++) {
                const double qlo[3] = {q.lo[0] + sh[0][ix], q.lo[1] + sh[1][iy], q.lo[2] + sh[2][iz]};
                const double qhi[3] = {q.hi[0] + sh[0][ix], q.hi[1] + sh[1][iy], q.hi[2] + sh[2][iz]};
                int sp = 0;
                stack[sp++] = 0;
                while (sp > 0) {
                    const int32_t c = stack[--sp];
                    Node nd;
                    load_node_ro(&nodes[c], nd);
                    const double r = s * fmax(q.hmax, nd.hmax) * margin;
                    const bool hit = (qlo[0] <= nd.hi[0] + r) && (nd.lo[0] - r <= qhi[0]) &&
                                     (qlo[1] <= nd.hi[1] + r) && (nd.lo[1] - r <= qhi[1]) &&
                                     (qlo[2] <= nd.hi[2] + r) && (nd.lo[2] - r <= qhi[2]);
                    if (!hit) continue;
                    if (c >= nin) {
                        if (count < cap) out[count] = (uint32_t)(c - nin);
                        ++count;
                    } else {
                        if (sp + 2 > kStackDepth) {
                            atomicOr(flags, kErrStack);
                            sp = 0;
                            break;
                        }
                        stack[sp++] = child[2 * c + 1];
                        stack[sp++] = child[2 * c];
                    }
                }
            }
    if (count > cap) {
        atomicOr(flags, kErrCandOverflow);
        cand_cnt[g] = (uint32_t)count;
        return;
    }
    if (nsh[0] * nsh[1] * nsh[2] > 1) {
        // merge the image lists: sort ascending and drop repeats (only the nearest image is used later)
        for (int i = 1; i < count; i++) {
            const uint32_t v = out[i];
            int j = i - 1;
            while (j >= 0 && out[j] > v) {
                out[j + 1] = out[j];
                --j;
            }
            out[j + 1] = v;
        }
        int m = 0;
        for (int i = 0; i < count; i++)
            if (m == 0 || out[i] != out[m - 1]) out[m++] = out[i];
        count = m;
    }
    cand_cnt[g] = (uint32_t)count;
}

// ------------------------------------------------------------------ stage 2: per-particle filter
__device__ __forceinline__ int wrap_cell(int d, int periodic) {
    return periodic ? (((d + 512) & 1023) - 512) : d;
}

// FP32 squared distance between a and b from cell-relative coordinates (direction irrelevant).
__device__ __forceinline__ float rel_r2(const float4 A, const float4 B, const Geo &geo) {
    const uint32_t pa = __float_as_uint(A.w), pb = __float_as_uint(B.w);
    const int dix = wrap_cell((int)((pb >> 20) & 1023u) - (int)((pa >> 20) & 1023u), geo.periodic);
    const int diy = wrap_cell((int)((pb >> 10) & 1023u) - (int)((pa >> 10) & 1023u), geo.periodic);
    const int diz = wrap_cell((int)(pb & 1023u) - (int)(pa & 1023u), geo.periodic);
    const float dx = fmaf((float)dix, geo.cell[0], B.x - A.x);
    const float dy = fmaf((float)diy, geo.cell[1], B.y - A.y);
    const float dz = fmaf((float)diz, geo.cell[2], B.z - A.z);
    return dx * dx + dy * dy + dz * dz;
}

// The definition, in FP64 and in the order of the oracle: r^2 = (dx*dx + dy*dy) + dz*dz < (s*max h)^2.
__device__ __forceinline__ bool exact_pair(int64_t a, int64_t b, const double *__restrict__ x,
                                           const double *__restrict__ y, const double *__restrict__ z,
                                           const double *__restrict__ h, double s, const Geo &geo) {
    const double dx = min_image(x[b] - x[a], geo.L[0], geo.halfL[0], geo.periodic);
    const double dy = min_image(y[b] - y[a], geo.L[1], geo.halfL[1], geo.periodic);
    const double dz = min_image(z[b] - z[a], geo.L[2], geo.halfL[2], geo.periodic);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double ha = h[a], hb = h[b];
    const double hm = ha > hb ? ha : hb;
    const double rad = __dmul_rn(s, hm);
    return r2 < __dmul_rn(rad, rad);
}

constexpr int kS2Warps = 4;
constexpr float kBand = 1.0f / 1024.0f;

template <bool kFill>
__global__ void __launch_bounds__(kS2Warps * 32) k_stage2(
    int64_t n, int64_t G, const int64_t *__restrict__ leaf_first, const uint32_t *__restrict__ cand,
    const uint32_t *__restrict__ cand_cnt, int cap, const float4 *__restrict__ rel, const float *__restrict__ h32,
    const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
    const double *__restrict__ h, double s, Geo geo, uint32_t *__restrict__ nb_cnt, int64_t *__restrict__ grp_slots,
    const int64_t *__restrict__ grp_off, uint32_t *__restrict__ nb_ids, DevScalars *sc) {
    __shared__ float4 s_rel[kS2Warps][32];
    __shared__ float s_h[kS2Warps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * kS2Warps + warp;
    if (g >= G) return;
    const int64_t a = g * 32 + lane;
    const bool va = a < n;
    const float4 A = va ? rel[a] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float hA = va ? h32[a] : 0.f;
    const float s32 = (float)s;
    const uint32_t *cl = cand + (size_t)g * cap;
    const int ncand = (int)min(cand_cnt[g], (uint32_t)cap);
    uint32_t cnt = 0;
    const int64_t off = kFill ? grp_off[g] + lane : 0;
    const uint32_t slots = kFill ? (uint32_t)((grp_off[g + 1] - grp_off[g]) / 32) : 0u;
    int ci = 0;
    while (ci < ncand) {
        uint32_t j = cl[ci++];
        const int64_t s0 = leaf_first[j];
        int64_t e0 = leaf_first[j + 1];
        while (ci < ncand && cl[ci] == j + 1) {
            ++j;
            e0 = leaf_first[j + 1];
            ++ci;
        }
        for (int64_t base = s0; base < e0; base += 32) {
            const int64_t b = base + lane;
            if (b < e0) {
                s_rel[warp][lane] = rel[b];
                s_h[warp][lane] = h32[b];
            }
            __syncwarp();
            const int m = (e0 - base) < 32 ? (int)(e0 - base) : 32;
            if (va) {
                for (int jj = 0; jj < m; jj++) {
                    const int64_t bi = base + jj;
                    if (bi == a) continue;
                    const float4 B = s_rel[warp][jj];
                    const float hm = fmaxf(hA, s_h[warp][jj]);
                    const float t = s32 * hm;
                    const float thr = t * t;
                    const float r2 = rel_r2(A, B, geo);
                    bool in;
                    if (r2 < thr * (1.0f - kBand)) in = true;
                    else if (r2 > thr * (1.0f + kBand)) in = false;
                    else in = exact_pair(a, bi, x, y, z, h, s, geo);
                    if (in) {
                        if (kFill && cnt < slots) nb_ids[off + (int64_t)cnt * 32] = (uint32_t)bi;
                        ++cnt;
                    }
                }
            }
            __syncwarp();
        }
    }
    if (!kFill) {
        if (va) nb_cnt[a] = cnt;
        uint32_t mx = cnt, sum = cnt;
        for (int o = 16; o > 0; o >>= 1) {
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
        }
        if (lane == 0) {
            grp_slots[g] = (int64_t)mx * 32;
            atomicAdd((unsigned long long *)&sc->n_pairs, (unsigned long long)sum);
        }
    }
}

__global__ void k_h32(int64_t n, const double *__restrict__ h, float *__restrict__ h32, double *__restrict__ hb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = h[i];
    h32[i] = (float)v;
    hb[i] = v;
}

int neighbours_build(sph_ctx *c, const sph_state *s) {
    if (!c->tree_valid) return fail(c, SPH_ERR_ORDER, "sph_find_neighbours before sph_build_tree");
    const int64_t n = s->n;
    const int64_t G = (n + 31) / 32;
    const int64_t L = c->n_leaves;
    const Geo geo = make_geo(c->p);
    const double sc = 2.0 * c->p.cache_tol;   // R_kern * chi
    c->cache_valid = false;
    c->n_groups = G;

    k_h32<<<grid_for(n, 256), 256, 0, c->stream>>>(n, s->h, c->h32, c->h_base);
    SPH_LAUNCH_CHECK(c, "k_h32");
    k_group_boxes<<<grid_for(G * 32, 128), 128, 0, c->stream>>>(n, G, s->x, s->y, s->z, s->h, c->gbox);
    SPH_LAUNCH_CHECK(c, "k_group_boxes");

    for (int attempt = 0;; attempt++) {
        SPH_CUDA(c, cudaMemsetAsync(&c->dscal->flags, 0, sizeof(uint32_t), c->stream));
        k_walk<<<grid_for(G, 128), 128, 0, c->stream>>>(G, L, c->gbox, c->nodes, c->child, sc, geo, c->cand,
                                                        c->cand_cnt, c->cand_cap, &c->dscal->flags);
        SPH_LAUNCH_CHECK(c, "k_walk");
        SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->flags, &c->dscal->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                    c->stream));
        SPH_CUDA(c, cudaStreamSynchronize(c->stream));
        const uint32_t fl = c->hscal->flags;
        if (fl & kErrStack) return fail(c, SPH_ERR_CAPACITY, "tree walk stack overflow");
        if (!(fl & kErrCandOverflow)) break;
        if (attempt >= 6) return fail(c, SPH_ERR_CAPACITY, "candidate leaf list overflow (cap %d)", c->cand_cap);
        // grow the candidate capacity (x2) and retry
        const int newcap = c->cand_cap * 2;
        uint32_t *nc = nullptr;
        if (cudaMalloc(&nc, (size_t)G * newcap * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, SPH_ERR_OOM, "candidate list of %lld x %d", (long long)G, newcap);
        }
        SPH_CUDA(c, cudaFree(c->cand));
        c->cand = nc;
        c->cand_cap = newcap;
    }

    SPH_CUDA(c, cudaMemsetAsync(&c->dscal->n_pairs, 0, sizeof(int64_t), c->stream));
    const unsigned blocks = grid_for(G, kS2Warps);
    k_stage2<false><<<blocks, kS2Warps * 32, 0, c->stream>>>(n, G, c->leaf_first, c->cand, c->cand_cnt, c->cand_cap,
                                                             c->rel, c->h32, s->x, s->y, s->z, s->h, sc, geo,
                                                             c->nb_cnt, c->grp_slots, nullptr, nullptr, c->dscal);
    SPH_LAUNCH_CHECK(c, "k_stage2<count>");
    int r = exclusive_scan_i64(c, c->grp_slots, c->grp_off, G);
    if (r) return r;
    SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->total_slots, &c->grp_off[G], sizeof(int64_t), cudaMemcpyDeviceToHost,
                                c->stream));
    SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->n_pairs, &c->dscal->n_pairs, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                c->stream));
    SPH_CUDA(c, cudaStreamSynchronize(c->stream));
    const int64_t total = c->hscal->total_slots;
    if (total > c->nb_cap) {
        const int64_t newcap = total + total / 4 + 1024;
        SPH_CUDA(c, cudaFree(c->nb_ids));
        c->nb_ids = nullptr;
        if (cudaMalloc(&c->nb_ids, (size_t)newcap * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            c->nb_cap = 0;
            return fail(c, SPH_ERR_OOM, "neighbour cache of %lld entries", (long long)newcap);
        }
        c->nb_cap = newcap;
    }
    k_stage2<true><<<blocks, kS2Warps * 32, 0, c->stream>>>(n, G, c->leaf_first, c->cand, c->cand_cnt, c->cand_cap,
                                                            c->rel, c->h32, s->x, s->y, s->z, s->h, sc, geo,
                                                            nullptr, nullptr, c->grp_off, c->nb_ids, c->dscal);
    SPH_LAUNCH_CHECK(c, "k_stage2<fill>");
    c->total_slots = total;
    c->n_pairs = c->hscal->n_pairs;
    c->stats.n_pairs = c->n_pairs;
    c->stats.cache_slots = total;
    c->stats.n_groups = G;
    c->cache_valid = true;
    return SPH_OK;
}

}  // namespace sph

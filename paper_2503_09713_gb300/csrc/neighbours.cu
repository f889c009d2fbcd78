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

// Candidates are stored as particle-index ranges [x, y): consecutive leaves found by the walk are
// merged into one range (leaves are contiguous runs of the Morton order).
__device__ __forceinline__ void push_leaf(uint2 *out, int cap, int &count, uint32_t first, uint32_t last) {
    if (count > 0 && count <= cap && out[count - 1].y == first) {
        out[count - 1].y = last;
        return;
    }
    if (count < cap) out[count] = make_uint2(first, last);
    ++count;
}

__global__ void __launch_bounds__(128) k_walk(int64_t G, int64_t L, const Node *__restrict__ gbox,
                                             const Node *__restrict__ nodes, const int32_t *__restrict__ child,
                                             const int64_t *__restrict__ leaf_first, double s, Geo geo,
                                             uint2 *__restrict__ cand, uint32_t *__restrict__ cand_cnt, int cap,
                                             uint32_t *flags) {
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
    uint2 *out = cand + (size_t)g * cap;
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
                        const int64_t j = c - nin;
                        push_leaf(out, cap, count, (uint32_t)leaf_first[j], (uint32_t)leaf_first[j + 1]);
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
        // several images: sort the ranges by start and merge overlapping or touching ones, so every
        // particle appears once (the nearest image is chosen later)
        for (int i = 1; i < count; i++) {
            const uint2 v = out[i];
            int j = i - 1;
            while (j >= 0 && out[j].x > v.x) {
                out[j + 1] = out[j];
                --j;
            }
            out[j + 1] = v;
        }
        int m = 0;
        for (int i = 0; i < count; i++) {
            if (m > 0 && out[i].x <= out[m - 1].y) {
                out[m - 1].y = max(out[m - 1].y, out[i].y);
            } else {
                out[m++] = out[i];
            }
        }
        count = m;
    }
    cand_cnt[g] = (uint32_t)count;
}

// ------------------------------------------------------------------ stage 2: per-particle filter
__device__ __forceinline__ int wrap_cell(int d, int periodic) {
    return periodic ? (((d + 512) & 1023) - 512) : d;
}

// Cell index components of a packed relative coordinate.
__device__ __forceinline__ void unpack_cell(const float4 P, int &cx, int &cy, int &cz) {
    const uint32_t p = __float_as_uint(P.w);
    cx = (int)((p >> 20) & 1023u);
    cy = (int)((p >> 10) & 1023u);
    cz = (int)(p & 1023u);
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
constexpr float kBandLo = 1.0f - 1.0f / 1024.0f;
constexpr float kBandHi = 1.0f + 1.0f / 1024.0f;

// One warp per group.  Every particle (the group's and the candidates') is expressed in FP32
// relative to the cell of the group's first particle, with the periodic wrap done once per
// particle on the integer cell index; a test is then three differences, r^2 and one compare.
// A true neighbour b of a group particle a lies within ext + s*h_max of that cell (ext: group box
// extent, h_max: largest h in the tree), so its wrapped coordinate is its nearest image whenever
// ext + s*h_max is below half a box; the kernel asks for a quarter box (checked per group,
// warp-uniform) and otherwise wraps every separation on its own.
template <bool kFill>
__global__ void __launch_bounds__(kS2Warps * 32) k_stage2(
    int64_t n, int64_t G, const uint2 *__restrict__ cand, const uint32_t *__restrict__ cand_cnt, int cap,
    const Node *__restrict__ gbox, const Node *__restrict__ nodes, const float4 *__restrict__ rel,
    const float *__restrict__ h32,
    const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
    const double *__restrict__ h, double s, float quarter_box, Geo geo, uint32_t *__restrict__ nb_cnt,
    int64_t *__restrict__ grp_slots, const int64_t *__restrict__ grp_off, uint32_t *__restrict__ nb_ids,
    DevScalars *sc) {
    __shared__ float4 s_pos[kS2Warps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * kS2Warps + warp;
    if (g >= G) return;
    const int64_t a = g * 32 + lane;
    const bool va = a < n;
    const float s32 = (float)s;
    const float4 Araw = rel[va ? a : g * 32];
    int rcx, rcy, rcz;
    unpack_cell(rel[g * 32], rcx, rcy, rcz);
    // group-relative FP32 coordinates of a particle from its packed cell and offset
    auto grel = [&](const float4 P, float &px, float &py, float &pz) {
        int cx, cy, cz;
        unpack_cell(P, cx, cy, cz);
        px = fmaf((float)wrap_cell(cx - rcx, geo.periodic), geo.cell[0], P.x);
        py = fmaf((float)wrap_cell(cy - rcy, geo.periodic), geo.cell[1], P.y);
        pz = fmaf((float)wrap_cell(cz - rcz, geo.periodic), geo.cell[2], P.z);
    };
    float ax, ay, az;
    grel(Araw, ax, ay, az);
    const float hA = va ? h32[a] : 0.f;
    const float tA = (s32 * hA) * (s32 * hA);
    const Node q = gbox[g];
    const double hroot = nodes[0].hmax;
    const float ext = (float)fmax(fmax(q.hi[0] - q.lo[0], q.hi[1] - q.lo[1]), q.hi[2] - q.lo[2]);
    const bool compact = ext + (float)(s * hroot) < quarter_box;   // warp-uniform
    const uint2 *cl = cand + (size_t)g * cap;
    const int ncand = (int)min(cand_cnt[g], (uint32_t)cap);
    uint32_t cnt = 0;
    const int64_t off = kFill ? grp_off[g] + lane : 0;
    const uint32_t slots = kFill ? (uint32_t)((grp_off[g + 1] - grp_off[g]) / 32) : 0u;
    for (int ci = 0; ci < ncand; ci++) {
        const uint2 rg = cl[ci];
        for (int64_t base = rg.x; base < rg.y; base += 32) {
            const int64_t b = base + lane;
            if (b < rg.y) {
                const float4 P = rel[b];
                const float hb = h32[b];
                float px, py, pz;
                if (compact) grel(P, px, py, pz);
                else { px = P.x; py = P.y; pz = P.z; }
                s_pos[warp][lane] = make_float4(px, py, pz, compact ? (s32 * hb) * (s32 * hb) : P.w);
            }
            __syncwarp();
            const int m = (rg.y - base) < 32 ? (int)(rg.y - base) : 32;
            if (va) {
                for (int jj = 0; jj < m; jj++) {
                    const float4 B = s_pos[warp][jj];
                    float r2, thr;
                    if (compact) {
                        const float dx = B.x - ax, dy = B.y - ay, dz = B.z - az;
                        r2 = dx * dx + dy * dy + dz * dz;
                        thr = fmaxf(tA, B.w);
                    } else {
                        const int64_t bj = base + jj;
                        int ca[3], cb[3];
                        unpack_cell(Araw, ca[0], ca[1], ca[2]);
                        unpack_cell(B, cb[0], cb[1], cb[2]);
                        const float dx = fmaf((float)wrap_cell(cb[0] - ca[0], geo.periodic), geo.cell[0], B.x - Araw.x);
                        const float dy = fmaf((float)wrap_cell(cb[1] - ca[1], geo.periodic), geo.cell[1], B.y - Araw.y);
                        const float dz = fmaf((float)wrap_cell(cb[2] - ca[2], geo.periodic), geo.cell[2], B.z - Araw.z);
                        r2 = dx * dx + dy * dy + dz * dz;
                        const float hm = fmaxf(hA, h32[bj]);
                        thr = (s32 * hm) * (s32 * hm);
                    }
                    if (r2 > thr * kBandHi) continue;
                    const int64_t bi = base + jj;
                    if (bi == a) continue;
                    const bool in = (r2 < thr * kBandLo) || exact_pair(a, bi, x, y, z, h, s, geo);
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
        k_walk<<<grid_for(G, 128), 128, 0, c->stream>>>(G, L, c->gbox, c->nodes, c->child, c->leaf_first, sc, geo,
                                                        c->cand, c->cand_cnt, c->cand_cap, &c->dscal->flags);
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
        uint2 *nc = nullptr;
        if (cudaMalloc(&nc, (size_t)G * newcap * sizeof(uint2)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, SPH_ERR_OOM, "candidate list of %lld x %d", (long long)G, newcap);
        }
        SPH_CUDA(c, cudaFree(c->cand));
        c->cand = nc;
        c->cand_cap = newcap;
    }

    SPH_CUDA(c, cudaMemsetAsync(&c->dscal->n_pairs, 0, sizeof(int64_t), c->stream));
    const unsigned blocks = grid_for(G, kS2Warps);
    const float qbox = (float)(0.25 * fmin(fmin(geo.L[0], geo.L[1]), geo.L[2]));
    k_stage2<false><<<blocks, kS2Warps * 32, 0, c->stream>>>(n, G, c->cand, c->cand_cnt, c->cand_cap, c->gbox,
                                                             c->nodes, c->rel, c->h32, s->x, s->y, s->z, s->h, sc, qbox, geo,
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
    k_stage2<true><<<blocks, kS2Warps * 32, 0, c->stream>>>(n, G, c->cand, c->cand_cnt, c->cand_cap, c->gbox,
                                                            c->nodes, c->rel, c->h32, s->x, s->y, s->z, s->h, sc, qbox, geo,
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

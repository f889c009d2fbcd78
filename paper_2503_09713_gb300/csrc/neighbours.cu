// Neighbour cache (App. C "Two-stages neighbour cache", App. D interaction criteria).
//
// Stage 1: every group (a tree node of at most 32 particles, see Groups) walks the radix tree once with
// a group-cell criterion: dist(AABB_g, AABB_c) <= s*max(h_max,g, h_max,c),  s = R_kern*chi (the
// Euclidean distance between the boxes: the cell box grown by a ball rather than the per-axis
// expansion, so corner cells that hold no possible pair are not visited), shifting the group box by
// the periodic images it can reach.  The walk runs on FP32 copies of the boxes rounded outwards, with
// the distance rounded down and the radius up, so it keeps every cell that can hold a pair of the
// object-object criterion.  Leaves found one after the other are merged into particle ranges
// (leaves are contiguous runs of the Morton order).
// Stage 2: one warp per group, lane = particle a, tests the candidates of the ranges, 32 at a time
// from shared memory, against  |r_ab|^2 < (s*max(h_a,h_b))^2  (object-object criterion with the cache
// tolerance of App. F); candidates farther from the group's box than any threshold of the group are
// dropped first, one test per candidate.  The test runs in FP32 on coordinates relative to the
// group; pairs within a relative 2^-10 of the radius are decided in FP64 exactly as the definition
// states, so the kept set is the FP64 set.  The count pass stores, per 32-candidate chunk and lane,
// the bit mask of kept candidates; after a scan over groups the fill pass only expands those masks.
// Layout of the cache: particle a = start_g + lane of a group of size_g particles owns entries
// k = 4 r + j, k < count_a, at off_g + 4 size_g r + 4 lane + j (16-byte quads, see nb_list).
#include <cuda/atomic>
#include <cmath>

#include "physics.cuh"

namespace sph {

struct Geo {
    double lo[3], L[3], halfL[3];
    float unit[3];   // length of one step of the fixed-point positions
    float Lf[3];     // box side in FP32
    int periodic;
};

// Stage 2 tests in the frame of a group's first particle when the group's extent plus the largest
// search radius stays below this: half the smallest box side less a margin of 2/1024 of the largest
// side (far above the rounding of the FP32 sum it is compared with), rounded down.
static float frame_limit(const Geo &geo) {
    const double lmin = fmin(fmin(geo.L[0], geo.L[1]), geo.L[2]);
    const double cmax = fmax(fmax(geo.L[0], geo.L[1]), geo.L[2]) / 1024.0;
    const double v = 0.5 * lmin - 2.0 * cmax;
    float f = (float)v;
    if ((double)f > v) f = std::nextafter(f, -INFINITY);
    return f;
}

static Geo make_geo(const sph_params &p) {
    Geo g;
    for (int k = 0; k < 3; k++) {
        g.lo[k] = p.box_lo[k];
        g.L[k] = p.box_hi[k] - p.box_lo[k];
        g.halfL[k] = 0.5 * g.L[k];
        g.unit[k] = (float)(g.L[k] * (p.periodic ? 0x1p-32 : 0x1p-30));
        g.Lf[k] = (float)g.L[k];
    }
    g.periodic = p.periodic;
    return g;
}

// ------------------------------------------------------------------ group boxes (warp per group)
// FP32 box of each group, rounded outwards from the FP64 positions (min/max in FP32 on the ALU
// pipe: the walk and the stage-2 extent only need a box that contains the group).
__global__ void k_group_boxes(Groups gr, Count Gc, const double *__restrict__ x, const double *__restrict__ y,
                              const double *__restrict__ z, const double *__restrict__ h, NodeF *__restrict__ gboxf) {
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= read_count(Gc, kAbortTree)) return;
    const int64_t a = group_first(gr, g) + lane;
    const bool va = a < group_end(gr, g);
    const double p[3] = {va ? x[a] : 0.0, va ? y[a] : 0.0, va ? z[a] : 0.0};
    NodeF b;
    for (int k = 0; k < 3; k++) {
        b.lo[k] = warp_min_f(va ? __double2float_rd(p[k]) : INFINITY);
        b.hi[k] = warp_max_f(va ? __double2float_ru(p[k]) : -INFINITY);
    }
    b.hmax = warp_max_f(va ? __double2float_ru(h[a]) : 0.f);
    b.pad = 0.f;
    if (lane == 0) gboxf[g] = b;
}

// ------------------------------------------------------------------ stage 1: tree walk per group
__device__ __forceinline__ NodeF load_nodef(const NodeF *p) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
    const float4 a = __ldg(q), b = __ldg(q + 1);
    NodeF o;
    o.lo[0] = a.x; o.lo[1] = a.y; o.lo[2] = a.z; o.hmax = a.w;
    o.hi[0] = b.x; o.hi[1] = b.y; o.hi[2] = b.z; o.pad = b.w;
    return o;
}

// Candidates are particle-index ranges [x, y); a leaf that continues the previous range extends it.
__device__ __forceinline__ void push_leaf(uint2 *out, int cap, int &count, uint32_t first, uint32_t last) {
    if (count > 0 && count <= cap && out[count - 1].y == first) {
        out[count - 1].y = last;
        return;
    }
    if (count < cap) out[count] = make_uint2(first, last);
    ++count;
}

// Upward-rounded s * max(h1, h2) with a relative margin that covers the FP32 products.
__device__ __forceinline__ float walk_radius(float s, float h1, float h2) {
    return __fmul_ru(__fmul_ru(s, fmaxf(h1, h2)), 1.0f + 1.0f / 65536.0f);
}

__global__ void __launch_bounds__(256) k_walk(Groups gr, Count Gc, Count Lc, const NodeF *__restrict__ gboxf,
                                             const NodeF *__restrict__ nodesf, const WNode *__restrict__ wnodes,
                                             const int64_t *__restrict__ leaf_first,
                                             const int32_t *__restrict__ box_root, float s, Geo geo,
                                             uint2 *__restrict__ cand, uint32_t *__restrict__ cand_cnt, int cap,
                                             int64_t *__restrict__ grp_chunks, uint32_t *flags) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= read_count(Gc, kAbortTree)) return;
    const int64_t L = read_count(Lc, kAbortTree);
    const int32_t rootc = box_root[group_box_of(gr, g)];   // the walk stays inside the group's box
    const NodeF q = load_nodef(&gboxf[g]);
    const NodeF root = load_nodef(&nodesf[rootc]);
    const float rmax = walk_radius(s, q.hmax, root.hmax);
    // periodic images of the group box that can reach the box (offsets added with outward rounding)
    int nsh[3];
    float sh[3][3];
    for (int k = 0; k < 3; k++) {
        nsh[k] = 1;
        sh[k][0] = 0.f;
        if (geo.periodic) {
            const float lo = (float)geo.lo[k];
            if (__fadd_ru(__fadd_ru(q.hi[k], -lo), rmax) >= geo.Lf[k] * (1.0f - 1e-6f)) sh[k][nsh[k]++] = -geo.Lf[k];
            if (__fadd_rd(__fadd_rd(q.lo[k], -lo), -rmax) <= geo.Lf[k] * 1e-6f) sh[k][nsh[k]++] = geo.Lf[k];
        }
    }
    uint2 *out = cand + (size_t)g * cap;
    int count = 0;
    int32_t stack[kStackDepth];
    const int64_t nin = L - 1;
    for (int ix = 0; ix < nsh[0]; ix++)
        for (int iy = 0; iy < nsh[1]; iy++)
            for (int iz = 0; iz < nsh[2]; iz++) {
                const float qlo[3] = {__fadd_rd(q.lo[0], sh[0][ix]), __fadd_rd(q.lo[1], sh[1][iy]),
                                      __fadd_rd(q.lo[2], sh[2][iz])};
                const float qhi[3] = {__fadd_ru(q.hi[0], sh[0][ix]), __fadd_ru(q.hi[1], sh[1][iy]),
                                      __fadd_ru(q.hi[2], sh[2][iz])};
                // Depth-first walk over hit nodes: a node's two children are loaded (one 64-byte
                // record of their boxes and ids, WNode) and tested together when the node is popped,
                // and only hits are pushed (right, then left, so leaves come out in Morton order).
                auto hits = [&](const NodeF &nd) {
                    const float r = walk_radius(s, q.hmax, nd.hmax);
                    // squared distance between the two boxes, rounded down, against r^2 rounded up
                    float d2 = 0.f;
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        const float gap = fmaxf(fmaxf(__fsub_rd(nd.lo[k], qhi[k]), __fsub_rd(qlo[k], nd.hi[k])), 0.f);
                        d2 = __fmaf_rd(gap, gap, d2);
                    }
                    return d2 <= __fmul_ru(r, r);
                };
                int sp = 0;
                if (hits(root)) stack[sp++] = rootc;
                while (sp > 0) {
                    const int32_t c = stack[--sp];
                    if (c >= nin) {
                        const int64_t j = c - nin;
                        push_leaf(out, cap, count, (uint32_t)leaf_first[j], (uint32_t)leaf_first[j + 1]);
                        continue;
                    }
                    const NodeF nl = load_nodef(&wnodes[c].l), nr = load_nodef(&wnodes[c].r);
                    const int2 ch = make_int2(__float_as_int(nl.pad), __float_as_int(nr.pad));
                    const bool hl = hits(nl), hr = hits(nr);
                    if (sp + 2 > kStackDepth) {
                        atomicOr(flags, kErrStack);
                        sp = 0;
                        break;
                    }
                    if (hr) stack[sp++] = ch.y;
                    if (hl) stack[sp++] = ch.x;
                }
            }
    if (count > cap) {
        atomicOr(flags, kErrCandOverflow);
        cand_cnt[g] = (uint32_t)count;
        grp_chunks[g] = 0;
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
    int64_t total = 0;
    for (int i = 0; i < count; i++) total += out[i].y - out[i].x;
    cand_cnt[g] = (uint32_t)count;
    grp_chunks[g] = (total + 31) / 32;   // stage 2 takes the concatenated ranges 32 at a time
}

// ------------------------------------------------------------------ stage 2: per-particle filter
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

constexpr int kS2MaxWarps = 8;   // stage-2 warps per block: 1 .. 8 (sph_launch.stage2_warps)
constexpr float kBandLo = 1.0f - 1.0f / 1024.0f;
constexpr float kBandHi = 1.0f + 1.0f / 1024.0f;
constexpr float kInvHi = 1.0f / kBandHi, kInvLo = 1.0f / kBandLo;   // the band applied to r^2 instead
constexpr float kPreHi = 1.0f + 1.0f / 512.0f;   // candidate filter: wider than the band and its rounding

constexpr unsigned long long kGrpAgg = 1ULL << 62;
constexpr unsigned long long kGrpInc = 2ULL << 62;
constexpr unsigned long long kGrpVal = (1ULL << 62) - 1;
constexpr uint32_t kGrpSpinLimit = 1u << 22;

// Stage 2 in one pass.  Groups are taken in launch order from a ticket.  For its group a warp
// (1) tests the candidates and keeps, per 32-candidate chunk and lane, the bit mask of kept
// candidates; (2) obtains the group's offset in the cache by decoupled look-back over the
// preceding groups (the group needs 32 x its largest count entries); (3) expands its masks, which
// are still in L2, into the cache.  Tests run in FP32 relative to the group's first particle: the
// int32 difference of fixed-point counts (one per particle) is the image nearest to that particle.
// A true neighbour b of a group particle lies within ext + s*h_max of it (ext: group extent, h_max:
// largest h in the box), so that image is b's nearest image from every particle of the group whenever
// ext + s*h_max stays below half a box (with a margin, see frame_limit); a candidate taken in another
// image is not a true neighbour and is never nearer than its nearest image, so it is rejected either
// way.  The condition is
// warp-uniform; a group that fails it wraps every separation on its own.  Pairs within a relative
// 2^-10 of the radius are decided in FP64 (exact_pair).
__global__ void __launch_bounds__(kS2MaxWarps * 32) k_stage2(
    Groups gr, const int32_t *__restrict__ box_root, Count Gc, const uint2 *__restrict__ cand, const uint32_t *__restrict__ cand_cnt, int cap,
    const int64_t *__restrict__ chunk_off, int64_t masks_cap, const NodeF *__restrict__ gboxf, const Node *__restrict__ nodes,
    const uint4 *__restrict__ qpos, const double *__restrict__ x,
    const double *__restrict__ y, const double *__restrict__ z, const double *__restrict__ h, double s,
    float frame_lim, Geo geo, uint32_t *__restrict__ masks, uint32_t *__restrict__ nb_cnt,
    unsigned long long *__restrict__ nb_ptr, unsigned long long *lookback, uint32_t *ticket, int64_t *__restrict__ grp_off, uint32_t *__restrict__ nb_ids,
    int64_t nb_cap, DevScalars *sc, uint32_t spin_limit) {
    // per warp: 32 candidates (group-frame position and (s h_b)^2, or the fixed-point position), and
    // h_b (wrapped path) or the chunk position of each compacted candidate (group-frame path)
    extern __shared__ float4 s2_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *s_posw = s2_smem + warp * 32;
    float *s_hb = reinterpret_cast<float *>(s2_smem + (blockDim.x >> 5) * 32) + warp * 64;
    int *s_jj = reinterpret_cast<int *>(s_hb + 32);
    // group count and the mask capacity: the same decision in every block, taken before any ticket
    const int64_t G = read_count(Gc, kAbortStage2);
    if (G == 0) return;
    if (chunk_off[G] * kChunkWords > masks_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&sc->flags, kErrCapacity);
        return;
    }
    int64_t g = 0;
    if (lane == 0) g = atomicAdd(ticket, 1u);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= G) return;
    if (g == 0 && lane == 0) sc->total_chunks = chunk_off[G];
    const int64_t first = group_first(gr, g);
    const int64_t a = first + lane;
    const int64_t gsize = group_end(gr, g) - first;
    const bool va = lane < gsize;
    const float s32 = (float)s;
    const uint4 Araw = qpos[va ? a : first];
    const uint4 F = qpos[first];
    // coordinates in the frame of the group's first particle (nearest image of each)
    auto grel = [&](const uint4 P, float &px, float &py, float &pz) {
        px = (float)(int)(P.x - F.x) * geo.unit[0];
        py = (float)(int)(P.y - F.y) * geo.unit[1];
        pz = (float)(int)(P.z - F.z) * geo.unit[2];
    };
    float ax, ay, az;
    grel(Araw, ax, ay, az);
    const float hA = va ? __uint_as_float(Araw.w) : 0.f;
    const float tA = (s32 * hA) * (s32 * hA);
    // the group's box in the same relative FP32 coordinates, and its largest h (candidate filter)
    const float glo[3] = {warp_min_f(va ? ax : INFINITY), warp_min_f(va ? ay : INFINITY),
                          warp_min_f(va ? az : INFINITY)};
    const float ghi[3] = {warp_max_f(va ? ax : -INFINITY), warp_max_f(va ? ay : -INFINITY),
                          warp_max_f(va ? az : -INFINITY)};
    const float hmax_g = warp_max_f(hA);
    const NodeF q = gboxf[g];
    const double hroot = nodes[box_root[group_box_of(gr, g)]].hmax;
    const float ext = fmaxf(fmaxf(__fsub_ru(q.hi[0], q.lo[0]), __fsub_ru(q.hi[1], q.lo[1])), __fsub_ru(q.hi[2], q.lo[2]));
    const bool compact = ext + (float)(s * hroot) < frame_lim;   // warp-uniform
    const uint2 *cl = cand + (size_t)g * cap;
    const int ncand = (int)min(cand_cnt[g], (uint32_t)cap);
    const int64_t nchunks = chunk_off[g + 1] - chunk_off[g];
    uint32_t *const gbase = masks + (size_t)chunk_off[g] * kChunkWords;
    uint32_t cnt = 0;
    // cursor over the concatenated candidate ranges (warp-uniform)
    int ci = 0;
    int64_t cur = 0, rend = 0;
    if (ncand > 0) {
        const uint2 r0 = cl[0];
        cur = r0.x;
        rend = r0.y;
    }
    // the lane's candidate of the next chunk (the next 32 of the concatenated ranges) and its record
    auto fill = [&](int64_t &bn, int &fn) {
        bn = -1;
        fn = 0;
        while (fn < 32 && ci < ncand) {
            const int take = (int)min((int64_t)(32 - fn), rend - cur);
            if (lane >= fn && lane < fn + take) bn = cur + (lane - fn);
            fn += take;
            cur += take;
            if (cur == rend && ++ci < ncand) {
                const uint2 r = cl[ci];
                cur = r.x;
                rend = r.y;
            }
        }
    };
    int64_t b_next;
    int f_next;
    fill(b_next, f_next);
    uint4 Q_next = b_next >= 0 ? qpos[b_next] : make_uint4(0u, 0u, 0u, 0u);
    // ---- (1) tests, 32 candidates of the concatenated ranges per chunk; the next chunk's records
    // are loaded while this one is tested
    for (int64_t chunk = 0; chunk < nchunks; ++chunk) {
        uint32_t *gch = gbase + (size_t)chunk * kChunkWords;   // [0, 32): masks, [32, 64): candidates
        const int64_t b = b_next;   // this lane's candidate
        const int filled = f_next;
        const uint4 Qc = Q_next;
        if (chunk + 1 < nchunks) {
            fill(b_next, f_next);
            Q_next = b_next >= 0 ? qpos[b_next] : make_uint4(0u, 0u, 0u, 0u);
        }
        // compact: group-frame position and (s h_b)^2; otherwise the fixed-point position
        float4 P = make_float4(1e30f, 1e30f, 1e30f, 0.f);
        float hb = 0.f;
        if (b >= 0) {
            const uint4 Q = Qc;
            hb = __uint_as_float(Q.w);
            if (compact) {
                float px, py, pz;
                grel(Q, px, py, pz);
                P = make_float4(px, py, pz, (s32 * hb) * (s32 * hb));
            } else {
                P = make_float4(__uint_as_float(Q.x), __uint_as_float(Q.y), __uint_as_float(Q.z), 0.f);
            }
        }
        // The group's own particles are consecutive in the (sorted, duplicate-free) candidate stream
        // and pass every filter: lane a's own slot is found from the first of them in this chunk.
        const uint32_t mg = __ballot_sync(0xffffffffu, b >= first && b < first + gsize);
        int jself = -1;
        if (mg) {
            const int j0 = __ffs(mg) - 1;
            const int64_t d = a - __shfl_sync(0xffffffffu, b, j0);
            if (va && d >= 0 && d < __popc(mg)) jself = j0 + (int)d;
        }
        uint32_t hi = 0;
        if (compact) {
            // Candidate filter (lane = candidate): drop a candidate farther from the group's box
            // than (s max(h_max,g, h_b))^2 (1 + 2^-9).  Per axis |B - A| >= the gap to the box
            // in FP32 too (rounding is monotone), the squared sums below are formed in the same
            // order as the pair test, and a kept pair has r^2 < max(t_a, t_b) (1 + 2^-10) (up to
            // one rounding of r^2), so no particle of the group would keep a dropped candidate.
            const float gx = fmaxf(fmaxf(glo[0] - P.x, P.x - ghi[0]), 0.f);
            const float gy = fmaxf(fmaxf(glo[1] - P.y, P.y - ghi[1]), 0.f);
            const float gz = fmaxf(fmaxf(glo[2] - P.z, P.z - ghi[2]), 0.f);
            const float hm = fmaxf(hmax_g, hb);
            const bool need = fmaf(gz, gz, fmaf(gy, gy, gx * gx)) <= (s32 * hm) * (s32 * hm) * kPreHi;
            const uint32_t needm = __ballot_sync(0xffffffffu, need);
            if (need) {   // compacted: kept candidate k in slot k, its index beside the masks
                const int slot = __popc(needm & ((1u << lane) - 1u));
                s_posw[slot] = P;
                s_jj[slot] = (int)b;
                gch[32 + slot] = (uint32_t)b;
            }
            __syncwarp();
            // Every lane tests the kept candidates (warp-uniform loop).  Each decision is the sign
            // of a fused difference, r^2 (1 -+ 2^-10)^-1 - T rounded once (the exact sign), moved
            // into bit k of the masks by one funnel shift: possibly inside (hi), surely inside (lc).
            const int nk = __popc(needm);
            uint32_t lc = 0;
#pragma unroll 4
            for (int k = nk - 1; k >= 0; --k) {
                const float4 B = s_posw[k];   // .w = (s h_b)^2
                const float dx = B.x - ax, dy = B.y - ay, dz = B.z - az;
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const float T = fmaxf(tA, B.w);
                hi = __funnelshift_l(__float_as_uint(fmaf(r2, kInvHi, -T)), hi, 1);
                lc = __funnelshift_l(__float_as_uint(fmaf(r2, kInvLo, -T)), lc, 1);
            }
            if (!va) hi = 0;   // lanes past the group keep nothing
            if (jself >= 0 && ((needm >> jself) & 1u))   // not its own neighbour
                hi &= ~(1u << __popc(needm & ((1u << jself) - 1u)));
            uint32_t band = hi & ~lc;   // inside the band: FP64 decides
            while (band) {
                const int k = __ffs(band) - 1;
                band &= band - 1;
                if (!exact_pair(a, s_jj[k], x, y, z, h, s, geo)) hi &= ~(1u << k);
            }
        } else {
            s_posw[lane] = P;
            s_hb[lane] = hb;
            s_jj[lane] = (int)b;
            gch[32 + lane] = (uint32_t)b;
            __syncwarp();
            uint32_t lo = 0;
            for (int jj = 0; jj < filled; jj++) {
                const float4 B = s_posw[jj];   // fixed-point counts
                const float dx = (float)(int)(__float_as_uint(B.x) - Araw.x) * geo.unit[0];
                const float dy = (float)(int)(__float_as_uint(B.y) - Araw.y) * geo.unit[1];
                const float dz = (float)(int)(__float_as_uint(B.z) - Araw.z) * geo.unit[2];
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const float hm = fmaxf(hA, s_hb[jj]);
                const float t = (s32 * hm) * (s32 * hm);
                if (r2 <= t * kBandHi) hi |= 1u << jj;
                if (r2 < t * kBandLo) lo |= 1u << jj;
            }
            if (!va) hi = lo = 0;   // lanes past the group keep nothing
            if (jself >= 0) hi &= ~(1u << jself);   // not its own neighbour
            uint32_t band = hi & ~lo;   // inside the band: FP64 decides
            while (band) {
                const int jj = __ffs(band) - 1;
                band &= band - 1;
                if (!exact_pair(a, s_jj[jj], x, y, z, h, s, geo)) hi &= ~(1u << jj);
            }
        }
        gch[lane] = hi;
        cnt += __popc(hi);
        __syncwarp();
    }
    if (va) nb_cnt[a] = cnt;
    uint32_t mx = cnt, sum = cnt;
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    const unsigned long long slots = (((unsigned long long)mx + 3ULL) & ~3ULL) * (unsigned long long)gsize;
    // ---- (2) decoupled look-back over the preceding groups (lane k reads group g-1-k)
    if (lane == 0) {
        cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> mine(lookback[g]);
        mine.store((g == 0 ? kGrpInc : kGrpAgg) | slots, cuda::memory_order_relaxed);
    }
    unsigned long long excl = 0;
    if (g > 0) {
        int64_t jb = g - 1;
        uint32_t spins = 0;
        for (;;) {
            const int64_t j = jb - lane;
            unsigned long long w = kGrpInc;   // before the first group: inclusive zero
            if (j >= 0) {
                cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> other(lookback[j]);
                w = other.load(cuda::memory_order_relaxed);
            }
            const unsigned long long fl = w & ~kGrpVal;
            const unsigned inc = __ballot_sync(0xffffffffu, fl == kGrpInc);
            const unsigned notready = __ballot_sync(0xffffffffu, fl == 0ULL);
            const unsigned need = inc ? (((inc & (0u - inc)) << 1) - 1u) : 0xffffffffu;
            if (notready & need) {
                if (++spins > spin_limit) {
                    if (lane == 0) atomicOr(&sc->flags, kErrTimeoutS2);
                    break;
                }
                __nanosleep(32);
                continue;
            }
            unsigned long long v = ((1u << lane) & need) ? (w & kGrpVal) : 0ULL;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            excl += v;
            if (inc) break;
            jb -= 32;
        }
        if (lane == 0) {
            cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> mine(lookback[g]);
            mine.store(kGrpInc | (excl + slots), cuda::memory_order_relaxed);
        }
    }
    const int64_t off_g = (int64_t)excl;
    if (va) nb_ptr[a] = pack_nb_ptr(off_g + 4 * lane, gsize);
    if (lane == 0) {
        grp_off[g] = off_g;
        if (g == G - 1) {
            grp_off[G] = off_g + (int64_t)slots;
            sc->total_slots = off_g + (int64_t)slots;
        }
        atomicAdd((unsigned long long *)&sc->n_pairs, (unsigned long long)sum);
    }
    if (off_g + (int64_t)slots > nb_cap) {   // cache too small: the host grows it and runs again
        if (lane == 0) atomicOr(&sc->flags, kErrCacheOverflow);
        return;
    }
    // ---- (3) expand the masks into the cache, one 16-byte quad per four entries
    uint32_t *dst = nb_ids + off_g + 4 * lane;
    const int64_t row = 4 * gsize;
    uint4 quad = make_uint4(0u, 0u, 0u, 0u);
    uint32_t k = 0;
    // the next chunk's mask and candidates are loaded while the current one is expanded
    uint32_t m_next = nchunks > 0 ? gbase[lane] : 0u, id_next = nchunks > 0 ? gbase[32 + lane] : 0u;
    for (int64_t chunk = 0; chunk < nchunks; ++chunk) {
        uint32_t m = m_next;
        s_jj[lane] = (int)id_next;   // the chunk's candidates (slots without a mask bit unused)
        if (chunk + 1 < nchunks) {
            const uint32_t *nxt = gbase + (size_t)(chunk + 1) * kChunkWords;
            m_next = nxt[lane];
            id_next = nxt[32 + lane];
        }
        __syncwarp();
        while (m) {
            const int jj = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t v = (uint32_t)s_jj[jj], j = k & 3u;
            quad.x = j == 0u ? v : quad.x;
            quad.y = j == 1u ? v : quad.y;
            quad.z = j == 2u ? v : quad.z;
            quad.w = v;
            if (j == 3u) *reinterpret_cast<uint4 *>(dst + (int64_t)(k >> 2) * row) = quad;
            ++k;
        }
        __syncwarp();
    }
    if (k & 3u) *reinterpret_cast<uint4 *>(dst + (int64_t)(k >> 2) * row) = quad;   // last, partial quad
}

// h^n of the cache (the FP64 copy the density iteration measures its steps against) and the FP32 h
// in the fixed-point positions' .w, which the stage-2 tests read.
__global__ void k_h_base(int64_t n, const double *__restrict__ h, uint4 *__restrict__ qpos, double *__restrict__ hb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = h[i];
    qpos[i].w = __float_as_uint((float)v);
    hb[i] = v;
}

template <typename T>
static int ensure(sph_ctx *c, T **p, int64_t &cap, int64_t need, const char *what) {
    if (need <= cap) return SPH_OK;
    ++c->gen;   // a captured step holds the old pointer
    const int64_t newcap = need + need / 4 + 1024;
    SPH_CUDA(c, cudaFree(*p));
    *p = nullptr;
    if (cudaMalloc((void **)p, (size_t)newcap * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        cap = 0;
        return fail(c, SPH_ERR_OOM, "%s of %lld entries", what, (long long)newcap);
    }
    cap = newcap;
    return SPH_OK;
}

// Failure-detection hook: stage 2 run again on the current candidates as one block of one warp
// whose group ticket starts at 1, so group 0 never publishes its look-back word and the bounded
// wait of group 1 runs out after `spins` rounds.  Group 1's tests, masks and (partial) cache rows
// stay inside the arrays sized for all groups by the last cache build; the cache is marked invalid.
int debug_stage2_timeout(sph_ctx *c, const sph_state *s, uint32_t spins) {
    if (!c->cache_valid || c->n_groups < 2) return fail(c, SPH_ERR_ORDER, "the probe needs a cache of two groups");
    const Geo geo = make_geo(c->p);
    const double sc = kernel_radius(c->p.kernel) * c->p.cache_tol;
    const float qbox = frame_limit(geo);
    const uint32_t one = 1;
    c->cache_valid = false;
    SPH_CUDA(c, cudaMemsetAsync(&c->dscal->flags, 0, sizeof(uint32_t), c->stream));
    SPH_CUDA(c, cudaMemcpyAsync(&c->dscal->s2_ticket, &one, sizeof one, cudaMemcpyHostToDevice, c->stream));
    SPH_CUDA(c, cudaMemsetAsync(c->grp_slots, 0, (size_t)c->n_groups * sizeof(int64_t), c->stream));
    k_stage2<<<1, 32, 32 * (sizeof(float4) + sizeof(float2)), c->stream>>>(
        make_groups(c), c->box_root, group_count(c), c->cand, c->cand_cnt, c->cand_cap, c->chunk_off, c->masks_cap,
        c->gboxf, c->nodes, c->qpos, s->x, s->y, s->z, s->h, sc, qbox, geo, c->masks, c->nb_cnt, c->nb_ptr,
        (unsigned long long *)c->grp_slots, &c->dscal->s2_ticket, c->grp_off, c->nb_ids, c->nb_cap, c->dscal, spins);
    SPH_LAUNCH_CHECK(c, "k_stage2 (probe)");
    SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->flags, &c->dscal->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                c->stream));
    SPH_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->hscal->flags & kErrTimeoutS2) return fail(c, SPH_ERR_TIMEOUT, "stage-2 look-back wait ran out (probe)");
    return SPH_OK;
}

int neighbours_build(sph_ctx *c, const sph_state *s) {
    if (!c->tree_valid) return fail(c, SPH_ERR_ORDER, "sph_find_neighbours before sph_build_tree");
    const int64_t n = s->n;
    const int64_t G = launch_groups(c);   // the group count, or the capacity in a captured step
    const Groups gr = make_groups(c);
    const Geo geo = make_geo(c->p);
    const double sc = kernel_radius(c->p.kernel) * c->p.cache_tol;   // R_kern * chi
    c->cache_valid = false;

    k_h_base<<<grid_for(n, 256), 256, 0, c->stream>>>(n, s->h, c->qpos, c->h_base);
    SPH_LAUNCH_CHECK(c, "k_h_base");
    k_group_boxes<<<grid_for(G * 32, 128), 128, 0, c->stream>>>(gr, group_count(c), s->x, s->y, s->z, s->h,
                                                                c->gboxf);
    SPH_LAUNCH_CHECK(c, "k_group_boxes");

    // stage 1, growing the candidate capacity while a list overflows
    for (int attempt = 0;; attempt++) {
        if (!c->capturing) SPH_CUDA(c, cudaMemsetAsync(&c->dscal->flags, 0, sizeof(uint32_t), c->stream));
        k_walk<<<grid_for(G, c->launch.walk_block), c->launch.walk_block, 0, c->stream>>>(
            gr, group_count(c), leaf_count(c), c->gboxf, c->nodesf, c->wnodes, c->leaf_first, c->box_root, (float)sc,
            geo, c->cand, c->cand_cnt, c->cand_cap, c->grp_chunks, &c->dscal->flags);
        SPH_LAUNCH_CHECK(c, "k_walk");
        int r = exclusive_scan_i64_dev(c, c->grp_chunks, c->chunk_off, &c->dscal->n_groups, G);
        if (r) return r;
        if (c->capturing) break;   // overflow is flagged on the device and the host redoes the step
        SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->flags, &c->dscal->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                    c->stream));
        SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->total_chunks, &c->chunk_off[G], sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, c->stream));
        SPH_CUDA(c, cudaStreamSynchronize(c->stream));
        const uint32_t fl = c->hscal->flags;
        if (fl & kErrStack) return fail(c, SPH_ERR_CAPACITY, "tree walk stack overflow");
        if (!(fl & kErrCandOverflow)) break;
        if (attempt >= 6) return fail(c, SPH_ERR_CAPACITY, "candidate range list overflow (cap %d)", c->cand_cap);
        const int newcap = c->cand_cap * 2;
        ++c->gen;
        uint2 *nc = nullptr;
        if (cudaMalloc(&nc, (size_t)c->g_cap * newcap * sizeof(uint2)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, SPH_ERR_OOM, "candidate list of %lld x %d", (long long)c->g_cap, newcap);
        }
        SPH_CUDA(c, cudaFree(c->cand));
        c->cand = nc;
        c->cand_cap = newcap;
    }
    const int64_t chunks = c->capturing ? 0 : c->hscal->total_chunks;
    int r = ensure(c, &c->masks, c->masks_cap, chunks * kChunkWords, "candidate masks");
    if (r) return r;

    // stage 2 in one pass; if the cache turns out too small it grows and the pass runs again
    const int s2w = c->launch.stage2_warps;
    const unsigned blocks = grid_for(G, s2w);
    const size_t s2_smem = (size_t)s2w * 32 * (sizeof(float4) + sizeof(float2));
    const float qbox = frame_limit(geo);
    int64_t total = 0;
    for (int attempt = 0;; attempt++) {
        SPH_CUDA(c, cudaMemsetAsync(&c->dscal->n_pairs, 0, sizeof(int64_t), c->stream));
        if (!c->capturing) SPH_CUDA(c, cudaMemsetAsync(&c->dscal->flags, 0, sizeof(uint32_t), c->stream));
        SPH_CUDA(c, cudaMemsetAsync(&c->dscal->s2_ticket, 0, sizeof(uint32_t), c->stream));
        SPH_CUDA(c, cudaMemsetAsync(c->grp_slots, 0, (size_t)G * sizeof(int64_t), c->stream));
        k_stage2<<<blocks, s2w * 32, s2_smem, c->stream>>>(
            gr, c->box_root, group_count(c), c->cand, c->cand_cnt, c->cand_cap, c->chunk_off, c->masks_cap, c->gboxf,
            c->nodes, c->qpos, s->x, s->y, s->z, s->h, sc, qbox, geo, c->masks, c->nb_cnt, c->nb_ptr,
            (unsigned long long *)c->grp_slots, &c->dscal->s2_ticket, c->grp_off, c->nb_ids, c->nb_cap, c->dscal,
            kGrpSpinLimit);
        SPH_LAUNCH_CHECK(c, "k_stage2");
        if (c->capturing) {   // counts and overflow stay on the device until the step is read back
            c->cache_valid = true;
            return SPH_OK;
        }
        SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->total_slots, &c->grp_off[G], sizeof(int64_t), cudaMemcpyDeviceToHost,
                                    c->stream));
        SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->n_pairs, &c->dscal->n_pairs, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                    c->stream));
        SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->flags, &c->dscal->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                    c->stream));
        SPH_CUDA(c, cudaStreamSynchronize(c->stream));
        if (c->hscal->flags & kErrTimeoutS2) return fail(c, SPH_ERR_TIMEOUT, "stage-2 look-back wait ran out");
        total = c->hscal->total_slots;
        if (!(c->hscal->flags & kErrCacheOverflow) && total <= c->nb_cap) break;
        if (attempt >= 2) return fail(c, SPH_ERR_CAPACITY, "neighbour cache does not fit");
        r = ensure(c, &c->nb_ids, c->nb_cap, total, "neighbour cache");
        if (r) return r;
    }
    c->total_slots = total;
    c->n_pairs = c->hscal->n_pairs;
    c->stats.n_pairs = c->n_pairs;
    c->stats.cache_slots = total;
    c->stats.n_groups = G;
    c->stats.cand_chunks = chunks;
    c->cache_valid = true;
    return SPH_OK;
}

}  // namespace sph

// Tree build (App. B-C): Morton codes, stable radix sort by key (onesweep, decoupled look-back),
// reorder of the particle arrays, duplicate mask + reduction passes (Alg. mortonmask), compaction
// into leaves, Karras radix tree (Table arrays_fig_karras) and bottom-up tight boxes + h_max.
#include <cuda/atomic>
#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>

#include "sph_internal.cuh"

namespace sph {

// ====================================================================================== Morton
// 21 bits per axis spread to every third bit (bit i -> bit 3i).
__device__ __forceinline__ uint64_t spread3(uint64_t v) {
    v &= 0x1fffffULL;
    v = (v | (v << 32)) & 0x1f00000000ffffULL;
    v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
    v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v << 2)) & 0x1249249249249249ULL;
    return v;
}

// min(floor(g), top) for g >= 0, 0 for g < 0 or NaN, read from the bits of g: exact, and on the
// integer pipe (FP64 floor and conversion would take the FP64 pipe, which is 1/64 of FP32 here).
__device__ __forceinline__ uint64_t floor_clamped(double g, uint64_t top) {
    const long long b = __double_as_longlong(g);
    if (b < 0) return 0;                                    // negative or -0.0
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    const uint64_t frac = (uint64_t)b & ((1ULL << 52) - 1);
    if (e < 0) return 0;                                    // [0, 1)
    if (e == 1024) return frac ? 0 : top;                   // NaN, +inf
    if (e >= 52) return top;
    const uint64_t f = (frac | (1ULL << 52)) >> (52 - e);
    return f > top ? top : f;
}

// App. B "Morton codes": remap to [0,1) by (x-lo)/(hi-lo), integer grid of 2^21 per axis,
// interleave X0 Y0 Z0 X1 ... with x most significant.  inv_span is 1/span when span is a power of
// two (then the product equals the quotient bit for bit, and one product by inv_span 2^bits equals
// the two exact scalings) and 0 otherwise (divide).
__device__ __forceinline__ uint64_t quantise(double x, double lo, double span, double inv_span, int bits = 21) {
    const double scale = (double)(1ULL << bits);   // exact power of two
    const double g = inv_span != 0.0 ? (x - lo) * (inv_span * scale) : ((x - lo) / span) * scale;
    return floor_clamped(g, (1ULL << bits) - 1);
}

struct Box3 {
    double lo[3], span[3];
    double inv_span[3];   // exact reciprocal when span is a power of two, else 0
};

// Grid scale of the box for k_morton: k = 2^bits / span on every axis when all spans are powers of
// two (an exact product, so (x - lo) k equals ((x - lo) / span) 2^bits bit for bit), else 0.
struct Quant {
    double lo[3], span[3], k[3];
    int pow2;
};

// The finiteness of a double (exponent field not all ones) and h > 0 from the bits (integer pipe).
__device__ __forceinline__ bool finite_bits(double v) {
    return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ULL) != 0x7ff0000000000000ULL;
}

// In a batch the key is (box index << 3*bits) | Morton code with `bits` bits per axis, so that the
// sort keeps each box's particles together and every box is a subtree of the radix tree.
__global__ void k_morton(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                         const double *__restrict__ z, const double *__restrict__ h, Quant b,
                         uint64_t *__restrict__ keys, uint32_t *__restrict__ vals, uint32_t *flags,
                         const uint16_t *__restrict__ box_of, int bits) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double px = x[i], py = y[i], pz = z[i], ph = h[i];
    if (!finite_bits(px) || !finite_bits(py) || !finite_bits(pz) || !finite_bits(ph) || __double_as_longlong(ph) <= 0)
        atomicOr(flags, kErrNonFinite);
    const uint64_t top = (1ULL << bits) - 1;
    uint64_t X, Y, Z;
    if (b.pow2) {
        X = floor_clamped((px - b.lo[0]) * b.k[0], top);
        Y = floor_clamped((py - b.lo[1]) * b.k[1], top);
        Z = floor_clamped((pz - b.lo[2]) * b.k[2], top);
    } else {
        const double scale = (double)(1ULL << bits);
        X = floor_clamped(((px - b.lo[0]) / b.span[0]) * scale, top);
        Y = floor_clamped(((py - b.lo[1]) / b.span[1]) * scale, top);
        Z = floor_clamped(((pz - b.lo[2]) / b.span[2]) * scale, top);
    }
    uint64_t key = (spread3(X) << 2) | (spread3(Y) << 1) | spread3(Z);
    if (box_of) key |= (uint64_t)box_of[i] << (3 * bits);
    keys[i] = key;
    vals[i] = (uint32_t)i;
}

// ====================================================================================== radix sort
// LSD radix sort of (63-bit key, u32 value) pairs, 8 passes of 8-bit digits.  One kernel per pass
// ranks a 2048-key tile (kSortTile) in shared memory (warp multi-split with match.any, stable), obtains the
// tile's global digit offsets by decoupled look-back over earlier tiles, and writes each digit run
// contiguously.
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = kSortTile / kRsThreads;
static_assert(kRsItems * kRsThreads == kSortTile, "tile = threads x keys per thread");
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarpKeys = 32 * kRsItems;
constexpr uint32_t kLbAgg = 1u << 30;
constexpr uint32_t kLbInc = 2u << 30;
constexpr uint32_t kLbMask = (1u << 30) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;

__global__ void __launch_bounds__(256) k_digit_hist(const uint64_t *__restrict__ keys, int64_t n,
                                                     uint32_t *__restrict__ hist) {
    __shared__ uint32_t sh[8 * 256];
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t k = keys[i];
#pragma unroll
        for (int p = 0; p < 8; p++) atomicAdd(&sh[p * 256 + ((k >> (8 * p)) & 255)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// In place: hist[p][d] -> exclusive prefix over d.  One block of 256 threads per pass.
__global__ void k_digit_scan(uint32_t *hist) {
    uint32_t *h = hist + blockIdx.x * 256;
    int64_t tot;
    const int64_t ex = block_exclusive_scan<256>((int64_t)h[threadIdx.x], tot);
    h[threadIdx.x] = (uint32_t)ex;
}

__global__ void __launch_bounds__(kRsThreads) k_onesweep(const uint64_t *__restrict__ kin,
                                                         const uint32_t *__restrict__ vin,
                                                         uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                         int64_t n, int shift, const uint32_t *__restrict__ digit_off,
                                                         uint32_t *lookback, uint32_t *tile_ctr, uint32_t *flags,
                                                         uint32_t spin_limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw);                 // [kRsTile]
    uint32_t *sv = reinterpret_cast<uint32_t *>(sk + kRsTile);             // [kRsTile]
    uint32_t *whist = sv + kRsTile;                                        // [kRsWarps][256]
    uint32_t *tstart = whist + kRsWarps * 256;                             // [256]
    uint32_t *gbase = tstart + 256;                                        // [256]
    uint32_t *stile = gbase + 256;                                         // [1]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kRsWarps * 256; i += kRsThreads) whist[i] = 0;
    if (tid == 0) stile[0] = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const int64_t tile = stile[0];
    const int64_t base = tile * kRsTile;
    const int64_t wbase = base + (int64_t)warp * kRsWarpKeys;

    uint64_t k[kRsItems];
    uint32_t v[kRsItems];
    uint32_t rank[kRsItems];
#pragma unroll
    for (int i = 0; i < kRsItems; i++) {
        const int64_t idx = wbase + i * 32 + lane;
        if (idx < n) {
            k[i] = kin[idx];
            v[i] = vin[idx];
        } else {
            k[i] = 0;
            v[i] = 0;
        }
    }
    uint32_t *mh = whist + warp * 256;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < kRsItems; i++) {
        const bool valid = (wbase + i * 32 + lane) < n;
        const uint32_t d = valid ? (uint32_t)((k[i] >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = 31 - __clz((int)peers);
        const uint32_t before = valid ? mh[d] : 0u;
        __syncwarp();
        if (valid && lane == leader) mh[d] = before + (uint32_t)__popc(peers);
        __syncwarp();
        rank[i] = before + (uint32_t)__popc(peers & lt);
    }
    __syncthreads();

    // per digit (thread tid = digit): exclusive prefix over warps and tile total
    const int d = tid;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; w++) {
        const uint32_t cnt = whist[w * 256 + d];
        whist[w * 256 + d] = run;
        run += cnt;
    }
    const uint32_t total = run;
    cuda::atomic_ref<uint32_t, cuda::thread_scope_device> mine(lookback[tile * 256 + d]);
    mine.store((tile == 0 ? kLbInc : kLbAgg) | total, cuda::memory_order_relaxed);

    int64_t tot_unused;
    const uint32_t ts = (uint32_t)block_exclusive_scan<kRsThreads>((int64_t)total, tot_unused);
    tstart[d] = ts;

    uint32_t excl = 0;
    if (tile > 0) {
        // look-back over the preceding tiles, kLbBatch words per round trip (tile 0 is inclusive, so
        // the walk never passes it)
        constexpr int kLbBatch = 8;
        int64_t j = tile - 1;
        uint32_t spins = 0;
        bool done = false;
        while (!done && j >= 0) {
            uint32_t w[kLbBatch];
#pragma unroll
            for (int q = 0; q < kLbBatch; q++) {
                w[q] = kLbInc;
                if (j - q >= 0) {
                    cuda::atomic_ref<uint32_t, cuda::thread_scope_device> other(lookback[(j - q) * 256 + d]);
                    w[q] = other.load(cuda::memory_order_relaxed);
                }
            }
            int q = 0;
            for (; q < kLbBatch; q++) {
                const uint32_t fl = w[q] & ~kLbMask;
                if (fl == 0u) break;   // not published yet: read again from here
                excl += w[q] & kLbMask;
                if (fl == kLbInc) {
                    done = true;
                    break;
                }
            }
            if (done) break;
            j -= q;
            if (q < kLbBatch) {
                if (++spins > spin_limit) {
                    atomicOr(flags, kErrTimeout);
                    break;
                }
                __nanosleep(32);
            }
        }
        mine.store(kLbInc | (excl + total), cuda::memory_order_relaxed);
    }
    gbase[d] = digit_off[d] + excl;
    __syncthreads();

#pragma unroll
    for (int i = 0; i < kRsItems; i++) {
        if ((wbase + i * 32 + lane) < n) {
            const uint32_t dd = (uint32_t)((k[i] >> shift) & 255u);
            const uint32_t pos = tstart[dd] + mh[dd] + rank[i];
            sk[pos] = k[i];
            sv[pos] = v[i];
        }
    }
    __syncthreads();
    const int64_t rem = n - base;
    const int tile_n = rem < kRsTile ? (int)rem : kRsTile;
    for (int j = tid; j < tile_n; j += kRsThreads) {
        const uint64_t key = sk[j];
        const uint32_t dd = (uint32_t)((key >> shift) & 255u);
        const uint32_t o = gbase[dd] + ((uint32_t)j - tstart[dd]);
        if (o < (uint64_t)n) {   // always true unless a look-back wait ran out (flagged)
            kout[o] = key;
            vout[o] = sv[j];
        }
    }
}

static size_t onesweep_smem() {
    return (size_t)kRsTile * 8 + (size_t)kRsTile * 4 + (size_t)kRsWarps * 256 * 4 + 256 * 4 * 2 + 16;
}

// k_onesweep needs more than the default 48 KiB of dynamic shared memory (opted in once per device).
static cudaError_t onesweep_opt_in(size_t sm) { return smem_opt_in<k_onesweep>(sm); }

// keys[0], vals[0] hold the input; one pass per 8-bit digit of the key_bits significant bits; the
// result is in keys[passes & 1], vals[passes & 1] (returned).
static int radix_sort(sph_ctx *c, int64_t n, int key_bits, int *out_buf) {
    const int passes = std::max(1, (key_bits + 7) / 8);
    const int64_t tiles = (n + kRsTile - 1) / kRsTile;
    SPH_CUDA(c, cudaMemsetAsync(c->digit_hist, 0, 8 * 256 * sizeof(uint32_t), c->stream));
    SPH_CUDA(c, cudaMemsetAsync(c->lookback, 0, (size_t)8 * tiles * 256 * sizeof(uint32_t), c->stream));
    SPH_CUDA(c, cudaMemsetAsync(c->tile_ctr, 0, 8 * sizeof(uint32_t), c->stream));
    unsigned hb = (unsigned)std::min<int64_t>(grid_for(n, 256), (int64_t)c->num_sms * 8);
    if (hb == 0) hb = 1;
    k_digit_hist<<<hb, 256, 0, c->stream>>>(c->keys[0], n, c->digit_hist);
    SPH_LAUNCH_CHECK(c, "k_digit_hist");
    k_digit_scan<<<8, 256, 0, c->stream>>>(c->digit_hist);
    SPH_LAUNCH_CHECK(c, "k_digit_scan");
    const size_t sm = onesweep_smem();
    SPH_CUDA(c, onesweep_opt_in(sm));
    for (int p = 0; p < passes; p++) {
        const int src = p & 1, dst = src ^ 1;
        k_onesweep<<<(unsigned)tiles, kRsThreads, sm, c->stream>>>(
            c->keys[src], c->vals[src], c->keys[dst], c->vals[dst], n, 8 * p, c->digit_hist + 256 * p,
            c->lookback + (size_t)p * tiles * 256, c->tile_ctr + p, &c->dscal->flags, kSpinLimit);
        SPH_LAUNCH_CHECK(c, "k_onesweep");
    }
    *out_buf = passes & 1;
    return SPH_OK;
}

// ====================================================================================== reorder
struct GatherArgs {
    const double *src[16];
    double *dst[16];
    int nf;
    const uint32_t *id_src;
    uint32_t *id_dst;
};

// The reorder touches only the particles whose index changes (perm[i] != i): from one step to the
// next a particle keeps its rank in Morton order unless its code passes a neighbour's, so the
// permutation is mostly the identity.  Marks, an exclusive scan and a compaction list those
// positions (the count stays on the device, at pos[n]); the gather and the copy back run over the
// list.  Pure data movement: the same bits as gathering every particle.
// Moved positions, counted per 2048-position chunk (flags from perm on the fly), then listed after
// a scan of the chunk counts; the count goes to moved_n.
constexpr int kMvThreads = 256;
constexpr int kMvItems = 8;
constexpr int kMvChunk = kMvThreads * kMvItems;

__global__ void k_moved_sums(int64_t n, const uint32_t *__restrict__ perm, int64_t *__restrict__ bsum) {
    const int64_t base = (int64_t)blockIdx.x * kMvChunk + (int64_t)threadIdx.x * kMvItems;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kMvItems; k++)
        if (base + k < n) s += perm[base + k] != (uint32_t)(base + k);
    int64_t tot;
    block_exclusive_scan<kMvThreads>(s, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_moved_list(int64_t n, const uint32_t *__restrict__ perm, const int64_t *__restrict__ boff,
                             uint32_t *__restrict__ moved, int64_t *__restrict__ moved_n) {
    const int64_t base = (int64_t)blockIdx.x * kMvChunk + (int64_t)threadIdx.x * kMvItems;
    bool f[kMvItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kMvItems; k++) {
        f[k] = base + k < n && perm[base + k] != (uint32_t)(base + k);
        s += f[k];
    }
    int64_t tot;
    int64_t pos = boff[blockIdx.x] + block_exclusive_scan<kMvThreads>(s, tot);
#pragma unroll
    for (int k = 0; k < kMvItems; k++)
        if (f[k]) moved[pos++] = (uint32_t)(base + k);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *moved_n = boff[blockIdx.x] + tot;
}

__global__ void k_gather_moved(const int64_t *__restrict__ count, const uint32_t *__restrict__ moved,
                               const uint32_t *__restrict__ perm, GatherArgs g, int64_t n) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= __ldg(count)) return;
    const uint32_t i = moved[j];
    uint32_t p = perm[i];
    if (p >= (uint64_t)n) p = 0;   // only after a flagged sort failure
    for (int f = 0; f < g.nf; f++) g.dst[f][j] = g.src[f][p];
    if (g.id_dst) g.id_dst[j] = g.id_src ? g.id_src[p] : p;
}

__global__ void k_copy_back_moved(const int64_t *__restrict__ count, const uint32_t *__restrict__ moved,
                                  GatherArgs g) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= __ldg(count)) return;
    const uint32_t i = moved[j];
    for (int f = 0; f < g.nf; f++) g.dst[f][i] = g.src[f][j];
    if (g.id_dst) g.id_dst[i] = g.id_src[j];
}

// Fixed-point positions (see QScale): per axis floor((p - lo) k) modulo 2^32; .w is written by the
// neighbour search (FP32 h).
__device__ __forceinline__ uint32_t fixed_count(double p, double lo, double k) {
    return (uint32_t)(unsigned long long)__double2ll_rd((p - lo) * k);
}

__global__ void k_qpos(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                       const double *__restrict__ z, QScale q, uint4 *__restrict__ qpos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    qpos[i] = make_uint4(fixed_count(x[i], q.lo[0], q.k[0]), fixed_count(y[i], q.lo[1], q.k[1]),
                         fixed_count(z[i], q.lo[2], q.k[2]), 0u);
}

// ====================================================================================== mask
__global__ void k_mask_init(int64_t n, const uint64_t *__restrict__ mu, uint8_t *__restrict__ xi) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    xi[i] = (i == 0) ? 1 : (mu[i] != mu[i - 1]);
}

// One reduction pass of Alg. mortonmask: code i (kept) is removed when
// delta(mu_{i-2}, mu_{i-1}) < delta(mu_{i-1}, mu_i) > delta(mu_i, mu_{i+1}) over kept codes; a
// missing neighbour gives delta = -1.  Reads the previous mask, writes a new one.
__device__ __forceinline__ int dlt(uint64_t a, uint64_t b) { return __clzll((long long)(a ^ b)); }

__global__ void k_reduce_pass(int64_t n, const uint64_t *__restrict__ mu, const uint8_t *__restrict__ in,
                              uint8_t *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!in[i]) {
        out[i] = 0;
        return;
    }
    int64_t im1 = i - 1;
    while (im1 >= 0 && !in[im1]) --im1;
    int64_t im2 = im1 - 1;
    while (im2 >= 0 && !in[im2]) --im2;
    int64_t ip1 = i + 1;
    while (ip1 < n && !in[ip1]) ++ip1;
    const uint64_t mi = mu[i];
    const int d0 = (ip1 < n) ? dlt(mi, mu[ip1]) : -1;
    const int dm1 = (im1 >= 0) ? dlt(mu[im1], mi) : -1;
    const int dm2 = (im2 >= 0) ? dlt(mu[im2], mu[im1]) : -1;
    out[i] = !(d0 < dm1 && dm2 < dm1);
}

// All reduction passes in one launch: a tile of kRdTile codes is loaded with kRdHalo codes on either
// side into shared memory, duplicates are masked, and each pass lists the kept positions of the
// extended range (block scan) and applies the rule above to every listed code, a neighbour beyond
// the extended range counting as missing.  Such decisions are exact only where the neighbours they
// read have exact states, so after each pass the range of exact states shrinks from either end by
// the kept codes next to it (two on the left, one on the right); a tile whose own codes do not all
// stay inside that range (long runs of removed codes near its ends, e.g. many particles at one
// position) raises kErrHalo and the host runs the passes one launch each instead.  Results are the
// same bits as the pass-by-pass kernels.
constexpr int kRdTile = 4096;
constexpr int kRdHalo = 512;
constexpr int kRdExt = kRdTile + 2 * kRdHalo;
constexpr int kRdThreads = 256;
constexpr int kRdPer = kRdExt / kRdThreads;
static_assert(kRdExt % kRdThreads == 0 && kRdExt <= 65535, "list positions are 16-bit");
constexpr size_t kRdSmem = (size_t)kRdExt * (sizeof(uint64_t) + sizeof(uint8_t) + sizeof(uint16_t));

__global__ void __launch_bounds__(kRdThreads) k_reduce_fused(int64_t n, const uint64_t *__restrict__ mu, int n_red,
                                                             uint8_t *__restrict__ xi, uint32_t *flags) {
    extern __shared__ __align__(16) unsigned char rd_smem[];
    uint64_t *code = reinterpret_cast<uint64_t *>(rd_smem);                      // [kRdExt]
    uint16_t *list = reinterpret_cast<uint16_t *>(code + kRdExt);                // [kRdExt]
    uint8_t *kept = reinterpret_cast<uint8_t *>(list + kRdExt);                  // [kRdExt]
    __shared__ int s_j0, s_j1;
    const int64_t t0 = (int64_t)blockIdx.x * kRdTile;
    const int64_t ext_lo = t0 > kRdHalo ? t0 - kRdHalo : 0;
    const int64_t ext_hi = t0 + kRdTile + kRdHalo < n ? t0 + kRdTile + kRdHalo : n;
    const int m = (int)(ext_hi - ext_lo);
    for (int i = threadIdx.x; i < m; i += kRdThreads) code[i] = mu[ext_lo + i];
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += kRdThreads) {
        const int64_t g = ext_lo + i;
        kept[i] = g == 0 ? 1 : (i > 0 ? code[i] != code[i - 1] : mu[g] != mu[g - 1]);
    }
    const bool lo_end = ext_lo == 0, hi_end = ext_hi == n;
    int64_t lo = ext_lo, hi = ext_hi;   // the states of positions in [lo, hi) are exact
    __syncthreads();
    for (int p = 0; p < n_red; p++) {
        const int b0 = threadIdx.x * kRdPer;
        int cnt = 0;
        for (int i = 0; i < kRdPer; i++) cnt += (b0 + i < m) ? kept[b0 + i] : 0;
        int64_t tot;
        int pos = (int)block_exclusive_scan<kRdThreads>((int64_t)cnt, tot);
        for (int i = 0; i < kRdPer; i++)
            if (b0 + i < m && kept[b0 + i]) list[pos++] = (uint16_t)(b0 + i);
        const int len = (int)tot;
        if (threadIdx.x == 0) {
            s_j0 = len;   // first listed position >= lo
            s_j1 = -1;    // last listed position < hi
        }
        __syncthreads();
        for (int j = threadIdx.x; j < len; j += kRdThreads) {
            const int64_t x = ext_lo + list[j];
            if (x >= lo && (j == 0 || ext_lo + list[j - 1] < lo)) s_j0 = j;
            if (x < hi && (j == len - 1 || ext_lo + list[j + 1] >= hi)) s_j1 = j;
            const uint64_t cx = code[list[j]];
            const int d0 = j + 1 < len ? dlt(cx, code[list[j + 1]]) : -1;
            const int dm1 = j >= 1 ? dlt(code[list[j - 1]], cx) : -1;
            const int dm2 = j >= 2 ? dlt(code[list[j - 2]], code[list[j - 1]]) : -1;
            kept[list[j]] = !(d0 < dm1 && dm2 < dm1);
        }
        __syncthreads();
        const int j0 = s_j0, j1 = s_j1;
        if (!lo_end) lo = (j0 + 2 < len) ? ext_lo + list[j0 + 2] : hi;
        if (!hi_end) hi = (j1 >= 0 && j1 < len) ? ext_lo + list[j1] : lo;
        __syncthreads();
    }
    const int64_t t1 = t0 + kRdTile < n ? t0 + kRdTile : n;
    if (t0 < lo || t1 > hi) {
        if (threadIdx.x == 0) atomicOr(flags, kErrHalo);
        return;
    }
    for (int64_t i = t0 + threadIdx.x; i < t1; i += kRdThreads) xi[i] = kept[i - ext_lo];
}

// ====================================================================================== compaction
constexpr int kCpThreads = 256;
constexpr int kCpItems = 8;
constexpr int kCpChunk = kCpThreads * kCpItems;

__global__ void k_flag_sums(int64_t n, const uint8_t *__restrict__ xi, int64_t *__restrict__ bsum) {
    const int64_t base = (int64_t)blockIdx.x * kCpChunk + (int64_t)threadIdx.x * kCpItems;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kCpItems; k++)
        if (base + k < n) s += xi[base + k];
    int64_t tot;
    block_exclusive_scan<kCpThreads>(s, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_compact(int64_t n, const uint8_t *__restrict__ xi, const uint64_t *__restrict__ mu,
                          const int64_t *__restrict__ boff, int64_t *__restrict__ leaf_first,
                          uint64_t *__restrict__ mu_leaf, DevScalars *sc) {
    const int64_t base = (int64_t)blockIdx.x * kCpChunk + (int64_t)threadIdx.x * kCpItems;
    uint8_t f[kCpItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kCpItems; k++) {
        f[k] = (base + k < n) ? xi[base + k] : 0;
        s += f[k];
    }
    int64_t tot;
    const int64_t ex = block_exclusive_scan<kCpThreads>(s, tot);
    int64_t pos = boff[blockIdx.x] + ex;
#pragma unroll
    for (int k = 0; k < kCpItems; k++) {
        if (f[k]) {
            leaf_first[pos] = base + k;
            mu_leaf[pos] = mu[base + k];
            ++pos;
        }
        if (base + k == n - 1) {
            leaf_first[pos] = n;
            sc->n_leaves = pos;
        }
    }
}

// ====================================================================================== Karras
// Karras (2012) parallel construction over L sorted distinct codes: internal node i covers the
// range between i and endrange[i]; children at the split gamma (App. B, "Karras algorithm").
__device__ __forceinline__ int kdelta(const uint64_t *mu, int64_t L, int64_t i, int64_t j) {
    if (j < 0 || j >= L) return -1;
    return __clzll((long long)(mu[i] ^ mu[j]));
}

__global__ void k_karras(Count Lc, const uint64_t *__restrict__ mu, int32_t *__restrict__ lchild,
                         int32_t *__restrict__ rchild, uint8_t *__restrict__ lflag, uint8_t *__restrict__ rflag,
                         int32_t *__restrict__ endrange, int32_t *__restrict__ child,
                         int32_t *__restrict__ node_parent, int32_t *__restrict__ leaf_parent) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t L = read_count(Lc, kAbortTree);
    if (i >= L - 1) return;
    const int dir = (kdelta(mu, L, i, i + 1) - kdelta(mu, L, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = kdelta(mu, L, i, i - dir);
    int64_t lmax = 2;
    while (kdelta(mu, L, i, i + lmax * dir) > dmin) lmax *= 2;
    int64_t l = 0;
    for (int64_t t = lmax / 2; t >= 1; t /= 2)
        if (kdelta(mu, L, i, i + (l + t) * dir) > dmin) l += t;
    const int64_t j = i + l * dir;
    const int dnode = kdelta(mu, L, i, j);
    int64_t s = 0;
    int64_t t = l;
    do {
        t = (t + 1) >> 1;
        if (kdelta(mu, L, i, i + (s + t) * dir) > dnode) s += t;
    } while (t > 1);
    const int64_t gamma = i + s * dir + (dir < 0 ? -1 : 0);
    const int64_t first = i < j ? i : j, last = i < j ? j : i;
    const bool lf = (first == gamma), rf = (last == gamma + 1);
    lchild[i] = (int32_t)gamma;
    rchild[i] = (int32_t)(gamma + 1);
    lflag[i] = lf;
    rflag[i] = rf;
    endrange[i] = (int32_t)j;
    const int64_t nin = L - 1;
    child[2 * i] = (int32_t)(lf ? nin + gamma : gamma);
    child[2 * i + 1] = (int32_t)(rf ? nin + gamma + 1 : gamma + 1);
    if (lf) leaf_parent[gamma] = (int32_t)i;
    else node_parent[gamma] = (int32_t)i;
    if (rf) leaf_parent[gamma + 1] = (int32_t)i;
    else node_parent[gamma + 1] = (int32_t)i;
    if (i == 0) node_parent[0] = -1;
}

// ====================================================================================== boxes
// Leaf boxes from their particles, then a climb: the second child to arrive at a node merges both
// children (min/max are exact, so the result does not depend on the arrival order).
__device__ __forceinline__ void load_node(const Node *nd, Node &o) {
    const double2 *p = reinterpret_cast<const double2 *>(nd);
    double2 a = __ldcg(p), b = __ldcg(p + 1), cc = __ldcg(p + 2), dd = __ldcg(p + 3);
    o.lo[0] = a.x; o.lo[1] = a.y; o.lo[2] = b.x; o.hmax = b.y;
    o.hi[0] = cc.x; o.hi[1] = cc.y; o.hi[2] = dd.x; o.pad = dd.y;
}

__global__ void k_boxes(Count Lc, const int64_t *__restrict__ leaf_first, const double *__restrict__ x,
                        const double *__restrict__ y, const double *__restrict__ z, const double *__restrict__ h,
                        const int32_t *__restrict__ child, const int32_t *__restrict__ node_parent,
                        const int32_t *__restrict__ leaf_parent, uint32_t *visit, Node *nodes, NodeF *nodesf,
                        WNode *wnodes) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t L = read_count(Lc, kAbortTree);
    if (j >= L) return;
    // min / max over the leaf's particles as signed integers that order like the doubles (exact, on
    // the integer pipe)
    long long klo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, khi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN}, kh = 0;
    for (int64_t p = leaf_first[j]; p < leaf_first[j + 1]; p++) {
        const long long r[3] = {order_key(x[p]), order_key(y[p]), order_key(z[p])};
        for (int k = 0; k < 3; k++) {
            klo[k] = min(klo[k], r[k]);
            khi[k] = max(khi[k], r[k]);
        }
        kh = max(kh, __double_as_longlong(h[p]));   // h > 0: its bits order like its value
    }
    Node b;
    for (int k = 0; k < 3; k++) {
        b.lo[k] = from_order_key(klo[k]);
        b.hi[k] = from_order_key(khi[k]);
    }
    b.hmax = __longlong_as_double(kh);
    b.pad = 0.0;
    const int64_t nin = L - 1;
    nodes[nin + j] = b;
    nodesf[nin + j] = to_float_outward(b);
    if (L == 1) return;
    int64_t node = leaf_parent[j];
    while (node >= 0) {
        __threadfence();
        const uint32_t old = atomicAdd(&visit[node], 1u);
        if (old == 0) return;
        __threadfence();
        Node l, r;
        const int32_t cl = child[2 * node], cr = child[2 * node + 1];
        load_node(&nodes[cl], l);
        load_node(&nodes[cr], r);
        NodeF fl = to_float_outward(l), fr = to_float_outward(r);   // the walk's copy of both children
        fl.pad = __int_as_float(cl);
        fr.pad = __int_as_float(cr);
        wnodes[node].l = fl;
        wnodes[node].r = fr;
        Node m;
        for (int k = 0; k < 3; k++) {
            m.lo[k] = fmin(l.lo[k], r.lo[k]);
            m.hi[k] = fmax(l.hi[k], r.hi[k]);
        }
        m.hmax = fmax(l.hmax, r.hmax);
        m.pad = 0.0;
        nodes[node] = m;
        nodesf[node] = to_float_outward(m);
        node = node_parent[node];
    }
}

// Root of each box's subtree (batch): the node whose leaves all carry the box index and whose parent
// mixes boxes; a box with one leaf has that leaf as its root.
__global__ void k_box_roots(Count Lc, const uint64_t *__restrict__ mu_leaf, const int32_t *__restrict__ endrange,
                            const int32_t *__restrict__ node_parent, const int32_t *__restrict__ leaf_parent,
                            int shift, int32_t *__restrict__ box_root) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t L = read_count(Lc, kAbortTree);
    const int64_t nin = L - 1;
    if (t >= nin + L) return;
    auto range_box = [&](int64_t node, uint64_t &b_lo, uint64_t &b_hi) {
        int64_t lo, hi;
        if (node < nin) {
            const int64_t e = endrange[node];
            lo = node < e ? node : e;
            hi = node < e ? e : node;
        } else {
            lo = hi = node - nin;
        }
        b_lo = mu_leaf[lo] >> shift;
        b_hi = mu_leaf[hi] >> shift;
    };
    uint64_t a0, a1;
    range_box(t, a0, a1);
    if (a0 != a1) return;
    const int64_t parent = (t < nin) ? node_parent[t] : (L > 1 ? leaf_parent[t - nin] : -1);
    if (parent >= 0) {
        uint64_t p0, p1;
        range_box(parent, p0, p1);
        if (p0 == p1) return;
    }
    box_root[a0] = (int32_t)t;
}

// ====================================================================================== groups
// Groups of the neighbour search: the largest nodes with at most kGroup particles inside one box.
// Node t marks the first particle of its range when it qualifies and its parent does not; a leaf
// with more than kGroup particles marks every kGroup-th particle; in a batch every box start is
// marked too.  An exclusive scan of the marks numbers the groups in particle order.
__global__ void k_group_marks(Count Lc, int64_t n, const int64_t *__restrict__ leaf_first,
                              const uint64_t *__restrict__ mu_leaf, const int32_t *__restrict__ endrange,
                              const int32_t *__restrict__ node_parent, const int32_t *__restrict__ leaf_parent,
                              int shift, const uint16_t *__restrict__ box_of, int64_t *__restrict__ marks) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t L = read_count(Lc, kAbortTree);
    const int64_t nin = L - 1;
    if (t < n && (t == 0 || (box_of && box_of[t] != box_of[t - 1]))) marks[t] = 1;
    if (t >= nin + L) return;
    auto leaves = [&](int64_t node, int64_t &lo, int64_t &hi) {
        if (node < nin) {
            const int64_t e = endrange[node];
            lo = node < e ? node : e;
            hi = node < e ? e : node;
        } else {
            lo = hi = node - nin;
        }
    };
    auto qualifies = [&](int64_t node) {
        int64_t lo, hi;
        leaves(node, lo, hi);
        return leaf_first[hi + 1] - leaf_first[lo] <= kGroup && (mu_leaf[lo] >> shift) == (mu_leaf[hi] >> shift);
    };
    int64_t lo, hi;
    leaves(t, lo, hi);
    const int64_t pf = leaf_first[lo], pl = leaf_first[hi + 1];
    if (qualifies(t)) {
        const int64_t parent = (t < nin) ? node_parent[t] : (L > 1 ? leaf_parent[t - nin] : -1);
        if (parent < 0 || !qualifies(parent)) marks[pf] = 1;
    } else if (t >= nin) {
        for (int64_t q = pf; q < pl; q += kGroup) marks[q] = 1;
    }
}

// Group table from the scanned marks; the group count pos[n] goes to sc->n_groups (checked against
// the capacity g_cap of the per-group arrays).
__global__ void k_group_table(int64_t n, const int64_t *__restrict__ marks, const int64_t *__restrict__ pos,
                              const uint16_t *__restrict__ box_of, int64_t *__restrict__ gstart,
                              uint16_t *__restrict__ group_box, int64_t g_cap, DevScalars *sc,
                              const uint32_t *abort) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n || aborted(abort, kAbortTree)) return;
    const int64_t G = pos[n];
    if (t == n - 1) sc->n_groups = G;
    if (G > g_cap) {
        if (t == 0) atomicOr(&sc->flags, kErrCapacity);
        return;
    }
    if (marks[t]) {
        const int64_t g = pos[t];
        gstart[g] = t;
        if (box_of) group_box[g] = box_of[t];
    }
    if (t == n - 1) gstart[G] = n;
}

static int make_group_table(sph_ctx *c, int64_t n) {
    const int64_t L = launch_leaves(c);
    int64_t *marks = reinterpret_cast<int64_t *>(c->gather_tmp);   // free after the reorder
    int64_t *pos = marks + c->n_cap;                                // [n + 1]
    SPH_CUDA(c, cudaMemsetAsync(marks, 0, (size_t)n * sizeof(int64_t), c->stream));
    const int64_t threads = std::max<int64_t>(n, 2 * L - 1);
    k_group_marks<<<grid_for(threads, 256), 256, 0, c->stream>>>(
        leaf_count(c), n, c->leaf_first, c->mu_leaf, c->endrange, c->node_parent, c->leaf_parent,
        3 * c->morton_bits, c->batch ? c->box_of : nullptr, marks);
    SPH_LAUNCH_CHECK(c, "k_group_marks");
    int r = exclusive_scan_i64(c, marks, pos, n);
    if (r) return r;
    if (!c->capturing) {   // a captured step keeps the group count on the device
        SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->n_groups, &pos[n], sizeof(int64_t), cudaMemcpyDeviceToHost,
                                    c->stream));
        SPH_CUDA(c, cudaStreamSynchronize(c->stream));
        const int64_t G = c->hscal->n_groups;
        if (G < 1 || G > n) return fail(c, SPH_ERR_CUDA, "bad group count %lld", (long long)G);
        r = ensure_groups(c, G);
        if (r) return r;
        c->n_groups = G;
        c->stats.n_groups = G;
    }
    k_group_table<<<grid_for(n, 256), 256, 0, c->stream>>>(n, marks, pos, c->batch ? c->box_of : nullptr,
                                                           c->gstart, c->group_box, c->g_cap, c->dscal,
                                                           abort_word(c));
    SPH_LAUNCH_CHECK(c, "k_group_table");
    return SPH_OK;
}

// A4: exclusive scan of the keep flags and compaction into leaf_first / mu_leaf (leaf count to the
// device scalars).
static int compact_leaves(sph_ctx *c, int64_t n, const uint8_t *keep) {
    const int64_t nb = (n + kCpChunk - 1) / kCpChunk;
    int64_t *bsum = c->scan_tmp;                       // [nb]
    int64_t *boff = c->scan_tmp + nb + 1;              // [nb + 1]
    int64_t *rest = c->scan_tmp + 2 * (nb + 1);
    k_flag_sums<<<(unsigned)nb, kCpThreads, 0, c->stream>>>(n, keep, bsum);
    SPH_LAUNCH_CHECK(c, "k_flag_sums");
    {
        int64_t *save = c->scan_tmp;
        c->scan_tmp = rest;
        const int r = exclusive_scan_i64(c, bsum, boff, nb);
        c->scan_tmp = save;
        if (r) return r;
    }
    k_compact<<<(unsigned)nb, kCpThreads, 0, c->stream>>>(n, keep, c->mu, boff, c->leaf_first, c->mu_leaf, c->dscal);
    SPH_LAUNCH_CHECK(c, "k_compact");
    return SPH_OK;
}

static double pow2_reciprocal(double v) {
    int e = 0;
    const double m = std::frexp(v, &e);
    return (m == 0.5) ? std::ldexp(1.0, 1 - e) : 0.0;
}

static Box3 make_box(const sph_params &p) {
    Box3 b;
    for (int k = 0; k < 3; k++) {
        b.lo[k] = p.box_lo[k];
        b.span[k] = p.box_hi[k] - p.box_lo[k];
        b.inv_span[k] = pow2_reciprocal(b.span[k]);
    }
    return b;
}

static int boxes(sph_ctx *c, const sph_state *s) {
    const int64_t L = launch_leaves(c);
    if (L > 1) SPH_CUDA(c, cudaMemsetAsync(c->visit, 0, (size_t)(L - 1) * sizeof(uint32_t), c->stream));
    k_boxes<<<grid_for(L, 128), 128, 0, c->stream>>>(leaf_count(c), c->leaf_first, s->x, s->y, s->z, s->h, c->child,
                                                     c->node_parent, c->leaf_parent, c->visit, c->nodes,
                                                     c->nodesf, c->wnodes);
    SPH_LAUNCH_CHECK(c, "k_boxes");
    return SPH_OK;
}

int tree_boxes(sph_ctx *c, const sph_state *s) { return boxes(c, s); }

// Failure-detection hook: one onesweep pass over two tiles of keys, launched as a single block
// whose tile ticket starts at 1, so tile 0 never publishes its look-back word and the block's
// bounded wait runs out after `spins` rounds.  Every access stays inside the two-tile buffers (the
// output is written only at positions below n).  Own buffers; the context's tree is not touched.
int debug_sort_timeout(sph_ctx *c, uint32_t spins) {
    const int64_t n = 2 * kRsTile;
    uint64_t *k = nullptr;
    uint32_t *v = nullptr, *words = nullptr;
    const size_t nwords = 2 * 256 + 256 + 8;   // look-back words of 2 tiles, digit offsets, counter + flags
    if (cudaMalloc(&k, (size_t)2 * n * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&v, (size_t)2 * n * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&words, nwords * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(k); cudaFree(v); cudaFree(words);
        return fail(c, SPH_ERR_OOM, "timeout probe buffers");
    }
    uint32_t *lookback = words, *digit_off = words + 512, *tile_ctr = words + 768, *flags = words + 769;
    const uint32_t one = 1;
    int r = SPH_OK;
    uint32_t fl = 0;
    if (cudaMemsetAsync(k, 0, (size_t)2 * n * sizeof(uint64_t), c->stream) != cudaSuccess ||
        cudaMemsetAsync(v, 0, (size_t)2 * n * sizeof(uint32_t), c->stream) != cudaSuccess ||
        cudaMemsetAsync(words, 0, nwords * sizeof(uint32_t), c->stream) != cudaSuccess ||
        cudaMemcpyAsync(tile_ctr, &one, sizeof one, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        onesweep_opt_in(onesweep_smem()) != cudaSuccess) {
        r = SPH_ERR_CUDA;
    } else {
        k_onesweep<<<1, kRsThreads, onesweep_smem(), c->stream>>>(k, v, k + n, v + n, n, 0, digit_off, lookback,
                                                                   tile_ctr, flags, spins);
        ++c->launches;
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&fl, flags, sizeof fl, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            r = SPH_ERR_CUDA;
    }
    cudaFree(k); cudaFree(v); cudaFree(words);
    if (r) return fail(c, r, "timeout probe launch");
    return (fl & kErrTimeout) ? fail(c, SPH_ERR_TIMEOUT, "radix sort look-back wait ran out (probe)") : SPH_OK;
}

int tree_build(sph_ctx *c, sph_state *s, bool gather_outputs) {
    const int64_t n = s->n;
    const Box3 bx = make_box(c->p);
    c->tree_valid = false;
    c->cache_valid = false;
    SPH_CUDA(c, cudaMemsetAsync(&c->dscal->flags, 0, sizeof(uint32_t), c->stream));

    // A1 Morton codes
    Quant qb;
    qb.pow2 = 1;
    for (int k = 0; k < 3; k++) {
        qb.lo[k] = bx.lo[k];
        qb.span[k] = bx.span[k];
        qb.k[k] = bx.inv_span[k] * (double)(1ULL << c->morton_bits);   // exact: powers of two
        if (bx.inv_span[k] == 0.0) qb.pow2 = 0;
    }
    k_morton<<<grid_for(n, 256), 256, 0, c->stream>>>(n, s->x, s->y, s->z, s->h, qb, c->keys[0], c->vals[0],
                                                      &c->dscal->flags, c->batch ? c->box_of : nullptr,
                                                      c->morton_bits);
    SPH_LAUNCH_CHECK(c, "k_morton");
    // A2 sort
    int buf = 0;
    int r = radix_sort(c, n, 3 * c->morton_bits + c->box_bits, &buf);
    if (r) return r;
    c->mu = c->keys[buf];
    c->perm = c->vals[buf];

    // reorder the particle arrays, kGatherBatch fields per pass through the scratch block
    const double *fields[18];
    double *fields_dst[18];
    const double *all[15] = {s->x, s->y, s->z, s->vx, s->vy, s->vz, s->u, s->h, s->ax, s->ay, s->az, s->du,
                             s->rho, s->omega, s->vsig};
    const int nf_all = gather_outputs ? 15 : 12;
    int nf = 0;
    for (int f = 0; f < nf_all; f++)
        if (all[f]) fields[nf++] = all[f];
    if (c->dhdt_valid) fields[nf++] = c->dhdt;   // dh/dt of the last force pass travels with its particles
    if (s->alpha) fields[nf++] = s->alpha;       // per-particle alpha of the shock switch
    for (int f = 0; f < nf; f++) fields_dst[f] = const_cast<double *>(fields[f]);
    // positions that change: chunk counts and their scan in the scan scratch (laid out as the leaf
    // compaction lays it out; it is free until then), the list in the free half of the value buffers,
    // the count after the chunk offsets
    static_assert(kMvChunk == kCpChunk, "the scan scratch is sized for chunks of kCpChunk");
    const int64_t mv_nb = (n + kMvChunk - 1) / kMvChunk;
    int64_t *mv_boff = c->scan_tmp + mv_nb + 1;   // [mv_nb + 1]
    {
        int64_t *bsum = c->scan_tmp;              // [mv_nb]
        k_moved_sums<<<(unsigned)mv_nb, kMvThreads, 0, c->stream>>>(n, c->perm, bsum);
        SPH_LAUNCH_CHECK(c, "k_moved_sums");
        int64_t *save = c->scan_tmp;
        c->scan_tmp = c->scan_tmp + 2 * (mv_nb + 1);
        r = exclusive_scan_i64(c, bsum, mv_boff, mv_nb);
        c->scan_tmp = save;
        if (r) return r;
        k_moved_list<<<(unsigned)mv_nb, kMvThreads, 0, c->stream>>>(n, c->perm, mv_boff, c->vals[buf ^ 1],
                                                                    mv_boff + mv_nb);
        SPH_LAUNCH_CHECK(c, "k_moved_list");
    }
    uint32_t *moved = c->vals[buf ^ 1];
    const int64_t *n_moved = mv_boff + mv_nb;
    for (int f0 = 0; f0 < nf || (f0 == 0 && s->id); f0 += kGatherBatch) {
        GatherArgs g{};
        g.nf = std::min(kGatherBatch, nf - f0);
        for (int k = 0; k < g.nf; k++) {
            g.src[k] = fields[f0 + k];
            g.dst[k] = c->gather_tmp + (size_t)k * c->n_cap;
        }
        g.id_src = s->id;
        g.id_dst = (f0 == 0 && s->id) ? c->id_tmp : nullptr;
        k_gather_moved<<<grid_for(n, 256), 256, 0, c->stream>>>(n_moved, moved, c->perm, g, n);
        SPH_LAUNCH_CHECK(c, "k_gather_moved");
        GatherArgs b{};
        b.nf = g.nf;
        for (int k = 0; k < g.nf; k++) {
            b.src[k] = g.dst[k];
            b.dst[k] = fields_dst[f0 + k];
        }
        b.id_src = g.id_dst ? c->id_tmp : nullptr;   // the id is complete after the first block
        b.id_dst = g.id_dst ? s->id : nullptr;
        k_copy_back_moved<<<grid_for(n, 256), 256, 0, c->stream>>>(n_moved, moved, b);
        SPH_LAUNCH_CHECK(c, "k_copy_back_moved");
    }
    k_qpos<<<grid_for(n, 256), 256, 0, c->stream>>>(n, s->x, s->y, s->z,
                                                    qpos_scale(c->p.box_lo, c->p.box_hi, c->p.periodic), c->qpos);
    SPH_LAUNCH_CHECK(c, "k_qpos");

    // A3 mask + reduction (all passes in one launch; pass by pass where a tile's halo is too short)
    // and A4 scan + compaction
    SPH_CUDA(c, smem_opt_in<k_reduce_fused>(kRdSmem));
    k_reduce_fused<<<(unsigned)((n + kRdTile - 1) / kRdTile), kRdThreads, kRdSmem, c->stream>>>(
        n, c->mu, c->p.reduction_level, c->mask[0], &c->dscal->flags);
    SPH_LAUNCH_CHECK(c, "k_reduce_fused");
    r = compact_leaves(c, n, c->mask[0]);
    if (r) return r;
    if (!c->capturing) {   // a captured step keeps the leaf count on the device
        SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->n_leaves, &c->dscal->n_leaves, sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, c->stream));
        SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->flags, &c->dscal->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                    c->stream));
        SPH_CUDA(c, cudaStreamSynchronize(c->stream));
        if (c->hscal->flags & kErrHalo) {   // pass by pass, double-buffered
            k_mask_init<<<grid_for(n, 256), 256, 0, c->stream>>>(n, c->mu, c->mask[0]);
            SPH_LAUNCH_CHECK(c, "k_mask_init");
            int cur = 0;
            for (int pass = 0; pass < c->p.reduction_level; pass++) {
                k_reduce_pass<<<grid_for(n, 256), 256, 0, c->stream>>>(n, c->mu, c->mask[cur], c->mask[cur ^ 1]);
                SPH_LAUNCH_CHECK(c, "k_reduce_pass");
                cur ^= 1;
            }
            if ((r = compact_leaves(c, n, c->mask[cur]))) return r;
            SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->n_leaves, &c->dscal->n_leaves, sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, c->stream));
            SPH_CUDA(c, cudaStreamSynchronize(c->stream));
            c->hscal->flags &= ~kErrHalo;
            SPH_CUDA(c, cudaMemsetAsync(&c->dscal->flags, 0, sizeof(uint32_t), c->stream));
        }
        if (c->hscal->flags & kErrNonFinite) return fail(c, SPH_ERR_NONFINITE, "non-finite position or h <= 0");
        if (c->hscal->flags & kErrTimeout) return fail(c, SPH_ERR_TIMEOUT, "radix sort look-back wait ran out");
        const int64_t L = c->hscal->n_leaves;
        if (L < 1 || L > n) return fail(c, SPH_ERR_CUDA, "bad leaf count %lld", (long long)L);
        c->n_leaves = L;
        r = ensure_tree(c, L);
        if (r) return r;
    }
    const int64_t L = launch_leaves(c);

    // A5 Karras
    if (L > 1) {
        k_karras<<<grid_for(L - 1, 256), 256, 0, c->stream>>>(leaf_count(c), c->mu_leaf, c->lchild, c->rchild, c->lflag,
                                                               c->rflag, c->endrange, c->child, c->node_parent,
                                                               c->leaf_parent);
        SPH_LAUNCH_CHECK(c, "k_karras");
    }
    // subtree root of every box
    if (c->batch) {
        k_box_roots<<<grid_for(2 * L - 1, 256), 256, 0, c->stream>>>(leaf_count(c), c->mu_leaf, c->endrange, c->node_parent,
                                                                     c->leaf_parent, 3 * c->morton_bits, c->box_root);
        SPH_LAUNCH_CHECK(c, "k_box_roots");
    }
    // groups of the neighbour search (tree nodes of at most kGroup particles)
    r = make_group_table(c, n);
    if (r) return r;
    // A6 boxes + h_max
    r = boxes(c, s);
    if (r) return r;
    c->tree_valid = true;
    c->stats.n = n;
    c->stats.n_leaves = c->n_leaves;
    c->stats.n_red = c->p.reduction_level;
    return SPH_OK;
}

}  // namespace sph

// ====================================================================================== no-alloc sort
// Morton codes + stable radix sort for callers that must not allocate device memory.  Some callers
// cannot call cudaMalloc/cudaFree: an application whose device memory is owned by another allocator
// (a framework's caching allocator or a fixed arena that already holds the free memory, so a fresh
// cudaMalloc fails or fragments it), or a latency-bound caller that cannot accept the implicit
// device synchronisation cudaFree performs.  This variant keeps all its scratch (one ping-pong side
// of the sort, histograms, look-back words, counters) in one file-scope device array of fixed size.
namespace sph {
namespace {

constexpr int64_t kNoAllocMaxN = 262144;                       // largest n accepted (64^3 particles)
constexpr int64_t kNoAllocTiles = kNoAllocMaxN / kRsTile;      // sort tiles at the largest n

struct NoAllocScratch {
    uint64_t keys[kNoAllocMaxN];                  // ping-pong side of the sort (2 MiB)
    uint32_t vals[kNoAllocMaxN];                  // (1 MiB)
    uint32_t lookback[8 * kNoAllocTiles * 256];   // decoupled look-back words (1 MiB)
    uint32_t hist[8 * 256];                       // digit histograms -> offsets
    uint32_t tile_ctr[8];
    uint32_t flags;
};

// Shared by every call on a device: it keeps the last call's contents.  4 MiB per device, held by
// every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
NoAllocScratch *g_noalloc_ptr[kNoAllocMaxDevices] = {};

__global__ void k_morton_codes(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                               const double *__restrict__ z, Box3 b, uint64_t *__restrict__ keys,
                               uint32_t *__restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t X = quantise(x[i], b.lo[0], b.span[0], b.inv_span[0]);
    const uint64_t Y = quantise(y[i], b.lo[1], b.span[1], b.inv_span[1]);
    const uint64_t Z = quantise(z[i], b.lo[2], b.span[2], b.inv_span[2]);
    keys[i] = (spread3(X) << 2) | (spread3(Y) << 1) | spread3(Z);
    vals[i] = (uint32_t)i;
}

// Device address of the scratch array on the current device.  The symbol name is only a host-side
// stand-in; the address comes from cudaGetSymbolAddress, once per device, with that device current.
int noalloc_scratch(NoAllocScratch **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return SPH_ERR_CUDA; }
    if (dev < 0 || dev >= kNoAllocMaxDevices) return SPH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SPH_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = static_cast<NoAllocScratch *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return SPH_OK;
}

}  // namespace
}  // namespace sph

extern "C" int sph_sort_morton_noalloc(int64_t n, const double *x, const double *y, const double *z,
                                       const double *box_lo, const double *box_hi, uint64_t *codes_out,
                                       uint32_t *perm_out, void *stream) {
    using namespace sph;
    if (n < 0) return SPH_ERR_INVALID_ARG;
    if (n > kNoAllocMaxN) return SPH_ERR_CAPACITY;
    if (n == 0) return SPH_OK;   // nothing to sort; the outputs are not touched
    if (!x || !y || !z || !box_lo || !box_hi || !codes_out || !perm_out) return SPH_ERR_INVALID_ARG;
    // an error left by an earlier, unrelated runtime call must not be reported as this call's
    cudaGetLastError();
    Box3 b;
    for (int k = 0; k < 3; k++) {
        if (!(box_hi[k] > box_lo[k])) return SPH_ERR_INVALID_ARG;
        b.lo[k] = box_lo[k];
        b.span[k] = box_hi[k] - box_lo[k];
        b.inv_span[k] = pow2_reciprocal(b.span[k]);
    }
    NoAllocScratch *sc = nullptr;
    int r = noalloc_scratch(&sc);
    if (r) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t tiles = (n + kRsTile - 1) / kRsTile;
    const size_t sm = onesweep_smem();
    // what must start at zero: histograms, look-back words, tile counters, the error word
    if (cudaMemsetAsync(sc->hist, 0, sizeof(sc->hist), st) != cudaSuccess ||
        cudaMemsetAsync(sc->lookback, 0, sizeof(sc->lookback), st) != cudaSuccess ||
        cudaMemsetAsync(sc->tile_ctr, 0, sizeof(sc->tile_ctr) + sizeof(sc->flags), st) != cudaSuccess ||
        onesweep_opt_in(sm) != cudaSuccess) {
        cudaGetLastError();
        return SPH_ERR_CUDA;
    }
    // codes start in the caller's output; 8 passes alternate output -> scratch -> output, so the
    // last (odd) pass writes the result into the output
    k_morton_codes<<<grid_for(n, 256), 256, 0, st>>>(n, x, y, z, b, codes_out, perm_out);
    unsigned hb = (unsigned)grid_for(n, 256);
    k_digit_hist<<<hb, 256, 0, st>>>(codes_out, n, sc->hist);
    k_digit_scan<<<8, 256, 0, st>>>(sc->hist);
    for (int p = 0; p < 8; p++) {
        const bool even = (p & 1) == 0;
        k_onesweep<<<(unsigned)tiles, kRsThreads, sm, st>>>(
            even ? codes_out : sc->keys, even ? perm_out : sc->vals, even ? sc->keys : codes_out,
            even ? sc->vals : perm_out, n, 8 * p, sc->hist + 256 * p, sc->lookback + (size_t)p * tiles * 256,
            sc->tile_ctr + p, &sc->flags, kSpinLimit);
    }
    if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
    uint32_t flags = 0;
    if (cudaMemcpyAsync(&flags, &sc->flags, sizeof flags, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return SPH_ERR_CUDA;
    }
    return (flags & kErrTimeout) ? SPH_ERR_TIMEOUT : SPH_OK;
}


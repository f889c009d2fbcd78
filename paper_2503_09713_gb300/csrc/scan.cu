// Device-wide exclusive scans (reduce-then-scan, 2048 elements per block) used by the leaf
// compaction (App. C, "Reduction": exclusive scan + stream compaction) and by the neighbour-cache
// offsets (App. C, Alg. neighcachedirect).
#include "sph_internal.cuh"

namespace sph {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

// dn (optional): the element count is min(*dn, n), read on the device; blocks past it write zero sums.
__device__ __forceinline__ int64_t scan_count(const int64_t *dn, int64_t n) {
    if (!dn) return n;
    const int64_t v = *dn;
    return v < n ? (v < 0 ? 0 : v) : n;
}

__global__ void k_scan_reduce(const int64_t *__restrict__ in, int64_t n, int64_t *__restrict__ bsum,
                              const int64_t *__restrict__ dn) {
    n = scan_count(dn, n);
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++)
        if (base + k < n) s += in[base + k];
    int64_t tot;
    block_exclusive_scan<kScanThreads>(s, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// out[i] = boff[block] + exclusive prefix inside the block; the block holding element n-1 (or
// block 0 when n == 0) also writes out[n] = total.
__global__ void k_scan_apply(const int64_t *__restrict__ in, int64_t n, const int64_t *__restrict__ boff,
                             int64_t *__restrict__ out, const int64_t *__restrict__ dn) {
    n = scan_count(dn, n);
    if ((int64_t)blockIdx.x * kScanChunk > n) return;
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int64_t tot;
    const int64_t ex = block_exclusive_scan<kScanThreads>(s, tot);
    const int64_t off = boff ? boff[blockIdx.x] : 0;
    int64_t run = off + ex;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    const int64_t last_block = (n > 0) ? (n - 1) / kScanChunk : 0;
    if ((int64_t)blockIdx.x == last_block && threadIdx.x == 0) out[n] = off + tot;
}

// Scratch needed by exclusive_scan_i64 for n elements (all recursion levels).
int64_t scan_scratch_elems(int64_t n) {
    int64_t tot = 0;
    int64_t m = n;
    while (m > kScanChunk) {
        int64_t b = (m + kScanChunk - 1) / kScanChunk;
        tot += 2 * (b + 1);
        m = b;
    }
    return tot + 16;
}

// Only the top level has a device count: the block sums below it are a full array of nb entries.
static int scan_rec(sph_ctx *c, const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, const int64_t *dn) {
    const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb <= 1) {
        k_scan_apply<<<1, kScanThreads, 0, c->stream>>>(in, n, nullptr, out, dn);
        SPH_LAUNCH_CHECK(c, "k_scan_apply");
        return SPH_OK;
    }
    int64_t *bsum = tmp;
    int64_t *boff = tmp + nb + 1;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, c->stream>>>(in, n, bsum, dn);
    SPH_LAUNCH_CHECK(c, "k_scan_reduce");
    int r = scan_rec(c, bsum, boff, nb, tmp + 2 * (nb + 1), nullptr);
    if (r) return r;
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, c->stream>>>(in, n, boff, out, dn);
    SPH_LAUNCH_CHECK(c, "k_scan_apply");
    return SPH_OK;
}

int exclusive_scan_i64(sph_ctx *c, const int64_t *in, int64_t *out, int64_t n) {
    return scan_rec(c, in, out, n, c->scan_tmp, nullptr);
}

int exclusive_scan_i64_dev(sph_ctx *c, const int64_t *in, int64_t *out, const int64_t *dn, int64_t cap) {
    return scan_rec(c, in, out, cap, c->scan_tmp, dn);
}

}  // namespace sph

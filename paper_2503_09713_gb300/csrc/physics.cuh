// Device helpers of the SPH pair loops: M4 kernel (Sect. 2.1), geometry of the neighbour cache,
// Kahan summation for the FP32 pair sums of the mixed-precision path.
#pragma once
#include <climits>

#include "sph_internal.cuh"

namespace sph {

constexpr double kInvPi = 0.31830988618379067154;
constexpr float kInvPiF = 0.31830988618379067154f;

// M4 cubic spline, R_kern = 2: f(q) = 1 - 3/2 q^2 + 3/4 q^3 (q<1), (2-q)^3/4 (1<=q<2), 0 beyond;
// df = df/dq.  W = f(q)/(pi h^3).
template <typename T>
__device__ __forceinline__ void m4(T q, T &f, T &df) {
    if (q < T(1)) {
        f = T(1) + q * q * (T(-1.5) + T(0.75) * q);
        df = q * (T(-3) + T(2.25) * q);
    } else if (q < T(2)) {
        const T t = T(2) - q;
        f = T(0.25) * t * t * t;
        df = T(-0.75) * t * t;
    } else {
        f = T(0);
        df = T(0);
    }
}

// Order of non-negative doubles through their bit patterns: an integer compare on the ALU pipe
// gives the same answer as the FP64 compare, which would occupy the FP64 pipe (the limiter of the
// FP64 pair loops on this GPU, where FP64 issues at 1/64 of FP32).
__device__ __forceinline__ bool nonneg_lt(double a, double b) {
    return __double_as_longlong(a) < __double_as_longlong(b);
}
__device__ __forceinline__ double nonneg_max(double a, double b) { return nonneg_lt(a, b) ? b : a; }

// M4 for q >= 0 in FP64 with the piece chosen by nonneg_lt.
__device__ __forceinline__ void m4d(double q, double &f, double &df) {
    if (nonneg_lt(q, 1.0)) {
        f = 1.0 + q * q * (-1.5 + 0.75 * q);
        df = q * (-3.0 + 2.25 * q);
    } else if (nonneg_lt(q, 2.0)) {
        const double t = 2.0 - q;
        f = 0.25 * t * t * t;
        df = -0.75 * t * t;
    } else {
        f = 0.0;
        df = 0.0;
    }
}
__device__ __forceinline__ double m4d_d2(double q) {
    if (nonneg_lt(q, 1.0)) return 4.5 * q - 3.0;
    if (nonneg_lt(q, 2.0)) return 1.5 * (2.0 - q);
    return 0.0;
}

// d2f/dq2 of M4: 9/2 q - 3 (q<1), 3/2 (2-q) (1<=q<2), 0 beyond.
template <typename T>
__device__ __forceinline__ T m4_d2(T q) {
    if (q < T(1)) return T(4.5) * q - T(3);
    if (q < T(2)) return T(1.5) * (T(2) - q);
    return T(0);
}

// dW/dq shape of M4 without branches (both pieces evaluated, one selected): lanes of a warp hold
// different q, so a branch would run both pieces anyway.
__device__ __forceinline__ float m4_df_sel(float q) {
    const float t = fmaxf(2.f - q, 0.f);
    const float outer = -0.75f * t * t;
    const float inner = q * fmaf(2.25f, q, -3.f);
    return q < 1.f ? inner : outer;
}

// L2 prefetch of the neighbour-list entries of a warp's particles.  Within a group the lists are
// interleaved and consecutive groups follow each other in the cache, so the entries of 32
// consecutive particles form one contiguous range; the warp prefetches it line by line so that the
// list loads of the pair loop hit L2 instead of DRAM.  All 32 lanes call it; [beg, end) is the
// lane's own range (empty for a lane without a particle).
__device__ __forceinline__ void prefetch_lists_l2(const uint32_t *nb_ids, int64_t beg, int64_t end) {
    long long lo = end > beg ? beg : LLONG_MAX, hi = end > beg ? end : 0;
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lo >= hi) return;
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(nb_ids + lo) & ~(uintptr_t)127;
    const uintptr_t a1 = reinterpret_cast<uintptr_t>(nb_ids + hi);
    for (uintptr_t ad = a0 + (uintptr_t)(threadIdx.x & 31) * 128; ad < a1; ad += 32 * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(ad));
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

__device__ __forceinline__ double kahan_value(float s, float c) { return (double)s - (double)c; }

// Geometry shared by the pair loops.
struct PairGeo {
    double L[3], halfL[3];
    float cell[3];
    int periodic;
};

inline PairGeo make_pair_geo(const sph_params &p) {
    PairGeo g;
    for (int k = 0; k < 3; k++) {
        g.L[k] = p.box_hi[k] - p.box_lo[k];
        g.halfL[k] = 0.5 * g.L[k];
        g.cell[k] = (float)(g.L[k] / 1024.0);
    }
    g.periodic = p.periodic;
    return g;
}

// FP32 separation r_a - r_b from cell-relative coordinates (nearest periodic image).
__device__ __forceinline__ void rel_sep(const float4 A, const float4 B, const PairGeo &geo, float &dx, float &dy,
                                        float &dz) {
    const uint32_t pa = __float_as_uint(A.w), pb = __float_as_uint(B.w);
    int dix = (int)((pa >> 20) & 1023u) - (int)((pb >> 20) & 1023u);
    int diy = (int)((pa >> 10) & 1023u) - (int)((pb >> 10) & 1023u);
    int diz = (int)(pa & 1023u) - (int)(pb & 1023u);
    if (geo.periodic) {
        dix = ((dix + 512) & 1023) - 512;
        diy = ((diy + 512) & 1023) - 512;
        diz = ((diz + 512) & 1023) - 512;
    }
    dx = fmaf((float)dix, geo.cell[0], A.x - B.x);
    dy = fmaf((float)diy, geo.cell[1], A.y - B.y);
    dz = fmaf((float)diz, geo.cell[2], A.z - B.z);
}

// Same separation, plus the periodic image shift (in box lengths, -1/0/+1 per axis) that turns the
// FP64 difference r_a - r_b into the nearest image: the cell-index difference is wrapped into
// [-512, 511]; a wrap of +-1024 cells is an image shift of -+1 box.
__device__ __forceinline__ void rel_sep_shift(const float4 A, const float4 B, const PairGeo &geo, float &dx,
                                              float &dy, float &dz, int &sx, int &sy, int &sz) {
    const uint32_t pa = __float_as_uint(A.w), pb = __float_as_uint(B.w);
    const int rx = (int)((pa >> 20) & 1023u) - (int)((pb >> 20) & 1023u);
    const int ry = (int)((pa >> 10) & 1023u) - (int)((pb >> 10) & 1023u);
    const int rz = (int)(pa & 1023u) - (int)(pb & 1023u);
    int wx = rx, wy = ry, wz = rz;
    if (geo.periodic) {
        wx = ((rx + 512) & 1023) - 512;
        wy = ((ry + 512) & 1023) - 512;
        wz = ((rz + 512) & 1023) - 512;
    }
    sx = (wx - rx) / 1024;
    sy = (wy - ry) / 1024;
    sz = (wz - rz) / 1024;
    dx = fmaf((float)wx, geo.cell[0], A.x - B.x);
    dy = fmaf((float)wy, geo.cell[1], A.y - B.y);
    dz = fmaf((float)wz, geo.cell[2], A.z - B.z);
}

// FP64 nearest-image difference a - b given the shift from rel_sep_shift (the shift is zero for all
// but boundary-crossing pairs; adding -L gives the same rounding as subtracting L).
__device__ __forceinline__ double image_diff(double a, double b, int s, double L) {
    double d = a - b;
    if (s != 0) d += (double)s * L;
    return d;
}

// Relative band of the FP32 pre-test: FP32 separations carry relative errors below 1e-6, so a pair
// whose FP32 q^2 exceeds the limit by more than 2^-10 is certainly outside in FP64 as well.
constexpr float kPreBand = 1.0f + 1.0f / 1024.0f;

}  // namespace sph

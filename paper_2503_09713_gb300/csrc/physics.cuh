// Device helpers of the SPH pair loops: smoothing kernels (Sect. 2.1), geometry of the neighbour cache,
// Kahan summation for the FP32 pair sums of the mixed-precision path.
#pragma once
#include <climits>
#include <type_traits>

#include "sph_internal.cuh"

namespace sph {

// Order of non-negative doubles through their bit patterns: an integer compare on the ALU pipe
// gives the same answer as the FP64 compare, which would occupy the FP64 pipe (the limiter of the
// FP64 pair loops on this GPU, where FP64 issues at 1/64 of FP32).
__device__ __forceinline__ bool nonneg_lt(double a, double b) {
    return __double_as_longlong(a) < __double_as_longlong(b);
}
__device__ __forceinline__ double nonneg_max(double a, double b) { return nonneg_lt(a, b) ? b : a; }

// Positive part (a - q)_+ for q >= 0 (FP64: integer compare; FP32: max).
__device__ __forceinline__ double posp(double a, double q) { return nonneg_lt(q, a) ? a - q : 0.0; }
__device__ __forceinline__ float posp(float a, float q) { return fmaxf(a - q, 0.f); }

// ------------------------------------------------------------------ smoothing kernels (Sect. 2.1)
// W(r, h) = C f(q) / h^3, q = r/h, f = 0 for q >= R; normalised in 3-D (4 pi C int f q^2 dq = 1).
// B-splines as sums of truncated powers (Schoenberg):  M4 = (2-q)_+^3/4 - (1-q)_+^3,
// M5 = (5/2-q)_+^4 - 5 (3/2-q)_+^4 + 10 (1/2-q)_+^4, M6 = (3-q)_+^5 - 6 (2-q)_+^5 + 15 (1-q)_+^5;
// Wendland functions with t = (1 - q/2)_+:  C2 = t^4 (1 + 2q), C4 = t^6 (1 + 3q + 35/12 q^2),
// C6 = t^8 (1 + 4q + 25/4 q^2 + 4q^3).  Every branch is evaluated and selected (no divergence).
// eval: f and f' = df/dq; d2: f''.
template <int K>
struct Kernel;

template <>
struct Kernel<SPH_KERNEL_M4> {
    static constexpr double R = 2.0, C = 0.31830988618379067154, F0 = 1.0;
    template <typename T>
    __device__ static void eval(T q, T &f, T &df) {
        const T t2 = posp(T(2), q), t1 = posp(T(1), q);
        f = T(0.25) * t2 * t2 * t2 - t1 * t1 * t1;
        df = T(-0.75) * t2 * t2 + T(3) * t1 * t1;
    }
    // FP64: the same function as one polynomial per piece in Horner form, the piece chosen by integer
    // compares of q's bits, so f and f' cost 3 + 2 fused multiply-adds on the FP64 pipe instead of
    // the 11 FP64 operations of the truncated powers (near q = 2 the expanded form loses the relative
    // accuracy of the small value, not the absolute one: |error| <= a few ulp(2) = 1e-15):
    //   q < 1:      f = 1 - 3/2 q^2 + 3/4 q^3,        f' = -3 q + 9/4 q^2
    //   1 <= q < 2: f = 2 - 3 q + 3/2 q^2 - 1/4 q^3,  f' = -3 + 3 q - 3/4 q^2
    __device__ static void eval(double q, double &f, double &df) {
        const bool in1 = nonneg_lt(q, 1.0), in2 = nonneg_lt(q, 2.0);
        const double c3 = in1 ? 0.75 : -0.25, c2 = in1 ? -1.5 : 1.5, c1 = in1 ? 0.0 : -3.0, c0 = in1 ? 1.0 : 2.0;
        f = in2 ? fma(fma(fma(c3, q, c2), q, c1), q, c0) : 0.0;
        df = in2 ? dfdq_piece(q, in1) : 0.0;
    }
    __device__ static double dfdq(double q) { return nonneg_lt(q, 2.0) ? dfdq_piece(q, nonneg_lt(q, 1.0)) : 0.0; }
    __device__ static double dfdq_piece(double q, bool in1) {
        const double d2 = in1 ? 2.25 : -0.75, d1 = in1 ? -3.0 : 3.0, d0 = in1 ? 0.0 : -3.0;
        return fma(fma(d2, q, d1), q, d0);
    }
    template <typename T>
    __device__ static T d2(T q) { return T(1.5) * posp(T(2), q) - T(6) * posp(T(1), q); }
};

// f'(q) alone (the force loops need no f): from eval, except for M4, where the FP64 loop takes the
// Horner form above and the FP32 loop the two pieces q (9/4 q - 3) (q < 1) and -3/4 (2-q)^2
// (1 <= q < 2), one operation fewer than the truncated powers.
__device__ __forceinline__ bool below_one(double q) { return nonneg_lt(q, 1.0); }
__device__ __forceinline__ bool below_one(float q) { return q < 1.f; }
template <typename K, typename T>
__device__ __forceinline__ T kernel_df(T q) {
    if constexpr (std::is_same<K, Kernel<SPH_KERNEL_M4>>::value && std::is_same<T, double>::value) {
        return K::dfdq(q);
    } else if constexpr (std::is_same<K, Kernel<SPH_KERNEL_M4>>::value) {
        const T t2 = posp(T(2), q);
        const T outer = T(-0.75) * t2 * t2;
        const T inner = q * (T(2.25) * q - T(3));
        return below_one(q) ? inner : outer;
    } else {
        T f, df;
        K::eval(q, f, df);
        return df;
    }
}

template <>
struct Kernel<SPH_KERNEL_M5> {
    static constexpr double R = 2.5, C = 0.31830988618379067154 / 20.0, F0 = 14.375;
    template <typename T>
    __device__ static void eval(T q, T &f, T &df) {
        const T a = posp(T(2.5), q), b = posp(T(1.5), q), c = posp(T(0.5), q);
        const T a3 = a * a * a, b3 = b * b * b, c3 = c * c * c;
        f = a3 * a - T(5) * b3 * b + T(10) * c3 * c;
        df = T(-4) * (a3 - T(5) * b3 + T(10) * c3);
    }
    template <typename T>
    __device__ static T d2(T q) {
        const T a = posp(T(2.5), q), b = posp(T(1.5), q), c = posp(T(0.5), q);
        return T(12) * (a * a - T(5) * b * b + T(10) * c * c);
    }
};

template <>
struct Kernel<SPH_KERNEL_M6> {
    static constexpr double R = 3.0, C = 0.31830988618379067154 / 120.0, F0 = 66.0;
    template <typename T>
    __device__ static void eval(T q, T &f, T &df) {
        const T a = posp(T(3), q), b = posp(T(2), q), c = posp(T(1), q);
        const T a4 = (a * a) * (a * a), b4 = (b * b) * (b * b), c4 = (c * c) * (c * c);
        f = a4 * a - T(6) * b4 * b + T(15) * c4 * c;
        df = T(-5) * (a4 - T(6) * b4 + T(15) * c4);
    }
    template <typename T>
    __device__ static T d2(T q) {
        const T a = posp(T(3), q), b = posp(T(2), q), c = posp(T(1), q);
        return T(20) * (a * a * a - T(6) * b * b * b + T(15) * c * c * c);
    }
};

template <>
struct Kernel<SPH_KERNEL_C2> {
    static constexpr double R = 2.0, C = 21.0 / 16.0 * 0.31830988618379067154, F0 = 1.0;
    template <typename T>
    __device__ static void eval(T q, T &f, T &df) {
        const T t = T(0.5) * posp(T(2), q), t3 = t * t * t;
        f = t3 * t * (T(1) + T(2) * q);
        df = T(-5) * q * t3;
    }
    template <typename T>
    __device__ static T d2(T q) {
        const T t = T(0.5) * posp(T(2), q);
        return t * t * (T(10) * q - T(5));
    }
};

template <>
struct Kernel<SPH_KERNEL_C4> {
    static constexpr double R = 2.0, C = 495.0 / 256.0 * 0.31830988618379067154, F0 = 1.0;
    template <typename T>
    __device__ static void eval(T q, T &f, T &df) {
        const T t = T(0.5) * posp(T(2), q), t2 = t * t, t5 = t2 * t2 * t;
        f = t5 * t * (T(1) + q * (T(3) + T(35.0 / 12.0) * q));
        df = T(-14.0 / 3.0) * q * (T(1) + T(2.5) * q) * t5;
    }
    template <typename T>
    __device__ static T d2(T q) {
        const T t = T(0.5) * posp(T(2), q), t2 = t * t;
        return T(-14.0 / 3.0) * t2 * t2 * (T(1) + q * (T(2) - T(8.75) * q));
    }
};

template <>
struct Kernel<SPH_KERNEL_C6> {
    static constexpr double R = 2.0, C = 1365.0 / 512.0 * 0.31830988618379067154, F0 = 1.0;
    template <typename T>
    __device__ static void eval(T q, T &f, T &df) {
        const T t = T(0.5) * posp(T(2), q), t2 = t * t, t4 = t2 * t2, t7 = t4 * t2 * t;
        f = t7 * t * (T(1) + q * (T(4) + q * (T(6.25) + T(4) * q)));
        df = T(-5.5) * q * (T(1) + q * (T(3.5) + T(4) * q)) * t7;
    }
    template <typename T>
    __device__ static T d2(T q) {
        const T t = T(0.5) * posp(T(2), q), t2 = t * t;
        return T(-5.5) * t2 * t2 * t2 * (T(1) + q * (T(3) + q * (T(-3.75) - T(20) * q)));
    }
};

// Support radius of a kernel id (host side).
inline double kernel_radius(int k) {
    switch (k) {
        case SPH_KERNEL_M5: return Kernel<SPH_KERNEL_M5>::R;
        case SPH_KERNEL_M6: return Kernel<SPH_KERNEL_M6>::R;
        case SPH_KERNEL_C2: return Kernel<SPH_KERNEL_C2>::R;
        case SPH_KERNEL_C4: return Kernel<SPH_KERNEL_C4>::R;
        case SPH_KERNEL_C6: return Kernel<SPH_KERNEL_C6>::R;
        default: return Kernel<SPH_KERNEL_M4>::R;
    }
}

// Calls body(Kernel<K>{}) with the kernel of id k (host side, for launch dispatch).
template <typename F>
inline auto with_kernel(int k, F &&body) {
    switch (k) {
        case SPH_KERNEL_M5: return body(Kernel<SPH_KERNEL_M5>{});
        case SPH_KERNEL_M6: return body(Kernel<SPH_KERNEL_M6>{});
        case SPH_KERNEL_C2: return body(Kernel<SPH_KERNEL_C2>{});
        case SPH_KERNEL_C4: return body(Kernel<SPH_KERNEL_C4>{});
        case SPH_KERNEL_C6: return body(Kernel<SPH_KERNEL_C6>{});
        default: return body(Kernel<SPH_KERNEL_M4>{});
    }
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
    double lo[3], L[3], halfL[3];
    float unit[3];   // length of one step of the fixed-point positions (see qpos_scale)
    float wmargin;   // 2^-20 of the largest box side (see may_cross_face)
    int periodic;
};

inline PairGeo make_pair_geo(const sph_params &p) {
    PairGeo g;
    for (int k = 0; k < 3; k++) {
        g.lo[k] = p.box_lo[k];
        g.L[k] = p.box_hi[k] - p.box_lo[k];
        g.halfL[k] = 0.5 * g.L[k];
        g.unit[k] = (float)(g.L[k] * (p.periodic ? 0x1p-32 : 0x1p-30));
    }
    g.wmargin = (float)(0x1p-20 * std::max(g.L[0], std::max(g.L[1], g.L[2])));
    g.periodic = p.periodic;
    return g;
}

// Distance of a position to the nearest face of a periodic box (FP32; +inf for an open box).
__device__ __forceinline__ float face_distance(double px, double py, double pz, const PairGeo &geo) {
    if (!geo.periodic) return INFINITY;
    const double p[3] = {px, py, pz};
    double d = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; k++) d = fmin(d, fmin(p[k] - geo.lo[k], geo.lo[k] + geo.L[k] - p[k]));
    return (float)d;
}

// Whether a neighbour whose separation components are at most `reach` (FP32, nearest image) may lie
// across a periodic face from a particle `dface` from the nearest face.  If not, the particle's
// position minus the separation stays inside the box on every axis, so the plain FP64 difference
// of the stored positions is already the nearest image.  The margins cover the FP32 separation's
// error (2^-24 relative plus one fixed-point step) and the rounding of dface.
__device__ __forceinline__ bool may_cross_face(float reach, float dface, const PairGeo &geo) {
    return geo.periodic && !(reach * 1.001f + geo.wmargin < dface);
}

// FP32 separation r_a - r_b (nearest periodic image) from fixed-point positions.
__device__ __forceinline__ void rel_sep(const uint4 A, const uint4 B, const PairGeo &geo, float &dx, float &dy,
                                        float &dz) {
    dx = (float)(int)(A.x - B.x) * geo.unit[0];
    dy = (float)(int)(A.y - B.y) * geo.unit[1];
    dz = (float)(int)(A.z - B.z) * geo.unit[2];
}

// FP64 nearest image of a separation: |d| > L/2 moves it by one box length (integer compare).
__device__ __forceinline__ double nearest_image(double d, double L, double halfL, int periodic) {
    if (periodic && nonneg_lt(halfL, fabs(d))) d -= copysign(L, d);
    return d;
}

// Relative band of the FP32 pre-test: FP32 separations carry relative errors below 1e-6, so a pair
// whose FP32 q^2 exceeds the limit by more than 2^-10 is certainly outside in FP64 as well.
constexpr float kPreBand = 1.0f + 1.0f / 1024.0f;

}  // namespace sph

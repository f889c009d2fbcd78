// Device helpers of the SPH pair loops: M4 kernel (Sect. 2.1), geometry of the neighbour cache,
// Kahan summation for the FP32 pair sums of the mixed-precision path.
#pragma once
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

}  // namespace sph

// Pair force loop (Sect. 2.1, Eqs. sphvel, sphuint, q^a_ab, v_sig, Lambda_cond, F_ab) and the CFL
// time step (App. G).
//
//   a_a    = - sum_b m [ (P_a + q^a_ab)/(rho_a^2 Omega_a) F_ab(h_a) + (P_b + q^b_ab)/(rho_b^2 Omega_b) F_ab(h_b) ] rhat_ab
//   du_a/dt=   sum_b m (P_a + q^a_ab)/(rho_a^2 Omega_a) (v_ab . rhat_ab) F_ab(h_a)
//            + sum_b m alpha_u v_sig^u (u_a - u_b) 1/2 [F_ab(h_a)/(Omega_a rho_a) + F_ab(h_b)/(Omega_b rho_b)]
//   q^a_ab = -1/2 rho_a (alpha c_s,a + beta |v_ab.rhat|) (v_ab.rhat)  when v_ab.rhat < 0, else 0
//   v_sig^dt_a = max_b (alpha c_s,a + beta max(0, -v_ab.rhat)),  alpha c_s,a without neighbours
// over pairs with r_ab < R_kern max(h_a, h_b).  Per-particle factors (P/(rho^2 Omega), 1/(rho Omega), c_s,
// P, rho, 1/h) are computed once per particle by a preparation kernel.  The mixed path evaluates
// each pair in FP32 from fixed-point positions and accumulates with Kahan compensation.
#include "physics.cuh"

namespace sph {

struct ForceParams {
    double mass, gamma, alpha_av, beta_av, alpha_u, c_cour, c_force;
    int m4_poly;               // FP64 records carry the M4 gradient as polynomials (FRec)
    double kern_c;             // C_norm of the smoothing kernel
    double kern_r;             // its support radius R_kern (in units of h)
    PairGeo geo;
    const double *box_mass;    // per-box particle mass (batch) or nullptr
    const double *box_gamma;   // per-box adiabatic index (batch) or nullptr
    const uint16_t *box_of;    // box of each particle (batch) or nullptr
    unsigned long long *box_dt_next;   // per-box CFL minimum (bits) or nullptr
    const uint32_t *abort;     // captured step: skip when an earlier stage failed
};

// Per-particle FP64 record of the force loop: 176 bytes, read as double2.
// pre = P/(rho^2 Omega), hqf = 1/(2 rho Omega), acs = alpha_AV c_s, rh2 = (R_kern h)^2 (a pair
// interacts when r^2 < max(rh2_a, rh2_b), the same bits as (R max h)^2), and for the conductivity
// term au = alpha_u u and P2 = 2 P (one FP64 product fewer per pair each).  k[]: the smoothing
// kernel's gradient.  In general k0 = 1/h and k1 = C_norm/h^4, so F_ab(h) = k1 f'(r k0).  For M4
// the loop needs F(r)/r only, which on each piece is a polynomial in r^2 and 1/r:
//   r < h:      F/r = g2i r^2 (1/r) + g1i,          g2i = 9/4 k h^-2,  g1i = -3 k h^-1
//   h <= r < 2h: F/r = (g2o r^2 + g0o) (1/r) + g1o,  g2o = -3/4 k h^-2, g1o = 3 k h^-1, g0o = -3 k
// with k = C_norm/h^4 (from f'(q) = -3q + 9/4 q^2 and -3 + 3q - 3/4 q^2); then k0 = h^2 (the piece
// boundary, compared with r^2), k1 = g0o, k2 = g1i, k3 = g1o, k4 = g2i, k5 = g2o.  av1 = -acs hqf and
// av2 = beta_AV hqf carry the artificial viscosity: for an approaching pair (v.rhat < 0)
//   pre + q_ab/(rho^2 Omega) = pre - (acs - beta v.rhat) v.rhat hqf = (av2 v.rhat + av1) v.rhat + pre,
// two fused multiply-adds per side.
struct __align__(16) FRec {
    double x, y, z, h;
    double vx, vy, vz, au;
    double pre, hqf, acs, P2;
    double rho, rh2, k0, k1;
    double k2, k3, k4, k5;
    double av1, av2;
};
static_assert(sizeof(FRec) == 176, "FP64 force record");

__global__ void k_force_prep(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                             const double *__restrict__ z, const double *__restrict__ vx,
                             const double *__restrict__ vy, const double *__restrict__ vz,
                             const double *__restrict__ u, const double *__restrict__ h,
                             const double *__restrict__ rho, const double *__restrict__ omega,
                             const double *__restrict__ alpha, ForceParams fp, int mixed, FRec *__restrict__ rec, float4 *__restrict__ m_v, float4 *__restrict__ m_t,
                             float4 *__restrict__ m_r, uint4 *__restrict__ qpos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || aborted(fp.abort, kAbortStep)) return;
    const double gam = fp.box_gamma ? fp.box_gamma[fp.box_of[i]] : fp.gamma;
    if (mixed) {
        // FP32 records for the FP32 pair sums: P = (gamma-1) rho u, c_s = sqrt(gamma (gamma-1) u),
        // P/(rho^2 Omega) = (gamma-1) u / (rho Omega), 1/(rho Omega), 1/(pi h^4)
        const float r = (float)rho[i], om = (float)omega[i], ui = (float)u[i], g = (float)gam;
        const float qf = 1.f / (r * om);
        const float hinvf = 1.f / (float)h[i];
        m_v[i] = make_float4((float)vx[i], (float)vy[i], (float)vz[i], hinvf);
        const float al = (float)(alpha ? alpha[i] : fp.alpha_av);
        m_t[i] = make_float4((g - 1.f) * ui * qf, qf, al * sqrtf(g * (g - 1.f) * ui),
                             (g - 1.f) * r * ui);
        m_r[i] = make_float4(r, ui, hinvf * hinvf * hinvf * hinvf * (float)fp.kern_c, 0.f);
    } else {
        // the same quantities in FP64, with two divisions and one square root per particle
        const double r = rho[i], om = omega[i], ui = u[i], hi = h[i];
        const double qf = 1.0 / (r * om);
        const double hinv = 1.0 / hi;
        FRec f;
        f.x = x[i]; f.y = y[i]; f.z = z[i]; f.h = hi;
        f.vx = vx[i]; f.vy = vy[i]; f.vz = vz[i]; f.au = fp.alpha_u * ui;
        f.pre = (gam - 1.0) * ui * qf; f.hqf = 0.5 * qf;
        f.acs = (alpha ? alpha[i] : fp.alpha_av) * sqrt(gam * (gam - 1.0) * ui);
        f.av1 = -f.acs * f.hqf;
        f.av2 = fp.beta_av * f.hqf;
        f.P2 = 2.0 * ((gam - 1.0) * r * ui);
        f.rho = r;
        const double fn = hinv * hinv * hinv * hinv * fp.kern_c;
        const double rad = __dmul_rn(fp.kern_r, hi);
        f.rh2 = __dmul_rn(rad, rad);
        if (fp.m4_poly) {
            f.k0 = hi * hi;
            f.k1 = -3.0 * fn;
            f.k2 = -3.0 * fn * hinv;
            f.k3 = 3.0 * fn * hinv;
            f.k4 = 2.25 * fn * hinv * hinv;
            f.k5 = -0.75 * fn * hinv * hinv;
        } else {
            f.k0 = hinv;
            f.k1 = fn;
            f.k2 = f.k3 = f.k4 = f.k5 = 0.0;
        }
        rec[i] = f;
        qpos[i].w = __float_as_uint((float)hi);   // the FP32 h of the pre-test
    }
}

template <bool kPoly>
__device__ __forceinline__ void load_rec(const FRec *p, FRec &o) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 t;
    t = __ldg(q + 0); o.x = t.x; o.y = t.y;
    t = __ldg(q + 1); o.z = t.x; o.h = t.y;
    t = __ldg(q + 2); o.vx = t.x; o.vy = t.y;
    t = __ldg(q + 3); o.vz = t.x; o.au = t.y;
    t = __ldg(q + 4); o.pre = t.x; o.hqf = t.y;
    t = __ldg(q + 5); o.acs = t.x; o.P2 = t.y;
    t = __ldg(q + 6); o.rho = t.x; o.rh2 = t.y;
    t = __ldg(q + 7); o.k0 = t.x; o.k1 = t.y;
    if (kPoly) {
        t = __ldg(q + 8); o.k2 = t.x; o.k3 = t.y;
        t = __ldg(q + 9); o.k4 = t.x; o.k5 = t.y;
    }
    t = __ldg(q + 10); o.av1 = t.x; o.av2 = t.y;
}

// F_ab(h)/r of one side of a pair from its record (see FRec), r2 = r^2, rinv = 1/r, inside the
// interaction range of that side (r^2 < rh2) or zero.
template <typename K>
__device__ __forceinline__ double grad_over_r(const FRec &R, double r2, double rinv) {
    if constexpr (std::is_same<K, Kernel<SPH_KERNEL_M4>>::value) {
        const bool in1 = nonneg_lt(r2, R.k0), in2 = nonneg_lt(r2, R.rh2);
        const double g2 = in1 ? R.k4 : R.k5, g0 = in1 ? 0.0 : R.k1, g1 = in1 ? R.k2 : R.k3;
        return in2 ? fma(fma(g2, r2, g0), rinv, g1) : 0.0;
    } else {
        return kernel_df<K>(r2 * rinv * R.k0) * R.k1 * rinv;
    }
}

// 1/sqrt(x) for 2^-125 <= x < 2^127 without FP32/FP64 conversion instructions (they issue on the
// FP64 pipe, this loop's bound): x narrowed to FP32 by truncating its bits (relative error below
// 2^-23), its FP32 reciprocal square root widened back by its bits (exact), then one Newton-Raphson
// step y <- y + y (1 - x y^2) / 2, which squares the relative error (below 1e-13).
__device__ __forceinline__ bool fp32_normal_range(double x) {
    const uint32_t e = (uint32_t)((unsigned long long)__double_as_longlong(x) >> 52);   // x > 0: no sign bit
    return e >= 1023u - 125u && e <= 1023u + 126u;
}
__device__ __forceinline__ double rsqrt_via_fp32(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t xf = (((uint32_t)(b >> 52) - (1023u - 127u)) << 23) | (uint32_t)((b >> 29) & 0x7fffffu);
    const uint32_t u = __float_as_uint(rsqrtf(__uint_as_float(xf)));
    const double y = __longlong_as_double((long long)(((unsigned long long)((u >> 23) + (1023u - 127u)) << 52) |
                                                      ((unsigned long long)(u & 0x7fffffu) << 29)));
    return fma(0.5 * y, fma(-x * y, y, 1.0), y);
}

struct ForceOut {
    double *ax, *ay, *az, *du, *vsig;
    double *dhdt;   // dh/dt = -h/(3 rho Omega) sum_b m v_ab . grad_a W_ab(h_a)  (Eq. rhoh with the SPH
                    // continuity equation); only the initial guess of the next h iteration uses it
};

// CFL candidate of one particle (App. G): min(C_cour h / v_sig, C_force sqrt(h/|a|)).
__device__ __forceinline__ double dt_candidate(double h, double vs, double ax, double ay, double az,
                                               const ForceParams &fp) {
    const double t1 = fp.c_cour * h / vs;
    const double am = sqrt(ax * ax + ay * ay + az * az);
    const double t2 = am > 0.0 ? fp.c_force * sqrt(h / am) : INFINITY;
    return fmin(t1, t2);
}

// Warp minimum of the CFL candidates and warp sum of the in-range pair counts (all 32 lanes
// participate), then one atomic each per warp; positive doubles order like their bit patterns.  A
// warp whose particles lie in one box updates that box's minimum once; a warp across a box boundary
// updates it lane by lane.
__device__ __forceinline__ void dt_reduce(double t, unsigned long long npair, DevScalars *sc,
                                          unsigned long long *box_dt_next, int box) {
    double tw = t;
    for (int o = 16; o > 0; o >>= 1) {
        tw = fmin(tw, __shfl_xor_sync(0xffffffffu, tw, o));
        npair += __shfl_xor_sync(0xffffffffu, npair, o);
    }
    const bool lane0 = (threadIdx.x & 31) == 0;
    if (lane0) {
        if (tw > 0.0 && tw < INFINITY) atomicMin(&sc->dt_min_bits, dbits(tw));
        atomicAdd(&sc->inrange_pairs, npair);
    }
    if (box_dt_next) {
        const int box0 = __shfl_sync(0xffffffffu, box, 0);
        if (__all_sync(0xffffffffu, box == box0)) {
            if (lane0 && tw > 0.0 && tw < INFINITY) atomicMin(&box_dt_next[box0], dbits(tw));
        } else if (t > 0.0 && t < INFINITY) {
            atomicMin(&box_dt_next[box], dbits(t));
        }
    }
}

// FP64 pair loop in two phases per chunk, so that the FP64 work runs with converged lanes.  Phase 1
// walks the particle's cached candidates and keeps those that pass an FP32 test on the fixed-point
// separations against the current h (kPreBand margin: every pair inside R max(h_a, h_b) passes), up to
// kForceQueue of them, in a per-thread queue in shared memory; phase 2 evaluates the queued pairs in
// FP64, all lanes of the warp stepping through their queues together.  (Tested and evaluated in one
// loop, ~30% of the candidates fail while other lanes of the warp evaluate, and the FP64 pipe, this
// loop's bound, runs for every candidate of the warp.)  The FP64 separation takes the nearest image
// by |d| > L/2, which for every queued pair is the image of the fixed-point test.  The mass factor is
// applied once per particle.
constexpr int kForceQueue = 32;   // queued candidates per thread: 4 bytes each in shared memory

template <typename K>
__global__ void __launch_bounds__(256) k_forces_fp64(int64_t n, const FRec *__restrict__ rec,
                                                     const uint4 *__restrict__ qpos,
                                                     const uint32_t *__restrict__ nb_cnt,
                                                     const unsigned long long *__restrict__ nb_ptr,
                                                     const uint32_t *__restrict__ nb_ids, ForceParams fp, ForceOut out,
                                                     DevScalars *sc) {
    extern __shared__ uint32_t fq[];   // [kForceQueue][blockDim.x]: thread t's queue is column t
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // one thread per particle
    if (a - (threadIdx.x & 31) >= n) return;   // whole warp past the end
    if (aborted(fp.abort, kAbortStep)) return;
    const bool va = a < n;
    const int box = (va && fp.box_of) ? fp.box_of[a] : 0;
    double tdt = INFINITY;
    unsigned long long npair = 0;
    const uint32_t cnt = va ? nb_cnt[a] : 0u;
    const unsigned long long pw = va ? nb_ptr[a] : 0ULL;
    uint32_t st;
    const uint32_t *ids = nb_list(nb_ids, pw, st);
    const int64_t lbeg = ids - nb_ids;
    prefetch_lists_l2(nb_ids, lbeg, lbeg + nb_span(cnt, st));
    constexpr bool kPoly = std::is_same<K, Kernel<SPH_KERNEL_M4>>::value;
    FRec A;
    load_rec<kPoly>(&rec[va ? a : 0], A);
    const uint4 PA = qpos[va ? a : 0];
    const float hA = va ? __uint_as_float(PA.w) : 0.f;
    const PairGeo &geo = fp.geo;
    double axs = 0.0, ays = 0.0, azs = 0.0, dus = 0.0, divs = 0.0;
    double vs = A.acs;
    uint32_t *q = fq + threadIdx.x;
    const int qs = blockDim.x;
    const float dface = va ? face_distance(A.x, A.y, A.z, geo) : INFINITY;
    uint32_t k = 0;
    for (;;) {
        // phase 1: FP32 pre-test, queue the survivors
        int nq = 0;
        float reach = 0.f;   // largest |separation| component of a queued candidate
        while (nq < kForceQueue && k < cnt) {
            const uint32_t b = nb_at(ids, k, st);
            ++k;
            float fx, fy, fz;
            const uint4 PB = qpos[b];
            rel_sep(PA, PB, geo, fx, fy, fz);
            const float hmf = fmaxf(hA, __uint_as_float(PB.w));
            if (!(fx * fx + fy * fy + fz * fz > (float)(K::R * K::R) * kPreBand * hmf * hmf)) {
                q[(nq++) * qs] = b;
                reach = fmaxf(reach, fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))));
            }
        }
        const int nq_max = __reduce_max_sync(0xffffffffu, (unsigned)nq);
        const bool wrap = __any_sync(0xffffffffu, may_cross_face(reach, dface, geo));
        // phase 2: the queued pairs in FP64, with the nearest-image step only where some lane of the
        // warp may have a neighbour across a periodic face (warp-uniform)
        auto evaluate = [&](auto wrap_c) {
        for (int j = 0; j < nq_max; j++) {
            if (j >= nq) continue;
            const uint32_t b = q[j * qs];
            FRec B;
            load_rec<kPoly>(&rec[b], B);
            double dx = A.x - B.x, dy = A.y - B.y, dz = A.z - B.z;
            if (decltype(wrap_c)::value) {
                dx = nearest_image(dx, geo.L[0], geo.halfL[0], geo.periodic);
                dy = nearest_image(dy, geo.L[1], geo.halfL[1], geo.periodic);
                dz = nearest_image(dz, geo.L[2], geo.halfL[2], geo.periodic);
            }
            // r < R max(h_a, h_b); both kernels and their derivatives vanish at R, so the rounding of
            // r^2 (fused here) only decides pairs whose terms are zero
            const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            if (!nonneg_lt(r2, nonneg_max(A.rh2, B.rh2))) continue;
            ++npair;
            // the warp takes the FP32-seeded form when every active lane's r^2 is in its range
            double rinv;
            if (__all_sync(__activemask(), fp32_normal_range(r2))) rinv = rsqrt_via_fp32(r2);
            else rinv = rsqrt(r2);
            // G = F_ab/r of both sides: F rhat = G (r_a - r_b), v_ab . rhat F = (v_ab . (r_a - r_b)) G
            const double Ga = grad_over_r<K>(A, r2, rinv), Gb = grad_over_r<K>(B, r2, rinv);
            const double vd = (A.vx - B.vx) * dx + (A.vy - B.vy) * dy + (A.vz - B.vz) * dz;
            const double vdotr = vd * rinv;
            double Aa = A.pre, Ab = B.pre;
            if (__double_as_longlong(vdotr) < 0) {   // sign bit: approaching (-0 changes nothing below)
                Aa = fma(fma(A.av2, vdotr, A.av1), vdotr, Aa);
                Ab = fma(fma(B.av2, vdotr, B.av1), vdotr, Ab);
                vs = nonneg_max(vs, fma(-fp.beta_av, vdotr, A.acs));   // alpha c_s + beta |v.rhat|
            }
            const double sc_ = Aa * Ga + Ab * Gb;
            axs -= sc_ * dx;
            ays -= sc_ * dy;
            azs -= sc_ * dz;
            const double vfa = vd * Ga;   // (v_ab . rhat) F_ab(h_a)
            dus = fma(Aa, vfa, dus);
            divs += vfa;
            if (fp.alpha_u != 0.0) {
                const double t = fabs(A.P2 - B.P2);   // 2 |P_a - P_b|; v_sig^u = sqrt(t / (rho_a + rho_b))
                if (__double_as_longlong(t) > 0) {
                    const double xu = t * (A.rho + B.rho);
                    double ru;
                    if (__all_sync(__activemask(), fp32_normal_range(xu))) ru = rsqrt_via_fp32(xu);
                    else ru = rsqrt(xu);
                    const double vsu = t * ru;
                    // F_a hqf_a + F_b hqf_b = r (G_a hqf_a + G_b hqf_b)
                    dus += vsu * (A.au - B.au) * ((r2 * rinv) * (Ga * A.hqf + Gb * B.hqf));
                }
            }
        }
        };
        if (wrap) evaluate(std::true_type{});
        else evaluate(std::false_type{});
        if (!__any_sync(0xffffffffu, k < cnt)) break;
    }
    if (va) {
        const double m = fp.box_mass ? fp.box_mass[box] : fp.mass;
        axs *= m;
        ays *= m;
        azs *= m;
        dus *= m;
        out.ax[a] = axs;
        out.ay[a] = ays;
        out.az[a] = azs;
        out.du[a] = dus;
        out.vsig[a] = vs;
        out.dhdt[a] = -A.h * (2.0 * A.hqf) * (1.0 / 3.0) * m * divs;
        tdt = dt_candidate(A.h, vs, axs, ays, azs, fp);
    }
    dt_reduce(tdt, npair, sc, fp.box_dt_next, box);
}

template <typename K>
__global__ void __launch_bounds__(256) k_forces_mixed(int64_t n, const uint4 *__restrict__ qpos,
                                                      const float4 *__restrict__ m_v, const float4 *__restrict__ m_t,
                                                      const float4 *__restrict__ m_r, const double *__restrict__ h,
                                                      const uint32_t *__restrict__ nb_cnt,
                                                      const unsigned long long *__restrict__ nb_ptr,
                                                      const uint32_t *__restrict__ nb_ids, ForceParams fp,
                                                      ForceOut out, DevScalars *sc) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // one thread per particle
    if (a - (threadIdx.x & 31) >= n) return;   // whole warp past the end
    if (aborted(fp.abort, kAbortStep)) return;
    const int box = (a < n && fp.box_of) ? fp.box_of[a] : 0;
    double tdt = INFINITY;
    unsigned long long npair = 0;
    const uint32_t cnt = a < n ? nb_cnt[a] : 0u;
    const unsigned long long pw = a < n ? nb_ptr[a] : 0ULL;
    uint32_t st;
    const uint32_t *ids = nb_list(nb_ids, pw, st);
    const int64_t lbeg = ids - nb_ids;
    prefetch_lists_l2(nb_ids, lbeg, lbeg + nb_span(cnt, st));
    if (a < n) {
    const uint4 PA = qpos[a];
    const float4 VA = m_v[a], TA = m_t[a], RA = m_r[a];
    const double mass_d = fp.box_mass ? fp.box_mass[box] : fp.mass;
    const float mass = (float)mass_d, beta = (float)fp.beta_av, au = (float)fp.alpha_u;
    // the mass factor is applied once per particle; the sums are the pair terms divided by m
    float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f, sz = 0.f, cz = 0.f, su = 0.f, cu = 0.f, sdiv = 0.f;
    float vs = TA.z;   // alpha_AV c_s,a
    const float hia = VA.w;
    const float Fa_n = RA.z;   // C_norm/h_a^4
    // one pair; B's position and velocity are already loaded
    auto pair = [&](uint32_t b, const uint4 PB, const float4 VB) {
        float dx, dy, dz;
        rel_sep(PA, PB, fp.geo, dx, dy, dz);
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float him = fminf(hia, VB.w);
        if (!(r2 * him * him < (float)(K::R * K::R))) return;
        ++npair;
        const float4 TB = m_t[b];
        const float4 RB = m_r[b];
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        const float dfa = kernel_df<K>(r * hia), dfb = kernel_df<K>(r * VB.w);
        const float Fa = dfa * Fa_n;
        const float Fb = dfb * RB.z;
        const float vdotr = fmaf(VA.z - VB.z, dz, fmaf(VA.y - VB.y, dy, (VA.x - VB.x) * dx)) * rinv;
        float Aa = TA.x, Ab = TB.x;
        if (vdotr < 0.f) {
            const float w = beta * vdotr;   // -beta |v.rhat|
            Aa = fmaf(-0.5f * (TA.z - w) * vdotr, TA.y, Aa);
            Ab = fmaf(-0.5f * (TB.z - w) * vdotr, TB.y, Ab);
            vs = fmaxf(vs, TA.z - w);
        }
        const float sc_ = fmaf(Aa, Fa, Ab * Fb) * rinv;
        kahan_add(sx, cx, -sc_ * dx);
        kahan_add(sy, cy, -sc_ * dy);
        kahan_add(sz, cz, -sc_ * dz);
        const float vfa = vdotr * Fa;
        float dut = Aa * vfa;
        sdiv += vfa;
        if (au != 0.f) {
            // v_sig^u = sqrt(|P_a - P_b| / (rho_a + rho_b)/2) = t / sqrt(t (rho_a + rho_b)/2)
            const float t = fabsf(TA.w - TB.w);
            const float vsu = t > 0.f ? t * rsqrtf(0.5f * t * (RA.x + RB.x)) : 0.f;
            dut = fmaf(au * vsu * (RA.y - RB.y) * 0.5f, fmaf(Fa, TA.y, Fb * TB.y), dut);
        }
        kahan_add(su, cu, dut);
    };
    // two neighbours per iteration, their gathers issued together; the next pair of indices is
    // loaded one iteration ahead
    uint32_t k = 0;
    uint2 nbp = make_uint2(0u, 0u);
    if (cnt >= 2) nbp = nb_pair(ids, 0, st);
    for (; k + 2 <= cnt; k += 2) {
        const uint32_t b0 = nbp.x, b1 = nbp.y;
        if (k + 4 <= cnt) nbp = nb_pair(ids, k + 2, st);
        const uint4 P0 = qpos[b0], P1 = qpos[b1];
        const float4 V0 = m_v[b0], V1 = m_v[b1];
        pair(b0, P0, V0);
        pair(b1, P1, V1);
    }
    if (k < cnt) {
        const uint32_t b = nb_at(ids, k, st);
        pair(b, qpos[b], m_v[b]);
    }
    const double axs = mass_d * kahan_value(sx, cx), ays = mass_d * kahan_value(sy, cy),
                 azs = mass_d * kahan_value(sz, cz);
    out.ax[a] = axs;
    out.ay[a] = ays;
    out.az[a] = azs;
    out.du[a] = mass_d * kahan_value(su, cu);
    out.vsig[a] = (double)vs;
    const float ha = (float)h[a];
    out.dhdt[a] = (double)(-ha * TA.y * (1.0f / 3.0f) * mass * sdiv);
    // CFL candidate in FP32 (a time-step estimate; the FP64 path evaluates it in FP64)
    const float am = sqrtf((float)(axs * axs + ays * ays + azs * azs));
    const float t1 = (float)fp.c_cour * ha / vs;
    const float t2 = am > 0.f ? (float)fp.c_force * sqrtf(ha / am) : INFINITY;
    tdt = (double)fminf(t1, t2);
    }
    dt_reduce(tdt, npair, sc, fp.box_dt_next, box);
}

__global__ void k_reset_dt(DevScalars *sc, unsigned long long *box_dt_next, int n_boxes) {
    if (threadIdx.x == 0) {
        sc->dt_min_bits = 0x7ff0000000000000ULL;
        sc->inrange_pairs = 0ULL;
    }
    if (box_dt_next)
        for (int b = threadIdx.x; b < n_boxes; b += blockDim.x) box_dt_next[b] = 0x7ff0000000000000ULL;
}

int forces_run(sph_ctx *c, sph_state *s, double *ax, double *ay, double *az, double *du) {
    if (!c->cache_valid) return fail(c, SPH_ERR_ORDER, "forces before sph_find_neighbours");
    const int64_t n = s->n;
    ForceParams fp;
    fp.mass = s->mass;
    fp.gamma = c->p.gamma;
    fp.alpha_av = c->p.alpha_av;
    fp.beta_av = c->p.beta_av;
    fp.alpha_u = c->p.alpha_u;
    fp.c_cour = c->p.c_cour;
    fp.c_force = c->p.c_force;
    fp.kern_c = with_kernel(c->p.kernel, [](auto kern) { return decltype(kern)::C; });
    fp.kern_r = kernel_radius(c->p.kernel);
    fp.m4_poly = c->p.kernel == SPH_KERNEL_M4;
    fp.geo = make_pair_geo(c->p);
    fp.box_mass = c->batch ? c->box_mass : nullptr;
    fp.box_gamma = c->batch ? c->box_gamma : nullptr;
    fp.box_of = c->batch ? c->box_of : nullptr;
    fp.box_dt_next = c->batch ? c->box_dt_next : nullptr;
    fp.abort = abort_word(c);
    const int mixed = c->p.precision == SPH_MIXED;
    int r = ensure_force_records(c);
    if (r) return r;
    if ((r = stage_begin(c, kStForcePrep))) return r;
    k_force_prep<<<grid_for(n, 256), 256, 0, c->stream>>>(n, s->x, s->y, s->z, s->vx, s->vy, s->vz, s->u, s->h,
                                                           s->rho, s->omega, c->p.av_switch ? s->alpha : nullptr,
                                                           fp, mixed, (FRec *)c->frec, c->m_v,
                                                           c->m_t, c->m_r, c->qpos);
    SPH_LAUNCH_CHECK(c, "k_force_prep");
    k_reset_dt<<<1, 32, 0, c->stream>>>(c->dscal, fp.box_dt_next, c->n_boxes);
    SPH_LAUNCH_CHECK(c, "k_reset_dt");
    if ((r = stage_end(c, kStForcePrep)) || (r = stage_begin(c, kStForces))) return r;
    ForceOut out{ax, ay, az, du, s->vsig, c->dhdt};
    const int blk = c->launch.forces_block;
    const size_t fsm = (size_t)kForceQueue * blk * sizeof(uint32_t);
    cudaError_t oe = cudaSuccess;
    with_kernel(c->p.kernel, [&](auto kern) {
        using K = decltype(kern);
        if (!mixed) oe = smem_opt_in<k_forces_fp64<K>>(fsm);
        return 0;
    });
    SPH_CUDA(c, oe);
    with_kernel(c->p.kernel, [&](auto kern) {
        using K = decltype(kern);
        if (mixed)
            k_forces_mixed<K><<<grid_for(n, blk), blk, 0, c->stream>>>(n, c->qpos, c->m_v, c->m_t, c->m_r, s->h,
                                                                       c->nb_cnt, c->nb_ptr, c->nb_ids, fp, out,
                                                                       c->dscal);
        else
            k_forces_fp64<K><<<grid_for(n, blk), blk, fsm, c->stream>>>(
                n, (const FRec *)c->frec, c->qpos,
                                                                      c->nb_cnt, c->nb_ptr, c->nb_ids, fp, out,
                                                                      c->dscal);
        return 0;
    });
    SPH_LAUNCH_CHECK(c, "k_forces");
    return stage_end(c, kStForces);
}

}  // namespace sph

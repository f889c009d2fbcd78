// Smoothing-length / density iteration (App. F, Alg. smoothinglenghtupdate) and Omega (Eq. sphomega).
//
// Each particle's equation  rho_sum(h_a) = m (hfact/h_a)^3  involves only its own h_a, so a thread
// iterates Newton-Raphson on its own particle until |dh|/h^n <= eps_c (the paper iterates all
// particles until the largest eps is below eps_c; once a particle meets the criterion its further
// updates are below eps_c^2).  Steps are clamped to [h/lambda, h*lambda]; an h above chi*h^n is
// clamped there and flagged so the host rebuilds the cache (outer loop of Alg. F).  After
// convergence rho = rho(h) (Eq. rhoh) and Omega = 1 + h/(3 rho) sum_b m dW/dh at the final h, the
// sum carried from the last Newton evaluation to the final h by its h-derivative (second-order
// error in a step below eps_c h^n), so no further pass over the neighbours is needed.
// FP64 path: all pair arithmetic in FP64.  Mixed path: pair sums in FP32 (Kahan) on separations
// from fixed-point positions; Newton update, h, rho and Omega in FP64.
#include <cstddef>

#include "physics.cuh"

namespace sph {

struct DensParams {
    double mass, hfact, h_tol, h_clamp, inv_h_clamp, chi;
    int max_iter;
    PairGeo geo;
    const double *box_mass;   // per-box particle mass (batch) or nullptr
    const uint16_t *box_of;   // box of each particle (batch) or nullptr
};

// A positive normal float as a double, from its bits: exponent rebiased (127 -> 1023), mantissa
// moved up by 29 bits.  Exact (IEEE 754 binary32 -> binary64) and on the integer pipe.
__device__ __forceinline__ double widen_normal(float f) {
    const uint32_t u = __float_as_uint(f);
    const unsigned long long d = ((unsigned long long)((u >> 23) + (1023u - 127u)) << 52) |
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

constexpr int kDensQueue = 32;   // FP64 path: queued candidates per thread (8 bytes each in shared memory)

// Sums over the neighbours of a at smoothing length h (kernel K):  sf = sum f(q),
// sg = sum (3 f + q f'),  sk = sum (12 f + 8 q f' + q^2 f'')  (self term included: f(0) times 1, 3
// and 12), so that rho_sum = m C sf / h^3,  sum m dW/dh = -m C sg / h^4,
// sum m d2W/dh2 = m C sk / h^5.
template <typename K, bool kMixed>
__device__ __forceinline__ void density_sums(int64_t a, double ha, uint32_t cnt, const uint32_t *__restrict__ ids,
                                             uint32_t st,
                                             const double *__restrict__ x, const double *__restrict__ y,
                                             const double *__restrict__ z, const uint4 *__restrict__ qpos,
                                             const PairGeo &geo, double &sf, double &sg, double &sk,
                                             uint32_t &nin, uint2 *queue) {
    const double hinv = 1.0 / ha;
    if (!kMixed) {
        // Two phases per chunk so that the FP64 work runs with converged lanes: an FP32 pre-test on the
        // fixed-point positions queues (up to kDensQueue) the candidates that may lie inside R h (the
        // others are clearly outside); then every lane of the warp evaluates its queued candidates in
        // FP64 together, the nearest image taken by |d| > L/2.  All 32 lanes call this function (a lane
        // without a particle passes cnt = 0).
        const double xa = x[a], ya = y[a], za = z[a];
        const double hinv2 = hinv * hinv;
        const uint4 A = qpos[a];
        const float lim = (float)(K::R * K::R) * kPreBand / ((float)hinv2);
        const float hinv2f = (float)hinv2;
        double f0 = K::F0, gq = 0.0;   // sum f and sum q f' (sum (3 f + q f') = 3 sum f + sum q f')
        float k0 = (float)(12.0 * K::F0);
        const int qs = blockDim.x;
        const float dface = face_distance(xa, ya, za, geo);
        uint32_t k = 0;
        for (;;) {
            int nq = 0;
            float reach = 0.f;   // largest |separation| component of a queued candidate
            while (nq < kDensQueue && k < cnt) {
                const uint32_t b = nb_at(ids, k, st);
                ++k;
                float fx, fy, fz;
                rel_sep(A, qpos[b], geo, fx, fy, fz);
                const float r2f = fx * fx + fy * fy + fz * fz;
                if (r2f > lim) continue;
                queue[(nq++) * qs] = make_uint2(b, __float_as_uint(r2f));
                reach = fmaxf(reach, fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))));
            }
            const int nq_max = __reduce_max_sync(0xffffffffu, (unsigned)nq);
            const bool wrap = __any_sync(0xffffffffu, may_cross_face(reach, dface, geo));
            // the next queued neighbour's position is loaded while the current one is evaluated
            uint2 e = queue[0];
            double bx = 0.0, by = 0.0, bz = 0.0;
            if (nq > 0) {
                bx = x[e.x];
                by = y[e.x];
                bz = z[e.x];
            }
            // the FP64 evaluation, with the nearest-image step only where some lane of the warp may
            // have a neighbour across a periodic face (warp-uniform)
            auto evaluate = [&](auto wrap_c) {
            for (int j = 0; j < nq_max; j++) {
                if (j >= nq) continue;
                const uint2 ec = e;
                const double cx = bx, cy = by, cz = bz;
                if (j + 1 < nq) {
                    e = queue[(j + 1) * qs];
                    bx = x[e.x];
                    by = y[e.x];
                    bz = z[e.x];
                }
                double dx = xa - cx, dy = ya - cy, dz = za - cz;
                if (decltype(wrap_c)::value) {
                    dx = nearest_image(dx, geo.L[0], geo.halfL[0], geo.periodic);
                    dy = nearest_image(dy, geo.L[1], geo.halfL[1], geo.periodic);
                    dz = nearest_image(dz, geo.L[2], geo.halfL[2], geo.periodic);
                }
                const double q2 = (dx * dx + dy * dy + dz * dz) * hinv2;
                if (!nonneg_lt(q2, K::R * K::R)) continue;
                ++nin;
                const float q2f = __uint_as_float(ec.y) * hinv2f;
                const float qf = sqrtf(q2f);
                // q = sqrt(q2) by one Newton-Raphson step from the FP32 root of the FP32 separation
                // (relative error below 1e-13); the two FP32 values are widened by their bits
                // (exact for normal numbers, integer pipe)
                const double q = qf >= 0x1p-126f ? fma(fma(-widen_normal(qf), widen_normal(qf), q2),
                                                       widen_normal(0.5f / qf), widen_normal(qf))
                                                 : sqrt(q2);
                double f, df;
                K::eval(q, f, df);
                f0 += f;
                gq = fma(q, df, gq);
                // sum m d2W/dh2 only carries Omega over the last Newton step (below eps_c h^n, reading
                // of Eq. sphomega): FP32 terms from the FP32 separation are far more accurate than
                // that and keep the FP64 pipe free
                float ff, dff;
                K::eval(qf, ff, dff);
                k0 += 12.f * ff + 8.f * qf * dff + q2f * K::d2(qf);
            }
            };
            if (wrap) evaluate(std::true_type{});
            else evaluate(std::false_type{});
            if (!__any_sync(0xffffffffu, k < cnt)) break;
        }
        sf = f0;
        sg = fma(3.0, f0, gq);
        sk = (double)k0;
    } else {
        // FP32 path: four neighbours per iteration so that four independent gathers are in flight
        const uint4 A = qpos[a];
        const float hi = (float)hinv;
        const float hi2 = hi * hi;
        constexpr float R2 = (float)(K::R * K::R);
        float s0 = (float)K::F0, c0 = 0.f, s1 = (float)(3.0 * K::F0), c1 = 0.f, s2 = (float)(12.0 * K::F0);
        auto acc = [&](const uint4 B) {
            float dx, dy, dz;
            rel_sep(A, B, geo, dx, dy, dz);
            const float q2 = (dx * dx + dy * dy + dz * dz) * hi2;
            if (q2 < R2) {
                ++nin;
                const float q = sqrtf(q2);
                float f, df;
                K::eval(q, f, df);
                const float qdf = q * df;
                kahan_add(s0, c0, f);
                kahan_add(s1, c1, 3.f * f + qdf);
                s2 += 12.f * f + 8.f * qdf + q2 * K::d2(q);   // only scales a step of order eps_c
            }
        };
        // software pipeline: the indices of the next four neighbours are loaded while the current
        // four are gathered and summed
        uint32_t k = 0;
        uint4 nq = make_uint4(0u, 0u, 0u, 0u);
        if (cnt >= 4) nq = nb_quad(ids, 0, st);
        for (; k + 4 <= cnt; k += 4) {
            const uint4 bq = nq;
            if (k + 8 <= cnt) nq = nb_quad(ids, (k >> 2) + 1, st);
            const uint4 B0 = qpos[bq.x], B1 = qpos[bq.y], B2 = qpos[bq.z], B3 = qpos[bq.w];
            acc(B0);
            acc(B1);
            acc(B2);
            acc(B3);
        }
        for (; k < cnt; k++) acc(qpos[nb_at(ids, k, st)]);
        sf = kahan_value(s0, c0);
        sg = kahan_value(s1, c1);
        sk = (double)s2;
    }
}

template <typename K, bool kMixed>
__global__ void __launch_bounds__(256, kMixed ? 4 : 1) k_density(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                                                 const double *__restrict__ z, const uint4 *__restrict__ qpos,
                                                 double *__restrict__ h, const double *__restrict__ h_base,
                                                 const uint32_t *__restrict__ nb_cnt,
                                                 const unsigned long long *__restrict__ nb_ptr,
                                                 const uint32_t *__restrict__ nb_ids, DensParams dp,
                                                 double *__restrict__ rho, double *__restrict__ omega, DevScalars *sc,
                                                 const uint32_t *abort) {
    extern __shared__ uint2 dq[];   // FP64 path: [kDensQueue][blockDim.x], thread t's queue is column t
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // one thread per particle
    if (a - (threadIdx.x & 31) >= n) return;   // whole warp past the end
    if (aborted(abort, kAbortDensity)) return;   // captured step: the cache is incomplete
    int it = 0;
    uint32_t nin = 0, evals = 0, flag = 0;
    // The Newton loop runs while any lane of the warp iterates (the FP64 sums are warp-collective); a
    // lane whose particle has converged, gone stale or hit the cap takes part with no candidates.
    bool active = a < n;
    const int64_t ai = active ? a : 0;
    const uint32_t cnt = active ? nb_cnt[a] : 0u;
    uint32_t st;
    const uint32_t *ids = nb_list(nb_ids, active ? nb_ptr[a] : 0ULL, st);
    double ha = h[ai];
    const double hn = h_base[ai];
    const double m = dp.box_mass ? dp.box_mass[dp.box_of[ai]] : dp.mass;
    const double hf3 = dp.hfact * dp.hfact * dp.hfact;
    bool stale = false, conv = false;
    double dsum_new = 0.0;
    while (__any_sync(0xffffffffu, active)) {
        if (active) ++it;
        double sf, sg, sk;
        density_sums<K, kMixed>(ai, ha, active ? cnt : 0u, ids, st, x, y, z, qpos, dp.geo, sf, sg, sk, nin,
                                dq + threadIdx.x);
        if (!active) continue;
        // one division for 1/h and one for the Newton step; the clamps and tests compare the
        // bits of the doubles (integer pipe) and |dh| <= eps_c h^n needs no quotient
        const double hinv = 1.0 / ha;
        const double hinv3 = hinv * hinv * hinv;
        const double mch3 = m * K::C * hinv3;
        const double rho_sum = mch3 * sf;
        const double dsum = -mch3 * sg * hinv;   // sum_b m dW/dh
        const double rho_h = m * hf3 * hinv3;
        double hnew = ha - (rho_sum - rho_h) / (dsum + 3.0 * rho_h * hinv);
        if (!nan_bits(hnew)) {   // step clamped to [h / lambda, h lambda]
            const double hi_c = ha * dp.h_clamp, lo_c = ha * dp.inv_h_clamp;
            const long long kn = order_key(hnew);
            if (kn > order_key(hi_c)) hnew = hi_c;
            else if (kn < order_key(lo_c)) hnew = lo_c;
        }
        const double dh = hnew - ha;
        const bool small = !nonneg_lt(dp.h_tol * hn, fabs(dh));   // |dh| <= eps_c h^n (NaN: no)
        if (!nan_bits(hnew) && nonneg_lt(hn * dp.chi, hnew)) {
            hnew = hn * dp.chi;
            stale = true;
        }
        // sum m dW/dh at the new h, to first order in the step (|dh| <= eps_c h^n at convergence,
        // so the neglected term is O(eps_c^2))
        dsum_new = dsum + mch3 * sk * hinv * hinv * (hnew - ha);
        ha = hnew;
        if (stale) active = false;
        else if (small) conv = true, active = false;
        else if (it >= dp.max_iter) active = false;
    }
    if (a < n) {
        h[a] = ha;
        flag = stale ? kErrStale : (conv ? 0u : kErrNotConverged);
        // rho = rho(h) (Eq. rhoh) and Omega (Eq. sphomega) at the final h
        const double hinv = 1.0 / ha;
        const double rho_h = m * hf3 * hinv * hinv * hinv;
        rho[a] = rho_h;
        omega[a] = 1.0 + ha / (3.0 * rho_h) * dsum_new;
        evals = cnt * (uint32_t)it;
    }
    // counters: one atomic per warp (same-address atomics from every thread serialise in L2)
    const uint32_t wit = __reduce_max_sync(0xffffffffu, (uint32_t)it);
    const uint32_t wev = __reduce_add_sync(0xffffffffu, evals);
    const uint32_t wnin = __reduce_add_sync(0xffffffffu, nin);
    const uint32_t wfl = __reduce_or_sync(0xffffffffu, flag);
    if ((threadIdx.x & 31) == 0) {
        if (wfl) atomicOr(&sc->flags, wfl);
        atomicMax(&sc->max_iters, wit);
        atomicAdd(&sc->pair_evals, (unsigned long long)wev);
        atomicAdd(&sc->dens_inrange, (unsigned long long)wnin);
    }
}

int density_run(sph_ctx *c, sph_state *s, int *iters, bool *stale) {
    if (!c->cache_valid) return fail(c, SPH_ERR_ORDER, "density before sph_find_neighbours");
    const int64_t n = s->n;
    DensParams dp;
    dp.mass = s->mass;
    dp.hfact = c->p.hfact;
    dp.h_tol = c->p.h_tol;
    dp.h_clamp = c->p.h_clamp;
    dp.inv_h_clamp = 1.0 / c->p.h_clamp;
    dp.chi = c->p.cache_tol;
    dp.max_iter = c->p.h_max_iter;
    dp.geo = make_pair_geo(c->p);
    dp.box_mass = c->batch ? c->box_mass : nullptr;
    dp.box_of = c->batch ? c->box_of : nullptr;
    const int blk = c->launch.density_block;
    if (!c->capturing) SPH_CUDA(c, cudaMemsetAsync(&c->dscal->flags, 0, sizeof(uint32_t), c->stream));
    SPH_CUDA(c, cudaMemsetAsync(&c->dscal->max_iters, 0, sizeof(uint32_t), c->stream));
    SPH_CUDA(c, cudaMemsetAsync(&c->dscal->pair_evals, 0, 2 * sizeof(unsigned long long), c->stream));
    const size_t dsm = (size_t)kDensQueue * blk * sizeof(uint2);
    cudaError_t oe = cudaSuccess;
    with_kernel(c->p.kernel, [&](auto kern) {
        using K = decltype(kern);
        if (c->p.precision != SPH_MIXED) oe = smem_opt_in<k_density<K, false>>(dsm);
        return 0;
    });
    SPH_CUDA(c, oe);
    with_kernel(c->p.kernel, [&](auto kern) {
        using K = decltype(kern);
        if (c->p.precision == SPH_MIXED)
            k_density<K, true><<<grid_for(n, blk), blk, 0, c->stream>>>(n, s->x, s->y, s->z, c->qpos, s->h, c->h_base,
                                                                        c->nb_cnt, c->nb_ptr, c->nb_ids, dp, s->rho,
                                                                        s->omega, c->dscal, abort_word(c));
        else
            k_density<K, false><<<grid_for(n, blk), blk, dsm, c->stream>>>(
                n, s->x, s->y, s->z, c->qpos, s->h, c->h_base,
                                                                         c->nb_cnt, c->nb_ptr, c->nb_ids, dp, s->rho,
                                                                         s->omega, c->dscal, abort_word(c));
        return 0;
    });
    SPH_LAUNCH_CHECK(c, "k_density");
    if (c->capturing) {   // iterations, stale and convergence flags are read back after the step
        *stale = false;
        return SPH_OK;
    }
    static_assert(offsetof(DevScalars, flags) == offsetof(DevScalars, max_iters) + sizeof(uint32_t), "layout");
    SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->max_iters, &c->dscal->max_iters, 2 * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, c->stream));
    SPH_CUDA(c, cudaStreamSynchronize(c->stream));
    SPH_CUDA(c, cudaMemcpyAsync(&c->hscal->pair_evals, &c->dscal->pair_evals, 2 * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, c->stream));
    SPH_CUDA(c, cudaStreamSynchronize(c->stream));
    c->stats.density_pair_evals = (int64_t)c->hscal->pair_evals;
    c->stats.density_inrange = (int64_t)c->hscal->dens_inrange;
    const uint32_t fl = c->hscal->flags;
    const int it = (int)c->hscal->max_iters;
    if (iters) *iters = it;
    c->stats.density_iters_max = it;
    *stale = (fl & kErrStale) != 0;
    if (fl & kErrNotConverged) return fail(c, SPH_ERR_H_NOT_CONVERGED, "h iteration exceeded %d", c->p.h_max_iter);
    c->density_valid = !*stale;
    return SPH_OK;
}

}  // namespace sph

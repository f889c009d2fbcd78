// Kick-drift-kick leapfrog (App. G, "Leapfrog integration"):
//   predictor:  v^{n+1/2} = v^n + dt/2 a^n;  r^{n+1} = r^n + dt v^{n+1/2} (wrapped);  v* = v^{n+1/2} + dt/2 a^n
//               (u advanced the same way with du/dt); h is moved to h + dt dh/dt (clamped to a factor
//               lambda) as the starting guess of the h iteration, dh/dt from the last force pass
//   corrector:  v^{n+1} = v* + dt/2 (a^{n+1} - a^n), likewise u; the correction dv_i (Eq. deltavi) is
//               reduced to max|dv_i| and sum |v_i|^2 for the check of Eq. cvleapfrog.
#include "sph_internal.cuh"

namespace sph {

struct IntParams {
    double dt;
    double h_clamp, inv_h_clamp;
    const double *box_dt;      // time step per box on the device (box_of nullptr: one box) or nullptr
    const uint16_t *box_of;
    double lo[3], hi[3];
    int periodic;
};

// x - L floor((x-lo)/L); a result equal to hi (rounding of a tiny negative offset) becomes lo.
// A particle moves less than a box length per step, so the floor is -1, 0 or 1: taken by compares
// (the same values as the quotient form), with the quotient form kept for anything further out.
__device__ __forceinline__ double wrap(double x, double lo, double hi) {
    const long long kx = order_key(x);
    if (kx >= order_key(lo) && kx < order_key(hi)) return x;   // inside (integer compares; NaN fails)
    const double L = hi - lo;
    double w;
    if (x >= hi && x < hi + L) w = x - L;
    else if (x < lo && x >= lo - L) w = x + L;
    else w = x - L * floor((x - lo) / L);
    if (w >= hi) w = lo;
    if (w < lo) w = lo;
    return w;
}

__global__ void k_predict(int64_t n, double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                          double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                          double *__restrict__ u, const double *__restrict__ ax, const double *__restrict__ ay,
                          const double *__restrict__ az, const double *__restrict__ du, double *__restrict__ h,
                          const double *__restrict__ dhdt, IntParams ip) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dt = ip.box_dt ? ip.box_dt[ip.box_of ? ip.box_of[i] : 0] : ip.dt;
    const double hdt = 0.5 * dt;
    const double kx = hdt * ax[i], ky = hdt * ay[i], kz = hdt * az[i], ku = hdt * du[i];
    const double hvx = vx[i] + kx, hvy = vy[i] + ky, hvz = vz[i] + kz;
    double px = x[i] + dt * hvx, py = y[i] + dt * hvy, pz = z[i] + dt * hvz;
    if (ip.periodic) {
        px = wrap(px, ip.lo[0], ip.hi[0]);
        py = wrap(py, ip.lo[1], ip.hi[1]);
        pz = wrap(pz, ip.lo[2], ip.hi[2]);
    }
    x[i] = px;
    y[i] = py;
    z[i] = pz;
    vx[i] = hvx + kx;
    vy[i] = hvy + ky;
    vz[i] = hvz + kz;
    u[i] = (u[i] + ku) + ku;
    if (dhdt) {
        const double h0 = h[i];
        const double hp = h0 + dt * dhdt[i];
        const double hlo = h0 * ip.inv_h_clamp, hhi = h0 * ip.h_clamp;
        // fmin(fmax(hp, hlo), hhi) by integer compares (NaN gives hlo, as fmax does)
        const long long k = order_key(hp);
        h[i] = (nan_bits(hp) || k < order_key(hlo)) ? hlo : (k > order_key(hhi) ? hhi : hp);
    }
}

__global__ void k_correct(int64_t n, double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                          double *__restrict__ u, double *__restrict__ ax, double *__restrict__ ay,
                          double *__restrict__ az, double *__restrict__ du, const double *__restrict__ anew,
                          int64_t stride, double dt, const double *__restrict__ box_dt,
                          const uint16_t *__restrict__ box_of, DevScalars *sc, double *__restrict__ block_part,
                          const uint32_t *abort) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float dv = 0.f, v2 = 0.f;
    if (i < n && !aborted(abort, kAbortStep)) {
        const double hdt = 0.5 * (box_dt ? box_dt[box_of ? box_of[i] : 0] : dt);
        const double nax = anew[i], nay = anew[stride + i], naz = anew[2 * stride + i], ndu = anew[3 * stride + i];
        const double dvx = hdt * (nax - ax[i]), dvy = hdt * (nay - ay[i]), dvz = hdt * (naz - az[i]);
        const double wx = vx[i] + dvx, wy = vy[i] + dvy, wz = vz[i] + dvz;
        vx[i] = wx;
        vy[i] = wy;
        vz[i] = wz;
        u[i] = u[i] + hdt * (ndu - du[i]);
        ax[i] = nax;
        ay[i] = nay;
        az[i] = naz;
        du[i] = ndu;
        // |dv| and |v|^2 only feed the step-quality ratio of Eq. cvleapfrog: FP32 is enough
        const float fx = (float)dvx, fy = (float)dvy, fz = (float)dvz;
        const float gx = (float)wx, gy = (float)wy, gz = (float)wz;
        dv = sqrtf(fx * fx + fy * fy + fz * fz);
        v2 = gx * gx + gy * gy + gz * gz;
    }
    for (int o = 16; o > 0; o >>= 1) {
        dv = fmaxf(dv, __shfl_xor_sync(0xffffffffu, dv, o));
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    }
    __shared__ double part[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        part[warp] = (double)v2;
        if (dv > 0.f) atomicMax(&sc->dv_max_bits, dbits((double)dv));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += part[w];
        block_part[blockIdx.x] = s;
    }
}

// Corrector pass k > 1 (App. G: the acceleration recomputed with v* <- v^{n+1}): from the saved
// v*, u*, a^n, du^n of the step, v^(k) = v* + dt/2 (a^(k) - a^n), likewise u; the change from the
// previous pass, |v^(k) - v^(k-1)| = dt/2 |a^(k) - a^(k-1)|, and |v^(k)|^2 feed the check of
// Eq. cvleapfrog as in the first pass.  a, du take a^(k), du^(k).
__global__ void k_correct_again(int64_t n, double *__restrict__ vx, double *__restrict__ vy,
                                double *__restrict__ vz, double *__restrict__ u, double *__restrict__ ax,
                                double *__restrict__ ay, double *__restrict__ az, double *__restrict__ du,
                                const double *__restrict__ anew, int64_t stride, const double *__restrict__ save,
                                double dt, const double *__restrict__ box_dt, const uint16_t *__restrict__ box_of,
                                DevScalars *sc, double *__restrict__ block_part, const uint32_t *abort) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float dv = 0.f, v2 = 0.f;
    if (i < n && !aborted(abort, kAbortStep)) {
        const double hdt = 0.5 * (box_dt ? box_dt[box_of ? box_of[i] : 0] : dt);
        const double nax = anew[i], nay = anew[stride + i], naz = anew[2 * stride + i], ndu = anew[3 * stride + i];
        const double ex = hdt * (nax - ax[i]), ey = hdt * (nay - ay[i]), ez = hdt * (naz - az[i]);
        const double wx = save[i] + hdt * (nax - save[4 * stride + i]);
        const double wy = save[stride + i] + hdt * (nay - save[5 * stride + i]);
        const double wz = save[2 * stride + i] + hdt * (naz - save[6 * stride + i]);
        vx[i] = wx;
        vy[i] = wy;
        vz[i] = wz;
        u[i] = save[3 * stride + i] + hdt * (ndu - save[7 * stride + i]);
        ax[i] = nax;
        ay[i] = nay;
        az[i] = naz;
        du[i] = ndu;
        const float fx = (float)ex, fy = (float)ey, fz = (float)ez;
        const float gx = (float)wx, gy = (float)wy, gz = (float)wz;
        dv = sqrtf(fx * fx + fy * fy + fz * fz);
        v2 = gx * gx + gy * gy + gz * gz;
    }
    for (int o = 16; o > 0; o >>= 1) {
        dv = fmaxf(dv, __shfl_xor_sync(0xffffffffu, dv, o));
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    }
    __shared__ double part[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        part[warp] = (double)v2;
        if (dv > 0.f) atomicMax(&sc->dv_max_bits, dbits((double)dv));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += part[w];
        block_part[blockIdx.x] = s;
    }
}

// Deterministic sum of the per-block partials (one block).
__global__ void k_sum_parts(const double *__restrict__ part, int64_t m, double *out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_reset_dv(DevScalars *sc) { sc->dv_max_bits = 0ULL; }

// v*, u*, a^n, du^n of the step into save[8][stride] for the corrector re-runs.
struct SaveArgs {
    const double *src[8];
};
__global__ void k_save(int64_t n, SaveArgs a, int64_t stride, double *__restrict__ save) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int f = 0; f < 8; f++) save[f * stride + i] = a.src[f][i];
}

int integrate_save(sph_ctx *c, sph_state *s) {
    SaveArgs a{{s->vx, s->vy, s->vz, s->u, s->ax, s->ay, s->az, s->du}};
    k_save<<<grid_for(s->n, 256), 256, 0, c->stream>>>(s->n, a, c->n_cap, c->rerun);
    SPH_LAUNCH_CHECK(c, "k_save");
    return SPH_OK;
}

int integrate_predict(sph_ctx *c, sph_state *s, double dt, const double *dhdt) {
    IntParams ip;
    ip.dt = dt;
    ip.h_clamp = c->p.h_clamp;
    ip.inv_h_clamp = 1.0 / c->p.h_clamp;
    ip.box_dt = c->box_dt;   // written by sph_step before the step
    ip.box_of = c->batch ? c->box_of : nullptr;
    for (int k = 0; k < 3; k++) {
        ip.lo[k] = c->p.box_lo[k];
        ip.hi[k] = c->p.box_hi[k];
    }
    ip.periodic = c->p.periodic;
    k_predict<<<grid_for(s->n, 256), 256, 0, c->stream>>>(s->n, s->x, s->y, s->z, s->vx, s->vy, s->vz, s->u, s->ax,
                                                           s->ay, s->az, s->du, s->h, dhdt, ip);
    SPH_LAUNCH_CHECK(c, "k_predict");
    return SPH_OK;
}

int integrate_correct(sph_ctx *c, sph_state *s, double dt) {
    const int64_t n = s->n;
    const unsigned blocks = grid_for(n, 256);
    k_reset_dv<<<1, 1, 0, c->stream>>>(c->dscal);
    SPH_LAUNCH_CHECK(c, "k_reset_dv");
    k_correct<<<blocks, 256, 0, c->stream>>>(n, s->vx, s->vy, s->vz, s->u, s->ax, s->ay, s->az, s->du, c->a_new,
                                             c->n_cap, dt, c->box_dt, c->batch ? c->box_of : nullptr, c->dscal,
                                             c->block_part, abort_word(c));
    SPH_LAUNCH_CHECK(c, "k_correct");
    k_sum_parts<<<1, 256, 0, c->stream>>>(c->block_part, blocks, &c->dscal->v2_sum);
    SPH_LAUNCH_CHECK(c, "k_sum_parts");
    return SPH_OK;
}

int integrate_correct_again(sph_ctx *c, sph_state *s, double dt) {
    const int64_t n = s->n;
    const unsigned blocks = grid_for(n, 256);
    k_reset_dv<<<1, 1, 0, c->stream>>>(c->dscal);
    SPH_LAUNCH_CHECK(c, "k_reset_dv");
    k_correct_again<<<blocks, 256, 0, c->stream>>>(n, s->vx, s->vy, s->vz, s->u, s->ax, s->ay, s->az, s->du,
                                                   c->a_new, c->n_cap, c->rerun, dt, c->box_dt,
                                                   c->batch ? c->box_of : nullptr, c->dscal, c->block_part,
                                                   abort_word(c));
    SPH_LAUNCH_CHECK(c, "k_correct_again");
    k_sum_parts<<<1, 256, 0, c->stream>>>(c->block_part, blocks, &c->dscal->v2_sum);
    SPH_LAUNCH_CHECK(c, "k_sum_parts");
    return SPH_OK;
}

}  // namespace sph

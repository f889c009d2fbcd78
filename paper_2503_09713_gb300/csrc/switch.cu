// Shock detection (App. G, Eq. evolalphaanalytic and its implicit step): per-particle alpha_AV
// evolved towards alpha_loc(v*, grad v*, grad a^n) after the predictor and the h iteration.  The
// switch follows the Phantom scheme the paper cites:
//   (d_j v^i)_a = -1/(Omega_a rho_a) sum_b m (v_a^i - v_b^i) F_ab(h_a) rhat_ab^j  (likewise a^n),
//   d(div v)/dt = div a - (d_i v^j)(d_j v^i),  xi_a = |div v|^2 / (|div v|^2 + |curl v|^2),
//   A_a = xi_a max(-d(div v)/dt, 0),  alpha_loc = max(alpha_min, min(10 h^2 A / c_s^2, alpha_max)),
//   tau_a = h_a / (sigma_decay c_s,a),
//   alpha^{n+1} = max((alpha^n + alpha_loc dt/tau)/(1 + dt/tau), alpha_loc),
// alpha_max = alpha_av.  The sums run over the cached neighbours with r < R_kern h_a.  FP64 path:
// FP64 sums; mixed path: FP32 sums on fixed-point separations (alpha is a limiter: the paper notes
// that Phantom keeps alpha and div v in single precision).
#include "physics.cuh"

namespace sph {

struct SwitchParams {
    double mass, hfact, gamma, alpha_max, alpha_min, sigma_decay, dt;
    const double *box_mass, *box_gamma, *box_dt;
    const uint16_t *box_of;
    PairGeo geo;
    const uint32_t *abort;     // captured step: skip when an earlier stage failed
};

template <typename K, bool kMixed>
__global__ void __launch_bounds__(128) k_alpha(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                                               const double *__restrict__ z, const uint4 *__restrict__ qpos,
                                               const double *__restrict__ vx, const double *__restrict__ vy,
                                               const double *__restrict__ vz, const double *__restrict__ ax,
                                               const double *__restrict__ ay, const double *__restrict__ az,
                                               const double *__restrict__ u, const double *__restrict__ h,
                                               const double *__restrict__ omega, const uint32_t *__restrict__ nb_cnt,
                                               const unsigned long long *__restrict__ nb_ptr,
                                               const uint32_t *__restrict__ nb_ids, SwitchParams sp,
                                               double *__restrict__ alpha) {
    using T = typename std::conditional<kMixed, float, double>::type;
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n || aborted(sp.abort, kAbortStep)) return;
    const int box = sp.box_of ? sp.box_of[a] : 0;
    const double m = sp.box_mass ? sp.box_mass[box] : sp.mass;
    const double gam = sp.box_gamma ? sp.box_gamma[box] : sp.gamma;
    const double dt = sp.box_dt ? sp.box_dt[box] : sp.dt;
    const uint32_t cnt = nb_cnt[a];
    uint32_t st;
    const uint32_t *ids = nb_list(nb_ids, nb_ptr[a], st);
    const double ha = h[a];
    const T hinv = (T)(1.0 / ha);
    const T fn = (T)(K::C) * hinv * hinv * hinv * hinv;   // F_ab(h_a) = C f'(q) / h^4
    const T R2 = (T)(K::R * K::R);
    const T vax = (T)vx[a], vay = (T)vy[a], vaz = (T)vz[a];
    const T aax = (T)ax[a], aay = (T)ay[a], aaz = (T)az[a];
    T G[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
    T diva = T(0);
    const uint4 A = qpos[a];
    const double xa = x[a], ya = y[a], za = z[a];
    for (uint32_t k = 0; k < cnt; k++) {
        const uint32_t b = nb_at(ids, k, st);
        T dx, dy, dz;
        if (kMixed) {
            float fx, fy, fz;
            rel_sep(A, qpos[b], sp.geo, fx, fy, fz);
            dx = (T)fx; dy = (T)fy; dz = (T)fz;
        } else {
            dx = (T)nearest_image(xa - x[b], sp.geo.L[0], sp.geo.halfL[0], sp.geo.periodic);
            dy = (T)nearest_image(ya - y[b], sp.geo.L[1], sp.geo.halfL[1], sp.geo.periodic);
            dz = (T)nearest_image(za - z[b], sp.geo.L[2], sp.geo.halfL[2], sp.geo.periodic);
        }
        const T r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 * hinv * hinv < R2) || !(r2 > T(0))) continue;
        const T rinv = T(1) / sqrt(r2);
        T f, df;
        K::eval(sqrt(r2) * hinv, f, df);
        const T w = df * fn * rinv;   // F_ab(h_a) / r: times (r_a - r_b)^j gives F rhat^j
        const T dv[3] = {vax - (T)vx[b], vay - (T)vy[b], vaz - (T)vz[b]};
        const T d[3] = {dx, dy, dz};
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) G[i][j] += dv[i] * w * d[j];
        diva += ((aax - (T)ax[b]) * dx + (aay - (T)ay[b]) * dy + (aaz - (T)az[b]) * dz) * w;
    }
    const double rho = m * (sp.hfact / ha) * (sp.hfact / ha) * (sp.hfact / ha);
    const double fac = -m / (omega[a] * rho);
    double g[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) g[i][j] = fac * (double)G[i][j];   // d_j v^i
    const double div_a = fac * (double)diva;
    const double divv = g[0][0] + g[1][1] + g[2][2];
    const double cx = g[2][1] - g[1][2], cy = g[0][2] - g[2][0], cz = g[1][0] - g[0][1];
    double tr = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) tr += g[i][j] * g[j][i];
    const double ddiv = div_a - tr;
    const double den = divv * divv + (cx * cx + cy * cy + cz * cz);
    const double xi = den > 0.0 ? divv * divv / den : 0.0;
    const double Aa = xi * (ddiv < 0.0 ? -ddiv : 0.0);
    const double cs = sqrt(gam * (gam - 1.0) * u[a]);
    double aloc = Aa > 0.0 ? sp.alpha_max : 0.0;   // c_s = 0: the limit of the ratio
    if (cs > 0.0) aloc = fmin(10.0 * ha * ha * Aa / (cs * cs), sp.alpha_max);
    aloc = fmax(aloc, sp.alpha_min);
    const double q = cs > 0.0 ? dt * sp.sigma_decay * cs / ha : 0.0;   // dt / tau
    const double an = (alpha[a] + aloc * q) / (1.0 + q);
    alpha[a] = fmax(an, aloc);
}

int switch_run(sph_ctx *c, sph_state *s, double dt) {
    if (!c->cache_valid) return fail(c, SPH_ERR_ORDER, "shock switch before sph_find_neighbours");
    if (!s->alpha) return fail(c, SPH_ERR_INVALID_ARG, "av_switch needs sph_state.alpha");
    const int64_t n = s->n;
    SwitchParams sp;
    sp.mass = s->mass;
    sp.hfact = c->p.hfact;
    sp.gamma = c->p.gamma;
    sp.alpha_max = c->p.alpha_av;
    sp.alpha_min = c->p.alpha_min;
    sp.sigma_decay = c->p.sigma_decay;
    sp.dt = dt;
    sp.box_mass = c->batch ? c->box_mass : nullptr;
    sp.box_gamma = c->batch ? c->box_gamma : nullptr;
    sp.box_dt = c->box_dt;   // written by sph_step before the step
    sp.box_of = c->batch ? c->box_of : nullptr;
    sp.geo = make_pair_geo(c->p);
    sp.abort = abort_word(c);
    with_kernel(c->p.kernel, [&](auto kern) {
        using K = decltype(kern);
        if (c->p.precision == SPH_MIXED)
            k_alpha<K, true><<<grid_for(n, 128), 128, 0, c->stream>>>(
                n, s->x, s->y, s->z, c->qpos, s->vx, s->vy, s->vz, s->ax, s->ay, s->az, s->u, s->h, s->omega,
                c->nb_cnt, c->nb_ptr, c->nb_ids, sp, s->alpha);
        else
            k_alpha<K, false><<<grid_for(n, 128), 128, 0, c->stream>>>(
                n, s->x, s->y, s->z, c->qpos, s->vx, s->vy, s->vz, s->ax, s->ay, s->az, s->u, s->h, s->omega,
                c->nb_cnt, c->nb_ptr, c->nb_ids, sp, s->alpha);
        return 0;
    });
    SPH_LAUNCH_CHECK(c, "k_alpha");
    return SPH_OK;
}

}  // namespace sph

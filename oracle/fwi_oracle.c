/*
 * fwi_oracle.c -- plain, slow FP64 CPU oracle for the likelihood-guidance
 * gradient of "Robust Physics-Guided Diffusion for Full-Waveform Inversion"
 * (arXiv 2603.16393).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: it exists so that tests, the smoke check and the timed CPU
 * baseline can compare the CUDA library against an independent, readable
 * definition of what the method computes.  It shares no code, header, table
 * or constant generator with the CUDA library.
 *
 * Every function is single-threaded plain loops in double precision; callers
 * parallelise over independent (model, shot) units.
 *
 * Readings of the paper that this file fixes (the paper is silent or
 * ambiguous on them; the same readings are listed in the design notes):
 *   - 4th-order central Laplacian (the paper's solver is 8th order, Sec. 6.1;
 *     the hot path is specified at 4th order), 2nd-order leapfrog in time.
 *   - Absorbing layer: a damping sponge of width nb on the left, right and
 *     bottom sides, eta = eta0x (dx_cells/nb)^2 + eta0z (dz_cells/nb)^2 with
 *     eta0 = 3 v_ref ln(1/R) / (nb h) per axis, so that a wave at v_ref that
 *     crosses the layer and back is damped by exp(-int eta/2 dt) = R; the
 *     damped leapfrog is
 *     u+ = A (2u - B u- + kappa (L u + s)), A = 1/(1+eta dt/2), B = 1-eta dt/2.
 *   - Velocity in the layer is the edge-replicated physical model; its
 *     gradient is folded back onto the physical cell it copies.
 *   - Top boundary: top_bc = 0 puts zero ghost values above row 0;
 *     top_bc = 1 mirrors rows 1,2 into the ghosts (du/dn = 0, Eq. 1).
 *   - Source term s = f(n dt)/(dx dz) at the source cell (a discrete delta,
 *     Sec. 6.1); sample n of a trace is u^{n+1} at the receiver cell and sits
 *     at time t_n = n dt on the W2 time axis (Sec. 6.2).
 *   - W2: trapezoid CDF on t_k, generalised-inverse quantile with linear
 *     interpolation, trapezoid rule in xi on xi_j = j/(Nxi-1) (Sec. 6.2);
 *     J = sum W2 / S_obs (Eq. final_objective).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(iz, ix, NX) ((size_t)(iz) * (size_t)(NX) + (size_t)(ix))

/* ------------------------------------------------------------------------ */
/* Source wavelet, Sec. 6.1: f(t) = (1 - 2 pi^2 fp^2 (t-t0)^2) exp(-pi^2 fp^2 (t-t0)^2) */
double orc_ricker(double t, double fp, double t0)
{
    const double pi = 3.14159265358979323846;
    double a = pi * pi * fp * fp * (t - t0) * (t - t0);
    return (1.0 - 2.0 * a) * exp(-a);
}

void orc_ricker_series(int nt, double dt, double fp, double t0, double *f)
{
    for (int n = 0; n < nt; ++n)
        f[n] = orc_ricker((double)n * dt, fp, t0);
}

/* ------------------------------------------------------------------------ */
/* Model padding (reading C-5): the padded grid has NZ = nz + nb rows (no layer
 * above row 0, the reflecting top of Eq. 1) and NX = nx + 2 nb columns; every
 * padded cell copies the nearest physical cell. */
void orc_pad_model(int nz, int nx, int nb, const double *v, double *vpad)
{
    int NZ = nz + nb, NX = nx + 2 * nb;
    for (int pz = 0; pz < NZ; ++pz) {
        int iz = pz < nz ? pz : nz - 1;
        for (int px = 0; px < NX; ++px) {
            int ix = px - nb;
            if (ix < 0) ix = 0;
            if (ix > nx - 1) ix = nx - 1;
            vpad[IDX(pz, px, NX)] = v[IDX(iz, ix, nx)];
        }
    }
}

/* Fold of a padded-grid gradient onto the physical grid: the exact transpose
 * of orc_pad_model (each padded cell adds into the cell it copies). */
void orc_fold_add(int nz, int nx, int nb, const double *gpad, double *g)
{
    int NZ = nz + nb, NX = nx + 2 * nb;
    for (int pz = 0; pz < NZ; ++pz) {
        int iz = pz < nz ? pz : nz - 1;
        for (int px = 0; px < NX; ++px) {
            int ix = px - nb;
            if (ix < 0) ix = 0;
            if (ix > nx - 1) ix = nx - 1;
            g[IDX(iz, ix, nx)] += gpad[IDX(pz, px, NX)];
        }
    }
}

/* Damping profile eta(pz, px) in 1/s on the padded grid (reading C-4). */
void orc_damping(int nz, int nx, int nb, double dz, double dx, double v_ref,
                 double refl_R, double *eta)
{
    int NZ = nz + nb, NX = nx + 2 * nb;
    double lnR = log(1.0 / refl_R);
    double eta0x = nb > 0 ? 3.0 * v_ref * lnR / (nb * dx) : 0.0;
    double eta0z = nb > 0 ? 3.0 * v_ref * lnR / (nb * dz) : 0.0;
    for (int pz = 0; pz < NZ; ++pz) {
        double cz = pz > nz - 1 ? (double)(pz - (nz - 1)) : 0.0;
        for (int px = 0; px < NX; ++px) {
            double cx = 0.0;
            if (px < nb) cx = (double)(nb - px);
            if (px > nb + nx - 1) cx = (double)(px - (nb + nx - 1));
            double e = 0.0;
            if (nb > 0)
                e = eta0x * (cx / nb) * (cx / nb) + eta0z * (cz / nb) * (cz / nb);
            eta[IDX(pz, px, NX)] = e;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Central second-derivative weights: 4th order (-1/12, 4/3, -5/2, 4/3, -1/12),
 * the hot path's; 8th order (-1/560, 8/315, -1/5, 8/5, -205/72, ...), the
 * space order of the paper's solver (Sec. 6.1). */
static const double W4[5] = {-1.0 / 12.0, 4.0 / 3.0, -5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0};
static const double W8[9] = {-1.0 / 560.0, 8.0 / 315.0, -1.0 / 5.0, 8.0 / 5.0, -205.0 / 72.0,
                             8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

/* weights and radius of a space order (4 or 8) */
static const double *stencil(int order, int *radius)
{
    *radius = order == 8 ? 4 : 2;
    return order == 8 ? W8 : W4;
}

/* Value of u at (pz, px) with the boundary treatment of the padded grid:
 * outside left/right/bottom -> 0; above row 0 -> 0 (top_bc = 0) or the
 * mirrored row (top_bc = 1: u[-k] = u[k]).  Returns the cell index used, or
 * -1 for a zero ghost. */
static long ghost_map(int NZ, int NX, int top_bc, int pz, int px)
{
    if (px < 0 || px >= NX || pz >= NZ) return -1;
    if (pz < 0) {
        if (top_bc == 0) return -1;
        pz = -pz;
        if (pz >= NZ) return -1;
    }
    return (long)IDX(pz, px, NX);
}

/* out = L u, gather form: out[p] = sum_q w(p,q) u[q]. */
void orc_laplacian(int NZ, int NX, double dz, double dx, int top_bc, int order,
                   const double *u, double *out)
{
    int R;
    const double *W = stencil(order, &R);
    for (int pz = 0; pz < NZ; ++pz)
        for (int px = 0; px < NX; ++px) {
            double s = 0.0;
            for (int m = -R; m <= R; ++m) {
                long qx = ghost_map(NZ, NX, top_bc, pz, px + m);
                if (qx >= 0) s += W[m + R] * u[qx] / (dx * dx);
                long qz = ghost_map(NZ, NX, top_bc, pz + m, px);
                if (qz >= 0) s += W[m + R] * u[qz] / (dz * dz);
            }
            out[IDX(pz, px, NX)] = s;
        }
}

/* out = L^T w, scatter form of the very same stencil: every weight w(p,q)
 * used by orc_laplacian moves w[p] into out[q].  Equal to orc_laplacian for
 * top_bc = 0 (symmetric operator), different for top_bc = 1. */
void orc_laplacian_T(int NZ, int NX, double dz, double dx, int top_bc, int order,
                     const double *w, double *out)
{
    int R;
    const double *W = stencil(order, &R);
    size_t n = (size_t)NZ * NX;
    for (size_t i = 0; i < n; ++i) out[i] = 0.0;
    for (int pz = 0; pz < NZ; ++pz)
        for (int px = 0; px < NX; ++px) {
            double wp = w[IDX(pz, px, NX)];
            for (int m = -R; m <= R; ++m) {
                long qx = ghost_map(NZ, NX, top_bc, pz, px + m);
                if (qx >= 0) out[qx] += W[m + R] * wp / (dx * dx);
                long qz = ghost_map(NZ, NX, top_bc, pz + m, px);
                if (qz >= 0) out[qz] += W[m + R] * wp / (dz * dz);
            }
        }
}

/* ------------------------------------------------------------------------ */
/* Forward solve of Eq. (1) for one shot on the padded grid (Sec. 2.1, 6.1).
 *   u^{-1} = u^0 = 0
 *   u^{n+1} = A (2 u^n - B u^{n-1} + kappa (L u^n + s^n)),  n = 0..nt-1
 *   kappa = vpad^2 dt^2, s^n = f[n]/(dx dz) at the source cell
 *   d[r][n] = u^{n+1} at receiver r   (restriction R, Sec. 2.1)
 * u_all (optional, (nt+1) x NZ x NX) receives u^0 .. u^nt. */
void orc_forward_shot(int NZ, int NX, int top_bc, int order, int nt, double dz, double dx,
                      double dt, const double *vpad, const double *eta,
                      const double *wavelet, int src_pz, int src_px,
                      int nrec, const int *rec_pz, const int *rec_px,
                      double *d, double *u_all)
{
    size_t n = (size_t)NZ * NX;
    double *um = calloc(n, sizeof(double));   /* u^{n-1} */
    double *u0 = calloc(n, sizeof(double));   /* u^n     */
    double *up = calloc(n, sizeof(double));   /* u^{n+1} */
    double *lap = calloc(n, sizeof(double));
    if (u_all) memset(u_all, 0, n * sizeof(double));   /* u^0 */
    for (int it = 0; it < nt; ++it) {
        orc_laplacian(NZ, NX, dz, dx, top_bc, order, u0, lap);
        lap[IDX(src_pz, src_px, NX)] += wavelet[it] / (dx * dz);
        for (size_t i = 0; i < n; ++i) {
            double A = 1.0 / (1.0 + eta[i] * dt / 2.0);
            double B = 1.0 - eta[i] * dt / 2.0;
            double kappa = vpad[i] * vpad[i] * dt * dt;
            up[i] = A * (2.0 * u0[i] - B * um[i] + kappa * lap[i]);
        }
        for (int r = 0; r < nrec; ++r)
            d[(size_t)r * nt + it] = up[IDX(rec_pz[r], rec_px[r], NX)];
        if (u_all) memcpy(u_all + (size_t)(it + 1) * n, up, n * sizeof(double));
        double *tmp = um; um = u0; u0 = up; up = tmp;
    }
    free(um); free(u0); free(up); free(lap);
}

/* Discrete adjoint of orc_forward_shot (the exact transpose of the recurrence,
 * i.e. what reverse-mode differentiation of the solver produces, Sec. 5.2
 * "automatic differentiation" and the F'* of the DPS step, Sec. 4.2).
 *   mu^{nt+1} = mu^{nt+2} = 0
 *   mu^m = R^T r[., m-1] + 2 A mu^{m+1} + L^T(kappa A mu^{m+1}) - A B mu^{m+2}
 *   dJ/dkappa = sum_{n=0}^{nt-1} mu^{n+1} A (L u^n + s^n)
 *   dJ/dvpad  = dJ/dkappa * 2 vpad dt^2
 * adj is r = dJ/dd, nrec x nt; u_all holds u^0..u^{nt-1} from the forward. */
void orc_adjoint_shot(int NZ, int NX, int top_bc, int order, int nt, double dz, double dx,
                      double dt, const double *vpad, const double *eta,
                      const double *wavelet, int src_pz, int src_px,
                      int nrec, const int *rec_pz, const int *rec_px,
                      const double *adj, const double *u_all, double *grad_vpad)
{
    size_t n = (size_t)NZ * NX;
    double *mu1 = calloc(n, sizeof(double));   /* mu^{m+1} */
    double *mu2 = calloc(n, sizeof(double));   /* mu^{m+2} */
    double *mu = calloc(n, sizeof(double));    /* mu^m     */
    double *tmp = calloc(n, sizeof(double));
    double *ltmp = calloc(n, sizeof(double));
    double *lu = calloc(n, sizeof(double));
    double *gk = calloc(n, sizeof(double));
    for (int m = nt; m >= 1; --m) {
        for (size_t i = 0; i < n; ++i) {
            double A = 1.0 / (1.0 + eta[i] * dt / 2.0);
            double kappa = vpad[i] * vpad[i] * dt * dt;
            tmp[i] = kappa * A * mu1[i];
        }
        orc_laplacian_T(NZ, NX, dz, dx, top_bc, order, tmp, ltmp);
        for (size_t i = 0; i < n; ++i) {
            double A = 1.0 / (1.0 + eta[i] * dt / 2.0);
            double B = 1.0 - eta[i] * dt / 2.0;
            mu[i] = 2.0 * A * mu1[i] + ltmp[i] - A * B * mu2[i];
        }
        for (int r = 0; r < nrec; ++r)
            mu[IDX(rec_pz[r], rec_px[r], NX)] += adj[(size_t)r * nt + (m - 1)];
        /* imaging term for forward step n = m-1 */
        orc_laplacian(NZ, NX, dz, dx, top_bc, order, u_all + (size_t)(m - 1) * n, lu);
        lu[IDX(src_pz, src_px, NX)] += wavelet[m - 1] / (dx * dz);
        for (size_t i = 0; i < n; ++i) {
            double A = 1.0 / (1.0 + eta[i] * dt / 2.0);
            gk[i] += mu[i] * A * lu[i];
        }
        double *t = mu2; mu2 = mu1; mu1 = mu; mu = t;
    }
    for (size_t i = 0; i < n; ++i)
        grad_vpad[i] = gk[i] * 2.0 * vpad[i] * dt * dt;
    free(mu1); free(mu2); free(mu); free(tmp); free(ltmp); free(lu); free(gk);
}

/* ------------------------------------------------------------------------ */
/* W2 pieces, Sec. 5.1 (II) and Sec. 6.2. */

/* Trapezoid integral of y over t_0..t_{nt-1}. */
static double trapz(int nt, double dt, const double *y)
{
    double s = 0.0;
    for (int k = 0; k < nt; ++k) s += y[k];
    return dt * (s - 0.5 * (y[0] + y[nt - 1]));
}

/* Density and CDF of a nonnegative signal y (Eq. pdf_map with the eps' of
 * Sec. 6.2): p = y / (int y + eps), F_0 = 0, F_k = F_{k-1} + dt (p_{k-1}+p_k)/2. */
void orc_cdf(int nt, double dt, double eps, const double *y, double *p,
             double *F, double *Z)
{
    double z = trapz(nt, dt, y);
    for (int k = 0; k < nt; ++k) p[k] = y[k] / (z + eps);
    F[0] = 0.0;
    for (int k = 1; k < nt; ++k) F[k] = F[k - 1] + dt * 0.5 * (p[k - 1] + p[k]);
    *Z = z;
}

/* Quantiles Q_j = F^{-1}(xi_j), xi_j = j/(nxi-1), generalised inverse
 * inf{t : F(t) >= xi} with F linear between samples (Eq. Wp_1d, Sec. 6.2):
 *   k* = min{k : F_k >= xi}; k* = 0 -> t_0; no such k -> t_{nt-1};
 *   else t_{k*-1} + dt (xi - F_{k*-1}) / (F_{k*} - F_{k*-1}).
 * kstar[j] receives k* (nt when no such k).  Because xi_j increases with j,
 * the set {k : F_k >= xi_{j+1}} is contained in {k : F_k >= xi_j}, so the
 * search for j+1 may start at k*_j. */
void orc_quantiles(int nt, double dt, int nxi, const double *F, double *Q,
                   int *kstar)
{
    int k = 0;
    for (int j = 0; j < nxi; ++j) {
        double xi = (double)j / (double)(nxi - 1);
        while (k < nt && F[k] < xi) ++k;
        double q;
        if (k == 0) q = 0.0;
        else if (k == nt) q = (double)(nt - 1) * dt;
        else q = (double)(k - 1) * dt + dt * (xi - F[k - 1]) / (F[k] - F[k - 1]);
        Q[j] = q;
        if (kstar) kstar[j] = k;
    }
}

/* Trapezoid weight of node j on the xi grid. */
static double xi_weight(int j, int nxi)
{
    return (j == 0 || j == nxi - 1) ? 0.5 : 1.0;
}

/* (int_0^1 |Qa - Qb|^2 dxi)^(1/2) by the trapezoid rule on the xi grid. */
double orc_w2_from_quantiles(int nxi, const double *Qa, const double *Qb)
{
    double dxi = 1.0 / (double)(nxi - 1), s = 0.0;
    for (int j = 0; j < nxi; ++j) {
        double dq = Qa[j] - (Qb ? Qb[j] : 0.0);
        s += xi_weight(j, nxi) * dq * dq;
    }
    return sqrt(dxi * s);
}

/* W2 between two nonnegative signals through the density map (no weighting,
 * no shift): used to pin the density/quantile routine against closed forms. */
double orc_w2_signals(int nt, double dt, double eps, int nxi, const double *ya,
                      const double *yb)
{
    double *p = malloc(sizeof(double) * nt), *F = malloc(sizeof(double) * nt);
    double *Qa = malloc(sizeof(double) * nxi), *Qb = malloc(sizeof(double) * nxi);
    double Z;
    orc_cdf(nt, dt, eps, ya, p, F, &Z);
    orc_quantiles(nt, dt, nxi, F, Qa, NULL);
    orc_cdf(nt, dt, eps, yb, p, F, &Z);
    orc_quantiles(nt, dt, nxi, F, Qb, NULL);
    double w = orc_w2_from_quantiles(nxi, Qa, Qb);
    free(p); free(F); free(Qa); free(Qb);
    return w;
}

/* Observation preparation for one instance (one observed data cube
 * d_obs[ntr][nt], ntr = Ns*Nr traces):
 *   M = max |d_obs|                                   (Sec. 5.1 (I))
 *   omega = 1 / (1 + k |d_obs| / M)                   (Eq. omega_def)
 *   c'    = cfac |min_t omega d_obs|  per trace       (Sec. 5.1 (II), 6.2)
 *   Q_obs = quantiles of P(omega d_obs + c')          (Eq. pdf_map, Wp_1d)
 *   s_tr  = (int_0^1 |Q_obs|^2)^(1/2) per trace, S_obs = sum s_tr  (Sec. 5.1 (III))
 * Returns S_obs; M is written to *Mout. */
double orc_w2_prepare(int ntr, int nt, double dt, double k, double cfac,
                      double eps, int nxi, const double *dobs, double *omega,
                      double *cshift, double *Qobs, double *s_tr, double *Mout)
{
    size_t N = (size_t)ntr * nt;
    double M = 0.0;
    for (size_t i = 0; i < N; ++i)
        if (fabs(dobs[i]) > M) M = fabs(dobs[i]);
    for (size_t i = 0; i < N; ++i) {
        double a = M > 0.0 ? fabs(dobs[i]) / M : 0.0;
        omega[i] = 1.0 / (1.0 + k * a);
    }
    double *y = malloc(sizeof(double) * nt), *p = malloc(sizeof(double) * nt);
    double *F = malloc(sizeof(double) * nt);
    double S = 0.0;
    for (int tr = 0; tr < ntr; ++tr) {
        const double *d = dobs + (size_t)tr * nt;
        const double *w = omega + (size_t)tr * nt;
        double mn = w[0] * d[0];
        for (int t = 1; t < nt; ++t)
            if (w[t] * d[t] < mn) mn = w[t] * d[t];
        double c = cfac * fabs(mn);
        cshift[tr] = c;
        for (int t = 0; t < nt; ++t) y[t] = w[t] * d[t] + c;
        double Z;
        orc_cdf(nt, dt, eps, y, p, F, &Z);
        double *Q = Qobs + (size_t)tr * nxi;
        orc_quantiles(nt, dt, nxi, F, Q, NULL);
        s_tr[tr] = orc_w2_from_quantiles(nxi, Q, NULL);
        S += s_tr[tr];
    }
    free(y); free(p); free(F);
    *Mout = M;
    return S;
}

/* Weighted, normalised W2 misfit of ntr traces (Eq. final_objective) and its
 * exact derivative with respect to d_syn (the adjoint source).
 *   y = omega d_syn + c', p, F, Q_syn as in orc_cdf / orc_quantiles
 *   W2_tr = (trapz_xi (Q_obs - Q_syn)^2)^(1/2);  returns sum_tr W2_tr / S_obs
 * The derivative is written by reversing each step above by hand:
 *   Q_syn,j  <- dJ/dQ_j = dxi w_j (Q_syn,j - Q_obs,j) / (W2 S_obs)  (0 if W2 = 0)
 *   F_{k*-1}, F_{k*} <- through the interpolation formula (zero in the clamped cases)
 *   p <- the CDF recurrence walked backwards
 *   y <- p = y/(Z+eps) with Z = trapz(y)
 *   d_syn <- y = omega d_syn + c'
 * adj (nullable) has the layout of d_syn. */
double orc_w2_misfit(int ntr, int nt, double dt, double eps, int nxi,
                     const double *dsyn, const double *omega,
                     const double *cshift, const double *Qobs, double S_obs,
                     int squared, double *w2_out, double *adj)
{
    double *y = malloc(sizeof(double) * nt), *p = malloc(sizeof(double) * nt);
    double *F = malloc(sizeof(double) * nt), *Q = malloc(sizeof(double) * nxi);
    int *ks = malloc(sizeof(int) * nxi);
    double *Fbar = malloc(sizeof(double) * nt), *pbar = malloc(sizeof(double) * nt);
    double dxi = 1.0 / (double)(nxi - 1);
    double J = 0.0;
    for (int tr = 0; tr < ntr; ++tr) {
        const double *d = dsyn + (size_t)tr * nt;
        const double *w = omega + (size_t)tr * nt;
        const double *Qo = Qobs + (size_t)tr * nxi;
        for (int t = 0; t < nt; ++t) y[t] = w[t] * d[t] + cshift[tr];
        double Z;
        orc_cdf(nt, dt, eps, y, p, F, &Z);
        orc_quantiles(nt, dt, nxi, F, Q, ks);
        double W2 = orc_w2_from_quantiles(nxi, Q, Qo);
        /* squared: the raw baseline objective sum W2^2 / sum int |Qobs|^2
         * (Sec. 6.3, Baseline 1), S_obs then holding the denominator */
        double term = squared ? W2 * W2 : W2;
        if (w2_out) w2_out[tr] = term;
        J += term / S_obs;
        if (!adj) continue;
        double *a = adj + (size_t)tr * nt;
        if (!squared && W2 == 0.0) {   /* reading C-10: non-differentiable point, take 0 */
            for (int t = 0; t < nt; ++t) a[t] = 0.0;
            continue;
        }
        for (int t = 0; t < nt; ++t) Fbar[t] = 0.0;
        for (int j = 0; j < nxi; ++j) {
            int kk = ks[j];
            if (kk == 0 || kk == nt) continue;   /* clamped quantile */
            double xi = (double)j * dxi;
            double qbar = squared ? 2.0 * dxi * xi_weight(j, nxi) * (Q[j] - Qo[j]) / S_obs
                                  : dxi * xi_weight(j, nxi) * (Q[j] - Qo[j]) / (W2 * S_obs);
            double D = F[kk] - F[kk - 1];
            Fbar[kk - 1] += qbar * dt * (xi - F[kk]) / (D * D);
            Fbar[kk] += qbar * (-dt * (xi - F[kk - 1]) / (D * D));
        }
        /* reverse of F_k = F_{k-1} + dt (p_{k-1} + p_k)/2, k = nt-1 .. 1; F_0 = 0 is constant */
        for (int t = 0; t < nt; ++t) pbar[t] = 0.0;
        for (int kk = nt - 1; kk >= 1; --kk) {
            pbar[kk - 1] += 0.5 * dt * Fbar[kk];
            pbar[kk] += 0.5 * dt * Fbar[kk];
            Fbar[kk - 1] += Fbar[kk];
        }
        /* reverse of p_t = y_t / (Z + eps), Z = dt (sum y - (y_0 + y_{nt-1})/2) */
        double zbar = 0.0;
        for (int t = 0; t < nt; ++t) zbar -= pbar[t] * y[t] / ((Z + eps) * (Z + eps));
        for (int t = 0; t < nt; ++t) {
            double wt = (t == 0 || t == nt - 1) ? 0.5 : 1.0;
            double ybar = pbar[t] / (Z + eps) + zbar * dt * wt;
            a[t] = w[t] * ybar;   /* y = omega d + c' */
        }
    }
    free(y); free(p); free(F); free(Q); free(ks); free(Fbar); free(pbar);
    return J;
}

/* ------------------------------------------------------------------------ */
/* Preconditioned guided update of one instance, Sec. 5.2 and Algorithm 2:
 *   TV(v0hat) = (1/Ng) sum (|grad_x v| + |grad_z v|), forward differences,
 *               a difference that would leave the grid counts as 0  (Eq. tv)
 *   rho   = rho0 exp(-(TV - tau)_+ / c)                             (Eq. rho)
 *   kappa_j = ((||g||_inf + eps) / (|g_j| + eps))^gamma, optionally clipped
 *             to [kmin, kmax] when kmin < kmax                       (Eq. kappa)
 *   v_out = v' - rho kappa . h                                       (Eq. precond_step)
 * Arrays are nz x nx, row-major (z slow).  Returns rho. */
double orc_guided_step(int nz, int nx, double rho0, double c, double tau,
                       double gamma, double eps, double kmin, double kmax,
                       const double *vprime, const double *v0hat,
                       const double *g, const double *h, double *vout)
{
    double tv = 0.0;
    for (int iz = 0; iz < nz; ++iz)
        for (int ix = 0; ix < nx; ++ix) {
            double v = v0hat[IDX(iz, ix, nx)];
            if (ix + 1 < nx) tv += fabs(v0hat[IDX(iz, ix + 1, nx)] - v);
            if (iz + 1 < nz) tv += fabs(v0hat[IDX(iz + 1, ix, nx)] - v);
        }
    tv /= (double)nz * (double)nx;
    double excess = tv - tau > 0.0 ? tv - tau : 0.0;
    double rho = rho0 * exp(-excess / c);
    double ginf = 0.0;
    size_t n = (size_t)nz * nx;
    for (size_t i = 0; i < n; ++i)
        if (fabs(g[i]) > ginf) ginf = fabs(g[i]);
    for (size_t i = 0; i < n; ++i) {
        double kap = pow((ginf + eps) / (fabs(g[i]) + eps), gamma);
        if (kmin < kmax) {
            if (kap < kmin) kap = kmin;
            if (kap > kmax) kap = kmax;
        }
        vout[i] = vprime[i] - rho * kap * h[i];
    }
    return rho;
}

/* ------------------------------------------------------------------------ */
/* Least-squares potential of the DPS baseline (Sec. 4.2, Baseline 3):
 *   J = (1/2) sum (d_syn - d_obs)^2 / sigma^2,  adj = dJ/dd_syn = (d_syn - d_obs) / sigma^2
 * over n samples of one instance.  Returns J. */
double orc_l2_misfit(long n, double sigma2, const double *dobs, const double *dsyn,
                     double *adj)
{
    double J = 0.0;
    for (long i = 0; i < n; ++i) {
        double r = dsyn[i] - dobs[i];
        J += 0.5 * r * r / sigma2;
        if (adj) adj[i] = r / sigma2;
    }
    return J;
}

/* Total variation of the normalised field u = v / unit (Eq. tv, forward
 * differences, a difference leaving the grid counts as 0, divided by
 * N_g = nz nx) and h = g + alpha dTV(v / unit)/dv, the subgradient taking
 * sign(0) = 0 (the (sub)gradient steps of Baselines 1 and 2).  Returns TV. */
double orc_tv_grad(int nz, int nx, double alpha, double unit, const double *v,
                   const double *g, double *h)
{
    size_t n = (size_t)nz * nx;
    double ng = (double)n, tv = 0.0;
    for (size_t i = 0; i < n; ++i) h[i] = g ? g[i] : 0.0;
    for (int iz = 0; iz < nz; ++iz)
        for (int ix = 0; ix < nx; ++ix) {
            size_t i = IDX(iz, ix, nx);
            if (ix + 1 < nx) {
                double d = (v[i + 1] - v[i]) / unit;
                double sg = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
                tv += fabs(d);
                h[i + 1] += alpha * sg / (ng * unit);
                h[i] -= alpha * sg / (ng * unit);
            }
            if (iz + 1 < nz) {
                size_t k = IDX(iz + 1, ix, nx);
                double d = (v[k] - v[i]) / unit;
                double sg = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
                tv += fabs(d);
                h[k] += alpha * sg / (ng * unit);
                h[i] -= alpha * sg / (ng * unit);
            }
        }
    return tv / ng;
}

/* Reconstruction measures of Sec. 6.3 between a true and a reconstructed
 * field (nz x nx):
 *   out[0] = ||v_true - v_rec||_2 / ||v_true||_2
 *   out[1] = PSNR = 10 log10(R^2 / mean (v_true - v_rec)^2)   (R = data range)
 *   out[2] = SSIM: mean over every 11 x 11 window lying inside the grid of
 *            (2 mu_t mu_r + C1)(2 s_tr + C2) / ((mu_t^2 + mu_r^2 + C1)(s_t^2 + s_r^2 + C2)),
 *            window weights exp(-(a^2 + b^2) / (2 1.5^2)) normalised to sum 1,
 *            weighted means, variances and covariance, C1 = (0.01 R)^2,
 *            C2 = (0.03 R)^2 (Wang et al. 2004); NAN when the grid is
 *            smaller than a window */
void orc_image_metrics(int nz, int nx, double R, const double *vt, const double *vr,
                       double *out)
{
    size_t n = (size_t)nz * nx;
    double se = 0.0, st = 0.0;
    for (size_t i = 0; i < n; ++i) {
        double e = vt[i] - vr[i];
        se += e * e;
        st += vt[i] * vt[i];
    }
    out[0] = sqrt(se) / sqrt(st);
    out[1] = 10.0 * log10(R * R / (se / (double)n));
    const int W = 11, H = 5;
    double w[11][11], ws = 0.0;
    for (int a = 0; a < W; ++a)
        for (int b = 0; b < W; ++b) {
            w[a][b] = exp(-((double)(a - H) * (a - H) + (double)(b - H) * (b - H)) / (2.0 * 1.5 * 1.5));
            ws += w[a][b];
        }
    for (int a = 0; a < W; ++a)
        for (int b = 0; b < W; ++b) w[a][b] /= ws;
    double C1 = (0.01 * R) * (0.01 * R), C2 = (0.03 * R) * (0.03 * R);
    double sum = 0.0;
    long cnt = 0;
    for (int i = 0; i + W <= nz; ++i)
        for (int j = 0; j + W <= nx; ++j) {
            double mt = 0.0, mr = 0.0;
            for (int a = 0; a < W; ++a)
                for (int b = 0; b < W; ++b) {
                    mt += w[a][b] * vt[IDX(i + a, j + b, nx)];
                    mr += w[a][b] * vr[IDX(i + a, j + b, nx)];
                }
            double vtt = 0.0, vrr = 0.0, vtr = 0.0;
            for (int a = 0; a < W; ++a)
                for (int b = 0; b < W; ++b) {
                    double dt_ = vt[IDX(i + a, j + b, nx)] - mt, dr = vr[IDX(i + a, j + b, nx)] - mr;
                    vtt += w[a][b] * dt_ * dt_;
                    vrr += w[a][b] * dr * dr;
                    vtr += w[a][b] * dt_ * dr;
                }
            sum += (2.0 * mt * mr + C1) * (2.0 * vtr + C2) /
                   ((mt * mt + mr * mr + C1) * (vtt + vrr + C2));
            ++cnt;
        }
    out[2] = cnt ? sum / (double)cnt : NAN;
}

/*
 * Oracle fluid module: Fourier pseudo-spectral discretization (Sec. 2.4) of
 * the penalized Navier-Stokes equations in rotational form
 * (Eq. PNST_org_momentum, without the sponge term), advanced by Algorithm 1
 * with Adams-Bashforth 2 and an integrating factor for the viscous term.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Readings where the paper is silent:
 *  - 2/3 rule: cubic truncation per axis, keep |m_i| <= floor(n_i/3)
 *    (the Fig. BB-Spectra caption gives k_max = 256 (2 pi/4) for n = 768);
 *    `dealias_strict` keeps |m_i| < n_i/3 instead;
 *  - AB2 with integrating factor (Sec. 2.4 names it without the formula):
 *    AB2 on v = exp(nu |k|^2 t) u_hat with variable steps, mapped back; the
 *    first step is the integrating-factor Euler step;
 *  - time step: min(CFL min(dx,dy,dz) / max|u|, C_eta, dt_max), or fixed;
 *  - mean mode: held at u_inf (N_hat(0) = 0) or left free to evolve;
 *  - force (Eq. force_with_unst_corrections) and moment (Eq. moment_of_love)
 *    per colour; the unsteady correction is the backward difference of
 *    sum chi u_s dV over the previous step, zero on the first step; moments
 *    are taken about the body centre (body) or the wing pivot (wings).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double PI = 3.14159265358979323846;

static long n_half(const orc_params *p) { return (long)p->nz * p->ny * (p->nx / 2 + 1); }
static long n_phys(const orc_params *p) { return (long)p->nz * p->ny * p->nx; }

/* signed mode number along y or z: 0..n/2-1, then -n/2..-1 */
static int signed_mode(int j, int n) { return j < n / 2 ? j : j - n; }

static int cutoff(int n, int strict)
{
    if (strict && n % 3 == 0) return n / 3 - 1;
    return n / 3;
}

static void wavevector(const orc_params *p, int ix, int iy, int iz, double k[3])
{
    k[0] = 2.0 * PI * ix / p->Lx;
    k[1] = 2.0 * PI * signed_mode(iy, p->ny) / p->Ly;
    k[2] = 2.0 * PI * signed_mode(iz, p->nz) / p->Lz;
}

/* 2/3 rule (Sec. 2.4): zero every mode outside the retained cube. */
void orc_dealias(const orc_params *p, double complex *fh, int ncomp)
{
    int hx = p->nx / 2 + 1;
    int Kx = cutoff(p->nx, p->dealias_strict);
    int Ky = cutoff(p->ny, p->dealias_strict);
    int Kz = cutoff(p->nz, p->dealias_strict);
    long nh = n_half(p);
    for (int c = 0; c < ncomp; ++c) {
#pragma omp parallel for schedule(static)
        for (int iz = 0; iz < p->nz; ++iz)
            for (int iy = 0; iy < p->ny; ++iy)
                for (int ix = 0; ix < hx; ++ix) {
                    int my = abs(signed_mode(iy, p->ny));
                    int mz = abs(signed_mode(iz, p->nz));
                    if (ix > Kx || my > Ky || mz > Kz)
                        fh[c * nh + ((long)iz * p->ny + iy) * hx + ix] = 0;
                }
    }
}

/* Wake-removal regions (Sec. 2.3), a reading: the paper places a sponge and a
 * thinner Dirichlet layer at the domain borders without formulas; here each
 * is the union over axes of the end slab x_i >= L_i - width_i, mask 1 inside
 * (a grid-aligned layer, no smoothing). */
static double end_slab(const orc_params *p, const double *w, const double *X)
{
    const double L[3] = {p->Lx, p->Ly, p->Lz};
    for (int i = 0; i < 3; ++i)
        if (w[i] > 0 && X[i] >= L[i] - w[i]) return 1.0;
    return 0.0;
}

double orc_sponge_mask(const orc_params *p, const double *X) { return end_slab(p, p->sponge_width, X); }

double orc_layer_mask(const orc_params *p, const double *X) { return end_slab(p, p->layer_width, X); }

/* Vorticity sponge (Sec. 2.3, Eq. PNST_org_momentum): -(1/C_sp) curl of the
 * Biot-Savart-type inverse of chi_sp omega.  In Fourier space, with
 * vh = FFT(chi_sp omega)/N, the reading that makes the term damp the vorticity
 * (the printed 1/nabla^2 taken as division by |k|^2, i.e. the inverse of
 * -nabla^2) is  S_hat = -(i k x vh) / (C_sp |k|^2),  S_hat(0) = 0.  Then
 * curl S = -(1/C_sp) times the solenoidal part of chi_sp omega, the term is
 * divergence-free and leaves the mean unchanged. */
void orc_sponge_term(const orc_params *p, const double complex *vh, double complex *sh)
{
    int hx = p->nx / 2 + 1;
    long nh = n_half(p);
#pragma omp parallel for schedule(static)
    for (int iz = 0; iz < p->nz; ++iz)
        for (int iy = 0; iy < p->ny; ++iy)
            for (int ix = 0; ix < hx; ++ix) {
                long i = ((long)iz * p->ny + iy) * hx + ix;
                double k[3];
                wavevector(p, ix, iy, iz, k);
                double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                if (k2 == 0.0) {
                    for (int c = 0; c < 3; ++c) sh[c * nh + i] = 0;
                    continue;
                }
                double complex v0 = vh[i], v1 = vh[nh + i], v2 = vh[2 * nh + i];
                double complex cx = I * (k[1] * v2 - k[2] * v1);
                double complex cy = I * (k[2] * v0 - k[0] * v2);
                double complex cz = I * (k[0] * v1 - k[1] * v0);
                double f = -1.0 / (p->sponge_c * k2);
                sh[i] = f * cx;
                sh[nh + i] = f * cy;
                sh[2 * nh + i] = f * cz;
            }
}

/* Leray projection, Algorithm 1 step (d): F <- F - k (k.F)/|k|^2, k != 0.
 * This is the Fourier-space solution of Eq. PNST_UP_pressure_poisson_eqn. */
void orc_project(const orc_params *p, double complex *fh)
{
    int hx = p->nx / 2 + 1;
    long nh = n_half(p);
#pragma omp parallel for schedule(static)
    for (int iz = 0; iz < p->nz; ++iz)
        for (int iy = 0; iy < p->ny; ++iy)
            for (int ix = 0; ix < hx; ++ix) {
                double k[3];
                wavevector(p, ix, iy, iz, k);
                double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                if (k2 == 0.0) continue;
                long i = ((long)iz * p->ny + iy) * hx + ix;
                double complex kf = k[0] * fh[i] + k[1] * fh[nh + i] + k[2] * fh[2 * nh + i];
                for (int c = 0; c < 3; ++c) fh[c * nh + i] -= k[c] * kf / k2;
            }
}

/* Vorticity omega_hat = i k x u_hat (Sec. 2.4: grad -> i k). */
void orc_curl(const orc_params *p, const double complex *uh, double complex *wh)
{
    int hx = p->nx / 2 + 1;
    long nh = n_half(p);
#pragma omp parallel for schedule(static)
    for (int iz = 0; iz < p->nz; ++iz)
        for (int iy = 0; iy < p->ny; ++iy)
            for (int ix = 0; ix < hx; ++ix) {
                double k[3];
                wavevector(p, ix, iy, iz, k);
                long i = ((long)iz * p->ny + iy) * hx + ix;
                double complex ux = uh[i], uy = uh[nh + i], uz = uh[2 * nh + i];
                wh[i] = I * (k[1] * uz - k[2] * uy);
                wh[nh + i] = I * (k[2] * ux - k[0] * uz);
                wh[2 * nh + i] = I * (k[0] * uy - k[1] * ux);
            }
}

void orc_forward(const orc_params *p, const double *u, double complex *uh, int ncomp)
{
    long N = n_phys(p), nh = n_half(p);
    for (int c = 0; c < ncomp; ++c) {
        orc_fft3_r2c(p->nx, p->ny, p->nz, u + c * N, uh + c * nh);
        for (long i = 0; i < nh; ++i) uh[c * nh + i] /= (double)N;
    }
}

void orc_inverse(const orc_params *p, const double complex *uh, double *u, int ncomp)
{
    long N = n_phys(p), nh = n_half(p);
    for (int c = 0; c < ncomp; ++c)
        orc_fft3_c2r(p->nx, p->ny, p->nz, uh + c * nh, u + c * N);
}

int orc_set_state(const orc_params *p, const double *u, double complex *uh,
                  double complex *nh_prev, orc_scalars *s)
{
    long nh = n_half(p);
    orc_forward(p, u, uh, 3);
    orc_dealias(p, uh, 3);
    orc_project(p, uh);
    if (p->mean_mode == 0)
        for (int c = 0; c < 3; ++c) uh[c * nh] = p->u_inf[c];
    memset(nh_prev, 0, sizeof(double complex) * (size_t)(3 * nh));
    memset(s, 0, sizeof *s);
    return 0;
}

void orc_get_state(const orc_params *p, const double complex *uh, double *u)
{
    orc_inverse(p, uh, u, 3);
}

static double grid_h(const orc_params *p, const orc_insect *ins)
{
    double dx = p->Lx / p->nx, dy = p->Ly / p->ny, dz = p->Lz / p->nz;
    double d = dx > dy ? dx : dy;
    if (dz > d) d = dz;
    return ins->c_smth * d;
}

/*
 * Algorithm 1 steps (a) and (c) in physical space at time t: u and omega from
 * u_hat, then per grid point chi, colour, u_s and
 * nl = u x omega - chi/C_eta (u - u_s), plus the FP64 sums.  When `fields` is
 * not NULL it receives [u(3), omega(3), chi, colour, u_s(3), nl(3)] per point.
 * Returns 1 if a non-finite value was met, else 0.
 */
static int physical_terms(const orc_params *p, const orc_insect *ins, double t,
                          const double complex *uh, double *nl, double *sums, double *fields,
                          double *vsp)
{
    long N = n_phys(p), nhs = n_half(p);
    double complex *wh = malloc(sizeof(double complex) * (size_t)(3 * nhs));
    double *u = malloc(sizeof(double) * (size_t)(3 * N));
    double *w = malloc(sizeof(double) * (size_t)(3 * N));

    orc_curl(p, uh, wh);
    orc_inverse(p, uh, u, 3);
    orc_inverse(p, wh, w, 3);

    orc_frames fr;
    if (ins) orc_frames_at(ins, t, &fr);
    double h = ins ? grid_h(p, ins) : 0.0;
    double dx = p->Lx / p->nx, dy = p->Ly / p->ny, dz = p->Lz / p->nz;
    double dV = dx * dy * dz;
    memset(sums, 0, sizeof(double) * ORC_NSUMS);
    int bad = 0;
    /* sums[0 .. ORC_SUM_EKIN] add up, ORC_SUM_UMAX is a maximum; in the
     * OpenMP build (timing only) each thread keeps its own copies of them */
    double acc[ORC_SUM_EKIN + 1];
    memset(acc, 0, sizeof acc);
    double umax = 0.0;

#pragma omp parallel for schedule(static) reduction(+ : acc[:ORC_SUM_EKIN + 1]) reduction(max : umax) \
    reduction(| : bad)
    for (long iz = 0; iz < p->nz; ++iz)
        for (long iy = 0; iy < p->ny; ++iy)
            for (long ix = 0; ix < p->nx; ++ix) {
                long i = (iz * p->ny + iy) * p->nx + ix;
                double X[3] = {ix * dx, iy * dy, iz * dz};
                double uu[3] = {u[i], u[N + i], u[2 * N + i]};
                double ww[3] = {w[i], w[N + i], w[2 * N + i]};
                double chi = 0.0, us[3] = {0, 0, 0};
                int col = 0;
                if (ins) orc_solid_at(ins, &fr, h, X, &chi, &col, us);
                /* u x omega - chi/C_eta (u - u_s) */
                double lamb[3] = {uu[1] * ww[2] - uu[2] * ww[1],
                                  uu[2] * ww[0] - uu[0] * ww[2],
                                  uu[0] * ww[1] - uu[1] * ww[0]};
                /* Dirichlet layer u = u_inf (Sec. 2.3), a penalization of its own */
                double chi_d = orc_layer_mask(p, X);
                for (int c = 0; c < 3; ++c) {
                    double v = lamb[c] - chi / p->eta * (uu[c] - us[c]);
                    if (chi_d > 0) v -= chi_d / p->eta * (uu[c] - p->u_inf[c]);
                    nl[c * N + i] = v;
                    if (!isfinite(v) || !isfinite(uu[c])) bad = 1;
                }
                if (vsp) {
                    double chi_sp = orc_sponge_mask(p, X);
                    for (int c = 0; c < 3; ++c) vsp[c * N + i] = chi_sp * ww[c];
                }
                if (fields) {
                    for (int c = 0; c < 3; ++c) {
                        fields[c * N + i] = uu[c];
                        fields[(3 + c) * N + i] = ww[c];
                        fields[(8 + c) * N + i] = us[c];
                        fields[(11 + c) * N + i] = nl[c * N + i];
                    }
                    fields[6 * N + i] = chi;
                    fields[7 * N + i] = col;
                }
                double u2 = uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2];
                acc[ORC_SUM_EKIN] += 0.5 * u2 * dV;
                if (sqrt(u2) > umax) umax = sqrt(u2);
                if (col > 0) {
                    int c0 = col - 1;
                    const double *xr = col == 1 ? ins->x_cntr : fr.pivot_g[col - 2];
                    double r[3] = {X[0] - xr[0], X[1] - xr[1], X[2] - xr[2]};
                    double pen[3], cus[3], m1[3], m2[3];
                    for (int c = 0; c < 3; ++c) {
                        pen[c] = chi * (uu[c] - us[c]);
                        cus[c] = chi * us[c];
                    }
                    m1[0] = r[1] * pen[2] - r[2] * pen[1];
                    m1[1] = r[2] * pen[0] - r[0] * pen[2];
                    m1[2] = r[0] * pen[1] - r[1] * pen[0];
                    m2[0] = r[1] * cus[2] - r[2] * cus[1];
                    m2[1] = r[2] * cus[0] - r[0] * cus[2];
                    m2[2] = r[0] * cus[1] - r[1] * cus[0];
                    for (int c = 0; c < 3; ++c) {
                        acc[ORC_SUM_FP(c0) + c] += pen[c] * dV / p->eta;
                        acc[ORC_SUM_MP(c0) + c] += m1[c] * dV / p->eta;
                        acc[ORC_SUM_IS(c0) + c] += cus[c] * dV;
                        acc[ORC_SUM_JS(c0) + c] += m2[c] * dV;
                    }
                }
            }
    for (int k = 0; k <= ORC_SUM_EKIN; ++k) sums[k] = acc[k];
    sums[ORC_SUM_UMAX] = umax;
    sums[ORC_SUM_NONFINITE] = bad;
    free(w);
    free(u);
    free(wh);
    return bad;
}

void orc_physical_fields(const orc_params *p, const orc_insect *ins, double t,
                         const double complex *uh, double *fields)
{
    long N = n_phys(p);
    double *nl = malloc(sizeof(double) * (size_t)(3 * N));
    double sums[ORC_NSUMS];
    physical_terms(p, ins, t, uh, nl, sums, fields, NULL);
    free(nl);
}

/*
 * Right-hand side of Algorithm 1 steps (a), (c), (d) at time t:
 * nh = P D FFT(u x omega - chi/C_eta (u - u_s)) / N, plus the FP64 sums.
 * Returns 1 if a non-finite value was met, else 0.
 */
int orc_rhs(const orc_params *p, const orc_insect *ins, double t,
            const double complex *uh, double complex *nh, double *sums)
{
    long N = n_phys(p), nhs = n_half(p);
    double *nl = malloc(sizeof(double) * (size_t)(3 * N));
    double *vsp = p->sponge_c > 0 ? malloc(sizeof(double) * (size_t)(3 * N)) : NULL;
    int bad = physical_terms(p, ins, t, uh, nl, sums, NULL, vsp);

    orc_forward(p, nl, nh, 3);
    if (vsp) {
        /* Algorithm 1 step (c): the sponge term joins the sources */
        double complex *vh = malloc(sizeof(double complex) * (size_t)(3 * nhs));
        double complex *sh = malloc(sizeof(double complex) * (size_t)(3 * nhs));
        orc_forward(p, vsp, vh, 3);
        orc_sponge_term(p, vh, sh);
        for (long i = 0; i < 3 * nhs; ++i) nh[i] += sh[i];
        free(vh);
        free(sh);
        free(vsp);
    }
    orc_dealias(p, nh, 3);
    orc_project(p, nh);
    if (p->mean_mode == 0)
        for (int c = 0; c < 3; ++c) nh[c * nhs] = 0;

    free(nl);
    return bad;
}

/*
 * Integrating-factor AB2 (Algorithm 1 step (e)).  With v = e^{nu k^2 t} u_hat,
 * dv/dt = e^{nu k^2 t} N_hat; variable-step AB2 on v with r = dt/dt_prev,
 * multiplied back by e^{-nu k^2 t^{n+1}}:
 *   u^{n+1} = E1 u^n + dt [ (1 + r/2) E1 N^n - (r/2) E2 N^{n-1} ],
 *   E1 = e^{-nu k^2 dt},  E2 = e^{-nu k^2 (dt + dt_prev)};
 * on the first step (n = 0): u^1 = E1 (u^0 + dt N^0).
 */
void orc_ab2_update(const orc_params *p, double complex *uh,
                    const double complex *nh, const double complex *nh_prev,
                    double dt, double dt_prev, int64_t n)
{
    int hx = p->nx / 2 + 1;
    long nhs = n_half(p);
#pragma omp parallel for schedule(static)
    for (int iz = 0; iz < p->nz; ++iz)
        for (int iy = 0; iy < p->ny; ++iy)
            for (int ix = 0; ix < hx; ++ix) {
                double k[3];
                wavevector(p, ix, iy, iz, k);
                double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                double E1 = exp(-p->nu * k2 * dt);
                long i = ((long)iz * p->ny + iy) * hx + ix;
                for (int c = 0; c < 3; ++c) {
                    long j = c * nhs + i;
                    if (n == 0) {
                        uh[j] = E1 * (uh[j] + dt * nh[j]);
                    } else {
                        double r = dt / dt_prev;
                        double E2 = exp(-p->nu * k2 * (dt + dt_prev));
                        uh[j] = E1 * uh[j] +
                                dt * ((1.0 + 0.5 * r) * E1 * nh[j] - 0.5 * r * E2 * nh_prev[j]);
                    }
                }
            }
}

/* RK4 with explicit diffusion (Sec. 2.4 names it as the alternative to
 * IF-AB2): the classical four-stage combination
 * u^{n+1} = u^n + dt/6 (k1 + 2 k2 + 2 k3 + k4). */
void orc_rk4_combine(const orc_params *p, double complex *uh, const double complex *k1,
                     const double complex *k2, const double complex *k3,
                     const double complex *k4, double dt)
{
    long n = 3 * n_half(p);
    for (long i = 0; i < n; ++i) uh[i] += dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* k = N_hat - nu |k|^2 u_hat: the right-hand side with the viscous term explicit. */
static void add_viscous(const orc_params *p, const double complex *uh, double complex *k)
{
    int hx = p->nx / 2 + 1;
    long nhs = n_half(p);
#pragma omp parallel for schedule(static)
    for (int iz = 0; iz < p->nz; ++iz)
        for (int iy = 0; iy < p->ny; ++iy)
            for (int ix = 0; ix < hx; ++ix) {
                double kv[3];
                wavevector(p, ix, iy, iz, kv);
                double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
                long i = ((long)iz * p->ny + iy) * hx + ix;
                for (int c = 0; c < 3; ++c) k[c * nhs + i] -= p->nu * k2 * uh[c * nhs + i];
            }
}

/* Largest |k|^2 over the retained modes (the explicit-diffusion limit of RK4). */
static double k2_max(const orc_params *p)
{
    int K[3] = {cutoff(p->nx, p->dealias_strict), cutoff(p->ny, p->dealias_strict),
                cutoff(p->nz, p->dealias_strict)};
    double L[3] = {p->Lx, p->Ly, p->Lz}, k2 = 0;
    for (int i = 0; i < 3; ++i) {
        double k = 6.283185307179586476925286766559 * K[i] / L[i];
        k2 += k * k;
    }
    return k2;
}

/* One step of Algorithm 1 (without free flight and output). */
int orc_step(const orc_params *p, orc_insect *ins, double complex *uh,
             double complex *nh_prev, orc_scalars *s, double *row)
{
    if (ins && ins->free_flight && p->time_scheme == 1) return 2;   /* free flight is AB2 only */
    long nhs = n_half(p);
    double complex *nh = malloc(sizeof(double complex) * (size_t)(3 * nhs));
    double sums[ORC_NSUMS];
    int bad = orc_rhs(p, ins, s->t, uh, nh, sums);
    if (bad) {
        free(nh);
        return 1;
    }

    /* Algorithm 1 step (b): the time step.  RK4 adds the explicit-diffusion
     * limit dt <= 2.5 / (nu |k|^2_max) (a reading: inside the real-axis
     * stability interval of RK4, about [-2.78, 0]). */
    double dt;
    if (p->dt_fixed > 0) {
        dt = p->dt_fixed;
    } else {
        double dx = p->Lx / p->nx, dy = p->Ly / p->ny, dz = p->Lz / p->nz;
        double dmin = dx < dy ? dx : dy;
        if (dz < dmin) dmin = dz;
        dt = p->eta;
        double umax = sums[ORC_SUM_UMAX];
        if (umax > 0 && p->cfl * dmin / umax < dt) dt = p->cfl * dmin / umax;
        if (p->dt_max > 0 && p->dt_max < dt) dt = p->dt_max;
        if (p->time_scheme == 1 && p->nu > 0) {
            double lim = 2.5 / (p->nu * k2_max(p));
            if (lim < dt) dt = lim;
        }
    }

    if (p->time_scheme == 1) {
        /* stages at t, t + dt/2, t + dt/2, t + dt; the mask moves with them */
        long n3 = 3 * nhs;
        size_t bytes = sizeof(double complex) * (size_t)n3;
        double complex *k[4], *us = malloc(bytes);
        double stage_sums[ORC_NSUMS];
        for (int q = 0; q < 4; ++q) k[q] = malloc(bytes);
        memcpy(k[0], nh, bytes);
        add_viscous(p, uh, k[0]);
        const double frac[4] = {0.0, 0.5, 0.5, 1.0};
        for (int q = 1; q < 4 && !bad; ++q) {
            for (long i = 0; i < n3; ++i) us[i] = uh[i] + frac[q] * dt * k[q - 1][i];
            bad = orc_rhs(p, ins, s->t + frac[q] * dt, us, k[q], stage_sums);
            add_viscous(p, us, k[q]);
        }
        if (!bad) orc_rk4_combine(p, uh, k[0], k[1], k[2], k[3], dt);
        for (int q = 0; q < 4; ++q) free(k[q]);
        free(us);
        if (bad) {
            free(nh);
            return 1;
        }
    } else {
        orc_ab2_update(p, uh, nh, nh_prev, dt, s->dt_prev, s->n);
    }

    row[0] = s->t;
    row[1] = dt;
    for (int c = 0; c < ORC_NCOLOURS; ++c)
        for (int i = 0; i < 3; ++i) {
            double F = sums[ORC_SUM_FP(c) + i], M = sums[ORC_SUM_MP(c) + i];
            double Is = sums[ORC_SUM_IS(c) + i], Js = sums[ORC_SUM_JS(c) + i];
            if (s->n > 0) {
                F += (Is - s->Is_prev[c][i]) / s->dt_prev;
                M += (Js - s->Js_prev[c][i]) / s->dt_prev;
            }
            row[2 + c * 6 + i] = F;
            row[2 + c * 6 + 3 + i] = M;
            s->Is_prev[c][i] = Is;
            s->Js_prev[c][i] = Js;
        }
    row[20] = sums[ORC_SUM_EKIN];
    row[21] = sums[ORC_SUM_UMAX];

    /* power of the wings at t^n (Sec. 3.5) */
    orc_frames fr;
    if (ins) orc_frames_at(ins, s->t, &fr);
    row[22] = row[23] = row[24] = row[25] = 0.0;
    if (ins) orc_wing_power(ins, &fr, row, row + 22, row + 24);

    /* free flight (Sec. 3.6): the body state advances with the fluid's AB2
     * (same dt and ratio, Euler on the first step); the quaternion is
     * renormalized after each step (a reading).  Force: all colours; moment:
     * about x_cntr, the wings' moments moved from their pivots. */
    if (ins && ins->free_flight) {
        double F[3] = {0, 0, 0}, m[3] = {0, 0, 0}, mb[3], f[13], y[13];
        for (int c = 0; c < ORC_NCOLOURS; ++c)
            for (int i = 0; i < 3; ++i) {
                F[i] += row[2 + 6 * c + i];
                m[i] += row[2 + 6 * c + 3 + i];
            }
        for (int w = 0; w < 2 && w < ins->nwings; ++w) {
            const double *Fw = row + 2 + 6 * (1 + w);
            double r[3] = {fr.pivot_g[w][0] - ins->x_cntr[0], fr.pivot_g[w][1] - ins->x_cntr[1],
                           fr.pivot_g[w][2] - ins->x_cntr[2]};
            m[0] += r[1] * Fw[2] - r[2] * Fw[1];
            m[1] += r[2] * Fw[0] - r[0] * Fw[2];
            m[2] += r[0] * Fw[1] - r[1] * Fw[0];
        }
        for (int i = 0; i < 3; ++i)
            mb[i] = fr.M_body[3 * i] * m[0] + fr.M_body[3 * i + 1] * m[1] + fr.M_body[3 * i + 2] * m[2];
        orc_body_rhs(ins, F, mb, f);
        for (int i = 0; i < 3; ++i) {
            y[i] = ins->x_cntr[i];
            y[3 + i] = ins->u_cntr[i];
            y[10 + i] = ins->Omega_body[i];
        }
        for (int i = 0; i < 4; ++i) y[6 + i] = ins->quat[i];
        for (int i = 0; i < 13; ++i) {
            if (s->n == 0) {
                y[i] += dt * f[i];
            } else {
                double r = dt / s->dt_prev;
                y[i] += dt * ((1.0 + 0.5 * r) * f[i] - 0.5 * r * s->body_rhs_prev[i]);
            }
            s->body_rhs_prev[i] = f[i];
        }
        double qn = sqrt(y[6] * y[6] + y[7] * y[7] + y[8] * y[8] + y[9] * y[9]);
        for (int i = 0; i < 3; ++i) {
            ins->x_cntr[i] = y[i];
            ins->u_cntr[i] = y[3 + i];
            ins->Omega_body[i] = y[10 + i];
        }
        for (int i = 0; i < 4; ++i) ins->quat[i] = y[6 + i] / qn;
    }

    memcpy(nh_prev, nh, sizeof(double complex) * (size_t)(3 * nhs));
    s->t += dt;
    s->dt_prev = dt;
    s->n += 1;
    free(nh);
    return 0;
}

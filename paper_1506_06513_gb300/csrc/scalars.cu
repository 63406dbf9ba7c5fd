// Small single-block kernels of one step:
//  * kinematics: the insect frames at t^n (Sec. 3.1, 3.3; Eq. M_body_yawpitchroll),
//    in FP64, written as one Frame block read by every CTA of the physical pass;
//  * scalars: the deterministic final reduction of the physical pass's per-CTA
//    partial sums, the time step (Algorithm 1 step b), the integrating-factor
//    AB2 coefficients and exponential tables, and the force row
//    (Eqs. force_with_unst_corrections, moment_of_love);
//  * reset: the step state after a new initial condition.
#include "kernels.cuh"

#include "../../include/flusi.h"

namespace flusi {

namespace {

struct M3 {
    double a[9];
};

__device__ M3 rot_x(double xi)
{
    double c = cos(xi), s = sin(xi);
    return {{1, 0, 0, 0, c, s, 0, -s, c}};
}
__device__ M3 rot_y(double xi)
{
    double c = cos(xi), s = sin(xi);
    return {{c, 0, -s, 0, 1, 0, s, 0, c}};
}
__device__ M3 rot_z(double xi)
{
    double c = cos(xi), s = sin(xi);
    return {{c, s, 0, -s, c, 0, 0, 0, 1}};
}
__device__ M3 mul(const M3& A, const M3& B)
{
    M3 C;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            C.a[i * 3 + j] = A.a[i * 3] * B.a[j] + A.a[i * 3 + 1] * B.a[3 + j] + A.a[i * 3 + 2] * B.a[6 + j];
    return C;
}
// A^T x (the inverse of a rotation applied to x)
__device__ void apply_t(const M3& A, const double* x, double* y)
{
    double t0 = A.a[0] * x[0] + A.a[3] * x[1] + A.a[6] * x[2];
    double t1 = A.a[1] * x[0] + A.a[4] * x[1] + A.a[7] * x[2];
    double t2 = A.a[2] * x[0] + A.a[5] * x[1] + A.a[8] * x[2];
    y[0] = t0, y[1] = t1, y[2] = t2;
}

// a0/2 + sum a_i cos(2 pi i f t) + b_i sin(2 pi i f t) and its time derivative
__device__ void series(double a0, const double* a, const double* b, int nf, double f, double t,
                       double* v, double* dv)
{
    const double two_pi = 6.283185307179586476925286766559;
    double s = 0.5 * a0, d = 0.0;
    for (int i = 0; i < nf; ++i) {
        double w = two_pi * (i + 1) * f;
        double sn, cs;
        sincos(w * t, &sn, &cs);
        s += a[i] * cs + b[i] * sn;
        d += w * (b[i] * cs - a[i] * sn);
    }
    *v = s;
    *dv = d;
}

__device__ void box_grow(double* box, const double* p)
{
    for (int i = 0; i < 3; ++i) {
        box[2 * i] = fmin(box[2 * i], p[i]);
        box[2 * i + 1] = fmax(box[2 * i + 1], p[i]);
    }
}

}  // namespace

// frac = 0: at the state's time; frac > 0: at t0 + frac dt of the current
// step (the later RK4 stages, after k_scalars has written t0 and dt).
__global__ void k_kinematics(const flusi_insect* ins, const StepState* st, const StepCoef* coef, Frame* fr,
                             double h, double frac)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double t = frac > 0.0 ? coef->t0 + frac * coef->dt : st->t;
    Frame F;
    F.t = t;
    for (int i = 0; i < 3; ++i) {
        F.xc[i] = ins->x_cntr[i];
        F.uc[i] = ins->u_cntr[i];
    }
    // body frame: yaw, then pitch, then roll
    M3 Rx = rot_x(ins->psi), Ry = rot_y(ins->beta), Rz = rot_z(ins->gamma);
    M3 Mb = mul(mul(Rx, Ry), Rz);
    for (int i = 0; i < 9; ++i) F.Mb[i] = Mb.a[i];
    // body angular velocity in the global frame (nested form of Sec. 3.1)
    double v[3] = {ins->psi_dot, 0, 0};
    apply_t(Rx, v, v);
    v[1] += ins->beta_dot;
    apply_t(Ry, v, v);
    v[2] += ins->gamma_dot;
    apply_t(Rz, v, F.Ob);

    double phi, alpha, theta, dphi, dalpha, dtheta;
    int nf = ins->nfourier;
    series(ins->phi_a0, ins->phi_a, ins->phi_b, nf, ins->freq, t, &phi, &dphi);
    series(ins->alpha_a0, ins->alpha_a, ins->alpha_b, nf, ins->freq, t, &alpha, &dalpha);
    series(ins->theta_a0, ins->theta_a, ins->theta_b, nf, ins->freq, t, &theta, &dtheta);

    const double pi = 3.141592653589793238462643383279;
    for (int s = 0; s < 2; ++s) {
        // the right wing mirrors the left: R_x(pi) in the stroke matrix and
        // (phi, alpha) -> (-phi, -alpha) in the wing matrix
        double sg = s == 0 ? 1.0 : -1.0;
        M3 Ms = rot_y(ins->eta_stroke);
        if (s == 1) Ms = mul(rot_x(pi), Ms);
        M3 Ra = rot_y(sg * alpha), Rt = rot_z(-theta), Rp = rot_x(sg * phi);
        M3 Mw = mul(mul(Ra, Rt), Rp);
        M3 Mg = mul(mul(Mw, Ms), Mb);          // global -> wing frame
        for (int i = 0; i < 9; ++i) F.Mw[s][i] = Mg.a[i];
        // angular velocity in the stroke frame, then body, then global frame
        double w[3] = {0, sg * dalpha, 0};
        apply_t(Ra, w, w);
        w[2] += -dtheta;
        apply_t(Rt, w, w);
        w[0] += sg * dphi;
        apply_t(Rp, w, w);
        apply_t(Ms, w, w);
        apply_t(Mb, w, F.Ow[s]);
        const double* pb = s == 0 ? ins->pivot_l : ins->pivot_r;
        double pg[3];
        apply_t(Mb, pb, pg);
        for (int i = 0; i < 3; ++i) F.pv[s][i] = F.xc[i] + pg[i];
    }

    // bounding boxes (global) of the region where chi > 0
    for (int p = 0; p < 3; ++p) {
        for (int i = 0; i < 3; ++i) {
            F.box[p][2 * i] = 1e300;
            F.box[p][2 * i + 1] = -1e300;
        }
        F.active[p] = 0;
    }
    if (ins->body_type != 0) {
        // body-frame box of thorax, head and eyes, grown by h; its corners in
        // the global frame
        double lo[3], hi[3];
        const double ey = ins->body_type == 1 ? ins->body_a : ins->body_b;
        lo[0] = -ins->body_a;
        hi[0] = ins->body_a;
        lo[1] = lo[2] = -ey;
        hi[1] = hi[2] = ey;
        if (ins->body_type == 2 && ins->head_r > 0)
            for (int i = 0; i < 3; ++i) {
                lo[i] = fmin(lo[i], ins->head_x0[i] - ins->head_r);
                hi[i] = fmax(hi[i], ins->head_x0[i] + ins->head_r);
            }
        if (ins->body_type == 2 && ins->eye_r > 0)
            for (int i = 0; i < 3; ++i) {
                const double c = ins->eye_x0[i], m = i == 1 ? -c : c;   // both eyes
                lo[i] = fmin(lo[i], fmin(c, m) - ins->eye_r);
                hi[i] = fmax(hi[i], fmax(c, m) + ins->eye_r);
            }
        for (int c = 0; c < 8; ++c) {
            double q[3] = {(c & 1 ? hi[0] : lo[0]) + (c & 1 ? h : -h),
                           (c & 2 ? hi[1] : lo[1]) + (c & 2 ? h : -h),
                           (c & 4 ? hi[2] : lo[2]) + (c & 4 ? h : -h)}, gq[3];
            apply_t(Mb, q, gq);
            for (int i = 0; i < 3; ++i) gq[i] += F.xc[i];
            box_grow(F.box[0], gq);
        }
        F.active[0] = 1;
    }
    for (int s = 0; s < ins->nwings && s < 2; ++s) {
        M3 Mg;
        for (int i = 0; i < 9; ++i) Mg.a[i] = F.Mw[s][i];
        double xs[2] = {-ins->wing_c_te - h, ins->wing_c_le + h};
        double ys[2] = {-h, ins->wing_R + h};
        double zs[2] = {-0.5 * ins->wing_h - h, 0.5 * ins->wing_h + h};
        if (ins->wing_shape == 1) {
            // R(theta) <= a0/2 + sum sqrt(a_i^2 + b_i^2)
            double rb = 0.5 * ins->contour_a0;
            for (int i = 0; i < ins->ncontour; ++i)
                rb += sqrt(ins->contour_a[i] * ins->contour_a[i] + ins->contour_b[i] * ins->contour_b[i]);
            xs[0] = ins->contour_xc - rb - h;
            xs[1] = ins->contour_xc + rb + h;
            ys[0] = ins->contour_yc - rb - h;
            ys[1] = ins->contour_yc + rb + h;
        }
        for (int c = 0; c < 8; ++c) {
            double q[3] = {xs[c & 1], ys[(c >> 1) & 1], zs[(c >> 2) & 1]}, g[3];
            apply_t(Mg, q, g);
            for (int i = 0; i < 3; ++i) g[i] += F.pv[s][i];
            box_grow(F.box[1 + s], g);
        }
        F.active[1 + s] = 1;
    }
    *fr = F;
}

__global__ void k_reset_state(StepState* st, StepCoef* coef)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    StepState s = {};
    *st = s;
    StepCoef c = {};
    *coef = c;
}

// One block.  Reduces part[nparts][kNumSums] in a fixed order, then forms the
// step's scalars.  `opts` = {cfl, dt_fixed, dt_max}; dt_diff > 0 caps the
// adaptive step (the explicit-diffusion limit of RK4).
__global__ void k_scalars(Geom g, const double* part, int nparts, StepState* st, StepCoef* coef,
                          double* rows, int ring, double* etab, double3 opts, double dt_diff)
{
    __shared__ double red[kNumSums][33];
    __shared__ double tot[kNumSums];
    const int tid = threadIdx.x, T = blockDim.x;
    const int warp = tid / 32, lane = tid % 32;

    // every thread reads the state before the first barrier; thread 0 writes
    // it only after the last one
    const int status = st->status;
    const long long n = st->n;
    const double dt_prev = st->dt_prev;
    if (status != 0) {
        if (tid == 0) coef->skip = 1;
        return;
    }
    // per slot: strided partial by thread, warp tree, then warps in order
    for (int k = 0; k < kNumSums; ++k) {
        const bool is_max = (k == kSumUmax2 || k == kSumBad);
        double acc = 0.0;
        for (int i = tid; i < nparts; i += T) {
            double v = part[(size_t)i * kNumSums + k];
            acc = is_max ? fmax(acc, v) : acc + v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            double w = __shfl_down_sync(0xffffffffu, acc, o);
            acc = is_max ? fmax(acc, w) : acc + w;
        }
        if (lane == 0) red[k][warp] = acc;
    }
    __syncthreads();
    if (tid < kNumSums) {
        const bool is_max = (tid == kSumUmax2 || tid == kSumBad);
        double a = 0.0;
        for (int w = 0; w < T / 32; ++w) a = is_max ? fmax(a, red[tid][w]) : a + red[tid][w];
        tot[tid] = a;
    }
    __syncthreads();

    if (tot[kSumBad] != 0.0) {
        if (tid == 0) {
            st->status = FLUSI_ENONFINITE;
            coef->skip = 1;
        }
        return;
    }

    // time step (Algorithm 1 step b)
    const double umax = sqrt(tot[kSumUmax2]);
    double dt;
    if (opts.y > 0.0) {
        dt = opts.y;
    } else {
        const double dmin = fmin(g.dx, fmin(g.dy, g.dz));
        dt = g.eta;
        if (umax > 0.0) dt = fmin(dt, opts.x * dmin / umax);
        if (opts.z > 0.0) dt = fmin(dt, opts.z);
        if (dt_diff > 0.0) dt = fmin(dt, dt_diff);
    }
    const int first = (n == 0);

    // integrating factors, separable per axis: E1 = e^{-nu |k|^2 dt},
    // E2 = e^{-nu |k|^2 (dt + dt_prev)}; layout [E1x Mx][E1y My][E1z Mz][E2x][E2y][E2z]
    const double two_pi = 6.283185307179586476925286766559;
    const int Mt = g.Mx + g.My + g.Mz;
    for (int i = tid; i < 2 * Mt; i += T) {
        int which = i / Mt, r = i % Mt;
        double k, tau = which == 0 ? dt : dt + dt_prev;
        if (r < g.Mx) k = two_pi * r / g.Lx;
        else if (r < g.Mx + g.My) k = two_pi * mode_of(r - g.Mx, g.Ky) / g.Ly;
        else k = two_pi * mode_of(r - g.Mx - g.My, g.Kz) / g.Lz;
        etab[i] = exp(-g.nu * k * k * tau);
    }

    __syncthreads();
    if (tid == 0) {
        StepCoef c;
        c.dt = dt;
        c.n = n;
        c.first = first;
        c.t0 = st->t;
        c.skip = 0;
        if (first) {
            c.c_now = dt;
            c.c_old = 0.0;
        } else {
            double r = dt / dt_prev;
            c.c_now = dt * (1.0 + 0.5 * r);
            c.c_old = dt * 0.5 * r;
        }
        *coef = c;

        // force row
        const double dV = g.dx * g.dy * g.dz;
        double* row = rows + (size_t)(n % ring) * kRowCols;
        row[0] = st->t;
        row[1] = dt;
        for (int p = 0; p < 3; ++p) {
            const double* s = tot + 12 * p;
            for (int i = 0; i < 3; ++i) {
                double Fv = s[i] * dV / g.eta, Mv = s[3 + i] * dV / g.eta;
                double Is = s[6 + i] * dV, Js = s[9 + i] * dV;
                if (!first) {
                    Fv += (Is - st->Is_prev[p][i]) / dt_prev;
                    Mv += (Js - st->Js_prev[p][i]) / dt_prev;
                }
                row[2 + 6 * p + i] = Fv;
                row[5 + 6 * p + i] = Mv;
                st->Is_prev[p][i] = Is;
                st->Js_prev[p][i] = Js;
            }
        }
        row[20] = 0.5 * tot[kSumEkin] * dV;
        row[21] = umax;

        st->t += dt;
        st->dt_prev = dt;
        st->n = n + 1;
    }
}

}  // namespace flusi

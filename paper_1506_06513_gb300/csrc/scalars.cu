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

// A x
__device__ void apply(const M3& A, const double* x, double* y)
{
    double t0 = A.a[0] * x[0] + A.a[1] * x[1] + A.a[2] * x[2];
    double t1 = A.a[3] * x[0] + A.a[4] * x[1] + A.a[5] * x[2];
    double t2 = A.a[6] * x[0] + A.a[7] * x[1] + A.a[8] * x[2];
    y[0] = t0, y[1] = t1, y[2] = t2;
}

__device__ void cross3(const double* a, const double* b, double* c)
{
    double c0 = a[1] * b[2] - a[2] * b[1];
    double c1 = a[2] * b[0] - a[0] * b[2];
    double c2 = a[0] * b[1] - a[1] * b[0];
    c[0] = c0, c[1] = c1, c[2] = c2;
}

// a0/2 + sum a_i cos(2 pi i f t) + b_i sin(2 pi i f t) and its first two time
// derivatives
__device__ void series(double a0, const double* a, const double* b, int nf, double f, double t,
                       double* v, double* dv, double* ddv)
{
    const double two_pi = 6.283185307179586476925286766559;
    double s = 0.5 * a0, d = 0.0, dd = 0.0;
    for (int i = 0; i < nf; ++i) {
        double w = two_pi * (i + 1) * f;
        double sn, cs;
        sincos(w * t, &sn, &cs);
        const double c = a[i] * cs + b[i] * sn;
        s += c;
        d += w * (b[i] * cs - a[i] * sn);
        dd -= w * w * c;
    }
    *v = s;
    *dv = d;
    *ddv = dd;
}

// Body-to-global matrix of the quaternion (e0, e1, e2, e3) as printed in
// Sec. 3.6; its transpose is the global-to-body matrix M_body.
__device__ M3 quat_to_global(const double* e)
{
    const double a = e[0], b = e[1], c = e[2], d = e[3];
    return {{a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c),
             2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b),
             2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d}};
}

__device__ void box_grow(double* box, const double* p)
{
    for (int i = 0; i < 3; ++i) {
        box[2 * i] = fmin(box[2 * i], p[i]);
        box[2 * i + 1] = fmax(box[2 * i + 1], p[i]);
    }
}

// Free flight (Sec. 3.6, Eq. oh_my_god_look_a_vector): one AB2 step of the
// 13 body equations with the fluid step's dt and ratio r = dt/dt_prev (Euler
// when `first`).  State y = (x_cntr, u_cntr, quat, Omega_body); forcing: the
// row's total force and its total moment about x_cntr, taken into body axes.
__device__ void advance_body(flusi_insect* ins, StepState* st, const Frame& F, const double* row,
                             double dt, double r, int first)
{
    double Ft[3] = {0, 0, 0}, mg[3] = {0, 0, 0};
    for (int p = 0; p < 3; ++p)
        for (int i = 0; i < 3; ++i) {
            Ft[i] += row[2 + 6 * p + i];
            mg[i] += row[5 + 6 * p + i];
        }
    // a wing's moment is about its pivot: M_c = M_pivot + (pivot - x_cntr) x F
    for (int s = 0; s < 2 && s < ins->nwings; ++s) {
        const double arm[3] = {F.pv[s][0] - F.xc[0], F.pv[s][1] - F.xc[1], F.pv[s][2] - F.xc[2]};
        double c[3];
        cross3(arm, row + 2 + 6 * (1 + s), c);
        for (int i = 0; i < 3; ++i) mg[i] += c[i];
    }
    M3 Mb;
    for (int i = 0; i < 9; ++i) Mb.a[i] = F.Mb[i];
    double mb[3];
    apply(Mb, mg, mb);

    double y[13], f[13];
    const double* e = ins->quat;
    const double* W = ins->Omega_body;
    const double* J = ins->J_body;
    const double* dof = ins->dof;
    for (int i = 0; i < 3; ++i) {
        y[i] = ins->x_cntr[i];
        y[3 + i] = ins->u_cntr[i];
        y[10 + i] = W[i];
        f[i] = ins->u_cntr[i];
        f[3 + i] = dof[i] * Ft[i] / ins->mass;
    }
    f[5] -= dof[2] * ins->gravity;
    for (int i = 0; i < 4; ++i) y[6 + i] = e[i];
    // quaternion rate: half the product eps (x) (0, Omega^(b))
    f[6] = -0.5 * (e[1] * W[0] + e[2] * W[1] + e[3] * W[2]);
    f[7] = 0.5 * (e[0] * W[0] + e[2] * W[2] - e[3] * W[1]);
    f[8] = 0.5 * (e[0] * W[1] + e[3] * W[0] - e[1] * W[2]);
    f[9] = 0.5 * (e[0] * W[2] + e[1] * W[1] - e[2] * W[0]);
    // Euler's equations in principal body axes
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        f[10 + i] = dof[3 + i] * ((J[j] - J[k]) * W[j] * W[k] + mb[i]) / J[i];
    }
    for (int i = 0; i < 13; ++i) {
        const double step = first ? f[i] : (1.0 + 0.5 * r) * f[i] - 0.5 * r * st->body_rhs_prev[i];
        y[i] += dt * step;
        st->body_rhs_prev[i] = f[i];
    }
    const double qn = sqrt(y[6] * y[6] + y[7] * y[7] + y[8] * y[8] + y[9] * y[9]);
    for (int i = 0; i < 3; ++i) {
        ins->x_cntr[i] = y[i];
        ins->u_cntr[i] = y[3 + i];
        ins->Omega_body[i] = y[10 + i];
    }
    for (int i = 0; i < 4; ++i) ins->quat[i] = y[6 + i] / qn;
}

}  // namespace

// The FP64 frame block (one thread): body and wing orientations and angular
// velocities, pivots, and the parts' bounding boxes.  frac = 0: at the state's
// time; frac > 0: at t0 + frac dt of the current step (the later RK4 stages,
// after k_scalars has written t0 and dt).
static __device__ void kinematics_frame(const flusi_insect* ins, const StepState* st, const StepCoef* coef,
                                        Frame* fr, double h, double frac, const Member* mb)
{
    if (mb) {
        const Member& m = mb[blockIdx.z];
        ins = m.ins;
        st = m.st;
        coef = m.coef;
        fr = m.fr;
    }
    const double t = frac > 0.0 ? coef->t0 + frac * coef->dt : st->t;
    Frame F;
    F.t = t;
    for (int i = 0; i < 3; ++i) {
        F.xc[i] = ins->x_cntr[i];
        F.uc[i] = ins->u_cntr[i];
    }
    M3 Mb;
    if (ins->free_flight) {
        // Sec. 3.6: the orientation is the quaternion's, Omega^(b) is state
        const M3 Q = quat_to_global(ins->quat);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Mb.a[3 * i + j] = Q.a[3 * j + i];
        apply(Q, ins->Omega_body, F.Ob);
    } else {
        // body frame: yaw, then pitch, then roll
        M3 Rx = rot_x(ins->psi), Ry = rot_y(ins->beta), Rz = rot_z(ins->gamma);
        Mb = mul(mul(Rx, Ry), Rz);
        // body angular velocity in the global frame (nested form of Sec. 3.1)
        double v[3] = {ins->psi_dot, 0, 0};
        apply_t(Rx, v, v);
        v[1] += ins->beta_dot;
        apply_t(Ry, v, v);
        v[2] += ins->gamma_dot;
        apply_t(Rz, v, F.Ob);
    }
    for (int i = 0; i < 9; ++i) F.Mb[i] = Mb.a[i];

    double phi, alpha, theta, dphi, dalpha, dtheta, ddphi, ddalpha, ddtheta;
    int nf = ins->nfourier;
    series(ins->phi_a0, ins->phi_a, ins->phi_b, nf, ins->freq, t, &phi, &dphi, &ddphi);
    series(ins->alpha_a0, ins->alpha_a, ins->alpha_b, nf, ins->freq, t, &alpha, &dalpha, &ddalpha);
    series(ins->theta_a0, ins->theta_a, ins->theta_b, nf, ins->freq, t, &theta, &dtheta, &ddtheta);

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
        // In the wing frame Omega^(w) = e_a + Ra (e_t + Rt e_p) with
        // e_a = (0, alpha', 0), e_t = (0, 0, -theta'), e_p = (phi', 0, 0).  Both
        // factors are rotations about one fixed axis, so d/dt (Ra x) =
        // Ra x' - e_a x (Ra x) and d/dt (Rt x) = Rt x' - e_t x (Rt x).
        {
            const double ea[3] = {0, sg * dalpha, 0}, et[3] = {0, 0, -dtheta}, ep[3] = {sg * dphi, 0, 0};
            const double dea[3] = {0, sg * ddalpha, 0}, det[3] = {0, 0, -ddtheta};
            const double dep[3] = {sg * ddphi, 0, 0};
            double rp[3], in[3], v[3], dv[3], c[3], drp[3];
            apply(Rt, ep, rp);                          // Rt e_p
            for (int i = 0; i < 3; ++i) in[i] = et[i] + rp[i];
            apply(Ra, in, v);                           // Ra (e_t + Rt e_p)
            for (int i = 0; i < 3; ++i) F.Oww[s][i] = ea[i] + v[i];
            apply(Rt, dep, drp);
            cross3(et, rp, c);
            for (int i = 0; i < 3; ++i) dv[i] = det[i] + drp[i] - c[i];
            apply(Ra, dv, dv);
            cross3(ea, v, c);
            for (int i = 0; i < 3; ++i) F.dOww[s][i] = dea[i] + dv[i] - c[i];
        }
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
        if (ins->body_type == 3) {
            // the arc x = x_c + r_c sin th, z = z_c + r_c cos th over
            // th0 -+ a/r_c: its ends and the quarter angles inside, grown by b
            const double rc = ins->body_arc[0], xc = ins->body_arc[1], zc = ins->body_arc[2];
            const double th0 = atan2(-xc, -zc), t1 = th0 - ins->body_a / rc, t2 = th0 + ins->body_a / rc;
            const double half_pi = 1.5707963267948966192313216916398;
            lo[0] = lo[2] = 1e300;
            hi[0] = hi[2] = -1e300;
            const int k1 = (int)ceil(t1 / half_pi), k2 = (int)floor(t2 / half_pi);
            for (int k = k1 - 1; k <= k2 + 1; ++k) {
                const double th = k < k1 ? t1 : k > k2 ? t2 : k * half_pi;
                const double px = xc + rc * sin(th), pz = zc + rc * cos(th);
                lo[0] = fmin(lo[0], px - ins->body_b);
                hi[0] = fmax(hi[0], px + ins->body_b);
                lo[2] = fmin(lo[2], pz - ins->body_b);
                hi[2] = fmax(hi[2], pz + ins->body_b);
            }
        }
        if (ins->body_type >= 2 && ins->head_r > 0)
            for (int i = 0; i < 3; ++i) {
                lo[i] = fmin(lo[i], ins->head_x0[i] - ins->head_r);
                hi[i] = fmax(hi[i], ins->head_x0[i] + ins->head_r);
            }
        if (ins->body_type >= 2 && ins->eye_r > 0)
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

// One warp.  Thread 0 forms the FP64 frame block; with `with_t`, the warp
// then writes its FP32 and FP64 copies with the mask shape S (FrameT, at their
// offsets of the frame slot) for the x pass.
__global__ void k_kinematics(const flusi_insect* ins, const StepState* st, const StepCoef* coef, Frame* fr,
                             double h, double frac, const Member* mb, Shape S, int with_t, double inv_eta)
{
    __shared__ Shape sS;
    if (blockIdx.x != 0) return;
    if (mb) fr = mb[blockIdx.z].fr;
    if (threadIdx.x == 0) {
        kinematics_frame(ins, st, coef, fr, h, frac, mb);
        if (with_t) sS = S;
    }
    if (!with_t || threadIdx.x >= 32) return;
    __syncwarp();
    const int lane = threadIdx.x;
    frame_to_t<float>(const_cast<FrameT<float>*>(frame_t<float>(fr)), fr, &sS, inv_eta, lane);
    frame_to_t<double>(const_cast<FrameT<double>*>(frame_t<double>(fr)), fr, &sS, inv_eta, lane);
}


// A bounded wait on a barrier that nothing completes (the arrival count is 2
// and one thread arrives once): gives up after max_cycles and reports as the
// tile loads do.
__global__ void k_wait_probe(int* err, long long max_cycles)
{
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 2);
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&bar)) : "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, max_cycles);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicCAS(err, 0, (int)FLUSI_ETIMEOUT);
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
//
// FP64 arithmetic is a small fraction of FP32 here, and a warp instruction
// costs the FP64 units the same with one lane active as with 32: the work is
// spread over lanes (a slot and segment of CTAs per thread, a force or moment
// component per lane) and each scalar is computed once, not by every thread.
constexpr int kScalarSeg = 6;   // CTA segments per slot: kNumSums * 6 = 240 threads
static_assert(kNumSums * kScalarSeg <= 256, "k_scalars runs 256 threads");

__global__ void k_scalars(Geom g, const double* part, int nparts, StepState* st, StepCoef* coef, double* rows,
                          int ring, double* etab, double3 opts, double dt_diff, const Frame* fr, flusi_insect* ins,
                          const Member* mb)
{
    if (mb) {
        const Member& m = mb[blockIdx.z];
        part = m.part;
        st = m.st;
        coef = m.coef;
        rows = m.rows;
        etab = m.etab;
        fr = m.fr;
        ins = m.ins;
        g.nu = m.nu;
    }
    __shared__ double seg[kNumSums][kScalarSeg];
    __shared__ double tot[kNumSums];
    __shared__ double sh_dt;
    const int tid = threadIdx.x, T = blockDim.x;

    // every thread reads the state before the first barrier; thread 0 writes
    // it only after the last one
    const int status = st->status;
    const long long n = st->n;
    const double dt_prev = st->dt_prev;
    if (status != 0) {
        if (tid == 0) coef->skip = 1;
        return;
    }
    // slot k, segment s: the partials of CTAs [s c, (s + 1) c) in order; then
    // the segments in order
    if (tid < kNumSums * kScalarSeg) {
        const int k = tid % kNumSums, sg = tid / kNumSums;
        const int chunk = (nparts + kScalarSeg - 1) / kScalarSeg;
        const int i0 = sg * chunk, i1 = min(nparts, i0 + chunk);
        const bool is_max = (k == kSumUmax2 || k == kSumBad);
        double acc = 0.0;
#pragma unroll 4
        for (int i = i0; i < i1; ++i) {
            const double v = part[(size_t)i * kNumSums + k];
            acc = is_max ? fmax(acc, v) : acc + v;
        }
        seg[k][sg] = acc;
    }
    __syncthreads();
    if (tid < kNumSums) {
        const bool is_max = (tid == kSumUmax2 || tid == kSumBad);
        double a = 0.0;
        for (int s2 = 0; s2 < kScalarSeg; ++s2) a = is_max ? fmax(a, seg[tid][s2]) : a + seg[tid][s2];
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
    if (tid == 0) {
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
        sh_dt = dt;
    }
    __syncthreads();
    const double dt = sh_dt;
    const int first = (n == 0);

    // integrating factors, separable per axis: E1 = e^{-nu |k|^2 dt},
    // E2 = e^{-nu |k|^2 (dt + dt_prev)}; layout [E1x Mx][E1y My][E1z Mz][E2x][E2y][E2z]
    // in FP64, then the same 2 Mt values rounded to FP32 (the FP32 update reads
    // those and converts nothing per mode)
    const double two_pi = 6.283185307179586476925286766559;
    const int Mt = g.Mx + g.My + g.Mz;
    float* etab32 = reinterpret_cast<float*>(etab + 2 * Mt);
    for (int i = tid; i < 2 * Mt; i += T) {
        int which = i / Mt, r = i % Mt;
        double k, tau = which == 0 ? dt : dt + dt_prev;
        if (r < g.Mx) k = two_pi * r / g.Lx;
        else if (r < g.Mx + g.My) k = two_pi * mode_of(r - g.Mx, g.Ky) / g.Ly;
        else k = two_pi * mode_of(r - g.Mx - g.My, g.Kz) / g.Lz;
        const double e = exp(-g.nu * k * k * tau);
        etab[i] = e;
        etab32[i] = float(e);
    }

    // force row: lane 3 p + i of warp 0 takes component i of part p; then the
    // wing power (lanes 0, 1) and the rest (lane 0)
    double* row = rows + (size_t)(n % ring) * kRowCols;
    if (tid < 9) {
        const int p = tid / 3, i = tid % 3;
        const double dV = g.dx * g.dy * g.dz;
        const double* s = tot + 12 * p;
        double Fv = s[i] * dV / g.eta, Mv = s[3 + i] * dV / g.eta;
        const double Is = s[6 + i] * dV, Js = s[9 + i] * dV;
        if (!first) {
            const double inv_dtp = 1.0 / dt_prev;
            Fv += (Is - st->Is_prev[p][i]) * inv_dtp;
            Mv += (Js - st->Js_prev[p][i]) * inv_dtp;
        }
        row[2 + 6 * p + i] = Fv;
        row[5 + 6 * p + i] = Mv;
        st->Is_prev[p][i] = Is;
        st->Js_prev[p][i] = Js;
    }
    __syncwarp();
    const Frame& F = *fr;
    if (tid < 2) {   // wing power at t^n (Sec. 3.5, Eq. insect_power)
        const int s = tid;
        double pa = 0.0, pi = 0.0;
        if (s < ins->nwings) {
            const double* m = row + 5 + 6 * (1 + s);
            pa = -(m[0] * F.Ow[s][0] + m[1] * F.Ow[s][1] + m[2] * F.Ow[s][2]);
            const double* J = ins->J_wing;   // xx yy zz xy xz yz
            const M3 Jm = {{J[0], J[3], J[4], J[3], J[1], J[5], J[4], J[5], J[2]}};
            const double* w = F.Oww[s];
            double Jw[3], Jdw[3], c[3];
            apply(Jm, w, Jw);
            apply(Jm, F.dOww[s], Jdw);
            cross3(w, Jw, c);
            pi = w[0] * (Jdw[0] + c[0]) + w[1] * (Jdw[1] + c[1]) + w[2] * (Jdw[2] + c[2]);
        }
        row[22 + s] = pa;
        row[24 + s] = pi;
    }
    __syncwarp();
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
        row[0] = st->t;
        row[1] = dt;
        row[20] = 0.5 * tot[kSumEkin] * g.dx * g.dy * g.dz;
        row[21] = umax;

        if (ins->free_flight) advance_body(ins, st, F, row, dt, first ? 0.0 : dt / dt_prev, first);

        st->t += dt;
        st->dt_prev = dt;
        st->n = n + 1;
    }
}

}  // namespace flusi

/*
 * Oracle insect module: mask function chi and solid velocity u_s of a body
 * and up to two rigid flapping wings (Sec. 3 of the FluSI paper), computed
 * point by point in the order the paper gives, with no bounding boxes and
 * no precomputed combined matrices.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Readings where the paper is silent, garbled or at odds with itself:
 *  - union of parts: chi = max over parts of chi_part, colour = the part
 *    attaining it, ties to the lowest colour (body 1 < left 2 < right 3);
 *  - thorax signed distance (Sec. 3.2) extended outside |x| > a by the
 *    distance to the tip, sqrt(y^2 + z^2 + (|x| - a)^2);
 *  - rectangular wing (Eq. signed_distance_rectangular_wing) read as
 *    max(x - c_le, -x - c_te, y - R, -y, |z| - h/2) in the wing frame;
 *  - wing angular velocity in the wing frame: Omega_w^(w) =
 *    M_wing M_stroke Omega_w^(b) (the printed M_wing alone maps a body-frame
 *    vector only when M_stroke = I);
 *  - wing velocity back to the global frame:
 *    u_w^(g) = M_body^-1 M_stroke^-1 M_wing^-1 u_w^(w), the inverse of
 *    x^(w) = M_wing M_stroke x^(b) (the printed order swaps the two);
 *  - right wing: the left-wing angular-velocity formula with (phi, alpha)
 *    replaced by (-phi, -alpha), matching the printed M_wing,r;
 *  - kinematic angles: a0/2 + sum_i a_i cos(2 pi i f t) + b_i sin(2 pi i f t),
 *    the Fourier form of Eq. Fourier_radious_wing with time as argument.
 */
#include "oracle.h"

#include <math.h>
#include <string.h>

static const double PI = 3.14159265358979323846;

/* Rotation matrices printed at the start of Sec. 3 (row major). */
void orc_rot_x(double xi, double *R)
{
    double c = cos(xi), s = sin(xi);
    double M[9] = {1, 0, 0, 0, c, s, 0, -s, c};
    memcpy(R, M, sizeof M);
}

void orc_rot_y(double xi, double *R)
{
    double c = cos(xi), s = sin(xi);
    double M[9] = {c, 0, -s, 0, 1, 0, s, 0, c};
    memcpy(R, M, sizeof M);
}

void orc_rot_z(double xi, double *R)
{
    double c = cos(xi), s = sin(xi);
    double M[9] = {c, s, 0, -s, c, 0, 0, 0, 1};
    memcpy(R, M, sizeof M);
}

static void mat_mul(const double *A, const double *B, double *C)
{
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[i * 3 + k] * B[k * 3 + j];
            T[i * 3 + j] = s;
        }
    memcpy(C, T, sizeof T);
}

static void mat_vec(const double *A, const double *x, double *y)
{
    double t[3];
    for (int i = 0; i < 3; ++i)
        t[i] = A[i * 3 + 0] * x[0] + A[i * 3 + 1] * x[1] + A[i * 3 + 2] * x[2];
    memcpy(y, t, sizeof t);
}

/* y = A^T x, the inverse of a rotation matrix applied to x. */
static void mat_tvec(const double *A, const double *x, double *y)
{
    double t[3];
    for (int i = 0; i < 3; ++i)
        t[i] = A[0 * 3 + i] * x[0] + A[1 * 3 + i] * x[1] + A[2 * 3 + i] * x[2];
    memcpy(y, t, sizeof t);
}

static void cross(const double *a, const double *b, double *c)
{
    double t[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2],
                   a[0] * b[1] - a[1] * b[0]};
    memcpy(c, t, sizeof t);
}

static void fourier_series(double a0, const double *a, const double *b, int nf,
                           double f, double t, double *val, double *dval, double *ddval)
{
    double v = 0.5 * a0, dv = 0, ddv = 0;
    for (int i = 1; i <= nf; ++i) {
        double w = 2.0 * PI * i * f;
        v += a[i - 1] * cos(w * t) + b[i - 1] * sin(w * t);
        dv += w * (-a[i - 1] * sin(w * t) + b[i - 1] * cos(w * t));
        ddv -= w * w * (a[i - 1] * cos(w * t) + b[i - 1] * sin(w * t));
    }
    *val = v;
    *dval = dv;
    *ddval = ddv;
}

/* Derivatives of the passive rotations R_y, R_z with respect to the angle. */
static void rot_y_d(double xi, double *R)
{
    double c = cos(xi), s = sin(xi);
    double M[9] = {-s, 0, -c, 0, 0, 0, c, 0, -s};
    memcpy(R, M, sizeof M);
}

static void rot_z_d(double xi, double *R)
{
    double c = cos(xi), s = sin(xi);
    double M[9] = {-s, c, 0, -c, -s, 0, 0, 0, 0};
    memcpy(R, M, sizeof M);
}

/* Free-flight orientation (Sec. 3.6): the printed quaternion matrix maps body
 * to global coordinates, the transpose of M_body of Eq. M_body_yawpitchroll
 * (with the printed initial quaternion of (psi, beta, gamma) the two agree). */
static void quat_body_to_global(const double *e, double *R)
{
    double e0 = e[0], e1 = e[1], e2 = e[2], e3 = e[3];
    double M[9] = {e0 * e0 + e1 * e1 - e2 * e2 - e3 * e3, 2 * (e1 * e2 - e3 * e0), 2 * (e1 * e3 + e2 * e0),
                   2 * (e1 * e2 + e3 * e0), e0 * e0 - e1 * e1 + e2 * e2 - e3 * e3, 2 * (e2 * e3 - e1 * e0),
                   2 * (e1 * e3 - e2 * e0), 2 * (e2 * e3 + e1 * e0), e0 * e0 - e1 * e1 - e2 * e2 + e3 * e3};
    memcpy(R, M, sizeof M);
}

void orc_quat_from_angles(double psi, double beta, double gamma, double *eps)
{
    double cp = cos(0.5 * psi), sp = sin(0.5 * psi), cb = cos(0.5 * beta), sb = sin(0.5 * beta);
    double cg = cos(0.5 * gamma), sg = sin(0.5 * gamma);
    eps[0] = cp * cb * cg + sp * sb * sg;
    eps[1] = sp * cb * cg - cp * sb * sg;
    eps[2] = cp * sb * cg + sp * cb * sg;
    eps[3] = cp * cb * sg - sp * sb * cg;
}

/* Right-hand side of the 13 free-flight equations (Eq. oh_my_god_look_a_vector)
 * for the state in the descriptor: F the total aerodynamic force (global),
 * m_b the total aerodynamic moment about x_cntr in the body frame.  The six
 * dof flags multiply the accelerations. */
void orc_body_rhs(const orc_insect *ins, const double *F, const double *m_b, double *f)
{
    const double *e = ins->quat, *W = ins->Omega_body, *J = ins->J_body;
    for (int i = 0; i < 3; ++i) f[i] = ins->u_cntr[i];
    f[3] = ins->dof[0] * F[0] / ins->mass;
    f[4] = ins->dof[1] * F[1] / ins->mass;
    f[5] = ins->dof[2] * (F[2] / ins->mass - ins->gravity);
    f[6] = 0.5 * (-e[1] * W[0] - e[2] * W[1] - e[3] * W[2]);
    f[7] = 0.5 * (e[0] * W[0] - e[3] * W[1] + e[2] * W[2]);
    f[8] = 0.5 * (e[3] * W[0] + e[0] * W[1] - e[1] * W[2]);
    f[9] = 0.5 * (-e[2] * W[0] + e[1] * W[1] + e[0] * W[2]);
    f[10] = ins->dof[3] * ((J[1] - J[2]) * W[1] * W[2] + m_b[0]) / J[0];
    f[11] = ins->dof[4] * ((J[2] - J[0]) * W[2] * W[0] + m_b[1]) / J[1];
    f[12] = ins->dof[5] * ((J[0] - J[1]) * W[0] * W[1] + m_b[2]) / J[2];
}

/* Power of each wing (Sec. 3.5, Eq. insect_power): aerodynamic
 * P = -m . (Omega_w - Omega_b) with the wing's moment about its pivot (force
 * row) and its rotation rate relative to the body in the global frame;
 * inertial P = Omega^(w) . (J Omega'^(w) + Omega^(w) x J Omega^(w)). */
void orc_wing_power(const orc_insect *ins, const orc_frames *fr, const double *row, double *p_aero,
                    double *p_inert)
{
    const double *J6 = ins->J_wing;
    const double J[9] = {J6[0], J6[3], J6[4], J6[3], J6[1], J6[5], J6[4], J6[5], J6[2]};
    for (int s = 0; s < 2; ++s) {
        p_aero[s] = p_inert[s] = 0.0;
        if (s >= ins->nwings) continue;
        double wg[3];
        mat_tvec(fr->M_body, fr->Omega_w_b[s], wg);
        const double *m = row + 2 + (1 + s) * 6 + 3;
        p_aero[s] = -(m[0] * wg[0] + m[1] * wg[1] + m[2] * wg[2]);
        const double *w = fr->Omega_w_w[s], *dw = fr->dOmega_w_w[s];
        double Jw[3], Jdw[3], c[3];
        mat_vec(J, w, Jw);
        mat_vec(J, dw, Jdw);
        cross(w, Jw, c);
        p_inert[s] = w[0] * (Jdw[0] + c[0]) + w[1] * (Jdw[1] + c[1]) + w[2] * (Jdw[2] + c[2]);
    }
}

void orc_frames_at(const orc_insect *ins, double t, orc_frames *fr)
{
    double Rx[9], Ry[9], Rz[9], v[3];
    memset(fr, 0, sizeof *fr);

    if (ins->free_flight) {
        /* Sec. 3.6: orientation from the quaternion, Omega^(b) from the state */
        double Rq[9];
        quat_body_to_global(ins->quat, Rq);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) fr->M_body[3 * i + j] = Rq[3 * j + i];
        mat_tvec(fr->M_body, ins->Omega_body, fr->Omega_b_g);
    } else {
        /* Body frame, Eq. M_body_yawpitchroll: yaw, then pitch, then roll. */
        orc_rot_x(ins->psi, Rx);
        orc_rot_y(ins->beta, Ry);
        orc_rot_z(ins->gamma, Rz);
        mat_mul(Rx, Ry, fr->M_body);
        mat_mul(fr->M_body, Rz, fr->M_body);

        /* Body angular velocity in the global frame (Sec. 3.1, nested form). */
        double e_psi[3] = {ins->psi_dot, 0, 0};
        double e_beta[3] = {0, ins->beta_dot, 0};
        double e_gamma[3] = {0, 0, ins->gamma_dot};
        mat_tvec(Rx, e_psi, v);
        for (int i = 0; i < 3; ++i) v[i] += e_beta[i];
        mat_tvec(Ry, v, v);
        for (int i = 0; i < 3; ++i) v[i] += e_gamma[i];
        mat_tvec(Rz, v, fr->Omega_b_g);
    }

    /* Wing angles from their Fourier coefficients (Sec. 3.3). */
    int nf = ins->nfourier;
    fourier_series(ins->phi_a0, ins->phi_a, ins->phi_b, nf, ins->freq, t,
                   &fr->phi, &fr->phi_dot, &fr->phi_ddot);
    fourier_series(ins->alpha_a0, ins->alpha_a, ins->alpha_b, nf, ins->freq, t,
                   &fr->alpha, &fr->alpha_dot, &fr->alpha_ddot);
    fourier_series(ins->theta_a0, ins->theta_a, ins->theta_b, nf, ins->freq, t,
                   &fr->theta, &fr->theta_dot, &fr->theta_ddot);

    for (int s = 0; s < 2; ++s) {
        double sg = s == 0 ? 1.0 : -1.0;
        double phi = sg * fr->phi, alpha = sg * fr->alpha, theta = fr->theta;
        double phid = sg * fr->phi_dot, alphad = sg * fr->alpha_dot;
        double thetad = fr->theta_dot;

        /* M_stroke,l = R_y(eta); M_stroke,r = R_x(pi) R_y(eta). */
        orc_rot_y(ins->eta_stroke, Ry);
        if (s == 0) {
            memcpy(fr->M_stroke[s], Ry, sizeof Ry);
        } else {
            orc_rot_x(PI, Rx);
            mat_mul(Rx, Ry, fr->M_stroke[s]);
        }
        /* M_wing = R_y(alpha) R_z(-theta) R_x(phi) (signs flipped on the right). */
        double Ra[9], Rt[9], Rp[9];
        orc_rot_y(alpha, Ra);
        orc_rot_z(-theta, Rt);
        orc_rot_x(phi, Rp);
        mat_mul(Ra, Rt, fr->M_wing[s]);
        mat_mul(fr->M_wing[s], Rp, fr->M_wing[s]);

        /* Omega_w^(b): nested form of Sec. 3.3. */
        double e_alpha[3] = {0, alphad, 0};
        double e_theta[3] = {0, 0, -thetad};
        double e_phi[3] = {phid, 0, 0};
        mat_tvec(Ra, e_alpha, v);
        for (int i = 0; i < 3; ++i) v[i] += e_theta[i];
        mat_tvec(Rt, v, v);
        for (int i = 0; i < 3; ++i) v[i] += e_phi[i];
        mat_tvec(Rp, v, v);
        mat_tvec(fr->M_stroke[s], v, fr->Omega_w_b[s]);

        /* Omega_w^(w) = M_wing M_stroke Omega_w^(b). */
        mat_vec(fr->M_stroke[s], fr->Omega_w_b[s], v);
        mat_vec(fr->M_wing[s], v, fr->Omega_w_w[s]);

        /* its time derivative: Omega^(w) = e_alpha + Ra e_theta + Ra Rt e_phi, so
         * d/dt = e_alpha' + Ra' e_theta + Ra e_theta' + (Ra' Rt + Ra Rt') e_phi
         * + Ra Rt e_phi' with Ra' = alpha' dR_y, Rt' = -theta' dR_z */
        {
            double alphadd = sg * fr->alpha_ddot, phidd = sg * fr->phi_ddot, thetadd = fr->theta_ddot;
            double dRa[9], dRt[9], A[9], B[9], t1[3], t2[3], t3[3];
            rot_y_d(alpha, dRa);
            rot_z_d(-theta, dRt);
            for (int i = 0; i < 9; ++i) {
                dRa[i] *= alphad;
                dRt[i] *= -thetad;
            }
            double d_theta[3] = {0, 0, -thetadd}, d_phi[3] = {phidd, 0, 0};
            double *out = fr->dOmega_w_w[s];
            out[0] = 0;
            out[1] = alphadd;
            out[2] = 0;
            mat_vec(dRa, e_theta, t1);
            mat_vec(Ra, d_theta, t2);
            mat_mul(dRa, Rt, A);
            mat_mul(Ra, dRt, B);
            for (int i = 0; i < 9; ++i) A[i] += B[i];
            mat_vec(A, e_phi, t3);
            for (int i = 0; i < 3; ++i) out[i] += t1[i] + t2[i] + t3[i];
            mat_mul(Ra, Rt, A);
            mat_vec(A, d_phi, t1);
            for (int i = 0; i < 3; ++i) out[i] += t1[i];
        }

        /* Pivot in the global frame: x_cntr + M_body^-1 x_pivot^(b). */
        const double *pb = s == 0 ? ins->pivot_l : ins->pivot_r;
        mat_tvec(fr->M_body, pb, v);
        for (int i = 0; i < 3; ++i) fr->pivot_g[s][i] = ins->x_cntr[i] + v[i];
    }
}

/* Smoothed mask as a function of the signed distance (Eq.
 * smoothing_mask_as_function_of_delta), or the tanh layer. */
double orc_mask_profile(int profile, double delta, double h)
{
    if (profile == 1) return 0.5 * (1.0 - tanh(delta / h));
    if (delta <= -h) return 1.0;
    if (delta >= h) return 0.0;
    return 0.5 * (1.0 + cos(PI * (delta + h) / (2.0 * h)));
}

/* Signed distance of the body in its frame (Sec. 3.2).  The thorax is the
 * ellipsoid rotationally symmetric about x^(b); head and eyes are spheres
 * |x - x0| - r (the printed forms omit the radius).  The parts are joined
 * by the minimum of their distances, the union of negative-inside sets (the
 * printed max would be their intersection). */
/* Thorax whose centre line is an arc of the circle of radius rc about
 * (xc, 0, zc), with circular cross-sections centred on the arc (the
 * fruit-fly body of Sec. 5.3 has this form).  Along the arc the
 * thorax profile of the straight body applies with the arc length s, measured
 * from the arc point in the direction of the body origin, in place of x^(b):
 * radius b sqrt(1 - (s/a)^2) for |s| <= a, beyond it the distance to the arc's
 * end point. */
static double curved_thorax_distance(const orc_insect *ins, const double *xb)
{
    const double a = ins->body_a, b = ins->body_b;
    const double rc = ins->body_arc[0], xc = ins->body_arc[1], zc = ins->body_arc[2];
    /* angles about the circle's centre, from +z^(b) towards +x^(b) */
    const double th0 = atan2(-xc, -zc);
    const double vx = xb[0] - xc, vz = xb[2] - zc;
    double dth = atan2(vx, vz) - th0;
    while (dth > PI) dth -= 2.0 * PI;
    while (dth <= -PI) dth += 2.0 * PI;
    const double s = rc * dth;
    const double rp = sqrt(vx * vx + vz * vz);
    if (fabs(s) <= a) {
        const double dc = sqrt((rp - rc) * (rp - rc) + xb[1] * xb[1]);
        return dc - b * sqrt(1.0 - (s / a) * (s / a));
    }
    const double te = th0 + (s > 0 ? a : -a) / rc;
    const double ex = xc + rc * sin(te), ez = zc + rc * cos(te);
    return sqrt((xb[0] - ex) * (xb[0] - ex) + xb[1] * xb[1] + (xb[2] - ez) * (xb[2] - ez));
}

double orc_body_distance(const orc_insect *ins, const double *xb)
{
    if (ins->body_type == 1)
        return sqrt(xb[0] * xb[0] + xb[1] * xb[1] + xb[2] * xb[2]) - ins->body_a;
    double d;
    if (ins->body_type == 3) {
        d = curved_thorax_distance(ins, xb);
    } else {
        double a = ins->body_a, b = ins->body_b;
        double rr = sqrt(xb[1] * xb[1] + xb[2] * xb[2]);
        double ax = fabs(xb[0]);
        if (ax <= a) d = rr - sqrt(b * b * (1.0 - (xb[0] / a) * (xb[0] / a)));
        else d = sqrt(rr * rr + (ax - a) * (ax - a));
    }
    if (ins->head_r > 0) {
        double e[3] = {xb[0] - ins->head_x0[0], xb[1] - ins->head_x0[1], xb[2] - ins->head_x0[2]};
        double dh = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) - ins->head_r;
        if (dh < d) d = dh;
    }
    if (ins->eye_r > 0) {
        for (int s = 0; s < 2; ++s) {
            double y0 = s == 0 ? ins->eye_x0[1] : -ins->eye_x0[1];
            double e[3] = {xb[0] - ins->eye_x0[0], xb[1] - y0, xb[2] - ins->eye_x0[2]};
            double de = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]) - ins->eye_r;
            if (de < d) d = de;
        }
    }
    return d;
}

/* Contour radius R(theta), Eq. Fourier_radious_wing with the angle in
 * radians (the printed argument 2 pi i theta takes theta in turns). */
static double contour_radius(const orc_insect *ins, double th)
{
    double R = 0.5 * ins->contour_a0;
    for (int i = 1; i <= ins->ncontour; ++i)
        R += ins->contour_a[i - 1] * cos(i * th) + ins->contour_b[i - 1] * sin(i * th);
    return R;
}

/* Signed distance of a wing in its frame (Sec. 3.4). */
double orc_wing_distance(const orc_insect *ins, const double *xw)
{
    double dz = fabs(xw[2]) - 0.5 * ins->wing_h;
    if (ins->wing_shape == 1) {
        double dx = xw[0] - ins->contour_xc, dy = xw[1] - ins->contour_yc;
        double r = sqrt(dx * dx + dy * dy);
        double d = r - contour_radius(ins, atan2(dy, dx));
        return dz > d ? dz : d;
    }
    double d = xw[0] - ins->wing_c_le;
    double e;
    e = -xw[0] - ins->wing_c_te;
    if (e > d) d = e;
    e = xw[1] - ins->wing_R;
    if (e > d) d = e;
    e = -xw[1];
    if (e > d) d = e;
    if (dz > d) d = dz;
    return d;
}

void orc_solid_at(const orc_insect *ins, const orc_frames *fr, double h,
                  const double x[3], double *chi, int *colour, double us[3])
{
    double r[3], xb[3], Ob_b[3], ub[3], v[3];
    for (int i = 0; i < 3; ++i) r[i] = x[i] - ins->x_cntr[i];
    mat_vec(fr->M_body, r, xb);

    /* body velocity field, Eq. body_velocity_field */
    mat_vec(fr->M_body, fr->Omega_b_g, Ob_b);
    cross(Ob_b, xb, v);
    mat_tvec(fr->M_body, v, v);
    for (int i = 0; i < 3; ++i) ub[i] = ins->u_cntr[i] + v[i];

    *chi = 0.0;
    *colour = 0;
    us[0] = us[1] = us[2] = 0.0;

    if (ins->body_type != 0) {
        double c = orc_mask_profile(ins->profile, orc_body_distance(ins, xb), h);
        if (c > *chi) {
            *chi = c;
            *colour = 1;
            for (int i = 0; i < 3; ++i) us[i] = ub[i];
        }
    }
    for (int s = 0; s < ins->nwings && s < 2; ++s) {
        const double *pb = s == 0 ? ins->pivot_l : ins->pivot_r;
        double xs[3], xw[3];
        for (int i = 0; i < 3; ++i) xs[i] = xb[i] - pb[i];
        mat_vec(fr->M_stroke[s], xs, xs);
        mat_vec(fr->M_wing[s], xs, xw);
        double c = orc_mask_profile(ins->profile, orc_wing_distance(ins, xw), h);
        if (c > *chi) {
            /* Eq. wing_velocity_field, then u_s = u_w + u_b */
            double uw[3];
            cross(fr->Omega_w_w[s], xw, uw);
            mat_tvec(fr->M_wing[s], uw, uw);
            mat_tvec(fr->M_stroke[s], uw, uw);
            mat_tvec(fr->M_body, uw, uw);
            *chi = c;
            *colour = 2 + s;
            for (int i = 0; i < 3; ++i) us[i] = uw[i] + ub[i];
        }
    }
}

static double layer_h(const orc_params *p, const orc_insect *ins)
{
    double dx = p->Lx / p->nx, dy = p->Ly / p->ny, dz = p->Lz / p->nz;
    double d = dx > dy ? dx : dy;
    if (dz > d) d = dz;
    return ins->c_smth * d;
}

void orc_mask_grid(const orc_params *p, const orc_insect *ins, double t,
                   double *chi, int32_t *colour, double *us)
{
    orc_frames fr;
    orc_frames_at(ins, t, &fr);
    double h = layer_h(p, ins);
    long N = (long)p->nx * p->ny * p->nz;
    for (long z = 0; z < p->nz; ++z)
        for (long y = 0; y < p->ny; ++y)
            for (long x = 0; x < p->nx; ++x) {
                long idx = (z * p->ny + y) * p->nx + x;
                double X[3] = {x * p->Lx / p->nx, y * p->Ly / p->ny, z * p->Lz / p->nz};
                double c, u3[3];
                int col;
                orc_solid_at(ins, &fr, h, X, &c, &col, u3);
                chi[idx] = c;
                colour[idx] = col;
                for (int i = 0; i < 3; ++i) us[i * N + idx] = u3[i];
            }
}

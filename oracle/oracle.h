/*
 * Plain FP64 CPU oracle for one time step of the volume-penalized
 * incompressible Navier-Stokes equations in rotational form, solved by a
 * Fourier pseudo-spectral method in a periodic box (Engels, Kolomenskiy,
 * Schneider, Sesterhenn, "FluSI", Sec. 2 and Sec. 3, Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path; it
 * is slow on purpose and is called only by the tests, the smoke check and
 * the CPU-baseline leg of the benchmark.  It shares no code, header or table
 * with the CUDA library.
 *
 * Conventions (readings of the paper where it is silent):
 *   grid        x_i = i*Lx/nx, i = 0..nx-1 (same for y, z)
 *   physical    u[c][z][y][x], x fastest, c = 0..2
 *   spectral    uh[c][z][y][x], x = 0..nx/2 (half spectrum), complex
 *   transform   uh = FFT(u)/N  so that  u(x) = sum_k uh_k exp(i k.x)
 *   wavenumber  k = 2*pi*m/L with m_x in 0..nx/2 and m_y, m_z in
 *               {0..n/2-1, -n/2..-1}
 */
#ifndef FLUSI_ORACLE_H
#define FLUSI_ORACLE_H

#include <complex.h>
#include <stdint.h>

#define ORC_MAX_FOURIER 8
#define ORC_MAX_CONTOUR 32   /* harmonics of a wing contour R(theta)     */
#define ORC_NCOLOURS 3   /* 1 = body, 2 = left wing, 3 = right wing */
#define ORC_ROW_COLS 26  /* t, dt, {F[3], M[3]} x 3 colours, E_kin, u_max,
                            P_aero (left, right wing), P_inert (left, right) */

typedef struct {
    int nx, ny, nz;
    int dealias_strict;  /* 0: keep |m| <= floor(n/3); 1: keep |m| < n/3 */
    double Lx, Ly, Lz;
    double nu;           /* kinematic viscosity                           */
    double eta;          /* penalization constant C_eta                   */
    double cfl;          /* CFL number for the adaptive step              */
    double dt_fixed;     /* > 0: fixed step; 0: adaptive                  */
    double dt_max;       /* > 0: upper bound on the adaptive step         */
    int mean_mode;       /* 0: k = 0 mode held at u_inf; 1: evolves       */
    int pad_;
    double u_inf[3];
    /* Wake removal (Sec. 2.3).  Vorticity sponge: constant C_sp (0: off) and
     * the sponge region, the union over axes i of x_i >= L_i - sponge_width[i]
     * (width 0: none on that axis).  Dirichlet layer: u = u_inf penalized with
     * C_eta in x_i >= L_i - layer_width[i] (width 0: none).                 */
    double sponge_c;
    double sponge_width[3];
    double layer_width[3];
    int time_scheme;     /* 0: integrating-factor AB2; 1: RK4, explicit diffusion */
    int pad2_;
} orc_params;

typedef struct {
    int body_type;       /* 0 none, 1 sphere, 2 ellipsoid (thorax), 3 thorax on a circular centre line */
    int nwings;          /* 0, 1 (left only) or 2                         */
    int profile;         /* 0: cosine layer of Sec. 2.2, 1: tanh layer    */
    int nfourier;        /* harmonics used in the kinematics series       */
    double c_smth;       /* layer half-thickness h = c_smth * dx          */
    double x_cntr[3], u_cntr[3];
    double psi, beta, gamma;             /* roll, pitch, yaw              */
    double psi_dot, beta_dot, gamma_dot;
    double body_a, body_b;               /* sphere radius = body_a         */
    double pivot_l[3], pivot_r[3];       /* body frame                     */
    double eta_stroke;                   /* anatomical stroke-plane angle  */
    double wing_c_le, wing_c_te, wing_R, wing_h;
    double freq;
    double phi_a0, phi_a[ORC_MAX_FOURIER], phi_b[ORC_MAX_FOURIER];
    double alpha_a0, alpha_a[ORC_MAX_FOURIER], alpha_b[ORC_MAX_FOURIER];
    double theta_a0, theta_a[ORC_MAX_FOURIER], theta_b[ORC_MAX_FOURIER];
    /* Head and eye spheres joined to the thorax (Sec. 3.2), body frame;
     * radius 0: absent.  The right eye mirrors the left one in y^(b). */
    double head_x0[3], head_r;
    double eye_x0[3], eye_r;
    /* Wing outline (Sec. 3.4): 0 = rectangular plate (wing_c_le, wing_c_te,
     * wing_R); 1 = contour R(theta) = a0/2 + sum a_i cos(i theta) + b_i sin(i theta)
     * about (contour_xc, contour_yc) in the wing plane, theta measured from
     * x^(w) towards y^(w). */
    int wing_shape;
    int ncontour;
    double contour_xc, contour_yc;
    double contour_a0, contour_a[ORC_MAX_CONTOUR], contour_b[ORC_MAX_CONTOUR];
    /* Wing tensor of inertia in the wing frame (xx, yy, zz, xy, xz, yz) for
     * the inertial power (Sec. 3.5). */
    double J_wing[6];
    /* Free flight (Sec. 3.6): 0 = tethered (the body moves as the fields
     * above prescribe); 1 = x_cntr, u_cntr, quat and Omega_body are the state
     * of the Newton-Euler system, advanced by each step. */
    int free_flight;
    int pad3_;
    double mass, gravity;       /* M and g (gravity along -z)                    */
    double J_body[3];           /* principal moments of inertia, body axes        */
    double dof[6];              /* 1/0 on du_x, du_y, du_z, dOmega_x, dOmega_y, dOmega_z */
    double quat[4];             /* orientation epsilon_0..3 (free flight)         */
    double Omega_body[3];       /* Omega^(b) (free flight)                        */
    /* body_type 3: centre-line circle of radius body_arc[0] about
     * (body_arc[1], 0, body_arc[2]) in the x^(b)-z^(b) plane (Sec. 5.3). */
    double body_arc[3];
} orc_insect;

/* Time-level data of the AB2 scheme besides the two spectral fields. */
typedef struct {
    double t;
    double dt_prev;
    int64_t n;
    double Is_prev[ORC_NCOLOURS][3];   /* sum chi u_s dV per colour          */
    double Js_prev[ORC_NCOLOURS][3];   /* sum r x chi u_s dV per colour      */
    double body_rhs_prev[13];          /* free flight: previous ODE right-hand side */
} orc_scalars;

/* Frames of Sec. 3 evaluated at one instant (for the pins). */
typedef struct {
    double M_body[9];
    double Omega_b_g[3];
    double M_stroke[2][9], M_wing[2][9];
    double Omega_w_b[2][3], Omega_w_w[2][3];
    double dOmega_w_w[2][3];           /* time derivative of Omega_w^(w)    */
    double pivot_g[2][3];
    double phi, alpha, theta, phi_dot, alpha_dot, theta_dot;
    double phi_ddot, alpha_ddot, theta_ddot;
} orc_frames;

/* ---- FFT (own code; no library) ---- */
void orc_fft1(int n, double complex *data, int sign);
void orc_fft3_r2c(int nx, int ny, int nz, const double *in, double complex *out);
void orc_fft3_c2r(int nx, int ny, int nz, const double complex *in, double *out);
void orc_dft3_r2c(int nx, int ny, int nz, const double *in, double complex *out);

/* ---- insect module (Sec. 3) ---- */
void orc_rot_x(double xi, double *R);
void orc_rot_y(double xi, double *R);
void orc_rot_z(double xi, double *R);
void orc_frames_at(const orc_insect *ins, double t, orc_frames *fr);
void orc_quat_from_angles(double psi, double beta, double gamma, double *eps);
void orc_body_rhs(const orc_insect *ins, const double *F, const double *m_b, double *f);
void orc_wing_power(const orc_insect *ins, const orc_frames *fr, const double *row, double *p_aero,
                    double *p_inert);
double orc_mask_profile(int profile, double delta, double h);
double orc_body_distance(const orc_insect *ins, const double *xb);
double orc_wing_distance(const orc_insect *ins, const double *xw);
void orc_solid_at(const orc_insect *ins, const orc_frames *fr, double h,
                  const double x[3], double *chi, int *colour, double us[3]);
void orc_mask_grid(const orc_params *p, const orc_insect *ins, double t,
                   double *chi, int32_t *colour, double *us);

/* ---- spectral operators (Sec. 2.4) ---- */
void orc_dealias(const orc_params *p, double complex *fh, int ncomp);
double orc_sponge_mask(const orc_params *p, const double *X);
double orc_layer_mask(const orc_params *p, const double *X);
void orc_sponge_term(const orc_params *p, const double complex *vh, double complex *sh);
void orc_project(const orc_params *p, double complex *fh);
void orc_curl(const orc_params *p, const double complex *uh, double complex *wh);
void orc_forward(const orc_params *p, const double *u, double complex *uh, int ncomp);
void orc_inverse(const orc_params *p, const double complex *uh, double *u, int ncomp);

/* ---- time stepping (Algorithm 1) ---- */
int orc_set_state(const orc_params *p, const double *u, double complex *uh,
                  double complex *nh_prev, orc_scalars *s);
void orc_get_state(const orc_params *p, const double complex *uh, double *u);
int orc_rhs(const orc_params *p, const orc_insect *ins, double t,
            const double complex *uh, double complex *nh, double *sums);
/* fields [14][nz][ny][nx]: u(3), omega(3), chi, colour, u_s(3),
 * u x omega - chi/C_eta (u - u_s) (3) */
void orc_physical_fields(const orc_params *p, const orc_insect *ins, double t,
                         const double complex *uh, double *fields);
void orc_rk4_combine(const orc_params *p, double complex *uh, const double complex *k1,
                     const double complex *k2, const double complex *k3,
                     const double complex *k4, double dt);
void orc_ab2_update(const orc_params *p, double complex *uh,
                    const double complex *nh, const double complex *nh_prev,
                    double dt, double dt_prev, int64_t n);
int orc_step(const orc_params *p, orc_insect *ins, double complex *uh,
             double complex *nh_prev, orc_scalars *s, double *row);

/* Layout of the sums written by orc_rhs (doubles). */
#define ORC_SUM_FP(c) ((c) * 12 + 0)  /* sum chi (u - u_s) dV / C_eta      */
#define ORC_SUM_MP(c) ((c) * 12 + 3)  /* sum r x chi (u - u_s) dV / C_eta  */
#define ORC_SUM_IS(c) ((c) * 12 + 6)  /* sum chi u_s dV                     */
#define ORC_SUM_JS(c) ((c) * 12 + 9)  /* sum r x chi u_s dV                 */
#define ORC_SUM_EKIN 36               /* 1/2 sum |u|^2 dV                  */
#define ORC_SUM_UMAX 37               /* max |u|                           */
#define ORC_SUM_NONFINITE 38          /* 1 if any u or NL value not finite */
#define ORC_NSUMS 39

#endif

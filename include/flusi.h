/*
 * libflusi -- one time step of the volume-penalized incompressible
 * Navier-Stokes equations in rotational form, solved by a Fourier
 * pseudo-spectral method in a periodic box, on one GB300 GPU (sm_103a).
 *
 * Method: Engels, Kolomenskiy, Schneider, Sesterhenn, "FluSI: a novel
 * parallel simulation tool for flapping insect flight using a Fourier method
 * with volume penalization" (arXiv 1506.06513): Eq. PNST_org_momentum (the
 * vorticity sponge and the Dirichlet inflow layer of Sec. 2.3 as options),
 * Sec. 2.4 (discretization, 2/3 rule, AB2 with integrating factor, or RK4),
 * Sec. 3 (insect geometry, kinematics, power and free flight), Algorithm 1
 * (one step).
 *
 * Conventions shared by every entry point
 *  - Grid x_i = i*Lx/nx (same for y, z); physical fields are [3][nz][ny][nx],
 *    x fastest, component-major.
 *  - Spectral fields returned to the caller are the half spectrum
 *    [3][nz][ny][nx/2+1] of u_hat = FFT(u)/N, so u(x) = sum_k u_hat_k e^{i k.x};
 *    k = 2 pi m / L with m_x in 0..nx/2 and m_y, m_z in {0..n/2-1, -n/2..-1}.
 *  - Every call returns a status code (flusi_status); nothing aborts or throws
 *    across the ABI.  flusi_last_error() describes the last failure.
 *  - A handle is not thread-safe; use one host thread per handle.
 *  - Host arrays are owned by the caller and copied synchronously on the bound
 *    stream, except by flusi_forces_async, which only enqueues its copy.
 *    Device pointers passed in are owned by the caller.
 *  - Errors found on the device (a non-finite velocity or nonlinear term) land
 *    in a device status word; they surface at the next call that synchronizes
 *    (flusi_forces, flusi_get_state, flusi_get_spectrum, flusi_sync), after
 *    which flusi_step returns FLUSI_ESTATE until the next flusi_set_state.
 */
#ifndef FLUSI_H
#define FLUSI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct flusi_s *flusi_t;

typedef enum {
    FLUSI_OK = 0,
    FLUSI_EINVAL = 1,    /* bad argument (size, pointer, option, call order)   */
    FLUSI_ENOMEM = 2,    /* bound workspace smaller than flusi_workspace_bytes */
    FLUSI_ECUDA = 3,     /* a CUDA runtime call failed                         */
    FLUSI_ENONFINITE = 4,/* a non-finite u or u x omega - chi/C_eta (u - u_s)  */
    FLUSI_ETIMEOUT = 5,  /* a device-side wait gave up                        */
    FLUSI_ESTATE = 6     /* no state set, not bound, or poisoned by an error   */
} flusi_status;

/* Arithmetic of the state, the FFTs and the pointwise products.  Force,
 * energy and CFL reductions and the kinematics are FP64 in all of them.
 *  FLUSI_FP64, FLUSI_FP32: every transform and product in that precision.
 *  FLUSI_FP32_SPLITBF16: FP32 state, y and z transforms and pointwise
 *    products; the DFT stages of the physical x pass (the c2r transforms of
 *    u and omega and the r2c transforms of the nonlinear term, Sec. 2.4) run
 *    on the tensor cores as BF16 matrix products with FP32 accumulation, each
 *    operand split into a hi + lo pair of BF16 values and the product taken
 *    as hi*hi + hi*lo + lo*hi (relative error of a product about 2^-16).
 *  FLUSI_FP32_SPLITBF16X3: the same with hi + mid + lo pieces and the six
 *    products of order up to 2^-16 (error at the FP32 rounding level).
 * The split forms need nx = 256 or 512 (else flusi_create fails with
 * FLUSI_EINVAL); the vorticity sponge's extra x round trip, set_state and
 * get_state transforms stay in FP32 arithmetic. */
typedef enum {
    FLUSI_FP64 = 0,
    FLUSI_FP32 = 1,
    FLUSI_FP32_SPLITBF16 = 2,
    FLUSI_FP32_SPLITBF16X3 = 3
} flusi_precision;

/* Where an array passed to set_state / get_state lives. */
typedef enum { FLUSI_HOST_FP64 = 0, FLUSI_HOST_FP32 = 1, FLUSI_DEVICE = 2 } flusi_where;

#define FLUSI_MAX_FOURIER 8
#define FLUSI_MAX_CONTOUR 32
#define FLUSI_FORCE_COLS 26

/* Columns of one force row (Eqs. force_with_unst_corrections and
 * moment_of_love, one block per mask colour: 0 body, 1 left wing, 2 right;
 * the moment of the body about x_cntr, of a wing about its pivot), then the
 * power of each wing (Sec. 3.5, Eq. insect_power): aerodynamic
 * P = -M_wing . (Omega_wing - Omega_body), global frame, and inertial
 * P = Omega^(w) . (J Omega'^(w) + Omega^(w) x J Omega^(w)), wing frame. */
#define FLUSI_COL_T 0
#define FLUSI_COL_DT 1
#define FLUSI_COL_F(colour) (2 + 6 * (colour))
#define FLUSI_COL_M(colour) (5 + 6 * (colour))
#define FLUSI_COL_EKIN 20
#define FLUSI_COL_UMAX 21
#define FLUSI_COL_PAERO(wing) (22 + (wing))
#define FLUSI_COL_PINERT(wing) (24 + (wing))

typedef struct flusi_options {
    double cfl;            /* CFL number of the adaptive step (default 0.1)            */
    double dt_fixed;       /* > 0: fixed step; 0: adaptive (default 0)                  */
    double dt_max;         /* > 0: cap on the adaptive step (default 0 = none)          */
    double u_inf[3];       /* mean flow held at k = 0 when mean_mode = 0 (default 0)    */
    int mean_mode;         /* 0: k = 0 mode held at u_inf; 1: evolves freely            */
    int dealias_strict;    /* 0: keep |m| <= floor(n/3); 1: keep |m| < n/3              */
    int force_ring;        /* device rows kept between flusi_forces calls (default 4096)*/
    int use_graph;         /* 1: replay a captured CUDA graph per step (default 1)      */
    /* Wake removal (Sec. 2.3).  Vorticity sponge -(1/C_sp) curl (chi_sp omega)/nabla^2
     * with C_sp = sponge_c (0: off, the default) over the region where some
     * x_i >= L_i - sponge_width[i] (width 0: no slab on that axis).  Dirichlet
     * layer: u = u_inf penalized with C_eta where some x_i >= L_i - layer_width[i].
     * Both masks are 1 inside their slabs and 0 elsewhere.                      */
    double sponge_c;
    double sponge_width[3];
    double layer_width[3];
    /* Time scheme (Sec. 2.4): 0 = integrating-factor AB2 (default); 1 = RK4
     * with explicit diffusion, four right-hand sides per step at t, t + dt/2,
     * t + dt/2, t + dt, the mask moved to each, and the step further limited
     * to dt <= 2.5/(nu |k|^2_max).  RK4 needs one more state-sized buffer, so
     * it is fixed at flusi_bind.                                             */
    int time_scheme;
    /* 1 (default): the y and z passes receive their tiles by TMA boxes
     * (cp.async.bulk.tensor) where a box fits; 0: by 16-byte asynchronous
     * copies everywhere.  Both give identical results. */
    int use_tma;
} flusi_options;

/* Insect geometry and kinematics (Sec. 3).  Angles in radians.  Kinematic
 * angles are Fourier series a0/2 + sum_i a[i] cos(2 pi (i+1) f t)
 * + b[i] sin(2 pi (i+1) f t), i < nfourier. */
typedef struct flusi_insect {
    int body_type;             /* 0 none, 1 sphere (radius body_a), 2 ellipsoid thorax,
                                  3 thorax on a circular centre line (body_arc)        */
    int nwings;                /* 0, 1 (left wing only) or 2                            */
    int profile;               /* 0: cosine layer (Sec. 2.2); 1: 1/2 (1 - tanh(delta/h)) */
    int nfourier;              /* harmonics used, <= FLUSI_MAX_FOURIER                  */
    double c_smth;             /* layer half-width h = c_smth * max(dx, dy, dz)          */
    double x_cntr[3], u_cntr[3];           /* body centre and its velocity (global)    */
    double psi, beta, gamma;               /* roll, pitch, yaw (Eq. M_body_yawpitchroll) */
    double psi_dot, beta_dot, gamma_dot;   /* their rates (body angular velocity)       */
    double body_a, body_b;                 /* thorax semi-axes (x; y and z)             */
    double pivot_l[3], pivot_r[3];         /* wing pivots in the body frame             */
    double eta_stroke;                     /* anatomical stroke-plane angle             */
    double wing_c_le, wing_c_te, wing_R, wing_h; /* plate: chord extents, span, thickness */
    double freq;
    double phi_a0, phi_a[FLUSI_MAX_FOURIER], phi_b[FLUSI_MAX_FOURIER];
    double alpha_a0, alpha_a[FLUSI_MAX_FOURIER], alpha_b[FLUSI_MAX_FOURIER];
    double theta_a0, theta_a[FLUSI_MAX_FOURIER], theta_b[FLUSI_MAX_FOURIER];
    /* Head and eye spheres joined to an ellipsoid thorax (Sec. 3.2, Eq.
     * DELTA_body_jerry), body frame; radius 0: absent.  The right eye mirrors
     * the left one in y^(b).  The parts are joined by the minimum of their
     * signed distances (their union). */
    double head_x0[3], head_r;
    double eye_x0[3], eye_r;
    /* Wing outline (Sec. 3.4): wing_shape 0 = the rectangular plate above;
     * 1 = the contour R(theta) = a0/2 + sum_{i<=ncontour} a_i cos(i theta) +
     * b_i sin(i theta) (Eq. Fourier_radious_wing, theta in radians from x^(w)
     * towards y^(w)) about (contour_xc, contour_yc) in the wing plane, with
     * thickness wing_h.  R is evaluated exactly (no lookup table). */
    int wing_shape;
    int ncontour;              /* <= FLUSI_MAX_CONTOUR */
    double contour_xc, contour_yc;
    double contour_a0, contour_a[FLUSI_MAX_CONTOUR], contour_b[FLUSI_MAX_CONTOUR];
    /* Tensor of inertia of one wing in its own frame (xx, yy, zz, xy, xz, yz),
     * used only by the inertial power column (Sec. 3.5). */
    double J_wing[6];
    /* Free flight (Sec. 3.6, Eq. oh_my_god_look_a_vector).  0: the body moves
     * as x_cntr, u_cntr and the angles above prescribe (tethered).  1: x_cntr,
     * u_cntr, quat and Omega_body are the initial state of the 13 Newton-Euler
     * equations, which every step advances on the device with the fluid's AB2
     * weights (Euler on the first step), driven by the step's total force and
     * its moment about x_cntr (the wings' moments moved from their pivots);
     * the quaternion is renormalized after each step.  The orientation is
     * then the quaternion's (the angles and their rates are not used), the
     * printed quaternion matrix being the body-to-global map.  Free flight
     * needs time_scheme 0.  flusi_get_body reads the state back. */
    int free_flight;
    int pad2_;
    double mass, gravity;      /* M; g > 0 pulls along -z                         */
    double J_body[3];          /* principal moments of inertia (body axes), > 0   */
    double dof[6];             /* factors on du_x, du_y, du_z and dOmega_x, _y, _z:
                                  1 free, 0 held                                 */
    double quat[4];            /* epsilon_0..3; all zero: from (psi, beta, gamma)  */
    double Omega_body[3];      /* Omega^(b), body frame                           */
    /* body_type 3 (the fruit-fly body of Sec. 5.3): the thorax (body_a, body_b)
     * bent along an arc of the circle of radius body_arc[0] about
     * (body_arc[1], 0, body_arc[2]) in the x^(b)-z^(b) plane, with circular
     * cross-sections of radius body_b sqrt(1 - (s/body_a)^2) centred on the
     * arc, s the arc length from the arc point towards the body origin; beyond
     * |s| = body_a the distance is that to the arc's end point.  Needs
     * body_b < body_arc[0], body_a < pi body_arc[0], and the circle's centre
     * away from the body origin.  Head and eyes join it as for type 2. */
    double body_arc[3];
} flusi_insect;

/* Create a solver for an nx x ny x nz periodic grid over the box L[3], with
 * kinematic viscosity nu and penalization constant eta (C_eta of Eq.
 * PNST_org_momentum).  Each n_i must be 2^a 3^b with 8 <= n_i <= 1024 and nx
 * even.  precision is a flusi_precision.  Allocates only a small host struct;
 * device memory is bound later (flusi_bind).  Returns FLUSI_EINVAL for bad
 * sizes or a NULL `out`. */
int flusi_create(int nx, int ny, int nz, const double L[3], double nu, double eta,
                 int precision, flusi_t *out);

/* Fill *opt with the defaults listed in flusi_options. */
void flusi_default_options(flusi_options *opt);

/* Replace the options (Algorithm 1 step b time-step rule, mean mode, 2/3-rule
 * variant, force ring size, graph use).  Allowed before flusi_bind; after it,
 * only options that keep the workspace size.  Invalidates a captured graph. */
int flusi_set_options(flusi_t h, const flusi_options *opt);

/* Bytes of device workspace the handle needs with its current options. */
int flusi_workspace_bytes(flusi_t h, size_t *bytes);

/* Bind a caller-owned device workspace (>= flusi_workspace_bytes, 256-byte
 * aligned, outliving the handle) and a CUDA stream (cudaStream_t; NULL is the
 * legacy default stream).  All later work is enqueued on that stream: a step
 * runs its two single-block kernels on a private stream that forks from it
 * and joins back into it within the step, so work ordered on the bound stream
 * before and after a step sees the whole step.  Zeroes the workspace and
 * builds the FFT twiddle tables.  FLUSI_ENOMEM if too small. */
int flusi_bind(flusi_t h, void *dev_workspace, size_t bytes, void *cuda_stream);

/* Set the velocity u [3][nz][ny][nx] (Algorithm 1 step 1, initial condition):
 * where = FLUSI_HOST_FP64 / FLUSI_HOST_FP32 (host array) or FLUSI_DEVICE (a
 * device array in the handle's precision).  The field is transformed,
 * truncated by the 2/3 rule and projected onto divergence-free fields; with
 * mean_mode 0 its mean is replaced by u_inf.  Resets t = 0, the step count,
 * the AB2 history, the force rows and the device status word. */
int flusi_set_state(flusi_t h, const void *u, int where);

/* Set the insect (Sec. 3): body, wings, kinematics.  Without a call (or with
 * NULL) there is no mask.  May be called between steps; with free flight it
 * replaces the body's state (the ODE's AB2 history is kept).  FLUSI_EINVAL
 * for a bad descriptor, or free flight with time_scheme 1.  On a bound
 * handle the descriptor is copied into one of 8 page-locked slots of the
 * handle and uploaded in stream order without waiting for the enqueued
 * steps; the call waits only when the slot it reuses still has its copy
 * pending (the host is 8 calls ahead of the GPU). */
int flusi_set_kinematics(flusi_t h, const flusi_insect *insect);

/* Free flight (Sec. 3.6): the body state after the steps enqueued so far,
 * state[13] = x_cntr[3], u_cntr[3], quat[4], Omega_body[3] (host).  Without
 * free flight it is the descriptor's (constant) values.  Synchronizes;
 * FLUSI_ESTATE without an insect or when not bound. */
int flusi_get_body(flusi_t h, double state[13]);

/* Enqueue n time steps (Algorithm 1 steps a-e) on the bound stream and
 * return without waiting.  Only argument and call-order errors are reported
 * here; device errors surface at the next synchronizing call. */
int flusi_step(flusi_t h, int n);

/* Wait for the enqueued work and check the device status word. */
int flusi_sync(flusi_t h);

/* Drain the force rows produced since the last call (in step order) into
 * rows[count][FLUSI_FORCE_COLS] (host, capacity `cap` rows).  Row columns:
 * t, dt, then per colour F[3], M[3], then E_kin = 1/2 sum |u|^2 dV and
 * max |u|, then the aerodynamic and the inertial power of each wing.  Synchronizes.  Rows beyond force_ring since the last call are
 * lost; *lost (may be NULL) receives their number. */
int flusi_forces(flusi_t h, double *rows, int cap, int *count, long long *lost);

/* The same drain without waiting: enqueues on the bound stream the copy of the
 * rows of every step enqueued since the last drain (at most `cap`, the oldest
 * first; rows beyond force_ring are lost as above) into rows[count][...] and
 * returns.  The rows are there once the stream has run the copy (after the
 * next synchronizing call, or an event or synchronization of the stream).
 * `rows` should be page-locked host memory (cudaHostAlloc, or a pinned
 * torch tensor): from pageable memory the copy, and so the call, waits for
 * the enqueued steps.  A step that failed on the device writes no row; the
 * failure surfaces at the next synchronizing call, and the rows counted
 * for the steps after it are undefined. */
int flusi_forces_async(flusi_t h, double *rows, int cap, int *count, long long *lost);

/* Copy the velocity u [3][nz][ny][nx] to host FP64 (where = FLUSI_HOST_FP64),
 * host FP32, or a caller device array in the handle's precision, with the
 * time t and step count (either may be NULL).  Synchronizes. */
int flusi_get_state(flusi_t h, void *u_out, int where, double *t, long long *step);

/* Divergence of the current state (Eq. PNST_UP_pressure_poisson_eqn: the
 * Leray projection keeps k . u_hat = 0): *div_max = max over the kept modes of
 * |k . u_hat| and, when ku_max is not NULL, *ku_max = max of |k| |u_hat| (its
 * scale; the ratio is the relative divergence, round-off after a step).  Both
 * reduced in FP64 on the device from the state in the handle's precision.
 * Waits for the enqueued steps; a non-finite state gives a NaN maximum. */
int flusi_divergence(flusi_t h, double *div_max, double *ku_max);

/* Copy u_hat to host FP64 complex, half-spectrum layout [3][nz][ny][nx/2+1]
 * (interleaved re, im), zero outside the 2/3-rule set.  Synchronizes. */
int flusi_get_spectrum(flusi_t h, double *uh_out);

/* Diagnostic: evaluate the physical-space fields of the current state at the
 * current time into the caller's device array out [14][nz][ny][nx] in the
 * handle's precision: u[3], omega[3], chi, colour, u_s[3], and the term
 * u x omega - chi/C_eta (u - u_s) [3] (Sec. 2.1, Algorithm 1 step c).
 * Enqueued on the bound stream. */
int flusi_debug_fields(flusi_t h, void *out_dev);

/* Diagnostic: time each kernel of one step with CUDA events on the bound
 * stream over n un-captured steps (which advance the state).  ms[i] gets the
 * mean duration of kernel i, names[i] its name (RK4 stages 2..4 carry a ".2",
 * ".3", ".4" suffix); *nk the number of kernels (at most FLUSI_PROFILE_MAX;
 * ms and names must hold that many).  Synchronizes. */
#define FLUSI_PROFILE_MAX 40
int flusi_profile_step(flusi_t h, int n, double *ms, const char **names, int *nk);

/* Diagnostic of the device-side failure path (no passage of the paper): one
 * block waits, bounded by about `milliseconds` of SM clock, on an mbarrier
 * that nothing completes -- the same bounded wait the tile loads of the y and
 * z passes use -- and, when it gives up, sets FLUSI_ETIMEOUT in the device
 * status word exactly as they do.  The next synchronizing call reports it
 * and the handle answers FLUSI_ESTATE until flusi_set_state; the context
 * stays usable.  0 < milliseconds <= 1000, else FLUSI_EINVAL. */
int flusi_debug_wait_timeout(flusi_t h, double milliseconds);

/* Host-side fault injection for testing the failure path (no passage of the
 * paper; nothing on the device is made to fault): write re + i im into the
 * state's Fourier coefficient of mode (mx, my, mz) of velocity component
 * `component` (0..2), after the steps already enqueued.  mx in 0..Kx, my in
 * -Ky..Ky, mz in -Kz..Kz (the kept modes, K = floor(n/3)), else FLUSI_EINVAL;
 * FLUSI_ESTATE without a state.  A non-finite value makes the next step set
 * FLUSI_ENONFINITE in the device status word (reported by the next
 * synchronizing call; steps are refused until flusi_set_state).  No
 * projection is applied to the written value.  Synchronizes. */
int flusi_debug_inject(flusi_t h, int component, int mx, int my, int mz, double re, double im);

/* Kernels launched per step (for launch accounting). */
int flusi_kernels_per_step(flusi_t h, int *count);

/* ---- FFT plans and tile shapes, and their autotuner.  The paper takes its
 * 1-D transforms from a library (Sec. 4, P3DFFT over FFTW); here each axis
 * pass is the project's own kernel, and how a length is factored into radix
 * stages and how many columns a y or z tile holds are choices whose best
 * value depends on the grid and the GPU.  Every setting computes the same
 * transforms; results differ only by rounding.
 *
 * Plans (y_plan, zf_plan): 0 radix 8 first, then one 4 or 2 (and 3 for each
 * factor 3; 16 = 4 4); 1 (default) as 0, but 2^(3q+1) takes one radix-16
 * stage in place of 4 4 or 8 2 (1024 = 16 8 8, 128 = 16 8, 16 = 16);
 * 2 fewest stages: as 1, and 2^(3q+2) with q >= 2 takes 16 16 in place of
 * 8 8 4 (256 = 16 16).  The inverse z pass always takes plan 0 (its kernel
 * has no radix-16 variant).
 * Tile columns (y_cols, z_cols): 0 (default) the widest tile that fits a
 * block's 64 KB, else a cap on the tile's columns (x columns times z planes
 * for y; columns of the flattened (y, x) plane for z), a power of two of at
 * least 32 bytes of complex values (4 in FP32, 2 in FP64) and at most 256.
 * x_kernel: 0 (default) the register-resident line kernel where one exists
 * (nx = 128, 256, 512, 1024, and its rectangular form at nx = 64, 96), 1 the
 * shared-memory kernel of every length.
 * y_pair: 1 the y passes' paired kernel, a cluster of two CTAs per tile,
 * each holding the grid rows of one parity and transforming them at half the
 * length, joined by a radix-2 step through distributed shared memory, so
 * that tiles keep 128-byte rows at twice the length (ny even); 0 (default)
 * one CTA per tile.  With it, y_cols caps the paired tile.
 *
 * flusi_get_tuning fills every field, including the read-only ones: the
 * radices each pass takes (0-terminated), the columns a tile takes, and
 * whether the x pass runs the register-resident kernel.
 * flusi_set_tuning takes the six settings (the rest is ignored); any
 * other value is FLUSI_EINVAL with nothing changed.  On a bound handle it
 * waits for the handle's stream, uploads the new digit-reversal tables and
 * rebuilds the TMA descriptors; the state is kept.  No device work on an
 * unbound handle.
 *
 * flusi_autotune: on a bound handle with a state, coordinate descent over
 * the settings (y_plan, y_pair, y_cols, zf_plan, z_cols, x_kernel, in that order):
 * each candidate runs one untimed step and `steps` (1..1000) timed steps,
 * and is scored by the CUDA-event time of the kernels it changes
 * (flusi_profile_step's per-kernel times); the best is kept.  The state,
 * time, step count and free-flight body state are saved before and restored
 * after, as by flusi_save/flusi_load, so the run continues where it was;
 * undrained force rows are dropped, as by flusi_load.  cache_path (NULL: no
 * cache) names a text file of lines "key y_plan zf_plan y_cols z_cols
 * x_kernel y_pair", key = GPU name (spaces as '_'), SM count, grid, precision,
 * time scheme and wake terms: a line with this handle's key is applied
 * without timing; otherwise the result is appended (a file that cannot be
 * written is FLUSI_EINVAL after the tuning is applied).  *out (may be
 * NULL) receives the chosen settings as flusi_get_tuning does.  The saved
 * state is held in host memory the call allocates and frees (two state-sized
 * spectra; FLUSI_ENOMEM when it cannot); a failing candidate step restores
 * the state and returns its error.  FLUSI_ESTATE without a bound workspace or
 * a state, or on a poisoned handle.  Synchronizes. */
#define FLUSI_MAX_STAGES 8
typedef struct flusi_tuning {
    int y_plan, zf_plan;       /* 0, 1 (default) or 2                      */
    int y_cols, z_cols;        /* 0 (default) or a power of two cap        */
    int x_kernel;              /* 0 (default) or 1                         */
    int y_pair;                /* 0 (default) or 1                         */
    /* read-only, filled by flusi_get_tuning (y_radix: the paired kernel's
     * half-length plan when y_paired is 1) */
    int y_radix[FLUSI_MAX_STAGES], zf_radix[FLUSI_MAX_STAGES], zi_radix[FLUSI_MAX_STAGES];
    int y_tile_cols, z_tile_cols, x_line_kernel, y_paired;
} flusi_tuning;
int flusi_get_tuning(flusi_t h, flusi_tuning *out);
int flusi_set_tuning(flusi_t h, const flusi_tuning *tuning);
int flusi_autotune(flusi_t h, int steps, const char *cache_path, flusi_tuning *out);

/* Largest grid (points) and output length of flusi_penalization_sums_noalloc. */
#define FLUSI_NOALLOC_MAX_POINTS (1024LL * 1024LL * 1024LL)
#define FLUSI_NOALLOC_SUMS 38

/* Force, moment, energy and CFL sums of a velocity field, without allocating.
 * The paper has no counterpart: this is a library convenience for callers
 * that cannot allocate device memory -- their device memory belongs to
 * another allocator's pool, or they cannot accept a cudaMalloc/cudaFree and
 * its implicit device synchronization where they run.  It needs no handle
 * and no workspace.
 *
 * Inputs: grid nx, ny, nz (at most FLUSI_NOALLOC_MAX_POINTS points, else
 * FLUSI_EINVAL with a message in flusi_last_error(NULL)), box L[3], penalization
 * constant eta (C_eta), the insect (NULL: no mask) evaluated at time t, and
 * u_dev, a caller-owned device array [3][nz][ny][nx] of FP64 velocity.
 * Output: sums_out, a caller-owned host array of FLUSI_NOALLOC_SUMS doubles:
 * per colour (body, left wing, right wing) sum chi (u - u_s) dV / C_eta [3],
 * sum r x chi (u - u_s) dV / C_eta [3], sum chi u_s dV [3],
 * sum r x chi u_s dV [3] (r from the body centre or the wing pivot), then
 * 1/2 sum |u|^2 dV and max |u|.  These are the quantities the step reduces
 * into its force rows; a step's row adds the unsteady correction (the change
 * of sum chi u_s dV over the previous step) to them.
 *
 * Scratch: a fixed array of about 332 KB in the library's own device memory
 * (every GPU that loads the library holds it until the process exits).  The
 * first call on a device looks up that array's device address, and looks it
 * up again whenever the device's current CUDA context has changed since (after
 * cudaDeviceReset the library's device memory is reloaded and can move); make
 * that first call, and the first after a reset, before any stream capture.
 * Every call shares the array and
 * leaves its contents behind, so calls that overlap on the GPU (two streams,
 * two host threads) race and corrupt each other's results.  The work is
 * enqueued on cuda_stream (NULL: legacy default stream) and the call waits for
 * it.  Returns FLUSI_ENONFINITE when u holds a non-finite value. */
int flusi_penalization_sums_noalloc(int nx, int ny, int nz, const double L[3], double eta,
                                    const flusi_insect *insect, double t, const double *u_dev,
                                    double *sums_out, void *cuda_stream);

/* ---- Checkpoint and exact restart.  The paper writes flow fields to disk but
 * describes no restart; an AB2 step depends on u_hat, the history N_hat^{n-1},
 * t, dt_{n-1}, the step count and the previous solid integrals of the
 * unsteady force correction (Eq. force_with_unst_corrections), and a
 * checkpoint holds exactly those, in the handle's precision and internal
 * layout (kept modes only), so a run restarted from it continues bit for bit.
 * In free flight it also holds the body state and the ODE's previous
 * right-hand side; loading writes the body state into the current insect when
 * that is in free flight.  Options and kinematics are not stored otherwise:
 * set them as they were, before flusi_load.
 *
 * flusi_checkpoint_bytes: size of a checkpoint of this handle (no device work).
 * flusi_save: write one into the caller's host buffer of `bytes` (at least that
 *   size, else FLUSI_EINVAL); FLUSI_ESTATE without a state or on a poisoned
 *   handle.  Synchronizes.
 * flusi_load: restore one into a bound handle of the same grid, box, nu, eta,
 *   precision and 2/3 rule (else FLUSI_EINVAL, checked before anything else);
 *   replaces the state as flusi_set_state does.  Force rows from before the
 *   save are not restored; the next drained row is the next step's.
 *   Synchronizes. */
int flusi_checkpoint_bytes(flusi_t h, size_t *bytes);
int flusi_save(flusi_t h, void *host_buf, size_t bytes);
int flusi_load(flusi_t h, const void *host_buf, size_t bytes);

/* ---- Ensembles of independent runs (uneven grids, kinematics, Reynolds
 * numbers).  The paper runs one simulation at a time; this batches many small
 * ones into one CUDA graph per ensemble step so that their kernels fill the
 * GPU together.
 *
 * flusi_ensemble_create: `members` are `count` (1..FLUSI_ENSEMBLE_MAX) bound
 * handles with a state, each with its own workspace; the array is copied and
 * the handles stay owned by the caller (they must outlive the ensemble and
 * must not be destroyed or re-bound while it exists).  `cuda_stream` is the
 * stream the ensemble's steps are enqueued on (NULL: legacy default stream).
 * FLUSI_EINVAL for a NULL or repeated member, FLUSI_ESTATE for one that is not
 * bound or has no state.  Ensemble calls leave their failure message in
 * flusi_last_error(NULL).
 *
 * flusi_ensemble_step: enqueue n steps of every member (Algorithm 1 steps
 * a-e, each member with its own adaptive dt) and return without waiting.  The
 * first call captures one graph holding one step of all members, forked from
 * and joined back into the ensemble stream; later calls launch it n times.
 * Members with the same grid, box, C_eta, precision, options, tuning and mask
 * shape, stepped with AB2, without the vorticity sponge, on the CUDA-core x
 * pass (nu and the kinematics may differ) share their launches: one launch
 * per kernel covers the whole group, each member's blocks reading its own
 * buffers; the others step with launches of their own.  Every member's
 * arithmetic is the same either way (its results equal a solo run's bit for
 * bit).
 * Work already enqueued on a member's bound stream runs before, and work
 * enqueued there afterwards runs after, so flusi_forces / flusi_get_state on a
 * member see the ensemble's steps.  A member with a device error stops
 * stepping (its kernels return at entry) and reports it at its next
 * synchronizing call; the others are unaffected.  Options and kinematics of
 * the members are those at the first call; changing a member's options, its
 * tuning (flusi_set_tuning, flusi_autotune) or the shape of its insect
 * afterwards needs a new ensemble (FLUSI_ESTATE).
 *
 * flusi_ensemble_destroy: release the ensemble (not the members).  NULL is a
 * no-op. */
#define FLUSI_ENSEMBLE_MAX 1024
typedef struct flusi_ensemble_s *flusi_ensemble_t;
int flusi_ensemble_create(const flusi_t *members, int count, void *cuda_stream,
                          flusi_ensemble_t *out);
int flusi_ensemble_step(flusi_ensemble_t e, int n);
int flusi_ensemble_destroy(flusi_ensemble_t e);
/* After the first flusi_ensemble_step: the number of groups whose members
 * share launches, and how many members they hold (both 0 before). */
int flusi_ensemble_batches(flusi_ensemble_t e, int *groups, int *members);

/* Release the handle (not the caller's workspace).  NULL is a no-op. */
int flusi_destroy(flusi_t h);

/* Message of the last failed call on h; with h NULL, of the calling thread's
 * last failed call that had no handle (flusi_create, the allocation-free
 * entry point).  Valid until the next failing call of the same kind. */
const char *flusi_last_error(flusi_t h);

/* Measured arithmetic peak of the current device: the rate of independent
 * dependent chains of fused multiply-adds in FP32 (fp64 = 0) or FP64
 * (fp64 = 1), every SM full, in flop/s (2 per FMA) into *flops_per_s, the
 * timed kernel's duration in ms into *ms (may be NULL).  The chain length is
 * calibrated so that one launch takes about target_ms (0 < target_ms <= 1e4);
 * the best of three launches counts.  A measuring aid with no counterpart in
 * the paper: the arithmetic rooflines of the x pass and of the FP64 path are
 * quoted against it.  Changes no clock or power setting; synchronizes. */
int flusi_fma_peak(int fp64, double target_ms, double *flops_per_s, double *ms);

/* Identity of the build: a digest of the library's sources, headers and
 * compiler flags (the build script's source hash), or "unstamped" for a build
 * made without it.  Lets a caller refuse a library built from other sources. */
const char *flusi_build_id(void);

#ifdef __cplusplus
}
#endif
#endif

// C-ABI of libflusi (include/flusi.h): handle, workspace layout, FFT plans
// and twiddle tables, the kernel sequence of one step (Algorithm 1 steps
// a-e) and its capture into a CUDA graph, and the host<->device marshalling
// of states and force rows.  Host code only; all arithmetic of the step runs
// in the kernels.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <initializer_list>
#include <memory>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/flusi.h"
#include "kernels.cuh"

using namespace flusi;

// the ensemble batch of the launches this host thread makes (see Batch)
Batch& flusi::current_batch()
{
    static thread_local Batch b;
    return b;
}

constexpr int kStageSlots = 8;   // pinned insect-descriptor slots per handle

struct flusi_s {
    int nx = 0, ny = 0, nz = 0, prec = 0;
    double L[3] = {0, 0, 0}, nu = 0, eta = 0;
    flusi_options opt{};
    flusi_tuning tune{};           // plans, tile caps and x kernel (flusi_set_tuning)
    flusi_insect ins{};
    int have_ins = 0;
    Geom g{};
    FftPlan px{}, py{}, pz{}, pzi{};   // pzi: the inverse z pass's plan (no radix-16 stage)
    FftPlan pyh{};                 // half the y length, for the paired y kernel (ny even)
    YMaps ymaps{};                 // TMA descriptors of W for the y passes (built at bind)
    ZMaps zmaps{};                 // TMA descriptors of U, the RK4 stage state and W for the z passes
    // workspace
    char* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    int bound = 0;
    size_t oU = 0, oH = 0, oUt = 0, oW = 0, otx = 0, oty = 0, otz = 0, opx = 0, opy = 0, opz = 0, opzi = 0, opyh = 0,
           oframe = 0, oins = 0, ostate = 0, ocoef = 0, oetab = 0, opart = 0, orows = 0, total = 0;
    int part_cap = 0, xgrid = 0;
    // run state
    int has_state = 0, poisoned = 0;
    long long rows_read = 0;
    long long n_enq = 0;          // the device step count once the enqueued steps complete
    // page-locked staging slots of the insect descriptor: its upload is
    // asynchronous; a slot is reused once the copy out of it has run
    flusi_insect* ins_stage = nullptr;
    cudaEvent_t stage_ev[8] = {};
    int stage_next = 0;
    cudaStream_t cap_stream = nullptr;
    // side branch of the step: the kinematics run beside the inverse z and y
    // passes, the scalar kernel beside the forward y pass
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_kin = nullptr, ev_x = nullptr, ev_sc = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_ok = 0;
    long long generation = 0;   // bumped whenever captured step graphs go stale
    std::string err;
};

namespace {

// errors without a handle (creation, the allocation-free entry point), per
// calling thread
thread_local std::string g_create_err;

}  // namespace

void flusi::set_global_error(const char* msg) { g_create_err = msg; }

namespace {

int fail(flusi_t h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    else g_create_err = msg;
    return code;
}

int cuda_fail(flusi_t h, cudaError_t e, const char* what)
{
    return fail(h, FLUSI_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

bool smooth_size(int n)
{
    if (n < 8 || n > kMaxN) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

// Radix order: 3s first (their stages divide), then 8s, then a 4 or 4*4 or 2.
// `tws` is the stride of the twiddle table the transform reads (its table has
// n*tws entries), folded into the per-stage twiddle steps.
// Radix stages of a length n = 2^a 3^b: the factors 3 first, then (a = 3q + r)
// mode 0: 8^q and one 4 (r = 2) or 2 (r = 1), except that 2^(3q+1) with
//   q >= 1 ends in 4 4 (16 = 4 4, 128 = 8 4 4, 1024 = 8 8 4 4);
// mode 1: as 0, but 2^(3q+1) with q >= 1 takes one radix-16 stage in place of
//   that 4 4 (16, 16 8, 16 8 8): one pass through shared memory fewer;
// mode 2: as 1, and 2^(3q+2) with q >= 2 takes 16 16 in place of 8 8 4
//   (256 = 16 16).
// Modes 1 and 2 are for the y and forward z passes, whose kernels have
// radix-16 variants.
FftPlan make_plan(int n, int tws, int mode = 0)
{
    FftPlan p{};
    p.n = n;
    std::vector<int> r;
    int m = n;
    while (m % 3 == 0) { r.push_back(3); m /= 3; }
    int a = 0;
    while (m % 2 == 0) { ++a; m /= 2; }
    int q = a / 3, rem = a % 3, n16 = 0;
    if (rem == 1 && q >= 1) {
        q -= 1;
        if (mode >= 1) { n16 = 1; rem = 0; } else rem = 4;
    } else if (rem == 2 && q >= 2 && mode == 2) {
        q -= 2;
        n16 = 2;
        rem = 0;
    }
    for (int i = 0; i < n16; ++i) r.push_back(16);
    for (int i = 0; i < q; ++i) r.push_back(8);
    if (rem == 2) r.push_back(4);
    if (rem == 1) r.push_back(2);
    if (rem == 4) { r.push_back(4); r.push_back(4); }
    p.nst = (int)r.size();
    int Ls = n;
    for (int s = 0; s < p.nst; ++s) {
        p.radix[s] = r[s];
        p.ls[s] = Ls;
        p.m[s] = Ls / r[s];
        p.mshift[s] = (p.m[s] & (p.m[s] - 1)) == 0 ? __builtin_ctz(p.m[s]) : -1;
        p.tstep[s] = (n / Ls) * tws;
        Ls = p.m[s];
    }
    return p;
}

// Row of frequency f after the in-place decimation-in-frequency transform:
// f = d_0 + r_0 (d_1 + r_1 (...))  ->  sum_s d_s m_s.
std::vector<int> digit_reversal(const FftPlan& p)
{
    std::vector<int> pos(p.n);
    for (int f = 0; f < p.n; ++f) {
        int ff = f, at = 0;
        for (int s = 0; s < p.nst; ++s) {
            at += (ff % p.radix[s]) * p.m[s];
            ff /= p.radix[s];
        }
        pos[f] = at;
    }
    return pos;
}

// exp(-2 pi i j / n), j < n, from long double sines and cosines.
std::vector<double2> twiddles(int n)
{
    std::vector<double2> t(n);
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int j = 0; j < n; ++j) {
        long double a = two_pi * (long double)j / (long double)n;
        t[j].x = (double)cosl(a);
        t[j].y = -(double)sinl(a);
    }
    return t;
}

// the table rounded to FP32 (stored after the FP64 one: the FP32 kernels read it)
std::vector<float2> twiddles32(const std::vector<double2>& t)
{
    std::vector<float2> f(t.size());
    for (size_t j = 0; j < t.size(); ++j) f[j] = make_float2((float)t[j].x, (float)t[j].y);
    return f;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int cutoff(int n, int strict) { return (strict && n % 3 == 0) ? n / 3 - 1 : n / 3; }

void layout(flusi_t h)
{
    Geom& g = h->g;
    const int strict = h->opt.dealias_strict;
    g.nx = h->nx;
    g.ny = h->ny;
    g.nz = h->nz;
    g.Kx = cutoff(h->nx, strict);
    g.Ky = cutoff(h->ny, strict);
    g.Kz = cutoff(h->nz, strict);
    g.Mx = g.Kx + 1;
    g.My = 2 * g.Ky + 1;
    g.Mz = 2 * g.Kz + 1;
    g.Mxp = (g.Mx + 3) / 4 * 4;
    g.Lx = h->L[0];
    g.Ly = h->L[1];
    g.Lz = h->L[2];
    g.dx = h->L[0] / h->nx;
    g.dy = h->L[1] / h->ny;
    g.dz = h->L[2] / h->nz;
    g.nu = h->nu;
    g.eta = h->eta;

    const size_t cs = h->prec == FLUSI_FP64 ? 16 : 8;
    const size_t spec = (size_t)3 * g.Mz * g.My * g.Mxp * cs;
    const size_t work = (size_t)6 * g.nz * g.ny * g.Mxp * cs;
    const int rb_min = 1;
    h->part_cap = std::min(8192, (g.nz * g.ny + rb_min - 1) / rb_min);
    size_t o = 0;
    h->oU = o; o = align256(o + spec);
    h->oH = o; o = align256(o + spec);
    h->oUt = o; o = align256(o + (h->opt.time_scheme == 1 ? spec : 0));   // RK4 stage state
    h->oW = o; o = align256(o + work);
    // twiddle tables: n values in FP64, then the same rounded to FP32
    h->otx = o; o = align256(o + (sizeof(double2) + sizeof(float2)) * g.nx);
    h->oty = o; o = align256(o + (sizeof(double2) + sizeof(float2)) * g.ny);
    h->otz = o; o = align256(o + (sizeof(double2) + sizeof(float2)) * g.nz);
    h->opx = o; o = align256(o + sizeof(int) * (g.nx / 2));
    h->opy = o; o = align256(o + sizeof(int) * g.ny);
    h->opz = o; o = align256(o + sizeof(int) * g.nz);
    h->opzi = o; o = align256(o + sizeof(int) * g.nz);
    h->opyh = o; o = align256(o + sizeof(int) * (g.ny / 2));
    h->oframe = o; o = align256(o + kFrameSlot);
    h->oins = o; o = align256(o + sizeof(flusi_insect));
    h->ostate = o; o = align256(o + sizeof(StepState));
    h->ocoef = o; o = align256(o + sizeof(StepCoef));
    h->oetab = o; o = align256(o + (sizeof(double) + sizeof(float)) * 2 * (g.Mx + g.My + g.Mz));
    h->opart = o; o = align256(o + sizeof(double) * kNumSums * h->part_cap);
    h->orows = o; o = align256(o + sizeof(double) * kRowCols * h->opt.force_ring);
    h->total = o;
    h->px = make_plan(h->nx / 2, 2);
    h->py = make_plan(h->ny, 1, h->tune.y_plan);
    h->pz = make_plan(h->nz, 1, h->tune.zf_plan);
    // the inverse z pass holds more live values per thread (the curl's side
    // rows); a radix-16 stage there costs it a block per SM, more than it saves
    h->pzi = make_plan(h->nz, 1, 0);
    h->pyh = h->ny % 2 == 0 ? make_plan(h->ny / 2, 1, h->tune.y_plan) : FftPlan{};
    g.ycols = h->tune.y_cols;
    g.ypair = h->tune.y_pair;
    g.zcols = h->tune.z_cols;
    g.xgeneric = h->tune.x_kernel;
    g.xtc = h->prec == FLUSI_FP32_SPLITBF16 ? 2 : h->prec == FLUSI_FP32_SPLITBF16X3 ? 3 : 0;
}

template <typename P> P* at(flusi_t h, size_t off) { return reinterpret_cast<P*>(h->ws + off); }

Shape make_shape(flusi_t h)
{
    if (!h->have_ins) return Shape{};
    const double d = std::max(h->g.dx, std::max(h->g.dy, h->g.dz));
    return shape_of(h->ins, h->ins.c_smth * d);
}

// Half-width used to grow the bounding boxes: the cosine layer vanishes
// beyond h; the tanh layer never does, so its boxes cover everything.
double box_margin(flusi_t h)
{
    Shape s = make_shape(h);
    return s.profile == 1 ? 1e300 : s.h;
}

// Names of the kernels of a step, in launch order; RK4 stages 2..4 repeat the
// right-hand-side kernels with a stage suffix.
const char* kStageNames[4][8] = {
    {"kinematics", "zinv_curl", "yinv", "xpass_phys", "sponge_x", "yfwd", "zfwd", "update"},
    {"kinematics.2", "zinv_curl.2", "yinv.2", "xpass_phys.2", "sponge_x.2", "yfwd.2", "zfwd.2", "update.2"},
    {"kinematics.3", "zinv_curl.3", "yinv.3", "xpass_phys.3", "sponge_x.3", "yfwd.3", "zfwd.3", "update.3"},
    {"kinematics.4", "zinv_curl.4", "yinv.4", "xpass_phys.4", "sponge_x.4", "yfwd.4", "zfwd.4", "update.4"}};
// the physical x pass on the tensor cores (split-BF16 precisions)
const char* kTcNames[4] = {"xpass_tc", "xpass_tc.2", "xpass_tc.3", "xpass_tc.4"};
constexpr int kMaxStepKernels = 4 * 8 + 1;

bool has_sponge(flusi_t h) { return h->opt.sponge_c > 0; }

bool is_rk4(flusi_t h) { return h->opt.time_scheme == 1; }

// device status word of the handle (where a device-side wait that gives up reports)
int* status_word(flusi_t h) { return &reinterpret_cast<StepState*>(h->ws + h->ostate)->status; }

// The square x pass forms chi_sp omega itself; other grids take a separate
// x round trip of the vorticity.
bool sponge_kernel(flusi_t h) { return has_sponge(h) && !xpass_fuses_sponge(h->prec == FLUSI_FP64, h->g); }

// Kernels per step: per right-hand side kinematics, z inverse, y inverse, x
// pass, (sponge x pass), y forward, z forward, update; the scalar kernel once.
int step_kernels(flusi_t h) { return (is_rk4(h) ? 4 : 1) * (7 + (sponge_kernel(h) ? 1 : 0)) + 1; }

// Explicit-diffusion cap of the RK4 step: 2.5 / (nu |k|^2_max) over the kept modes.
double rk4_dt_diff(flusi_t h)
{
    if (!is_rk4(h) || !(h->nu > 0)) return 0.0;
    const double two_pi = 6.283185307179586476925286766559;
    const int K[3] = {h->g.Kx, h->g.Ky, h->g.Kz};
    double k2 = 0;
    for (int i = 0; i < 3; ++i) {
        const double k = two_pi * K[i] / h->L[i];
        k2 += k * k;
    }
    return 2.5 / (h->nu * k2);
}

ZfwdExtra zextra(flusi_t h)
{
    ZfwdExtra ze{};
    ze.coef = at<StepCoef>(h, h->ocoef);
    ze.etab = at<double>(h, h->oetab);
    for (int i = 0; i < 3; ++i) ze.u_inf[i] = h->opt.u_inf[i];
    ze.mean_free = h->opt.mean_mode;
    ze.sponge_c = h->opt.sponge_c;
    return ze;
}

// First grid index of the end slab x_i >= L_i - w (i * L_i/n_i compared in
// FP64 as the oracle does); n when w = 0.
int slab_start(int n, double L, double w)
{
    if (!(w > 0)) return n;
    const double d = L / n;
    for (int i = 0; i < n; ++i)
        if (i * d >= L - w) return i;
    return n;
}

// Wake-removal fields of an x-pass descriptor (Sec. 2.3).
void set_wake(flusi_t h, XExtra& xe)
{
    const int n[3] = {h->nx, h->ny, h->nz};
    for (int i = 0; i < 3; ++i) {
        xe.layer0[i] = slab_start(n[i], h->L[i], h->opt.layer_width[i]);
        xe.sponge0[i] = slab_start(n[i], h->L[i], h->opt.sponge_width[i]);
        xe.u_inf[i] = h->opt.u_inf[i];
    }
}

// Enqueue one step.  With `ev` (step_kernels + 1 events) it records an event
// before each kernel and after the last, and names[i] the kernel after event i.
cudaError_t enqueue_step(flusi_t h, cudaStream_t s, cudaEvent_t* ev, const char** names = nullptr)
{
    const Geom& g = h->g;
    const int fp64 = h->prec == FLUSI_FP64;
    StepState* st = at<StepState>(h, h->ostate);
    StepCoef* coef = at<StepCoef>(h, h->ocoef);
    void* W = h->ws + h->oW;
    const double2* tx = at<double2>(h, h->otx);
    const double2* ty = at<double2>(h, h->oty);
    const double2* tz = at<double2>(h, h->otz);
    cudaError_t e;
    int k = 0;
    auto mark = [&](const char* next) {
        if (ev) cudaEventRecord(ev[k], s);
        if (names) names[k] = next;
        ++k;
    };
    // Without per-kernel events the two single-block kernels of the first
    // right-hand side run on the side stream: the kinematics only have to
    // finish before the x pass, the scalars (dt, coefficients, force row) only
    // before the update.
    const bool branch = ev == nullptr;
    cudaStream_t sk = branch ? h->side : s;
    const int nfwd = has_sponge(h) ? 6 : 3;
    const int stages = is_rk4(h) ? 4 : 1;
    const double frac[4] = {0.0, 0.5, 0.5, 1.0};
    for (int q = 0; q < stages; ++q) {
        const char* const* nm = kStageNames[q];
        // the right-hand side at the stage state: u^n first, then the RK4 stage buffer
        void* ustage = q == 0 ? h->ws + h->oU : h->ws + h->oUt;
        cudaStream_t skq = q == 0 ? sk : s;
        const bool br = branch && q == 0;
        mark(nm[0]);
        if (br) {
            if ((e = cudaEventRecord(h->ev_fork, s))) return e;
            if ((e = cudaStreamWaitEvent(sk, h->ev_fork, 0))) return e;
        }
        k_kinematics<<<dim3(1, 1, current_batch().n), 32, 0, skq>>>(
            at<flusi_insect>(h, h->oins), st, coef, at<Frame>(h, h->oframe), box_margin(h), frac[q],
            current_batch().mb, make_shape(h), 1, 1.0 / g.eta);
        if ((e = cudaGetLastError())) return e;
        if (br && (e = cudaEventRecord(h->ev_kin, sk))) return e;
        mark(nm[1]);
        const CUtensorMap* umap = q == 0 ? &h->zmaps.u : &h->zmaps.ut;
        const int ubh = q == 0 ? h->zmaps.u_bh : h->zmaps.ut_bh;
        if ((e = launch_zinv(fp64, ustage, W, g, h->pzi, tz, at<int>(h, h->opzi), 6, st, umap, ubh, &st->status, s)))
            return e;
        mark(nm[2]);
        if ((e = launch_ypass(fp64, true, W, g, h->py, ty, at<int>(h, h->opy), 6, st, &h->ymaps, &st->status, s, &h->pyh, at<int>(h, h->opyh)))) return e;
        mark(g.xtc ? kTcNames[q] : nm[3]);
        if (br && (e = cudaStreamWaitEvent(s, h->ev_kin, 0))) return e;
        XExtra xe{};
        xe.frame = at<Frame>(h, h->oframe);
        xe.shape = make_shape(h);
        xe.part = at<double>(h, h->opart);
        xe.comp0 = 0;
        set_wake(h, xe);
        xe.sponge_fused = has_sponge(h) && !sponge_kernel(h);
        xe.err = &st->status;
        if ((e = launch_xpass(fp64, XP_PHYS, W, g, h->px, tx, at<int>(h, h->opx), xe, st, s))) return e;
        if (q == 0) {
            mark("scalars");
            if (branch) {
                if ((e = cudaEventRecord(h->ev_x, s))) return e;
                if ((e = cudaStreamWaitEvent(sk, h->ev_x, 0))) return e;
            }
            double3 opts = make_double3(h->opt.cfl, h->opt.dt_fixed, h->opt.dt_max);
            k_scalars<<<dim3(1, 1, current_batch().n), 256, 0, sk>>>(g, at<double>(h, h->opart), h->xgrid, st, coef, at<double>(h, h->orows),
                                         h->opt.force_ring, at<double>(h, h->oetab), opts, rk4_dt_diff(h),
                                         at<Frame>(h, h->oframe), at<flusi_insect>(h, h->oins), current_batch().mb);
            if ((e = cudaGetLastError())) return e;
            if (branch && (e = cudaEventRecord(h->ev_sc, sk))) return e;
        }
        if (sponge_kernel(h)) {
            mark(nm[4]);
            // chi_sp omega of the vorticity still in W[3..5] (x transformed back in place)
            XExtra xs{};
            xs.ncomp = 3;
            xs.comp0 = 3;
            set_wake(h, xs);
            if ((e = launch_xpass(fp64, XP_SPONGE, W, g, h->px, tx, at<int>(h, h->opx), xs, st, s))) return e;
        }
        mark(nm[5]);
        if ((e = launch_ypass(fp64, false, W, g, h->py, ty, at<int>(h, h->opy), nfwd, st, &h->ymaps, &st->status, s, &h->pyh, at<int>(h, h->opyh)))) return e;
        mark(nm[6]);
        if ((e = launch_zfwd(fp64, W, nfwd, g, h->pz, tz, at<int>(h, h->opz), st, &h->zmaps.w, h->zmaps.w_bh,
                             &st->status, s)))
            return e;
        mark(nm[7]);
        if (q == 0 && branch && (e = cudaStreamWaitEvent(s, h->ev_sc, 0))) return e;
        ZfwdExtra ze = zextra(h);
        ze.stage = h->ws + h->oUt;
        if ((e = launch_zupdate(fp64, is_rk4(h) ? 2 + q : 0, W, h->ws + h->oU, h->ws + h->oH, g, ze, st, s)))
            return e;
    }
    mark(nullptr);
    return cudaSuccess;
}

int check_ready(flusi_t h, bool need_state)
{
    if (!h) return FLUSI_EINVAL;
    if (!h->bound) return fail(h, FLUSI_ESTATE, "no workspace bound (flusi_bind)");
    if (need_state && !h->has_state) return fail(h, FLUSI_ESTATE, "no state set (flusi_set_state)");
    return FLUSI_OK;
}

void drop_graph(flusi_t h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->graph_ok = 0;
    ++h->generation;
}

int read_status(flusi_t h, StepState* out)
{
    StepState st;
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    CK(cudaMemcpy(&st, h->ws + h->ostate, sizeof st, cudaMemcpyDeviceToHost), "read step state");
    if (out) *out = st;
    if (st.status != 0) {
        h->poisoned = 1;
        return fail(h, st.status, st.status == FLUSI_ENONFINITE
                                      ? "non-finite velocity or nonlinear term on the device"
                                      : "device-side failure");
    }
    return FLUSI_OK;
}

// Quaternion of the yaw-pitch-roll orientation (psi, beta, gamma) of Eq.
// M_body_yawpitchroll.  M_body = R_x(psi) R_y(beta) R_z(gamma) maps global to
// body coordinates, so the body-to-global map is the active rotation by gamma
// about z after beta about y after psi about x: eps = q_z (x) q_y (x) q_x, with
// q_n(a) = (cos a/2, sin a/2 n) and (x) the quaternion product.
void quat_of_angles(double psi, double beta, double gamma, double* eps)
{
    auto mulq = [](const double* a, const double* b, double* c) {
        double r[4] = {a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3],
                       a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2],
                       a[0] * b[2] + a[2] * b[0] + a[3] * b[1] - a[1] * b[3],
                       a[0] * b[3] + a[3] * b[0] + a[1] * b[2] - a[2] * b[1]};
        std::memcpy(c, r, sizeof r);
    };
    const double qx[4] = {std::cos(0.5 * psi), std::sin(0.5 * psi), 0, 0};
    const double qy[4] = {std::cos(0.5 * beta), 0, std::sin(0.5 * beta), 0};
    const double qz[4] = {std::cos(0.5 * gamma), 0, 0, std::sin(0.5 * gamma)};
    double t[4];
    mulq(qz, qy, t);
    mulq(t, qx, eps);
}

// TMA descriptors of the bound workspace (none with use_tma = 0).
int prepare_maps(flusi_t h)
{
    h->ymaps = YMaps{};
    h->zmaps = ZMaps{};
    if (!h->opt.use_tma) return FLUSI_OK;
    CK(prepare_ymaps(h->prec == FLUSI_FP64, h->ws + h->oW, h->g, &h->ymaps), "y tensor maps");
    CK(prepare_zmaps(h->prec == FLUSI_FP64, h->ws + h->oU, is_rk4(h) ? h->ws + h->oUt : nullptr, h->ws + h->oW,
                     h->g, &h->zmaps),
       "z tensor maps");
    return FLUSI_OK;
}

// Shapes are value-initialized, padding included, so bytes compare fields.
bool same_shape(const Shape& a, const Shape& b) { return std::memcmp(&a, &b, sizeof a) == 0; }

size_t real_size(int where, int prec)
{
    if (where == FLUSI_HOST_FP64) return 8;
    if (where == FLUSI_HOST_FP32) return 4;
    return prec == FLUSI_FP64 ? 8 : 4;
}

}  // namespace

extern "C" {

void flusi_default_options(flusi_options* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->cfl = 0.1;
    o->force_ring = 4096;
    o->use_graph = 1;
    o->use_tma = 1;
}

int flusi_create(int nx, int ny, int nz, const double L[3], double nu, double eta, int precision,
                 flusi_t* out)
{
    if (!out) return fail(nullptr, FLUSI_EINVAL, "out is NULL");
    *out = nullptr;
    if (!smooth_size(nx) || !smooth_size(ny) || !smooth_size(nz) || nx % 2 != 0)
        return fail(nullptr, FLUSI_EINVAL, "each n must be 2^a 3^b in [8, 1024], nx even");
    if (!L || !(L[0] > 0) || !(L[1] > 0) || !(L[2] > 0)) return fail(nullptr, FLUSI_EINVAL, "box sides must be > 0");
    if (!(nu >= 0) || !(eta > 0)) return fail(nullptr, FLUSI_EINVAL, "need nu >= 0 and eta > 0");
    if (precision < FLUSI_FP64 || precision > FLUSI_FP32_SPLITBF16X3) return fail(nullptr, FLUSI_EINVAL, "bad precision");
    if (precision >= FLUSI_FP32_SPLITBF16 && !xpass_tc_supported(nx))
        return fail(nullptr, FLUSI_EINVAL, "split-BF16 tensor-core stages are built for nx = 256 and 512");
    flusi_t h = new (std::nothrow) flusi_s();
    if (!h) return fail(nullptr, FLUSI_ENOMEM, "host allocation failed");
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->prec = precision;
    for (int i = 0; i < 3; ++i) h->L[i] = L[i];
    h->nu = nu;
    h->eta = eta;
    flusi_default_options(&h->opt);
    h->tune.y_plan = h->tune.zf_plan = 1;
    layout(h);
    *out = h;
    return FLUSI_OK;
}

int flusi_set_options(flusi_t h, const flusi_options* o)
{
    if (!h || !o) return fail(h, FLUSI_EINVAL, "NULL argument");
    if (!(o->cfl > 0) || o->dt_fixed < 0 || o->dt_max < 0 || o->force_ring < 1 ||
        (o->mean_mode != 0 && o->mean_mode != 1) || (o->dealias_strict != 0 && o->dealias_strict != 1))
        return fail(h, FLUSI_EINVAL, "bad option value");
    if (!(o->sponge_c >= 0) || !std::isfinite(o->sponge_c))
        return fail(h, FLUSI_EINVAL, "sponge_c must be >= 0 (0: no sponge)");
    if (o->time_scheme != 0 && o->time_scheme != 1) return fail(h, FLUSI_EINVAL, "time_scheme must be 0 or 1");
    if (o->use_tma != 0 && o->use_tma != 1) return fail(h, FLUSI_EINVAL, "use_tma must be 0 or 1");
    if (h->bound && o->time_scheme != h->opt.time_scheme)
        return fail(h, FLUSI_EINVAL, "time_scheme cannot change after flusi_bind");
    if (o->time_scheme != 0 && h->have_ins && h->ins.free_flight)
        return fail(h, FLUSI_EINVAL, "free flight needs time_scheme 0");
    for (int i = 0; i < 3; ++i)
        if (!(o->sponge_width[i] >= 0 && o->sponge_width[i] <= h->L[i]) ||
            !(o->layer_width[i] >= 0 && o->layer_width[i] <= h->L[i]))
            return fail(h, FLUSI_EINVAL, "sponge and layer widths must lie in [0, L]");
    if (h->bound && (o->force_ring != h->opt.force_ring || o->dealias_strict != h->opt.dealias_strict))
        return fail(h, FLUSI_EINVAL, "force_ring and dealias_strict cannot change after flusi_bind");
    h->opt = *o;
    layout(h);
    drop_graph(h);
    if (h->bound) {
        int rc = prepare_maps(h);
        if (rc) return rc;
    }
    return FLUSI_OK;
}

int flusi_workspace_bytes(flusi_t h, size_t* bytes)
{
    if (!h || !bytes) return fail(h, FLUSI_EINVAL, "NULL argument");
    *bytes = h->total;
    return FLUSI_OK;
}

int flusi_bind(flusi_t h, void* ws, size_t bytes, void* stream)
{
    if (!h || !ws) return fail(h, FLUSI_EINVAL, "NULL argument");
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return fail(h, FLUSI_EINVAL, "workspace not 256-byte aligned");
    if (bytes < h->total) return fail(h, FLUSI_ENOMEM, "workspace smaller than flusi_workspace_bytes");
    {
        // kernel attributes (shared-memory limits), once per device
        static std::mutex mu;
        static std::vector<int> done;
        int dev = 0;
        CK(cudaGetDevice(&dev), "cudaGetDevice");
        std::lock_guard<std::mutex> lock(mu);
        if (std::find(done.begin(), done.end(), dev) == done.end()) {
            CK(configure_ypass(), "configure y pass");
            CK(configure_zpass(), "configure z pass");
            CK(configure_xpass(), "configure x pass");
            CK(configure_xpass_tc(), "configure tensor-core x pass");
            done.push_back(dev);
        }
    }
    drop_graph(h);
    h->ws = static_cast<char*>(ws);
    h->ws_bytes = bytes;
    h->stream = static_cast<cudaStream_t>(stream);
    h->xgrid = xpass_grid(h->prec == FLUSI_FP64, h->g);
    int rc = prepare_maps(h);
    if (rc) return rc;
    if (h->xgrid > h->part_cap) h->xgrid = h->part_cap;
    CK(cudaMemsetAsync(h->ws, 0, h->total, h->stream), "clear workspace");
    auto tx = twiddles(h->nx), ty = twiddles(h->ny), tz = twiddles(h->nz);
    auto fx = twiddles32(tx), fy = twiddles32(ty), fz = twiddles32(tz);
    auto px = digit_reversal(h->px), py = digit_reversal(h->py), pz = digit_reversal(h->pz);
    auto pzi = digit_reversal(h->pzi);
    struct Tab {
        size_t off;
        const std::vector<double2>* d;
        const std::vector<float2>* f;
    };
    for (const Tab& t : {Tab{h->otx, &tx, &fx}, Tab{h->oty, &ty, &fy}, Tab{h->otz, &tz, &fz}}) {
        const size_t n = t.d->size();
        CK(cudaMemcpyAsync(h->ws + t.off, t.d->data(), sizeof(double2) * n, cudaMemcpyHostToDevice, h->stream),
           "twiddles");
        CK(cudaMemcpyAsync(h->ws + t.off + sizeof(double2) * n, t.f->data(), sizeof(float2) * n,
                           cudaMemcpyHostToDevice, h->stream),
           "twiddles");
    }
    CK(cudaMemcpyAsync(h->ws + h->opx, px.data(), sizeof(int) * px.size(), cudaMemcpyHostToDevice, h->stream), "digit reversal");
    CK(cudaMemcpyAsync(h->ws + h->opy, py.data(), sizeof(int) * py.size(), cudaMemcpyHostToDevice, h->stream), "digit reversal");
    CK(cudaMemcpyAsync(h->ws + h->opz, pz.data(), sizeof(int) * pz.size(), cudaMemcpyHostToDevice, h->stream), "digit reversal");
    CK(cudaMemcpyAsync(h->ws + h->opzi, pzi.data(), sizeof(int) * pzi.size(), cudaMemcpyHostToDevice, h->stream),
       "digit reversal");
    std::vector<int> pyh;
    if (h->pyh.n > 0) {
        pyh = digit_reversal(h->pyh);
        CK(cudaMemcpyAsync(h->ws + h->opyh, pyh.data(), sizeof(int) * pyh.size(), cudaMemcpyHostToDevice,
                           h->stream),
           "digit reversal");
    }
    // the host tables must outlive the asynchronous copies
    CK(cudaStreamSynchronize(h->stream), "bind tables");
    if (h->have_ins)
        CK(cudaMemcpyAsync(h->ws + h->oins, &h->ins, sizeof h->ins, cudaMemcpyHostToDevice, h->stream), "insect");
    CK(cudaStreamSynchronize(h->stream), "bind");
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "capture stream");
    if (!h->side) CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking), "side stream");
    for (cudaEvent_t* ev : {&h->ev_fork, &h->ev_kin, &h->ev_x, &h->ev_sc})
        if (!*ev) CK(cudaEventCreateWithFlags(ev, cudaEventDisableTiming), "step events");
    h->bound = 1;
    h->has_state = 0;
    return FLUSI_OK;
}

int flusi_set_kinematics(flusi_t h, const flusi_insect* ins)
{
    if (!h) return FLUSI_EINVAL;
    const Shape before = make_shape(h);
    double qn = 0.0;
    if (ins) {
        if (const char* why = insect_error(*ins)) return fail(h, FLUSI_EINVAL, why);
        if (ins->free_flight != 0 && ins->free_flight != 1) return fail(h, FLUSI_EINVAL, "free_flight must be 0 or 1");
        if (ins->free_flight) {
            bool ok = ins->mass > 0 && std::isfinite(ins->gravity) && h->opt.time_scheme == 0;
            for (int i = 0; i < 3; ++i) ok = ok && ins->J_body[i] > 0 && std::isfinite(ins->Omega_body[i]);
            for (int i = 0; i < 6; ++i) ok = ok && std::isfinite(ins->dof[i]);
            if (!ok)
                return fail(h, FLUSI_EINVAL, "free flight needs mass > 0, J_body > 0, finite gravity, dof and "
                                             "Omega_body, and time_scheme 0");
        }
        for (int i = 0; i < 4; ++i) qn += ins->quat[i] * ins->quat[i];
        if (!std::isfinite(qn)) return fail(h, FLUSI_EINVAL, "bad quaternion");
    }
    // page-locked upload slots, before anything of the handle changes: made
    // into locals and handed to the handle only when every part exists, so a
    // failure leaves the handle as it was (and the next call tries again)
    if (h->bound && !h->ins_stage) {
        flusi_insect* stage = nullptr;
        cudaEvent_t ev[kStageSlots] = {};
        cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&stage), sizeof(flusi_insect) * kStageSlots,
                                      cudaHostAllocDefault);
        for (int k = 0; k < kStageSlots && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (cudaEvent_t x : ev)
                if (x) cudaEventDestroy(x);
            if (stage) cudaFreeHost(stage);
            return fail(h, FLUSI_ECUDA, (std::string("pinned descriptor slots: ") + cudaGetErrorString(e)).c_str());
        }
        h->ins_stage = stage;
        for (int k = 0; k < kStageSlots; ++k) h->stage_ev[k] = ev[k];
    }
    if (ins) {
        h->ins = *ins;
        h->have_ins = 1;
        if (qn == 0.0) {
            quat_of_angles(ins->psi, ins->beta, ins->gamma, h->ins.quat);
        } else if (qn != 1.0) {
            for (int i = 0; i < 4; ++i) h->ins.quat[i] = ins->quat[i] / std::sqrt(qn);
        }
    } else {
        std::memset(&h->ins, 0, sizeof h->ins);
        h->have_ins = 0;
    }
    // the step kernels read the descriptor from device memory in stream order;
    // only the mask shape is baked into the captured kernel arguments
    if (h->bound) {
        const int k = h->stage_next;
        h->stage_next = (k + 1) % kStageSlots;
        CK(cudaEventSynchronize(h->stage_ev[k]), "descriptor slot");   // its previous copy has run
        h->ins_stage[k] = h->ins;
        CK(cudaMemcpyAsync(h->ws + h->oins, &h->ins_stage[k], sizeof h->ins, cudaMemcpyHostToDevice, h->stream),
           "insect");
        CK(cudaEventRecord(h->stage_ev[k], h->stream), "descriptor slot");
    }
    if (!same_shape(before, make_shape(h))) drop_graph(h);
    return FLUSI_OK;
}

namespace {

// The 13 body-state values inside a device descriptor: x_cntr and u_cntr
// are adjacent, so are quat and Omega_body.
constexpr size_t kBodyA = offsetof(flusi_insect, x_cntr), kBodyB = offsetof(flusi_insect, quat);
static_assert(offsetof(flusi_insect, u_cntr) == kBodyA + 3 * sizeof(double), "x_cntr, u_cntr adjacent");
static_assert(offsetof(flusi_insect, Omega_body) == kBodyB + 4 * sizeof(double), "quat, Omega_body adjacent");

cudaError_t read_body(flusi_t h, double* y)
{
    cudaError_t e = cudaMemcpy(y, h->ws + h->oins + kBodyA, 6 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e) return e;
    return cudaMemcpy(y + 6, h->ws + h->oins + kBodyB, 7 * sizeof(double), cudaMemcpyDeviceToHost);
}

cudaError_t write_body(flusi_t h, const double* y)
{
    cudaError_t e = cudaMemcpy(h->ws + h->oins + kBodyA, y, 6 * sizeof(double), cudaMemcpyHostToDevice);
    if (e) return e;
    return cudaMemcpy(h->ws + h->oins + kBodyB, y + 6, 7 * sizeof(double), cudaMemcpyHostToDevice);
}

}  // namespace

int flusi_get_body(flusi_t h, double* state)
{
    if (!h || !state) return fail(h, FLUSI_EINVAL, "NULL argument");
    int rc = check_ready(h, false);
    if (rc) return rc;
    if (!h->have_ins) return fail(h, FLUSI_ESTATE, "no insect set");
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    CK(read_body(h, state), "read body state");
    return FLUSI_OK;
}

int flusi_set_state(flusi_t h, const void* u, int where)
{
    int rc = check_ready(h, false);
    if (rc) return rc;
    if (!u) return fail(h, FLUSI_EINVAL, "u is NULL");
    if (where < FLUSI_HOST_FP64 || where > FLUSI_DEVICE) return fail(h, FLUSI_EINVAL, "bad `where`");
    const Geom& g = h->g;
    const int fp64 = h->prec == FLUSI_FP64;
    const size_t N = (size_t)g.nx * g.ny * g.nz;
    void* W = h->ws + h->oW;
    const double2* tx = at<double2>(h, h->otx);
    cudaStream_t s = h->stream;
    CK(cudaStreamSynchronize(s), "sync before set_state");
    k_reset_state<<<1, 1, 0, s>>>(at<StepState>(h, h->ostate), at<StepCoef>(h, h->ocoef));
    CK(cudaGetLastError(), "reset");
    XExtra xe{};
    xe.cstride = (long long)N;
    if (where == FLUSI_DEVICE) {
        xe.rin = u;
        xe.real_fp64 = fp64;
        xe.ncomp = 3;
        xe.comp0 = 0;
        CK(launch_xpass(fp64, XP_R2C, W, g, h->px, tx, at<int>(h, h->opx), xe, nullptr, s), "x r2c");
    } else {
        const size_t es = real_size(where, h->prec);
        char* stage = h->ws + h->oW + (size_t)3 * g.nz * g.ny * g.Mxp * (fp64 ? 16 : 8);
        for (int c = 0; c < 3; ++c) {
            CK(cudaMemcpyAsync(stage, static_cast<const char*>(u) + c * N * es, N * es,
                               cudaMemcpyHostToDevice, s), "copy state in");
            xe.rin = stage;
            xe.real_fp64 = where == FLUSI_HOST_FP64;
            xe.ncomp = 1;
            xe.comp0 = c;
            CK(launch_xpass(fp64, XP_R2C, W, g, h->px, tx, at<int>(h, h->opx), xe, nullptr, s), "x r2c");
        }
    }
    CK(launch_ypass(fp64, false, W, g, h->py, at<double2>(h, h->oty), at<int>(h, h->opy), 3, nullptr,
                    &h->ymaps, status_word(h), s, &h->pyh, at<int>(h, h->opyh)), "y forward");
    CK(launch_zfwd(fp64, W, 3, g, h->pz, at<double2>(h, h->otz), at<int>(h, h->opz), nullptr, &h->zmaps.w,
                   h->zmaps.w_bh, status_word(h), s),
       "z forward");
    ZfwdExtra ze = zextra(h);
    ze.coef = nullptr;
    ze.etab = nullptr;
    ze.sponge_c = 0;
    CK(launch_zupdate(fp64, 1, W, h->ws + h->oU, h->ws + h->oH, g, ze, nullptr, s), "spectral set");
    CK(cudaStreamSynchronize(s), "set_state");
    h->has_state = 1;
    h->poisoned = 0;
    h->rows_read = 0;
    h->n_enq = 0;
    return FLUSI_OK;
}

int flusi_step(flusi_t h, int n)
{
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (n < 0) return fail(h, FLUSI_EINVAL, "n < 0");
    if (h->poisoned) return fail(h, FLUSI_ESTATE, "a device error poisoned the handle; set a new state");
    if (n == 0) return FLUSI_OK;
    if (!h->opt.use_graph) {
        for (int i = 0; i < n; ++i) {
            CK(enqueue_step(h, h->stream, nullptr), "enqueue step");
            ++h->n_enq;
        }
        return FLUSI_OK;
    }
    if (!h->graph_ok) {
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e = enqueue_step(h, h->cap_stream, nullptr);
        cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(h, e, "capture step");
        }
        CK(e2, "end capture");
        e = cudaGraphInstantiate(&h->gexec, graph, 0);
        cudaGraphDestroy(graph);
        CK(e, "instantiate graph");
        h->graph_ok = 1;
    }
    for (int i = 0; i < n; ++i) {
        CK(cudaGraphLaunch(h->gexec, h->stream), "graph launch");
        ++h->n_enq;
    }
    return FLUSI_OK;
}

int flusi_sync(flusi_t h)
{
    int rc = check_ready(h, false);
    if (rc) return rc;
    return read_status(h, nullptr);
}

int flusi_forces(flusi_t h, double* rows, int cap, int* count, long long* lost)
{
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (!rows || !count || cap < 0) return fail(h, FLUSI_EINVAL, "bad argument");
    *count = 0;
    if (lost) *lost = 0;
    StepState st;
    rc = read_status(h, &st);
    if (rc) return rc;
    const long long ring = h->opt.force_ring;
    long long avail = st.n - h->rows_read;
    long long dropped = avail > ring ? avail - ring : 0;
    long long first = h->rows_read + dropped;
    long long take = std::min<long long>(avail - dropped, cap);
    const double* dev = at<double>(h, h->orows);
    long long done = 0;
    while (done < take) {
        long long idx = (first + done) % ring;
        long long chunk = std::min(take - done, ring - idx);
        CK(cudaMemcpy(rows + done * kRowCols, dev + idx * kRowCols, sizeof(double) * kRowCols * chunk,
                      cudaMemcpyDeviceToHost), "read force rows");
        done += chunk;
    }
    h->rows_read = first + take;
    *count = (int)take;
    if (lost) *lost = dropped;
    return FLUSI_OK;
}

int flusi_forces_async(flusi_t h, double* rows, int cap, int* count, long long* lost)
{
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (!rows || !count || cap < 0) return fail(h, FLUSI_EINVAL, "bad argument");
    if (h->poisoned) return fail(h, FLUSI_ESTATE, "a device error poisoned the handle");
    *count = 0;
    if (lost) *lost = 0;
    const long long ring = h->opt.force_ring;
    const long long avail = h->n_enq - h->rows_read;
    const long long dropped = avail > ring ? avail - ring : 0;
    const long long first = h->rows_read + dropped;
    const long long take = std::min<long long>(avail - dropped, cap);
    const double* dev = at<double>(h, h->orows);
    long long done = 0;
    while (done < take) {
        const long long idx = (first + done) % ring;
        const long long chunk = std::min(take - done, ring - idx);
        CK(cudaMemcpyAsync(rows + done * kRowCols, dev + idx * kRowCols, sizeof(double) * kRowCols * chunk,
                           cudaMemcpyDeviceToHost, h->stream),
           "enqueue force rows");
        done += chunk;
    }
    h->rows_read = first + take;
    *count = (int)take;
    if (lost) *lost = dropped;
    return FLUSI_OK;
}

int flusi_get_state(flusi_t h, void* u_out, int where, double* t, long long* step)
{
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (!u_out) return fail(h, FLUSI_EINVAL, "u_out is NULL");
    if (where < FLUSI_HOST_FP64 || where > FLUSI_DEVICE) return fail(h, FLUSI_EINVAL, "bad `where`");
    StepState st;
    rc = read_status(h, &st);
    if (rc) return rc;
    const Geom& g = h->g;
    const int fp64 = h->prec == FLUSI_FP64;
    const size_t N = (size_t)g.nx * g.ny * g.nz;
    void* W = h->ws + h->oW;
    cudaStream_t s = h->stream;
    CK(launch_zinv(fp64, h->ws + h->oU, W, g, h->pzi, at<double2>(h, h->otz), at<int>(h, h->opzi), 3, nullptr,
                   &h->zmaps.u, h->zmaps.u_bh, status_word(h), s),
       "z inverse");
    CK(launch_ypass(fp64, true, W, g, h->py, at<double2>(h, h->oty), at<int>(h, h->opy), 3, nullptr,
                    &h->ymaps, status_word(h), s, &h->pyh, at<int>(h, h->opyh)), "y inverse");
    XExtra xe{};
    xe.cstride = (long long)N;
    if (where == FLUSI_DEVICE) {
        xe.rout = u_out;
        xe.real_fp64 = fp64;
        xe.ncomp = 3;
        xe.comp0 = 0;
        CK(launch_xpass(fp64, XP_C2R, W, g, h->px, at<double2>(h, h->otx), at<int>(h, h->opx), xe, nullptr, s), "x c2r");
        CK(cudaStreamSynchronize(s), "get_state");
    } else {
        const size_t es = real_size(where, h->prec);
        char* stage = h->ws + h->oW + (size_t)3 * g.nz * g.ny * g.Mxp * (fp64 ? 16 : 8);
        for (int c = 0; c < 3; ++c) {
            xe.rout = stage;
            xe.real_fp64 = where == FLUSI_HOST_FP64;
            xe.ncomp = 1;
            xe.comp0 = c;
            CK(launch_xpass(fp64, XP_C2R, W, g, h->px, at<double2>(h, h->otx), at<int>(h, h->opx), xe, nullptr, s), "x c2r");
            CK(cudaMemcpyAsync(static_cast<char*>(u_out) + c * N * es, stage, N * es,
                               cudaMemcpyDeviceToHost, s), "copy state out");
        }
        CK(cudaStreamSynchronize(s), "get_state");
    }
    if (t) *t = st.t;
    if (step) *step = st.n;
    return FLUSI_OK;
}

int flusi_divergence(flusi_t h, double* div_max, double* ku_max)
{
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (!div_max) return fail(h, FLUSI_EINVAL, "div_max is NULL");
    rc = read_status(h, nullptr);
    if (rc) return rc;
    // the per-CTA partial-sum rows are free between steps (stream order)
    unsigned long long* slot = at<unsigned long long>(h, h->opart);
    CK(launch_divergence(h->prec == FLUSI_FP64, h->ws + h->oU, h->g, slot, h->stream), "divergence");
    unsigned long long bits[2] = {0, 0};
    CK(cudaMemcpyAsync(bits, slot, sizeof bits, cudaMemcpyDeviceToHost, h->stream), "read divergence");
    CK(cudaStreamSynchronize(h->stream), "divergence");
    std::memcpy(div_max, &bits[0], sizeof(double));
    if (ku_max) std::memcpy(ku_max, &bits[1], sizeof(double));
    return FLUSI_OK;
}

int flusi_get_spectrum(flusi_t h, double* uh_out)
{
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (!uh_out) return fail(h, FLUSI_EINVAL, "uh_out is NULL");
    rc = read_status(h, nullptr);
    if (rc) return rc;
    const Geom& g = h->g;
    const int fp64 = h->prec == FLUSI_FP64;
    const size_t cnt = (size_t)3 * g.Mz * g.My * g.Mxp;
    std::vector<double> host(cnt * 2);
    if (fp64) {
        CK(cudaMemcpy(host.data(), h->ws + h->oU, cnt * 16, cudaMemcpyDeviceToHost), "read spectrum");
    } else {
        std::vector<float> f(cnt * 2);
        CK(cudaMemcpy(f.data(), h->ws + h->oU, cnt * 8, cudaMemcpyDeviceToHost), "read spectrum");
        for (size_t i = 0; i < f.size(); ++i) host[i] = f[i];
    }
    const int hx = g.nx / 2 + 1;
    const size_t full = (size_t)g.nz * g.ny * hx;
    std::memset(uh_out, 0, sizeof(double) * 2 * 3 * full);
    for (int c = 0; c < 3; ++c)
        for (int jz = 0; jz < g.Mz; ++jz)
            for (int jy = 0; jy < g.My; ++jy)
                for (int x = 0; x < g.Mx; ++x) {
                    const int iz = slot_of(jz, g.Kz, g.nz), iy = slot_of(jy, g.Ky, g.ny);
                    const size_t src = (((size_t)c * g.Mz + jz) * g.My + jy) * g.Mxp + x;
                    const size_t dst = c * full + ((size_t)iz * g.ny + iy) * hx + x;
                    uh_out[2 * dst] = host[2 * src];
                    uh_out[2 * dst + 1] = host[2 * src + 1];
                }
    return FLUSI_OK;
}

int flusi_debug_wait_timeout(flusi_t h, double milliseconds)
{
    int rc = check_ready(h, false);
    if (rc) return rc;
    if (!(milliseconds > 0 && milliseconds <= 1000)) return fail(h, FLUSI_EINVAL, "milliseconds must be in (0, 1000]");
    int dev = 0, khz = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev), "clock rate");
    if (khz <= 0) khz = 2000000;
    const long long cycles = (long long)(milliseconds * khz);
    k_wait_probe<<<1, 32, 0, h->stream>>>(status_word(h), cycles);
    CK(cudaGetLastError(), "wait probe");
    return FLUSI_OK;
}

int flusi_debug_inject(flusi_t h, int component, int mx, int my, int mz, double re, double im)
{
    int rc = check_ready(h, true);
    if (rc) return rc;
    const Geom& g = h->g;
    if (component < 0 || component > 2 || mx < 0 || mx > g.Kx || my < -g.Ky || my > g.Ky || mz < -g.Kz ||
        mz > g.Kz)
        return fail(h, FLUSI_EINVAL, "component or mode outside the kept modes");
    const int jy = my >= 0 ? my : g.My + my, jz = mz >= 0 ? mz : g.Mz + mz;
    const size_t idx = (size_t)component * g.Mz * g.My * g.Mxp + ((size_t)jz * g.My + jy) * g.Mxp + mx;
    // after the enqueued steps; the next step reads it
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (h->prec == FLUSI_FP64) {
        const double v[2] = {re, im};
        CK(cudaMemcpy(h->ws + h->oU + idx * sizeof(v), v, sizeof(v), cudaMemcpyHostToDevice), "inject");
    } else {
        const float v[2] = {(float)re, (float)im};
        CK(cudaMemcpy(h->ws + h->oU + idx * sizeof(v), v, sizeof(v), cudaMemcpyHostToDevice), "inject");
    }
    return FLUSI_OK;
}

int flusi_debug_fields(flusi_t h, void* out_dev)
{
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (!out_dev) return fail(h, FLUSI_EINVAL, "out_dev is NULL");
    const Geom& g = h->g;
    const int fp64 = h->prec == FLUSI_FP64;
    cudaStream_t s = h->stream;
    void* W = h->ws + h->oW;
    StepState* st = at<StepState>(h, h->ostate);
    k_kinematics<<<1, 32, 0, s>>>(at<flusi_insect>(h, h->oins), st, at<StepCoef>(h, h->ocoef),
                                  at<Frame>(h, h->oframe), box_margin(h), 0.0, nullptr, make_shape(h), 1,
                                  1.0 / g.eta);
    CK(cudaGetLastError(), "kinematics");
    CK(launch_zinv(fp64, h->ws + h->oU, W, g, h->pzi, at<double2>(h, h->otz), at<int>(h, h->opzi), 6, nullptr,
                   &h->zmaps.u, h->zmaps.u_bh, status_word(h), s),
       "z inverse");
    CK(launch_ypass(fp64, true, W, g, h->py, at<double2>(h, h->oty), at<int>(h, h->opy), 6, nullptr,
                    &h->ymaps, status_word(h), s, &h->pyh, at<int>(h, h->opyh)), "y inverse");
    XExtra xe{};
    xe.frame = at<Frame>(h, h->oframe);
    xe.shape = make_shape(h);
    xe.rout = out_dev;
    xe.comp0 = 0;
    set_wake(h, xe);
    CK(launch_xpass(fp64, XP_DUMP, W, g, h->px, at<double2>(h, h->otx), at<int>(h, h->opx), xe, nullptr, s), "x dump");
    return FLUSI_OK;
}

int flusi_profile_step(flusi_t h, int n, double* ms, const char** names, int* nk)
{
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (n < 1 || !ms || !nk) return fail(h, FLUSI_EINVAL, "bad argument");
    if (h->poisoned) return fail(h, FLUSI_ESTATE, "handle poisoned");
    const int nk_step = step_kernels(h);
    if (nk_step > FLUSI_PROFILE_MAX) return fail(h, FLUSI_EINVAL, "too many kernels per step to profile");
    cudaEvent_t ev[kMaxStepKernels + 1];
    const char* nm[kMaxStepKernels + 1];
    for (auto& e : ev) CK(cudaEventCreate(&e), "event");
    std::vector<double> acc(nk_step, 0.0);
    for (int i = 0; i < n; ++i) {
        CK(enqueue_step(h, h->stream, ev, nm), "enqueue step");
        ++h->n_enq;
        CK(cudaEventSynchronize(ev[nk_step]), "event sync");
        for (int k = 0; k < nk_step; ++k) {
            float t = 0;
            CK(cudaEventElapsedTime(&t, ev[k], ev[k + 1]), "elapsed");
            acc[k] += t;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    for (int k = 0; k < nk_step; ++k) {
        ms[k] = acc[k] / n;
        if (names) names[k] = nm[k];
    }
    *nk = nk_step;
    return read_status(h, nullptr);
}

int flusi_kernels_per_step(flusi_t h, int* count)
{
    if (!h || !count) return FLUSI_EINVAL;
    *count = step_kernels(h);
    return FLUSI_OK;
}

// ---------------------------------------------------------------- tuning

namespace {

int tuning_error(flusi_t h, const flusi_tuning& t)
{
    const int cmin = h->prec == FLUSI_FP64 ? 2 : 4;   // 32 bytes of complex values
    auto cols_ok = [&](int c) { return c == 0 || (c >= cmin && c <= 256 && (c & (c - 1)) == 0); };
    if (t.y_plan < 0 || t.y_plan > 2 || t.zf_plan < 0 || t.zf_plan > 2)
        return fail(h, FLUSI_EINVAL, "y_plan and zf_plan must be 0, 1 or 2");
    if (!cols_ok(t.y_cols) || !cols_ok(t.z_cols))
        return fail(h, FLUSI_EINVAL, "y_cols and z_cols must be 0 or a power of two in [32 bytes, 256]");
    if (t.x_kernel != 0 && t.x_kernel != 1) return fail(h, FLUSI_EINVAL, "x_kernel must be 0 or 1");
    if (t.y_pair != 0 && t.y_pair != 1) return fail(h, FLUSI_EINVAL, "y_pair must be 0 or 1");
    return FLUSI_OK;
}

void radices(const FftPlan& p, int* out)
{
    for (int s = 0; s < FLUSI_MAX_STAGES; ++s) out[s] = s < p.nst ? p.radix[s] : 0;
}

// Sum of the mean per-kernel times (ms) of the kernels whose names, stage
// suffix removed, are in `names`, over `steps` un-captured steps after one
// untimed step.
int time_kernels(flusi_t h, int steps, const char* const names[2], double* ms_out)
{
    double ms[FLUSI_PROFILE_MAX];
    const char* nm[FLUSI_PROFILE_MAX];
    int nk = 0;
    int rc = flusi_profile_step(h, 1, ms, nm, &nk);
    if (rc) return rc;
    rc = flusi_profile_step(h, steps, ms, nm, &nk);
    if (rc) return rc;
    double sum = 0;
    for (int k = 0; k < nk; ++k) {
        const std::string base = std::string(nm[k]).substr(0, std::string(nm[k]).find('.'));
        for (int i = 0; i < 2; ++i)
            if (names[i] && base == names[i]) sum += ms[k];
    }
    *ms_out = sum;
    return FLUSI_OK;
}

std::string tuning_key(flusi_t h)
{
    int dev = 0;
    cudaDeviceProp prop{};
    cudaGetDevice(&dev);
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) cudaGetLastError();
    std::string name = prop.name;
    for (char& c : name)
        if (c == ' ' || c == '\t') c = '_';
    const bool wake = h->opt.sponge_c > 0 || h->opt.layer_width[0] > 0 || h->opt.layer_width[1] > 0 ||
                      h->opt.layer_width[2] > 0;
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s|%d|%dx%dx%d|%s|%s|%s|d%d", name.empty() ? "gpu" : name.c_str(),
                  prop.multiProcessorCount, h->nx, h->ny, h->nz,
                  h->prec == FLUSI_FP64 ? "fp64" : h->prec == FLUSI_FP32 ? "fp32" : h->prec == FLUSI_FP32_SPLITBF16 ? "bf16x2" : "bf16x3",
                  is_rk4(h) ? "rk4" : "ab2", wake ? "wake" : "nowake", h->opt.dealias_strict);
    return buf;
}

// the last line of the cache with this key, if any
bool cache_lookup(const char* path, const std::string& key, flusi_tuning* t)
{
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        std::istringstream in(line);
        std::string k;
        flusi_tuning c{};
        if (!(in >> k >> c.y_plan >> c.zf_plan >> c.y_cols >> c.z_cols >> c.x_kernel >> c.y_pair)) continue;
        if (k == key) {
            *t = c;
            found = true;
        }
    }
    return found;
}

}  // namespace

int flusi_get_tuning(flusi_t h, flusi_tuning* out)
{
    if (!h || !out) return fail(h, FLUSI_EINVAL, "NULL argument");
    *out = h->tune;
    const int fp64 = h->prec == FLUSI_FP64;
    out->y_paired = ypass_paired(fp64, h->g);
    radices(out->y_paired ? h->pyh : h->py, out->y_radix);
    radices(h->pz, out->zf_radix);
    radices(h->pzi, out->zi_radix);
    out->y_tile_cols = ypass_tile_cols(fp64, h->g);
    out->z_tile_cols = zpass_tile_cols(fp64, h->g);
    out->x_line_kernel = xpass_fuses_sponge(fp64, h->g);
    return FLUSI_OK;
}

int flusi_set_tuning(flusi_t h, const flusi_tuning* t)
{
    if (!h || !t) return fail(h, FLUSI_EINVAL, "NULL argument");
    int rc = tuning_error(h, *t);
    if (rc) return rc;
    if (h->bound) CK(cudaStreamSynchronize(h->stream), "wait before retuning");
    h->tune = flusi_tuning{};
    h->tune.y_plan = t->y_plan;
    h->tune.zf_plan = t->zf_plan;
    h->tune.y_cols = t->y_cols;
    h->tune.z_cols = t->z_cols;
    h->tune.x_kernel = t->x_kernel;
    h->tune.y_pair = t->y_pair;
    layout(h);
    drop_graph(h);
    if (!h->bound) return FLUSI_OK;
    const auto py = digit_reversal(h->py), pz = digit_reversal(h->pz);
    CK(cudaMemcpyAsync(h->ws + h->opy, py.data(), sizeof(int) * py.size(), cudaMemcpyHostToDevice, h->stream),
       "digit reversal");
    std::vector<int> pyh;
    if (h->pyh.n > 0) {
        pyh = digit_reversal(h->pyh);
        CK(cudaMemcpyAsync(h->ws + h->opyh, pyh.data(), sizeof(int) * pyh.size(), cudaMemcpyHostToDevice,
                           h->stream),
           "digit reversal");
    }
    CK(cudaMemcpyAsync(h->ws + h->opz, pz.data(), sizeof(int) * pz.size(), cudaMemcpyHostToDevice, h->stream),
       "digit reversal");
    CK(cudaStreamSynchronize(h->stream), "retune tables");
    h->xgrid = std::min(xpass_grid(h->prec == FLUSI_FP64, h->g), h->part_cap);
    return prepare_maps(h);
}

int flusi_autotune(flusi_t h, int steps, const char* cache_path, flusi_tuning* out)
{
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (steps < 1 || steps > 1000) return fail(h, FLUSI_EINVAL, "steps must lie in [1, 1000]");
    if (h->poisoned) return fail(h, FLUSI_ESTATE, "a device error poisoned the handle");
    const std::string key = tuning_key(h);
    flusi_tuning best{};
    if (cache_path && cache_lookup(cache_path, key, &best)) {
        rc = flusi_set_tuning(h, &best);
        if (rc) return rc;
        return out ? flusi_get_tuning(h, out) : FLUSI_OK;
    }
    size_t bytes = 0;
    flusi_checkpoint_bytes(h, &bytes);
    std::unique_ptr<char[]> saved(new (std::nothrow) char[bytes]);   // nothing throws across the ABI
    if (!saved) return fail(h, FLUSI_ENOMEM, "no host memory for the state while tuning");
    rc = flusi_save(h, saved.get(), bytes);
    if (rc) return rc;
    flusi_get_tuning(h, &best);
    struct Knob {
        int flusi_tuning::*field;
        const char* kernels[2];
    };
    const Knob knobs[] = {{&flusi_tuning::y_plan, {"yinv", "yfwd"}},
                          {&flusi_tuning::y_pair, {"yinv", "yfwd"}},
                          {&flusi_tuning::y_cols, {"yinv", "yfwd"}},
                          {&flusi_tuning::zf_plan, {"zfwd", nullptr}},
                          {&flusi_tuning::z_cols, {"zinv_curl", "zfwd"}},
                          {&flusi_tuning::x_kernel, {"xpass_phys", "sponge_x"}}};
    for (const Knob& kb : knobs) {
        // candidate values: the plans, or the default tile and two halvings
        std::vector<int> vals;
        if (kb.field == &flusi_tuning::y_plan || kb.field == &flusi_tuning::zf_plan) vals = {1, 0, 2};
        else if (kb.field == &flusi_tuning::y_pair) vals = {0, 1};
        else if (kb.field == &flusi_tuning::x_kernel) vals = {0, 1};
        else {
            flusi_tuning d = best;
            d.*kb.field = 0;
            rc = flusi_set_tuning(h, &d);
            if (rc) break;
            flusi_tuning got{};
            flusi_get_tuning(h, &got);
            const int c0 = kb.field == &flusi_tuning::y_cols ? got.y_tile_cols : got.z_tile_cols;
            vals = {0};
            const int cmin = h->prec == FLUSI_FP64 ? 2 : 4;
            for (int c = c0 / 2; c >= cmin && c >= c0 / 4; c /= 2) vals.push_back(c);
        }
        std::vector<std::string> seen;
        double best_ms = 0;
        int best_v = best.*kb.field, timed = 0;
        for (int v : vals) {
            flusi_tuning t = best;
            t.*kb.field = v;
            rc = flusi_set_tuning(h, &t);
            if (rc) break;
            // settings that give the same plans, tiles and kernels are timed once
            flusi_tuning got{};
            flusi_get_tuning(h, &got);
            std::string sig;
            for (int i = 0; i < FLUSI_MAX_STAGES; ++i)
                sig += std::to_string(got.y_radix[i]) + "," + std::to_string(got.zf_radix[i]) + ",";
            sig += std::to_string(got.y_tile_cols) + "," + std::to_string(got.z_tile_cols) + "," +
                   std::to_string(got.x_line_kernel) + "," + std::to_string(got.y_paired);
            if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
            seen.push_back(sig);
            double ms = 0;
            rc = time_kernels(h, steps, kb.kernels, &ms);
            if (rc) break;
            if (!timed || ms < best_ms) {
                best_ms = ms;
                best_v = v;
            }
            timed = 1;
        }
        if (rc) break;
        best.*kb.field = best_v;
    }
    if (rc) {   // restore the state; the error stays the result
        const std::string msg = h->err;
        if (flusi_load(h, saved.get(), bytes) == FLUSI_OK) h->err = msg;
        return rc;
    }
    rc = flusi_set_tuning(h, &best);
    if (rc) return rc;
    rc = flusi_load(h, saved.get(), bytes);
    if (rc) return rc;
    if (out) flusi_get_tuning(h, out);
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        f << key << ' ' << best.y_plan << ' ' << best.zf_plan << ' ' << best.y_cols << ' ' << best.z_cols << ' '
          << best.x_kernel << ' ' << best.y_pair << '\n';
        if (!f) return fail(h, FLUSI_EINVAL, "cannot append to the tuning cache");
    }
    return FLUSI_OK;
}

// ---------------------------------------------------------------- checkpoints

namespace {

struct CkptHeader {
    char magic[8];               // "FLUSICK2"
    int prec, nx, ny, nz, Mx, My, Mz, Mxp;
    int dealias_strict;
    double L[3], nu, eta;
    unsigned long long spec_bytes;  // one of U, H
};

// after the step state: the free-flight body state (13 doubles, padded)
constexpr size_t kCkptBody = 16 * sizeof(double);

size_t spec_bytes(flusi_t h)
{
    const size_t cs = h->prec == FLUSI_FP64 ? 16 : 8;
    return (size_t)3 * h->g.Mz * h->g.My * h->g.Mxp * cs;
}

CkptHeader make_header(flusi_t h)
{
    CkptHeader c{};
    std::memcpy(c.magic, "FLUSICK2", 8);
    c.prec = h->prec;
    c.nx = h->nx;
    c.ny = h->ny;
    c.nz = h->nz;
    c.Mx = h->g.Mx;
    c.My = h->g.My;
    c.Mz = h->g.Mz;
    c.Mxp = h->g.Mxp;
    c.dealias_strict = h->opt.dealias_strict;
    for (int i = 0; i < 3; ++i) c.L[i] = h->L[i];
    c.nu = h->nu;
    c.eta = h->eta;
    c.spec_bytes = spec_bytes(h);
    return c;
}

}  // namespace

int flusi_checkpoint_bytes(flusi_t h, size_t* bytes)
{
    if (!h || !bytes) return fail(h, FLUSI_EINVAL, "NULL argument");
    *bytes = sizeof(CkptHeader) + sizeof(StepState) + kCkptBody + 2 * spec_bytes(h);
    return FLUSI_OK;
}

int flusi_save(flusi_t h, void* host_buf, size_t bytes)
{
    size_t need = 0;
    if (!h || !host_buf) return fail(h, FLUSI_EINVAL, "NULL argument");
    flusi_checkpoint_bytes(h, &need);
    if (bytes < need) return fail(h, FLUSI_EINVAL, "checkpoint buffer too small");
    int rc = check_ready(h, true);
    if (rc) return rc;
    if (h->poisoned) return fail(h, FLUSI_ESTATE, "a device error poisoned the handle");
    StepState st;
    rc = read_status(h, &st);       // synchronizes; fails on a device error
    if (rc) return rc;
    char* p = static_cast<char*>(host_buf);
    const CkptHeader hd = make_header(h);
    std::memcpy(p, &hd, sizeof hd);
    std::memcpy(p + sizeof hd, &st, sizeof st);
    double body[16] = {};
    if (h->have_ins) CK(read_body(h, body), "save body state");
    std::memcpy(p + sizeof hd + sizeof st, body, kCkptBody);
    char* q = p + sizeof hd + sizeof st + kCkptBody;
    CK(cudaMemcpy(q, h->ws + h->oU, hd.spec_bytes, cudaMemcpyDeviceToHost), "save u_hat");
    CK(cudaMemcpy(q + hd.spec_bytes, h->ws + h->oH, hd.spec_bytes, cudaMemcpyDeviceToHost), "save history");
    return FLUSI_OK;
}

int flusi_load(flusi_t h, const void* host_buf, size_t bytes)
{
    size_t need = 0;
    if (!h || !host_buf) return fail(h, FLUSI_EINVAL, "NULL argument");
    flusi_checkpoint_bytes(h, &need);
    if (bytes < need) return fail(h, FLUSI_EINVAL, "checkpoint buffer too small");
    const char* p = static_cast<const char*>(host_buf);
    CkptHeader hd, mine = make_header(h);
    std::memcpy(&hd, p, sizeof hd);
    if (std::memcmp(hd.magic, mine.magic, 8) != 0) return fail(h, FLUSI_EINVAL, "not a flusi checkpoint");
    if (hd.prec != mine.prec || hd.nx != mine.nx || hd.ny != mine.ny || hd.nz != mine.nz ||
        hd.Mx != mine.Mx || hd.My != mine.My || hd.Mz != mine.Mz || hd.Mxp != mine.Mxp ||
        hd.dealias_strict != mine.dealias_strict || hd.nu != mine.nu || hd.eta != mine.eta ||
        hd.L[0] != mine.L[0] || hd.L[1] != mine.L[1] || hd.L[2] != mine.L[2])
        return fail(h, FLUSI_EINVAL, "checkpoint of another grid, box, nu, eta, precision or 2/3 rule");
    int rc = check_ready(h, false);
    if (rc) return rc;
    StepState st;
    std::memcpy(&st, p + sizeof hd, sizeof st);
    if (st.status != 0 || st.n < 0) return fail(h, FLUSI_EINVAL, "checkpoint holds a failed or invalid state");
    double body[16];
    std::memcpy(body, p + sizeof hd + sizeof st, kCkptBody);
    const char* q = p + sizeof hd + sizeof st + kCkptBody;
    CK(cudaStreamSynchronize(h->stream), "sync before load");
    CK(cudaMemcpy(h->ws + h->ostate, &st, sizeof st, cudaMemcpyHostToDevice), "load step state");
    if (h->have_ins && h->ins.free_flight) {
        CK(write_body(h, body), "load body state");
        std::memcpy(h->ins.x_cntr, body, 3 * sizeof(double));
        std::memcpy(h->ins.u_cntr, body + 3, 3 * sizeof(double));
        std::memcpy(h->ins.quat, body + 6, 4 * sizeof(double));
        std::memcpy(h->ins.Omega_body, body + 10, 3 * sizeof(double));
    }
    CK(cudaMemcpy(h->ws + h->oU, q, hd.spec_bytes, cudaMemcpyHostToDevice), "load u_hat");
    CK(cudaMemcpy(h->ws + h->oH, q + hd.spec_bytes, hd.spec_bytes, cudaMemcpyHostToDevice), "load history");
    h->has_state = 1;
    h->poisoned = 0;
    h->rows_read = st.n;
    h->n_enq = st.n;
    return FLUSI_OK;
}

// ---------------------------------------------------------------- ensembles

struct flusi_ensemble_s {
    std::vector<flusi_t> m;
    std::vector<long long> gen;            // member generations at capture
    cudaStream_t stream = nullptr;         // the caller's stream
    cudaStream_t cap = nullptr;            // private capture origin
    cudaEvent_t fork = nullptr, done = nullptr;
    std::vector<cudaEvent_t> join, pre;
    cudaGraphExec_t gexec = nullptr;
    Member* dev_members = nullptr;         // the batched groups' member tables
    int batches = 0, batched_members = 0;  // of the captured graph
};

namespace {

int ens_fail(int code, const std::string& msg) { return fail(nullptr, code, msg); }

int ens_cuda(cudaError_t e, const char* what)
{
    return ens_fail(FLUSI_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CKE(call, what)                                 \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return ens_cuda(e_, what); \
    } while (0)

void ens_release(flusi_ensemble_t e)
{
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    if (e->dev_members) cudaFree(e->dev_members);
    if (e->cap) cudaStreamDestroy(e->cap);
    if (e->fork) cudaEventDestroy(e->fork);
    if (e->done) cudaEventDestroy(e->done);
    for (cudaEvent_t ev : e->join)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : e->pre)
        if (ev) cudaEventDestroy(ev);
    delete e;
}

// Members whose steps can run as one launch per kernel: the same grid, box,
// C_eta, precision, options (all but nu), tuning, mask shape and x-pass grid,
// with the AB2 scheme, no vorticity sponge, the CUDA-core x pass and one-CTA
// y tiles.  nu differs freely (it enters only through the scalars' tables).
bool batchable(flusi_t h)
{
    return h->opt.time_scheme == 0 && !(h->opt.sponge_c > 0) && !h->g.xtc && h->g.ypair == 0;
}

bool same_batch(flusi_t a, flusi_t b)
{
    const Geom &x = a->g, &y = b->g;
    const bool geom = x.nx == y.nx && x.ny == y.ny && x.nz == y.nz && x.Kx == y.Kx && x.Ky == y.Ky &&
                      x.Kz == y.Kz && x.Mxp == y.Mxp && x.Lx == y.Lx && x.Ly == y.Ly && x.Lz == y.Lz &&
                      x.eta == y.eta && x.ycols == y.ycols && x.zcols == y.zcols && x.xgeneric == y.xgeneric &&
                      x.ypair == y.ypair && x.xtc == y.xtc;
    const flusi_options &o = a->opt, &q = b->opt;
    bool opts = o.cfl == q.cfl && o.dt_fixed == q.dt_fixed && o.dt_max == q.dt_max && o.mean_mode == q.mean_mode &&
                o.dealias_strict == q.dealias_strict && o.force_ring == q.force_ring && o.time_scheme == q.time_scheme &&
                o.sponge_c == q.sponge_c;
    for (int i = 0; i < 3; ++i)
        opts = opts && o.u_inf[i] == q.u_inf[i] && o.layer_width[i] == q.layer_width[i] &&
               o.sponge_width[i] == q.sponge_width[i];
    return geom && opts && a->prec == b->prec && a->tune.y_plan == b->tune.y_plan &&
           a->tune.zf_plan == b->tune.zf_plan && a->xgrid == b->xgrid &&
           same_shape(make_shape(a), make_shape(b)) && box_margin(a) == box_margin(b);
}

Member member_of(flusi_t h)
{
    Member m;
    m.W = h->ws + h->oW;
    m.U = h->ws + h->oU;
    m.H = h->ws + h->oH;
    m.st = at<StepState>(h, h->ostate);
    m.coef = at<StepCoef>(h, h->ocoef);
    m.fr = at<Frame>(h, h->oframe);
    m.ins = at<flusi_insect>(h, h->oins);
    m.etab = at<double>(h, h->oetab);
    m.part = at<double>(h, h->opart);
    m.rows = at<double>(h, h->orows);
    m.nu = h->nu;
    return m;
}

// One graph: fork from the capture origin, then per group of members that
// can share launches (same_batch) one step whose launches cover the whole
// group (gridDim.z = members, each kernel taking its member's buffers from a
// device table), and for every other member one step of its own, each on its
// own capture stream; join back.
int ens_capture(flusi_ensemble_t e)
{
    const size_t M = e->m.size();
    std::vector<int> group(M, -1);
    std::vector<std::vector<int>> groups;
    for (size_t i = 0; i < M; ++i) {
        if (group[i] >= 0) continue;
        group[i] = (int)groups.size();
        groups.push_back({(int)i});
        if (!batchable(e->m[i])) continue;
        for (size_t j = i + 1; j < M; ++j)
            if (group[j] < 0 && batchable(e->m[j]) && same_batch(e->m[i], e->m[j])) {
                group[j] = group[i];
                groups.back().push_back((int)j);
            }
    }
    // the member tables of the batched groups, in one device array
    std::vector<Member> table;
    std::vector<size_t> first(groups.size(), 0);
    for (size_t k = 0; k < groups.size(); ++k) {
        first[k] = table.size();
        if (groups[k].size() > 1)
            for (int i : groups[k]) table.push_back(member_of(e->m[i]));
    }
    if (e->dev_members) {
        cudaFree(e->dev_members);
        e->dev_members = nullptr;
    }
    if (!table.empty()) {
        CKE(cudaMalloc(&e->dev_members, sizeof(Member) * table.size()), "ensemble: member tables");
        CKE(cudaMemcpy(e->dev_members, table.data(), sizeof(Member) * table.size(), cudaMemcpyHostToDevice),
            "ensemble: member tables");
    }
    cudaGraph_t graph = nullptr;
    CKE(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal), "ensemble: begin capture");
    cudaError_t err = cudaEventRecord(e->fork, e->cap);
    e->batches = e->batched_members = 0;
    for (size_t k = 0; k < groups.size() && err == cudaSuccess; ++k) {
        const int lead = groups[k][0];
        flusi_t h = e->m[lead];
        err = cudaStreamWaitEvent(h->cap_stream, e->fork, 0);
        if (err == cudaSuccess) {
            Batch& B = current_batch();
            if (groups[k].size() > 1) {
                B.mb = e->dev_members + first[k];
                B.n = (int)groups[k].size();
                ++e->batches;
                e->batched_members += B.n;
            }
            err = enqueue_step(h, h->cap_stream, nullptr);
            B = Batch{};
        }
        if (err == cudaSuccess) err = cudaEventRecord(e->join[lead], h->cap_stream);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(e->cap, e->join[lead], 0);
    }
    cudaError_t err2 = cudaStreamEndCapture(e->cap, &graph);
    if (err != cudaSuccess || err2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return ens_cuda(err != cudaSuccess ? err : err2, "ensemble: capture step");
    }
    err = cudaGraphInstantiate(&e->gexec, graph, 0);
    cudaGraphDestroy(graph);
    CKE(err, "ensemble: instantiate graph");
    for (size_t i = 0; i < e->m.size(); ++i) e->gen[i] = e->m[i]->generation;
    return FLUSI_OK;
}

}  // namespace

int flusi_ensemble_create(const flusi_t* members, int count, void* cuda_stream,
                          flusi_ensemble_t* out)
{
    if (!out) return ens_fail(FLUSI_EINVAL, "out is NULL");
    *out = nullptr;
    if (!members || count < 1 || count > FLUSI_ENSEMBLE_MAX)
        return ens_fail(FLUSI_EINVAL, "members must be 1.." + std::to_string(FLUSI_ENSEMBLE_MAX) + " handles");
    for (int i = 0; i < count; ++i) {
        if (!members[i]) return ens_fail(FLUSI_EINVAL, "member " + std::to_string(i) + " is NULL");
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i])
                return ens_fail(FLUSI_EINVAL, "member " + std::to_string(i) + " repeats member " + std::to_string(j));
    }
    for (int i = 0; i < count; ++i) {
        flusi_t h = members[i];
        if (!h->bound) return ens_fail(FLUSI_ESTATE, "member " + std::to_string(i) + " has no workspace (flusi_bind)");
        if (!h->has_state) return ens_fail(FLUSI_ESTATE, "member " + std::to_string(i) + " has no state (flusi_set_state)");
    }
    flusi_ensemble_t e = new (std::nothrow) flusi_ensemble_s;
    if (!e) return ens_fail(FLUSI_ENOMEM, "out of host memory");
    e->m.assign(members, members + count);
    e->gen.assign(count, -1);
    e->stream = (cudaStream_t)cuda_stream;
    e->join.assign(count, nullptr);
    e->pre.assign(count, nullptr);
    cudaError_t err = cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->done, cudaEventDisableTiming);
    for (int i = 0; i < count && err == cudaSuccess; ++i) {
        err = cudaEventCreateWithFlags(&e->join[i], cudaEventDisableTiming);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->pre[i], cudaEventDisableTiming);
    }
    if (err != cudaSuccess) {
        ens_release(e);
        return ens_cuda(err, "ensemble: streams and events");
    }
    *out = e;
    return FLUSI_OK;
}

int flusi_ensemble_step(flusi_ensemble_t e, int n)
{
    if (!e) return ens_fail(FLUSI_EINVAL, "ensemble is NULL");
    if (n < 0) return ens_fail(FLUSI_EINVAL, "n < 0");
    for (size_t i = 0; i < e->m.size(); ++i) {
        flusi_t h = e->m[i];
        if (!h->bound || !h->has_state)
            return ens_fail(FLUSI_ESTATE, "member " + std::to_string(i) + " is not bound or has no state");
        if (e->gexec && e->gen[i] != h->generation)
            return ens_fail(FLUSI_ESTATE, "member " + std::to_string(i) +
                                              " changed options, tuning, workspace or insect shape; create a new ensemble");
    }
    if (n == 0) return FLUSI_OK;
    if (!e->gexec) {
        int rc = ens_capture(e);
        if (rc) return rc;
    }
    // order after the members' streams, run, and order the members' streams after
    for (size_t i = 0; i < e->m.size(); ++i) {
        CKE(cudaEventRecord(e->pre[i], e->m[i]->stream), "ensemble: order after members");
        CKE(cudaStreamWaitEvent(e->stream, e->pre[i], 0), "ensemble: order after members");
    }
    for (int k = 0; k < n; ++k) CKE(cudaGraphLaunch(e->gexec, e->stream), "ensemble: graph launch");
    for (flusi_t h : e->m) h->n_enq += n;
    CKE(cudaEventRecord(e->done, e->stream), "ensemble: order members after");
    for (flusi_t h : e->m) CKE(cudaStreamWaitEvent(h->stream, e->done, 0), "ensemble: order members after");
    return FLUSI_OK;
}

int flusi_ensemble_batches(flusi_ensemble_t e, int* groups, int* members)
{
    if (!e || !groups || !members) return ens_fail(FLUSI_EINVAL, "NULL argument");
    *groups = e->batches;
    *members = e->batched_members;
    return FLUSI_OK;
}

int flusi_ensemble_destroy(flusi_ensemble_t e)
{
    if (!e) return FLUSI_OK;
    ens_release(e);
    return FLUSI_OK;
}

int flusi_destroy(flusi_t h)
{
    if (!h) return FLUSI_OK;
    drop_graph(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->side) cudaStreamDestroy(h->side);
    for (cudaEvent_t ev : {h->ev_fork, h->ev_kin, h->ev_x, h->ev_sc})
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : h->stage_ev)
        if (ev) cudaEventDestroy(ev);
    if (h->ins_stage) cudaFreeHost(h->ins_stage);
    delete h;
    return FLUSI_OK;
}

const char* flusi_last_error(flusi_t h)
{
    return h ? h->err.c_str() : g_create_err.c_str();
}

#ifndef FLUSI_SOURCE_HASH
#define FLUSI_SOURCE_HASH "unstamped"
#endif
const char* flusi_build_id(void) { return FLUSI_SOURCE_HASH; }

}  // extern "C"

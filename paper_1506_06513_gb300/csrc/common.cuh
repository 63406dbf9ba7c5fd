// Shared device types of libflusi: complex arithmetic, the grid geometry
// passed to every kernel, the per-step frame block written by the kinematics
// kernel, and the device-side step state.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstddef>

#include "../../include/flusi.h"

namespace flusi {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mkc(T r, T i)
{
    cplx<T> c;
    c.x = r;
    c.y = i;
    return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// a * i
template <typename C> __device__ __forceinline__ C cmuli(C a) { C r; r.x = -a.y; r.y = a.x; return r; }
// a * (-i)
template <typename C> __device__ __forceinline__ C cmulmi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) { a.x *= s; a.y *= s; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// Largest FFT length along any axis (the x transform runs at nx/2).
constexpr int kMaxN = 1024;
constexpr int kMaxStages = 10;
constexpr int kNumSums = 40;     // per-CTA partial sums of the physical pass
constexpr int kRowCols = 26;     // one force row

// Partial-sum slots: per colour c (0 body, 1 left, 2 right) 12 doubles:
// [0..2] sum chi (u - u_s), [3..5] sum r x chi (u - u_s),
// [6..8] sum chi u_s, [9..11] sum r x chi u_s, with r = x - x_ref the arm
// from the body centre (body) or the wing pivot (wings); all without dV.
constexpr int kSumEkin = 36;     // sum |u|^2
constexpr int kSumUmax2 = 37;    // max |u|^2
constexpr int kSumBad = 38;      // 1 if a non-finite value was met

// Radix plan of one 1-D transform (mixed radix 2, 3, 4, 8, 16; in-place
// decimation in frequency / time, see fft.cuh).
struct FftPlan {
    int n;                   // transform length
    int nst;                 // number of stages
    int radix[kMaxStages];
    int m[kMaxStages];       // butterfly span: rows b*ls + k + t*m
    int mshift[kMaxStages];  // log2(m) when m is a power of two, else -1
    int ls[kMaxStages];      // block length radix*m
    int tstep[kMaxStages];   // twiddle index step (n/ls times the table stride)
};

// Grid and spectral truncation, shared by all kernels.
struct Geom {
    int nx, ny, nz;
    int Kx, Ky, Kz;          // 2/3-rule cutoffs: kept |m| <= K
    int Mx, My, Mz;          // retained modes: Kx + 1, 2 Ky + 1, 2 Kz + 1
    int Mxp;                 // Mx padded to a multiple of 4 (row pitch of spectral rows)
    double Lx, Ly, Lz;
    double dx, dy, dz;
    double nu, eta;
    // tile and kernel choices (0: defaults): caps on the columns of a y and a
    // z tile, the shared-memory x kernel in place of the line kernel, and the
    // paired (two-CTA) y kernel where ny is even
    int ycols, zcols, xgeneric, ypair;
    // physical x pass on the tensor cores with the operands split into xtc
    // BF16 pieces (2 or 3); 0: FP32 (or FP64) arithmetic units
    int xtc;
};

// Per-step geometry of the insect, written by the kinematics kernel (FP64).
struct Frame {
    double t;
    double xc[3];            // body centre (global)
    double uc[3];            // centre velocity
    double Ob[3];            // body angular velocity (global frame)
    double Mb[9];            // global -> body frame (row major)
    double Mw[2][9];         // global -> wing frame, per wing
    double pv[2][3];         // wing pivots (global)
    double Ow[2][3];         // wing angular velocity relative to the body (global frame)
    double Oww[2][3];        // the same in the wing's own frame
    double dOww[2][3];       // its time derivative (inertial power)
    double box[3][6];        // bounding box per part: xmin xmax ymin ymax zmin zmax
    int active[3];           // part present
    int pad;
};

// Insect parameters needed per grid point (set with the kinematics).
struct Shape {
    int body_type;           // 0 none, 1 sphere, 2 ellipsoid
    int nwings;
    int profile;             // 0 cosine layer, 1 tanh layer
    int wing_shape;          // 0 plate, 1 contour R(theta)
    double h;                // smoothing half-width
    double body_a, body_b;
    double c_le, c_te, R, ht;
    double head_x0[3], head_r, eye_x0[3], eye_r;   // body frame; radius 0: absent
    int ncontour, pad;
    double contour_xc, contour_yc, contour_a0;
    double contour_a[FLUSI_MAX_CONTOUR], contour_b[FLUSI_MAX_CONTOUR];
    // body_type 3: centre-line circle (radius, centre x, z), the unit vector
    // from its centre towards the body origin, and the arc's end points (x, z)
    double arc_r, arc_x, arc_z, arc_ux, arc_uz;
    double arc_end[2][2];
};

// The frame block and mask shape in the x pass's precision T.  The kinematics
// kernel writes one per precision after the FP64 frame, at fixed offsets of
// the frame slot (frame_t), so the x-pass blocks only copy bytes.
template <typename T> struct FrameT {
    T xc[3], uc[3], Ob[3], Mb[9], Mw[2][9], pv[2][3], Ow[2][3], box[3][6];
    int active[3];
    T h, a, b, c_le, c_te, R, ht, inv_eta;
    int body_type, profile, wing_shape, ncontour;
    T head_x0[3], head_r, eye_x0[3], eye_r;
    T cxc, cyc, ca0, ca[FLUSI_MAX_CONTOUR], cb[FLUSI_MAX_CONTOUR];
    T arc_r, arc_x, arc_z, arc_ux, arc_uz, arc_end[2][2];
};

constexpr size_t align16(size_t n) { return (n + 15) / 16 * 16; }
constexpr size_t kFrameT32Off = align16(sizeof(Frame));
constexpr size_t kFrameT64Off = kFrameT32Off + align16(sizeof(FrameT<float>));
constexpr size_t kFrameSlot = kFrameT64Off + align16(sizeof(FrameT<double>));   // bytes of a frame slot

template <typename T> __host__ __device__ inline const FrameT<T>* frame_t(const Frame* f)
{
    return reinterpret_cast<const FrameT<T>*>(reinterpret_cast<const char*>(f) +
                                              (sizeof(T) == 4 ? kFrameT32Off : kFrameT64Off));
}

// Runs of T fields of FrameT that mirror runs of doubles of Frame or Shape,
// in the same order (checked below), so the lanes of a warp convert them
// with uniform code.
template <typename T> struct FrameTRuns {
    static_assert(offsetof(FrameT<T>, box) == offsetof(FrameT<T>, xc) + 48 * sizeof(T), "FrameT xc..Ow");
    static_assert(offsetof(Frame, Oww) == offsetof(Frame, xc) + 48 * sizeof(double), "Frame xc..Ow");
    static_assert(offsetof(FrameT<T>, inv_eta) == offsetof(FrameT<T>, h) + 7 * sizeof(T), "FrameT h..ht");
    static_assert(offsetof(Shape, head_x0) == offsetof(Shape, h) + 7 * sizeof(double), "Shape h..ht");
    static_assert(offsetof(FrameT<T>, cxc) == offsetof(FrameT<T>, head_x0) + 8 * sizeof(T), "FrameT head, eyes");
    static_assert(offsetof(Shape, ncontour) == offsetof(Shape, head_x0) + 8 * sizeof(double), "Shape head, eyes");
    static_assert(offsetof(FrameT<T>, arc_end) + 4 * sizeof(T) == offsetof(FrameT<T>, cxc) + 76 * sizeof(T),
                  "FrameT contour..arc");
    static_assert(sizeof(Shape) == offsetof(Shape, contour_xc) + 76 * sizeof(double), "Shape contour..arc");
};

// FrameT<T> from the frame block and the shape, by the 32 lanes of one warp
// (lane = 0..31); `F` and `S` readable by every lane.
template <typename T>
__device__ inline void frame_to_t(FrameT<T>* f, const Frame* F, const Shape* S, double inv_eta, int lane)
{
    (void)sizeof(FrameTRuns<T>);
    auto run = [&](size_t dst, const void* base, size_t src, int n) {
        T* d = reinterpret_cast<T*>(reinterpret_cast<char*>(f) + dst);
        const double* q = reinterpret_cast<const double*>(reinterpret_cast<const char*>(base) + src);
        for (int i = lane; i < n; i += 32) d[i] = T(q[i]);
    };
    run(offsetof(FrameT<T>, xc), F, offsetof(Frame, xc), 48);
    run(offsetof(FrameT<T>, box), F, offsetof(Frame, box), 18);
    run(offsetof(FrameT<T>, h), S, offsetof(Shape, h), 7);
    run(offsetof(FrameT<T>, head_x0), S, offsetof(Shape, head_x0), 8);
    run(offsetof(FrameT<T>, cxc), S, offsetof(Shape, contour_xc), 76);
    if (lane < 3) {
        const bool absent = (lane == 0 && S->body_type == 0) || (lane == 1 && S->nwings < 1) ||
                            (lane == 2 && S->nwings < 2);
        f->active[lane] = absent ? 0 : F->active[lane];
    } else if (lane == 3) {
        f->inv_eta = T(inv_eta);
        f->body_type = S->body_type;
        f->profile = S->profile;
        f->wing_shape = S->wing_shape;
        f->ncontour = S->ncontour;
    }
}

// Why a descriptor cannot be used, or nullptr (checks shared by every entry
// point that takes one; the free-flight fields are checked where they apply).
inline const char* insect_error(const flusi_insect& I)
{
    if (I.body_type < 0 || I.body_type > 3 || I.nwings < 0 || I.nwings > 2 || I.profile < 0 ||
        I.profile > 1 || I.nfourier < 0 || I.nfourier > FLUSI_MAX_FOURIER || !(I.c_smth > 0))
        return "bad insect descriptor (body_type, nwings, profile, nfourier or c_smth)";
    if ((I.body_type == 1 && !(I.body_a > 0)) || (I.body_type >= 2 && !(I.body_a > 0 && I.body_b > 0)))
        return "bad insect descriptor (body axes)";
    if (I.body_type == 3) {
        const double pi = 3.141592653589793238462643383279;
        const double d = std::sqrt(I.body_arc[1] * I.body_arc[1] + I.body_arc[2] * I.body_arc[2]);
        if (!(I.body_arc[0] > I.body_b) || !(I.body_a < pi * I.body_arc[0]) || !(d > 0) || !std::isfinite(d))
            return "bad insect descriptor (body_arc: need body_b < radius, body_a < pi radius, "
                   "centre away from the body origin)";
    }
    if (!(I.head_r >= 0) || !(I.eye_r >= 0) || I.wing_shape < 0 || I.wing_shape > 1 || I.ncontour < 0 ||
        I.ncontour > FLUSI_MAX_CONTOUR || (I.wing_shape == 1 && !(I.contour_a0 > 0)))
        return "bad insect descriptor (head, eyes or wing outline)";
    return nullptr;
}

// Mask shape of an insect descriptor with smoothing half-width h.
inline Shape shape_of(const flusi_insect& I, double h)
{
    Shape s{};
    s.body_type = I.body_type;
    s.nwings = I.nwings;
    s.profile = I.profile;
    s.wing_shape = I.wing_shape;
    s.h = h;
    s.body_a = I.body_a;
    s.body_b = I.body_b;
    s.c_le = I.wing_c_le;
    s.c_te = I.wing_c_te;
    s.R = I.wing_R;
    s.ht = I.wing_h;
    for (int i = 0; i < 3; ++i) {
        s.head_x0[i] = I.head_x0[i];
        s.eye_x0[i] = I.eye_x0[i];
    }
    s.head_r = I.head_r;
    s.eye_r = I.eye_r;
    s.ncontour = I.ncontour;
    s.contour_xc = I.contour_xc;
    s.contour_yc = I.contour_yc;
    s.contour_a0 = I.contour_a0;
    for (int i = 0; i < FLUSI_MAX_CONTOUR; ++i) {
        s.contour_a[i] = i < I.ncontour ? I.contour_a[i] : 0.0;
        s.contour_b[i] = i < I.ncontour ? I.contour_b[i] : 0.0;
    }
    if (I.body_type == 3) {
        s.arc_r = I.body_arc[0];
        s.arc_x = I.body_arc[1];
        s.arc_z = I.body_arc[2];
        const double d = std::sqrt(s.arc_x * s.arc_x + s.arc_z * s.arc_z);
        s.arc_ux = -s.arc_x / d;
        s.arc_uz = -s.arc_z / d;
        // end points at the angles theta_0 -+ a / r_c about the centre
        // (angles from +z^(b) towards +x^(b))
        for (int e = 0; e < 2; ++e) {
            const double dth = (e == 0 ? -1.0 : 1.0) * I.body_a / s.arc_r;
            const double c = std::cos(dth), sn = std::sin(dth);
            // rotate (ux, uz) = (sin theta_0, cos theta_0) by dth
            const double ux = s.arc_ux * c + s.arc_uz * sn, uz = s.arc_uz * c - s.arc_ux * sn;
            s.arc_end[e][0] = s.arc_x + s.arc_r * ux;
            s.arc_end[e][1] = s.arc_z + s.arc_r * uz;
        }
    }
    return s;
}

// Device-resident step state (persists across steps).
struct StepState {
    double t;
    double dt_prev;
    long long n;             // steps taken
    int status;              // flusi_status of the first device-side failure
    int pad;
    double Is_prev[3][3];
    double Js_prev[3][3];
    double body_rhs_prev[13];   // free flight: the ODE right-hand side of the previous step
    double pad2;
};

// Coefficients of the current step, written by the scalar kernel and read by
// the spectral update.
struct StepCoef {
    double dt;
    double c_now;            // dt (1 + r/2), or dt on the first step
    double c_old;            // dt r/2, or 0 on the first step
    long long n;
    int first;
    int skip;                // 1 when the step is abandoned (status set)
    double t0;               // time at the start of the step (RK stages)
};

// One ensemble member's buffers, for launches that cover several members of
// the same grid, options and tuning at once (blockIdx.z picks the member):
// everything that differs between such members lives here.
struct Member {
    void* W;                 // work fields
    void* U;                 // state u_hat
    void* H;                 // AB2 history
    StepState* st;
    StepCoef* coef;
    Frame* fr;
    flusi_insect* ins;       // device descriptor
    double* etab;            // integrating-factor tables
    double* part;            // per-CTA partial sums of the physical pass
    double* rows;            // force-row ring
    double nu;
};

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Rows per TMA box for an inverse tile of length n that keeps modes 0..K and
// -K..-1 (rows 0..K and K..2K of the source, two parts of K + 1 rows): the
// part split into the fewest equal boxes of at most 256 rows whose
// destinations (row offsets times row_bytes) start on 128-byte boundaries;
// 0 if there is none (the pass then copies by 16 bytes).
inline int inverse_box_rows(int n, int K, size_t row_bytes)
{
    if (((size_t)(n - K - 1) * row_bytes) % 128 != 0) return 0;
    for (int k = 1; k <= 8; ++k) {
        if ((K + 1) % k != 0) continue;
        const int bh = (K + 1) / k;
        if (bh > 256) continue;
        if (k > 1 && ((size_t)bh * row_bytes) % 128 != 0) continue;
        return bh;
    }
    return 0;
}

inline bool plan_has_radix16(const FftPlan& p)
{
    for (int s = 0; s < p.nst; ++s)
        if (p.radix[s] == 16) return true;
    return false;
}

// Asynchronous global -> shared copies of one complex value (8 or 16 bytes):
// a tile's loads are all issued back to back, then waited for at once.
template <typename T>
__device__ __forceinline__ void cp_async_cplx(cplx<T>* smem_dst, const cplx<T>* gmem_src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    if (sizeof(cplx<T>) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src));
}

// 16-byte asynchronous copy (two FP32 complex values or one FP64 value).
__device__ __forceinline__ void cp_async_16(void* smem_dst, const void* gmem_src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src));
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Bulk prefetch of `bytes` (a multiple of 16) from a 16-byte aligned global
// address into L2; no completion to wait for.
__device__ __forceinline__ void prefetch_l2_bulk(const void* gmem_src, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gmem_src), "r"(bytes) : "memory");
}

// ---- TMA (cp.async.bulk.tensor) with an mbarrier, one elected thread
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous (TMA) proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// order this thread's earlier generic-proxy shared-memory accesses before the
// asynchronous proxy's (a TMA write into a buffer the block used before)
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// one 3-D box of the tensor map into shared memory (coordinates innermost first)
__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, int c0, int c1, int c2,
                                            unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of the barrier: false when it gave up after
// about 0.2 s of SM clock (each try_wait itself blocks for a short,
// hardware-bounded time).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          long long max_cycles = 400000000LL)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > max_cycles) return false;
    return true;
}

// Signed mode of a stored spectral index j in [0, M) with M = 2K + 1.
__host__ __device__ __forceinline__ int mode_of(int j, int K) { return j <= K ? j : j - (2 * K + 1); }
// FFT frequency slot of a stored index j for a length-n transform.
__host__ __device__ __forceinline__ int slot_of(int j, int K, int n) { return j <= K ? j : n - (2 * K + 1) + j; }

}  // namespace flusi

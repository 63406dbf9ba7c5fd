// Physical-space pieces of the x pass shared by its kernels: the FP64 frame
// block turned into the pass's precision, the signed distances of the
// insect's parts and the smoothed mask (Sec. 3, Eq.
// smoothing_mask_as_function_of_delta), the solid velocity (Eqs.
// body_velocity_field, wing_velocity_field), and the pre- and
// post-processing that turns a length-nx real transform into a length-nx/2
// complex one.
#pragma once

#include "kernels.cuh"

namespace flusi {
namespace {

// The block's copy of the frame in T (written by the kinematics kernel),
// by every thread of the block in 4-byte words.
template <typename T> __device__ __forceinline__ void load_frame_t(FrameT<T>* dst, const Frame* fr)
{
    static_assert(sizeof(FrameT<T>) % 4 == 0, "word copy");
    const unsigned* src = reinterpret_cast<const unsigned*>(frame_t<T>(fr));
    unsigned* d = reinterpret_cast<unsigned*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(FrameT<T>) / 4); i += blockDim.x) d[i] = src[i];
}

// The pass's copy of the frame (FP64 on the device) and mask shape in T.
template <typename T>
__device__ void setup_frame(FrameT<T>& f, const Frame& F, const Shape& S, double inv_eta)
{
    for (int i = 0; i < 3; ++i) {
        f.xc[i] = T(F.xc[i]);
        f.uc[i] = T(F.uc[i]);
        f.Ob[i] = T(F.Ob[i]);
        f.active[i] = F.active[i];
        for (int s2 = 0; s2 < 2; ++s2) {
            f.pv[s2][i] = T(F.pv[s2][i]);
            f.Ow[s2][i] = T(F.Ow[s2][i]);
        }
        for (int k = 0; k < 6; ++k) f.box[i][k] = T(F.box[i][k]);
        f.head_x0[i] = T(S.head_x0[i]);
        f.eye_x0[i] = T(S.eye_x0[i]);
    }
    for (int i = 0; i < 9; ++i) {
        f.Mb[i] = T(F.Mb[i]);
        f.Mw[0][i] = T(F.Mw[0][i]);
        f.Mw[1][i] = T(F.Mw[1][i]);
    }
    f.h = T(S.h);
    f.a = T(S.body_a);
    f.b = T(S.body_b);
    f.c_le = T(S.c_le);
    f.c_te = T(S.c_te);
    f.R = T(S.R);
    f.ht = T(S.ht);
    f.inv_eta = T(inv_eta);
    f.body_type = S.body_type;
    f.profile = S.profile;
    f.wing_shape = S.wing_shape;
    f.ncontour = S.ncontour;
    f.head_r = T(S.head_r);
    f.eye_r = T(S.eye_r);
    f.cxc = T(S.contour_xc);
    f.cyc = T(S.contour_yc);
    f.ca0 = T(S.contour_a0);
    for (int i = 0; i < FLUSI_MAX_CONTOUR; ++i) {
        f.ca[i] = T(S.contour_a[i]);
        f.cb[i] = T(S.contour_b[i]);
    }
    f.arc_r = T(S.arc_r);
    f.arc_x = T(S.arc_x);
    f.arc_z = T(S.arc_z);
    f.arc_ux = T(S.arc_ux);
    f.arc_uz = T(S.arc_uz);
    for (int e = 0; e < 2; ++e) {
        f.arc_end[e][0] = T(S.arc_end[e][0]);
        f.arc_end[e][1] = T(S.arc_end[e][1]);
    }
    if (S.body_type == 0) f.active[0] = 0;
    if (S.nwings < 1) f.active[1] = 0;
    if (S.nwings < 2) f.active[2] = 0;
}

// Signed distance of the body in its frame (Sec. 3.2): thorax (sphere,
// ellipsoid, or the ellipsoid bent along a circular arc as for the fruit fly
// of Sec. 5.3), joined with the head and eye spheres by the minimum.
template <typename T>
__device__ __forceinline__ T body_delta(const FrameT<T>& F, const T* xb)
{
    T delta;
    if (F.body_type == 1) {
        delta = sqrt(xb[0] * xb[0] + xb[1] * xb[1] + xb[2] * xb[2]) - F.a;
    } else {
        if (F.body_type == 3) {
            // arc length s of the point's angle about the circle's centre,
            // from the direction u towards the body origin; the offset from
            // the centre line in the circle's plane is r - r_c, across it y
            const T vx = xb[0] - F.arc_x, vz = xb[2] - F.arc_z;
            const T s = F.arc_r * atan2(vx * F.arc_uz - vz * F.arc_ux, vx * F.arc_ux + vz * F.arc_uz);
            if (fabs(s) <= F.a) {
                const T dr = sqrt(vx * vx + vz * vz) - F.arc_r, q = s / F.a;
                delta = sqrt(dr * dr + xb[1] * xb[1]) - F.b * sqrt(fmax(T(0), T(1) - q * q));
            } else {
                const T* e = F.arc_end[s > T(0) ? 1 : 0];
                const T ex = xb[0] - e[0], ez = xb[2] - e[1];
                delta = sqrt(ex * ex + xb[1] * xb[1] + ez * ez);
            }
        } else {
            T rr = sqrt(xb[1] * xb[1] + xb[2] * xb[2]), ax = fabs(xb[0]);
            if (ax <= F.a) {
                T q = xb[0] / F.a;
                delta = rr - F.b * sqrt(fmax(T(0), T(1) - q * q));
            } else {
                delta = sqrt(rr * rr + (ax - F.a) * (ax - F.a));
            }
        }
        if (F.head_r > T(0)) {
            const T e0 = xb[0] - F.head_x0[0], e1 = xb[1] - F.head_x0[1], e2 = xb[2] - F.head_x0[2];
            delta = fmin(delta, sqrt(e0 * e0 + e1 * e1 + e2 * e2) - F.head_r);
        }
        if (F.eye_r > T(0)) {
            for (int s = 0; s < 2; ++s) {
                const T y0 = s == 0 ? F.eye_x0[1] : -F.eye_x0[1];
                const T e0 = xb[0] - F.eye_x0[0], e1 = xb[1] - y0, e2 = xb[2] - F.eye_x0[2];
                delta = fmin(delta, sqrt(e0 * e0 + e1 * e1 + e2 * e2) - F.eye_r);
            }
        }
    }
    return delta;
}

// Signed distance of a wing in its frame (Sec. 3.4): the rectangular plate,
// or the contour R(theta) = a0/2 + sum a_i cos(i theta) + b_i sin(i theta)
// with cos, sin of i theta from the angle-addition recurrence.
template <typename T>
__device__ __forceinline__ T wing_delta(const FrameT<T>& F, const T* xw)
{
    const T dz = fabs(xw[2]) - T(0.5) * F.ht;
    if (F.wing_shape == 1) {
        const T dx = xw[0] - F.cxc, dy = xw[1] - F.cyc;
        const T r = sqrt(dx * dx + dy * dy);
        const T c1 = r > T(0) ? dx / r : T(1), s1 = r > T(0) ? dy / r : T(0);
        T R = T(0.5) * F.ca0, ci = c1, si = s1;
        for (int i = 0; i < F.ncontour; ++i) {
            R += F.ca[i] * ci + F.cb[i] * si;
            const T cn = ci * c1 - si * s1;
            si = si * c1 + ci * s1;
            ci = cn;
        }
        return fmax(dz, r - R);
    }
    return fmax(fmax(xw[0] - F.c_le, -xw[0] - F.c_te), fmax(fmax(xw[1] - F.R, -xw[1]), dz));
}

template <typename T> __device__ __forceinline__ T profile_chi(int profile, T d, T h)
{
    if (profile == 1) return T(0.5) * (T(1) - tanh(d / h));
    if (d <= -h) return T(1);
    if (d >= h) return T(0);
    return T(0.5) * (T(1) + cospi((d + h) / (T(2) * h)));
}

template <typename T>
__device__ __forceinline__ void cross3(const T* a, const T* b, T* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Mask, colour (0 fluid, 1 body, 2/3 wings) and solid velocity at X.
template <typename T>
__device__ __forceinline__ void solid_at(const FrameT<T>& F, const T* X, const bool* inrow, T& chi,
                                         int& col, T* us)
{
    chi = T(0);
    col = 0;
    us[0] = us[1] = us[2] = T(0);
    if (!(inrow[0] | inrow[1] | inrow[2])) return;
    T d[3] = {X[0] - F.xc[0], X[1] - F.xc[1], X[2] - F.xc[2]};
    if (inrow[0] && X[0] >= F.box[0][0] && X[0] <= F.box[0][1]) {
        T xb[3];
        for (int i = 0; i < 3; ++i) xb[i] = F.Mb[3 * i] * d[0] + F.Mb[3 * i + 1] * d[1] + F.Mb[3 * i + 2] * d[2];
        const T delta = body_delta(F, xb);
        T c = profile_chi(F.profile, delta, F.h);
        if (c > chi) {
            chi = c;
            col = 1;
            T w[3];
            cross3(F.Ob, d, w);
            for (int i = 0; i < 3; ++i) us[i] = F.uc[i] + w[i];
        }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (!(inrow[1 + s] && X[0] >= F.box[1 + s][0] && X[0] <= F.box[1 + s][1])) continue;
        const T* M = F.Mw[s];
        T e[3] = {X[0] - F.pv[s][0], X[1] - F.pv[s][1], X[2] - F.pv[s][2]};
        T xw[3];
        for (int i = 0; i < 3; ++i) xw[i] = M[3 * i] * e[0] + M[3 * i + 1] * e[1] + M[3 * i + 2] * e[2];
        const T delta = wing_delta(F, xw);
        T c = profile_chi(F.profile, delta, F.h);
        if (c > chi) {
            chi = c;
            col = 2 + s;
            T w[3], v[3];
            cross3(F.Ob, d, w);
            cross3(F.Ow[s], e, v);
            for (int i = 0; i < 3; ++i) us[i] = F.uc[i] + w[i] + v[i];
        }
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}


// a b + c, rounded once
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// c2r pre-processing: Z[k] = (X[k] + X*[m]) + i (X[k] - X*[m]) w^{-k} with the
// mirror value Xm = X[nh - k].
// The warp totals of 12 per-lane values in FP64, added into w[0..11]: a
// reduce-scatter over 16 slots (12 values, 4 zeros), halving the slots per
// lane at each of the xor-16, 8, 4, 2 exchanges, then one xor-1 add; lane
// 2i + 1 (bits 4..1 = i) ends with the total of slot i.  16 FP64 adds a warp
// instead of the 60 of twelve separate butterflies (FP64 is slow here).
// Every lane of the warp calls it.
template <typename T>
__device__ __forceinline__ void warp_sums12(const T* v, double* w, int lane)
{
    double d[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) d[k] = k < 12 ? double(v[k]) : 0.0;
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
        const bool up = (lane & (2 * h)) != 0;   // this lane keeps the upper half
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const double send = up ? d[k] : d[k + h];
            const double keep = up ? d[k + h] : d[k];
            d[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * h);
        }
    }
    d[0] += __shfl_xor_sync(0xffffffffu, d[0], 1);
    const int slot = (lane >> 1) & 15;
    if ((lane & 1) && slot < 12) w[slot] += d[0];
}

template <typename T>
__device__ __forceinline__ cplx<T> c2r_pre(cplx<T> Xk, cplx<T> Xm, cplx<T> wk)
{
    // s + i d conj(w) with s = Xk + conj(Xm), d = Xk - conj(Xm), as fused
    // multiply-adds: (s.x - d.y w.x + d.x w.y, s.y + d.x w.x + d.y w.y)
    const T sx = Xk.x + Xm.x, sy = Xk.y - Xm.y, dx = Xk.x - Xm.x, dy = Xk.y + Xm.y;
    return mkc<T>(fmadd(dx, wk.y, fmadd(-dy, wk.x, sx)), fmadd(dy, wk.y, fmadd(dx, wk.x, sy)));
}

// r2c post-processing: X[k] = E + w^k O, E = (Z[k] + Z*[m])/2, O = -i (Z[k] - Z*[m])/2.
template <typename T>
__device__ __forceinline__ cplx<T> r2c_post(cplx<T> Zk, cplx<T> Zm, cplx<T> wk)
{
    // with a = Zk + conj(Zm), b = Zk - conj(Zm): E + w O = (a + w (-i b)) / 2
    // = (a.x + w.x b.y + w.y b.x, a.y + w.y b.y - w.x b.x) / 2, as fused
    // multiply-adds (the halving is exact)
    const T ax = Zk.x + Zm.x, ay = Zk.y - Zm.y, bx = Zk.x - Zm.x, by = Zk.y + Zm.y;
    return mkc<T>(T(0.5) * fmadd(wk.y, bx, fmadd(wk.x, by, ax)), T(0.5) * fmadd(-wk.x, bx, fmadd(wk.y, by, ay)));
}

template <typename T, int R, int L>
__device__ __forceinline__ void sq_exchange_pre(cplx<T>* x, int j, const cplx<T>* twx)
{
    // x[t] holds X[j + L t]; on return x[t] = Z[j + L t] (c2r pre-processing).
    // The mirror nh - k of k = j + L t is element R-1-t of lane L-j for j != 0,
    // and lane 0's own element R-t (t = 0: X[nh], a dropped mode, zero).  One
    // branch-free loop serves both: lane 0 "sends itself" elements s+1 and R-s
    // where the other lanes send elements s and R-1-s.  The pairs (s, R-1-s)
    // go from the middle outwards, so every element read is still unmodified
    // (element s+1 was overwritten the iteration before: carried from there).
    const int partner = (L - j) & (L - 1);
    const bool self = j == 0;
    cplx<T> carry = x[R / 2];   // the original element s + 1
#pragma unroll
    for (int s = R / 2 - 1; s >= 0; --s) {
        const cplx<T> xs = x[s], xt = x[R - 1 - s];
        const cplx<T> up = s == 0 ? mkc<T>(0, 0) : x[s == 0 ? 0 : R - s];
        const cplx<T> sa = self ? carry : xs;   // mirror of element R-1-s
        const cplx<T> sb = self ? up : xt;      // mirror of element s
        cplx<T> a, b;
        a.x = __shfl_sync(0xffffffffu, sa.x, partner, L);
        a.y = __shfl_sync(0xffffffffu, sa.y, partner, L);
        b.x = __shfl_sync(0xffffffffu, sb.x, partner, L);
        b.y = __shfl_sync(0xffffffffu, sb.y, partner, L);
        x[s] = c2r_pre<T>(xs, b, twx[j + L * s]);
        x[R - 1 - s] = c2r_pre<T>(xt, a, twx[j + L * (R - 1 - s)]);
        carry = xs;
    }
}

}  // namespace
}  // namespace flusi

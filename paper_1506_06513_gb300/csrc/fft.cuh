// Batched 1-D FFT in shared memory: mixed-radix (2, 3, 4, 8) in-place
// Cooley-Tukey transforms of C columns of length n held as buf[row*ld + col].
//
// Radices r_0..r_{S-1} (plan order).  Stage s works on blocks of length
// Ls = n / (r_0 ... r_{s-1}); a butterfly (block b, k < m_s = Ls / r_s) owns
// rows b Ls + k + t m_s, t < r_s, so each butterfly reads and writes its own
// rows and a stage needs only one barrier.
//   fft_dif: natural order in -> digit-reversed out.  Stage s = 0..S-1:
//            R-point DFT, then output q times w_Ls^{k q}.
//   fft_dit: digit-reversed in -> natural order out.  Stage s = S-1..0:
//            input t times w_Ls^{k t}, then the R-point DFT.
// (fft_dit is the transpose of fft_dif; the DFT matrix is symmetric.)
// Frequency f = d_0 + r_0 (d_1 + r_1 (...)) sits at row pos[f] = sum_s d_s m_s.
// w = exp(-2 pi i / n) forward, exp(+2 pi i / n) inverse; unnormalized.
// The twiddle w_Ls^{k t} is tw[k t tstep_s], tstep_s = (n / Ls) * (table stride).
//
// Threads own one column (col = tid % C) and stride over its butterflies
// (P = blockDim / C threads per column).
#pragma once

#include "common.cuh"

namespace flusi {
// A row index of a transform (n <= 1024) in the blocks' shared-memory tables:
// 16 bits, so that a 1024-row tile of 64 KB, its twiddles and this table fit
// three blocks on an SM.
using rowidx_t = unsigned short;
}  // namespace flusi

namespace flusi {

// R-point DFT in registers: forward uses exp(-2 pi i/R), inverse exp(+2 pi i/R).
template <typename T, int R, bool INV> struct Dft;

template <typename T, bool INV> struct Dft<T, 2, INV> {
    __device__ __forceinline__ static void run(cplx<T>* v)
    {
        cplx<T> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <typename T, bool INV> struct Dft<T, 4, INV> {
    __device__ __forceinline__ static void run(cplx<T>* v)
    {
        cplx<T> a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        cplx<T> a2 = cadd(v[1], v[3]);
        cplx<T> d = csub(v[1], v[3]);
        cplx<T> a3 = INV ? cmuli(d) : cmulmi(d);
        v[0] = cadd(a0, a2);
        v[2] = csub(a0, a2);
        v[1] = cadd(a1, a3);
        v[3] = csub(a1, a3);
    }
};

template <typename T, bool INV> struct Dft<T, 8, INV> {
    __device__ __forceinline__ static void run(cplx<T>* v)
    {
        // even and odd 4-point transforms, recombined with w8^q
        cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
        cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
        Dft<T, 4, INV>::run(e);
        Dft<T, 4, INV>::run(o);
        const T r = T(0.70710678118654752440084436210484903928);
        // w8 = (1 -+ i)/sqrt2 ; w8^2 = -+i ; w8^3 = (-1 -+ i)/sqrt2
        cplx<T> o1, o2, o3;
        if (INV) {
            o1 = mkc<T>(r * (o[1].x - o[1].y), r * (o[1].x + o[1].y));
            o2 = cmuli(o[2]);
            o3 = mkc<T>(-r * (o[3].x + o[3].y), r * (o[3].x - o[3].y));
        } else {
            o1 = mkc<T>(r * (o[1].x + o[1].y), r * (o[1].y - o[1].x));
            o2 = cmulmi(o[2]);
            o3 = mkc<T>(r * (o[3].y - o[3].x), -r * (o[3].x + o[3].y));
        }
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

// 16-point DFT as 4 x 4: X[k1 + 4 k2] = sum_n2 w16^{n2 k1} (sum_n1 x[4 n1 + n2] w4^{n1 k1}) w4^{n2 k2}.
template <typename T, bool INV> struct Dft<T, 16, INV> {
    __device__ __forceinline__ static void run(cplx<T>* v)
    {
        // cos and sin of 2 pi k / 16, k = 0..3
        const T c1 = T(0.92387953251128675612818318939678828682);
        const T s1 = T(0.38268343236508977172845998403039886676);
        const T r = T(0.70710678118654752440084436210484903928);
        cplx<T> y[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            cplx<T> a[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
            Dft<T, 4, INV>::run(a);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = a[k1];
        }
        // y[n2][k1] *= w16^{n2 k1}; exponents 1, 2, 3, 2, 4, 6, 3, 6, 9
        const T sg = INV ? T(1) : T(-1);
        auto rot = [&](cplx<T> x, T c, T s) {   // x * (c + i sg s)
            return mkc<T>(x.x * c - sg * x.y * s, x.y * c + sg * x.x * s);
        };
        y[1][1] = rot(y[1][1], c1, s1);
        y[1][2] = rot(y[1][2], r, r);
        y[1][3] = rot(y[1][3], s1, c1);
        y[2][1] = rot(y[2][1], r, r);
        y[2][2] = INV ? cmuli(y[2][2]) : cmulmi(y[2][2]);
        y[2][3] = rot(y[2][3], -r, r);
        y[3][1] = rot(y[3][1], s1, c1);
        y[3][2] = rot(y[3][2], -r, r);
        y[3][3] = rot(y[3][3], -c1, -s1);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            cplx<T> a[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
            Dft<T, 4, INV>::run(a);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = a[k2];
        }
    }
};

template <typename T, bool INV> struct Dft<T, 3, INV> {
    __device__ __forceinline__ static void run(cplx<T>* v)
    {
        // w3 = -1/2 -+ i sqrt(3)/2
        const T s = T(0.86602540378443864676372317075293618347);
        cplx<T> t1 = cadd(v[1], v[2]);
        cplx<T> t2 = csub(v[0], cscale(t1, T(0.5)));
        cplx<T> d = cscale(csub(v[1], v[2]), s);
        cplx<T> t3 = INV ? cmuli(d) : cmulmi(d);
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    }
};

// 12-point DFT as 4 x 3: with n = n1 + 3 n2 and k = 4 k1 + k2,
// X[4 k1 + k2] = sum_n1 w3^{n1 k1} w12^{n1 k2} (sum_n2 x[n1 + 3 n2] w4^{n2 k2}).
template <typename T, bool INV> struct Dft<T, 12, INV> {
    __device__ __forceinline__ static void run(cplx<T>* v)
    {
        const T h = T(0.5), c = T(0.86602540378443864676372317075293618347);   // cos, sin of pi/6
        cplx<T> a[3][4];
#pragma unroll
        for (int n1 = 0; n1 < 3; ++n1) {
            cplx<T> b[4] = {v[n1], v[n1 + 3], v[n1 + 6], v[n1 + 9]};
            Dft<T, 4, INV>::run(b);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) a[n1][k2] = b[k2];
        }
        // a[n1][k2] *= w12^{n1 k2}: exponents 1, 2, 3 (n1 = 1) and 2, 4, 6 (n1 = 2)
        const T sg = INV ? T(1) : T(-1);
        auto rot = [&](cplx<T> x, T cr, T si) {   // x * (cr + i sg si)
            return mkc<T>(x.x * cr - sg * x.y * si, x.y * cr + sg * x.x * si);
        };
        a[1][1] = rot(a[1][1], c, h);
        a[1][2] = rot(a[1][2], h, c);
        a[1][3] = INV ? cmuli(a[1][3]) : cmulmi(a[1][3]);
        a[2][1] = rot(a[2][1], h, c);
        a[2][2] = rot(a[2][2], -h, c);
        a[2][3] = mkc<T>(-a[2][3].x, -a[2][3].y);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            cplx<T> b[3] = {a[0][k2], a[1][k2], a[2][k2]};
            Dft<T, 3, INV>::run(b);
#pragma unroll
            for (int k1 = 0; k1 < 3; ++k1) v[4 * k1 + k2] = b[k1];
        }
    }
};

// v[t] *= w^(k t) for t = 1..R-1 from the table (conjugated for the inverse):
// tw[k * step] holds w^k.
template <typename T, int R, bool INV>
__device__ __forceinline__ void twiddle_table(cplx<T>* v, const cplx<T>* tw, int kstep)
{
#pragma unroll
    for (int t = 1; t < R; ++t) {
        cplx<T> w = tw[kstep * t];
        if (INV) w.y = -w.y;
        v[t] = cmul(v[t], w);
    }
}

// V adjacent complex values of one tile row (16-byte accesses for V = 2 in FP32).
template <typename T, int V>
__device__ __forceinline__ void ld_row(const cplx<T>* p, cplx<T>* o)
{
    if constexpr (V % 2 == 0 && sizeof(T) == 4) {
#pragma unroll
        for (int c = 0; c < V; c += 2) {
            const float4 q = *reinterpret_cast<const float4*>(p + c);
            o[c] = mkc<T>(q.x, q.y);
            o[c + 1] = mkc<T>(q.z, q.w);
        }
    } else {
#pragma unroll
        for (int c = 0; c < V; ++c) o[c] = p[c];
    }
}

template <typename T, int V>
__device__ __forceinline__ void st_row(cplx<T>* p, const cplx<T>* o)
{
    if constexpr (V % 2 == 0 && sizeof(T) == 4) {
#pragma unroll
        for (int c = 0; c < V; c += 2)
            *reinterpret_cast<float4*>(p + c) = make_float4(o[c].x, o[c].y, o[c + 1].x, o[c + 1].y);
    } else {
#pragma unroll
        for (int c = 0; c < V; ++c) p[c] = o[c];
    }
}

// One stage on V adjacent columns per thread (they share the butterfly's
// addresses and twiddles).  Butterfly j of the stage: rows b*ls + k + t*m.
template <typename T, int R, bool INV, bool DIF, int V>
__device__ __forceinline__ void fft_stage(cplx<T>* buf, int ld, int col, int jt, int P, int nbf,
                                          int m, int msh, int ls, int tstep, const cplx<T>* tw)
{
    constexpr int kUnroll = V == 1 ? 2 : 1;
#pragma unroll kUnroll
    for (int j = jt; j < nbf; j += P) {
        const int b = msh >= 0 ? (j >> msh) : (j / m);
        const int k = j - b * m;
        cplx<T>* p = buf + (b * ls + k) * ld + col;
        const int step = m * ld;
        cplx<T> v[V][R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            cplx<T> r[V];
            ld_row<T, V>(p + t * step, r);
#pragma unroll
            for (int c = 0; c < V; ++c) v[c][t] = r[c];
        }
        if (DIF) {
#pragma unroll
            for (int c = 0; c < V; ++c) Dft<T, R, INV>::run(v[c]);
        }
        if (k != 0) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                cplx<T> w = tw[k * tstep * t];
                if (INV) w.y = -w.y;
#pragma unroll
                for (int c = 0; c < V; ++c) v[c][t] = cmul(v[c][t], w);
            }
        }
        if (!DIF) {
#pragma unroll
            for (int c = 0; c < V; ++c) Dft<T, R, INV>::run(v[c]);
        }
#pragma unroll
        for (int t = 0; t < R; ++t) {
            cplx<T> r[V];
#pragma unroll
            for (int c = 0; c < V; ++c) r[c] = v[c][t];
            st_row<T, V>(p + t * step, r);
        }
    }
    __syncthreads();
}

// Stages s in [s0, s1): ascending for DIF, descending for DIT.  Thread map:
// column group (threadIdx.x % (C/V)) * V, butterflies jt, jt + P, ...
// R16: the plan may hold radix-16 stages (a separate instantiation, so the
// kernels without them keep their register budget).
template <typename T, bool INV, bool DIF, int V = 1, bool R16 = false>
__device__ __forceinline__ void fft_run(cplx<T>* buf, int C, int ld, const FftPlan& plan,
                                        const cplx<T>* tw, int s0, int s1)
{
    const int G = C / V;
    const int P = blockDim.x / G;
    const int col = (threadIdx.x % G) * V;
    const int jt = threadIdx.x / G;
    for (int i = s0; i < s1; ++i) {
        const int s = DIF ? i : s0 + s1 - 1 - i;
        const int R = plan.radix[s];
        const int nbf = plan.n / R;
        const int m = plan.m[s], msh = plan.mshift[s], ls = plan.ls[s], ts = plan.tstep[s];
        if constexpr (R16) {
            if (R == 16) {
                fft_stage<T, 16, INV, DIF, V>(buf, ld, col, jt, P, nbf, m, msh, ls, ts, tw);
                continue;
            }
        }
        switch (R) {
        case 8: fft_stage<T, 8, INV, DIF, V>(buf, ld, col, jt, P, nbf, m, msh, ls, ts, tw); break;
        case 4: fft_stage<T, 4, INV, DIF, V>(buf, ld, col, jt, P, nbf, m, msh, ls, ts, tw); break;
        case 3: fft_stage<T, 3, INV, DIF, V>(buf, ld, col, jt, P, nbf, m, msh, ls, ts, tw); break;
        default: fft_stage<T, 2, INV, DIF, V>(buf, ld, col, jt, P, nbf, m, msh, ls, ts, tw); break;
        }
    }
}

// Natural order in, digit-reversed out (row pos[f] holds frequency/point f).
// Columns 0..C-1, C must divide blockDim.x; all threads must call.
template <typename T, bool INV>
__device__ void fft_dif(cplx<T>* buf, int C, int ld, const FftPlan& plan, const cplx<T>* tw,
                        int s0 = 0, int s1 = -1)
{
    fft_run<T, INV, true>(buf, C, ld, plan, tw, s0, s1 < 0 ? plan.nst : s1);
}

// Digit-reversed in (row pos[f] holds f), natural order out.
template <typename T, bool INV>
__device__ void fft_dit(cplx<T>* buf, int C, int ld, const FftPlan& plan, const cplx<T>* tw,
                        int s0 = 0, int s1 = -1)
{
    fft_run<T, INV, false>(buf, C, ld, plan, tw, s0, s1 < 0 ? plan.nst : s1);
}

// ---------------------------------------------------------------------------
// Column transforms with their first stage fed from registers loaded by a
// functor and (optionally) their last stage handing results to a functor, so
// the tile goes through shared memory only between stages.  V adjacent
// columns per thread (the map of fft_run):
//   load(row, out[V])   input row `row` (natural order) of this thread's columns
//   store(f, in[V])     output frequency f of this thread's columns

// DIF stage 0: butterfly j takes rows j + m t (m = n / R) and, after the
// twiddles w^{j t}, leaves them where fft_stage would.
template <typename T, int R, bool INV, int V, class Load>
__device__ __forceinline__ void fft_stage_first(cplx<T>* buf, int ld, int col, int jt, int P, int m,
                                                int tstep, const cplx<T>* tw, Load& load)
{
    constexpr int kUnroll = V == 1 ? 2 : 1;
#pragma unroll kUnroll
    for (int j = jt; j < m; j += P) {
        cplx<T> v[V][R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            cplx<T> r[V];
            load(j + t * m, r);
#pragma unroll
            for (int c = 0; c < V; ++c) v[c][t] = r[c];
        }
#pragma unroll
        for (int c = 0; c < V; ++c) Dft<T, R, INV>::run(v[c]);
        if (j != 0) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                cplx<T> w = tw[j * tstep * t];
                if (INV) w.y = -w.y;
#pragma unroll
                for (int c = 0; c < V; ++c) v[c][t] = cmul(v[c][t], w);
            }
        }
        cplx<T>* p = buf + j * ld + col;
#pragma unroll
        for (int t = 0; t < R; ++t) {
            cplx<T> r[V];
#pragma unroll
            for (int c = 0; c < V; ++c) r[c] = v[c][t];
            st_row<T, V>(p + t * m * ld, r);
        }
    }
    __syncthreads();
}

// DIF last stage (span 1, no twiddles): butterfly j holds rows j R + t, which
// are frequencies f0 + t fstep with f0 the frequency of row j R and fstep = n / R.
// With AUX the store is an object that also takes one side-input row per
// output (store.aux(f, a) reads it, store.put(f, v, a) writes); the side rows
// of the first half of a butterfly's outputs are read before its DFT, so
// their latency overlaps it, those of the second half after the first puts
// (half the registers of holding all R).
template <typename T, int R, bool INV, int V, bool AUX, class Store>
__device__ __forceinline__ void fft_stage_last(const cplx<T>* buf, int ld, int col, int jt, int P,
                                               int nbf, int fstep, const rowidx_t* sinv, Store& store)
{
    constexpr int kUnroll = V == 1 ? 2 : 1;
    constexpr int H = AUX ? (R + 1) / 2 : 1;
#pragma unroll kUnroll
    for (int j = jt; j < nbf; j += P) {
        const int f0 = sinv[j * R];
        cplx<T> a[H][V];
        if constexpr (AUX) {
#pragma unroll
            for (int t = 0; t < H; ++t) store.aux(f0 + t * fstep, a[t]);
        }
        cplx<T> v[V][R];
        const cplx<T>* p = buf + j * R * ld + col;
#pragma unroll
        for (int t = 0; t < R; ++t) {
            cplx<T> r[V];
            ld_row<T, V>(p + t * ld, r);
#pragma unroll
            for (int c = 0; c < V; ++c) v[c][t] = r[c];
        }
#pragma unroll
        for (int c = 0; c < V; ++c) Dft<T, R, INV>::run(v[c]);
#pragma unroll
        for (int t = 0; t < R; ++t) {
            cplx<T> r[V];
#pragma unroll
            for (int c = 0; c < V; ++c) r[c] = v[c][t];
            if constexpr (AUX) {
                if (t == H) {
#pragma unroll
                    for (int u = 0; u < H && H + u < R; ++u) store.aux(f0 + (H + u) * fstep, a[u]);
                }
                store.put(f0 + t * fstep, r, a[t % H]);
            } else {
                store(f0 + t * fstep, r);
            }
        }
    }
}

template <typename T, bool INV, int V, bool AUX = false, bool R16 = false, class Store>
__device__ __forceinline__ void fft_last_to(const cplx<T>* buf, int ld, int col, int jt, int P,
                                            const FftPlan& plan, const rowidx_t* sinv, Store& store)
{
    const int last = plan.nst - 1;
    const int R = plan.radix[last], nbf = plan.n / R, fstep = plan.n / R;
    if constexpr (R16) {
        if (R == 16) {
            fft_stage_last<T, 16, INV, V, AUX>(buf, ld, col, jt, P, nbf, fstep, sinv, store);
            return;
        }
    }
    switch (R) {
    case 8: fft_stage_last<T, 8, INV, V, AUX>(buf, ld, col, jt, P, nbf, fstep, sinv, store); break;
    case 4: fft_stage_last<T, 4, INV, V, AUX>(buf, ld, col, jt, P, nbf, fstep, sinv, store); break;
    case 3: fft_stage_last<T, 3, INV, V, AUX>(buf, ld, col, jt, P, nbf, fstep, sinv, store); break;
    default: fft_stage_last<T, 2, INV, V, AUX>(buf, ld, col, jt, P, nbf, fstep, sinv, store); break;
    }
}

// Stage 0 from `load`, the middle stages in shared memory, the last stage to
// `store` (sinv[row] = frequency held by that row).  All threads must call.
template <typename T, bool INV, int V, bool AUX = false, bool R16 = false, class Load, class Store>
__device__ void fft_dif_io(cplx<T>* buf, int C, int ld, const FftPlan& plan, const cplx<T>* tw,
                           const rowidx_t* sinv, Load load, Store store)
{
    const int G = C / V, P = blockDim.x / G, col = (threadIdx.x % G) * V, jt = threadIdx.x / G;
    const int m = plan.m[0], ts = plan.tstep[0];
    if (R16 && plan.radix[0] == 16) {
        if constexpr (R16) fft_stage_first<T, 16, INV, V>(buf, ld, col, jt, P, m, ts, tw, load);
    } else
    switch (plan.radix[0]) {
    case 8: fft_stage_first<T, 8, INV, V>(buf, ld, col, jt, P, m, ts, tw, load); break;
    case 4: fft_stage_first<T, 4, INV, V>(buf, ld, col, jt, P, m, ts, tw, load); break;
    case 3: fft_stage_first<T, 3, INV, V>(buf, ld, col, jt, P, m, ts, tw, load); break;
    default: fft_stage_first<T, 2, INV, V>(buf, ld, col, jt, P, m, ts, tw, load); break;
    }
    const int last = plan.nst - 1;
    if (last == 0) {   // a one-stage transform is in natural order already
        for (int f = jt; f < plan.n; f += P) {
            cplx<T> r[V];
            ld_row<T, V>(buf + f * ld + col, r);
            if constexpr (AUX) {
                cplx<T> a[V];
                store.aux(f, a);
                store.put(f, r, a);
            } else {
                store(f, r);
            }
        }
        return;
    }
    fft_run<T, INV, true, V, R16>(buf, C, ld, plan, tw, 1, last);
    fft_last_to<T, INV, V, AUX, R16>(buf, ld, col, jt, P, plan, sinv, store);
}

// All stages but the last in shared memory (input tile in natural order), the
// last stage to `store`.  All threads must call.
template <typename T, bool INV, int V, bool AUX = false, bool R16 = false, class Store>
__device__ void fft_dif_out(cplx<T>* buf, int C, int ld, const FftPlan& plan, const cplx<T>* tw,
                            const rowidx_t* sinv, Store store)
{
    const int G = C / V, P = blockDim.x / G, col = (threadIdx.x % G) * V, jt = threadIdx.x / G;
    fft_run<T, INV, true, V, R16>(buf, C, ld, plan, tw, 0, plan.nst - 1);
    fft_last_to<T, INV, V, AUX, R16>(buf, ld, col, jt, P, plan, sinv, store);
}

// Inverse digit-reversal table in shared memory: sinv[pos[f]] = f.
__device__ __forceinline__ void load_inverse_pos(rowidx_t* sinv, const int* pos_src, int n)
{
    for (int f = threadIdx.x; f < n; f += blockDim.x) sinv[pos_src[f]] = (rowidx_t)f;
}

// Copy the twiddle table (global; ntw entries exp(-2 pi i j / ntw) in FP64,
// followed by the same ntw entries in FP32, read by the FP32 kernels) and the
// n-entry digit-reversal table into shared memory.
template <typename T>
__device__ __forceinline__ void load_tables(cplx<T>* dst, int* pos_dst, const double2* src,
                                            const int* pos_src, int ntw, int n)
{
    if constexpr (sizeof(T) == 4) {
        const float2* f = reinterpret_cast<const float2*>(src + ntw);
        for (int i = threadIdx.x; i < ntw; i += blockDim.x) dst[i] = mkc<T>(f[i].x, f[i].y);
    } else {
        for (int i = threadIdx.x; i < ntw; i += blockDim.x) {
            double2 w = src[i];
            dst[i] = mkc<T>(T(w.x), T(w.y));
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) pos_dst[i] = pos_src[i];
}

}  // namespace flusi

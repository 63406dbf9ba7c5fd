// x-axis pass: real-to-complex and complex-to-real transforms along x, fused
// with the physical-space work of Algorithm 1 step c.
//
// A tile is RB consecutive (z, y) rows.  Each real line of length nx is
// transformed through a complex transform of length nh = nx/2 on
// z[p] = x[2p] + i x[2p+1]:
//   c2r: Z[k] = (X[k] + X*[nh-k]) + i (X[k] - X*[nh-k]) w^{-k},  z = iFFT_nh(Z)
//   r2c: X[k] = E + w^k O,  E = (Z[k] + Z*[nh-k])/2,  O = -i (Z[k] - Z*[nh-k])/2
// with w = exp(-2 pi i / nx); only the kept x-modes k < Mx are read/written.
//
// XP_PHYS, per grid point (Sec. 2.1, Sec. 3):
//   chi, colour, u_s from the body and wing signed distances (Eq.
//   smoothing_mask_as_function_of_delta), u_s = u_b + Omega_w x (x - x_pivot)
//   (Eqs. body_velocity_field, wing_velocity_field), and
//   NL = u x omega - chi/C_eta (u - u_s)  (Eq. PNST_org_momentum),
//   plus FP64 partial sums of chi (u - u_s), r x chi (u - u_s), chi u_s,
//   r x chi u_s per colour, |u|^2, max |u|^2 and a non-finite flag.
// The grid is persistent (a multiple of the SM count); each CTA writes one
// row of partial sums, reduced in a fixed order by the scalar kernel.
#include <algorithm>
#include <mutex>
#include <utility>

#include "fft.cuh"
#include "kernels.cuh"
#include "xphys.cuh"

namespace flusi {

namespace {

constexpr int kThreadsX = 192;
constexpr int kWarpsX = kThreadsX / 32;
// complex elements per tile: 48 KiB of shared memory
template <typename T> constexpr int tile_elems() { return sizeof(T) == 4 ? 6144 : 3072; }

// The first inverse (DIF) stage of the length-nh transforms fused with the
// c2r pre-processing.  Stage 0 has butterflies j < m0 on rows j + m0 t; the
// mirror rows nh - (j + m0 t) belong to butterfly m0 - j, so one thread takes
// the pair (j, m0 - j) and reads only rows k < Mx (the kept modes; buf rows
// beyond Mx are not read).  tws is the length-nx table w^k = exp(-2 pi i k/nx).
template <typename T, int R>
__device__ __forceinline__ void x_first_inverse(cplx<T>* buf, int C, int ld, int Mx,
                                                const FftPlan& plan, const cplx<T>* tws)
{
    const int m0 = plan.m[0], ts = plan.tstep[0];
    const int npairs = m0 / 2 + 1;
    for (int i = threadIdx.x; i < C * npairs; i += blockDim.x) {
        const int col = i / npairs, j = i - col * npairs;
        const int jp = m0 - j;
        const bool two = (jp != j) && (jp < m0);
        cplx<T> xj[R], xp[R], a[R], b[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int k = j + m0 * t;
            xj[t] = k < Mx ? buf[k * ld + col] : mkc<T>(0, 0);
            const int kp = jp + m0 * t;
            xp[t] = (two && kp < Mx) ? buf[kp * ld + col] : mkc<T>(0, 0);
        }
        if (j == 0) xj[0].y = T(0);   // a real line has a real mean
#pragma unroll
        for (int t = 0; t < R; ++t) {
            cplx<T> xm;
            if (j == 0) xm = t == 0 ? mkc<T>(0, 0) : xj[R - t];
            else xm = two ? xp[R - 1 - t] : xj[R - 1 - t];
            a[t] = c2r_pre<T>(xj[t], xm, tws[j + m0 * t]);
            b[t] = c2r_pre<T>(xp[t], xj[R - 1 - t], tws[(two ? jp : 0) + m0 * t]);
        }
        Dft<T, R, true>::run(a);
        if (j != 0) twiddle_table<T, R, true>(a, tws, j * ts);
#pragma unroll
        for (int q = 0; q < R; ++q) buf[(j + m0 * q) * ld + col] = a[q];
        if (two) {
            Dft<T, R, true>::run(b);
            twiddle_table<T, R, true>(b, tws, jp * ts);
#pragma unroll
            for (int q = 0; q < R; ++q) buf[(jp + m0 * q) * ld + col] = b[q];
        }
    }
    __syncthreads();
}

// The last forward (DIT) stage fused with the r2c post-processing and the
// store of the kept x-modes (zeros in the row padding Mx..Mxp-1).
template <typename T, int R>
__device__ __forceinline__ void x_last_forward(const cplx<T>* buf, int C, int ld, int Mx, int Mxp,
                                               const FftPlan& plan, const cplx<T>* tws,
                                               cplx<T>* W, int comp0, int lgRB, int row0,
                                               int nrows)
{
    const int m0 = plan.m[0], ts = plan.tstep[0];
    const int npairs = m0 / 2 + 1;
    const int RB = 1 << lgRB;
    for (int i = threadIdx.x; i < C * npairs; i += blockDim.x) {
        const int col = i / npairs, j = i - col * npairs;
        const int f = col >> lgRB, r = row0 + (col & (RB - 1));
        if (r >= nrows) continue;
        const int jp = m0 - j;
        const bool two = (jp != j) && (jp < m0);
        cplx<T> a[R], b[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            a[t] = buf[(j + m0 * t) * ld + col];
            b[t] = two ? buf[(jp + m0 * t) * ld + col] : mkc<T>(0, 0);
        }
        if (j != 0) twiddle_table<T, R, false>(a, tws, j * ts);
        Dft<T, R, false>::run(a);
        if (two) {
            twiddle_table<T, R, false>(b, tws, jp * ts);
            Dft<T, R, false>::run(b);
        }
        cplx<T>* out = W + ((size_t)(comp0 + f) * nrows + r) * Mxp;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int k = j + m0 * q;
            if (k < Mxp) {
                cplx<T> zm;
                if (j == 0) zm = q == 0 ? a[0] : a[R - q];
                else zm = two ? b[R - 1 - q] : a[R - 1 - q];
                out[k] = k < Mx ? r2c_post<T>(a[q], zm, tws[k]) : mkc<T>(0, 0);
            }
            if (two) {
                const int kp = jp + m0 * q;
                if (kp < Mxp) out[kp] = kp < Mx ? r2c_post<T>(b[q], a[R - 1 - q], tws[kp]) : mkc<T>(0, 0);
            }
        }
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void x_first_inverse_any(cplx<T>* buf, int C, int ld, int Mx,
                                                    const FftPlan& plan, const cplx<T>* tws)
{
    switch (plan.radix[0]) {
    case 8: x_first_inverse<T, 8>(buf, C, ld, Mx, plan, tws); break;
    case 4: x_first_inverse<T, 4>(buf, C, ld, Mx, plan, tws); break;
    case 3: x_first_inverse<T, 3>(buf, C, ld, Mx, plan, tws); break;
    default: x_first_inverse<T, 2>(buf, C, ld, Mx, plan, tws); break;
    }
}

template <typename T>
__device__ __forceinline__ void x_last_forward_any(const cplx<T>* buf, int C, int ld, int Mx,
                                                   int Mxp, const FftPlan& plan,
                                                   const cplx<T>* tws, cplx<T>* W, int comp0,
                                                   int lgRB, int row0, int nrows)
{
    switch (plan.radix[0]) {
    case 8: x_last_forward<T, 8>(buf, C, ld, Mx, Mxp, plan, tws, W, comp0, lgRB, row0, nrows); break;
    case 4: x_last_forward<T, 4>(buf, C, ld, Mx, Mxp, plan, tws, W, comp0, lgRB, row0, nrows); break;
    case 3: x_last_forward<T, 3>(buf, C, ld, Mx, Mxp, plan, tws, W, comp0, lgRB, row0, nrows); break;
    default: x_last_forward<T, 2>(buf, C, ld, Mx, Mxp, plan, tws, W, comp0, lgRB, row0, nrows); break;
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreadsX, sizeof(T) == 4 ? 3 : 1)
k_xpass(cplx<T>* __restrict__ W, Geom g, FftPlan plan, const double2* __restrict__ tw,
        const int* __restrict__ pos, XExtra ex, int lgRB, const StepState* __restrict__ st,
        const Member* __restrict__ mb)
{
    if (mb) {   // one member of an ensemble batch
        const Member& m = mb[blockIdx.z];
        W = static_cast<cplx<T>*>(m.W);
        st = m.st;
        ex.frame = m.fr;
        ex.part = m.part;
    }
    if (st && st->status != 0) return;
    constexpr bool kPhys = (MODE == XP_PHYS || MODE == XP_DUMP);
    const int RB = 1 << lgRB;
    const int NF = kPhys ? 6 : ex.ncomp;
    const int C = NF * RB;
    const int ld = C | 1;
    const int nh = g.nx / 2, nx = g.nx;
    const int nrows = g.nz * g.ny;
    const int ntiles = ceil_div(nrows, RB);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* wacc = reinterpret_cast<double*>(smem_raw);                    // [warps][36]
    FrameT<T>* Fs = reinterpret_cast<FrameT<T>*>(wacc + kWarpsX * 36);
    cplx<T>* tws = reinterpret_cast<cplx<T>*>(
        reinterpret_cast<unsigned char*>(Fs) + ((sizeof(FrameT<T>) + 15) / 16) * 16);
    cplx<T>* buf = tws + nx;
    int* spos = reinterpret_cast<int*>(buf + (size_t)nh * ld);
    int* ipos = spos + nh;                       // row -> point pair p (inverse of pos)

    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    load_tables<T>(tws, spos, tw, pos, nx, nh);
    if (kPhys) {
        for (int i = tid; i < kWarpsX * 36; i += kThreadsX) wacc[i] = 0.0;
        load_frame_t<T>(Fs, ex.frame);
    }
    __syncthreads();
    for (int p = tid; p < nh; p += kThreadsX) ipos[spos[p]] = p;
    __syncthreads();

    __shared__ int rowmask[32];     // per tile row: bit q set if part q's box meets the row
    double e_acc = 0.0;             // FP64 across tiles; FP32 partials within a tile
    T m_acc = T(0);                 // max |u|^2 (a max is exact in any precision)
    int bad = 0;
    const T dxT = T(g.dx), dyT = T(g.dy), dzT = T(g.dz);

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row0 = tile * RB;
        if (kPhys && tid < RB) {
            const int r = row0 + tid;
            int mask = 0;
            if (r < nrows) {
                const FrameT<T>& F = *Fs;
                const int z = r / g.ny, y = r - z * g.ny;
                const T Y = T(y) * dyT, Z = T(z) * dzT;
                for (int q = 0; q < 3; ++q)
                    if (F.active[q] && Y >= F.box[q][2] && Y <= F.box[q][3] && Z >= F.box[q][4] &&
                        Z <= F.box[q][5])
                        mask |= 1 << q;
            }
            rowmask[tid] = mask;
        }

        // ---- load: spectral rows -> Z (c2r input) or real rows -> z (r2c input)
        if (MODE == XP_R2C) {
            for (int i = tid; i < C * nh; i += kThreadsX) {
                const int col = i / nh, p = i - col * nh;
                const int f = col >> lgRB, r = row0 + (col & (RB - 1));
                cplx<T> z = mkc<T>(0, 0);
                if (r < nrows) {
                    const long long o = f * ex.cstride + (long long)r * nx + 2 * p;
                    if (ex.real_fp64) {
                        const double* s = (const double*)ex.rin;
                        z = mkc<T>(T(s[o]), T(s[o + 1]));
                    } else {
                        const float* s = (const float*)ex.rin;
                        z = mkc<T>(T(s[o]), T(s[o + 1]));
                    }
                }
                buf[spos[p] * ld + col] = z;
            }
        } else {
            // kept x-modes of each row straight into column (field, row) of buf
            const int Mx = g.Mx;
            for (int i = tid; i < C * Mx; i += kThreadsX) {
                const int col = i / Mx, k = i - col * Mx;
                const int f = col >> lgRB, r = row0 + (col & (RB - 1));
                if (r < nrows)
                    cp_async_cplx<T>(buf + k * ld + col,
                                     W + ((size_t)(ex.comp0 + f) * nrows + r) * g.Mxp + k);
                else
                    buf[k * ld + col] = mkc<T>(0, 0);
            }
            cp_async_wait_all();
        }
        __syncthreads();

        if (MODE != XP_R2C) {                 // z[p] ends at row pos[p]
            x_first_inverse_any<T>(buf, C, ld, g.Mx, plan, tws);
            fft_dif<T, true>(buf, C, ld, plan, tws, 1, plan.nst);
        }

        if (MODE == XP_SPONGE) {
            // chi_sp omega (Sec. 2.3): keep the points of the sponge slabs
            for (int i = tid; i < C * nh; i += kThreadsX) {
                const int row = i / C, col = i - row * C;
                const int r = row0 + (col & (RB - 1));
                const int p = ipos[row];
                const int z = r / g.ny, y = r - z * g.ny;
                const bool in_row = y >= ex.sponge0[1] || z >= ex.sponge0[2];
                cplx<T>& b = buf[row * ld + col];
                b.x = (in_row || 2 * p >= ex.sponge0[0]) ? b.x : T(0);
                b.y = (in_row || 2 * p + 1 >= ex.sponge0[0]) ? b.y : T(0);
            }
            __syncthreads();
        }


        if (MODE == XP_C2R) {
            for (int i = tid; i < C * nh; i += kThreadsX) {
                const int col = i / nh, p = i - col * nh;
                const int f = col >> lgRB, r = row0 + (col & (RB - 1));
                if (r >= nrows) continue;
                const cplx<T> z = buf[spos[p] * ld + col];
                const long long o = f * ex.cstride + (long long)r * nx + 2 * p;
                if (ex.real_fp64) {
                    double* d = (double*)ex.rout;
                    d[o] = double(z.x);
                    d[o + 1] = double(z.y);
                } else {
                    float* d = (float*)ex.rout;
                    d[o] = float(z.x);
                    d[o + 1] = float(z.y);
                }
            }
            __syncthreads();
            continue;
        }

        if (kPhys) {
            const FrameT<T>& F = *Fs;
            const int items = RB * nh;
            const int niter = ceil_div(items, kThreadsX);
            T e_tile = T(0);
            for (int it = 0; it < niter; ++it) {
                // consecutive lanes take consecutive buffer rows (conflict-free);
                // row holds the point pair p = ipos[row] after the inverse transform
                const int i = tid + it * kThreadsX;
                const int rr = i / nh, row = i - rr * nh;
                const bool valid = (i < items) && (row0 + rr < nrows);
                const int p = valid ? ipos[row] : 0;
                const int r = row0 + rr;
                const int mask = valid ? rowmask[rr] : 0;
                T nl[2][3], chi2[2] = {T(0), T(0)}, us2[2][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
                int colr[2] = {0, 0};
                T u[2][3], om[2][3], X[2][3];
                if (valid) {
                    const int z = r / g.ny, y = r - z * g.ny;
                    const T Y = T(y) * dyT, Z = T(z) * dzT;
                    cplx<T> uv[3], wv[3];
                    for (int c = 0; c < 3; ++c) {
                        uv[c] = buf[row * ld + c * RB + rr];
                        wv[c] = buf[row * ld + (3 + c) * RB + rr];
                    }
                    for (int h = 0; h < 2; ++h) {
                        for (int c = 0; c < 3; ++c) {
                            u[h][c] = h ? uv[c].y : uv[c].x;
                            om[h][c] = h ? wv[c].y : wv[c].x;
                        }
                        X[h][0] = T(2 * p + h) * dxT;
                        X[h][1] = Y;
                        X[h][2] = Z;
                        if (mask != 0) {
                            const bool inrow[3] = {(mask & 1) != 0, (mask & 2) != 0, (mask & 4) != 0};
                            solid_at(F, X[h], inrow, chi2[h], colr[h], us2[h]);
                        }
                        T lamb[3];
                        cross3(u[h], om[h], lamb);
                        const T pen = chi2[h] * F.inv_eta;
                        // Dirichlet layer u = u_inf (Sec. 2.3), penalized with C_eta
                        const bool lay = y >= ex.layer0[1] || z >= ex.layer0[2] || 2 * p + h >= ex.layer0[0];
                        T uu = T(0);
                        for (int c = 0; c < 3; ++c) {
                            nl[h][c] = lamb[c] - pen * (u[h][c] - us2[h][c]);
                            if (lay) nl[h][c] -= F.inv_eta * (u[h][c] - T(ex.u_inf[c]));
                            uu += u[h][c] * u[h][c];
                            if (!isfinite(nl[h][c]) || !isfinite(u[h][c])) bad = 1;
                        }
                        e_tile += uu;
                        m_acc = fmax(m_acc, uu);
                    }
                    if (MODE == XP_DUMP) {
                        T* out = (T*)ex.rout;
                        const long long Nn = (long long)nrows * nx;
                        for (int h = 0; h < 2; ++h) {
                            const long long o = (long long)r * nx + 2 * p + h;
                            for (int c = 0; c < 3; ++c) {
                                out[c * Nn + o] = u[h][c];
                                out[(3 + c) * Nn + o] = om[h][c];
                                out[(8 + c) * Nn + o] = us2[h][c];
                                out[(11 + c) * Nn + o] = nl[h][c];
                            }
                            out[6 * Nn + o] = chi2[h];
                            out[7 * Nn + o] = T(colr[h]);
                        }
                    } else {
                        for (int c = 0; c < 3; ++c)
                            buf[row * ld + c * RB + rr] = mkc<T>(nl[0][c], nl[1][c]);
                    }
                }
                // penalization sums per colour, only in warps whose rows meet a part
                if (MODE == XP_PHYS && __any_sync(0xffffffffu, mask != 0)) {
                    for (int cc = 0; cc < 3; ++cc) {
                        const bool has = valid && (colr[0] == cc + 1 || colr[1] == cc + 1);
                        if (!__any_sync(0xffffffffu, has)) continue;
                        T v[12];   // this lane's contribution, in T
                        for (int k = 0; k < 12; ++k) v[k] = T(0);
                        if (has) {
                            for (int h = 0; h < 2; ++h) {
                                if (colr[h] != cc + 1) continue;
                                const T* ref = cc == 0 ? F.xc : F.pv[cc - 1];
                                T rv[3] = {X[h][0] - ref[0], X[h][1] - ref[1], X[h][2] - ref[2]};
                                T pu[3], cu[3], m1[3], m2[3];
                                for (int c = 0; c < 3; ++c) {
                                    pu[c] = chi2[h] * (u[h][c] - us2[h][c]);
                                    cu[c] = chi2[h] * us2[h][c];
                                }
                                cross3(rv, pu, m1);
                                cross3(rv, cu, m2);
                                for (int c = 0; c < 3; ++c) {
                                    v[c] += pu[c];
                                    v[3 + c] += m1[c];
                                    v[6 + c] += cu[c];
                                    v[9 + c] += m2[c];
                                }
                            }
                        }
                        // a lane's points in T, everything above it in FP64
                        warp_sums12<T>(v, wacc + warp * 36 + cc * 12, lane);
                    }
                }
            }
            e_acc += double(e_tile);
            __syncthreads();
            if (MODE == XP_DUMP) continue;
        }

        // ---- r2c of the first 3 (or ncomp) fields and store of the kept x-modes
        const int Cf = kPhys ? 3 * RB : C;
        fft_dit<T, false>(buf, Cf, ld, plan, tws, 1, plan.nst);
        x_last_forward_any<T>(buf, Cf, ld, g.Mx, g.Mxp, plan, tws, W, ex.comp0, lgRB, row0, nrows);
    }

    if (MODE == XP_PHYS) {
        __shared__ double red[kWarpsX][3];
        e_acc = warp_sum(e_acc);
        double m_d = double(m_acc);
        for (int o = 16; o > 0; o >>= 1) m_d = fmax(m_d, __shfl_xor_sync(0xffffffffu, m_d, o));
        const int anybad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            red[warp][0] = e_acc;
            red[warp][1] = m_d;
            red[warp][2] = anybad ? 1.0 : 0.0;
        }
        __syncthreads();
        double* out = ex.part + (size_t)blockIdx.x * kNumSums;
        if (tid < 36) {
            double s = 0.0;
            for (int w = 0; w < kWarpsX; ++w) s += wacc[w * 36 + tid];
            out[tid] = s;
        } else if (tid == kSumEkin) {
            double s = 0.0;
            for (int w = 0; w < kWarpsX; ++w) s += red[w][0];
            out[tid] = s;
        } else if (tid == kSumUmax2) {
            double s = 0.0;
            for (int w = 0; w < kWarpsX; ++w) s = fmax(s, red[w][1]);
            out[tid] = s;
        } else if (tid == kSumBad) {
            double s = 0.0;
            for (int w = 0; w < kWarpsX; ++w) s = fmax(s, red[w][2]);
            out[tid] = s;
        } else if (tid < kNumSums) {
            out[tid] = 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// x pass for nh = nx/2 = S R^2 (S = 1: nx = 512 with R = 16, 128 with R = 8;
// S = 2: nx = 1024, 256).  Each line (one field of one row) belongs to
// L = S R consecutive lanes, which hold R values each, lane j the points
// j + L t.  The inverse transform of length nh is a register-resident
// radix-R pass over t, the twiddles w_nh^{j k1}, then for S = 1 a radix-R
// pass over j and for S = 2 a radix-R pass over j' (j = 2 j' + p, lane pair
// p = 0, 1 for each k1) and a radix-2 step between the pair (lanes k1 and
// k1 + R) with the twiddles w_2R^{k'}; the forward transform runs the same
// steps transposed, in reverse.  The passes exchange through the line's own
// shared-memory slice, so they need __syncwarp only; XOR swizzles keep both
// sides of each exchange free of bank conflicts without padding.  The c2r
// mirror values X[nh - k] and the r2c mirror values Z[nh - k] are exchanged
// between lanes j and L - j with warp shuffles; inputs are loaded from global
// memory straight into registers and outputs are stored from registers.
// After the inverse, logical row l R + d of a line holds the point pair
// (l % R) + R d + R^2 (l / R) (SqMap).
//
// S = 0 is the rectangular form nh = 4 R (R = 12: nx = 96; R = 8: nx = 64):
// L = 4 lanes per line, lane j holding Z[j + 4 t]; the radix-R pass over t
// and the twiddles w_nh^{j n1} as above, then the R radix-4 transforms over
// j, R/4 per lane (lane j takes n1 = j + 4 m), through one exchange in the
// line's slice; the pairs n1 + R n2 are then stored in natural order.  Slices
// are nh + 4 values apart and the exchange slots XOR-swizzled, so the 16
// lanes (4 lines) of a half-warp meet 16 distinct banks on every access.
// ---------------------------------------------------------------------------
// rows per tile: each group of L lanes inverse-transforms two lines (u and
// omega fields) and forward-transforms one (the three NL fields)
template <int L> constexpr int sq_rows() { return 384 / (6 * L); }

template <int R, int S> constexpr int sq_lanes() { return S == 0 ? 4 : S * R; }
template <int R, int S> constexpr int sq_nh() { return S == 0 ? 4 * R : S * R * R; }
template <int R, int S> constexpr int sq_slice() { return S == 0 ? 4 * R + 4 : S * R * R; }

template <int R, int S> struct SqMap {
    // point pair held by logical row lrow after the inverse, and its inverse map
    __device__ __forceinline__ static int point(int lrow)
    {
        const int l = lrow / R, d = lrow % R;
        return (l % R) + R * d + R * R * (l / R);
    }
    __device__ __forceinline__ static int lrow(int pp)
    {
        return (pp % R + R * (pp / (R * R))) * R + (pp / R) % R;
    }
};

// Shared-memory slot of logical row R q + j of a line slice: the column
// index is XOR-ed with the row, so both the column-wise (pass 1) and the
// row-wise (pass 2) accesses of R lanes meet R distinct banks.
template <int R> __device__ __forceinline__ int sq_slot(int lrow)
{
    return (lrow & ~(R - 1)) | ((lrow ^ (lrow / R)) & (R - 1));
}

// FP32 radix-16 lines (nx = 512): column c of row q at c ^ (2 q mod 16), an
// even mask, so the pairs (2 i, 2 i + 1) of a row stay adjacent and in order
// and a row moves as eight 16-byte accesses; a quarter-warp (8 lanes, 8
// rows) meets 8 distinct 16-byte bank groups, a half-warp column access 16
// distinct 8-byte ones.  Other lines: c ^ q.
template <typename T, int R, int S> constexpr bool sq_wide() { return S == 1 && R == 16 && sizeof(T) == 4; }
template <typename T, int R, int S> __device__ __forceinline__ int sq_swz(int q)
{
    if constexpr (sq_wide<T, R, S>()) return (2 * q) & (R - 1);
    else return q;
}
template <typename T, int R, int S> __device__ __forceinline__ void sq_ld_row(const cplx<T>* row, int sw, cplx<T>* v)
{
    if constexpr (sq_wide<T, R, S>()) {
#pragma unroll
        for (int i = 0; i < R; i += 2) {
            const float4 p = *reinterpret_cast<const float4*>(row + (i ^ sw));
            v[i] = mkc<T>(p.x, p.y);
            v[i + 1] = mkc<T>(p.z, p.w);
        }
    } else {
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = row[i ^ sw];
    }
}
template <typename T, int R, int S> __device__ __forceinline__ void sq_st_row(cplx<T>* row, int sw, const cplx<T>* v)
{
    if constexpr (sq_wide<T, R, S>()) {
#pragma unroll
        for (int i = 0; i < R; i += 2)
            *reinterpret_cast<float4*>(row + (i ^ sw)) = make_float4(v[i].x, v[i].y, v[i + 1].x, v[i + 1].y);
    } else {
#pragma unroll
        for (int i = 0; i < R; ++i) row[i ^ sw] = v[i];
    }
}

// the rectangular form keeps the point pairs in natural order
template <int R> struct SqMap<R, 0> {
    __device__ __forceinline__ static int point(int lrow) { return lrow; }
    __device__ __forceinline__ static int lrow(int pp) { return pp; }
};

// slot of logical row lrow in a line slice
template <typename T, int R, int S> __device__ __forceinline__ int sq_line_slot(int lrow)
{
    if constexpr (S == 0) return lrow;
    else if constexpr (sq_wide<T, R, S>()) return (lrow & ~(R - 1)) | ((lrow ^ sq_swz<T, R, S>(lrow / R)) & (R - 1));
    else return sq_slot<R>(lrow);
}

template <typename T, int R, int S, bool LAYER, bool SPONGE>
__global__ void __launch_bounds__(192, sizeof(T) == 4 ? (S == 2 ? 3 : 4) : 1)
k_xpass_sq(cplx<T>* __restrict__ W, Geom g, const double2* __restrict__ tw, XExtra ex,
           const StepState* __restrict__ st, const Member* __restrict__ mb)
{
    if (mb) {   // one member of an ensemble batch
        const Member& m = mb[blockIdx.z];
        W = static_cast<cplx<T>*>(m.W);
        st = m.st;
        ex.frame = m.fr;
        ex.part = m.part;
    }
    if (st && st->status != 0) return;
    constexpr int L = sq_lanes<R, S>();    // lanes per line
    constexpr int RB = sq_rows<L>();
    constexpr int NH = sq_nh<R, S>();
    using Map = SqMap<R, S>;
    constexpr int CS = sq_slice<R, S>();   // line slice (S > 0: logical row R q + j at R q + (j ^ q))
    const int nx = g.nx, Mx = g.Mx, Mxp = g.Mxp;
    const int nrows = g.nz * g.ny;
    const int ntiles = ceil_div(nrows, RB);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* wacc = reinterpret_cast<double*>(smem_raw);                    // [warps][36]
    FrameT<T>* Fs = reinterpret_cast<FrameT<T>*>(wacc + kWarpsX * 36);
    cplx<T>* twx = reinterpret_cast<cplx<T>*>(
        reinterpret_cast<unsigned char*>(Fs) + ((sizeof(FrameT<T>) + 15) / 16) * 16);
    // w_nh^{j q} (q < R, j < L) at q L + (j ^ q): conflict-free both for a
    // fixed q across lanes j and for a fixed j across lanes q
    cplx<T>* tw2 = twx + NH;
    cplx<T>* buf = tw2 + NH;               // C line slices of CS values
    __shared__ int rowmask[RB];

    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int c = tid / L, j = tid % L;    // this lane's line and index within it
    // w_nx^k for k < nh: the c2r/r2c mirror steps use no higher power
    // (the FP32 copy of the table follows the FP64 one)
    auto twv = [&](int k) -> cplx<T> {
        if constexpr (sizeof(T) == 4) {
            const float2 w = reinterpret_cast<const float2*>(tw + nx)[k];
            return mkc<T>(w.x, w.y);
        } else {
            return mkc<T>(tw[k].x, tw[k].y);
        }
    };
    for (int i = tid; i < NH; i += blockDim.x) twx[i] = twv(i);
    for (int i = tid; i < NH; i += blockDim.x) {
        const int q = i / L, jj = i % L;
        tw2[q * L + (S == 0 ? jj : (jj ^ q))] = twv((2 * jj * q) % nx);
    }
    load_frame_t<T>(Fs, ex.frame);

    const T dxT = T(g.dx), dyT = T(g.dy), dzT = T(g.dz);
    const FrameT<T>& F = *Fs;
    constexpr int NG = 192 / L;            // lane groups; group c owns lines c and c + NG
    constexpr bool has_layer = LAYER;   // a Dirichlet layer is set
    const T uinf[3] = {T(ex.u_inf[0]), T(ex.u_inf[1]), T(ex.u_inf[2])};

    // virtual CTA vb: its tiles in order into its own row of partial sums, so
    // the sums do not depend on how many CTAs the launch runs
    const int P = ex.nvirt > 0 ? ex.nvirt : (int)gridDim.x;
#pragma unroll 1
    for (int vb = blockIdx.x; vb < P; vb += gridDim.x) {
    for (int i = tid; i < kWarpsX * 36; i += blockDim.x) wacc[i] = 0.0;
    __syncthreads();
    double e_acc = 0.0;
    T m_acc = T(0);
    int bad = 0;
    for (int tile = vb; tile < ntiles; tile += P) {
        const int row0 = tile * RB;
        cplx<T> v[R];
        // the six input lines of this block's next tile on their way into L2
        if (tid < 6) {
            const int next0 = (tile + P) * RB;
            if (next0 < nrows) {
                const int nr = min(RB, nrows - next0);
                prefetch_l2_bulk(W + ((size_t)tid * nrows + next0) * Mxp,
                                 (unsigned)(nr * Mxp * sizeof(cplx<T>)));
            }
        }
        if (tid < RB) {
            const int r = row0 + tid;
            int mask = 0;
            if (r < nrows) {
                const int z = r / g.ny, y = r - z * g.ny;
                const T Y = T(y) * dyT, Z = T(z) * dzT;
                for (int q = 0; q < 3; ++q)
                    if (F.active[q] && Y >= F.box[q][2] && Y <= F.box[q][3] && Z >= F.box[q][4] &&
                        Z <= F.box[q][5])
                        mask |= 1 << q;
            }
            rowmask[tid] = mask;
        }
#pragma unroll 1
        for (int li = 0; li < 2; ++li) {
            const int cl = c + li * NG;
            const int fld = cl / RB, lrr = cl % RB;
            cplx<T>* line = buf + cl * CS;
            // ---- this lane's kept x-modes, straight from global memory into registers
            const int r = row0 + lrr;
            const cplx<T>* src = W + ((size_t)fld * nrows + (r < nrows ? r : 0)) * Mxp;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int k = j + L * t;
                v[t] = (r < nrows && k < Mx) ? src[k] : mkc<T>(0, 0);
            }
            if (j == 0) v[0].y = T(0);     // a real line has a real mean
            // ---- inverse: c2r pre-processing, radix R over t and the twiddles
            //      w_nh^{j k1}, then the second pass(es)
            sq_exchange_pre<T, R, L>(v, j, twx);
            Dft<T, R, true>::run(v);
#pragma unroll
            for (int q = 1; q < R; ++q) v[q] = cmul(v[q], cconj(tw2[q * L + (S == 0 ? j : (j ^ q))]));
            if constexpr (S == 0) {
                // Y[j][n1] at n1 L + (j ^ n1 % L); lane j then takes n1 = j + L m
#pragma unroll
                for (int q = 0; q < R; ++q) line[q * L + (j ^ (q % L))] = v[q];
                __syncwarp();
#pragma unroll
                for (int m = 0; m < R / L; ++m) {
                    const int n1 = j + L * m;
                    cplx<T> a[L];
#pragma unroll
                    for (int i = 0; i < L; ++i) a[i] = line[n1 * L + (i ^ j)];
                    Dft<T, L, true>::run(a);   // over j -> n2: the pair n1 + R n2
#pragma unroll
                    for (int i = 0; i < L; ++i) v[m * L + i] = a[i];
                }
                __syncwarp();
#pragma unroll
                for (int m = 0; m < R / L; ++m) {
#pragma unroll
                    for (int i = 0; i < L; ++i) line[j + L * m + R * i] = v[m * L + i];
                }
            } else if constexpr (S == 1) {
#pragma unroll
                for (int q = 0; q < R; ++q) line[R * q + (j ^ sq_swz<T, R, S>(q))] = v[q];
                __syncwarp();
                sq_ld_row<T, R, S>(line + R * j, sq_swz<T, R, S>(j), v);
                Dft<T, R, true>::run(v);
                sq_st_row<T, R, S>(line + R * j, sq_swz<T, R, S>(j), v);
            } else {
                // Y[j][k1] at L k1 + (j ^ k1); lane j turns into (k1, p) = (j % R, j / R)
#pragma unroll
                for (int q = 0; q < R; ++q) line[L * q + (j ^ q)] = v[q];
                __syncwarp();
                const int k1 = j % R, p = j / R;
#pragma unroll
                for (int i = 0; i < R; ++i) v[i] = line[L * k1 + ((2 * i + p) ^ k1)];
                Dft<T, R, true>::run(v);   // over j' -> k'
                if (p) {
#pragma unroll
                    for (int d = 1; d < R; ++d) v[d] = cmul(v[d], cconj(twx[2 * R * d]));   // w_2R^{k'}
                }
                // radix 2 between the lane pair: outputs k1 + R k' + R^2 p
#pragma unroll
                for (int d = 0; d < R; ++d) {
                    cplx<T> o;
                    o.x = __shfl_xor_sync(0xffffffffu, v[d].x, R);
                    o.y = __shfl_xor_sync(0xffffffffu, v[d].y, R);
                    v[d] = p ? csub(o, v[d]) : cadd(v[d], o);
                }
                __syncwarp();
#pragma unroll
                for (int d = 0; d < R; ++d) line[sq_slot<R>(R * j + d)] = v[d];
            }
        }
        __syncthreads();

        // ---- physical space, every point: NL = u x omega into the omega lines,
        //      energy and max |u|^2.  A non-finite velocity makes the energy sum
        //      non-finite; NL can only be non-finite through u (omega, u_s and
        //      the penalization are finite for a finite state), so the energy
        //      sum is the check.
        //      FP32 radix-16 and rectangular lines without the wake terms: two
        //      point pairs per thread (logical rows 2m, 2m + 1 sit in adjacent
        //      slots of those layouts), as 16-byte accesses.
        if constexpr (sizeof(T) == 4 && (sq_wide<T, R, S>() || S == 0) && !SPONGE && !LAYER) {
            constexpr int NH2 = NH / 2;
            const int items = RB * NH2;
            T e_tile = T(0);
            for (int it = 0; it < (items + 191) / 192; ++it) {
                const int i = tid + it * 192;
                const int rr = i / NH2, lrow = 2 * (i % NH2);
                if (i < items && row0 + rr < nrows) {
                    const int slot = sq_line_slot<T, R, S>(lrow);   // even; row lrow + 1 at slot + 1
                    float4 uq[3], wq[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        uq[q] = *reinterpret_cast<const float4*>(buf + (q * RB + rr) * CS + slot);
                        wq[q] = *reinterpret_cast<const float4*>(buf + ((3 + q) * RB + rr) * CS + slot);
                    }
                    T nl[4][3];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        T u[3], om[3];
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            u[q] = h == 0 ? uq[q].x : h == 1 ? uq[q].y : h == 2 ? uq[q].z : uq[q].w;
                            om[q] = h == 0 ? wq[q].x : h == 1 ? wq[q].y : h == 2 ? wq[q].z : wq[q].w;
                        }
                        cross3(u, om, nl[h]);
                        const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                        e_tile += uu;
                        m_acc = fmax(m_acc, uu);
                    }
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        *reinterpret_cast<float4*>(buf + ((3 + q) * RB + rr) * CS + slot) =
                            make_float4(nl[0][q], nl[1][q], nl[2][q], nl[3][q]);
                }
            }
            e_acc += double(e_tile);
            if (!isfinite(e_tile)) bad = 1;
        } else {
            const int items = RB * NH;
            T e_tile = T(0);
            for (int it = 0; it < (items + 191) / 192; ++it) {
                const int i = tid + it * 192;
                const int rr = i / NH, lrow = i % NH;
                if (i < items && row0 + rr < nrows) {
                    const int slot = sq_line_slot<T, R, S>(lrow);
                    cplx<T> uv[3], wv[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        uv[q] = buf[(q * RB + rr) * CS + slot];
                        wv[q] = buf[((3 + q) * RB + rr) * CS + slot];
                    }
                    if (SPONGE) {   // chi_sp omega (Sec. 2.3) into the sponge lines
                        const int r = row0 + rr, z = r / g.ny, y = r - z * g.ny;
                        const int pp = Map::point(lrow);
                        const bool in_row = y >= ex.sponge0[1] || z >= ex.sponge0[2];
                        const T s0 = (in_row || 2 * pp >= ex.sponge0[0]) ? T(1) : T(0);
                        const T s1 = (in_row || 2 * pp + 1 >= ex.sponge0[0]) ? T(1) : T(0);
#pragma unroll
                        for (int q = 0; q < 3; ++q)
                            buf[((6 + q) * RB + rr) * CS + slot] = mkc<T>(s0 * wv[q].x, s1 * wv[q].y);
                    }
                    T nl[2][3];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        T u[3], om[3];
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            u[q] = h ? uv[q].y : uv[q].x;
                            om[q] = h ? wv[q].y : wv[q].x;
                        }
                        cross3(u, om, nl[h]);
                        if (has_layer) {   // Dirichlet layer u = u_inf (Sec. 2.3)
                            const int r = row0 + rr, z = r / g.ny, y = r - z * g.ny;
                            const int pp = Map::point(lrow);
                            if (y >= ex.layer0[1] || z >= ex.layer0[2] || 2 * pp + h >= ex.layer0[0]) {
#pragma unroll
                                for (int q = 0; q < 3; ++q) nl[h][q] -= F.inv_eta * (u[q] - uinf[q]);
                            }
                        }
                        const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                        e_tile += uu;
                        m_acc = fmax(m_acc, uu);
                    }
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        buf[((3 + q) * RB + rr) * CS + slot] = mkc<T>(nl[0][q], nl[1][q]);
                }
            }
            e_acc += double(e_tile);
            if (!isfinite(e_tile)) bad = 1;
        }

        // ---- penalization, only in tiles with a row that meets a part's box:
        //      chi, u_s, NL -= chi/C_eta (u - u_s) and the per-colour sums
        int tile_any = 0;
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) tile_any |= rowmask[rr];
        if (tile_any) {   // uniform over the block
            __syncthreads();
            constexpr int NX = 2 * NH;
            for (int i0 = 0; i0 < RB * NX; i0 += 192) {
                const int i = i0 + tid;
                const int rr = i / NX, xi = i % NX;
                const int r = row0 + rr;
                const int mask = (i < RB * NX && r < nrows) ? rowmask[rr] : 0;
                T chi = T(0), us[3] = {T(0), T(0), T(0)}, X[3] = {T(0), T(0), T(0)};
                T u[3] = {T(0), T(0), T(0)};
                int colr = 0;
                if (mask != 0) {
                    const int z = r / g.ny, y = r - z * g.ny;
                    X[0] = T(xi) * dxT;
                    X[1] = T(y) * dyT;
                    X[2] = T(z) * dzT;
                    const bool inrow[3] = {(mask & 1) != 0, (mask & 2) != 0, (mask & 4) != 0};
                    solid_at(F, X, inrow, chi, colr, us);
                    if (chi > T(0)) {
                        // point xi is half h of pair pp, held at logical row Map::lrow(pp)
                        const int pp = xi >> 1, h = xi & 1;
                        const int lrow = Map::lrow(pp);
                        const int slot = sq_line_slot<T, R, S>(lrow);
                        const T pen = chi * F.inv_eta;
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            const T* ul = reinterpret_cast<const T*>(buf + (q * RB + rr) * CS + slot);
                            T* nl = reinterpret_cast<T*>(buf + ((3 + q) * RB + rr) * CS + slot);
                            u[q] = ul[h];
                            nl[h] -= pen * (u[q] - us[q]);
                        }
                    }
                }
                if (__any_sync(0xffffffffu, colr != 0)) {
                    for (int cc = 0; cc < 3; ++cc) {
                        const bool has = colr == cc + 1;
                        if (!__any_sync(0xffffffffu, has)) continue;
                        T acc[12];   // this lane's contribution, in T
#pragma unroll
                        for (int k2 = 0; k2 < 12; ++k2) acc[k2] = T(0);
                        if (has) {
                            const T* ref = cc == 0 ? F.xc : F.pv[cc - 1];
                            T rv[3] = {X[0] - ref[0], X[1] - ref[1], X[2] - ref[2]};
                            T pu[3], cu[3], m1[3], m2[3];
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                pu[q] = chi * (u[q] - us[q]);
                                cu[q] = chi * us[q];
                            }
                            cross3(rv, pu, m1);
                            cross3(rv, cu, m2);
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                acc[q] = pu[q];
                                acc[3 + q] = m1[q];
                                acc[6 + q] = cu[q];
                                acc[9 + q] = m2[q];
                            }
                        }
                        // one point per lane in T; the sums across lanes, warps
                        // and blocks in FP64
                        warp_sums12<T>(acc, wacc + warp * 36 + cc * 12, lane);
                    }
                }
            }
        }
        __syncthreads();

        // ---- forward on the three NL lines of each row (one per lane group) and,
        //      with the sponge, the three chi_sp omega lines (a second one):
        //      DIT stage 1, stage 0, r2c post-processing and store
#pragma unroll 1
        for (int li = 0; li < (SPONGE ? 2 : 1); ++li) {
            cplx<T>* line = buf + (3 * RB + c + li * NG) * CS;
            const int fld = 3 * li + c / RB, lrr = c % RB;
            if constexpr (S == 0) {
                // lane j takes n1 = j + L m: radix L over its pairs n1 + R i,
                // the twiddles w_nh^{n1 jj}, U[n1][jj] at n1 L + (jj ^ j)
#pragma unroll
                for (int m = 0; m < R / L; ++m) {
                    const int n1 = j + L * m;
                    cplx<T> a[L];
#pragma unroll
                    for (int i = 0; i < L; ++i) a[i] = line[n1 + R * i];
                    Dft<T, L, false>::run(a);
#pragma unroll
                    for (int i = 1; i < L; ++i) a[i] = cmul(a[i], tw2[n1 * L + i]);
#pragma unroll
                    for (int i = 0; i < L; ++i) v[m * L + i] = a[i];
                }
                __syncwarp();
#pragma unroll
                for (int m = 0; m < R / L; ++m) {
#pragma unroll
                    for (int i = 0; i < L; ++i) line[(j + L * m) * L + (i ^ j)] = v[m * L + i];
                }
                __syncwarp();
#pragma unroll
                for (int q = 0; q < R; ++q) v[q] = line[q * L + (j ^ (q % L))];
            } else if constexpr (S == 1) {
                sq_ld_row<T, R, S>(line + R * j, sq_swz<T, R, S>(j), v);
                Dft<T, R, false>::run(v);
                sq_st_row<T, R, S>(line + R * j, sq_swz<T, R, S>(j), v);
                __syncwarp();
#pragma unroll
                for (int t = 0; t < R; ++t) v[t] = line[R * t + (j ^ sq_swz<T, R, S>(t))];
#pragma unroll
                for (int t = 1; t < R; ++t) v[t] = cmul(v[t], tw2[t * R + (j ^ t)]);
            } else {
                // lane j = (k1, p): radix 2 over the two halves h of its points
                // k1 + R k' + R^2 h, the twiddles w_2R^{p k'}, radix R over k',
                // then w_nh^{k1 (2 j' + p)}
                const int k1 = j % R, p = j / R;
#pragma unroll
                for (int d = 0; d < R; ++d) {
                    const cplx<T> a = line[sq_slot<R>(R * j + d)];
                    const cplx<T> b = line[sq_slot<R>(R * (j ^ R) + d)];
                    v[d] = p ? csub(b, a) : cadd(a, b);
                }
                if (p) {
#pragma unroll
                    for (int d = 1; d < R; ++d) v[d] = cmul(v[d], twx[2 * R * d]);
                }
                Dft<T, R, false>::run(v);   // over k' -> j'
#pragma unroll
                for (int i = 0; i < R; ++i) v[i] = cmul(v[i], tw2[k1 * L + ((2 * i + p) ^ k1)]);
                __syncwarp();
#pragma unroll
                for (int i = 0; i < R; ++i) line[L * k1 + ((2 * i + p) ^ k1)] = v[i];
                __syncwarp();
#pragma unroll
                for (int q = 0; q < R; ++q) v[q] = line[L * q + (j ^ q)];
            }
            Dft<T, R, false>::run(v);      // v[q] = Z[j + L q]
            const int r = row0 + lrr;
            cplx<T>* out = W + ((size_t)fld * nrows + (r < nrows ? r : 0)) * Mxp;
#pragma unroll
            for (int s2 = 0; s2 < R / 2; ++s2) {
                cplx<T> a, b;   // partner's Z[s2] and Z[R-1-s2]
                a.x = __shfl_sync(0xffffffffu, v[s2].x, (L - j) & (L - 1), L);
                a.y = __shfl_sync(0xffffffffu, v[s2].y, (L - j) & (L - 1), L);
                b.x = __shfl_sync(0xffffffffu, v[R - 1 - s2].x, (L - j) & (L - 1), L);
                b.y = __shfl_sync(0xffffffffu, v[R - 1 - s2].y, (L - j) & (L - 1), L);
                if (r < nrows) {
                    const int q1 = s2, q2 = R - 1 - s2;
                    const int k1 = j + L * q1, k2 = j + L * q2;
                    cplx<T> m1, m2;
                    if (j != 0) {
                        m1 = b;    // Z[nh - k1] = partner's Z[R-1-q1]
                        m2 = a;
                    } else {
                        m1 = v[(R - q1) % R];
                        m2 = v[(R - q2) % R];
                    }
                    if (k1 < Mxp) out[k1] = k1 < Mx ? r2c_post<T>(v[q1], m1, twx[k1]) : mkc<T>(0, 0);
                    if (k2 < Mxp) out[k2] = k2 < Mx ? r2c_post<T>(v[q2], m2, twx[k2]) : mkc<T>(0, 0);
                }
            }
        }
        // No block barrier before the next tile: its inverse lines go to
        // slices c and c + NG of group c (3 RB = NG in every layout), that is
        // a u line, whose last readers (the physical-space phases) are behind
        // the barrier above, and the group's own forward line; rowmask is
        // read between the first and the last barrier of a tile only.  The
        // lanes of a group still order their reads before their writes.
        __syncwarp();
    }

    __shared__ double red[kWarpsX][3];
    e_acc = warp_sum(e_acc);
    double m_d = double(m_acc);
    for (int o = 16; o > 0; o >>= 1) m_d = fmax(m_d, __shfl_xor_sync(0xffffffffu, m_d, o));
    const int anybad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        red[warp][0] = e_acc;
        red[warp][1] = m_d;
        red[warp][2] = anybad ? 1.0 : 0.0;
    }
    __syncthreads();
    double* outp = ex.part + (size_t)vb * kNumSums;
    if (tid < 36) {
        double s2 = 0.0;
        for (int w = 0; w < kWarpsX; ++w) s2 += wacc[w * 36 + tid];
        outp[tid] = s2;
    } else if (tid == kSumEkin) {
        double s2 = 0.0;
        for (int w = 0; w < kWarpsX; ++w) s2 += red[w][0];
        outp[tid] = s2;
    } else if (tid == kSumUmax2 || tid == kSumBad) {
        double s2 = 0.0;
        for (int w = 0; w < kWarpsX; ++w) s2 = fmax(s2, red[w][tid == kSumUmax2 ? 1 : 2]);
        outp[tid] = s2;
    } else if (tid < kNumSums) {
        outp[tid] = 0.0;
    }
    __syncthreads();   // wacc and red read before the next virtual CTA clears them
    }   // virtual CTAs
}

template <typename T, int R, int S> size_t sq_smem(const Geom& g, bool sponge = false)
{
    const int RB = sq_rows<sq_lanes<R, S>()>(), NH = sq_nh<R, S>(), CS = sq_slice<R, S>();
    size_t s = sizeof(double) * kWarpsX * 36 + ((sizeof(FrameT<T>) + 15) / 16) * 16;
    s += sizeof(cplx<T>) * ((size_t)2 * NH + (size_t)(sponge ? 9 : 6) * RB * CS);
    return s;
}

// grid = the virtual CTAs (rows of partial sums, x_grid); a batch of n
// members runs about one resident wave in all, each CTA taking several
// virtual ones, instead of n full grids of CTAs that each take one or two
// tiles and pay their table and frame loads for them.
template <typename T, int R, int S>
void launch_sq(bool layer, bool sponge, cplx<T>* w, const Geom& g, const double2* tw, const XExtra& ex0,
               const StepState* st, cudaStream_t s, int grid)
{
    const size_t smem = sq_smem<T, R, S>(g, sponge);
    const Batch& B = current_batch();
    XExtra ex = ex0;
    ex.nvirt = grid;
    int run = grid;
    if (B.n > 1) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_xpass_sq<T, R, S, false, false>, 192, smem);
        const int resident = std::max(1, sms * std::max(1, per_sm));
        run = std::min(grid, std::max(1, ceil_div(resident, B.n)));
    }
    const dim3 gd(run, 1, B.n);
    if (layer && sponge)
        k_xpass_sq<T, R, S, true, true><<<gd, 192, smem, s>>>(w, g, tw, ex, st, B.mb);
    else if (layer)
        k_xpass_sq<T, R, S, true, false><<<gd, 192, smem, s>>>(w, g, tw, ex, st, B.mb);
    else if (sponge)
        k_xpass_sq<T, R, S, false, true><<<gd, 192, smem, s>>>(w, g, tw, ex, st, B.mb);
    else
        k_xpass_sq<T, R, S, false, false><<<gd, 192, smem, s>>>(w, g, tw, ex, st, B.mb);
}

// the register-resident kernel for this grid: 10 R + S (R = 16 or 8 with
// S = 1 or 2; R = 12 or 8 with S = 0, the rectangular form), or 0 for the
// generic one
template <typename T> int sq_kind(const Geom& g)
{
    if (g.xgeneric) return 0;
    switch (g.nx) {
    case 512: return 161;
    case 128: return 81;
    case 1024: return 162;
    case 256: return 82;
    case 96: return 120;
    case 64: return 80;
    default: return 0;
    }
}

template <typename T> int x_lgrb(const Geom& g)
{
    const int nh = g.nx / 2;
    int RB = 32;
    while (RB > 1 && nh * 6 * RB > tile_elems<T>()) RB >>= 1;
    return __builtin_ctz(RB);
}

template <typename T> size_t x_smem(const Geom& g, int lgRB, int NF)
{
    const int C = NF << lgRB;
    const int ld = C | 1;
    size_t s = sizeof(double) * kWarpsX * 36 + ((sizeof(FrameT<T>) + 15) / 16) * 16;
    s += sizeof(cplx<T>) * ((size_t)g.nx + (size_t)(g.nx / 2) * ld) + 2 * sizeof(int) * (g.nx / 2);
    return s;
}

template <typename T> int x_grid(const Geom& g)
{
    int dev = 0, sm_count = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (sm_count <= 0) sm_count = 1;
    int per_sm = 0, ntiles = 0;
    const int kind = sq_kind<T>(g);
#define FLUSI_SQ_OCC(R, S)                                                                          \
    ntiles = ceil_div(g.nz * g.ny, sq_rows<sq_lanes<R, S>()>());                                               \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_xpass_sq<T, R, S, false, false>, 192, \
                                                  sq_smem<T, R, S>(g));
    if (kind == 161) {
        FLUSI_SQ_OCC(16, 1)
    } else if (kind == 81) {
        FLUSI_SQ_OCC(8, 1)
    } else if (kind == 162) {
        FLUSI_SQ_OCC(16, 2)
    } else if (kind == 82) {
        FLUSI_SQ_OCC(8, 2)
    } else if (kind == 120) {
        FLUSI_SQ_OCC(12, 0)
    } else if (kind == 80) {
        FLUSI_SQ_OCC(8, 0)
    } else {
        const int lg = x_lgrb<T>(g);
        ntiles = ceil_div(g.nz * g.ny, 1 << lg);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_xpass<T, XP_PHYS>, kThreadsX,
                                                      x_smem<T>(g, lg, 6));
    }
#undef FLUSI_SQ_OCC
    if (per_sm <= 0) per_sm = 1;
    int grid = sm_count * per_sm;
    return grid < ntiles ? grid : ntiles;
}

template <typename T>
cudaError_t launch_x(int mode, void* W, const Geom& g, const FftPlan& plan, const double2* tw,
                     const int* pos, const XExtra& ex, const StepState* st, cudaStream_t s)
{
    const int lg = x_lgrb<T>(g);
    const int RB = 1 << lg;
    const int ntiles = ceil_div(g.nz * g.ny, RB);
    const int NF = (mode == XP_PHYS || mode == XP_DUMP) ? 6 : ex.ncomp;
    if (NF < 1 || NF > 6 || (g.nx / 2) * NF * RB > tile_elems<T>()) return cudaErrorInvalidValue;
    if (kThreadsX % (NF * RB) != 0) return cudaErrorInvalidValue;
    const size_t smem = x_smem<T>(g, lg, NF);
    cplx<T>* w = (cplx<T>*)W;
    const bool layer = ex.layer0[0] < g.nx || ex.layer0[1] < g.ny || ex.layer0[2] < g.nz;
    const bool sponge = ex.sponge_fused != 0;
    switch (mode) {
    case XP_PHYS:
        switch (sq_kind<T>(g)) {
        case 161: launch_sq<T, 16, 1>(layer, sponge, w, g, tw, ex, st, s, x_grid<T>(g)); break;
        case 81: launch_sq<T, 8, 1>(layer, sponge, w, g, tw, ex, st, s, x_grid<T>(g)); break;
        case 162: launch_sq<T, 16, 2>(layer, sponge, w, g, tw, ex, st, s, x_grid<T>(g)); break;
        case 82: launch_sq<T, 8, 2>(layer, sponge, w, g, tw, ex, st, s, x_grid<T>(g)); break;
        case 120: launch_sq<T, 12, 0>(layer, sponge, w, g, tw, ex, st, s, x_grid<T>(g)); break;
        case 80: launch_sq<T, 8, 0>(layer, sponge, w, g, tw, ex, st, s, x_grid<T>(g)); break;
        default:
            k_xpass<T, XP_PHYS><<<dim3(x_grid<T>(g), 1, current_batch().n), kThreadsX, smem, s>>>(
                w, g, plan, tw, pos, ex, lg, st, current_batch().mb);
        }
        break;
    case XP_R2C:
        k_xpass<T, XP_R2C><<<ntiles, kThreadsX, smem, s>>>(w, g, plan, tw, pos, ex, lg, st, nullptr);
        break;
    case XP_C2R:
        k_xpass<T, XP_C2R><<<ntiles, kThreadsX, smem, s>>>(w, g, plan, tw, pos, ex, lg, st, nullptr);
        break;
    case XP_SPONGE:
        k_xpass<T, XP_SPONGE><<<ntiles, kThreadsX, smem, s>>>(w, g, plan, tw, pos, ex, lg, st, nullptr);
        break;
    default:
        k_xpass<T, XP_DUMP><<<ntiles, kThreadsX, smem, s>>>(w, g, plan, tw, pos, ex, lg, st, nullptr);
        break;
    }
    return cudaGetLastError();
}

}  // namespace

int xpass_grid(int fp64, const Geom& g)
{
    if (!fp64 && g.xtc) return xpass_tc_grid(g);
    return fp64 ? x_grid<double>(g) : x_grid<float>(g);
}

// 1 when the physical x pass (square kernel) forms and transforms chi_sp omega itself
int xpass_fuses_sponge(int fp64, const Geom& g)
{
    if (!fp64 && g.xtc) return 0;
    return fp64 ? sq_kind<double>(g) != 0 : sq_kind<float>(g) != 0;
}

cudaError_t launch_xpass(int fp64, int mode, void* W, const Geom& g, const FftPlan& plan,
                         const double2* tw, const int* pos, const XExtra& ex, const StepState* st,
                         cudaStream_t s)
{
    // ensemble batches cover the physical pass of the CUDA-core kernels only
    if (current_batch().mb && (mode != XP_PHYS || (!fp64 && g.xtc) || ex.sponge_fused))
        return cudaErrorInvalidValue;
    if (!fp64 && g.xtc && mode == XP_PHYS) return launch_xpass_tc(W, g, tw, ex, st, s);
    return fp64 ? launch_x<double>(mode, W, g, plan, tw, pos, ex, st, s)
                : launch_x<float>(mode, W, g, plan, tw, pos, ex, st, s);
}

cudaError_t configure_xpass()
{
    const int big = 200 * 1024;
    cudaError_t e;
#define FLUSI_SMEM(fn) \
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    FLUSI_SMEM((k_xpass<float, XP_PHYS>))
    FLUSI_SMEM((k_xpass<float, XP_R2C>))
    FLUSI_SMEM((k_xpass<float, XP_C2R>))
    FLUSI_SMEM((k_xpass<float, XP_DUMP>))
    FLUSI_SMEM((k_xpass<float, XP_SPONGE>))
    FLUSI_SMEM((k_xpass<double, XP_SPONGE>))
    FLUSI_SMEM((k_xpass<double, XP_PHYS>))
    FLUSI_SMEM((k_xpass<double, XP_R2C>))
    FLUSI_SMEM((k_xpass<double, XP_C2R>))
    FLUSI_SMEM((k_xpass<double, XP_DUMP>))
#define FLUSI_SMEM_SQ(T, R, S)                              \
    FLUSI_SMEM((k_xpass_sq<T, R, S, false, false>))         \
    FLUSI_SMEM((k_xpass_sq<T, R, S, true, false>))          \
    FLUSI_SMEM((k_xpass_sq<T, R, S, false, true>))          \
    FLUSI_SMEM((k_xpass_sq<T, R, S, true, true>))
    FLUSI_SMEM_SQ(float, 16, 1)
    FLUSI_SMEM_SQ(float, 8, 1)
    FLUSI_SMEM_SQ(float, 16, 2)
    FLUSI_SMEM_SQ(float, 8, 2)
    FLUSI_SMEM_SQ(float, 12, 0)
    FLUSI_SMEM_SQ(float, 8, 0)
    FLUSI_SMEM_SQ(double, 12, 0)
    FLUSI_SMEM_SQ(double, 8, 0)
    FLUSI_SMEM_SQ(double, 16, 1)
    FLUSI_SMEM_SQ(double, 8, 1)
    FLUSI_SMEM_SQ(double, 16, 2)
    FLUSI_SMEM_SQ(double, 8, 2)
#undef FLUSI_SMEM_SQ
#undef FLUSI_SMEM
    return cudaSuccess;
}

}  // namespace flusi

// ---------------------------------------------------------------------------
// Allocation-free variant of the physical pass's reduction.
//
// Some callers cannot allocate device memory at all: their device memory is
// owned by another allocator's pool (a framework's caching allocator, a
// real-time loop that reserves everything up front), or they cannot accept a
// cudaMalloc / cudaFree and its implicit device synchronization where they
// run.  This entry point gives them the force, moment, energy and CFL sums of
// a velocity field they already hold, with no handle and no workspace: its
// scratch (the insect descriptor, the frame block, one row of FP64 partial
// sums per CTA and the reduced sums) lives in a fixed array in the library's
// own device memory.
// ---------------------------------------------------------------------------
namespace flusi {

namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocWarps = kNoallocThreads / 32;
constexpr int kNoallocMaxCtas = 1024;                       // partial-sum rows
constexpr long long kNoallocMaxPoints = 1024LL * 1024 * 1024;
constexpr int kNoallocHeader = 512;                         // doubles: descriptor, time, frame

// Scratch of the allocation-free entry point: [header | partials | sums],
// 8 * (512 + 1024 * 40 + 40) bytes (about 332 KB), held by every GPU that
// loads the library until the process exits.
constexpr size_t kNoallocDoubles = kNoallocHeader + (size_t)kNoallocMaxCtas * kNumSums + kNumSums;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

static_assert(sizeof(flusi_insect) + sizeof(StepState) + sizeof(Frame) + 32 <= kNoallocHeader * 8,
              "scratch header too small");

// Copies the caller's descriptor and time into the scratch header.
__global__ void k_noalloc_header(flusi_insect ins, double t, flusi_insect* d_ins, StepState* d_st)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *d_ins = ins;
    StepState st = {};
    st.t = t;
    *d_st = st;
}

__global__ void __launch_bounds__(kNoallocThreads)
k_noalloc_sums(const double* __restrict__ u, int nx, int ny, int nz, double dx, double dy, double dz,
               const Frame* __restrict__ frame, Shape S, double* __restrict__ part)
{
    __shared__ FrameT<double> F;
    __shared__ double wacc[kNoallocWarps * 36];
    __shared__ double red[kNoallocWarps][3];
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    for (int i = tid; i < kNoallocWarps * 36; i += kNoallocThreads) wacc[i] = 0.0;
    if (tid == 0) setup_frame<double>(F, *frame, S, 0.0);
    __syncthreads();

    const long long N = (long long)nx * ny * nz;
    double e_acc = 0.0, m_acc = 0.0;
    int bad = 0;
    // block-uniform trip count, so whole warps reach the votes below
    for (long long base = (long long)blockIdx.x * kNoallocThreads; base < N;
         base += (long long)gridDim.x * kNoallocThreads) {
        const long long i = base + tid;
        const bool valid = i < N;
        double chi = 0.0, us[3] = {0, 0, 0}, uu[3] = {0, 0, 0}, X[3] = {0, 0, 0};
        int col = 0;
        if (valid) {
            const int x = (int)(i % nx);
            const long long r = i / nx;
            const int y = (int)(r % ny), z = (int)(r / ny);
            X[0] = x * dx;
            X[1] = y * dy;
            X[2] = z * dz;
            for (int c = 0; c < 3; ++c) uu[c] = u[c * N + i];
            bool inrow[3];
            for (int q = 0; q < 3; ++q)
                inrow[q] = F.active[q] && X[1] >= F.box[q][2] && X[1] <= F.box[q][3] &&
                           X[2] >= F.box[q][4] && X[2] <= F.box[q][5];
            solid_at(F, X, inrow, chi, col, us);
            const double u2 = uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2];
            e_acc += u2;
            m_acc = fmax(m_acc, u2);
            if (!isfinite(u2)) bad = 1;
        }
        for (int cc = 0; cc < 3; ++cc) {
            const bool has = valid && col == cc + 1;
            if (!__any_sync(0xffffffffu, has)) continue;
            double v[12];
            for (int k = 0; k < 12; ++k) v[k] = 0.0;
            if (has) {
                const double* ref = cc == 0 ? F.xc : F.pv[cc - 1];
                double rv[3] = {X[0] - ref[0], X[1] - ref[1], X[2] - ref[2]};
                double pu[3], cu[3], m1[3], m2[3];
                for (int c = 0; c < 3; ++c) {
                    pu[c] = chi * (uu[c] - us[c]);
                    cu[c] = chi * us[c];
                }
                cross3(rv, pu, m1);
                cross3(rv, cu, m2);
                for (int c = 0; c < 3; ++c) {
                    v[c] = pu[c];
                    v[3 + c] = m1[c];
                    v[6 + c] = cu[c];
                    v[9 + c] = m2[c];
                }
            }
            for (int k = 0; k < 12; ++k) v[k] = warp_sum(v[k]);
            if (lane == 0)
                for (int k = 0; k < 12; ++k) wacc[warp * 36 + cc * 12 + k] += v[k];
        }
    }
    e_acc = warp_sum(e_acc);
    for (int o = 16; o > 0; o >>= 1) m_acc = fmax(m_acc, __shfl_xor_sync(0xffffffffu, m_acc, o));
    const int anybad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        red[warp][0] = e_acc;
        red[warp][1] = m_acc;
        red[warp][2] = anybad ? 1.0 : 0.0;
    }
    __syncthreads();
    double* out = part + (size_t)blockIdx.x * kNumSums;
    if (tid < 36) {
        double s = 0.0;
        for (int w = 0; w < kNoallocWarps; ++w) s += wacc[w * 36 + tid];
        out[tid] = s;
    } else if (tid == kSumEkin) {
        double s = 0.0;
        for (int w = 0; w < kNoallocWarps; ++w) s += red[w][0];
        out[tid] = s;
    } else if (tid == kSumUmax2 || tid == kSumBad) {
        double s = 0.0;
        for (int w = 0; w < kNoallocWarps; ++w) s = fmax(s, red[w][tid == kSumUmax2 ? 1 : 2]);
        out[tid] = s;
    } else if (tid < kNumSums) {
        out[tid] = 0.0;
    }
}

// One block: partial rows reduced in a fixed order, then scaled into the
// output layout (per colour F[3], M[3], I[3], J[3]; then E_kin, max |u|,
// and the non-finite flag).
__global__ void k_noalloc_reduce(const double* __restrict__ part, int nparts, double dV, double eta,
                                 double* __restrict__ out)
{
    __shared__ double tot[kNumSums];
    const int k = threadIdx.x;
    if (k < kNumSums) {
        const bool is_max = (k == kSumUmax2 || k == kSumBad);
        double a = 0.0;
        for (int i = 0; i < nparts; ++i) {
            const double v = part[(size_t)i * kNumSums + k];
            a = is_max ? fmax(a, v) : a + v;
        }
        tot[k] = a;
    }
    __syncthreads();
    if (k < 36) {
        out[k] = (k % 12) < 6 ? tot[k] * dV / eta : tot[k] * dV;
    } else if (k == 36) {
        out[36] = 0.5 * tot[kSumEkin] * dV;
    } else if (k == 37) {
        out[37] = sqrt(tot[kSumUmax2]);
    } else if (k == 38) {
        out[38] = tot[kSumBad];
    }
}

// Device address of the scratch array, looked up once per device and CUDA
// context.  A module's device globals live in one context: after
// cudaDeviceReset (or any teardown of the primary context) the library's
// module is loaded again into the new context and the array can move, so the
// cached address is kept together with the unique id of the context it was
// found in (cuCtxGetId) and looked up again when that id changes.
constexpr int kNoallocMaxDevices = 64;
struct NoallocSlot {
    std::mutex m;
    unsigned long long ctx_id = 0;   // 0: nothing cached
    double* ptr = nullptr;
};
NoallocSlot g_noalloc_slot[kNoallocMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context, or 0 when there is none
// or the driver cannot tell (then nothing is cached).
unsigned long long current_context_id()
{
    static const std::pair<CtxGetCurrentFn, CtxGetIdFn> fns = [] {
        void* cur = nullptr;
        void* id = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &cur, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            cur = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &id, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            id = nullptr;
        cudaGetLastError();
        return std::make_pair(reinterpret_cast<CtxGetCurrentFn>(cur), reinterpret_cast<CtxGetIdFn>(id));
    }();
    if (!fns.first || !fns.second) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (fns.first(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (fns.second(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

}  // namespace

}  // namespace flusi

extern "C" int flusi_penalization_sums_noalloc(int nx, int ny, int nz, const double L[3],
                                               double eta, const flusi_insect* insect, double t,
                                               const double* u_dev, double* sums_out,
                                               void* cuda_stream)
{
    using namespace flusi;
    if (nx < 1 || ny < 1 || nz < 1 || !L || !(L[0] > 0) || !(L[1] > 0) || !(L[2] > 0) ||
        !(eta > 0) || !u_dev || !sums_out) {
        set_global_error("flusi_penalization_sums_noalloc: bad sizes, box, eta or NULL pointer");
        return FLUSI_EINVAL;
    }
    const long long N = (long long)nx * ny * nz;
    if (N > kNoallocMaxPoints) {
        set_global_error("flusi_penalization_sums_noalloc: grid has more than "
                         "FLUSI_NOALLOC_MAX_POINTS (2^30) points");
        return FLUSI_EINVAL;
    }
    if (insect && insect_error(*insect)) {
        set_global_error("flusi_penalization_sums_noalloc: bad insect descriptor");
        return FLUSI_EINVAL;
    }

    // set-up, once per device and context: the device address of the
    // scratch array (host code holds only a stand-in for the symbol)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
        set_global_error("flusi_penalization_sums_noalloc: no usable current device");
        return FLUSI_ECUDA;
    }
    double* scratch = nullptr;
    {
        NoallocSlot& slot = g_noalloc_slot[dev];
        std::lock_guard<std::mutex> lock(slot.m);
        const unsigned long long id = current_context_id();
        if (slot.ptr && id != 0 && id == slot.ctx_id) {
            scratch = slot.ptr;
        } else {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                set_global_error("flusi_penalization_sums_noalloc: cudaGetSymbolAddress failed");
                return FLUSI_ECUDA;
            }
            scratch = static_cast<double*>(p);
            // the lookup made the device's primary context current if it was not
            slot.ctx_id = current_context_id();
            slot.ptr = slot.ctx_id != 0 ? scratch : nullptr;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    // header: descriptor, step state (only t is read), frame block
    char* head = reinterpret_cast<char*>(scratch);
    flusi_insect* d_ins = reinterpret_cast<flusi_insect*>(head);
    StepState* d_st = reinterpret_cast<StepState*>(head + ((sizeof(flusi_insect) + 15) / 16) * 16);
    Frame* d_fr = reinterpret_cast<Frame*>(reinterpret_cast<char*>(d_st) +
                                           ((sizeof(StepState) + 15) / 16) * 16);
    double* part = scratch + kNoallocHeader;
    double* sums = part + (size_t)kNoallocMaxCtas * kNumSums;

    flusi_insect ins{};
    if (insect) ins = *insect;
    const double dx = L[0] / nx, dy = L[1] / ny, dz = L[2] / nz;
    Shape sh{};
    if (insect) sh = shape_of(ins, ins.c_smth * fmax(dx, fmax(dy, dz)));
    const double margin = sh.profile == 1 ? 1e300 : sh.h;
    // every slot read below is written first in this call: nothing carried
    // over from an earlier call needs clearing
    const long long want = (N + kNoallocThreads - 1) / kNoallocThreads;
    const int grid = (int)(want < kNoallocMaxCtas ? want : kNoallocMaxCtas);
    k_noalloc_header<<<1, 1, 0, s>>>(ins, t, d_ins, d_st);
    k_kinematics<<<1, 32, 0, s>>>(d_ins, d_st, nullptr, d_fr, margin, 0.0, nullptr, sh, 0, 0.0);
    k_noalloc_sums<<<grid, kNoallocThreads, 0, s>>>(u_dev, nx, ny, nz, dx, dy, dz, d_fr, sh, part);
    k_noalloc_reduce<<<1, 64, 0, s>>>(part, grid, dx * dy * dz, eta, sums);
    cudaError_t e = cudaGetLastError();
    double host[kNumSums];
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, sums, sizeof(double) * 39, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return FLUSI_ECUDA;
    }
    for (int i = 0; i < 38; ++i) sums_out[i] = host[i];
    if (host[38] != 0.0) {
        set_global_error("flusi_penalization_sums_noalloc: non-finite velocity");
        return FLUSI_ENONFINITE;
    }
    return FLUSI_OK;
}

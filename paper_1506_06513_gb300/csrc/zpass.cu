// z-axis transform passes, fused with the spectral pointwise work.
//
// Columns along z are indexed by q = jy * Mxp + x over the kept y-modes: a
// tile is TX consecutive q, so every global access is a run of TX complex.
// Stored fields arrive by 16-byte asynchronous copies; the vorticity is formed
// in registers as the first FFT stage loads it.  The inverse pass stores its
// last stage's results from registers.
//
// zinv (Algorithm 1 step c, first half): loads the state u_hat, forms
//   omega_hat = i k x u_hat on the fly (Sec. 2.4: grad -> i k), fills the
//   dropped z-modes with zeros and transforms back to z grid points:
//   W[f] = iFFT_z(field f), f < 3 velocity, f = 3..5 vorticity.
// zfwd (Algorithm 1 steps d, e): transforms W[0..2] (the nonlinear term
//   after its x and y transforms) along z keeping only the 2/3-rule modes,
//   scales by 1/N, applies the Leray projection N <- N - k (k.N)/|k|^2
//   (Eq. PNST_UP_pressure_poisson_eqn in Fourier space) and
//   mode 0: the integrating-factor AB2 update
//     u^{n+1} = E1 u^n + c_now E1 N^n - c_old E2 N^{n-1},  N^{n-1} <- N^n,
//     with c_now = dt (1 + r/2), c_old = dt r/2 (first step: dt, 0) and the
//     separable factors E1 = e^{-nu |k|^2 dt}, E2 = e^{-nu |k|^2 (dt + dt_prev)};
//   mode 1: u_hat = N (initial condition), history cleared.
//   The k = 0 mode is held at u_inf (N(0) = 0) unless the mean is free.
#include "fft.cuh"
#include "kernels.cuh"

namespace flusi {

namespace {

constexpr int kThreadsInv = 256;
constexpr int kThreadsFwd = 384;
// complex elements per tile: 64 KiB (inverse) and 96 KiB (forward, 3 components)
template <typename T> constexpr int cap_zi() { return sizeof(T) == 4 ? 8192 : 4096; }
template <typename T> constexpr int cap_zf() { return sizeof(T) == 4 ? 12288 : 6144; }

template <typename T>
__global__ void __launch_bounds__(kThreadsInv)
k_zinv(const cplx<T>* __restrict__ U, cplx<T>* __restrict__ W, Geom g, FftPlan plan,
       const double2* __restrict__ tw, const int* __restrict__ pos, int nf, int lgTX,
       const StepState* __restrict__ st)
{
    if (st && st->status != 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TX = 1 << lgTX;
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* tws = buf + (g.nz << lgTX);
    int* sinv = reinterpret_cast<int*>(tws + g.nz);
    const int Q = g.My * g.Mxp;
    const int q0 = blockIdx.x * TX;
    const size_t Ustride = (size_t)g.Mz * Q;           // between components of U
    const size_t Wplane = (size_t)g.ny * g.Mxp;        // between z planes of W
    load_tables<T>(tws, nullptr, tw, nullptr, g.nz, 0);
    load_inverse_pos(sinv, pos, g.nz);

    // this thread's column is fixed across the strided loops (TX divides blockDim)
    const int tx = threadIdx.x & (TX - 1);
    const int q = q0 + tx;
    const bool qok = q < Q;
    const int jy = qok ? q / g.Mxp : 0;
    const int x = qok ? q - jy * g.Mxp : 0;
    const bool kept = qok && x < g.Mx;
    const T two_pi = T(6.283185307179586476925286766559);
    const T kx = two_pi * T(x) / T(g.Lx);
    const T ky = two_pi * T(mode_of(jy, g.Ky)) / T(g.Ly);
    const int nz = g.nz, Kz = g.Kz, Mz = g.Mz;
    __syncthreads();

    for (int f = 0; f < nf; ++f) {
        cplx<T>* out = W + (size_t)f * nz * Wplane + (qok ? q : 0);
        auto store = [&](int z, cplx<T> v) {
            if (qok) out[(size_t)z * Wplane] = v;
        };
        if (f < 3) {
            // U's row padding (x >= Mx) is zero
            // 16-byte asynchronous copies of VEC adjacent columns
            constexpr int VEC = 16 / sizeof(cplx<T>);
            const int lpr = TX / VEC;                  // lanes per row of the tile
            const int rstep = kThreadsInv / lpr;
            const int txv = (threadIdx.x % lpr) * VEC;
            const int qv = q0 + txv;                   // Q is a multiple of VEC
            for (int s = threadIdx.x / lpr; s < nz; s += rstep) {
                const int jz = s <= Kz ? s : (s >= nz - Kz ? s - nz + Mz : -1);
                cplx<T>* dst = buf + (s << lgTX) + txv;
                if (qv < Q && jz >= 0) {
                    cp_async_16(dst, U + f * Ustride + (size_t)jz * Q + qv);
                } else {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) dst[v] = mkc<T>(0, 0);
                }
            }
            cp_async_wait_all();
            __syncthreads();
            fft_dif_out<T, true>(buf, TX, TX, plan, tws, sinv, store);
        } else {
            // omega = i (k x u) from two velocity components
            const int cA = f == 3 ? 2 : f == 4 ? 0 : 1;
            const int cB = f == 3 ? 1 : f == 4 ? 2 : 0;
            const T kb = f == 3 ? T(0) : f == 4 ? kx : ky;   // kz enters per mode
            const T ka = f == 3 ? ky : f == 4 ? T(0) : kx;
            const cplx<T>* srcA = U + cA * Ustride + (qok ? q : 0);
            const cplx<T>* srcB = U + cB * Ustride + (qok ? q : 0);
            auto load = [&](int s) -> cplx<T> {
                const int jz = s <= Kz ? s : (s >= nz - Kz ? s - nz + Mz : -1);
                if (!kept || jz < 0) return mkc<T>(0, 0);
                const cplx<T> a = srcA[(size_t)jz * Q], b = srcB[(size_t)jz * Q];
                const T kz = two_pi * T(mode_of(jz, Kz)) / T(g.Lz);
                // f=3: ky uz - kz uy; f=4: kz ux - kx uz; f=5: kx uy - ky ux
                const T k1 = f == 4 ? kz : ka;
                const T k2 = f == 3 ? kz : kb;
                return cmuli(mkc<T>(k1 * a.x - k2 * b.x, k1 * a.y - k2 * b.y));
            };
            fft_dif_io<T, true>(buf, TX, TX, plan, tws, sinv, load, store);
        }
        __syncthreads();
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreadsFwd, 2)
k_zfwd(const cplx<T>* __restrict__ W, cplx<T>* __restrict__ U, cplx<T>* __restrict__ H, Geom g,
       FftPlan plan, const double2* __restrict__ tw, const int* __restrict__ pos, int lgTX,
       ZfwdExtra ex, const StepState* __restrict__ st)
{
    if (st && st->status != 0) return;
    if (MODE == 0 && ex.coef->skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TX = 1 << lgTX, C = 3 * TX;
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* tws = buf + g.nz * C;
    int* spos = reinterpret_cast<int*>(tws + g.nz);
    const int Q = g.My * g.Mxp;
    const int q0 = blockIdx.x * TX;
    const size_t Wplane = (size_t)g.ny * g.Mxp;
    const size_t Ustride = (size_t)g.Mz * Q;
    const int nz = g.nz;
    load_tables<T>(tws, spos, tw, pos, nz, nz);
    __syncthreads();
    {
        constexpr int VEC = 16 / sizeof(cplx<T>);
        const int lpr = C / VEC;               // lanes per row of the tile
        const int rstep = kThreadsFwd / lpr;
        const int col = (threadIdx.x % lpr) * VEC;
        const int c = col >> lgTX, q = q0 + (col & (TX - 1));
        for (int z = threadIdx.x / lpr; z < nz; z += rstep) {
            cplx<T>* dst = buf + z * C + col;
            if (q < Q) {
                cp_async_16(dst, W + ((size_t)c * nz + z) * Wplane + q);
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) dst[v] = mkc<T>(0, 0);
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();
    fft_dif<T, false>(buf, C, C, plan, tws);

    const T two_pi = T(6.283185307179586476925286766559);
    const T inv_n = T(1.0 / ((double)g.nx * g.ny * g.nz));
    double c_now = 0, c_old = 0;
    int first = 1;
    if (MODE == 0) {
        c_now = ex.coef->c_now;
        c_old = ex.coef->c_old;
        first = ex.coef->first;
    }
    const T cn = T(c_now), co = T(c_old);
    const double* E1x = ex.etab;
    const double* E1y = E1x + g.Mx;
    const double* E1z = E1y + g.My;
    const double* E2x = E1z + g.Mz;
    const double* E2y = E2x + g.Mx;
    const double* E2z = E2y + g.My;

    // two modes per batch: the twelve global loads of U and H are issued before
    // any of the arithmetic that needs them
    constexpr int kB = 2;
    const int total = g.Mz << lgTX;
    for (int e0 = threadIdx.x; e0 < total; e0 += kB * kThreadsFwd) {
        cplx<T> uo[kB][3], ho[kB][3];
        int jzs[kB], qs[kB];
#pragma unroll
        for (int bb = 0; bb < kB; ++bb) {
            const int e = e0 + bb * kThreadsFwd;
            const int jz = e >> lgTX, q = q0 + (e & (TX - 1));
            jzs[bb] = jz;
            qs[bb] = (e < total && q < Q) ? q : -1;
            const size_t o = (size_t)jz * Q + q;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                uo[bb][c] = mkc<T>(0, 0);
                ho[bb][c] = mkc<T>(0, 0);
                if (qs[bb] >= 0) {
                    if (MODE == 0) uo[bb][c] = U[c * Ustride + o];
                    if (MODE == 0 && !first) ho[bb][c] = H[c * Ustride + o];
                }
            }
        }
#pragma unroll
        for (int bb = 0; bb < kB; ++bb) {
            if (qs[bb] < 0) continue;
            const int jz = jzs[bb], q = qs[bb], tx = q - q0;
            const int jy = q / g.Mxp, x = q - jy * g.Mxp;
            const size_t o = (size_t)jz * Q + q;
            if (x >= g.Mx) {   // row padding stays zero
                for (int c = 0; c < 3; ++c) {
                    U[c * Ustride + o] = mkc<T>(0, 0);
                    H[c * Ustride + o] = mkc<T>(0, 0);
                }
                continue;
            }
            const int s = spos[slot_of(jz, g.Kz, nz)];
            cplx<T> N[3];
            for (int c = 0; c < 3; ++c) N[c] = cscale(buf[s * C + c * TX + tx], inv_n);
            const T kx = two_pi * T(x) / T(g.Lx);
            const T ky = two_pi * T(mode_of(jy, g.Ky)) / T(g.Ly);
            const T kz = two_pi * T(mode_of(jz, g.Kz)) / T(g.Lz);
            const T k2 = kx * kx + ky * ky + kz * kz;
            const bool zero_mode = (x == 0 && jy == 0 && jz == 0);
            if (!zero_mode) {
                const T inv_k2 = T(1) / k2;
                const T kNr = (kx * N[0].x + ky * N[1].x + kz * N[2].x) * inv_k2;
                const T kNi = (kx * N[0].y + ky * N[1].y + kz * N[2].y) * inv_k2;
                const T kk[3] = {kx, ky, kz};
                for (int c = 0; c < 3; ++c) {
                    N[c].x -= kk[c] * kNr;
                    N[c].y -= kk[c] * kNi;
                }
            } else if (!ex.mean_free) {
                N[0] = N[1] = N[2] = mkc<T>(0, 0);
            }
            if (MODE == 0) {
                // products of the per-axis factors in the state precision
                const T e1 = T(E1x[x]) * T(E1y[jy]) * T(E1z[jz]);
                const T e2 = first ? T(0) : T(E2x[x]) * T(E2y[jy]) * T(E2z[jz]);
                for (int c = 0; c < 3; ++c) {
                    const cplx<T> u = uo[bb][c], h = ho[bb][c];
                    cplx<T> r;
                    r.x = e1 * (u.x + cn * N[c].x) - co * e2 * h.x;
                    r.y = e1 * (u.y + cn * N[c].y) - co * e2 * h.y;
                    U[c * Ustride + o] = r;
                    H[c * Ustride + o] = N[c];
                }
            } else {
                for (int c = 0; c < 3; ++c) {
                    cplx<T> u = N[c];
                    if (zero_mode && !ex.mean_free) u = mkc<T>(T(ex.u_inf[c]), 0);
                    U[c * Ustride + o] = u;
                    H[c * Ustride + o] = mkc<T>(0, 0);
                }
            }
        }
    }
}

template <typename T> int zinv_tx(const Geom& g)
{
    int TX = sizeof(T) == 4 ? 16 : 8;
    while (TX > 1 && g.nz * TX > cap_zi<T>()) TX >>= 1;
    while (2 * TX * g.nz <= cap_zi<T>() && 2 * TX <= 64) TX *= 2;
    return TX;
}

template <typename T> int zfwd_tx(const Geom& g)
{
    int TX = sizeof(T) == 4 ? 8 : 4;
    while (TX > 1 && g.nz * 3 * TX > cap_zf<T>()) TX >>= 1;
    while (2 * TX * 3 * g.nz <= cap_zf<T>() && 2 * TX <= 32) TX *= 2;
    return TX;
}

template <typename T>
cudaError_t launch_zi(const void* U, void* W, const Geom& g, const FftPlan& plan, const double2* tw,
                      const int* pos, int nf, const StepState* st, cudaStream_t s)
{
    const int TX = zinv_tx<T>(g);
    if (g.nz * TX > cap_zi<T>() || kThreadsInv % TX != 0) return cudaErrorInvalidValue;
    const int blocks = ceil_div(g.My * g.Mxp, TX);
    const size_t smem = sizeof(cplx<T>) * ((size_t)g.nz + (size_t)g.nz * TX) + sizeof(int) * g.nz;
    k_zinv<T><<<blocks, kThreadsInv, smem, s>>>((const cplx<T>*)U, (cplx<T>*)W, g, plan, tw, pos, nf,
                                                __builtin_ctz(TX), st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zf(int mode, const void* W, void* U, void* H, const Geom& g, const FftPlan& plan,
                      const double2* tw, const int* pos, const ZfwdExtra& ex, const StepState* st,
                      cudaStream_t s)
{
    const int TX = zfwd_tx<T>(g);
    if (g.nz * 3 * TX > cap_zf<T>() || kThreadsFwd % (3 * TX) != 0) return cudaErrorInvalidValue;
    const int blocks = ceil_div(g.My * g.Mxp, TX);
    const size_t smem = sizeof(cplx<T>) * ((size_t)g.nz + (size_t)g.nz * 3 * TX) + sizeof(int) * g.nz;
    if (mode == 0)
        k_zfwd<T, 0><<<blocks, kThreadsFwd, smem, s>>>((const cplx<T>*)W, (cplx<T>*)U, (cplx<T>*)H, g,
                                                       plan, tw, pos, __builtin_ctz(TX), ex, st);
    else
        k_zfwd<T, 1><<<blocks, kThreadsFwd, smem, s>>>((const cplx<T>*)W, (cplx<T>*)U, (cplx<T>*)H, g,
                                                       plan, tw, pos, __builtin_ctz(TX), ex, st);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_zinv(int fp64, const void* U, void* W, const Geom& g, const FftPlan& plan,
                        const double2* tw, const int* pos, int nf, const StepState* st,
                        cudaStream_t s)
{
    return fp64 ? launch_zi<double>(U, W, g, plan, tw, pos, nf, st, s)
                : launch_zi<float>(U, W, g, plan, tw, pos, nf, st, s);
}

cudaError_t launch_zfwd(int fp64, int mode, const void* W, void* U, void* H, const Geom& g,
                        const FftPlan& plan, const double2* tw, const int* pos, const ZfwdExtra& ex,
                        const StepState* st, cudaStream_t s)
{
    return fp64 ? launch_zf<double>(mode, W, U, H, g, plan, tw, pos, ex, st, s)
                : launch_zf<float>(mode, W, U, H, g, plan, tw, pos, ex, st, s);
}

cudaError_t configure_zpass()
{
    const int big = 120 * 1024;
    cudaError_t e;
#define FLUSI_SMEM(fn) \
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    FLUSI_SMEM(k_zinv<float>)
    FLUSI_SMEM(k_zinv<double>)
    FLUSI_SMEM((k_zfwd<float, 0>))
    FLUSI_SMEM((k_zfwd<float, 1>))
    FLUSI_SMEM((k_zfwd<double, 0>))
    FLUSI_SMEM((k_zfwd<double, 1>))
#undef FLUSI_SMEM
    return cudaSuccess;
}

}  // namespace flusi

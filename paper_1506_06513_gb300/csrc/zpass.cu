// z-axis transform passes, fused with the spectral pointwise work.
//
// Columns along z are indexed by q = jy * Mxp + x over the kept y-modes: a
// tile is TX consecutive q, so every global access is a run of TX complex.
// Stored fields arrive by 16-byte asynchronous copies; the vorticity is formed
// in registers as the first FFT stage loads it.  The inverse pass stores its
// last stage's results from registers.
//
// zinv (Algorithm 1 step c, first half): loads the state u_hat, fills the
//   dropped z-modes with zeros and transforms back to z grid points:
//   W[f] = iFFT_z(field f), f < 3 velocity, f = 3..5 the vorticity
//   omega_hat = i k x u_hat (Sec. 2.4: grad -> i k), of which only the kz
//   terms take transforms of their own (five transforms for six fields).
// zfwd (Algorithm 1 step c, second half): transforms W[0..2] (the nonlinear
//   term after its x and y transforms) along z and keeps only the 2/3-rule
//   modes, in the state layout, in the free vorticity part of W.
// zupdate (Algorithm 1 steps d, e), a streaming pass over the kept modes:
//   scales by 1/N, applies the Leray projection N <- N - k (k.N)/|k|^2
//   (Eq. PNST_UP_pressure_poisson_eqn in Fourier space) and
//   mode 0: the integrating-factor AB2 update
//     u^{n+1} = E1 u^n + c_now E1 N^n - c_old E2 N^{n-1},  N^{n-1} <- N^n,
//     with c_now = dt (1 + r/2), c_old = dt r/2 (first step: dt, 0) and the
//     separable factors E1 = e^{-nu |k|^2 dt}, E2 = e^{-nu |k|^2 (dt + dt_prev)};
//   mode 1: u_hat = N (initial condition), history cleared.
//   The k = 0 mode is held at u_inf (N(0) = 0) unless the mean is free.
#include <algorithm>

#include "fft.cuh"
#include "kernels.cuh"

namespace flusi {

namespace {

constexpr int kThreadsInv = 256;
// complex elements per column tile (64 KiB)
template <typename T> constexpr int cap_zi() { return sizeof(T) == 4 ? 8192 : 4096; }
inline size_t ceil_div_sz(size_t a, size_t b) { return (a + b - 1) / b; }

// A row store marked streaming (st.global.cs: likely read once, so evicted
// from L2 first), for outputs the kernel does not read back.
template <typename T, int V>
__device__ __forceinline__ void st_row_cs(cplx<T>* p, const cplx<T>* o)
{
    if constexpr (V % 2 == 0 && sizeof(T) == 4) {
#pragma unroll
        for (int c = 0; c < V; c += 2)
            __stcs(reinterpret_cast<float4*>(p + c), make_float4(o[c].x, o[c].y, o[c + 1].x, o[c + 1].y));
    } else {
#pragma unroll
        for (int c = 0; c < V; ++c) __stcs(reinterpret_cast<double2*>(p + c), make_double2(o[c].x, o[c].y));
    }
}

// L2 eviction policies of the inverse pass: a velocity component is read
// twice by the same block with one transform between, and the transformed
// u_z and u_x are read back as side rows a phase or two after they are
// written, so those lines are kept (evict_last) until their last use, which
// marks them evict_first.
constexpr int kZinvHints = 2;   // 0 none, 1 the velocity loads, 2 also the side rows

__device__ __forceinline__ unsigned long long l2_evict_last()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ unsigned long long l2_evict_first()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// tma_load_3d with an L2 eviction policy for the lines it reads
__device__ __forceinline__ void tma_load_3d_hint(void* dst, const void* map, int c0, int c1, int c2,
                                                 unsigned long long* bar, unsigned long long policy)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;\n" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

template <typename T, int V>
__device__ __forceinline__ void st_row_hint(cplx<T>* p, const cplx<T>* o, unsigned long long pol)
{
    if constexpr (V % 2 == 0 && sizeof(T) == 4) {
#pragma unroll
        for (int c = 0; c < V; c += 2)
            asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p + c), "f"(o[c].x),
                         "f"(o[c].y), "f"(o[c + 1].x), "f"(o[c + 1].y), "l"(pol)
                         : "memory");
    } else {
#pragma unroll
        for (int c = 0; c < V; ++c)
            asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p + c), "d"(double(o[c].x)),
                         "d"(double(o[c].y)), "l"(pol)
                         : "memory");
    }
}

// Stores of k_zinv.  Plain: the transformed column to `out`.
template <typename T, int V> struct ZStore {
    cplx<T>* out;
    size_t plane;
    bool ok;
    bool keep = false;                 // the lines are read back later (evict_last)
    unsigned long long pol = 0;
    __device__ __forceinline__ void operator()(int z, const cplx<T>* v) const
    {
        if (!ok) return;
        if (keep) st_row_hint<T, V>(out + (size_t)z * plane, v, pol);
        else st_row<T, V>(out + (size_t)z * plane, v);
    }
};

// A vorticity component from a transform v and a side row a of an already
// transformed velocity component: out_c = i (cv v + ca a) per column, and v
// itself to out_v when that is set (both streaming stores: nothing reads
// them back here).  The side rows were written earlier in the same kernel by
// this block, so they are read through L2 (ld.cg).
template <typename T, int V> struct ZCurlStore {
    cplx<T>* out_v;
    cplx<T>* out_c;
    const cplx<T>* side;
    size_t plane;
    T cv[V], ca[V];
    bool ok;
    bool last = false;                 // the side rows' last use (evict_first)
    unsigned long long pol = 0;
    __device__ __forceinline__ void aux(int z, cplx<T>* a) const
    {
        if (!ok) {
#pragma unroll
            for (int c = 0; c < V; ++c) a[c] = mkc<T>(0, 0);
            return;
        }
        const cplx<T>* p = side + (size_t)z * plane;
        if (last) {
            if constexpr (sizeof(T) == 4 && V % 2 == 0) {
#pragma unroll
                for (int c = 0; c < V; c += 2) {
                    float4 q;
                    asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                                 : "=f"(q.x), "=f"(q.y), "=f"(q.z), "=f"(q.w)
                                 : "l"(p + c), "l"(pol));
                    a[c] = mkc<T>(q.x, q.y);
                    a[c + 1] = mkc<T>(q.z, q.w);
                }
            } else {
#pragma unroll
                for (int c = 0; c < V; ++c) {
                    double qx, qy;
                    asm volatile("ld.global.cg.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                                 : "=d"(qx), "=d"(qy)
                                 : "l"(p + c), "l"(pol));
                    a[c] = mkc<T>(T(qx), T(qy));
                }
            }
            return;
        }
        if constexpr (sizeof(T) == 4 && V % 2 == 0) {
#pragma unroll
            for (int c = 0; c < V; c += 2) {
                const float4 q = __ldcg(reinterpret_cast<const float4*>(p + c));
                a[c] = mkc<T>(q.x, q.y);
                a[c + 1] = mkc<T>(q.z, q.w);
            }
        } else {
#pragma unroll
            for (int c = 0; c < V; ++c) {
                const double2 q = __ldcg(reinterpret_cast<const double2*>(p + c));
                a[c] = mkc<T>(T(q.x), T(q.y));
            }
        }
    }
    __device__ __forceinline__ void put(int z, const cplx<T>* v, const cplx<T>* a) const
    {
        if (!ok) return;
        if (out_v) st_row_cs<T, V>(out_v + (size_t)z * plane, v);
        cplx<T> r[V];
#pragma unroll
        for (int c = 0; c < V; ++c)
            r[c] = cmuli(mkc<T>(cv[c] * v[c].x + ca[c] * a[c].x, cv[c] * v[c].y + ca[c] * a[c].y));
        st_row_cs<T, V>(out_c + (size_t)z * plane, r);
    }
};

// First-stage loads of kz times the staged tile (in place: the first stage
// reads and writes the same rows of each butterfly).
template <typename T, int V> struct ZLoadKz {
    const cplx<T>* buf;
    int ld, col, nz, Kz;
    T kunit;                                   // 2 pi / Lz
    __device__ __forceinline__ void operator()(int s, cplx<T>* r) const
    {
        ld_row<T, V>(buf + s * ld + col, r);
        const T kz = kunit * T(s <= Kz ? s : s - nz);   // rows of dropped modes are zero
#pragma unroll
        for (int c = 0; c < V; ++c) r[c] = cscale(r[c], kz);
    }
};

// The z transform is linear and kx, ky are constant along a column, so of
// omega = i k x u only the kz terms need transforms of their own:
//   W2 = Fz u_z;  W4 = i (Fz(kz u_x) - kx W2);  W0 = Fz u_x;
//   W3 = i (ky W2 - Fz(kz u_y));  W1 = Fz u_y, W5 = i (kx W1 - ky W0)
// five transforms, each velocity component read from DRAM once (its second
// read follows the first), the side rows read back from L2.  nf = 3: the
// velocity alone.
template <typename T, bool TMA, bool R16>
__global__ void __launch_bounds__(kThreadsInv, sizeof(T) == 4 ? 3 : 1)
k_zinv(const cplx<T>* __restrict__ U, cplx<T>* __restrict__ W, Geom g, FftPlan plan,
       const double2* __restrict__ tw, const int* __restrict__ pos, int nf, int lgTX,
       const StepState* __restrict__ st, const __grid_constant__ CUtensorMap umap, int bh, int* err,
       const Member* __restrict__ mb)
{
    if (mb) {   // one member of an ensemble batch (never with TMA)
        U = static_cast<const cplx<T>*>(mb[blockIdx.z].U);
        W = static_cast<cplx<T>*>(mb[blockIdx.z].W);
        st = mb[blockIdx.z].st;
        err = &mb[blockIdx.z].st->status;
    }
    if (st && st->status != 0) return;
    if (TMA && *(volatile int*)err != 0) return;   // a TMA wait gave up earlier
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int TX = 1 << lgTX;
    // the tile at a 128-byte boundary of shared memory (TMA destinations)
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));
    cplx<T>* tws = buf + (g.nz << lgTX);
    rowidx_t* sinv = reinterpret_cast<rowidx_t*>(tws + g.nz);
    const int Q = g.My * g.Mxp;
    const int q0 = blockIdx.x * TX;
    const size_t Ustride = (size_t)g.Mz * Q;           // between components of U
    const size_t Wplane = (size_t)g.ny * g.Mxp;        // between z planes of W
    const size_t Wfield = (size_t)g.nz * Wplane;       // between fields of W
    const int nz = g.nz, Kz = g.Kz, Mz = g.Mz;

    // the TMA boxes of one velocity component into buf (thread 0): modes
    // 0..Kz to rows 0..Kz, Kz..2Kz to rows nz-Kz-1..nz-1, the duplicate row
    // cleared with the dropped modes after the wait.
    // hint: 0 none, 1 keep the lines for a second read, 2 their last read
    __shared__ unsigned long long bar;
    unsigned phase = 0;
    auto issue = [&](int comp, int hint) {
        const unsigned box = (unsigned)(((size_t)bh << lgTX) * sizeof(cplx<T>));
        const int kb = (Kz + 1) / bh;   // boxes per part
        mbar_expect_tx(&bar, 2 * kb * box);
        if (kZinvHints >= 1 && hint) {
            const unsigned long long pol = hint == 1 ? l2_evict_last() : l2_evict_first();
            for (int b = 0; b < kb; ++b) {
                tma_load_3d_hint(buf + ((size_t)(b * bh) << lgTX), &umap, 2 * q0, b * bh, comp, &bar, pol);
                tma_load_3d_hint(buf + ((size_t)(nz - Kz - 1 + b * bh) << lgTX), &umap, 2 * q0, Kz + b * bh,
                                 comp, &bar, pol);
            }
        } else {
            for (int b = 0; b < kb; ++b) {
                tma_load_3d(buf + ((size_t)(b * bh) << lgTX), &umap, 2 * q0, b * bh, comp, &bar);
                tma_load_3d(buf + ((size_t)(nz - Kz - 1 + b * bh) << lgTX), &umap, 2 * q0, Kz + b * bh, comp,
                            &bar);
            }
        }
    };
    // the first component's boxes go out before the block loads its tables
    // (u_x for the velocity alone, u_z when the vorticity is formed too)
    bool pre_issued = false;
    if constexpr (TMA) {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            issue(nf < 6 ? 0 : 2, nf < 6 ? 0 : 2);
        }
        pre_issued = true;
    }
    load_tables<T>(tws, nullptr, tw, nullptr, g.nz, 0);
    load_inverse_pos(sinv, pos, g.nz);

    // this thread's two adjacent columns in the transform stages (fft_run's map
    // with V = 2); Mxp is a multiple of 4, so both lie in one row jy
    constexpr int V = 2;
    const int tx = (threadIdx.x % (TX / V)) * V;
    const int q = q0 + tx;
    const bool qok = q < Q;
    const int jy = qok ? q / g.Mxp : 0;
    const int x = qok ? q - jy * g.Mxp : 0;
    const T two_pi = T(6.283185307179586476925286766559);
    const T kxv[V] = {two_pi * T(x) / T(g.Lx), two_pi * T(x + 1) / T(g.Lx)};
    const T ky = two_pi * T(mode_of(jy, g.Ky)) / T(g.Ly);
    cplx<T>* Wq = W + (qok ? q : 0);
    __syncthreads();   // tables, and the barrier's initialisation before any thread waits on it

    // component `comp` of the tile into buf: kept modes at their z rows, zeros
    // elsewhere (U's row padding x >= Mx is zero); by two TMA boxes (modes
    // 0..Kz to rows 0..Kz, Kz..2Kz to rows nz-Kz-1..nz-1, the duplicate row
    // cleared with the dropped modes) or by 16-byte asynchronous copies.
    // false: a TMA wait gave up (status set; the block must leave).
    // hint: 0 none, 1 keep the lines for a second read, 2 their last read
    auto stage_in = [&](int comp, int hint) -> bool {
        if constexpr (TMA) {
            if (threadIdx.x == 0 && !pre_issued) {
                // earlier generic writes to buf before the asynchronous proxy's
                fence_proxy_async();
                issue(comp, hint);
            }
            pre_issued = false;
            const bool ok = mbar_wait(&bar, phase);
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicCAS(err, 0, (int)FLUSI_ETIMEOUT);
                mbar_wait(&bar, phase);   // let the copies in flight land
                return false;
            }
            phase ^= 1;
            const int nzero = (nz - Mz) << lgTX;
            cplx<T>* gap = buf + ((size_t)(Kz + 1) << lgTX);
            for (int i = threadIdx.x; i < nzero; i += kThreadsInv) gap[i] = mkc<T>(0, 0);
            __syncthreads();
            return true;
        }
        constexpr int VEC = 16 / sizeof(cplx<T>);
        const int lpr = TX / VEC;                  // lanes per row of the tile
        const int rstep = kThreadsInv / lpr;
        const int txv = (threadIdx.x % lpr) * VEC;
        const int qv = q0 + txv;                   // Q is a multiple of VEC
        for (int s = threadIdx.x / lpr; s < nz; s += rstep) {
            const int jz = s <= Kz ? s : (s >= nz - Kz ? s - nz + Mz : -1);
            cplx<T>* dst = buf + (s << lgTX) + txv;
            if (qv < Q && jz >= 0) {
                cp_async_16(dst, U + comp * Ustride + (size_t)jz * Q + qv);
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) dst[v] = mkc<T>(0, 0);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        return true;
    };
    // keep: the transformed component is read back as side rows (evict_last)
    auto velocity = [&](int comp, int hint, bool keep) -> bool {
        if (!stage_in(comp, hint)) return false;
        ZStore<T, V> out{Wq + comp * Wfield, Wplane, qok};
        if (kZinvHints >= 2 && keep) {
            out.keep = true;
            out.pol = l2_evict_last();
        }
        fft_dif_out<T, true, V, false, R16>(buf, TX, TX, plan, tws, sinv, out);
        __syncthreads();
        return true;
    };
    const ZLoadKz<T, V> kz_load{buf, TX, tx, nz, Kz, two_pi / T(g.Lz)};

    if (nf < 6) {
        for (int f = 0; f < nf; ++f)
            if (!velocity(f, 0, false)) return;
        return;
    }
    if (!velocity(2, 2, true)) return;
    {   // W4 = i (Fz(kz u_x) - kx W2)
        if (!stage_in(0, 1)) return;
        ZCurlStore<T, V> w4{nullptr, Wq + 4 * Wfield, Wq + 2 * Wfield, Wplane, {T(1), T(1)},
                            {-kxv[0], -kxv[1]}, qok};
        fft_dif_io<T, true, V, true, R16>(buf, TX, TX, plan, tws, sinv, kz_load, w4);
        __syncthreads();
    }
    if (!velocity(0, 2, true)) return;
    {   // W3 = i (ky W2 - Fz(kz u_y))
        if (!stage_in(1, 1)) return;
        ZCurlStore<T, V> w3{nullptr, Wq + 3 * Wfield, Wq + 2 * Wfield, Wplane, {T(-1), T(-1)}, {ky, ky}, qok};
        if (kZinvHints >= 2) {
            w3.last = true;
            w3.pol = l2_evict_first();
        }
        fft_dif_io<T, true, V, true, R16>(buf, TX, TX, plan, tws, sinv, kz_load, w3);
        __syncthreads();
    }
    {   // W1 = Fz u_y and W5 = i (kx W1 - ky W0)
        if (!stage_in(1, 2)) return;
        ZCurlStore<T, V> w5{Wq + 1 * Wfield, Wq + 5 * Wfield, Wq, Wplane, {kxv[0], kxv[1]}, {-ky, -ky}, qok};
        if (kZinvHints >= 2) {
            w5.last = true;
            w5.pol = l2_evict_first();
        }
        fft_dif_out<T, true, V, true, R16>(buf, TX, TX, plan, tws, sinv, w5);
    }
}

// Forward z transform of one component of a column tile: TX consecutive
// columns q of W[c] (A form, all nz rows) in by 16-byte asynchronous copies,
// the kept modes jz (2/3 rule) back into rows jz < Mz of the same columns
// (in place: a tile reads all of its rows before its first barrier).
template <typename T, bool TMA, bool R16>
__global__ void __launch_bounds__(kThreadsInv)
k_zfwd(cplx<T>* __restrict__ W, Geom g, FftPlan plan, const double2* __restrict__ tw,
       const int* __restrict__ pos, int lgTX, const StepState* __restrict__ st,
       const __grid_constant__ CUtensorMap wmap, int bh, int* err, const Member* __restrict__ mb)
{
    if (mb) {   // one member of an ensemble batch (never with TMA)
        W = static_cast<cplx<T>*>(mb[blockIdx.z].W);
        st = mb[blockIdx.z].st;
        err = &mb[blockIdx.z].st->status;
    }
    if (st && st->status != 0) return;
    if (TMA && *(volatile int*)err != 0) return;   // a TMA wait gave up earlier
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int TX = 1 << lgTX;
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));
    cplx<T>* tws = buf + (g.nz << lgTX);
    rowidx_t* sinv = reinterpret_cast<rowidx_t*>(tws + g.nz);
    const int Q = g.My * g.Mxp, nz = g.nz, Kz = g.Kz, Mz = g.Mz;
    const int nqb = ceil_div(Q, TX);
    const int c = blockIdx.x / nqb, q0 = (blockIdx.x - c * nqb) * TX;
    const size_t Wplane = (size_t)g.ny * g.Mxp;
    // the tile's TMA boxes (nz / bh boxes of bh rows of TX columns) go out
    // first, in flight while the block loads its tables
    __shared__ unsigned long long bar;
    if constexpr (TMA) {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            const unsigned box = (unsigned)(((size_t)bh << lgTX) * sizeof(cplx<T>));
            const int nb = nz / bh;
            mbar_expect_tx(&bar, nb * box);
            for (int b = 0; b < nb; ++b) tma_load_3d(buf + ((size_t)(b * bh) << lgTX), &wmap, 2 * q0, b * bh, c, &bar);
        }
    }
    load_tables<T>(tws, nullptr, tw, nullptr, nz, 0);
    load_inverse_pos(sinv, pos, nz);
    if constexpr (TMA) {
        __syncthreads();   // the barrier's initialisation, before any thread waits on it
        const bool ok = mbar_wait(&bar, 0);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicCAS(err, 0, (int)FLUSI_ETIMEOUT);
            mbar_wait(&bar, 0);
            return;
        }
    } else {
        constexpr int VEC = 16 / sizeof(cplx<T>);
        const int lpr = TX / VEC;              // lanes per row of the tile
        const int rstep = kThreadsInv / lpr;
        const int txv = (threadIdx.x % lpr) * VEC;
        const int qv = q0 + txv;               // Q is a multiple of VEC
        const cplx<T>* src = W + (size_t)c * nz * Wplane + qv;
        for (int z = threadIdx.x / lpr; z < nz; z += rstep) {
            cplx<T>* dst = buf + (z << lgTX) + txv;
            if (qv < Q) {
                cp_async_16(dst, src + (size_t)z * Wplane);
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) dst[v] = mkc<T>(0, 0);
            }
        }
        cp_async_wait_all();
    }
    __syncthreads();
    constexpr int V = 2;                       // adjacent columns per thread
    const int q = q0 + (threadIdx.x % (TX / V)) * V;
    const bool qok = q < Q;                    // Q is a multiple of 4
    cplx<T>* out = W + (size_t)c * nz * Wplane + (qok ? q : 0);
    auto store = [&](int f, const cplx<T>* v) {   // keep modes |m| <= Kz only
        const int jz = f <= Kz ? f : (f >= nz - Kz ? f - nz + Mz : -1);
        if (qok && jz >= 0) st_row<T, V>(out + (size_t)jz * Wplane, v);
    };
    fft_dif_out<T, false, V, false, R16>(buf, TX, TX, plan, tws, sinv, store);
}

// Pointwise spectral update over the kept modes, VEC adjacent columns per
// thread: N = N^ / N_points (the kept modes that k_zfwd left in rows jz of
// W[0..2]); with a sponge, N += -(i k x V^)/(C_sp |k|^2) with V^ the kept
// modes of chi_sp omega in W[3..5] (Sec. 2.3, read as a damping of the
// vorticity, zero at k = 0); Leray projection N <- N - k (k.N)/|k|^2, then
//   mode 0: IF-AB2  u^{n+1} = E1 (u^n + c_now N) - c_old E2 N^{n-1},  N^{n-1} <- N
//   mode 1: u_hat = N (the initial condition), history cleared.
//   modes 2..5: RK4 stage 1..4 with R = N - nu |k|^2 u_s, u_s the stage state
//     (U for stage 1, the stage buffer Ut after), H the accumulator:
//     1: H = R, Ut = U + dt/2 R;  2: H += 2R, Ut = U + dt/2 R;
//     3: H += 2R, Ut = U + dt R;  4: U += dt/6 (H + R).
// The mean (k = 0) is held at u_inf unless it is free.  Row padding x >= Mx
// is never written (it is zero from the workspace reset on).
template <typename T, int MODE, bool SPONGE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
k_zupdate(const cplx<T>* __restrict__ Wn, cplx<T>* __restrict__ U, cplx<T>* __restrict__ H, Geom g,
          ZfwdExtra ex, const StepState* __restrict__ st, const Member* __restrict__ mb)
{
    if (mb) {   // one member of an ensemble batch
        const Member& m = mb[blockIdx.z];
        Wn = static_cast<const cplx<T>*>(m.W);
        U = static_cast<cplx<T>*>(m.U);
        H = static_cast<cplx<T>*>(m.H);
        st = m.st;
        ex.coef = m.coef;
        ex.etab = m.etab;
        g.nu = m.nu;
    }
    if (st && st->status != 0) return;
    constexpr bool RK = MODE >= 2;
    constexpr int STAGE = MODE - 1;        // RK4 stage 1..4
    if ((MODE == 0 || RK) && ex.coef->skip) return;
    constexpr int VEC = 16 / sizeof(cplx<T>);
    cplx<T>* __restrict__ Ut = (cplx<T>*)ex.stage;
    const int Q = g.My * g.Mxp;
    const size_t S = (size_t)g.Mz * Q;     // values per component
    const size_t groups = S / VEC;         // Mxp is a multiple of 4
    const size_t Wplane = (size_t)g.ny * g.Mxp, Wfield = (size_t)g.nz * Wplane;
    constexpr bool sponge = (MODE == 0 || RK) && SPONGE;
    const T dt = RK ? T(ex.coef->dt) : T(0), nu = T(g.nu);
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
    // the factor tables in T: FP64, then their FP32 copy (written together)
    const int Mt = g.Mx + g.My + g.Mz;
    const T* E1x = sizeof(T) == 8 ? reinterpret_cast<const T*>(ex.etab)
                                  : reinterpret_cast<const T*>(ex.etab + 2 * Mt);
    const T* E1y = E1x + g.Mx;
    const T* E1z = E1y + g.My;
    const T* E2x = E1z + g.Mz;
    const T* E2y = E2x + g.Mx;
    const T* E2z = E2y + g.My;
    for (size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x; gi < groups;
         gi += (size_t)gridDim.x * blockDim.x) {
        const size_t o = gi * VEC;
        const int jz = (int)(o / Q), q = (int)(o - (size_t)jz * Q);
        const int jy = q / g.Mxp, x0 = q - jy * g.Mxp;
        if (x0 >= g.Mx) continue;
        cplx<T> n[3][VEC], u[3][VEC], h[3][VEC], sv[3][VEC], us[3][VEC];
        const size_t on = (size_t)jz * Wplane + q;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t oc = c * S + o;
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                n[c][v] = Wn[c * Wfield + on + v];
                sv[c][v] = sponge ? Wn[(3 + c) * Wfield + on + v] : mkc<T>(0, 0);
                u[c][v] = mkc<T>(0, 0);
                h[c][v] = mkc<T>(0, 0);
                us[c][v] = mkc<T>(0, 0);
                if (MODE == 0 || RK) u[c][v] = U[oc + v];
                if ((MODE == 0 && !first) || (RK && STAGE > 1)) h[c][v] = H[oc + v];
                if (RK && STAGE > 1) us[c][v] = Ut[oc + v];
            }
        }
        const T ky = two_pi * T(mode_of(jy, g.Ky)) / T(g.Ly);
        const T kz = two_pi * T(mode_of(jz, g.Kz)) / T(g.Lz);
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int x = x0 + v;
            if (x >= g.Mx) break;
            cplx<T> N[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) N[c] = cscale(n[c][v], inv_n);
            const T kx = two_pi * T(x) / T(g.Lx);
            const bool zero_mode = (x == 0 && jy == 0 && jz == 0);
            if (sponge && !zero_mode) {
                // -(i k x V)/(C_sp |k|^2): real part Im(k x V)/(C k^2), imaginary -Re(k x V)/(C k^2)
                cplx<T> Vs[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) Vs[c] = cscale(sv[c][v], inv_n);
                const T f = T(1) / (T(ex.sponge_c) * (kx * kx + ky * ky + kz * kz));
                const cplx<T> cr[3] = {csub(cscale(Vs[2], ky), cscale(Vs[1], kz)),
                                       csub(cscale(Vs[0], kz), cscale(Vs[2], kx)),
                                       csub(cscale(Vs[1], kx), cscale(Vs[0], ky))};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    N[c].x += f * cr[c].y;
                    N[c].y -= f * cr[c].x;
                }
            }
            if (!zero_mode) {
                const T inv_k2 = T(1) / (kx * kx + ky * ky + kz * kz);
                const T kNr = (kx * N[0].x + ky * N[1].x + kz * N[2].x) * inv_k2;
                const T kNi = (kx * N[0].y + ky * N[1].y + kz * N[2].y) * inv_k2;
                const T kk[3] = {kx, ky, kz};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    N[c].x -= kk[c] * kNr;
                    N[c].y -= kk[c] * kNi;
                }
            } else if (!ex.mean_free) {
                N[0] = N[1] = N[2] = mkc<T>(0, 0);
            }
            const size_t ov = o + v;
            if (MODE == 0) {
                // products of the per-axis factors in the state precision
                const T e1 = E1x[x] * E1y[jy] * E1z[jz];
                const T e2 = first ? T(0) : E2x[x] * E2y[jy] * E2z[jz];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    cplx<T> r;
                    r.x = e1 * (u[c][v].x + cn * N[c].x) - co * e2 * h[c][v].x;
                    r.y = e1 * (u[c][v].y + cn * N[c].y) - co * e2 * h[c][v].y;
                    U[c * S + ov] = r;
                    H[c * S + ov] = N[c];
                }
            } else if (RK) {
                const T k2 = kx * kx + ky * ky + kz * kz;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const cplx<T> ust = STAGE == 1 ? u[c][v] : us[c][v];
                    const cplx<T> R = csub(N[c], cscale(ust, nu * k2));
                    if (STAGE == 1) {
                        H[c * S + ov] = R;
                        Ut[c * S + ov] = cadd(u[c][v], cscale(R, T(0.5) * dt));
                    } else if (STAGE == 2 || STAGE == 3) {
                        H[c * S + ov] = cadd(h[c][v], cscale(R, T(2)));
                        Ut[c * S + ov] = cadd(u[c][v], cscale(R, STAGE == 2 ? T(0.5) * dt : dt));
                    } else {
                        U[c * S + ov] = cadd(u[c][v], cscale(cadd(h[c][v], R), dt / T(6)));
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    cplx<T> r = N[c];
                    if (zero_mode && !ex.mean_free) r = mkc<T>(T(ex.u_inf[c]), 0);
                    U[c * S + ov] = r;
                    H[c * S + ov] = mkc<T>(0, 0);
                }
            }
        }
    }
}

template <typename T> int zinv_tx(const Geom& g)
{
    const int cmax = g.zcols > 0 ? g.zcols : 64;   // columns per tile
    int TX = sizeof(T) == 4 ? 16 : 8;
    while (TX > 1 && (g.nz * TX > cap_zi<T>() || TX > cmax)) TX >>= 1;
    while (2 * TX * g.nz <= cap_zi<T>() && 2 * TX <= cmax) TX *= 2;
    return TX;
}

template <typename T>
cudaError_t launch_zi(const void* U, void* W, const Geom& g, const FftPlan& plan, const double2* tw,
                      const int* pos, int nf, const StepState* st, const CUtensorMap* map, int bh, int* err,
                      cudaStream_t s)
{
    const int TX = zinv_tx<T>(g);
    if (g.nz * TX > cap_zi<T>() || kThreadsInv % TX != 0) return cudaErrorInvalidValue;
    const int blocks = ceil_div(g.My * g.Mxp, TX);
    const size_t smem = sizeof(cplx<T>) * ((size_t)g.nz + (size_t)g.nz * TX) + sizeof(rowidx_t) * g.nz + 128;
    const cplx<T>* u = (const cplx<T>*)U;
    cplx<T>* w = (cplx<T>*)W;
    const bool tma = map && bh > 0 && err;
    CUtensorMap none{};
    const CUtensorMap& m = tma ? *map : none;
    const int lg = __builtin_ctz(TX);
    // the inverse z pass is built without radix-16 stages (its plan has none)
    if (plan_has_radix16(plan)) return cudaErrorInvalidValue;
    const Batch& B = current_batch();
    const dim3 grid(blocks, 1, B.n);
    if (tma && !B.mb)
        k_zinv<T, true, false><<<grid, kThreadsInv, smem, s>>>(u, w, g, plan, tw, pos, nf, lg, st, m, bh, err, nullptr);
    else
        k_zinv<T, false, false><<<grid, kThreadsInv, smem, s>>>(u, w, g, plan, tw, pos, nf, lg, st, m, 0, err, B.mb);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zf(void* W, int nf, const Geom& g, const FftPlan& plan, const double2* tw,
                      const int* pos, const StepState* st, const CUtensorMap* map, int bh, int* err,
                      cudaStream_t s)
{
    const int TX = zinv_tx<T>(g);
    if (g.nz * TX > cap_zi<T>() || kThreadsInv % TX != 0 || nf < 1 || nf > 6) return cudaErrorInvalidValue;
    const int blocks = nf * ceil_div(g.My * g.Mxp, TX);
    const size_t smem = sizeof(cplx<T>) * ((size_t)g.nz + (size_t)g.nz * TX) + sizeof(rowidx_t) * g.nz + 128;
    cplx<T>* w = (cplx<T>*)W;
    const bool tma = map && bh > 0 && err;
    CUtensorMap none{};
    const CUtensorMap& m = tma ? *map : none;
    const int lg = __builtin_ctz(TX);
    const Batch& B = current_batch();
    const dim3 grid(blocks, 1, B.n);
    const bool use_tma = tma && !B.mb;
    if (plan_has_radix16(plan)) {
        if (use_tma) k_zfwd<T, true, true><<<grid, kThreadsInv, smem, s>>>(w, g, plan, tw, pos, lg, st, m, bh, err, nullptr);
        else k_zfwd<T, false, true><<<grid, kThreadsInv, smem, s>>>(w, g, plan, tw, pos, lg, st, m, 0, err, B.mb);
    } else {
        if (use_tma) k_zfwd<T, true, false><<<grid, kThreadsInv, smem, s>>>(w, g, plan, tw, pos, lg, st, m, bh, err, nullptr);
        else k_zfwd<T, false, false><<<grid, kThreadsInv, smem, s>>>(w, g, plan, tw, pos, lg, st, m, 0, err, B.mb);
    }
    return cudaGetLastError();
}

// Tensor maps of the z sources: (2 Q reals, rows, components) with row stride
// rs and component stride cs (complex values); box (2 TX, bh, 1).  The
// inverse reads the kept rows of U (bh = Kz + 1, two boxes), the forward all
// nz rows of W (bh = nz or 256).  Boxes over 256 rows, destinations off a
// 128-byte boundary or a failed encoding leave that source to 16-byte copies.
template <typename T> cudaError_t prepare_z(void* U, void* Ut, void* W, const Geom& g, ZMaps* m)
{
    m->u_bh = m->ut_bh = m->w_bh = 0;
    const TensorMapEncoder encode = tensor_map_encoder();
    if (!encode) return cudaSuccess;   // no encoder: 16-byte copies
    const int TX = zinv_tx<T>(g);
    const size_t row_bytes = (size_t)TX * sizeof(cplx<T>);
    const size_t Q = (size_t)g.My * g.Mxp;
    const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    auto make = [&](CUtensorMap* map, void* base, size_t rows, size_t ncomp, size_t rs, size_t cs, int bh) {
        if (!base || bh <= 0 || bh > 256 || reinterpret_cast<uintptr_t>(base) % 16 != 0) return 0;
        const cuuint64_t dims[3] = {(cuuint64_t)(2 * Q), (cuuint64_t)rows, (cuuint64_t)ncomp};
        const cuuint64_t strides[2] = {(cuuint64_t)(rs * sizeof(cplx<T>)), (cuuint64_t)(cs * sizeof(cplx<T>))};
        const cuuint32_t box[3] = {(cuuint32_t)(2 * TX), (cuuint32_t)bh, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        const CUresult r = encode(map, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        return r == CUDA_SUCCESS ? bh : 0;
    };
    const int ibh = inverse_box_rows(g.nz, g.Kz, row_bytes);
    m->u_bh = make(&m->u, U, g.Mz, 3, Q, (size_t)g.Mz * Q, ibh);
    m->ut_bh = make(&m->ut, Ut, g.Mz, 3, Q, (size_t)g.Mz * Q, ibh);
    int fbh = g.nz <= 256 ? g.nz : (g.nz % 256 == 0 ? 256 : 0);
    if (((size_t)fbh * row_bytes) % 128 != 0) fbh = 0;
    const size_t Wplane = (size_t)g.ny * g.Mxp;
    m->w_bh = make(&m->w, W, g.nz, 6, Wplane, (size_t)g.nz * Wplane, fbh);
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_zu(int mode, const void* Nh, void* U, void* H, const Geom& g, const ZfwdExtra& ex,
                      const StepState* st, cudaStream_t s)
{
    constexpr int VEC = 16 / sizeof(cplx<T>);
    const size_t groups = (size_t)g.Mz * g.My * g.Mxp / VEC;
    const int blocks = (int)std::min<size_t>(ceil_div_sz(groups, 256), (size_t)152 * 64);
    const cplx<T>* n = (const cplx<T>*)Nh;
    cplx<T>* u = (cplx<T>*)U;
    cplx<T>* hh = (cplx<T>*)H;
    const bool sp = ex.sponge_c > 0 && mode != 1;
    const Batch& B = current_batch();
    const dim3 grid(blocks, 1, B.n);
#define FLUSI_ZU(M)                                                              \
    if (sp)                                                                      \
        k_zupdate<T, M, true><<<grid, 256, 0, s>>>(n, u, hh, g, ex, st, B.mb);   \
    else                                                                         \
        k_zupdate<T, M, false><<<grid, 256, 0, s>>>(n, u, hh, g, ex, st, B.mb);
    switch (mode) {
    case 0: FLUSI_ZU(0) break;
    case 1: k_zupdate<T, 1, false><<<grid, 256, 0, s>>>(n, u, hh, g, ex, st, B.mb); break;
    case 2: FLUSI_ZU(2) break;
    case 3: FLUSI_ZU(3) break;
    case 4: FLUSI_ZU(4) break;
    case 5: FLUSI_ZU(5) break;
    default: return cudaErrorInvalidValue;
    }
#undef FLUSI_ZU
    return cudaGetLastError();
}

}  // namespace

int zpass_tile_cols(int fp64, const Geom& g) { return fp64 ? zinv_tx<double>(g) : zinv_tx<float>(g); }

cudaError_t prepare_zmaps(int fp64, void* U, void* Ut, void* W, const Geom& g, ZMaps* maps)
{
    return fp64 ? prepare_z<double>(U, Ut, W, g, maps) : prepare_z<float>(U, Ut, W, g, maps);
}

cudaError_t launch_zinv(int fp64, const void* U, void* W, const Geom& g, const FftPlan& plan,
                        const double2* tw, const int* pos, int nf, const StepState* st,
                        const CUtensorMap* map, int bh, int* err, cudaStream_t s)
{
    return fp64 ? launch_zi<double>(U, W, g, plan, tw, pos, nf, st, map, bh, err, s)
                : launch_zi<float>(U, W, g, plan, tw, pos, nf, st, map, bh, err, s);
}

cudaError_t launch_zfwd(int fp64, void* W, int nf, const Geom& g, const FftPlan& plan,
                        const double2* tw, const int* pos, const StepState* st,
                        const CUtensorMap* map, int bh, int* err, cudaStream_t s)
{
    return fp64 ? launch_zf<double>(W, nf, g, plan, tw, pos, st, map, bh, err, s)
                : launch_zf<float>(W, nf, g, plan, tw, pos, st, map, bh, err, s);
}

cudaError_t launch_zupdate(int fp64, int mode, const void* W, void* U, void* H, const Geom& g,
                           const ZfwdExtra& ex, const StepState* st, cudaStream_t s)
{
    return fp64 ? launch_zu<double>(mode, W, U, H, g, ex, st, s)
                : launch_zu<float>(mode, W, U, H, g, ex, st, s);
}

// max over the kept modes of |k . u_hat| and of |k| |u_hat|, in FP64 from a
// state of precision T: the discrete divergence that the Leray projection
// (Eq. PNST_UP_pressure_poisson_eqn) removes, and its scale.  Non-negative
// doubles order like their bit patterns, so the maxima are kept with 64-bit
// integer atomics in out[0], out[1] (cleared by the caller).
template <typename T>
__global__ void __launch_bounds__(256) k_divergence(const cplx<T>* __restrict__ U, Geom g,
                                                     unsigned long long* __restrict__ out)
{
    const int Q = g.My * g.Mxp;
    const size_t S = (size_t)g.Mz * Q;
    const double two_pi = 6.283185307179586476925286766559;
    double dmax = 0.0, kumax = 0.0;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < S; o += (size_t)gridDim.x * blockDim.x) {
        const int jz = (int)(o / Q), q = (int)(o - (size_t)jz * Q);
        const int jy = q / g.Mxp, jx = q - jy * g.Mxp;
        if (jx >= g.Mx) continue;
        const double k[3] = {two_pi * jx / g.Lx, two_pi * mode_of(jy, g.Ky) / g.Ly, two_pi * mode_of(jz, g.Kz) / g.Lz};
        double dr = 0.0, di = 0.0, uu = 0.0;
        for (int c = 0; c < 3; ++c) {
            const cplx<T> u = U[c * S + o];
            dr += k[c] * double(u.x);
            di += k[c] * double(u.y);
            uu += double(u.x) * double(u.x) + double(u.y) * double(u.y);
        }
        const double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        dmax = fmax(dmax, sqrt(dr * dr + di * di));
        kumax = fmax(kumax, sqrt(kk * uu));
        if (!(dr == dr && di == di && uu == uu)) dmax = __longlong_as_double(0x7ff8000000000000LL);
    }
    for (int off = 16; off > 0; off >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
        kumax = fmax(kumax, __shfl_xor_sync(0xffffffffu, kumax, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(dmax));
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(kumax));
    }
}

cudaError_t launch_divergence(int fp64, const void* U, const Geom& g, unsigned long long* out, cudaStream_t s)
{
    const size_t S = (size_t)g.Mz * g.My * g.Mxp;
    const int grid = (int)std::min<size_t>(1024, (S + 255) / 256);
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), s);
    if (e) return e;
    if (fp64) k_divergence<double><<<grid, 256, 0, s>>>(static_cast<const cplx<double>*>(U), g, out);
    else k_divergence<float><<<grid, 256, 0, s>>>(static_cast<const cplx<float>*>(U), g, out);
    return cudaGetLastError();
}

cudaError_t configure_zpass()
{
    const int big = 120 * 1024;
    cudaError_t e;
#define FLUSI_SMEM(fn) \
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
#define FLUSI_SMEM_Z(T, R16)                  \
    FLUSI_SMEM((k_zfwd<T, false, R16>))       \
    FLUSI_SMEM((k_zfwd<T, true, R16>))
    FLUSI_SMEM_Z(float, false)
    FLUSI_SMEM_Z(double, false)
    FLUSI_SMEM_Z(float, true)
    FLUSI_SMEM_Z(double, true)
#undef FLUSI_SMEM_Z
    FLUSI_SMEM((k_zinv<float, false, false>))
    FLUSI_SMEM((k_zinv<float, true, false>))
    FLUSI_SMEM((k_zinv<double, false, false>))
    FLUSI_SMEM((k_zinv<double, true, false>))
#undef FLUSI_SMEM
    return cudaSuccess;
}

}  // namespace flusi

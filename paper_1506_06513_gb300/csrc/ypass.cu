// y-axis transform pass (part of the 3-D FFTs of Algorithm 1 step c).
//
// A tile is TX consecutive x-mode columns of NP consecutive z planes of one
// component: every global access is a run of TX complex values (128 bytes).
// Rows arrive by TMA: one thread issues the tile's boxes of a 3-D tensor map
// of W (dims: x reals, planes of all components, y rows, so a box lands in
// shared memory row-major as the transform wants it) against an mbarrier;
// where no map fits (box heights over 256 rows) by 16-byte asynchronous
// copies.  All FFT stages but the last run in shared memory and the last one
// stores its results to global memory from registers; the pass works in place
// (a tile reads all of its rows before its first barrier and writes after its
// last).
//   inverse: rows j < My hold the kept y-modes 0..Ky, -Ky..-1 -> ny grid rows
//   forward: ny grid rows -> the My kept y-modes (2/3 rule, pruned output)
#include <algorithm>

#include <cooperative_groups.h>

#include "fft.cuh"
#include "kernels.cuh"

namespace flusi {

namespace {

constexpr int kThreads = 256;
// complex elements per tile (64 KiB of shared memory)
template <typename T> constexpr int tile_elems() { return sizeof(T) == 4 ? 8192 : 4096; }

template <typename T, bool INV, bool TMA, bool R16>
__global__ void __launch_bounds__(kThreads)
k_ypass(cplx<T>* __restrict__ W, Geom g, FftPlan plan, const double2* __restrict__ tw,
        const int* __restrict__ pos, int ncomp, int lgTX, int lgNP, const StepState* __restrict__ st,
        const __grid_constant__ CUtensorMap tmap, int bh, int* err, const Member* __restrict__ mb)
{
    if (mb) {   // one member of an ensemble batch (never with TMA)
        W = static_cast<cplx<T>*>(mb[blockIdx.z].W);
        st = mb[blockIdx.z].st;
        err = &mb[blockIdx.z].st->status;
    }
    if (st && st->status != 0) return;
    // after a TMA wait gave up, the remaining blocks leave at once
    if (TMA && *(volatile int*)err != 0) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int TX = 1 << lgTX, lgC = lgTX + lgNP, C = 1 << lgC;
    // the tile at a 128-byte boundary of shared memory (TMA destinations)
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));
    cplx<T>* tws = buf + (g.ny << lgC);
    rowidx_t* sinv = reinterpret_cast<rowidx_t*>(tws + g.ny);
    const int nxb = ceil_div(g.Mxp, TX), nzb = ceil_div(g.nz, 1 << lgNP);
    int b = blockIdx.x;
    const int xb = b % nxb;
    b /= nxb;
    const int zb = b % nzb;
    const int c = b / nzb;
    if (c >= ncomp) return;
    const int x0 = xb * TX, z0 = zb << lgNP;
    const size_t plane = (size_t)g.ny * g.Mxp;
    cplx<T>* base = W + (size_t)c * g.nz * plane;
    const int ny = g.ny, My = g.My, Ky = g.Ky;

    // the tile's TMA boxes go out first, so that they are in flight while the
    // block loads its twiddle and digit-reversal tables
    __shared__ unsigned long long bar;
    if constexpr (TMA) {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            // coordinates: x in reals (2 x0 sizeof(T) is a multiple of 128
            // bytes), plane c nz + z0, row; a box is bh rows of NP planes of TX
            // columns
            const int xr = 2 * x0, pl = c * g.nz + z0;
            const unsigned box = (unsigned)(((size_t)bh << lgC) * sizeof(cplx<T>));
            if (INV) {
                // modes 0..Ky to rows 0..Ky; modes Ky..2Ky to rows ny-Ky-1..ny-1
                // (kb boxes of bh = (Ky + 1)/kb rows each; row ny-Ky-1 is
                // cleared below)
                const int kb = (Ky + 1) / bh;
                mbar_expect_tx(&bar, 2 * kb * box);
                for (int q = 0; q < kb; ++q) {
                    tma_load_3d(buf + ((size_t)(q * bh) << lgC), &tmap, xr, pl, q * bh, &bar);
                    tma_load_3d(buf + ((size_t)(ny - Ky - 1 + q * bh) << lgC), &tmap, xr, pl, Ky + q * bh, &bar);
                }
            } else {
                const int nb = ny / bh;
                mbar_expect_tx(&bar, nb * box);
                for (int q = 0; q < nb; ++q) tma_load_3d(buf + ((size_t)(q * bh) << lgC), &tmap, xr, pl, q * bh, &bar);
            }
        }
    }
    load_tables<T>(tws, nullptr, tw, nullptr, g.ny, 0);
    load_inverse_pos(sinv, pos, g.ny);
    const int ld = g.Mxp;   // row stride; a plane holds fewer than 2^31 values
    // this thread's two adjacent columns in the transform stages (fft_run's
    // map with V = 2; TX is even, so both lie in one plane)
    constexpr int V = 2;
    const int col = (threadIdx.x % (C / V)) * V;
    const int z = z0 + (col >> lgTX), x = x0 + (col & (TX - 1));
    const bool colok = z < g.nz && x < g.Mxp;   // Mxp is a multiple of 4
    cplx<T>* gcol = base + (size_t)(colok ? z : 0) * plane + (colok ? x : 0);
    if constexpr (TMA) {
        __syncthreads();   // the barrier's initialisation, before any thread waits on it
        const bool ok = mbar_wait(&bar, 0);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicCAS(err, 0, (int)FLUSI_ETIMEOUT);
            mbar_wait(&bar, 0);   // let the copies in flight land before the block leaves
            return;
        }
        if (INV) {
            // grid slots of the dropped modes are zero
            const int nzero = (ny - My) << lgC;
            cplx<T>* gap = buf + ((size_t)(Ky + 1) << lgC);
            for (int i = threadIdx.x; i < nzero; i += kThreads) gap[i] = mkc<T>(0, 0);
        }
    } else {
        // 16-byte asynchronous copies: each lane moves VEC adjacent columns
        constexpr int VEC = 16 / sizeof(cplx<T>);
        const int lanes_per_row = C / VEC;
        const int rstep = kThreads / lanes_per_row;
        const int cv = (threadIdx.x % lanes_per_row) * VEC;
        const int zv = z0 + (cv >> lgTX), xv = x0 + (cv & (TX - 1));
        const bool okv = zv < g.nz && xv < g.Mxp;   // Mxp and TX are multiples of VEC
        const cplx<T>* gv = base + (size_t)(okv ? zv : 0) * plane + (okv ? xv : 0);
        for (int s = threadIdx.x / lanes_per_row; s < ny; s += rstep) {
            // grid slot s <- row j(s) (inverse: modes 0..Ky, -Ky..-1 in rows j < My)
            const int j = INV ? (s <= Ky ? s : (s >= ny - Ky ? s - ny + My : -1)) : s;
            cplx<T>* dst = buf + (s << lgC) + cv;
            if (okv && j >= 0) {
                cp_async_16(dst, gv + j * ld);
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) dst[v] = mkc<T>(0, 0);
            }
        }
        cp_async_wait_all();
    }
    __syncthreads();
    if (INV) {
        auto store = [&](int f, const cplx<T>* v) {
            if (colok) st_row<T, V>(gcol + f * ld, v);
        };
        fft_dif_out<T, true, V, false, R16>(buf, C, C, plan, tws, sinv, store);
    } else {
        auto store = [&](int f, const cplx<T>* v) {   // keep modes |m| <= Ky only
            const int r = f <= Ky ? f : (f >= ny - Ky ? f - ny + My : -1);
            if (colok && r >= 0) st_row<T, V>(gcol + r * ld, v);
        };
        fft_dif_out<T, false, V, false, R16>(buf, C, C, plan, tws, sinv, store);
    }
}

// Paired variant (a cluster of two CTAs per tile), for lengths where a
// one-CTA tile of 128-byte rows would not fit its shared memory.  With
// n = 2 m, the CTA of cluster rank p holds the grid rows 2 s + p (s < m) of
// the tile, and transforms them at length m, every stage in shared memory
// (row pos_h[f] then holds frequency f).  The two halves are joined by one
// radix-2 decimation-in-time step: X[f] = E[f] + w_n^f O[f] and
// X[f + m] = E[f] - w_n^f O[f] (conjugate twiddles for the inverse), E from
// rank 0, O from rank 1, read across the cluster through distributed shared
// memory; rank p computes and stores the frequencies f + p m.  The loads are
// 16-byte asynchronous copies.  Both CTAs take every cluster barrier on every
// path (no early return), so neither can wait on a partner that has left.
template <typename T, bool INV, bool R16>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads)
k_ypass_pair(cplx<T>* __restrict__ W, Geom g, FftPlan plan_h, const double2* __restrict__ tw,
             const int* __restrict__ pos_h, int ncomp, int lgTX, int lgNP)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int p = (int)cluster.block_rank();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int TX = 1 << lgTX, lgC = lgTX + lgNP, C = 1 << lgC;
    const int ny = g.ny, m = ny / 2, My = g.My, Ky = g.Ky;
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));
    cplx<T>* tws = buf + ((size_t)m << lgC);     // w_m^j = w_n^(2j), j < m
    int* spos = reinterpret_cast<int*>(tws + m);  // row of frequency f after the length-m transform
    const int nxb = ceil_div(g.Mxp, TX), nzb = ceil_div(g.nz, 1 << lgNP);
    int b = blockIdx.x / 2;
    const int xb = b % nxb;
    b /= nxb;
    const int zb = b % nzb;
    const int c = min(b / nzb, ncomp - 1);        // the grid holds whole clusters of real tiles
    const int x0 = xb * TX, z0 = zb << lgNP;
    const size_t plane = (size_t)ny * g.Mxp;
    cplx<T>* base = W + (size_t)c * g.nz * plane;
    const int ld = g.Mxp;

    for (int i = threadIdx.x; i < m; i += kThreads) {
        const double2 w = tw[2 * i];
        tws[i] = mkc<T>(T(w.x), T(w.y));
        spos[i] = pos_h[i];
    }
    // rows 2 s + p of the tile: VEC adjacent columns per lane
    {
        constexpr int VEC = 16 / sizeof(cplx<T>);
        const int lanes_per_row = C / VEC;
        const int rstep = kThreads / lanes_per_row;
        const int cv = (threadIdx.x % lanes_per_row) * VEC;
        const int zv = z0 + (cv >> lgTX), xv = x0 + (cv & (TX - 1));
        const bool okv = zv < g.nz && xv < g.Mxp;   // Mxp and TX are multiples of VEC
        const cplx<T>* gv = base + (size_t)(okv ? zv : 0) * plane + (okv ? xv : 0);
        for (int sr = threadIdx.x / lanes_per_row; sr < m; sr += rstep) {
            const int s2 = 2 * sr + p;
            // inverse: grid slot s2 <- kept mode row j (modes 0..Ky, -Ky..-1 in rows j < My)
            const int j = INV ? (s2 <= Ky ? s2 : (s2 >= ny - Ky ? s2 - ny + My : -1)) : s2;
            cplx<T>* dst = buf + ((size_t)sr << lgC) + cv;
            if (okv && j >= 0) {
                cp_async_16(dst, gv + (size_t)j * ld);
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) dst[v] = mkc<T>(0, 0);
            }
        }
        cp_async_wait_all();
    }
    __syncthreads();
    fft_run<T, INV, true, 2, R16>(buf, C, C, plan_h, tws, 0, plan_h.nst);   // ends with a block barrier
    cluster.sync();   // both halves transformed: the partner's buffer is readable

    constexpr int V = 2;
    const int G = C / V, P = kThreads / G, col = (threadIdx.x % G) * V, jt = threadIdx.x / G;
    const int z = z0 + (col >> lgTX), x = x0 + (col & (TX - 1));
    const bool colok = z < g.nz && x < g.Mxp && b / nzb < ncomp;
    cplx<T>* gcol = base + (size_t)(colok ? z : 0) * plane + (colok ? x : 0);
    const cplx<T>* other = cluster.map_shared_rank(buf, p ^ 1);
    for (int f = jt; f < m; f += P) {
        const int r = spos[f];
        cplx<T> a[V], o[V];
        ld_row<T, V>(buf + ((size_t)r << lgC) + col, a);
        ld_row<T, V>(other + ((size_t)r << lgC) + col, o);
        const double2 wd = tw[f];
        const cplx<T> w = mkc<T>(T(wd.x), INV ? -T(wd.y) : T(wd.y));
        cplx<T> out[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            // own half: E for rank 0, O for rank 1
            const cplx<T> E = p ? o[v] : a[v], O = p ? a[v] : o[v];
            const cplx<T> t = cmul(w, O);
            out[v] = p ? csub(E, t) : cadd(E, t);
        }
        const int fr = f + p * m;   // the frequency this CTA stores
        if (INV) {
            if (colok) st_row<T, V>(gcol + (size_t)fr * ld, out);
        } else {
            const int r2 = fr <= Ky ? fr : (fr >= ny - Ky ? fr - ny + My : -1);
            if (colok && r2 >= 0) st_row<T, V>(gcol + (size_t)r2 * ld, out);
        }
    }
    cluster.sync();   // the partner has read this buffer
}

struct YTile {
    int lgTX, lgNP, blocks;
    size_t smem;
};

template <typename T> YTile y_tile(const Geom& g, int ncomp)
{
    YTile t;
    const int cap = tile_elems<T>();
    const int cmax = g.ycols > 0 ? g.ycols : kThreads;   // columns per tile
    int TX = sizeof(T) == 4 ? 16 : 8;                     // 128-byte runs
    while (TX > 1 && (g.ny * TX > cap || TX > cmax)) TX >>= 1;
    int NP = 1;
    while (2 * NP * TX * g.ny <= cap && 2 * NP * TX <= std::min(kThreads, cmax) && 2 * NP <= g.nz) NP *= 2;
    t.lgTX = __builtin_ctz(TX);
    t.lgNP = __builtin_ctz(NP);
    t.blocks = ceil_div(g.Mxp, TX) * ceil_div(g.nz, NP) * ncomp;
    t.smem = sizeof(cplx<T>) * ((size_t)g.ny + (size_t)g.ny * TX * NP) + sizeof(rowidx_t) * g.ny + 128;
    return t;
}

template <typename T, bool R16>
cudaError_t launch_y2(bool inverse, cplx<T>* w, const Geom& g, const FftPlan& plan, const double2* tw,
                      const int* pos, int ncomp, const StepState* st, const YMaps* maps, int* err,
                      const YTile& t, cudaStream_t s)
{
    const Batch& B = current_batch();
    const int bh = maps && !B.mb ? (inverse ? maps->inv_bh : maps->fwd_bh) : 0;
    const dim3 grid(t.blocks, 1, B.n);
    if (bh > 0 && err) {
        const CUtensorMap& m = inverse ? maps->inv : maps->fwd;
        if (inverse)
            k_ypass<T, true, true, R16><<<grid, kThreads, t.smem, s>>>(w, g, plan, tw, pos, ncomp, t.lgTX,
                                                                        t.lgNP, st, m, bh, err, B.mb);
        else
            k_ypass<T, false, true, R16><<<grid, kThreads, t.smem, s>>>(w, g, plan, tw, pos, ncomp, t.lgTX,
                                                                         t.lgNP, st, m, bh, err, B.mb);
    } else {
        CUtensorMap none{};
        if (inverse)
            k_ypass<T, true, false, R16><<<grid, kThreads, t.smem, s>>>(w, g, plan, tw, pos, ncomp, t.lgTX,
                                                                         t.lgNP, st, none, 0, err, B.mb);
        else
            k_ypass<T, false, false, R16><<<grid, kThreads, t.smem, s>>>(w, g, plan, tw, pos, ncomp, t.lgTX,
                                                                          t.lgNP, st, none, 0, err, B.mb);
    }
    return cudaGetLastError();
}

// The paired kernel's tile: a one-CTA tile for the half length m = ny / 2.
template <typename T> YTile y_tile_pair(const Geom& g, int ncomp)
{
    Geom h = g;
    h.ny = g.ny / 2;
    YTile t = y_tile<T>(h, ncomp);
    t.blocks *= 2;
    t.smem = sizeof(cplx<T>) * ((size_t)h.ny << (t.lgTX + t.lgNP)) + (sizeof(cplx<T>) + sizeof(int)) * h.ny + 128;
    return t;
}

// whether the y passes take the paired kernel: ypair 1 and ny even (at
// least 16).  It keeps 128-byte rows at n = 1024, but measured slower than
// one CTA per tile on 512^3 and 1024^3 (the second pass through shared
// memory, the 16-byte copies in place of TMA boxes and the reads across the
// cluster cost more than the narrower rows), so it is an autotuner candidate,
// not a default.
template <typename T> bool y_paired(const Geom& g) { return g.ypair == 1 && g.ny % 2 == 0 && g.ny >= 16; }

template <typename T>
cudaError_t launch_y(bool inverse, void* W, const Geom& g, const FftPlan& plan, const double2* tw,
                     const int* pos, int ncomp, const StepState* st, const YMaps* maps, int* err,
                     const FftPlan* half, const int* pos_half, cudaStream_t s)
{
    if (half && pos_half && y_paired<T>(g)) {
        if (current_batch().mb) return cudaErrorInvalidValue;   // batches take the one-CTA tiles
        const YTile t = y_tile_pair<T>(g, ncomp);
        if (((size_t)(g.ny / 2) << (t.lgTX + t.lgNP)) > (size_t)tile_elems<T>() || half->n != g.ny / 2)
            return cudaErrorInvalidValue;
        cplx<T>* w = (cplx<T>*)W;
        const bool r16 = plan_has_radix16(*half);
#define FLUSI_PAIR(I, R)                                                                                  \
    k_ypass_pair<T, I, R><<<t.blocks, kThreads, t.smem, s>>>(w, g, *half, tw, pos_half, ncomp, t.lgTX, t.lgNP)
        if (inverse) {
            if (r16) FLUSI_PAIR(true, true);
            else FLUSI_PAIR(true, false);
        } else {
            if (r16) FLUSI_PAIR(false, true);
            else FLUSI_PAIR(false, false);
        }
#undef FLUSI_PAIR
        return cudaGetLastError();
    }
    YTile t = y_tile<T>(g, ncomp);
    if ((size_t)g.ny << (t.lgTX + t.lgNP) > (size_t)tile_elems<T>()) return cudaErrorInvalidValue;
    cplx<T>* w = (cplx<T>*)W;
    return plan_has_radix16(plan) ? launch_y2<T, true>(inverse, w, g, plan, tw, pos, ncomp, st, maps, err, t, s)
                                  : launch_y2<T, false>(inverse, w, g, plan, tw, pos, ncomp, st, maps, err, t, s);
}

// Tensor maps of W for the y tiles: dims (2 Mxp reals, 6 nz planes, ny rows)
// with strides (plane ny Mxp, row Mxp complex); boxes (2 TX, NP, bh).  A box
// height over 256 (the hardware's limit) leaves that direction to 16-byte
// copies, as does a failed encoding.
template <typename T> cudaError_t prepare_y(void* W, const Geom& g, YMaps* m)
{
    m->inv_bh = m->fwd_bh = 0;
    const TensorMapEncoder encode = tensor_map_encoder();
    if (!encode) return cudaSuccess;   // no encoder: 16-byte copies
    if (reinterpret_cast<uintptr_t>(W) % 16 != 0) return cudaSuccess;
    const YTile t = y_tile<T>(g, 1);
    const cuuint64_t dims[3] = {(cuuint64_t)2 * g.Mxp, (cuuint64_t)6 * g.nz, (cuuint64_t)g.ny};
    const cuuint64_t strides[2] = {(cuuint64_t)g.ny * g.Mxp * sizeof(cplx<T>), (cuuint64_t)g.Mxp * sizeof(cplx<T>)};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    auto make = [&](CUtensorMap* map, int bh) {
        if (bh <= 0 || bh > 256) return 0;
        const cuuint32_t box[3] = {(cuuint32_t)(2 << t.lgTX), (cuuint32_t)(1 << t.lgNP), (cuuint32_t)bh};
        const CUresult r = encode(map, dt, 3, W, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        return r == CUDA_SUCCESS ? bh : 0;
    };
    // every box destination (row offsets of the tile) on a 128-byte boundary
    const size_t row_bytes = sizeof(cplx<T>) << (t.lgTX + t.lgNP);
    m->inv_bh = make(&m->inv, inverse_box_rows(g.ny, g.Ky, row_bytes));
    int fbh = g.ny <= 256 ? g.ny : (g.ny % 256 == 0 ? 256 : 0);
    if (((size_t)fbh * row_bytes) % 128 != 0) fbh = 0;
    m->fwd_bh = make(&m->fwd, fbh);
    return cudaSuccess;
}

}  // namespace

TensorMapEncoder tensor_map_encoder()
{
    static const TensorMapEncoder enc = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return TensorMapEncoder(nullptr);
        }
        return reinterpret_cast<TensorMapEncoder>(fn);
    }();
    return enc;
}

int ypass_tile_cols(int fp64, const Geom& g)
{
    YTile t;
    if (fp64) t = y_paired<double>(g) ? y_tile_pair<double>(g, 1) : y_tile<double>(g, 1);
    else t = y_paired<float>(g) ? y_tile_pair<float>(g, 1) : y_tile<float>(g, 1);
    return 1 << (t.lgTX + t.lgNP);
}

cudaError_t prepare_ymaps(int fp64, void* W, const Geom& g, YMaps* maps)
{
    return fp64 ? prepare_y<double>(W, g, maps) : prepare_y<float>(W, g, maps);
}

cudaError_t launch_ypass(int fp64, bool inverse, void* W, const Geom& g, const FftPlan& plan,
                         const double2* tw, const int* pos, int ncomp, const StepState* st,
                         const YMaps* maps, int* err, cudaStream_t s, const FftPlan* half,
                         const int* pos_half)
{
    return fp64 ? launch_y<double>(inverse, W, g, plan, tw, pos, ncomp, st, maps, err, half, pos_half, s)
                : launch_y<float>(inverse, W, g, plan, tw, pos, ncomp, st, maps, err, half, pos_half, s);
}

int ypass_paired(int fp64, const Geom& g) { return fp64 ? y_paired<double>(g) : y_paired<float>(g); }

cudaError_t configure_ypass()
{
    const int big = 100 * 1024;
    cudaError_t e;
#define FLUSI_SMEM(fn) \
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
#define FLUSI_SMEM_Y(T, R16)                         \
    FLUSI_SMEM((k_ypass<T, true, false, R16>))       \
    FLUSI_SMEM((k_ypass<T, false, false, R16>))      \
    FLUSI_SMEM((k_ypass<T, true, true, R16>))        \
    FLUSI_SMEM((k_ypass<T, false, true, R16>))
    FLUSI_SMEM_Y(float, false)
    FLUSI_SMEM_Y(double, false)
    FLUSI_SMEM_Y(float, true)
    FLUSI_SMEM_Y(double, true)
#undef FLUSI_SMEM_Y
#define FLUSI_SMEM_P(T, R16)                     \
    FLUSI_SMEM((k_ypass_pair<T, true, R16>))     \
    FLUSI_SMEM((k_ypass_pair<T, false, R16>))
    FLUSI_SMEM_P(float, false)
    FLUSI_SMEM_P(double, false)
    FLUSI_SMEM_P(float, true)
    FLUSI_SMEM_P(double, true)
#undef FLUSI_SMEM_P
#undef FLUSI_SMEM
    return cudaSuccess;
}

}  // namespace flusi

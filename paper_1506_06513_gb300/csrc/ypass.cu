// y-axis transform pass (part of the 3-D FFTs of Algorithm 1 step c).
//
// A tile is TX consecutive x-mode columns of NP consecutive z planes of one
// component: every global access is a run of TX complex values (128 bytes).
// Rows arrive by 16-byte asynchronous copies, all FFT stages but the last run
// in shared memory and the last one stores its results to global memory from
// registers; the pass works in place (a tile reads all of its rows before its
// first barrier and writes after its last).
//   inverse: rows j < My hold the kept y-modes 0..Ky, -Ky..-1 -> ny grid rows
//   forward: ny grid rows -> the My kept y-modes (2/3 rule, pruned output)
#include "fft.cuh"
#include "kernels.cuh"

namespace flusi {

namespace {

constexpr int kThreads = 256;
// complex elements per tile (64 KiB of shared memory)
template <typename T> constexpr int tile_elems() { return sizeof(T) == 4 ? 8192 : 4096; }

template <typename T, bool INV>
__global__ void __launch_bounds__(kThreads)
k_ypass(cplx<T>* __restrict__ W, Geom g, FftPlan plan, const double2* __restrict__ tw,
        const int* __restrict__ pos, int ncomp, int lgTX, int lgNP, const StepState* __restrict__ st)
{
    if (st && st->status != 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TX = 1 << lgTX, lgC = lgTX + lgNP, C = 1 << lgC;
    cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* tws = buf + (g.ny << lgC);
    int* sinv = reinterpret_cast<int*>(tws + g.ny);
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

    load_tables<T>(tws, nullptr, tw, nullptr, g.ny, 0);
    load_inverse_pos(sinv, pos, g.ny);
    const int ny = g.ny, My = g.My, Ky = g.Ky;
    const int ld = g.Mxp;   // row stride; a plane holds fewer than 2^31 values
    // this thread's two adjacent columns in the transform stages (fft_run's
    // map with V = 2; TX is even, so both lie in one plane)
    constexpr int V = 2;
    const int col = (threadIdx.x % (C / V)) * V;
    const int z = z0 + (col >> lgTX), x = x0 + (col & (TX - 1));
    const bool colok = z < g.nz && x < g.Mxp;   // Mxp is a multiple of 4
    cplx<T>* gcol = base + (size_t)(colok ? z : 0) * plane + (colok ? x : 0);
    {
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
        fft_dif_out<T, true, V>(buf, C, C, plan, tws, sinv, store);
    } else {
        auto store = [&](int f, const cplx<T>* v) {   // keep modes |m| <= Ky only
            const int r = f <= Ky ? f : (f >= ny - Ky ? f - ny + My : -1);
            if (colok && r >= 0) st_row<T, V>(gcol + r * ld, v);
        };
        fft_dif_out<T, false, V>(buf, C, C, plan, tws, sinv, store);
    }
}

struct YTile {
    int lgTX, lgNP, blocks;
    size_t smem;
};

template <typename T> YTile y_tile(const Geom& g, int ncomp)
{
    YTile t;
    const int cap = tile_elems<T>();
    int TX = sizeof(T) == 4 ? 16 : 8;               // 128-byte runs
    while (TX > 1 && g.ny * TX > cap) TX >>= 1;
    int NP = 1;
    while (2 * NP * TX * g.ny <= cap && 2 * NP * TX <= kThreads && 2 * NP <= g.nz) NP *= 2;
    t.lgTX = __builtin_ctz(TX);
    t.lgNP = __builtin_ctz(NP);
    t.blocks = ceil_div(g.Mxp, TX) * ceil_div(g.nz, NP) * ncomp;
    t.smem = sizeof(cplx<T>) * ((size_t)g.ny + (size_t)g.ny * TX * NP) + sizeof(int) * g.ny;
    return t;
}

template <typename T>
cudaError_t launch_y(bool inverse, void* W, const Geom& g, const FftPlan& plan, const double2* tw,
                     const int* pos, int ncomp, const StepState* st, cudaStream_t s)
{
    YTile t = y_tile<T>(g, ncomp);
    if ((size_t)g.ny << (t.lgTX + t.lgNP) > (size_t)tile_elems<T>()) return cudaErrorInvalidValue;
    if (inverse)
        k_ypass<T, true><<<t.blocks, kThreads, t.smem, s>>>((cplx<T>*)W, g, plan, tw, pos, ncomp,
                                                              t.lgTX, t.lgNP, st);
    else
        k_ypass<T, false><<<t.blocks, kThreads, t.smem, s>>>((cplx<T>*)W, g, plan, tw, pos, ncomp,
                                                               t.lgTX, t.lgNP, st);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ypass(int fp64, bool inverse, void* W, const Geom& g, const FftPlan& plan,
                         const double2* tw, const int* pos, int ncomp, const StepState* st,
                         cudaStream_t s)
{
    return fp64 ? launch_y<double>(inverse, W, g, plan, tw, pos, ncomp, st, s)
                : launch_y<float>(inverse, W, g, plan, tw, pos, ncomp, st, s);
}

cudaError_t configure_ypass()
{
    const int big = 100 * 1024;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_ypass<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_ypass<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_ypass<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    return cudaFuncSetAttribute(k_ypass<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

}  // namespace flusi

// Arithmetic peaks of the GPU the library runs on, measured: the FP32 and
// FP64 fused multiply-add rates that the arithmetic rooflines of the x pass
// (FP32) and of the FP64 path are reported against.  Plain kernels of
// independent dependent-FMA chains, timed with CUDA events; they change no
// clock or power setting.
#include <cuda_runtime.h>

#include "../../include/flusi.h"

namespace flusi {
namespace {

constexpr int kChains = 8;         // independent chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;    // 2048 threads per SM

__device__ double g_fma_sink;      // keeps the chains' results alive

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + 17 * c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == T(-1234.5)) g_fma_sink = double(s);   // never true; the store keeps the work
}

template <typename T>
cudaError_t timed(int grid, int iters, cudaStream_t s, float* ms)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e) return e;
    if ((e = cudaEventCreate(&e1))) {
        cudaEventDestroy(e0);
        return e;
    }
    k_fma_chains<T><<<grid, kThreads, 0, s>>>(iters, T(0.9999999), T(1e-7));   // warm-up
    cudaEventRecord(e0, s);
    k_fma_chains<T><<<grid, kThreads, 0, s>>>(iters, T(0.9999999), T(1e-7));
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (!e) e = cudaEventElapsedTime(ms, e0, e1);
    if (!e) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace
}  // namespace flusi

extern "C" int flusi_fma_peak(int fp64, double target_ms, double* flops_per_s, double* ms_out)
{
    using namespace flusi;
    if ((fp64 != 0 && fp64 != 1) || !flops_per_s || !(target_ms > 0) || target_ms > 10000) return FLUSI_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) || sms <= 0)
        return FLUSI_ECUDA;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) return FLUSI_ECUDA;
    const int grid = sms * kBlocksPerSm;
    // calibrate the chain length to about target_ms, then take the best of three
    int iters = 256;
    float ms = 0.f;
    cudaError_t e = fp64 ? timed<double>(grid, iters, s, &ms) : timed<float>(grid, iters, s, &ms);
    if (!e && ms > 0.f) {
        const double scale = target_ms / ms;
        const double want = iters * (scale > 1.0 ? scale : 1.0);
        iters = want > 1e8 ? 100000000 : (int)want;
    }
    float best = 0.f;
    for (int r = 0; r < 3 && !e; ++r) {
        e = fp64 ? timed<double>(grid, iters, s, &ms) : timed<float>(grid, iters, s, &ms);
        if (!e && (best == 0.f || ms < best)) best = ms;
    }
    cudaStreamDestroy(s);
    if (e || best <= 0.f) return FLUSI_ECUDA;
    const double flops = 2.0 * kChains * (double)iters * (double)grid * kThreads;
    *flops_per_s = flops / (best * 1e-3);
    if (ms_out) *ms_out = best;
    return FLUSI_OK;
}

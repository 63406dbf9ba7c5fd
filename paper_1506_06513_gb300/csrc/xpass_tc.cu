// x pass with its DFT stages on the fifth-generation tensor cores (tcgen05):
// the FP32 state's x transforms as BF16 matrix products with FP32
// accumulation, the operands split into P BF16 pieces (hi + lo, or
// hi + mid + lo), and tensor memory (TMEM) holding the transformed lines
// between the stages and through the physical-space work.
//
// A line of nx = 32 Q reals is transformed at half length NH = 16 Q (the
// c2r pre- and r2c post-processing of the square kernel, Sec. 2.4), by two
// Cooley-Tukey stages, each a product of a block of lines with the real form
// of a small DFT matrix F (K = 2n rows [Re x; Im x], N = 2n columns
// [Re y, Im y], F_ab = W_n^{ab}):
//   inverse, n = n1 + 16 n2:   Y[n1][k1] = sum_{n2} x[n1 + 16 n2] W_Q^{n2 k1}
//                              X[k1 + Q k2] = sum_{n1} W_NH^{n1 k1} Y[n1][k1] W_16^{n1 k2}
//   forward, n = n1 + Q n2:    Y[n1][k1] = sum_{n2} x[n1 + Q n2] W_16^{n2 k1}
//                              X[k1 + 16 k2] = sum_{n1} W_NH^{n1 k1} Y[n1][k1] W_Q^{n1 k2}
// (W = exp(+2 pi i / n) inverse, exp(-2 pi i / n) forward).  A matrix
// product takes 128 rows (M = 128): one row per (line, first index), so one
// tile is RB = 128 / Q grid rows and every thread of the 128-thread CTA owns
// one TMEM lane.  The stage-2 accumulator of an inverse field lands in TMEM
// lane (line, k1) with the line's point pairs k1 + Q k2 along its columns:
// the same lane of all six fields (u, omega) holds the same points, so the
// thread owning that lane forms u x omega - chi/C_eta (u - u_s) for them and
// writes the result straight into the first forward operand, whose row
// (line, n1 = k1) wants exactly those points.  No line ever goes through
// shared memory as FP32.
//
// Operands: stage-1 A (rows from registers) K-major; stage-2 A (the
// twiddled accumulator of a row, written as a K-row of the transposed block)
// MN-major; B (the DFT matrices, built once per CTA) K-major.  With pieces
// a = a_0 + a_1 (+ a_2), b likewise, D = sum over i + j < P of A_i B_j:
// P = 2 drops the a_1 b_1 term (relative error about 2^-16), P = 3 the terms
// of order 2^-24 (the FP32 rounding level).
//
// Force, moment and solid-velocity sums (Eqs. force_with_unst_corrections,
// moment_of_love) are accumulated per point in FP64.
#include "tcgen05.cuh"
#include "xphys.cuh"

namespace flusi {
namespace {

constexpr int kTcThreads = 128;
constexpr unsigned kTcCols = 256;          // TMEM columns per CTA (two CTAs per SM)
constexpr unsigned kTcMinSmem = 80 * 1024; // keeps at most two CTAs on an SM

// Shared-memory layout of one CTA (bytes).
template <int Q, int P> struct TcLayout {
    static constexpr int NH = 16 * Q, RB = 128 / Q;
    static constexpr unsigned kPiece = 8192;                   // 128 rows x 32 BF16
    static constexpr unsigned kBuf = kPiece * P;               // one operand, all pieces
    static constexpr unsigned kB16 = 2048;                     // 32 x 32 BF16: one piece of the 16-point matrix
    static constexpr unsigned kBQ = 8u * Q * Q;                // (2Q)^2 BF16: one piece of the Q-point matrix
    static constexpr unsigned oA = 0;                          // three operand buffers
    static_assert(kBuf % 1024 == 0, "operand buffers stay 1 KB aligned");
    static constexpr unsigned oB16 = oA + 3 * kBuf;            // [forward, inverse][piece]
    static constexpr unsigned oBQ = oB16 + 2 * P * kB16;       // [forward, inverse][piece] when Q != 16
    // input ring depth (fields in flight), as deep as two CTAs per SM allow
    static constexpr int kSlots = P == 2 ? 3 : (Q == 16 ? 2 : 1);
    static constexpr unsigned kMxpMax = (32u * Q / 3 + 4) / 4 * 4; // kept x-modes, padded to 4
    static constexpr unsigned kSlot = RB * kMxpMax * 8;          // one field's rows of a tile
    static constexpr unsigned oRing = oBQ + (Q == 16 ? 0u : 2 * P * kBQ);
    static constexpr unsigned oTwx = oRing + kSlots * kSlot;
    static constexpr unsigned oTw2 = oTwx + 8 * NH;
    static constexpr unsigned oFrame = oTw2 + 8 * NH;
    static constexpr unsigned oWacc = (oFrame + (unsigned)sizeof(FrameT<float>) + 15) / 16 * 16;
    static constexpr unsigned oMask = oWacc + 4 * 36 * 8;
    static constexpr unsigned oBar = (oMask + 4 * RB + 15) / 16 * 16;   // kSlots + 2 mbarriers, TMEM slot
    static constexpr unsigned kBytes = oBar + 8 * (kSlots + 2) + 16;
    static constexpr unsigned kSmem = kBytes > kTcMinSmem ? kBytes : kTcMinSmem;
};

// The real form of the n-point DFT matrix (forward W = exp(-2 pi i/n), or
// inverse), K-major with SBO = 16 K bytes, as P BF16 pieces of `piece` bytes:
// B[a][b] = B[n+a][n+b] = Re W^{ab}, B[a][n+b] = Im W^{ab}, B[n+a][b] = -Im W^{ab}.
// tw is the FP64 table exp(-2 pi i k/nx), k < nx.
template <int P>
__device__ void build_dft_b(char* dst, unsigned piece, int n, bool inverse, const double2* __restrict__ tw, int nx)
{
    const int K = 2 * n, sbo = 16 * K;
    for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
        const int kk = i / K, nn = i - kk * K;
        const int a = kk % n, b = nn % n;
        const double2 w = tw[(size_t)(nx / n) * ((a * b) % n)];
        const double c = w.x, s = inverse ? -w.y : w.y;
        const double v = kk < n ? (nn < n ? c : s) : (nn < n ? -s : c);
        const unsigned off = (nn / 8) * sbo + (kk / 8) * 128 + (nn % 8) * 16 + (kk % 8) * 2;
        double r = v;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const __nv_bfloat16 h = __float2bfloat16_rn((float)r);
            *reinterpret_cast<__nv_bfloat16*>(dst + p * piece + off) = h;
            r -= (double)__bfloat162float(h);
        }
    }
}

// Eight FP32 values as P BF16 pieces, 16 bytes each at dst + p * stride; each
// piece is the residual of the ones before rounded to nearest (the
// differences are exact in FP32).
template <int P>
__device__ __forceinline__ void store8(const float* v, char* dst, unsigned stride)
{
    float r[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = v[i];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            w[i] = tc::pack_bf16(r[2 * i], r[2 * i + 1]);
            if (p + 1 < P) {
                r[2 * i] -= tc::bf16_lo(w[i]);
                r[2 * i + 1] -= tc::bf16_hi(w[i]);
            }
        }
        *reinterpret_cast<uint4*>(dst + p * stride) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Four values, 8 bytes per piece.
template <int P>
__device__ __forceinline__ void store4(const float* v, char* dst, unsigned stride)
{
    float r[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) r[i] = v[i];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        uint32_t w[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            w[i] = tc::pack_bf16(r[2 * i], r[2 * i + 1]);
            if (p + 1 < P) {
                r[2 * i] -= tc::bf16_lo(w[i]);
                r[2 * i + 1] -= tc::bf16_hi(w[i]);
            }
        }
        *reinterpret_cast<uint2*>(dst + p * stride) = make_uint2(w[0], w[1]);
    }
}

// D = sum over the piece products i + j < P of A_i B_j (the smaller products
// first), K in slices of 16 (256 bytes of each operand's K blocks); one
// thread issues.
template <int P>
__device__ __forceinline__ void mma_split(unsigned d, const char* a, unsigned a_piece, unsigned a_sbo,
                                          const char* b, unsigned b_piece, unsigned b_sbo, int kslices,
                                          uint32_t idesc)
{
    unsigned acc = 0;
#pragma unroll
    for (int s = P - 1; s >= 0; --s) {
#pragma unroll
        for (int i = 0; i <= s; ++i) {
            const int j = s - i;
            for (int k = 0; k < kslices; ++k) {
                const uint64_t ad = tc::smem_desc(a + i * a_piece + k * 256, 128, a_sbo);
                const uint64_t bd = tc::smem_desc(b + j * b_piece + k * 256, 128, b_sbo);
                tc::mma_bf16(d, ad, bd, idesc, acc);
                acc = 1;
            }
        }
    }
}

template <int Q, int P, bool LAYER>
__global__ void __launch_bounds__(kTcThreads, 1)
k_xpass_tc(float2* __restrict__ W, Geom g, const double2* __restrict__ tw, XExtra ex,
           const StepState* __restrict__ st)
{
    if (st && st->status != 0) return;
    using Lt = TcLayout<Q, P>;
    constexpr int NH = Lt::NH, RB = Lt::RB, G = 16 / Q;   // G: 8-line groups of the 16-row stages
    constexpr int S = Lt::kSlots;
    constexpr unsigned SBO_Q = 32 * Q;                     // K = 2Q operands: 128 (K/8) bytes per 8 rows
    constexpr unsigned kD1 = 192;                          // TMEM: two stage-1 accumulators of 32 columns
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    char* sm = reinterpret_cast<char*>(smem_raw);
    char* abuf = sm + Lt::oA;                              // [A1 even | A1 odd | A2]
    const char* b16f = sm + Lt::oB16;
    const char* b16i = sm + Lt::oB16 + P * Lt::kB16;
    const char* bqf = Q == 16 ? b16f : sm + Lt::oBQ;
    const char* bqi = Q == 16 ? b16i : sm + Lt::oBQ + P * Lt::kBQ;
    const unsigned bq_piece = Q == 16 ? Lt::kB16 : Lt::kBQ;
    char* ring = sm + Lt::oRing;
    float2* twx = reinterpret_cast<float2*>(sm + Lt::oTwx);
    float2* tw2 = reinterpret_cast<float2*>(sm + Lt::oTw2);
    FrameT<float>* Fs = reinterpret_cast<FrameT<float>*>(sm + Lt::oFrame);
    double* wacc = reinterpret_cast<double*>(sm + Lt::oWacc);
    int* rowmask = reinterpret_cast<int*>(sm + Lt::oMask);
    unsigned long long* full = reinterpret_cast<unsigned long long*>(sm + Lt::oBar);   // [S] ring slots
    unsigned long long* bar1 = full + S;                                                // stage-1 products
    unsigned long long* bar2 = full + S + 1;                                            // stage-2 products
    unsigned* tslot = reinterpret_cast<unsigned*>(full + S + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nx = g.nx, Mx = g.Mx, Mxp = g.Mxp;
    const int nrows = g.nz * g.ny;
    const int ntiles = ceil_div(nrows, RB);

    // twiddles: w_nx^k (mirror steps), and W_NH^{ab} = w_nx^{2ab} (a < 16, b < Q,
    // between the stages) at a Q + (b ^ a % Q): the 16 lanes that read it with
    // a fixed b (inverse) or a fixed a (forward) meet distinct banks
    for (int i = tid; i < NH; i += kTcThreads) {
        twx[i] = make_float2((float)tw[i].x, (float)tw[i].y);
        const int a = i / Q, b = i % Q;
        const double2 w = tw[2 * a * b];
        tw2[a * Q + (b ^ (a % Q))] = make_float2((float)w.x, (float)w.y);
    }
    build_dft_b<P>(sm + Lt::oB16, Lt::kB16, 16, false, tw, nx);
    build_dft_b<P>(sm + Lt::oB16 + P * Lt::kB16, Lt::kB16, 16, true, tw, nx);
    if (Q != 16) {
        build_dft_b<P>(sm + Lt::oBQ, Lt::kBQ, Q, false, tw, nx);
        build_dft_b<P>(sm + Lt::oBQ + P * Lt::kBQ, Lt::kBQ, Q, true, tw, nx);
    }
    load_frame_t<float>(Fs, ex.frame);
    if (tid == 0)
        for (int i = 0; i < S + 2; ++i) mbar_init(full + i, 1);
    if (warp == 0) tc::tmem_alloc(tslot, kTcCols);
    fence_proxy_async();   // the B matrices, written by these threads, before the tensor cores read them
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const unsigned tb = *tslot;
    const unsigned tl = tb + ((unsigned)(warp * 32) << 16);   // this warp's quarter of the lanes

    // Input ring: load L is field L % 6 of this CTA's (L / 6)-th tile, the
    // tile's RB rows of kept x-modes (contiguous in W) in one bulk copy.
    int ring_hi = 0;   // thread 0: one past the last load issued
    auto ring_issue = [&](int L) {
        const int k = L / 6, f = L - 6 * k;
        const int tile = blockIdx.x + k * gridDim.x;
        if (tile >= ntiles) return;
        ring_hi = L + 1;
        const int r0 = tile * RB, nr = min(RB, nrows - r0);
        const unsigned bytes = (unsigned)(nr * Mxp) * (unsigned)sizeof(float2);
        unsigned long long* fb = full + (L % S);
        mbar_expect_tx(fb, bytes);
        tc::bulk_load(ring + (L % S) * Lt::kSlot, W + ((size_t)f * nrows + r0) * Mxp, bytes, fb);
    };
    if (tid == 0)
        for (int L = 0; L < S; ++L) ring_issue(L);

    unsigned ph1 = 0, ph2 = 0;   // completed phases of bar1, bar2
    int ring_lo = 0;             // loads consumed
    bool timed_out = false;

    double acc[3][12];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[c][k] = 0.0;
    double e_acc = 0.0;
    float m_acc = 0.f;
    int bad = 0;
    const FrameT<float>& F = *Fs;
    const float dxT = float(g.dx), dyT = float(g.dy), dzT = float(g.dz);
    const float uinf[3] = {float(ex.u_inf[0]), float(ex.u_inf[1]), float(ex.u_inf[2])};
    constexpr uint32_t id_inv1 = tc::idesc_bf16(128, 2 * Q, 0, 0);
    constexpr uint32_t id_inv2 = tc::idesc_bf16(128, 32, 1, 0);
    constexpr uint32_t id_fwd1 = tc::idesc_bf16(128, 32, 0, 0);
    constexpr uint32_t id_fwd2 = tc::idesc_bf16(128, 2 * Q, 1, 0);

    int k = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
        const int row0 = tile * RB;
        if (tid < RB) {
            const int r = row0 + tid;
            int mask = 0;
            if (r < nrows) {
                const int z = r / g.ny, y = r - z * g.ny;
                const float Y = float(y) * dyT, Z = float(z) * dzT;
                for (int q = 0; q < 3; ++q)
                    if (F.active[q] && Y >= F.box[q][2] && Y <= F.box[q][3] && Z >= F.box[q][4] &&
                        Z <= F.box[q][5])
                        mask |= 1 << q;
            }
            rowmask[tid] = mask;
        }

        // ---- inverse transforms of the six fields (u, omega), two deep:
        //      iteration f forms the stage-1 operands of field f while the
        //      tensor cores run field f-1's stage 1 and f-2's stage 2, then the
        //      stage-2 operands of field f-1.  Stage 2 of field f lands in TMEM
        //      columns [32 f, 32 f + 32); stage 1 alternates between [192, 224)
        //      and [224, 256).
#pragma unroll 1
        for (int f = 0; f <= 6; ++f) {
            bool fail = false;
            if (f < 6) {
                const int L = 6 * k + f, s = L % S;
                fail |= !mbar_wait(full + s, (unsigned)(L / S) & 1u);
                ring_lo = L + 1;
                const float2* rows = reinterpret_cast<const float2*>(ring + s * Lt::kSlot);
                char* a1 = abuf + (f & 1) * Lt::kBuf;
#pragma unroll
                for (int gi = 0; gi < G; ++gi) {
                    const int line = 8 * gi + (tid >> 4), n1 = tid & 15;
                    const bool in = row0 + line < nrows;
                    const float2* src = rows + line * Mxp;
                    float2 v[Q];
#pragma unroll
                    for (int t = 0; t < Q; ++t) {
                        const int kx = n1 + 16 * t;
                        v[t] = (in && kx < Mx) ? src[kx] : make_float2(0.f, 0.f);
                    }
                    if (n1 == 0) v[0].y = 0.f;   // a real line has a real mean
                    sq_exchange_pre<float, Q, 16>(v, n1, twx);
                    // row (line, n1) of group gi: K = [Re v_t | Im v_t], t < Q
                    char* row = a1 + gi * (16 * SBO_Q) + (tid >> 3) * SBO_Q + (tid & 7) * 16;
#pragma unroll
                    for (int kb = 0; kb < Q / 8; ++kb) {
                        float re[8], im[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            re[i] = v[8 * kb + i].x;
                            im[i] = v[8 * kb + i].y;
                        }
                        store8<P>(re, row + kb * 128, Lt::kPiece);
                        store8<P>(im, row + (Q / 8 + kb) * 128, Lt::kPiece);
                    }
                }
            }
            if (f >= 1) {
                // stage 1 of field f-1 done; stage 2 of f-2 done (its operand buffer is free)
                fail |= !mbar_wait(bar1, ph1 & 1u);
                ++ph1;
                if (f >= 2) {
                    fail |= !mbar_wait(bar2, ph2 & 1u);
                    ++ph2;
                }
                tc::fence_after_sync();
                const unsigned d1 = kD1 + 32u * ((f - 1) & 1);
                // twiddle conj(W_NH^{n1 k1}); the row (line, n1) becomes
                // K-row n1 of the transposed block (M = line Q + k1)
#pragma unroll
                for (int gi = 0; gi < G; ++gi) {
                    const int line = 8 * gi + (tid >> 4), n1 = tid & 15;
                    float y[2 * Q];
                    if constexpr (Q == 16) tc::ld32(tl + d1 + gi * 2 * Q, y);
                    else tc::ld16(tl + d1 + gi * 2 * Q, y);
                    float re[Q], im[Q];
#pragma unroll
                    for (int k1 = 0; k1 < Q; ++k1) {
                        const float2 w = tw2[n1 * Q + (k1 ^ (n1 % Q))];
                        re[k1] = y[k1] * w.x + y[Q + k1] * w.y;
                        im[k1] = y[Q + k1] * w.x - y[k1] * w.y;
                    }
#pragma unroll
                    for (int c = 0; c < Q / 8; ++c) {
                        const int M0 = line * Q + 8 * c;
                        char* base = abuf + 2 * Lt::kBuf + (M0 / 8) * 512 + (n1 % 8) * 16;
                        store8<P>(re + 8 * c, base + (n1 / 8) * 128, Lt::kPiece);
                        store8<P>(im + 8 * c, base + ((16 + n1) / 8) * 128, Lt::kPiece);
                    }
                }
            }
            // hand the operands to the tensor cores
            fence_proxy_async();
            tc::fence_before_sync();
            if (__syncthreads_or(fail)) {
                timed_out = true;
                break;
            }
            if (tid == 0) {
                tc::fence_after_sync();
                if (f < 6) ring_issue(6 * k + f + S);   // into the slot just read
                if (f >= 1) {
                    mma_split<P>(tb + 32u * (f - 1), abuf + 2 * Lt::kBuf, Lt::kPiece, 512, b16i, Lt::kB16, 512, 2,
                                 id_inv2);
                    tc::commit(bar2);
                }
                if (f < 6) {
                    const unsigned d1 = kD1 + 32u * (f & 1);
                    for (int gi = 0; gi < G; ++gi)
                        mma_split<P>(tb + d1 + gi * 2 * Q, abuf + (f & 1) * Lt::kBuf + gi * (16 * SBO_Q),
                                     Lt::kPiece, SBO_Q, bqi, bq_piece, SBO_Q, 2 * Q / 16, id_inv1);
                    tc::commit(bar1);
                }
            }
        }
        if (timed_out) break;
        {
            const bool ok = mbar_wait(bar2, ph2 & 1u);   // stage 2 of field 5
            ++ph2;
            tc::fence_after_sync();
            if (__syncthreads_or(!ok)) {
                timed_out = true;
                break;
            }
        }

        // ---- physical space: lane (line, k1) holds the pairs k1 + Q k2 of
        //      every field; NL into the forward stage-1 operands (row = lane)
        {
            const int line = tid / Q, k1 = tid % Q;
            const int r = row0 + line;
            const bool valid = r < nrows;
            const int mask = valid ? rowmask[line] : 0;
            const int z = valid ? r / g.ny : 0, y = valid ? r - z * g.ny : 0;
            const bool inrow[3] = {(mask & 1) != 0, (mask & 2) != 0, (mask & 4) != 0};
            float e_tile = 0.f, chk = 0.f;
            const unsigned arow = (tid >> 3) * 512 + (tid & 7) * 16;
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float ur[3][4], ui[3][4], wr[3][4], wi[3][4];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    tc::ld4x2(tl + 32u * q + 4 * c, 16, ur[q], ui[q]);
                    tc::ld4x2(tl + 32u * (3 + q) + 4 * c, 16, wr[q], wi[q]);
                }
                float nlr[3][4], nli[3][4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int pp = k1 + Q * (4 * c + i);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float u[3], om[3], nl[3];
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            u[q] = h ? ui[q][i] : ur[q][i];
                            om[q] = h ? wi[q][i] : wr[q][i];
                        }
                        cross3(u, om, nl);
                        if (LAYER && valid &&
                            (y >= ex.layer0[1] || z >= ex.layer0[2] || 2 * pp + h >= ex.layer0[0])) {
#pragma unroll
                            for (int q = 0; q < 3; ++q) nl[q] -= F.inv_eta * (u[q] - uinf[q]);
                        }
                        if (valid) {
                            const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                            e_tile += uu;
                            m_acc = fmaxf(m_acc, uu);
                            chk += nl[0] + nl[1] + nl[2];
                        }
                        if (mask) {
                            const float X[3] = {float(2 * pp + h) * dxT, float(y) * dyT, float(z) * dzT};
                            float chi, us[3];
                            int colr;
                            solid_at(F, X, inrow, chi, colr, us);
                            if (chi > 0.f) {
                                const float pen = chi * F.inv_eta;
                                float pu[3], cu[3], m1[3], m2[3];
#pragma unroll
                                for (int q = 0; q < 3; ++q) {
                                    nl[q] -= pen * (u[q] - us[q]);
                                    pu[q] = chi * (u[q] - us[q]);
                                    cu[q] = chi * us[q];
                                }
                                const float* ref = colr == 1 ? F.xc : F.pv[colr - 2];
                                const float rv[3] = {X[0] - ref[0], X[1] - ref[1], X[2] - ref[2]};
                                cross3(rv, pu, m1);
                                cross3(rv, cu, m2);
#pragma unroll
                                for (int cc = 0; cc < 3; ++cc) {
                                    if (colr != cc + 1) continue;
#pragma unroll
                                    for (int q = 0; q < 3; ++q) {
                                        acc[cc][q] += double(pu[q]);
                                        acc[cc][3 + q] += double(m1[q]);
                                        acc[cc][6 + q] += double(cu[q]);
                                        acc[cc][9 + q] += double(m2[q]);
                                    }
                                }
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            const float o = valid ? nl[q] : 0.f;
                            if (h) nli[q][i] = o;
                            else nlr[q][i] = o;
                        }
                    }
                }
                // K index k2 = 4c + i: Re in K blocks 0, 1; Im in 2, 3
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    char* a = abuf + q * Lt::kBuf + arow + (c % 2) * 8;
                    store4<P>(nlr[q], a + (c / 2) * 128, Lt::kPiece);
                    store4<P>(nli[q], a + (2 + c / 2) * 128, Lt::kPiece);
                }
            }
            e_acc += double(e_tile);
            if (!isfinite(e_tile) || !isfinite(chk)) bad = 1;
        }

        // ---- forward transforms of the three NL fields: stage 1 into the
        //      columns of u, stage 2 into those of omega; the stage-2 operands
        //      of a field are formed while the previous field's product runs
        fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            for (int q = 0; q < 3; ++q)
                mma_split<P>(tb + 32u * q, abuf + q * Lt::kBuf, Lt::kPiece, 512, b16f, Lt::kB16, 512, 2, id_fwd1);
            tc::commit(bar1);
        }
        bool fail = !mbar_wait(bar1, ph1 & 1u);
        ++ph1;
        tc::fence_after_sync();
        {
            const int line = tid / Q, n1 = tid % Q;
#pragma unroll 1
            for (int q = 0; q < 3; ++q) {
                float y[32];
                tc::ld32(tl + 32u * q, y);
                float re[16], im[16];
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {
                    const float2 w = tw2[kk * Q + (n1 ^ (kk % Q))];
                    re[kk] = y[kk] * w.x - y[16 + kk] * w.y;
                    im[kk] = y[kk] * w.y + y[16 + kk] * w.x;
                }
                // transposed block of group line / 8: M = (line % 8) 16 + kk, K = n1 (Re), Q + n1 (Im)
                char* base = abuf + q * Lt::kBuf + (line / 8) * (16 * SBO_Q) + (n1 % 8) * 16;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int M0 = (line % 8) * 16 + 8 * c;
                    store8<P>(re + 8 * c, base + (M0 / 8) * SBO_Q + (n1 / 8) * 128, Lt::kPiece);
                    store8<P>(im + 8 * c, base + (M0 / 8) * SBO_Q + ((Q + n1) / 8) * 128, Lt::kPiece);
                }
                fence_proxy_async();
                tc::fence_before_sync();
                if (__syncthreads_or(fail)) {
                    timed_out = true;
                    break;
                }
                if (tid == 0) {
                    tc::fence_after_sync();
                    for (int gi = 0; gi < G; ++gi)
                        mma_split<P>(tb + 96u + 32u * q + gi * 2 * Q, abuf + q * Lt::kBuf + gi * (16 * SBO_Q),
                                     Lt::kPiece, SBO_Q, bqf, bq_piece, SBO_Q, 2 * Q / 16, id_fwd2);
                    if (q == 2) tc::commit(bar2);
                }
            }
        }
        if (timed_out) break;
        {
            const bool ok = mbar_wait(bar2, ph2 & 1u);
            ++ph2;
            tc::fence_after_sync();
            if (__syncthreads_or(!ok)) {
                timed_out = true;
                break;
            }
        }
        // ---- r2c post-processing and the store of the kept x-modes: lane
        //      (line, j) holds Z[j + 16 k2], k2 < Q
#pragma unroll 1
        for (int q = 0; q < 3; ++q) {
#pragma unroll
            for (int gi = 0; gi < G; ++gi) {
                const int line = 8 * gi + (tid >> 4), j = tid & 15;
                const int r = row0 + line;
                float y[2 * Q];
                if constexpr (Q == 16) tc::ld32(tl + 96u + 32u * q + gi * 2 * Q, y);
                else tc::ld16(tl + 96u + 32u * q + gi * 2 * Q, y);
                float2 v[Q];
#pragma unroll
                for (int k2 = 0; k2 < Q; ++k2) v[k2] = make_float2(y[k2], y[Q + k2]);
                float2* out = W + ((size_t)q * nrows + (r < nrows ? r : 0)) * Mxp;
#pragma unroll
                for (int s2 = 0; s2 < Q / 2; ++s2) {
                    float2 a, b;   // partner's Z[s2] and Z[Q-1-s2]
                    a.x = __shfl_sync(0xffffffffu, v[s2].x, (16 - j) & 15, 16);
                    a.y = __shfl_sync(0xffffffffu, v[s2].y, (16 - j) & 15, 16);
                    b.x = __shfl_sync(0xffffffffu, v[Q - 1 - s2].x, (16 - j) & 15, 16);
                    b.y = __shfl_sync(0xffffffffu, v[Q - 1 - s2].y, (16 - j) & 15, 16);
                    if (r < nrows) {
                        const int q1 = s2, q2 = Q - 1 - s2;
                        const int k1 = j + 16 * q1, k2 = j + 16 * q2;
                        float2 m1, m2;
                        if (j != 0) {
                            m1 = b;   // Z[NH - k1] = partner's Z[Q-1-q1]
                            m2 = a;
                        } else {
                            m1 = v[(Q - q1) & (Q - 1)];
                            m2 = v[(Q - q2) & (Q - 1)];
                        }
                        if (k1 < Mxp) out[k1] = k1 < Mx ? r2c_post<float>(v[q1], m1, twx[k1]) : make_float2(0.f, 0.f);
                        if (k2 < Mxp) out[k2] = k2 < Mx ? r2c_post<float>(v[q2], m2, twx[k2]) : make_float2(0.f, 0.f);
                    }
                }
            }
        }
    }

    if (timed_out) {
        // a product or a copy that never completed: report, wait once more
        // (bounded) for what is in flight, give the tensor memory back, leave
        if (tid == 0) {
            atomicCAS(ex.err, 0, (int)FLUSI_ETIMEOUT);
            mbar_wait(bar1, ph1 & 1u);
            mbar_wait(bar2, ph2 & 1u);
            // input copies still on their way into this CTA's shared memory
            for (int L = ring_lo - 1 < 0 ? 0 : ring_lo - 1; L < ring_hi; ++L)
                mbar_wait(full + L % S, (unsigned)(L / S) & 1u);
        }
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) {
            tc::fence_after_sync();
            tc::tmem_dealloc(tb, kTcCols);
        }
        return;
    }

    // ---- the CTA's partial sums: FP64 across lanes and warps
    __shared__ double red[4][3];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
#pragma unroll
        for (int kk = 0; kk < 12; ++kk) {
            const double s2 = warp_sum(acc[cc][kk]);
            if (lane == 0) wacc[warp * 36 + cc * 12 + kk] = s2;
        }
    e_acc = warp_sum(e_acc);
    double m_d = double(m_acc);
    for (int o = 16; o > 0; o >>= 1) m_d = fmax(m_d, __shfl_xor_sync(0xffffffffu, m_d, o));
    const int anybad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        red[warp][0] = e_acc;
        red[warp][1] = m_d;
        red[warp][2] = anybad ? 1.0 : 0.0;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tb, kTcCols);
    }
    double* outp = ex.part + (size_t)blockIdx.x * kNumSums;
    if (tid < 36) {
        double s2 = 0.0;
        for (int w = 0; w < 4; ++w) s2 += wacc[w * 36 + tid];
        outp[tid] = s2;
    } else if (tid == kSumEkin) {
        double s2 = 0.0;
        for (int w = 0; w < 4; ++w) s2 += red[w][0];
        outp[tid] = s2;
    } else if (tid == kSumUmax2 || tid == kSumBad) {
        double s2 = 0.0;
        for (int w = 0; w < 4; ++w) s2 = fmax(s2, red[w][tid == kSumUmax2 ? 1 : 2]);
        outp[tid] = s2;
    } else if (tid < kNumSums) {
        outp[tid] = 0.0;
    }
}

template <int Q, int P>
cudaError_t launch_tc_qp(bool layer, float2* W, const Geom& g, const double2* tw, const XExtra& ex,
                         const StepState* st, cudaStream_t s, int grid)
{
    const size_t smem = TcLayout<Q, P>::kSmem;
    if (layer) k_xpass_tc<Q, P, true><<<grid, kTcThreads, smem, s>>>(W, g, tw, ex, st);
    else k_xpass_tc<Q, P, false><<<grid, kTcThreads, smem, s>>>(W, g, tw, ex, st);
    return cudaGetLastError();
}

// Resident CTAs per SM (at most two: two CTAs of 256 TMEM columns fill an
// SM's 512), from the SM's shared memory and registers.
template <int Q, int P> int tc_per_sm()
{
    int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0;
    cudaFuncAttributes fa{};
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, k_xpass_tc<Q, P, false>) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    const size_t per_cta = TcLayout<Q, P>::kSmem + fa.sharedSizeBytes + (size_t)reserved;
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;   // allocation granularity
    const bool two = 2 * per_cta <= (size_t)smem_sm && 2 * 4 * warp_regs <= regs_sm;
    return two ? 2 : 1;
}

}  // namespace

int xpass_tc_supported(int nx) { return nx == 512 || nx == 256; }

int xpass_tc_grid(const Geom& g)
{
    int dev = 0, sm_count = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (sm_count <= 0) sm_count = 1;
    int per_sm = 1;
    if (g.nx == 512) per_sm = g.xtc == 3 ? tc_per_sm<16, 3>() : tc_per_sm<16, 2>();
    else per_sm = g.xtc == 3 ? tc_per_sm<8, 3>() : tc_per_sm<8, 2>();
    const int RB = 128 / (g.nx / 32);
    const int ntiles = ceil_div(g.nz * g.ny, RB);
    const int grid = per_sm * sm_count;
    return grid < ntiles ? grid : ntiles;
}

cudaError_t launch_xpass_tc(void* W, const Geom& g, const double2* tw, const XExtra& ex, const StepState* st,
                            cudaStream_t s)
{
    float2* w = static_cast<float2*>(W);
    const bool layer = ex.layer0[0] < g.nx || ex.layer0[1] < g.ny || ex.layer0[2] < g.nz;
    const int grid = xpass_tc_grid(g);
    if (!ex.err || ex.sponge_fused) return cudaErrorInvalidValue;
    // the input ring's bulk copies need 16-byte aligned rows that fit a slot
    if ((reinterpret_cast<uintptr_t>(W) & 15) != 0 || (g.Mxp * sizeof(float2)) % 16 != 0)
        return cudaErrorInvalidValue;
    if ((g.nx == 512 && (unsigned)g.Mxp > TcLayout<16, 2>::kMxpMax) ||
        (g.nx == 256 && (unsigned)g.Mxp > TcLayout<8, 2>::kMxpMax))
        return cudaErrorInvalidValue;
    if (g.nx == 512 && g.xtc == 2) return launch_tc_qp<16, 2>(layer, w, g, tw, ex, st, s, grid);
    if (g.nx == 512 && g.xtc == 3) return launch_tc_qp<16, 3>(layer, w, g, tw, ex, st, s, grid);
    if (g.nx == 256 && g.xtc == 2) return launch_tc_qp<8, 2>(layer, w, g, tw, ex, st, s, grid);
    if (g.nx == 256 && g.xtc == 3) return launch_tc_qp<8, 3>(layer, w, g, tw, ex, st, s, grid);
    return cudaErrorInvalidValue;
}

cudaError_t configure_xpass_tc()
{
    cudaError_t e;
    // the largest shared-memory carveout, so that two CTAs fit an SM
#define FLUSI_TC_SMEM(Q, P)                                                                                \
    if ((e = cudaFuncSetAttribute(k_xpass_tc<Q, P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                  TcLayout<Q, P>::kSmem)))                                                 \
        return e;                                                                                          \
    if ((e = cudaFuncSetAttribute(k_xpass_tc<Q, P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                  TcLayout<Q, P>::kSmem)))                                                 \
        return e;                                                                                          \
    if ((e = cudaFuncSetAttribute(k_xpass_tc<Q, P, false>, cudaFuncAttributePreferredSharedMemoryCarveout, \
                                  (int)cudaSharedmemCarveoutMaxShared)))                                   \
        return e;                                                                                          \
    if ((e = cudaFuncSetAttribute(k_xpass_tc<Q, P, true>, cudaFuncAttributePreferredSharedMemoryCarveout,  \
                                  (int)cudaSharedmemCarveoutMaxShared)))                                   \
        return e;
    FLUSI_TC_SMEM(16, 2)
    FLUSI_TC_SMEM(16, 3)
    FLUSI_TC_SMEM(8, 2)
    FLUSI_TC_SMEM(8, 3)
#undef FLUSI_TC_SMEM
    return cudaSuccess;
}

}  // namespace flusi

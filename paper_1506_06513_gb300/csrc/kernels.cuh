// Kernels of libflusi and their host-side launchers.
//
// Device data layout (complex of the state precision T; N_r = nz*ny rows):
//   U, H   state u_hat and AB2 history N_hat^{n-1}: [3][Mz][My][Mxp], only the
//          modes kept by the 2/3 rule (m_y, m_z stored as 0..K, -K..-1)
//   W      work: [6][nz][ny][Mxp]; per z plane the first My rows hold
//          y-modes ("A" form, after the z transform) or all ny rows hold grid
//          y values ("B" form, after the y transform); each row carries the
//          Mx kept x-modes padded with zeros to Mxp.
// One step: kinematics -> zinv (u, omega) -> yinv -> xpass (c2r, physics, r2c)
//           -> scalars -> yfwd -> zfwd -> zupdate (projection, IF-AB2).
#pragma once

#include <cuda.h>   // CUtensorMap (descriptor type only; the encoder is fetched at run time)

#include "../../include/flusi.h"
#include "common.cuh"

namespace flusi {

// Ensemble batches.  While an ensemble step is captured, the launches made on
// this host thread can cover `n` members at once: the launchers then size
// gridDim.z = n and pass `mb`, the device array of the members' buffers, and
// each kernel takes its member's pointers from mb[blockIdx.z].  Outside a
// batch n = 1 and mb = nullptr (the kernels use their own arguments).
struct Batch {
    const Member* mb = nullptr;
    int n = 1;
};
Batch& current_batch();

// kinematics / scalars (scalars.cu); mb: see Batch
__global__ void k_kinematics(const flusi_insect* ins, const StepState* st, const StepCoef* coef, Frame* fr,
                             double h, double frac, const Member* mb, Shape S, int with_t, double inv_eta);
__global__ void k_reset_state(StepState* st, StepCoef* coef);
__global__ void k_wait_probe(int* err, long long max_cycles);
__global__ void k_scalars(Geom g, const double* part, int nparts, StepState* st, StepCoef* coef,
                          double* rows, int ring, double* etab, double3 opts, double dt_diff,
                          const Frame* fr, flusi_insect* ins, const Member* mb);

// y transform (ypass.cu): W[c] for c < ncomp, between A and B form.
// tw: twiddle table of the axis; pos: digit-reversal table of its plan.
// With maps (tensor descriptors of W built by prepare_ymaps for this handle's
// W) a tile arrives by TMA boxes, else by 16-byte asynchronous copies; a TMA
// wait that gives up sets *err = FLUSI_ETIMEOUT.
// cuTensorMapEncodeTiled through the runtime's driver entry point (fetched
// once, thread-safely), or nullptr when the driver does not offer it.
typedef CUresult (*TensorMapEncoder)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                     const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                     CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                     CUtensorMapFloatOOBfill);
TensorMapEncoder tensor_map_encoder();
struct YMaps {
    CUtensorMap inv, fwd;
    int inv_bh = 0, fwd_bh = 0;   // box heights (rows); 0: that direction copies by 16 bytes
};
cudaError_t prepare_ymaps(int fp64, void* W, const Geom& g, YMaps* maps);
// half, pos_half: the plan of length ny / 2 and its digit-reversal table, for
// the paired kernel (a cluster of two CTAs per tile; see ypass_paired);
// nullptr: one CTA per tile always
cudaError_t launch_ypass(int fp64, bool inverse, void* W, const Geom& g, const FftPlan& plan,
                         const double2* tw, const int* pos, int ncomp, const StepState* st,
                         const YMaps* maps, int* err, cudaStream_t s, const FftPlan* half = nullptr,
                         const int* pos_half = nullptr);
// 1 when the y passes of this grid take the paired kernel (Geom::ypair)
int ypass_paired(int fp64, const Geom& g);

// z transforms (zpass.cu)
//   zinv: U -> W[0..nf) in A form; nf = 3 (u) or 6 (u and omega = i k x u).
// TMA descriptors of the z passes' sources: the state U, the RK4 stage state
// and W, each as (2 Q reals, rows, components) with Q = My Mxp columns; box
// height 0: that source copies by 16 bytes.
struct ZMaps {
    CUtensorMap u, ut, w;
    int u_bh = 0, ut_bh = 0, w_bh = 0;
};
cudaError_t prepare_zmaps(int fp64, void* U, void* Ut, void* W, const Geom& g, ZMaps* maps);
// columns of a y tile and of a z tile for this grid and its tile caps
int ypass_tile_cols(int fp64, const Geom& g);
int zpass_tile_cols(int fp64, const Geom& g);
cudaError_t launch_zinv(int fp64, const void* U, void* W, const Geom& g, const FftPlan& plan,
                        const double2* tw, const int* pos, int nf, const StepState* st,
                        const CUtensorMap* map, int bh, int* err, cudaStream_t s);
// Extra arguments of the spectral update (launch_zupdate).
struct ZfwdExtra {
    const StepCoef* coef;     // mode 0
    const double* etab;       // mode 0: [E1x Mx][E1y My][E1z Mz][E2x][E2y][E2z] in FP64, then in FP32
    double u_inf[3];
    int mean_free;
    double sponge_c;          // modes 0, 2..5: > 0 adds the vorticity sponge of W[3..5]
    void* stage;              // modes 2..5: the RK4 stage state (state layout)
};
// forward z transform of W[0..nf-1] (A form), in place: the kept modes jz < Mz
// end in rows jz of each field's A-form layout
cudaError_t launch_zfwd(int fp64, void* W, int nf, const Geom& g, const FftPlan& plan,
                        const double2* tw, const int* pos, const StepState* st,
                        const CUtensorMap* map, int bh, int* err, cudaStream_t s);
// 1/N, sponge, projection and (mode 0) IF-AB2 update of U, H, (mode 1) U = N,
// H = 0, or (modes 2..5) RK4 stage 1..4, reading the kept modes that
// launch_zfwd left in W
cudaError_t launch_zupdate(int fp64, int mode, const void* W, void* U, void* H, const Geom& g,
                           const ZfwdExtra& ex, const StepState* st, cudaStream_t s);

// max |k . u_hat| and max |k| |u_hat| over the kept modes of a state, FP64,
// into out[0], out[1] (device; cleared here)
cudaError_t launch_divergence(int fp64, const void* U, const Geom& g, unsigned long long* out, cudaStream_t s);

// x pass (xpass.cu)
// XP_SPONGE: c2r of W[comp0 .. comp0+2], times the sponge mask, r2c back in place
enum XMode { XP_PHYS = 0, XP_R2C = 1, XP_C2R = 2, XP_DUMP = 3, XP_SPONGE = 4 };
struct XExtra {
    const Frame* frame;
    Shape shape;
    double* part;            // XP_PHYS: [grid][kNumSums]
    const void* rin;         // XP_R2C: real input [ncomp][nz][ny][nx]
    void* rout;              // XP_C2R: real output; XP_DUMP: [14][nz][ny][nx]
    int real_fp64;           // element type of rin / rout: 1 double, 0 float
    int ncomp;               // XP_R2C / XP_C2R: components
    int comp0;               // first W component written (R2C) or read (C2R)
    long long cstride;       // elements between components of rin / rout
    // Sec. 2.3 wake removal: first grid index of each axis' end slab (the
    // axis length when there is none)
    int layer0[3];           // XP_PHYS / XP_DUMP: Dirichlet layer u = u_inf
    int sponge0[3];          // XP_SPONGE, or XP_PHYS with sponge_fused: sponge region
    int sponge_fused;        // XP_PHYS: also form chi_sp omega and x-transform it into W[3..5]
    double u_inf[3];
    int* err;                // XP_PHYS on the tensor cores: status word for a wait that gives up
    // XP_PHYS, register-resident kernels: rows of partial sums ("virtual
    // CTAs", each taking tiles v, v + nvirt, ... in order); the launch may
    // run fewer CTAs, each taking virtual CTAs b, b + gridDim.x, ...  0: the
    // launch's own grid.
    int nvirt;
};
int xpass_fuses_sponge(int fp64, const Geom& g);
int xpass_grid(int fp64, const Geom& g);   // CTAs of the persistent physical pass
cudaError_t launch_xpass(int fp64, int mode, void* W, const Geom& g, const FftPlan& plan,
                         const double2* tw, const int* pos, const XExtra& ex, const StepState* st,
                         cudaStream_t s);

// x pass on the tensor cores (xpass_tc.cu): the physical pass of an FP32
// state with its DFT stages as split-BF16 tcgen05 products (g.xtc pieces),
// for nx = 256 and 512 without the fused sponge.
int xpass_tc_supported(int nx);
int xpass_tc_grid(const Geom& g);
cudaError_t launch_xpass_tc(void* W, const Geom& g, const double2* tw, const XExtra& ex, const StepState* st,
                            cudaStream_t s);
cudaError_t configure_xpass_tc();

// Message returned by flusi_last_error(NULL).
void set_global_error(const char* msg);

// Shared-memory limits of every instantiation (once per process and device).
cudaError_t configure_ypass();
cudaError_t configure_zpass();
cudaError_t configure_xpass();

}  // namespace flusi

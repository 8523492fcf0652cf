// lbm_internal.h -- shared between the host API (lbm_api.cu) and the sweep
// kernels (sweep_*.cu).  Not part of the public C ABI (include/lbm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace btrirt {

enum Problem { kCavity = 0, kStefan = 1 };

// What one launch of the lattice kernel does.
enum Mode {
    kSweep = 0,      // stream + collide, write the next populations
    kSweepDiag = 1,  // same, plus the fused FP64 diagnostics reductions
    kFields = 2,     // stream + macroscopic step only: write the fields, no populations
};

// FP64 diagnostics record living in device memory (one per handle).
struct DevRecord {
    double step;      // step the record belongs to
    double melt_sum;  // sum f_l
    double H_sum;     // sum H
    double Q_last;    // heated-wall inflow of the last step
    double Q_cum;     // running sum of Q_last
    double max_u;     // max |u|
    double nan_flag;  // 1 if a non-finite H or rho was seen
    double valid;     // 1 once the fields of `step` have been reduced
};

// Arguments of every lattice kernel, passed by value.
template <typename real>
struct SweepArgs {
    const real *src;       // 18 planes: f_0..f_8 then g_0..g_8
    real *dst;             // same layout (sweep modes)
    real *aux;             // init only: the other buffer, whose f planes are also
                           // set to w_i (they are never rewritten when flow is off)
    int nx, ny;            // lattice size
    int pitch;             // row pitch, elements
    long long pstride;     // plane stride, elements
    real k0, k1, k2;       // g rates (Eq. 2)
    real k0f, k1f, k2f;    // f rates
    real Lh, gbeta;        // latent heat, g*beta
    int strip_on;          // cavity: 1 if the heated segment is non-empty
    int lo2, hi2;          // cavity: crossing heated iff lo2 <= 2x + 1 - c_ix <= hi2
    // heated-wall inflow reduction (every sweep)
    double *qpart;         // one partial per wall-adjacent block
    unsigned *qcount;      // ticket counter, reset to 0 by the last block
    int nq;                // number of wall-adjacent blocks
    // diagnostics reduction (kSweepDiag, init)
    double *dpart;         // 4 partials per block
    unsigned *dcount;      // ticket counter, reset to 0 by the last block
    DevRecord *rec;
    long long step;        // step index the launch produces
    // field outputs (kFields), nx*ny doubles each, row-major; NULL = skip
    double *oH, *oT, *oFL, *oUX, *oUY, *oRHO;
};

// Launchers (defined in sweep_fp32.cu / sweep_fp64.cu).
template <typename real>
cudaError_t launch_lattice(const SweepArgs<real> &a, int problem, bool flow, int mode,
                           dim3 grid, dim3 block, cudaStream_t s);
template <typename real>
cudaError_t launch_init(const SweepArgs<real> &a, double amp, uint64_t seed, dim3 grid,
                        dim3 block, cudaStream_t s);
template <typename real>
cudaError_t launch_fields0(const SweepArgs<real> &a, bool flow, dim3 grid, dim3 block,
                           cudaStream_t s);

}  // namespace btrirt

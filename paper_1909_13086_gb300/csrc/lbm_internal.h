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
    kSweepDiag = 1,  // same, plus the fused diagnostics reductions
    kFields = 2,     // stream + macroscopic step only: write the fields, no populations
};

// How populations move from one step to the next.  Pull: two buffers, every
// sweep pulls f*_i(x - c_i) from src and writes f*_i(x) into its own slot i of
// dst ("the pull layout": slot i of cell x holds f*_i(x)).  One buffer, two
// alternating sweeps (src == dst; the AA pattern of Bailey et al. 2009):
//   push  -- from the pull layout: pull as above, then put f*_i(x) into slot
//            opp(i) of cell x + c_i, or into the cell's own slot i where
//            x + c_i lies beyond a wall;
//   local -- from the pushed layout: f_i(x) is the cell's own slot opp(i) (a
//            wall's incoming population then takes the wall rule), and f*_i(x)
//            goes to its own slot i: the pull layout again.
// Each cell reads and writes the same 18 locations in either sweep, so no two
// cells touch one location, and the populations are those of the pull sweeps.
enum Streaming { kPull = 0, kAAPush = 1, kAALocal = 2 };

// Population layout in device memory ("tile-major structure of arrays").
// The lattice is cut into column tiles of kTW cells.  Within a tile, each row
// holds the 18 planes (f_0..f_8, g_0..g_8) one after the other, kTW values
// each, and rows follow one another:
//     index(x, y, p) = ((x / kTW) * ny + y) * 18 * kTW + p * kTW + x % kTW.
// A warp's 18 loads of one cell row are then one base register plus
// compile-time offsets (plane p: p*kTW; row above / below: -/+ 18*kTW).
constexpr int kTW = 128;  // tile width = threads per block (fastest of 128/256/512 on GB300)
constexpr int kPlanes = 18;
constexpr int kRS = kPlanes * kTW;  // elements per tile row

__host__ __device__ inline long long pop_index(int x, int y, int p, int ny) {
    return ((long long)(x / kTW) * ny + y) * kRS + (long long)p * kTW + (x % kTW);
}

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
    unsigned long long counter;  // steps taken: advanced by every sweep on the
                                 // device, so that replayed CUDA graphs stamp
                                 // records correctly (an integer: GB300's FP64
                                 // pipe is narrow, and a sweep's warps would
                                 // each issue the predicated FP64 add)
    unsigned long long rng[2];   // stochastic-rounding step seeds, one word per buffer parity
    double timeout;   // 1 once a bounded device wait ran out (staged sweep)
};

// Arguments of every lattice kernel, passed by value.  16-byte aligned, so
// that a batch entry's argument sets start on 16-byte pieces.
template <typename real>
struct alignas(16) SweepArgs {
    // Population buffers, tile-major, of the storage type S the launcher was
    // instantiated with (float, double, __half or __nv_bfloat16).
    const void *src;       // populations of the previous step
    void *dst;             // populations written by this step
    void *aux;             // init only: the other buffer, whose f planes are also
                           // set to w_i (they are never rewritten when flow is off)
    int nx, ny;            // lattice size
    int ntx;               // number of column tiles
    int parity;            // index of the source buffer (selects the rounding seed word
                           // and the direction of the sweep over the row bands)
    int rows;              // rows per block (each thread walks them)
    int prefetch;          // > 0: each block asks L2 for the tile rows `prefetch`
                           // rows ahead of its own in the sweep's direction
                           // (one bulk prefetch per row)
    real k0, k1, k2;       // g rates (Eq. 2)
    real k0f, k1f, k2f;    // f rates
    real Lh, gbeta;        // latent heat, g*beta
    real inv_Lh;           // 1 / Lh
    int strip_on;          // cavity: 1 if the heated segment is non-empty
    int lo2, hi2;          // cavity: crossing heated iff lo2 <= 2x + 1 - c_ix <= hi2
    // heated-wall inflow reduction (every sweep)
    double *qpart;         // one partial per wall-adjacent block
    unsigned *qcount;      // ticket counter, reset to 0 by the last block
    int nq;                // number of wall-adjacent blocks
    // diagnostics (kSweepDiag, init): 4 partials per block, folded into the
    // record by a fold kernel launched right after on the same stream
    double *dpart;
    double *dpart2;        // fold kernel: 4 partials per fold block
    unsigned *dticket;     // fold kernel: ticket counter, reset by its last block
    DevRecord *rec;
    // optional history ring (lbm_set_history): entry k = 4 doubles {step, Q,
    // melt fraction, unused} for step k mod hist_cap; NULL = off
    double *hist;
    long long hist_cap;
    long long step;        // step index the launch produces (host bookkeeping only;
                           // the record takes its step from rec->counter)
    // staged sweep (16-bit storage): 1 = launch staged_kernel over the band
    // grid; its mbarrier waits give up after wait_limit + 1 tries, and
    // force_timeout = 1 makes each block first wait on a barrier that nothing
    // completes (tests of the timeout path)
    int staged;
    int force_timeout;
    long long wait_limit;
    // field outputs (kFields), nx*ny doubles each, row-major; NULL = skip
    double *oH, *oT, *oFL, *oUX, *oUY, *oRHO;
};

// Launchers, instantiated in sweep_fp32.cu / sweep_fp64.cu / sweep_f16.cu /
// sweep_bf16.cu for (compute real, storage codec S) = (float, float),
// (double, double), (float, F16<SR>), (float, BF16<SR>), SR = round to
// nearest (false) or stochastically (true).
template <bool SR>
struct F16;
template <bool SR>
struct BF16;
// pdl: launch the sweep with programmatic stream serialization, so that it
// is scheduled while the previous kernel of the stream drains (the kernel
// waits for that kernel's completion before it touches memory).
template <typename real, typename S>
cudaError_t launch_lattice(const SweepArgs<real> &a, int problem, bool flow, int mode,
                           dim3 grid, dim3 block, cudaStream_t s, bool pdl, int streaming = kPull);
template <typename real, typename S>
cudaError_t launch_init(const SweepArgs<real> &a, double amp, uint64_t seed, dim3 grid,
                        dim3 block, cudaStream_t s);
template <typename real, typename S>
cudaError_t launch_fields0(const SweepArgs<real> &a, bool flow, dim3 grid, dim3 block,
                           cudaStream_t s);
// One lattice of a batch launch: its arguments for both buffer parities and
// its place in the launch's block numbering.
template <typename real>
struct BatchEntry {
    SweepArgs<real> a[2];  // [p]: source buffer p, destination buffer 1 - p
    int start;             // first block of this lattice in the launch
    int gx, gy;            // tile columns and row bands
    int pad;
};

// One step of a batch: `entries` points at n device BatchEntry<real> records
// whose blocks, nblocks in all, run in one launch; starts[r] is entry r's first
// block (the entries' start fields, as a compact array for the block search);
// parity[r] is entry r's source buffer at step j = 0; uniform > 0 when every
// entry has that many blocks (0 otherwise); interleave (uniform batches only):
// block b belongs to entry b mod n instead of b / uniform.  diag: diagnostic
// sweep plus the per-entry fold.  streaming: kPull (buffer parity[r] ^ (j & 1)
// into the other), or the push (even j) / local (odd j) sweep of one-buffer
// streaming in buffer parity[r].
template <typename real, typename S>
cudaError_t launch_batch(const void *entries, const int *starts, const int *parity, int n,
                         int uniform, int interleave, int nblocks, int problem, bool flow, bool diag,
                         int j, cudaStream_t s, bool pdl, int streaming = kPull);
// Tile-major buffer <-> plane-major FP64 staging (18 planes of nx*ny, f then g).
// to_staging = true packs buf into stage; false unpacks stage into buf (and,
// if buf2 is non-NULL, the f planes into buf2 as well).  Values in the staging
// are the populations themselves, whatever the storage encoding.
template <typename S>
cudaError_t launch_repack(void *buf, void *buf2, double *stage, int nx, int ny, bool to_staging,
                          cudaStream_t s);

}  // namespace btrirt

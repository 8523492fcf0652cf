/*
 * lbm.h -- C ABI of the GB300 B-TriRT melting solver.
 *
 * One fused CUDA sweep per time step advances, on one GPU, the D2Q9 lattice of
 * the paper "Lattice Boltzmann simulations of melting in a rectangular cavity
 * heated locally from below at high Rayleigh number" (Zhao, Wu, Chai, Shi):
 *   - the total-enthalpy populations g_i with the block triple-relaxation-time
 *     (B-TriRT) collision of Eq. 2 and the equilibrium of Eq. 4, k1 from the
 *     thermal diffusivity by Eq. 5, optionally k2 = 2 - k1 (Eq. 6);
 *   - the per-cell inversion H -> (T, f_l) of H = C_p T + f_l L (Eq. 1);
 *   - the flow populations f_i with Boussinesq buoyancy and the liquid-fraction
 *     velocity suppression u = f_l u* (readings of Sec. 3.2, which cites its
 *     flow model without stating it);
 *   - pull streaming with half-way bounce-back (no-slip, adiabatic) and
 *     anti-bounce-back on the wall held at T_h (Sec. 3.1 left wall, Sec. 3.2
 *     heated strip of width D centred at C on the bottom wall).
 * Lattice units throughout: dx = dt = 1, c_s^2 = 1/3, C_p = rho0 = 1, T_m = 0,
 * T_h = 1.
 *
 * Conventions
 *   - Every call returns an int status: LBM_OK (0) or a negative LBM_ERR_*.
 *     lbm_last_error(h) gives a message (h may be NULL for create failures).
 *     No call throws or aborts.
 *   - The handle owns its device memory (allocated through the allocator hook
 *     if one is installed, else cudaMalloc).  Host arrays are owned by the
 *     caller and only read or written during the call.
 *   - Host field and population arrays are row-major FP64: cell (x, y) at index
 *     y*nx + x, 0 <= x < nx (width), 0 <= y < ny (height, y = 0 at the bottom
 *     wall).  Population arrays are plane-major: direction i (0..8) at offset
 *     i*nx*ny.  D2Q9 order: c_0 = (0,0), c_1 = (1,0), c_2 = (0,1), c_3 = (-1,0),
 *     c_4 = (0,-1), c_5 = (1,1), c_6 = (-1,1), c_7 = (-1,-1), c_8 = (1,-1).
 *   - Work is enqueued on the handle's CUDA stream (borrowed from the caller,
 *     or created by the library when NULL is passed).  Calls that return data
 *     to the host synchronise that stream.
 *   - One handle must not be used from two host threads at the same time.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_s *lbm_handle;

enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,      /* invalid argument or parameter set                */
    LBM_ERR_OOM = -2,      /* device or host allocation failed                 */
    LBM_ERR_CUDA = -3,     /* a CUDA runtime call failed                       */
    LBM_ERR_DIVERGED = -4, /* a non-finite H or rho was found by the diagnostics */
    LBM_ERR_STATE = -5,    /* call not valid in the handle's current state     */
    LBM_ERR_TIMEOUT = -6   /* a bounded device wait ran out (staged sweep)     */
};

/* Storage and arithmetic precision of the populations.  The 16-bit modes
 * store the populations in FP16 or BF16 -- f_i as its deviation f_i - w_i from
 * the rest state, g_i as it is (its rest state at T_m = 0 is zero) -- with all
 * arithmetic in FP32 and the diagnostics reductions as for LBM_FP32.  FP16
 * values are stored scaled by exact powers of two (g by 2^6, f - w by 2^10) so
 * that they stay in FP16's normal range: |g| <= 1000 and |f - w| <= 64.
 * LBM_FP16 / LBM_BF16 round to nearest; LBM_FP16_SR / LBM_BF16_SR round
 * stochastically with counter-based random bits (deterministic for a given
 * state and step), so that per-step increments below half an ulp are not
 * lost.  Population read-back and write-back round to nearest in every mode. */
enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16 = 2, LBM_BF16 = 3, LBM_FP16_SR = 4, LBM_BF16_SR = 5 };

/* Problem kind. */
enum {
    LBM_CAVITY = 0, /* Sec. 3.2: closed cavity, heated strip on the bottom wall  */
    LBM_STEFAN = 1  /* Sec. 3.1: left wall at T_h, right wall adiabatic, y periodic */
};

/* Problem parameters (Sec. 3.1, Sec. 3.2 and Eqs. 5-6). */
typedef struct {
    int problem;            /* LBM_CAVITY or LBM_STEFAN                                 */
    double Ra, Pr, Ste, Ma; /* Rayleigh, Prandtl, Stefan and Mach numbers.  Cavity units:
                               U = Ma c_s, nu = U ny sqrt(Pr/Ra), alpha = nu/Pr,
                               g beta = U^2/ny; L = 1/Ste                                */
    double strip_center;    /* C, heated-strip centre as a fraction of the width         */
    double strip_width;     /* D, heated-strip width as a fraction of the width; 0 = none */
    double k0, k2;          /* g rates of Eq. 2 in (0, 2); k2 < 0 selects k2 = 2 - k1    */
    double alpha_override;  /* > 0: thermal diffusivity alpha directly (nu = Pr alpha,
                               g beta from Ra); 0: from Ra, Pr, Ma; < 0 is rejected      */
    double k0f, k1f;        /* flow ghost and first-moment rates in (0, 2); the second-
                               moment rate is 1/(nu/c_s^2 + 1/2)                         */
    int flow_on;            /* 0: u = 0 and f is not evolved (Sec. 3.1 conduction)       */
    double init_amp;        /* amplitude a of the initial perturbation: H0 = a (2r - 1),
                               r = (splitmix64(seed xor (y nx + x)) >> 11) 2^-53          */
    uint64_t seed;
} lbm_params;

/* Parameters derived by lbm_set_params (lattice units). */
typedef struct {
    double nu, alpha, gbeta;
    double k0, k1, k2;       /* k1 from Eq. 5: 1/k1 = alpha/c_s^2 + 1/2                 */
    double k0f, k1f, k2f;
    double Lh;               /* latent heat 1/Ste                                        */
    double a, b;             /* heated segment [a, b] of the bottom wall, in cells       */
    double Href;             /* reference length: ny (cavity) or nx (Stefan)             */
    double heated_len;       /* b - a (cavity) or ny (Stefan)                            */
} lbm_derived;

/* Diagnostics of the current step, reduced on the device: sums over cells in
 * FP64 for LBM_FP64 lattices, exactly in 64-bit fixed point (2^-24 units, each
 * cell's value rounded once) for FP32 and 16-bit storage; delivered as FP64. */
typedef struct {
    long long step;          /* steps taken since lbm_set_params                        */
    double melt_fraction;    /* sum f_l / (nx ny)                                        */
    double H_total;          /* sum H                                                    */
    double Q_strip;          /* enthalpy entering through the T_h wall in the last step:
                                sum over heated crossings of 2 w_i T_h - 2 g*_opp(i)     */
    double Q_cum;            /* Q_strip summed over all steps since lbm_set_params       */
    double Nu;               /* Q_strip Href / (alpha dT heated_len)                     */
    double front_x;          /* sum f_l / ny: melt-front distance from x = 0 (Stefan)    */
    double max_u;            /* max |u|                                                  */
    int nan_flag;            /* 1 if any H or rho was not finite                         */
} lbm_diag;

/* Create a solver for an nx x ny lattice (nx, ny >= 2) in the given precision.
 * cuda_stream: a cudaStream_t to borrow, or NULL for a library-owned
 * non-blocking stream (NULL is never taken to mean the legacy default stream).
 * Limits: ny <= 65535, nx * ny <= 2^31.
 * Allocates the two population buffers (2 x 18 planes).  State is undefined
 * until lbm_set_params.  Errors: LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_create(int nx, int ny, int precision, void *cuda_stream, lbm_handle *out);

/* Validate and derive the parameters (Eqs. 5-6 and the unit mapping above),
 * then reset the state to step 0: f_i = w_i, g_i = g_eq(H0, T(H0), u = 0)
 * (Eq. 4).  Errors: LBM_ERR_ARG (rates outside (0, 2), Ste <= 0, ...). */
int lbm_set_params(lbm_handle h, const lbm_params *p);

/* Copy the derived parameters.  Error LBM_ERR_STATE before lbm_set_params. */
int lbm_get_derived(lbm_handle h, lbm_derived *out);

/* Advance n >= 0 time steps (one fused sweep each), asynchronously on the
 * stream.  The diagnostics reductions are fused into the last sweep (and into
 * every diag_every-th sweep, see lbm_set_diag_every).  Errors: LBM_ERR_ARG,
 * LBM_ERR_STATE (no parameters), LBM_ERR_CUDA. */
int lbm_step(lbm_handle h, long long n);

/* Fuse the diagnostics into every k-th sweep as well (k = 0: last sweep of
 * each lbm_step call only, the default). */
int lbm_set_diag_every(lbm_handle h, long long k);

/* Launch shape of the sweep (the tuner's knobs): rows of the lattice walked by
 * each thread of a block (1 to 1024, default 1, or 3 with 16-bit storage);
 * the distance, in rows, at which each block asks L2 to prefetch a later
 * block's tile rows (0 = off, default 16, or 32 with 16-bit storage); and
 * graph_chunk, the longest piece
 * of sweeps lbm_step replays from a CUDA graph (0 = launch every sweep
 * directly; default 128).  Successive sweeps visit the lattice's row bands in
 * opposite directions (the two wall bands first), each starting on the rows
 * the previous one wrote last, which are still in L2; the prefetch distance
 * counts along the sweep's direction.
 *
 * How lbm_step enqueues its n sweeps: it cuts them into pieces that end at
 * the diagnostic sweeps (every diag_every-th step and the call's last one)
 * and are at most graph_chunk long (with one-buffer streaming, see
 * lbm_set_streaming, the call's one-buffer sweeps are cut the same way, ending
 * at the diagnostic steps inside them, and its closing two-buffer sweeps form
 * the last piece).  A piece is identified by its length, whether it ends with
 * a diagnostic sweep, the buffer parity it starts from, and for one-buffer
 * pieces the sweep (push or local) it starts with.  The first time a piece is
 * asked for its sweeps are launched
 * directly; the second time it is captured into a CUDA graph, which is
 * replayed from then on (up to 16 pieces are remembered per handle, least
 * recently used first out).  So repeated calls of one length -- a serving
 * quantum, a fixed output interval -- run from graphs after the first, and a
 * one-off call never pays for a capture.  Every sweep, direct or replayed,
 * is launched with programmatic stream serialization: it is scheduled while
 * the previous sweep's last blocks drain and waits for that sweep's results
 * before it reads them.  When the caller is itself capturing the handle's
 * stream, lbm_step launches directly.  Results do not depend on any of these: the
 * populations never, and the diagnostics of FP32 and 16-bit storage neither
 * (their sums are exact fixed-point integer sums); the FP64 diagnostics sums
 * follow the grouping of cells, to within FP64 rounding.  Errors: LBM_ERR_ARG. */
int lbm_set_launch(lbm_handle h, int rows_per_block, int prefetch_rows, int graph_chunk);

/* How lbm_step moves the populations from one step to the next.
 * LBM_STREAM_TWO_BUFFERS: every sweep pulls from one buffer into the other.  LBM_STREAM_ONE_BUFFER: all but the last one or two sweeps of a
 * call work in place in one buffer, alternating two sweeps (the AA pattern of
 * Bailey et al., "Accelerating lattice Boltzmann fluid flow simulations using
 * graphics processors", 2009): a push sweep that pulls as usual and puts
 * each post-collision population f*_i(x) into slot opp(i) of cell x + c_i
 * (its own slot i where x + c_i lies beyond a wall), then a local sweep that
 * takes a cell's populations from its own slots (wall rules on the edge) and
 * writes them back to their own slots, which leaves the usual layout.  Each
 * cell reads and writes the same locations in either sweep.  The closing
 * sweeps of a call run over the two buffers, so between calls the handle's
 * state is exactly that of two-buffer streaming: results, fields, populations
 * and checkpoints do not depend on the mode, bit for bit.  One buffer halves
 * the working set of a step, so that more of what the previous step wrote is
 * still in L2 when the next one reads it.  Both buffers stay allocated.  The
 * staged 16-bit sweep and lbm_step_static always use two buffers; a batch has
 * its own setting (lbm_batch_set_streaming).
 * Default (set by lbm_create): one buffer (2048 x 1024 cavity on GB300: FP32
 * 41.4 -> 36.6 us per step, BF16-SR 26.1 -> 24.4 us), except for LBM_FP64,
 * which is bound by its arithmetic and keeps two buffers.  Takes effect at the
 * next lbm_step.  Errors: LBM_ERR_ARG. */
enum { LBM_STREAM_TWO_BUFFERS = 0, LBM_STREAM_ONE_BUFFER = 1 };
int lbm_set_streaming(lbm_handle h, int mode);

/* Sweep kernel for 16-bit storage.  The staged sweep (an option for LBM_FP16,
 * LBM_BF16, LBM_FP16_SR and LBM_BF16_SR; off by default) gives each block a band of
 * consecutive rows of one 128-cell tile column and streams the tile rows it
 * needs through a ring of shared-memory slots with TMA bulk copies, two rows
 * ahead of the row it computes, so that the loads are in flight while it
 * collides; it reads the 16-bit populations at the same addresses and
 * computes exactly what the row-per-block sweep computes.  On GB300 it is
 * slower than the row-per-block sweep (the 16-bit sweep is bound by
 * instruction issue, not by memory latency, and each tile row takes 27 bulk
 * copies), so it is off by default.  bands: -1 = automatic (as many bands
 * per tile column as give one wave of 8 blocks per SM, each at least 4 rows),
 * 0 = the row-per-block sweep (lbm_set_launch shape; the default), n > 0 = n
 * bands per tile column (capped at ny / 4).  FP32 and FP64 lattices always
 * take the row-per-block sweep.  Results do not depend on it.
 * Errors: LBM_ERR_ARG. */
int lbm_set_staging(lbm_handle h, int bands);

/* Every wait of the staged sweep on its shared-memory ring is bounded: after
 * tries + 1 unsuccessful tries (default 2^20, about a second) the block
 * records a timeout, waits for its copies still in flight and returns, and
 * the next lbm_diagnostics reports LBM_ERR_TIMEOUT; the state is then invalid
 * until lbm_set_params or lbm_write_populations.  force_timeout = 1 makes
 * every block first wait on a barrier that nothing completes, so that the
 * timeout path can be tested without a fault (0 for normal operation).
 * Errors: LBM_ERR_ARG. */
int lbm_set_wait_limit(lbm_handle h, long long tries, int force_timeout);

/* Counters of how the handle's sweeps were enqueued since lbm_create:
 * launched directly, replayed from captured graphs, and graphs captured. */
typedef struct {
    long long sweeps_direct;
    long long sweeps_replayed;
    long long graphs_captured;
} lbm_launch_stats;
int lbm_get_launch_stats(lbm_handle h, lbm_launch_stats *out);

/* Autotuner: times every launch shape of a small candidate set (rows per block
 * 1, 2, 3, 4; prefetch distance 0, 2, 4, 8, 16, 24, 32, 48 rows) for steps_per_trial
 * steps each (best of two, after a warm-up) on a scratch lattice with the
 * handle's size, precision and parameters -- the handle's own state is not
 * touched, but the scratch lattice is allocated and freed -- and applies the
 * fastest with lbm_set_launch (graph_chunk unchanged).  The choice is cached
 * per (nx, ny, precision, problem, flow_on) for the life of the process, so
 * later handles of the same kind are tuned without timing.  Outputs (may be
 * NULL): the chosen rows and prefetch, and its time per step in microseconds
 * (0 when it came from the cache).  Synchronises.  Errors: LBM_ERR_ARG,
 * LBM_ERR_STATE, LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_autotune(lbm_handle h, int steps_per_trial, int *rows, int *prefetch, float *us_per_step);

/* Bit mask selecting the fields of lbm_read_fields. */
enum { LBM_FIELD_H = 1, LBM_FIELD_T = 2, LBM_FIELD_FL = 4, LBM_FIELD_UX = 8,
       LBM_FIELD_UY = 16, LBM_FIELD_RHO = 32, LBM_FIELD_ALL = 63 };

/* Macroscopic fields of the current step n: the H, T, f_l, u (= f_l u*) and rho
 * computed inside step n from the streamed populations (at n = 0: the initial
 * fields, u = 0).  Each selected pointer receives nx*ny doubles; unselected or
 * NULL pointers are skipped.  Synchronises.  Errors: LBM_ERR_STATE right after
 * lbm_write_populations (no step taken yet), LBM_ERR_CUDA. */
int lbm_read_fields(lbm_handle h, unsigned mask, double *H, double *T, double *fl,
                    double *ux, double *uy, double *rho);

/* Diagnostics record of the current step.  Synchronises.  Returns
 * LBM_ERR_DIVERGED (with *out filled) if nan_flag is set, LBM_ERR_TIMEOUT if a
 * bounded device wait ran out since the state was last set. */
int lbm_diagnostics(lbm_handle h, lbm_diag *out);

/* History of the run (the melt-fraction and Nusselt histories of Sec. 3.2):
 * a device ring of `capacity` entries (0 frees it) that every step fills with
 * its heated-wall inflow Q and every diagnostic step also with its melt
 * fraction, without any host round trip (steps 1, 2, ...; the initial state
 * has no entry).  Cleared on (re)allocation. */
int lbm_set_history(lbm_handle h, long long capacity);

/* Read the newest min(max, capacity) history entries, oldest first: step, Q,
 * Nu (from Q, as in lbm_diag) and melt fraction (NaN on steps without
 * diagnostics).  Steps with no entry (a cavity without a heated strip between
 * diagnostic steps, or overwritten) are skipped.  Any output pointer may be
 * NULL; *count receives the number of entries.  Synchronises. */
int lbm_read_history(lbm_handle h, int max, long long *step, double *Q, double *Nu, double *melt,
                     int *count);

/* Checkpoint: the current post-collision populations (9*nx*ny doubles each
 * for f and g, plane-major) and the step counter.  Synchronises. */
int lbm_read_populations(lbm_handle h, double *f, double *g, long long *step);

/* Resume: overwrite the populations (rounded to the handle's precision) and
 * the step counter; Q_cum restarts at 0.  Fields and diagnostics are
 * undefined until the next step. */
int lbm_write_populations(lbm_handle h, const double *f, const double *g, long long step);

/* ---- Batches: many lattices advanced together ------------------------------
 * A batch advances all its lattices by one fused launch per step: the blocks
 * of every member lattice form one grid (each block looks up its lattice and
 * tile in a device table), so lattices too small to fill the GPU alone -- the
 * 256 x 128 requests of a serving stream -- share it, and the per-step launch
 * cost is paid once.  lbm_batch_step cuts its steps into pieces (128 plain
 * steps while more than 128 remain, then the rest, ending with the diagnostic
 * step) and, as lbm_step does, replays a piece from a CUDA graph from the
 * second time it is asked for (graphs are kept per batch composition); every
 * launch uses programmatic stream serialization.  The batch uses its own
 * launch shape (lbm_batch_set_launch, lbm_batch_autotune), whatever the
 * members' lbm_set_launch settings.  Each
 * step of a member computes exactly what lbm_step would: the populations are
 * bitwise those of stepping it alone, and so are the diagnostics except on
 * FP64 lattices (summation order, see lbm_set_launch).
 *
 * Members keep their own memory and state; lbm_diagnostics, lbm_read_fields
 * and friends keep working on them between batch steps.  Every member must
 * share the device, precision, problem kind and flow_on of the first one; the
 * last step of each lbm_batch_step is a diagnostic step for every member (their
 * diag_every setting does not apply inside a batch).  The batch orders its
 * work after what is queued on the members' streams and their streams after
 * it.  Errors of batch calls are reported by lbm_last_error(NULL). */
typedef struct lbm_batch_s *lbm_batch;

/* Create an empty batch for up to max_lattices lattices (1..65536) on the
 * current device; cuda_stream as in lbm_create.  Allocates the device table
 * (through the allocator hook if one is installed).  Errors: LBM_ERR_ARG,
 * LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_batch_create(int max_lattices, void *cuda_stream, lbm_batch *out);

/* Add a lattice (its parameters set) to the batch / remove it.  Membership
 * changes take effect at the next lbm_batch_step (the table is rebuilt and the
 * chunk graph re-captured then).  Errors: LBM_ERR_ARG (full, duplicate, not a
 * member, or precision / problem / flow_on differing from the batch's),
 * LBM_ERR_STATE (no parameters). */
int lbm_batch_add(lbm_batch b, lbm_handle h);
int lbm_batch_remove(lbm_batch b, lbm_handle h);

/* Number of lattices in the batch. */
int lbm_batch_count(lbm_batch b, int *count);

/* Advance every member n >= 0 steps, asynchronously on the batch's stream. */
int lbm_batch_step(lbm_batch b, long long n);

/* Launch shape of the batch's step kernel: rows of a member walked by each
 * block (0 = the default: 2, or 4 with 16-bit storage; up to 1024), the L2
 * prefetch distance in rows (-1 = the default: 4),
 * and interleave = 1 (the default) to number the blocks of a one-size batch
 * member after member (block b belongs to member b mod n) instead of member
 * by member (0; a batch whose members' block counts differ is always member
 * by member).  Results do not depend on it.  Takes effect at the next
 * lbm_batch_step.  Errors: LBM_ERR_ARG. */
int lbm_batch_set_launch(lbm_batch b, int rows_per_block, int prefetch_rows, int interleave);

/* Streaming of the batch's step kernel, as lbm_set_streaming for one lattice:
 * with LBM_STREAM_ONE_BUFFER all but the last one or two steps of an
 * lbm_batch_step call alternate push and local sweeps in each member's current
 * buffer, and the closing steps run over two buffers, so that between calls
 * every member's state is the two-buffer one (results do not depend on the
 * mode, bit for bit; members may be stepped alone or in other batches between
 * calls).  Until this is called the batch follows its precision: one buffer,
 * two for LBM_FP64.  Synchronises the batch's stream.  Errors: LBM_ERR_ARG. */
int lbm_batch_set_streaming(lbm_batch b, int mode);

/* Autotuner for a batch: times rows per block (1, 2, 3, 4) x prefetch distance
 * (0, 4, 8, 16 rows) x block order (member by
 * member, interleaved) for steps_per_trial steps each (best of three, after a
 * warm-up) on scratch lattices of the batch's composition -- the same sizes,
 * precision and parameters, allocated and freed here; the members' states are
 * not touched -- and applies the fastest with lbm_batch_set_launch.  The
 * choice is cached per composition (precision, problem, flow and the members'
 * sizes in order) for the life of the process.  Outputs (may be NULL): the
 * chosen shape and its time per step in microseconds (0 when it came from the
 * cache).  Synchronises.  Errors: LBM_ERR_ARG, LBM_ERR_STATE (empty batch),
 * LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_batch_autotune(lbm_batch b, int steps_per_trial, int *rows, int *prefetch, int *interleave,
                       float *us_per_step);

/* Free the batch (not its members). */
int lbm_batch_destroy(lbm_batch b);

/* One step with no allocation, for callers that cannot allocate device
 * memory at the moment they step: hosts that hand out device memory only from
 * a fixed arena of their own, plug-ins that must not touch the host program's
 * allocator, latency-critical loops that must never enter an allocator.  The
 * paper has no counterpart: it is an interface convenience, not part of the
 * method.
 *
 * Advances the lattice held in the caller's device buffer `src` by one fused
 * sweep with diagnostics (the same kernel and arithmetic as lbm_step) into the
 * caller's device buffer `dst` (distinct from src), on `cuda_stream` (NULL =
 * legacy default stream).  Both buffers use the library's tile-major layout:
 * element ((x / 128) * ny + y) * 2304 + p * 128 + x % 128 for plane p (0..8 =
 * f_0..f_8, 9..17 = g_0..g_8), ceil(nx / 128) * ny * 2304 elements of FP32
 * (LBM_FP32) or FP64 (LBM_FP64).  With flow_on = 0 the f planes are neither
 * read nor written.  `step` is the step number of src.  If `out` is non-NULL
 * the call synchronises the stream and fills it with the diagnostics of step
 * + 1, where Q_cum covers this call only; with out = NULL it returns without
 * synchronising.
 *
 * The reduction scratch is one file-scope device array of about 2.6 MB, held
 * by every GPU that loads the library until the process exits.  Maximum
 * lattice: ceil(nx / 128) * ny <= 65536 (e.g. 4096 x 2048); larger ones get
 * LBM_ERR_ARG -- use lbm_create / lbm_step.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current and keeps it for later calls; make that first call before any
 * stream capture.  The kept address belongs to the device's context as it was
 * then: after cudaDeviceReset (or any teardown of the primary context) it is
 * stale, so do not call lbm_step_static on a device after resetting it.  With
 * out non-NULL the call also synchronises the stream.  Every call shares
 * the one array, clearing what must start at zero: calls whose work overlaps
 * on the GPU (other streams, other host threads) race and must be serialised
 * by the caller.  Allocates nothing and calls no allocating routine.  Errors
 * (message in lbm_last_error(NULL)): LBM_ERR_ARG, LBM_ERR_CUDA,
 * LBM_ERR_DIVERGED (out filled). */
int lbm_step_static(const void *src, void *dst, int nx, int ny, int precision, const lbm_params *p,
                    long long step, void *cuda_stream, lbm_diag *out);

/* Free the handle's device memory (and its stream, if library-owned). */
int lbm_destroy(lbm_handle h);

/* Message of the last error on h (or of the calling thread's last create
 * failure when h is NULL).  Never NULL. */
const char *lbm_last_error(lbm_handle h);

/* Optional device allocator hook, used by every later lbm_create (e.g. to take
 * memory from a framework's caching allocator).  alloc returns a device
 * pointer of at least `bytes` bytes aligned to 256 B, or NULL; release frees
 * it.  Pass NULL, NULL to restore cudaMalloc/cudaFree.  Not thread-safe
 * against concurrent lbm_create calls. */
typedef void *(*lbm_alloc_fn)(size_t bytes, void *ctx);
typedef void (*lbm_free_fn)(void *ptr, void *ctx);
int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn release, void *ctx);

/* Library build identification: "btrirt <version> sm_103a". */
const char *lbm_version(void);

#ifdef __cplusplus
}
#endif
#endif

/*
 * swept.h -- C ABI of libswept.so: the swept time-space decomposition rule for
 * explicit 1D stencils on one GB300 GPU (sm_103a), beside a per-time-step kernel.
 *
 * Paper: Magee, Walker & Niemeyer, "Applying the swept rule for solving explicit
 * partial differential equations on heterogeneous computing systems".
 *   Section 4.1 / Fig. 1:  Up Triangle, Communication, Diamond, Down Triangle.
 *   Section 4.2:           the problem statement (grid size, block size, scheme)
 *                          and the two test equations.
 *   Section 4.2, Eq. 1:    the GPU work factor of the CPU/GPU split
 *                          (sw_run_hybrid).
 *   Section 4.3 / Fig. 2:  per-step ("Classic") decomposition, flattening and
 *                          lengthening; the 7-value Euler state per point.
 *
 * Conventions for every entry point:
 *  - All calls return an int status: 0 (SW_OK), a positive warning, or a
 *    negative error (SW_ERR_*). No call throws or aborts across the ABI.
 *  - Device pointers are CUDA global-memory pointers on the current device.
 *    `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Compute calls are asynchronous on that stream; errors detected on the
 *    device are latched in the handle and reported by sw_sync_status.
 *  - The caller owns every state buffer it passes; the library owns the
 *    scratch it allocates in sw_create and frees it in sw_destroy.
 *  - A handle is not thread-safe: one host thread (or external locking) per
 *    handle; calls on one handle must go to one stream at a time.
 *
 * State layout ("planes"): structure of arrays, plane-major, n cells per plane,
 * contiguous: plane k occupies elements [k*n, (k+1)*n).
 *   heat  FP64:      1 plane  of double (u)
 *   heat  FP32:      1 plane  of float  (u)
 *   heat  FP32_COMP: 2 planes of float  (u_hi, u_lo), value = hi + lo
 *   Euler FP64:      3 planes of double (rho, rho*u, E)
 *   Euler FP32:      3 planes of float
 *   Euler FP32_COMP: 6 planes of float  (rho_hi, m_hi, E_hi, rho_lo, m_lo, E_lo)
 * sw_pack_fp64 / sw_unpack_fp64 convert between FP64 planes and any layout.
 */
#ifndef SWEPT_H
#define SWEPT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* 2: sw_run_hybrid / sw_hybrid_split, SW_FLAG_EULER_FOLD / LENGTHENED / FLATTENED /
 * GRAPH, SW_ERR_CORRUPT and sw_debug_corrupt_guard.
 * 3: swept Euler runs default to the flattened form where W allows it;
 * SW_FLAG_LENGTHENED selects the lengthened form for swept runs too; sw_autotune
 * also picks the Euler form.
 * 4: the two-dimensional heat entry points sw2d_*; sw_batch_set_threads.
 * 5: sw2d_set_threads / sw2d_threads. */
#define SW_ABI_VERSION 5

#if defined(__GNUC__)
#define SW_API __attribute__((visibility("default")))
#else
#define SW_API
#endif

/* schemes (Section 4.2) */
#define SW_HEAT 0   /* FTCS heat equation, r = alpha dt / dx^2 */
#define SW_EULER 1  /* 2nd-order finite volume Euler, pressure-ratio minmod limiter */

/* working precision */
#define SW_FP64 0
#define SW_FP32 1
#define SW_FP32_COMP 2  /* FP32 hi/lo pair with compensated (TwoSum) state update */

/* boundary of the 1D domain */
#define SW_PERIODIC 0
#define SW_TRANSMISSIVE 1  /* zero-gradient: the ghost copies the end cell */

/* decomposition (Section 4.1: Swept vs Classic) */
#define SW_SWEPT 0    /* Up Triangle, Diamond x k, Down Triangle */
#define SW_PERSTEP 1  /* one launch per step (Euler: per stage, the flattened form) */

/* status codes */
#define SW_OK 0
#define SW_WARN_UNSTABLE 1       /* heat r > 1/2: runs, but FTCS is unstable */
#define SW_ERR_BAD_ARG (-1)
#define SW_ERR_CUDA (-2)
#define SW_ERR_OOM (-3)
#define SW_ERR_TIMEOUT (-4)      /* a bounded device-side wait expired */
#define SW_ERR_NONPHYSICAL (-5)  /* Euler: rho <= 0, p <= 0 or NaN found */
#define SW_ERR_UNSUPPORTED (-6)
#define SW_ERR_TOO_LARGE (-7)    /* sw_run_noalloc: needs more than SW_NOALLOC_SCRATCH_BYTES */
#define SW_ERR_CORRUPT (-8)      /* a guard word after a scratch buffer was overwritten */

#define SW_NOALLOC_SCRATCH_BYTES (16u << 20)

/* sw_problem.flags */
#define SW_FLAG_GENERIC 1  /* swept: use the generic shared-memory phase kernel for every
                              phase (no register-resident Diamond kernel); same results */
#define SW_FLAG_EULER_FOLD 2 /* swept Euler: run every phase with a complete (or no) upper
                                half on the register-resident kernel where it is instantiated
                                (W = 128; FP32 forms also W = 256), otherwise as without the
                                flag; same results. Off by default: on GB300 it measured
                                slower than the generic kernel, because the scheme is bound by
                                arithmetic and the folded kernel evaluates K + 1 faces per K
                                cells per level at a lower occupancy. Ignored with
                                SW_FLAG_GENERIC. */
/* The two data-structure strategies of Section 4.3 (Fig. 2) for the Euler step; every
   form gives the same bits. Lengthened: four 3-point sub-steps per step, the pressure
   ratio stored between them. Flattened: two 5-point stages per step. Without either
   flag, per-step runs are flattened (two launches per step) and swept runs are
   flattened whenever the base width allows radius-2 windows (W % 4 == 0, W >= 8),
   else lengthened; SW_FLAG_EULER_FOLD (swept) implies lengthened. The default
   follows the measured speed: on GB300 the flattened form is the faster one for
   both methods (fewer barriers per step, 722 against 943 thread instructions per
   cell-step in FP32 swept). Both flags at once: SW_ERR_BAD_ARG. */
#define SW_FLAG_LENGTHENED 4 /* Euler: the lengthened form (per-step: four launches per step) */
#define SW_FLAG_GRAPH 16     /* sw_run captures the run's launches once into a CUDA graph
                                (on a private stream, launch tracing off) and replays it on the
                                caller's stream; the handle keeps one graph, for the last
                                (state pointer, nsteps) pair, and captures again when either
                                changes. Same results. */
#define SW_FLAG_FLATTENED 8  /* Euler: the flattened form, two 5-point stages per step; swept:
                                windows widen and narrow by 2 cells per level, W/4 levels per
                                phase, W % 4 == 0 and W >= 8, generic kernel only (ignores
                                SW_FLAG_EULER_FOLD) */

#define SW_MIN_TILE 4
#define SW_MAX_TILE 1024

/* The problem statement of Section 4.2: grid size, scheme, dt/dx (as r for
 * heat, lambda = dt/dx for Euler), block (tile) base width. */
typedef struct sw_problem {
    int32_t scheme;     /* SW_HEAT or SW_EULER */
    int32_t precision;  /* SW_FP64, SW_FP32 or SW_FP32_COMP */
    int32_t boundary;   /* SW_PERIODIC or SW_TRANSMISSIVE */
    int32_t method;     /* SW_SWEPT or SW_PERSTEP */
    int64_t n;          /* number of cells, >= 2 * tile_width (swept) or >= 4 */
    double r;           /* heat: alpha * dt / dx^2 (> 0) */
    double dt_dx;       /* Euler: lambda = dt / dx (> 0) */
    double gamma;       /* Euler: ratio of specific heats (> 1) */
    int32_t tile_width; /* swept base width W: even, SW_MIN_TILE..SW_MAX_TILE,
                           divides n; 0 selects the library default */
    int32_t flags;      /* 0 or an OR of the SW_FLAG_* bits above (sw_run_noalloc:
                           SW_FLAG_GENERIC, SW_FLAG_LENGTHENED, SW_FLAG_FLATTENED only;
                           batches: 0, SW_FLAG_LENGTHENED or SW_FLAG_FLATTENED) */
} sw_problem;

typedef struct sw_handle sw_handle;

/* Validate `p` and allocate the scratch the run needs (flank buffers for the
 * swept phases, a ping-pong plane set for the per-step form, a status word) on
 * the current device. On success *out owns that memory. Errors: SW_ERR_BAD_ARG
 * (bad field; *out untouched), SW_ERR_OOM, SW_ERR_CUDA. Returns
 * SW_WARN_UNSTABLE (and a valid handle) for heat with r > 1/2. */
SW_API int sw_create(const sw_problem *p, sw_handle **out);

/* Release the handle and its scratch (synchronises the device first). NULL ok. */
SW_API void sw_destroy(sw_handle *h);

/* Number of planes (of the precision's element type) and bytes of one state. */
SW_API int sw_state_planes(const sw_problem *p);
SW_API int64_t sw_state_bytes(const sw_problem *p);

/* Advance the state in place by `nsteps` full time steps (Euler: 4 sub-steps
 * each) on `stream`. `state` is a device pointer in the layout above. Swept:
 * one launch per phase (Up, each Diamond, Down; Section 4.1); per-step: one
 * launch per step (heat) or per stage (Euler). nsteps == 0 is a no-op.
 * Errors: SW_ERR_BAD_ARG (NULL state, nsteps < 0), SW_ERR_CUDA (launch). */
SW_API int sw_run(sw_handle *h, void *state, int64_t nsteps, void *stream);

/* End-to-end form of sw_run: copy `state_in` (host memory, same layout) to the
 * handle's device buffer, advance it, copy it back to `state_out` (host; may
 * equal state_in), and wait for completion. Pinned host memory is fastest. */
SW_API int sw_run_host(sw_handle *h, const void *state_in, void *state_out, int64_t nsteps,
                void *stream);

/* The affinity split of Section 4.2 (Eq. 1, the GPU work factor WF = N_GPU / N_CPU,
 * counted in tiles): for `tiles` tiles, `cpu_threads` host threads each take
 * tiles_per_thread = floor(tiles / (work_factor + cpu_threads)) tiles and the GPU
 * the rest (gpu_tiles >= work_factor * tiles_per_thread). Pure host arithmetic.
 * Errors: SW_ERR_BAD_ARG when tiles < 2, work_factor < 1, cpu_threads outside
 * 1..4096 or tiles_per_thread would be 0. Output pointers may be NULL. */
SW_API int sw_hybrid_split(int64_t tiles, int32_t work_factor, int32_t cpu_threads, int64_t *gpu_tiles,
                           int64_t *tiles_per_thread);

/* Swept run shared between the GPU and `cpu_threads` host threads (Section 4.2's
 * heterogeneous decomposition, the split of sw_hybrid_split): in every phase the GPU
 * runs structures 0 .. gpu_tiles-1 and the host threads the rest, concurrently; the
 * host threads work on pinned host mirrors of the flank buffers and of the state,
 * and once per phase the one or two flank slots at the GPU/host boundaries cross
 * between device and host memory on `stream`. The host threads evaluate the same
 * per-cell arithmetic with the host's IEEE operations (no contraction), so the
 * result is bitwise that of sw_run. `state` is the device state (in place): the
 * host's tiles are read from it at the start and written back at the end.
 * Synchronous: returns when the run is complete. The first call allocates the host
 * mirrors (2 x the flank scratch + one state, pinned) and starts the threads; both
 * are kept by the handle until sw_destroy (a call with another thread count restarts
 * the threads). Not safe to call concurrently on one handle.
 * The host threads implement the lengthened Euler form only: an Euler handle must
 * run lengthened (SW_FLAG_LENGTHENED, or a width that rules out the flattened form).
 * Errors: SW_ERR_BAD_ARG (method not swept, a flattened Euler handle, the split
 * above, NULL state, nsteps < 0), SW_ERR_OOM, SW_ERR_CUDA. */
SW_API int sw_run_hybrid(sw_handle *h, void *state, int64_t nsteps, int32_t work_factor, int32_t cpu_threads,
                         void *stream);

/* Conversions between FP64 planes (nplanes_fp64 = 1 heat, 3 Euler, each n
 * doubles) and the working layout of `p`, on the device. FP32: round to
 * nearest; FP32_COMP: hi = float(x), lo = float(x - hi). */
SW_API int sw_pack_fp64(const sw_problem *p, const double *src_fp64, void *dst_state, void *stream);
SW_API int sw_unpack_fp64(const sw_problem *p, const void *src_state, double *dst_fp64, void *stream);

/* Deterministic FP64 sums of each conserved variable (heat: sum u; Euler: sum
 * rho, sum m, sum E; FP32_COMP sums hi + lo), written to sums_host[0..nv) after
 * the stream completes. Fixed-order tree: identical for identical inputs. */
SW_API int sw_conservation(sw_handle *h, const void *state, double *sums_host, void *stream);

/* Euler only: scan the state for rho <= 0, p <= 0 or NaN; latch the result.
 * Returns SW_OK or SW_ERR_NONPHYSICAL (after synchronising `stream`); the first
 * offending cell index is written to *cell (if non-NULL), else -1. */
SW_API int sw_check_physical(sw_handle *h, const void *state, int64_t *cell, void *stream);

/* Synchronise `stream` and return the latched device status (then clear it).
 * It also checks the guard words that follow each of the handle's scratch
 * buffers (flank buffers, per-step planes: 256 bytes of a fixed pattern written
 * at sw_create): if any changed, a kernel wrote past its buffer, and the call
 * returns SW_ERR_CORRUPT (the guards are rewritten, so the next call reports only
 * new damage). */
SW_API int sw_sync_status(sw_handle *h, void *stream);

/* Test hook: overwrite one byte of the guard after scratch buffer `which` (0, 1:
 * flank buffers; 2: per-step planes) from the host, so that tests can check the
 * detection in sw_sync_status without any kernel writing out of bounds.
 * SW_ERR_BAD_ARG when the handle has no such buffer. */
SW_API int sw_debug_corrupt_guard(sw_handle *h, int32_t which);

/* Number of kernel launches the last sw_run on this handle issued. */
SW_API int64_t sw_last_launch_count(const sw_handle *h);

/* Per-launch tracing. sw_set_timing(h, capacity) makes every following sw_run
 * record a CUDA event pair around each of its first `capacity` launches, on
 * the run's stream (capacity 0 turns it off; SW_ERR_OOM/SW_ERR_CUDA if the
 * events cannot be created). sw_launch_times waits for those events and writes
 * up to `cap` durations in milliseconds to ms[] and the launch kinds to kind[]
 * (0 Up Triangle, 1 Diamond, 2 Down Triangle, 3 per-step kernel); it returns
 * the number written, or a negative status. */
SW_API int sw_set_timing(sw_handle *h, int64_t capacity);
SW_API int64_t sw_launch_times(sw_handle *h, float *ms, int32_t *kind, int64_t cap);

/* Tile width actually used by the handle (after defaults). */
SW_API int32_t sw_tile_width(const sw_handle *h);

/* sw_run without any device allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- code running
 * inside a framework whose memory pool owns the device (a direct cudaMalloc
 * fails or escapes the pool's accounting) and latency-critical loops that
 * allow no allocation after start-up (cudaMalloc/cudaFree may synchronise).
 * It runs the same swept phases as sw_run (method must be SW_SWEPT; same default
 * width and Euler form; always the generic phase kernel, same bits), but the
 * flank buffers live in one static device array of SW_NOALLOC_SCRATCH_BYTES
 * (16 MiB) compiled into the library, which every GPU that loads the library
 * holds until the process exits. The caller passes the state, as for sw_run.
 * Scratch needed: 2 * round_up_256(K * (n/W + 1) * 2W * element_size) bytes,
 * K = 1 (heat FP64/FP32), 2 (heat FP32_COMP), 7 (Euler FP64/FP32 lengthened),
 * 6 (flattened), 10 (Euler FP32_COMP lengthened), 9 (flattened); larger problems
 * are rejected with SW_ERR_TOO_LARGE before any launch (e.g. heat FP64 at
 * W = 1024 fits n up to ~512k cells).
 * Every call looks up the array's device address (cudaGetSymbolAddress, a
 * host-side lookup that allocates nothing) with the caller's device current, so
 * a device reset cannot leave a stale address. The first call on a device also
 * loads the library's device code there; make that first call before any
 * stream capture. All calls share the array and it keeps the last call's
 * contents (nothing in it needs to start at zero); calls that overlap on the
 * GPU race on it and must be serialised by the caller. A CUDA error already
 * pending on the calling thread is reported as SW_ERR_CUDA without launching
 * (and is left pending); launches stop at the first that fails.
 * Returns SW_WARN_UNSTABLE after a successful heat run with r > 1/2, as sw_create.
 * Errors: SW_ERR_BAD_ARG (the rules of sw_create, method != SW_SWEPT, other
 * flags), SW_ERR_TOO_LARGE, SW_ERR_UNSUPPORTED, SW_ERR_CUDA. */
SW_API int sw_run_noalloc(const sw_problem *p, void *state, int64_t nsteps, void *stream);

/* ---- batches: many independent problems in one persistent launch ------------
 * (Section 6 of the paper tunes the block size per problem; the batched launch
 * and its device-side work queue are this library's addition.)
 * sw_batch_create: `count` problems (all of one precision, method SW_SWEPT,
 * the field rules of sw_create, each with an explicit tile_width; flags 0 or, for
 * an Euler problem, SW_FLAG_LENGTHENED or SW_FLAG_FLATTENED (then W % 4 == 0 and
 * W >= 8); each Euler problem runs in the form sw_run would take for it), problem
 * i's device state at
 * states[i] (layout as for sw_run, owned by the caller and used by every run),
 * each advanced `nsteps` time steps per sw_batch_run. Allocates the flank
 * buffers, per-structure completion flags and the work tables (owned by the
 * batch). Errors: SW_ERR_BAD_ARG, SW_ERR_OOM, SW_ERR_CUDA, SW_ERR_UNSUPPORTED. */
typedef struct sw_batch sw_batch;
SW_API int sw_batch_create(const sw_problem *probs, void *const *states, int32_t count, int64_t nsteps,
                           sw_batch **out);

/* Advance every problem of the batch by nsteps: one persistent kernel whose
 * CTAs take (phase, problem, chunk of structures) items from a device-side
 * counter and wait (bounded, ~1 s) for the two neighbouring structures of the
 * previous phase. The reset of the counter/flags and the launch are captured in
 * a CUDA graph on the first call and replayed on `stream` afterwards.
 * Asynchronous; results are bitwise those of sw_run on each problem. */
SW_API int sw_batch_run(sw_batch *b, void *stream);

/* Synchronise `stream`; return the last run's device status (SW_OK, or
 * SW_ERR_TIMEOUT if a dependency wait ran out and the launch was abandoned). */
SW_API int sw_batch_status(sw_batch *b, void *stream);

/* Work items per run (for reporting). */
SW_API int64_t sw_batch_items(const sw_batch *b);

/* Threads per CTA of the persistent kernel: 64, 128 (the default) or 256; each CTA
 * runs one structure at a time with all its threads, so narrow tiles leave fewer of
 * them idle with fewer threads and wide ones have more work per level. Synchronises
 * the device; the next sw_batch_run captures its graph again. Errors: SW_ERR_BAD_ARG,
 * SW_ERR_CUDA. */
SW_API int sw_batch_set_threads(sw_batch *b, int32_t threads);

/* Failure-injection hook for tests: set the dependency-wait budget in clock
 * cycles and, if drop_publish != 0, make structure 0 of problem 0 never
 * publish its first phase so that its neighbours' waits run out. */
SW_API int sw_batch_debug(sw_batch *b, int64_t wait_budget_cycles, int32_t drop_publish);

SW_API void sw_batch_destroy(sw_batch *b);

/* Tile-width autotuner (Section 6 advises tuning the block size on a
 * few short runs): times `probe_steps` steps of a probe state (heat: 1.5 +
 * a smooth sine, one sign, as the data-dependent FP64 integer-pipe path expects of
 * smooth fields; Euler: uniform, at rest) for each W in {32, ..., 1024} that divides
 * n (with n >= 2W),
 * using the problem's own flags (SW_FLAG_GENERIC tunes the generic kernel that
 * batches use), and writes the fastest to inout->tile_width. For an Euler
 * problem with neither SW_FLAG_LENGTHENED nor SW_FLAG_FLATTENED it times both
 * forms of Section 4.3 at each W and ORs the faster form's flag into
 * inout->flags. Allocates a temporary state; synchronises `stream`. */
SW_API int sw_autotune(sw_problem *inout, int64_t probe_steps, void *stream);

/* ---- two dimensions: FTCS heat on an nx x ny grid (the 5-point stencil) ----------
 * Section 6 names the extension of the swept rule to two dimensions as future work;
 * this is that extension for the heat equation, built as the product of two 1D swept
 * decompositions. At the levels between two full levels every cell belongs to one of
 * four kinds of region, each the product of a 1D lower (widening) or upper
 * (narrowing) window in x and in y: pyramids (upper x upper, self-contained),
 * x-bridges (lower x upper) and y-bridges (upper x lower), each importing the two
 * outermost cells of its neighbours per level on its widening sides, and
 * octahedra (lower x lower), which import from four bridges and the corners of four
 * pyramids, reach the full W x W tile and go on to build the next pyramid. One phase
 * = one bridges launch and one octahedra launch, W/2 levels; the 2-cell-deep strips
 * travel through HBM between them, as the flanks of the 1D rule do. No cell of any
 * level is computed twice.
 * Update, per cell: u' = fma(rx, fma(-2, u, a + b), fma(ry, fma(-2, u, d + e), u)),
 * a, b the x-neighbours and d, e the y-neighbours (a state constant along y gives the
 * 1D update bit for bit). State: nx * ny values, row-major, x fastest
 * (u[j * nx + i]), double (SW_FP64) or float (SW_FP32).
 * Swept runs are periodic; nx and ny multiples of W with at least two tiles each;
 * W even, 8 <= W <= the width the shared memory holds (FP64 118, FP32 166); a run
 * of L steps does floor(L / (W/2)) swept phases and the remaining L mod (W/2) steps
 * with the per-step kernel (same bits). Per-step runs: periodic or transmissive. */
typedef struct sw_heat2d {
    int32_t precision;  /* SW_FP64 or SW_FP32 */
    int32_t boundary;   /* SW_PERIODIC, or SW_TRANSMISSIVE (per-step only) */
    int32_t method;     /* SW_SWEPT or SW_PERSTEP */
    int32_t tile_width; /* W (swept); 0 = the library default (64) */
    int64_t nx, ny;     /* grid, each >= 4 (swept: >= 2W), nx * ny <= 2^36 */
    double rx, ry;      /* alpha dt / dx^2 and alpha dt / dy^2, each > 0 */
} sw_heat2d;

typedef struct sw_handle2d sw_handle2d;

/* Validate and allocate the strip buffers (swept) or a second plane (per-step) on the
 * current device. Errors: SW_ERR_BAD_ARG, SW_ERR_UNSUPPORTED (W beyond shared
 * memory), SW_ERR_OOM, SW_ERR_CUDA. SW_WARN_UNSTABLE (and a handle) when
 * rx + ry > 1/2. */
SW_API int sw2d_create(const sw_heat2d *p, sw_handle2d **out);
SW_API void sw2d_destroy(sw_handle2d *h);
/* Advance `state` (device, layout above) by nsteps in place on `stream`. */
SW_API int sw2d_run(sw_handle2d *h, void *state, int64_t nsteps, void *stream);
/* Launches issued by the last sw2d_run, and the tile width in use. */
SW_API int64_t sw2d_last_launch_count(const sw_handle2d *h);
SW_API int32_t sw2d_tile_width(const sw_handle2d *h);
/* Threads per CTA of the swept kernels of a swept handle: `threads` for the Up and
 * octahedra launches, `bridge_threads` for the bridges; each 128, 256 or 1024, 0 for the
 * default (FP32: 128 below W = 128, from there 1024 and 256 for the bridges; FP64: 256;
 * the fastest on 8192^2 x 2048 steps on GB300). A tuning choice only: every count
 * computes the same cells with the same arithmetic, so results are bitwise equal.
 * Takes effect at the next sw2d_run. SW_ERR_BAD_ARG for another count or a per-step
 * handle. sw2d_threads returns the count in use (bridges != 0: the bridges'), 0 for a
 * per-step handle. */
SW_API int sw2d_set_threads(sw_handle2d *h, int32_t threads, int32_t bridge_threads);
SW_API int32_t sw2d_threads(const sw_handle2d *h, int32_t bridges);
/* Tracing, as sw_set_timing / sw_launch_times (kinds: 0 Up pyramids, 1 bridges,
 * 2 octahedra, 3 per-step, 4 the last phase's octahedra). */
SW_API int sw2d_set_timing(sw_handle2d *h, int64_t capacity);
SW_API int64_t sw2d_launch_times(sw_handle2d *h, float *ms, int32_t *kind, int64_t cap);

SW_API const char *sw_status_string(int status);
SW_API int sw_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SWEPT_H */

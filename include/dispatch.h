/*
 * dispatch.h -- C ABI of the GB300 per-patch update library (libdispatch_gpu.so).
 *
 * The library advances a set of Cartesian patches of ideal MHD with local,
 * power-of-two time steps, as in DISPATCH (Nordlund et al. 2018, "DISPATCH: a
 * numerical simulation framework for the exa-scale era. I. Fundamentals"):
 *
 *   - each patch is a task with a position, a size, guard zones and a circular
 *     buffer of time slices (Sec. 2.1; Sec. 3 A);
 *   - before an update its guard zones are filled by linear (or quadratic)
 *     interpolation in time from its neighbours' slices, or extrapolation
 *     past a neighbour's newest slice when the grace allows it (Sec. 3 A;
 *     closing paragraph of Sec. 3 B);
 *   - a patch is ready when Eq. (1) holds for every neighbour:
 *     t_self <= t_nbor + g dt_nbor;
 *   - the update is one local Courant step (Sec. 5.1) of a MUSCL-Hancock
 *     scheme with HLL (or HLLD) fluxes and constrained transport of
 *     face-centred B (Secs. 4.1 and 4.3 name the solver family; the paper
 *     prints no scheme), optionally with the Ohmic and ambipolar terms of
 *     Sec. 4.3;
 *   - the new state overwrites the oldest slice (Sec. 3 A).
 *
 * Every call returns 0 on success or one of the negative DSP_ERR_* codes.
 * After DSP_ERR_UNPHYSICAL, DSP_ERR_TIMEOUT, DSP_ERR_DEADLOCK, DSP_ERR_BRACKET,
 * DSP_ERR_BOUNDS or DSP_ERR_CUDA the context is poisoned: only dsp_get_state, dsp_get_times,
 * dsp_get_schedule, dsp_diagnostics, dsp_last_error and dsp_destroy remain
 * valid.  Calls on one context are not thread-safe; distinct contexts are
 * independent.  All device work is issued on the stream given to dsp_create
 * and is ordered after the caller's earlier work on that stream.
 */
#ifndef DISPATCH_GPU_H
#define DISPATCH_GPU_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DSP_API __attribute__((visibility("default")))
#else
#define DSP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define DSP_OK 0
#define DSP_ERR_INVALID_ARG (-1)      /* bad pointer, size, layout or parameter */
#define DSP_ERR_OOM (-2)              /* device or host allocation failed */
#define DSP_ERR_CUDA (-3)             /* a CUDA runtime call failed */
#define DSP_ERR_UNPHYSICAL (-4)       /* rho <= 0 or p <= 0 in a new state */
#define DSP_ERR_TIMEOUT (-5)          /* a bounded device wait ran out */
#define DSP_ERR_DEADLOCK (-6)         /* no patch ready while some are behind t_end */
#define DSP_ERR_SCHEDULE_OVERFLOW (-7) /* the schedule log was larger than its capacity */
#define DSP_ERR_UNSUPPORTED (-8)      /* a valid request this build does not implement */
#define DSP_ERR_BRACKET (-9)          /* a neighbour's slices do not bracket a guard time */
#define DSP_ERR_BOUNDS (-10)          /* bounds-checked build only: a global address outside every buffer */

typedef struct dsp_ctx dsp_ctx;

/* One patch (Sec. 2.1, the patch data type): its refinement level, its
 * interior cells per axis (x, y, z) and the index of its first interior cell
 * in the level's cell index space (level l has base_cells * 2^l cells per
 * axis, cell size dx / 2^l).  Every patch has n > nguard on every axis.
 * Level-0 patches (sizes may differ) must tile the periodic box exactly.
 * Level-1 patches are optional: disjoint, each covering whole level-0 cells
 * (even lo and n).  Guard values across the resolution jump follow Sec. 3 A
 * (interpolation in space as well as in time): a level-1 guard cell that no
 * level-1 patch owns is its level-0 parent plus a quarter of the parent's
 * MC-limited slopes signed by the child's side; a level-1 guard face is the
 * level-0 face it lies on, or the mean of the parent's two faces along its
 * axis; a level-0 guard cell covered by level 1 is the mean of its 8
 * children, a face the mean of the 4 level-1 faces on it.  Level-0 patches
 * under the refined region are still advanced. */
typedef struct {
  int32_t level;
  int32_t n[3];
  int64_t lo[3];
} dsp_patch_desc;

/* Physics and execution parameters.
 *   gamma        adiabatic index of the gamma-law equation of state
 *   cfl          Courant number C of the local step dt = C dx / s_max
 *   t0           time of the initial state
 *   dt_max       upper bound on any step (0 = none); use a power of two
 *   grace        g of Eq. (1), 0 <= g < 1: a patch may step while up to g times
 *                a neighbour's last step ahead of it, that neighbour's guard
 *                values then extrapolated in time; a patch keeps its oldest
 *                slice while a neighbour that may step first still needs it.
 *                g > 0 needs the sweep dispatcher (DSP_ERR_UNSUPPORTED with
 *                the ready queue, whose result would depend on timing)
 *   box_lo, box_len   the periodic box; cells must be cubic
 *   base_cells   level-0 cells per axis
 *   nguard       guard zones per side (>= 2; the stencil reads two)
 *   nslices      time slices per patch (3 to 16; 4 or more for quadratic
 *                extrapolation with g > 0)
 *   precision    0: all state and arithmetic in FP64, no fused multiply-add
 *                   (bit-identical to a plain FP64 evaluation);
 *                1: FP32 state and stencil arithmetic, FP64 times and steps;
 *                2: FP64 state and arithmetic with fused multiply-adds
 *   time_mode    0: one global step per sweep (the smallest patch step);
 *                1: local steps, each patch its own
 *   dt_pow2      must be 1: steps are powers of two, so times are exact
 *   dispatcher   1: sweeps over the ready set (one kernel pair per sweep);
 *                0: persistent device ready queue (local steps only): one
 *                   launch runs every update to t_end; blocks claim (patch,
 *                   tile) work, and the block finishing a patch publishes it
 *                   and queues every neighbour it made ready
 *   tile_x, tile_y, tile_z   update tile in cells (0 = defaults)
 *   sched_capacity  entries kept in the schedule log (0 = no log)
 *   timing       1: time every update-kernel launch with CUDA events on the
 *                context's stream and report the total in dsp_stats
 *   wait_budget  ready-queue dispatcher only: SM clock cycles a device wait
 *                may spin without progress before the run stops with
 *                DSP_ERR_TIMEOUT (0 = default, about two seconds)
 *   variant      id of a compiled update-kernel variant of this precision and
 *                Riemann solver to use (-1 = the default; see dsp_autotune)
 *   graph        sweep dispatcher only: 1 = capture batches of 32 sweeps
 *                (plan + update kernels) in a CUDA graph and replay it; with
 *                a NULL stream the context then creates its own blocking
 *                stream (the legacy stream cannot be captured)
 *   riemann      face fluxes: 0 = HLL, 1 = HLLD (Miyoshi & Kusano 2005; the
 *                MHD solver whose cell-update cost Sec. 5.3 compares with
 *                RAMSES), which resolves isolated contacts and rotational
 *                discontinuities exactly; the edge EMFs stay the upwind HLL
 *                ones.  Any other value: DSP_ERR_INVALID_ARG
 *   eta          Ohmic resistivity eta_Ohm >= 0 (0 = no Ohmic term): the EMF
 *                gains eta J, J = curl B on the cell edges (DISPATCH I,
 *                Sec. 4.3, Eq. 2), and the step is limited to
 *                c_ohm dx^2 / eta (Eq. 4)
 *   gamma_ad     ambipolar drift coefficient gamma_AD >= 0 (0 = no ambipolar
 *                term): the EMF gains -v_D x B with v_D = J x B /
 *                (gamma_AD rho rho_i) (Eqs. 5-6), the step is limited to
 *                c_ad gamma_AD rho_i rho dx^2 / B^2 (Eq. 8)
 *   rho_i        ion density of the ambipolar term (> 0 when gamma_ad > 0)
 *   c_ohm, c_ad  Courant-like factors of the two limits (0 = 0.1, the
 *                paper's value).  The Poynting flux of the non-ideal EMF
 *                joins the energy flux, so total energy stays conserved and
 *                the heating of Eqs. 3 and 7 goes into the internal energy.
 *                A negative or non-finite coefficient: DSP_ERR_INVALID_ARG
 *   time_order   order of the time inter- and extrapolation of guard values:
 *                1 (or 0) linear between the two slices around the time (the
 *                newest two past the newest slice); 2 quadratic through those
 *                and the next older slice (the next newer where none is
 *                older; the newest three past the newest), which the closing
 *                paragraph of Sec. 3 B allows; any other value:
 *                DSP_ERR_INVALID_ARG
 *   owned        NULL: every patch is this context's own.  Else one byte per
 *                patch: 1 = owned (updated here), 0 = virtual, a copy of a
 *                patch that another process owns (Sec. 3 C, the MPI process
 *                view): never updated here, its new states arrive through
 *                dsp_unpack.  With virtual patches the layout is one
 *                process's share: it need not tile the box, but every guard
 *                cell (nguard layers) of an owned patch must lie in a patch of
 *                the layout (else DSP_ERR_INVALID_ARG); it needs local steps,
 *                g = 0, the sweep dispatcher and one level (else
 *                DSP_ERR_UNSUPPORTED); a sweep with no owned patch ready
 *                returns normally (it waits for other processes), and
 *                dsp_diagnostics counts owned patches only.  The array is
 *                read during dsp_create only */
typedef struct {
  double gamma, cfl, t0, dt_max, grace;
  double box_lo[3], box_len[3];
  int32_t base_cells[3];
  int32_t nguard, nslices, precision, time_mode, dt_pow2, dispatcher;
  int32_t tile_x, tile_y, tile_z;
  int64_t sched_capacity;
  int32_t timing;
  int64_t wait_budget;
  int32_t graph;
  int32_t variant;
  int32_t riemann;
  double eta, gamma_ad, rho_i, c_ohm, c_ad;
  int32_t time_order;
  const uint8_t *owned;
} dsp_params;

/* Counters of one dsp_advance call.  kernel_ms and kernel_launches are the
 * summed device time and the number of launches of the update kernel (only
 * when timing was requested); plan_launches counts the dispatcher kernels
 * (three per sweep) and, with two levels, the cross-level guard kernel.
 * fallbacks counts cells whose reconstruction fell back to first order (a
 * face state with rho <= 0 or p <= 0); floors counts cells of new slices
 * whose pressure recovery took the floor p >= 1e-20 rho (both 0 on smooth
 * inputs; the paper states neither, see dsp_params). */
typedef struct {
  int64_t patch_updates, cell_updates, sweeps, fallbacks;
  double t_min, t_max;
  int32_t status;
  double kernel_ms;
  int64_t kernel_launches, plan_launches;
  int64_t floors;
} dsp_stats;

/* One schedule entry: patch index, start time, step. */
typedef struct {
  int64_t patch;
  double t_start, dt;
} dsp_sched_entry;

/* Diagnostics of the newest slices: volume integrals of rho, m, E and of the
 * face fields (each face once), with FP64 compensated sums; the largest
 * |sum_d Delta_d b| over cells and the largest |b| over faces. */
typedef struct {
  double mass, mom[3], energy, bmean[3], max_divb, max_b;
} dsp_diag;

/* Create a context (the task list of Sec. 2.2 for a set of patches, each the
 * patch data type of Sec. 2.1 laid out as by the "cartesian" component of
 * Sec. 2.3, with nslices time slices of Sec. 3 A): validates the layout,
 * builds the neighbour ("nbor") tables, allocates every slice on the current
 * CUDA device.  stream is a
 * cudaStream_t (NULL = legacy default stream).  On success *out owns all
 * device memory until dsp_destroy.  Neighbours are symmetric: on the same
 * level, patches whose interior meets the padded box; across levels,
 * patches whose interior meets the cells a patch may read on the other
 * level.  Returns DSP_ERR_INVALID_ARG for a layout that breaks the rules of
 * dsp_patch_desc, DSP_ERR_UNSUPPORTED for levels other than 0 and 1, for two
 * levels with the ready-queue dispatcher, or for grace > 0 with the
 * ready-queue dispatcher. */
DSP_API int dsp_create(const dsp_patch_desc *patches, int32_t npatch, const dsp_params *params, void *stream,
               dsp_ctx **out);

/* Load the state of patches [first, first+count) (the interior state
 * variables of Sec. 3 A; guard zones are never stored, they are filled from
 * the neighbours' slices at each update) into their first slice at
 * time t0 (and reset every patch's time to t0 when first == 0 and count ==
 * npatch).  Arrays are the concatenation, in patch order, of each patch's
 * interior: U[5][nz][ny][nx] (rho, m_x, m_y, m_z, E), bx[nz][ny][nx+1],
 * by[nz][ny+1][nx], bz[nz+1][ny][nx], x fastest.  dtype: 0 = float64,
 * 1 = float32 (converted to the context's precision).  on_device: 1 if the
 * pointers are device memory.  The arrays are copied; the caller keeps them. */
DSP_API int dsp_set_state(dsp_ctx *ctx, int32_t first, int32_t count, const void *U, const void *bx, const void *by,
                  const void *bz, int32_t dtype, int32_t on_device);

/* Advance until every patch has reached t_end, or until max_sweeps sweeps
 * have run (<= 0: no limit; then t_end must be finite): the task list's
 * execute procedure of Sec. 2.2, which calls the update of Sec. 3 B (select
 * the ready tasks by Eq. 1, update each, re-check its neighbours) until every
 * task reached its final time.  Each patch update is the single-task cycle
 * of Sec. 3 A: guard zones by time interpolation, one local Courant step
 * (Sec. 5.1), the new state into the oldest slice.  Synchronous: returns
 * after the device work finished, with the status of the run (a non-zero
 * status also poisons the context, see above).  A sweep limit ends the call
 * between sweeps, leaving a consistent state.  out may be NULL. */
DSP_API int dsp_advance(dsp_ctx *ctx, double t_end, int64_t max_sweeps, dsp_stats *out);

/* Copy the newest slice (Sec. 3 A, the most recent state of the circular
 * buffer) of patches [first, first+count) out, same layout and
 * dtype/on_device conventions as dsp_set_state.  The caller owns the arrays;
 * host arrays are staged through a library-owned device buffer.  Valid on a
 * poisoned context. */
DSP_API int dsp_get_state(dsp_ctx *ctx, int32_t first, int32_t count, void *U, void *bx, void *by, void *bz,
                  int32_t dtype, int32_t on_device);

/* Per-patch time of the newest slice and last step (the task times and time
 * steps of Sec. 2.1 that Eq. 1 compares), into host arrays of npatch values
 * owned by the caller; dt_last may be NULL.  Valid on a poisoned context. */
DSP_API int dsp_get_times(dsp_ctx *ctx, double *t, double *dt_last);

/* Copy up to cap schedule entries (one per patch update: which task the
 * dispatcher of Sec. 3 B updated, from which time, by which step), in
 * execution order (patch order within a sweep), into the caller's host
 * buffer; *n receives the total recorded so far.  Returns
 * DSP_ERR_SCHEDULE_OVERFLOW if more updates ran than the log's capacity
 * (dsp_params.sched_capacity; the first capacity entries are still valid).
 * buf may be NULL to query *n.  Valid on a poisoned context. */
DSP_API int dsp_get_schedule(dsp_ctx *ctx, dsp_sched_entry *buf, int64_t cap, int64_t *n);

/* Diagnostics of the newest slices of every patch (see dsp_diag): the paper
 * has no counterpart (its validation, Sec. 5, compares runs rather than
 * sums); they serve the conservation and div B checks.  Every cell counts
 * with its own level's cell volume (level-0 cells under a refined region
 * too); each face counts once, as the low face of a cell; the sums are FP64
 * Neumaier-compensated per patch in a fixed order, then over patches in patch
 * order, so the result is deterministic.  Allocates a small device buffer
 * (10 doubles per patch) for the per-patch partials; writes *out on the
 * host.  Valid on a poisoned context. */
DSP_API int dsp_diagnostics(dsp_ctx *ctx, dsp_diag *out);

/* Autotuner: for each patch-size class of the context (each distinct patch
 * size, up to four, with the sweep dispatcher; else one class), time every
 * compiled variant of the update kernel that fits (tile shape, threads per
 * block, blocks per SM) with each z run of a work item (the patches' whole
 * height and half of it, or dsp_params.tile_z when set) on the next sweep's
 * real ready list of that class, `reps` launches each, and keep the fastest
 * per class; every sweep then launches each class's own variant.  The paper
 * has no autotuner; its Sec. 5.3 notes that the best patch size depends on
 * the problem and the hardware, and on a GPU so does the tiling of a patch.
 * Nothing is published and the state is unchanged (the update writes only
 * the patches' next slot); all variants and z runs compute bit-identical
 * results.  Call after dsp_set_state, before dsp_advance.  Writes the
 * variant chosen for class 0, and for up to cap candidates their ids
 * (class * 1000000 + z run * 1000 + variant id) and average milliseconds per
 * launch; *n receives the number of candidates timed; dsp_get_tuning gives
 * the choice of every class.  Any output pointer may be NULL. */
DSP_API int dsp_autotune(dsp_ctx *ctx, int32_t reps, int32_t *chosen, double *ms, int32_t *ids, int32_t cap,
                         int32_t *n);

/* The tuning in use: *ncls size classes; for each of the first cap classes
 * its patch size (sizes[3k..3k+2], x y z), update-kernel variant and z run.
 * Any output array may be NULL. */
DSP_API int dsp_get_tuning(dsp_ctx *ctx, int32_t cap, int32_t *ncls, int32_t *sizes, int32_t *variant,
                           int32_t *tile_z);

/* Maximum number of patches dsp_diagnostics_noalloc accepts. */
#define DSP_NOALLOC_MAX_PATCHES 16384

/* The diagnostics of dsp_diagnostics, computed from a state held in the
 * caller's own device arrays (the dsp_set_state layout: U, bx, by, bz
 * concatenated over npatch patches of n[0] x n[1] x n[2] cells, cell size dx;
 * dtype 0 = float64, 1 = float32), without allocating any device memory.
 * Unlike dsp_diagnostics, every patch must have the same size n and the
 * same cell size dx (one level, one patch size): mixed sizes or a second
 * level need dsp_diagnostics.
 * This entry point has no counterpart in the paper; it exists for callers
 * that cannot call cudaMalloc: a host application that hands all device
 * memory to its own pool allocator and forbids raw allocations, or a
 * latency-sensitive loop sharing the GPU with other streams, where
 * cudaMalloc's implicit device-wide synchronisation would stall the other
 * work.  Its scratch is a fixed file-scope device array sized for
 * DSP_NOALLOC_MAX_PATCHES patches (about 1.3 MB on every GPU that loads the
 * library, held until the process exits).  npatch above that limit, or any
 * invalid argument, returns DSP_ERR_INVALID_ARG before any work is issued.
 * The first call on a device looks up the array's device address (that
 * device must be current; make this first call before any stream capture).
 * Work is issued on `stream` (a cudaStream_t) and the call returns after it
 * finished, writing *out on the host.  All calls share the scratch array:
 * calls whose kernels overlap on one GPU race and may return wrong values. */
DSP_API int dsp_diagnostics_noalloc(const void *U, const void *bx, const void *by, const void *bz, int32_t dtype,
                                    int32_t npatch, const int32_t *n, double dx, void *stream, dsp_diag *out);

/* Save the whole dispatcher state (every slice, its time and signal speed,
 * the newest-slice index and last step of every patch) into host memory: a
 * snapshot suitable for restarting, as the I/O view of Sec. 3 E asks of
 * DISPATCH snapshots (one binary blob here, no file format).
 * Layout: a 40-byte header (char magic[8] = "DSPSAVE", int32 version = 1,
 * npatch, nslices, precision, int64 reserved, int64 slot_stride), then
 * double t[npatch][nslices], double smax[npatch][nslices], int32
 * newest[npatch], double dt_last[npatch], and the slices: nslices blocks of
 * slot_stride values (float64, or float32 for precision 1), each the
 * concatenation over patches of U, bx, by, bz in the dsp_set_state layout.
 * With buf == NULL only *used (the required size) is written.  dsp_load
 * restores a state saved from a context with the same layout and parameters;
 * a run resumed from it is bit-identical to the uninterrupted run. */
DSP_API int dsp_save(dsp_ctx *ctx, void *buf, size_t cap, size_t *used);
DSP_API int dsp_load(dsp_ctx *ctx, const void *buf, size_t size);

/* Packages between processes (Sec. 3 C, the MPI process view): after a
 * process updates a patch that other processes hold as a virtual copy, it
 * sends them the patch's whole interior and its time parameters, and each
 * receiver stores them as the copy's new slice.  The paper ships the whole
 * interior rather than guard layers only, which keeps packing simple; so do
 * these calls.  A package of patch P is its newest slice: the values of U,
 * bx, by, bz of P (dsp_set_state layout of one patch), contiguous, in the
 * context's precision (float64, or float32 for precision 1), and three
 * doubles of meta: the slice's time, P's last step, the slice's signal
 * speed.  A list's packages are concatenated in list order.
 *
 * dsp_package_len: the number of values (not bytes) of the packages of the
 * listed patches (distinct indices of this context).
 * dsp_pack: write the packages of the listed patches into buf and meta
 * (3 * count doubles); on_device: 1 if buf and meta are device memory, else
 * host memory staged through a library-owned device buffer.
 * dsp_unpack: store each listed package as the newest slice of its patch,
 * which must be virtual (DSP_ERR_INVALID_ARG otherwise): written into the
 * slot after the newest, which then becomes the newest, with the meta's
 * time, last step and signal speed.  Not on a poisoned context.
 * All three copy: the caller keeps its arrays; both are synchronous. */
DSP_API int dsp_package_len(dsp_ctx *ctx, const int32_t *ids, int32_t count, int64_t *values);
DSP_API int dsp_pack(dsp_ctx *ctx, const int32_t *ids, int32_t count, void *buf, double *meta, int32_t on_device);
DSP_API int dsp_unpack(dsp_ctx *ctx, const int32_t *ids, int32_t count, const void *buf, const double *meta,
                       int32_t on_device);

/* Message of the last error on this context ("" if none).  Valid until the
 * next call on the context.  No counterpart in the paper. */
DSP_API const char *dsp_last_error(dsp_ctx *ctx);

/* Release every device and host allocation of the context (after the
 * context's stream has finished its work).  NULL is ignored. */
DSP_API void dsp_destroy(dsp_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif

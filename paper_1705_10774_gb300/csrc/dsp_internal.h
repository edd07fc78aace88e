// dsp_internal.h -- device context shared by the library's translation units.
#pragma once
#include <cstdint>

#include "../../include/dispatch.h"

namespace dsp {

// Control words in device memory (int32 each).
enum Ctl : int {
  CTL_NREADY = 0,   // patches in the current ready list
  CTL_STATUS = 1,   // 0 or a DSP_ERR_* code (first error wins)
  CTL_DONE = 2,     // 1 once no patch is behind t_end
  CTL_ERRP = 3,     // patch of the first error
  CTL_ERRC = 4,     // cell (linear, patch-local) of the first error
  CTL_COUNT = 8
};

// 64-bit counters in device memory.
enum Cnt : int {
  CNT_PATCH_UPDATES = 0,
  CNT_CELL_UPDATES = 1,
  CNT_SWEEPS = 2,
  CNT_FALLBACKS = 3,
  CNT_NSCHED = 4,
  CNT_COUNT = 8
};

// Everything a kernel needs, passed by value.  Slices are stored slice-major:
// slice s of patch P starts at slab + s * slot_stride + P * patch_len
// (elements of the context's precision), and holds U[5][nz][ny][nx],
// bx[nz][ny][nx+1], by[nz][ny+1][nx], bz[nz+1][ny][nx].
struct DevCtx {
  int np, ns;
  int nx, ny, nz;
  int tx, ty, tz;          // tile extents in cells
  int ntx, nty, ntz;       // tiles per axis
  int tiles;               // tiles per patch
  long long nc, nfx, nfy, nfz, patch_len, slot_stride;
  double gamma, cfl, dx, dt_max;
  void *slab;
  double *t_slot;          // [np][ns]
  double *smax_slot;       // [np][ns]
  int *latest;             // [np]
  double *dt_last;         // [np]
  const int *nb27;         // [np][27] patch at offset (ox,oy,oz) in {-1,0,1}^3, index (oz+1)*9+(oy+1)*3+(ox+1)
  const int *nbl_off;      // [np+1] CSR of distinct neighbours (self excluded)
  const int *nbl;
  int *R;                  // [np] ready list of the current sweep
  double *dtR;             // [np] step of each ready patch
  unsigned long long *smax_new;  // [np] signal speed of the slice being written (double bits)
  int *ctl;                // [CTL_COUNT]
  long long *cnt;          // [CNT_COUNT]
  dsp_sched_entry *sched;  // [sched_cap]
  long long sched_cap;
  // persistent ready queue (dispatcher 0): a ring of np entries
  int *q_patch;                    // [np] patch of each ring slot
  double *q_dt;                    // [np] its step
  unsigned long long *q_seq;       // [np] sequence number published in the slot
  unsigned long long *q_free;      // [np] sequence number the slot may take next
  int *q_reads;                    // [np] tiles of the slot's entry claimed so far
  unsigned long long *q_ctl;       // [4]: 0 next work item, 1 next entry, 2 patches done
  int *p_state;                    // [np] 0 idle, 1 queued or being updated
  int *tiles_done;                 // [np]
  long long wait_budget;           // clock64 cycles a wait may spin before DSP_ERR_TIMEOUT
};

// Launchers implemented in the precision-specific translation units.
int launch_update_f64(const DevCtx &c, int grid, void *stream);
int launch_update_f32(const DevCtx &c, int grid, void *stream);
int launch_update_f64f(const DevCtx &c, int grid, void *stream);
int update_grid_f64f(const DevCtx &c);
int launch_queue_f64(const DevCtx &c, int grid, double t_end, void *stream);
int launch_queue_f64f(const DevCtx &c, int grid, double t_end, void *stream);
int launch_queue_f32(const DevCtx &c, int grid, double t_end, void *stream);
int update_grid_f64(const DevCtx &c);
int update_grid_f32(const DevCtx &c);
void update_tile_f64(int *tx, int *ty);
void update_tile_f32(int *tx, int *ty);

}  // namespace dsp

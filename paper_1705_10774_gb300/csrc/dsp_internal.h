// dsp_internal.h -- device context shared by the library's translation units.
#pragma once
#include <cstdint>

#include "../../include/dispatch.h"
#include "dsp_variants.h"

namespace dsp {

// Control words in device memory (int32 each).
enum Ctl : int {
  CTL_NREADY = 0,   // patches in the current ready list
  CTL_STATUS = 1,   // 0 or a DSP_ERR_* code (first error wins)
  CTL_DONE = 2,     // 1 once no patch is behind t_end
  CTL_ERRP = 3,     // patch of the first error
  CTL_ERRC = 4,     // cell (linear, patch-local) of the first error
  CTL_NOTDONE = 5,  // set by the readiness pass when some patch is behind t_end
  CTL_CLS = 8,      // [MAXCLS + 1]: first ready-list entry of each size class, then the end
  CTL_COUNT = 16
};

// Patch-size classes: each distinct patch size (up to MAXCLS of them) has its
// own update-kernel variant and z run, chosen by dsp_autotune; more sizes
// share one class.
constexpr int MAXCLS = 4;

// 64-bit counters in device memory.
enum Cnt : int {
  CNT_PATCH_UPDATES = 0,
  CNT_CELL_UPDATES = 1,
  CNT_SWEEPS = 2,
  CNT_FALLBACKS = 3,
  CNT_NSCHED = 4,
  CNT_FLOORS = 5,  // cells of new slices whose pressure recovery took the floor
  CNT_COUNT = 8
};

// Per-patch geometry (device memory).  Slice s of patch P starts at
// slab + s * slot_stride + off, and holds U[5][nz][ny][nx],
// bx[nz][ny][nx+1], by[nz][ny+1][nx], bz[nz+1][ny][nx] (elements of the
// context's precision).
struct PatchGeo {
  int n[3];       // interior cells per axis
  int nt[3];      // update tiles per axis
  int tiles;      // nt[0] * nt[1] * nt[2]
  int lo[3];      // first interior cell in the level's index space
  int level;      // refinement level (0, or 1 at half the cell size)
  int tz;         // z run of the patch's work items (cells)
  int cls;        // size class
  long long off;  // offset of the patch inside a slice
};

// Largest number of map blocks one work item's padded tile may touch.
constexpr int TABMAX = 128;

// Everything a kernel needs, passed by value.
struct DevCtx {
  int np, ns;
  int ncls;                // size classes (1..MAXCLS)
  long long total_tiles;   // tiles of all patches
  long long cls_tiles[MAXCLS];  // tiles of each class's patches
  long long slot_stride;   // elements of one slice of all patches
  const PatchGeo *geo;     // [np]
  // per level l: the periodic box of L[l] cells per axis cut into blocks of
  // bsz[l] cells.  omap[l][block] = the level-l patch owning the block, or -1
  // (level 1 outside the refined region).  gmap[l] is what a level-l patch's
  // guard gather uses: omap[l] except -1 wherever the value comes from the
  // other level (level 0: blocks covered by level 1; level 1: uncovered).
  int nlev;
  const int *omap[2];
  const int *gmap[2];
  int bsz[2][3], mapd[2][3], L[2][3];
  float binv[2][3];
  // cross-level guard values of each patch that has some (-1 otherwise):
  // a padded box of n + 4 cells per axis starting at lo - 2, laid out like a
  // patch slice, refilled before every update of the patch
  void *gbuf;
  long long gbuf_len;      // elements of gbuf
  const long long *gofs;   // [np] element offset into gbuf, or -1
  const long long *coff;   // [4][np+1] offsets of each patch in the caller's U, bx, by, bz arrays
  int *work_off;           // [np+1] first work item of each ready patch (prefix of tiles)
  double gamma, cfl, dx, dt_max;
  // non-ideal MHD (Sec. 4.3): Ohmic resistivity, ambipolar drift coefficient
  // and ion density, Courant-like factors of their step limits (0 = off)
  double eta, gad, rhoi, cohm, cad;
  // grace g of Eq. (1) and the order of the time inter- and extrapolation of
  // guard values (1 linear, 2 quadratic)
  double grace;
  int torder;
  void *slab;
  double *t_slot;          // [np][ns]
  double *smax_slot;       // [np][ns]
  int *latest;             // [np]
  double *dt_last;         // [np]
  // several processes (Sec. 3 C): owned[P] = 1 for a patch this context
  // updates, 0 for a virtual copy of a patch another process owns (NULL:
  // every patch is owned); partial = 1 when some patch is virtual
  const int *owned;
  int partial;
  const int *nbl_off;      // [np+1] CSR of distinct neighbours (self excluded)
  const int *nbl;
  int *R;                  // [np] ready list of the current sweep (patch order)
  int *Rk;                 // [np] the work list: indices into R grouped by size class
  int *rflag;              // [np] readiness of each patch (dispatcher scratch)
  double *rdt;             // [np] its step
  double *dtR;             // [np] step of each ready patch
  unsigned long long *smax_new;  // [np] signal speed of the slice being written (double bits)
  int *ctl;                // [CTL_COUNT]
  long long *cnt;          // [CNT_COUNT]
  dsp_sched_entry *sched;  // [sched_cap]
  long long sched_cap;
  // persistent ready queue (dispatcher 0): a ring of q_cap tile tickets,
  // each one work item (a tile of a queued patch)
  long long q_cap;                 // ring slots: twice the tiles of all patches, plus the blocks' tickets
  int *q_patch;                    // [q_cap] patch of each ring slot
  int *q_tile;                     // [q_cap] the tile of that patch
  double *q_dt;                    // [q_cap] its step
  unsigned long long *q_seq;       // [q_cap] ticket published in the slot
  unsigned long long *q_free;      // [q_cap] ticket the slot may take next
  unsigned long long *q_ctl;       // [4]: 0 next ticket to claim, 1 next ticket to push, 2 patches done
  int *p_state;                    // [np] 0 idle, 1 queued or being updated
  int *tiles_done;                 // [np]
  long long wait_budget;           // clock64 cycles a wait may spin before DSP_ERR_TIMEOUT
};

// A compiled variant of the update kernels (see dsp_variants.h).
struct KernelVariant {
  int id, precision;  // precision code of dsp_params
  int riemann;        // Riemann solver of the face fluxes (dsp_params.riemann)
  int nonideal;       // 1: with the non-ideal Ohmic and ambipolar terms
  int tx, ty, nt;     // tile and threads per block
  const char *name;
  int (*launch_update)(const DevCtx &c, int grid, void *stream, int cls, int cls_end);
  int (*launch_queue)(const DevCtx &c, int grid, double t_end, void *stream);
  int (*grid)(const DevCtx &c, int cls, int cls_end);
};

#define DSP_DECLARE_VARIANT(id, T, TX, TY, NT, MB, PREC, RS, NI) const KernelVariant *variant_##id();
DSP_VARIANT_LIST(DSP_DECLARE_VARIANT)
#undef DSP_DECLARE_VARIANT

}  // namespace dsp

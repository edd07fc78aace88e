// dsp_host.cu -- the C ABI (include/dispatch.h): context set-up, the sweep
// dispatcher, state transfer, diagnostics and save/load.
//
// Dispatcher (DISPATCH I, Sec. 3 B): each sweep runs three dispatcher kernels
// and the update kernel on the context's stream.  The first publishes the
// previous sweep (new slice becomes the newest, patch time += dt, schedule log
// entry), the second finds every patch that is ready by Eq. (1) (t_P < t_end
// and t_P <= t_N + g dt_N for every neighbour N, and with g > 0 its oldest
// slice no longer needed) and gives it its local Courant step, the third
// compacts the ready patches in index order.  The update kernel then
// advances every ready patch from the pre-sweep slices, and no patch writes a
// slice another ready patch reads, so any order of execution inside a sweep
// gives the same result; with g = 0 sweeping also gives the same per-patch
// schedule as a time-sorted ready queue.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "dsp_diag.cuh"
#include "dsp_dispatch.cuh"
#include "dsp_internal.h"
#include "dsp_levels.cuh"
#include "dsp_physics.cuh"

using namespace dsp;

struct dsp_ctx {
  DevCtx d;
  dsp_params prm;
  cudaStream_t stream;
  int precision;
  size_t esize;
  std::string err;
  int poisoned;
  // host copies of the tables
  std::vector<int> nbl_off, nbl;
  std::vector<PatchGeo> geo;
  std::vector<long long> coff;  // [4][np+1]
  // device allocations
  void *slab;
  double *t_slot, *smax_slot, *dt_last, *dtR;
  int *latest, *nbl_off_d, *nbl_d, *R, *ctl, *omap_d[2], *gmap0_d, *work_off_d, *rflag, *owned_d;
  std::vector<int> owned;      // host copy (1 owned, 0 virtual)
  int *pk_ids;                 // [np] patch list of a pack/unpack call
  long long *pk_off;           // [np+1] its package offsets
  double *pk_meta;             // [3 np] its meta values
  double *rdt;
  long long *gofs_d;
  void *gbuf;
  PatchGeo *geo_d;
  long long *coff_d;
  unsigned long long *smax_new;
  long long *cnt;
  dsp_sched_entry *sched;
  int *q_patch, *q_tile, *p_state, *tiles_done;
  double *q_dt;
  unsigned long long *q_seq, *q_free, *q_ctl;
  long long q_alloc;  // slots of the ready queue's ring as allocated
  void *staging;
  size_t staging_bytes;
  int *h_ctl;  // pinned
  int grid_update;                         // grid of the ready-queue kernel
  // size classes: each class's update-kernel variant, z run and grid
  std::vector<int> cls;                    // [np] class of each patch
  int ncls;
  int cls_n[MAXCLS][3];                    // patch size of each class
  const KernelVariant *var_cls[MAXCLS];
  int tz_cls[MAXCLS];
  int grid_cls[MAXCLS];
  // launch groups: consecutive classes with the same variant share one
  // launch over their stretches of the work list
  int ngrp, grp_lo[MAXCLS], grp_hi[MAXCLS], grid_grp[MAXCLS];
  int *Rk;
  cudaEvent_t ev[2 * 32];
  int nev;
  cudaGraphExec_t graph_exec;  // a captured batch of sweeps
  double graph_t_end;
  int graph_timing;
  int own_stream;  // the context created its stream (graph capture needs one)
  const KernelVariant *var;  // the update-kernel variant of class 0 (the ready queue's)
  int n_xlevel;              // patches with a cross-level guard buffer
  std::vector<dsp_patch_desc> patches;
};

namespace {

int fail(dsp_ctx *c, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(dsp_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
    if (code == DSP_ERR_CUDA) (void)cudaGetLastError();  // do not leak the error into later calls
    if (code == DSP_ERR_CUDA || code == DSP_ERR_UNPHYSICAL || code == DSP_ERR_TIMEOUT || code == DSP_ERR_DEADLOCK ||
        code == DSP_ERR_BRACKET || code == DSP_ERR_BOUNDS)
      c->poisoned = 1;
  }
  return code;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(c, DSP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// ------------------------------------------------------------------ kernels

__device__ void set_status(const DevCtx &c, int code, int P) {
  if (atomicCAS(&c.ctl[CTL_STATUS], 0, code) == 0) c.ctl[CTL_ERRP] = P;
}

constexpr int PLAN_NT = 1024;
constexpr int EVAL_NT = 256;

// Dispatcher step, part 1 (one thread per patch of the previous ready list):
// publish the previous sweep -- the new slice becomes the newest, its time
// is t + dt, its signal speed the one the update kernel reduced, and the
// schedule log gets (P, t, dt).  Cell counts are summed into the counters;
// the other counters move in part 3, after every entry is written.
__global__ void __launch_bounds__(EVAL_NT) plan_publish_kernel(DevCtx c) {
  const int nprev = c.ctl[CTL_NREADY];
  const long long s0 = c.cnt[CNT_NSCHED];
  const int ns = c.ns;
  __shared__ unsigned long long s_cells;
  if (threadIdx.x == 0) s_cells = 0;
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nprev) {
    const int P = c.R[r];
    atomicAdd(&s_cells, (unsigned long long)c.geo[P].n[0] * c.geo[P].n[1] * c.geo[P].n[2]);
    const double dt = c.dtR[r];
    const int L = c.latest[P], Ln = (L + 1) % ns;
    const double t = c.t_slot[(long long)P * ns + L];
    c.t_slot[(long long)P * ns + Ln] = t + dt;
    c.smax_slot[(long long)P * ns + Ln] = __longlong_as_double((long long)c.smax_new[P]);
    c.latest[P] = Ln;
    c.dt_last[P] = dt;
    const long long e = s0 + r;
    if (e < c.sched_cap) {
      c.sched[e].patch = P;
      c.sched[e].t_start = t;
      c.sched[e].dt = dt;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_cells) atomicAdd((unsigned long long *)&c.cnt[CNT_CELL_UPDATES], s_cells);
}

// Part 2 (one thread per patch): Eq. (1) and the local step of
// every ready patch; rflag/rdt per patch, and whether any patch is behind
// t_end.
__global__ void __launch_bounds__(EVAL_NT) plan_ready_kernel(DevCtx c, double t_end) {
  if (c.ctl[CTL_STATUS] != 0) return;
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= c.np) return;
  int flag = 0;
  double dtP = 0.0;
  const double t = c.t_slot[(long long)P * c.ns + c.latest[P]];
  if (t < t_end && (!c.owned || c.owned[P])) {
    c.ctl[CTL_NOTDONE] = 1;
    double tr;
    if (is_ready<false>(c, P, t_end, &tr)) {
      const int rc = patch_dt<false>(c, P, t, t_end, &dtP);
      if (rc != DSP_OK) set_status(c, rc, P);
      else flag = 1;
    }
  }
  c.rflag[P] = flag;
  c.rdt[P] = dtP;
}

// Block-wide exclusive scan of one flag per thread (ballot/popc per warp,
// then warp 0 over the warp sums): *pos = this thread's position among the
// flagged threads, returns their total.  Every thread of the block calls it.
__device__ __forceinline__ int block_scan_flag(int flag, int *s_wsum, int &s_total, int *pos) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) s_wsum[wid] = __popc(bal);
  __syncthreads();
  if (wid == 0) {
    const int v = s_wsum[lane];
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    s_wsum[lane] = incl - v;
    if (lane == 31) s_total = incl;
  }
  __syncthreads();
  *pos = s_wsum[wid] + __popc(bal & ((1u << lane) - 1u));
  const int total = s_total;
  __syncthreads();
  return total;
}

// Part 3 (one block): counters of the published sweep; the ready list R in
// patch order (publication and the schedule log follow it), the global step
// (smallest ready step) in global-step mode, the work list Rk -- the ready
// list's entries grouped by size class, each class's kernel taking its own
// stretch [ctl[CTL_CLS + k], ctl[CTL_CLS + k + 1]) -- with its work offsets,
// and done / deadlock.
__global__ void __launch_bounds__(PLAN_NT) plan_compact_kernel(DevCtx c, int global_mode, int publish_only) {
  __shared__ int s_wsum[PLAN_NT / 32];
  __shared__ int s_base, s_total;
  __shared__ unsigned long long s_dtmin;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    const int nprev = c.ctl[CTL_NREADY];
    if (nprev > 0) {
      c.cnt[CNT_NSCHED] += nprev;
      c.cnt[CNT_PATCH_UPDATES] += nprev;
      c.cnt[CNT_SWEEPS] += 1;
    }
    c.ctl[CTL_NREADY] = 0;
    for (int k = 0; k <= MAXCLS; k++) c.ctl[CTL_CLS + k] = 0;
    s_base = 0;
    s_dtmin = 0x7ff0000000000000ull;  // +inf
  }
  __syncthreads();
  const int notdone = c.ctl[CTL_NOTDONE];
  __syncthreads();
  if (tid == 0) c.ctl[CTL_NOTDONE] = 0;
  if (publish_only || c.ctl[CTL_STATUS] != 0) return;
  // the ready list in patch order; rflag[P] becomes P's index in it plus one
  for (int chunk = 0; chunk < c.np; chunk += PLAN_NT) {
    const int P = chunk + tid;
    const int flag = P < c.np ? c.rflag[P] : 0;
    int pos;
    const int total = block_scan_flag(flag, s_wsum, s_total, &pos);
    if (flag) {
      const double dtP = c.rdt[P];
      const int idx = s_base + pos;
      c.R[idx] = P;
      c.dtR[idx] = dtP;
      c.rflag[P] = idx + 1;
      c.smax_new[P] = 0ull;
      if (global_mode) atomicMin(&s_dtmin, (unsigned long long)__double_as_longlong(dtP));
    }
    if (tid == 0) s_base += total;
    __syncthreads();
  }
  const int nr = s_base;
  if (global_mode) {
    const double dtg = __longlong_as_double((long long)s_dtmin);
    for (int r = tid; r < nr; r += PLAN_NT) c.dtR[r] = dtg;
  }
  // the work list, grouped by size class
  __shared__ int s_kb;
  if (tid == 0) s_kb = 0;
  __syncthreads();
  for (int k = 0; k < c.ncls; k++) {
    if (tid == 0) c.ctl[CTL_CLS + k] = s_kb;
    for (int chunk = 0; chunk < c.np; chunk += PLAN_NT) {
      const int P = chunk + tid;
      const int ri = P < c.np ? c.rflag[P] : 0;
      const int flag = ri > 0 && c.geo[P].cls == k;
      int pos;
      const int total = block_scan_flag(flag, s_wsum, s_total, &pos);
      if (flag) c.Rk[s_kb + pos] = ri - 1;
      if (tid == 0) s_kb += total;
      __syncthreads();
    }
  }
  if (tid == 0) c.ctl[CTL_CLS + c.ncls] = s_kb;
  // work offsets: work-list entry i owns update work items [work_off[i], work_off[i+1])
  __shared__ int s_woff;
  if (tid == 0) s_woff = 0;
  __syncthreads();
  for (int chunk = 0; chunk < nr; chunk += PLAN_NT) {
    const int r = chunk + tid;
    const int v = r < nr ? c.geo[c.R[c.Rk[r]]].tiles : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) s_wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const int wv = s_wsum[lane];
      int wi = wv;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += u;
      }
      s_wsum[lane] = wi - wv;
      if (lane == 31) s_total = wi;
    }
    __syncthreads();
    if (r < nr) c.work_off[r] = s_woff + s_wsum[wid] + incl - v;
    __syncthreads();
    if (tid == 0) s_woff += s_total;
    __syncthreads();
  }
  if (tid == 0) c.work_off[nr] = s_woff;
  if (tid == 0) {
    if (c.ctl[CTL_STATUS] != 0) {
      c.ctl[CTL_NREADY] = 0;
      for (int k = 0; k <= MAXCLS; k++) c.ctl[CTL_CLS + k] = 0;
    } else {
      c.ctl[CTL_NREADY] = nr;
      if (nr == 0) {
        // in a context with virtual patches an empty sweep waits for the
        // packages of other processes; the caller detects a global deadlock
        if (!notdone) c.ctl[CTL_DONE] = 1;
        else if (!c.partial) set_status(c, DSP_ERR_DEADLOCK, -1);
      }
    }
  }
}

// Signal speed and positivity of slice s of every patch (one block per patch).
template <typename T>
__global__ void smax_kernel(DevCtx c, int slot, int first, int count) {
  const int P = first + blockIdx.x;
  if (P >= first + count) return;
  const PatchGeo &g = c.geo[P];
  const T *base = (const T *)c.slab + (long long)slot * c.slot_stride + g.off;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const long long nc = (long long)nx * ny * nz;
  const T *bxa = base + 5 * nc, *bya = bxa + (long long)(nx + 1) * ny * nz, *bza = bya + (long long)nx * (ny + 1) * nz;
  const T gamma = (T)c.gamma;
  double m = 0.0;
  for (long long id = threadIdx.x; id < nc; id += blockDim.x) {
    const int i = (int)(id % nx), j = (int)((id / nx) % ny), k = (int)(id / ((long long)nx * ny));
    T W[8];
    prim(base[id], base[nc + id], base[2 * nc + id], base[3 * nc + id], base[4 * nc + id],
         bxa[((long long)k * ny + j) * (nx + 1) + i], bxa[((long long)k * ny + j) * (nx + 1) + i + 1],
         bya[((long long)k * (ny + 1) + j) * nx + i], bya[((long long)k * (ny + 1) + j + 1) * nx + i],
         bza[((long long)k * ny + j) * nx + i], bza[((long long)(k + 1) * ny + j) * nx + i], gamma, W);
    if (!(W[RHO] > T(0)) || !(W[PR] > T(0))) set_status(c, DSP_ERR_UNPHYSICAL, P);
    T sig = signal_sum(W, gamma);
    if (c.eta > 0.0 || c.gad > 0.0)
      sig = tmax(sig, nonideal_speed(W, c.cfl, c.eta, c.gad, c.rhoi, c.cohm, c.cad, ldexp(c.dx, -g.level)));
    m = fmax(m, (double)sig);
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double u = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) u = fmax(u, __shfl_xor_sync(0xffffffffu, u, o));
    if (threadIdx.x == 0) c.smax_slot[(long long)P * c.ns + slot] = u;
  }
}

// Copy between the caller's four arrays (patches [first, first+count)) and
// the slices: dir 0 loads slot 0, dir 1 stores each patch's newest slot.
template <typename TS, typename TU>
__global__ void xfer_kernel(DevCtx c, int first, int count, TU *U, TU *bx, TU *by, TU *bz, int dir) {
  TU *arr[4] = {U, bx, by, bz};
  for (int P = first + blockIdx.x; P < first + count; P += gridDim.x) {
    const PatchGeo &g = c.geo[P];
    const long long nc = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long per[4] = {5 * nc, (long long)(g.n[0] + 1) * g.n[1] * g.n[2],
                              (long long)g.n[0] * (g.n[1] + 1) * g.n[2], (long long)g.n[0] * g.n[1] * (g.n[2] + 1)};
    const int s = dir == 0 ? 0 : c.latest[P];
    TS *slot = (TS *)c.slab + (long long)s * c.slot_stride + g.off;
    long long so = 0;
    for (int f = 0; f < 4; f++) {
      TU *a = arr[f] + (c.coff[f * (c.np + 1) + P] - c.coff[f * (c.np + 1) + first]);
      for (long long l = threadIdx.x; l < per[f]; l += blockDim.x) {
        if (dir == 0) slot[so + l] = (TS)a[l];
        else a[l] = (TU)slot[so + l];
      }
      so += per[f];
    }
  }
}

// Packages of several processes (Sec. 3 C): the newest slice of each listed
// patch -- its whole interior, U, bx, by, bz as laid out in a slice -- and
// its time parameters.  dir 0 (pack): newest slice -> buf + off[k], meta[k] =
// (time, last step, signal speed).  dir 1 (unpack): buf + off[k] -> the slot
// after the newest, which then becomes the newest with meta's time, step and
// signal speed.  One block per listed patch (the patches are distinct).
template <typename T>
__global__ void package_kernel(DevCtx c, const int *ids, const long long *off, int count, T *buf, double *meta,
                               int dir) {
  const int k = blockIdx.x;
  if (k >= count) return;
  const int P = ids[k];
  const PatchGeo &g = c.geo[P];
  const long long nc = (long long)g.n[0] * g.n[1] * g.n[2];
  const long long len = 5 * nc + (long long)(g.n[0] + 1) * g.n[1] * g.n[2] + (long long)g.n[0] * (g.n[1] + 1) * g.n[2] +
                        (long long)g.n[0] * g.n[1] * (g.n[2] + 1);
  const int L = c.latest[P];
  const int s = dir == 0 ? L : (L + 1) % c.ns;
  T *slot = (T *)c.slab + (long long)s * c.slot_stride + g.off;
  T *pkg = buf + off[k];
  for (long long l = threadIdx.x; l < len; l += blockDim.x) {
    if (dir == 0) pkg[l] = slot[l];
    else slot[l] = pkg[l];
  }
  if (threadIdx.x == 0) {
    const long long ts = (long long)P * c.ns;
    if (dir == 0) {
      meta[3 * k] = c.t_slot[ts + L];
      meta[3 * k + 1] = c.dt_last[P];
      meta[3 * k + 2] = c.smax_slot[ts + L];
    } else {
      c.t_slot[ts + s] = meta[3 * k];
      c.dt_last[P] = meta[3 * k + 1];
      c.smax_slot[ts + s] = meta[3 * k + 2];
      c.latest[P] = s;
    }
  }
}

__global__ void reset_times_kernel(DevCtx c, int first, int count, double t0) {
  for (int P = first + blockIdx.x * blockDim.x + threadIdx.x; P < first + count; P += gridDim.x * blockDim.x) {
    for (int s = 0; s < c.ns; s++) c.t_slot[(long long)P * c.ns + s] = s == 0 ? t0 : __longlong_as_double(0x7ff8000000000000ll);
    c.latest[P] = 0;
    c.dt_last[P] = 0.0;
  }
}

// Empties the ready queue's ring: slot s first takes ticket s.
__global__ void queue_ring_kernel(DevCtx c) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < c.q_cap; s += (long long)gridDim.x * blockDim.x) {
    c.q_free[s] = (unsigned long long)s;
    c.q_seq[s] = ~0ull;
  }
}

// Seeds the persistent ready queue from the ready list the plan kernel just
// built (the tiles of work-list entry r take tickets [work_off[r],
// work_off[r+1])), and resets the queue's control words (one block).
__global__ void queue_init_kernel(DevCtx c, double t_end) {
  const int nr = c.ctl[CTL_NREADY];
  for (int P = threadIdx.x; P < c.np; P += blockDim.x) {
    c.p_state[P] = 0;
    c.tiles_done[P] = 0;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nr; r += blockDim.x) {
    const int q = c.Rk[r], P = c.R[q];
    const int base = c.work_off[r], T = c.geo[P].tiles;
    for (int k = 0; k < T; k++) {
      c.q_patch[base + k] = P;
      c.q_tile[base + k] = k;
      c.q_dt[base + k] = c.dtR[q];
      c.q_seq[base + k] = (unsigned long long)(base + k);
    }
    c.p_state[P] = 1;
  }
  __shared__ int done;
  if (threadIdx.x == 0) done = 0;
  __syncthreads();
  for (int P = threadIdx.x; P < c.np; P += blockDim.x)
    if (!(c.t_slot[(long long)P * c.ns + c.latest[P]] < t_end)) atomicAdd(&done, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    c.q_ctl[0] = 0;
    c.q_ctl[1] = (unsigned long long)c.work_off[nr];
    c.q_ctl[2] = (unsigned long long)done;
    c.ctl[CTL_NREADY] = 0;
    if (nr == 0 && done < c.np) set_status(c, DSP_ERR_DEADLOCK, -1);
  }
}

// Per-patch diagnostics of the newest slice (dsp_diag.cuh): one block per
// patch, with the patch's own level's cell volume.
template <typename T>
__global__ void __launch_bounds__(DIAG_NT) diag_kernel(DevCtx c, double *out) {
  const int P = blockIdx.x;
  if (c.owned && !c.owned[P]) {  // a virtual patch: its owner counts it
    if (threadIdx.x < DIAG_PER) out[(long long)P * DIAG_PER + threadIdx.x] = 0.0;
    return;
  }
  const PatchGeo &g = c.geo[P];
  const T *base = (const T *)c.slab + (long long)c.latest[P] * c.slot_stride + g.off;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const long long nc = (long long)nx * ny * nz;
  const T *bxa = base + 5 * nc, *bya = bxa + (long long)(nx + 1) * ny * nz, *bza = bya + (long long)nx * (ny + 1) * nz;
  const double dxl = ldexp(c.dx, -g.level);
  diag_patch<T>(base, bxa, bya, bza, nx, ny, nz, dxl * dxl * dxl, out + (long long)P * DIAG_PER);
}

int launch_queue(dsp_ctx *c, double t_end) { return c->var->launch_queue(c->d, c->grid_update, t_end, c->stream); }

// The update kernels of a sweep: one launch per launch group (consecutive
// size classes with the same variant), over its stretch of the work list.
int launch_update(dsp_ctx *c) {
  for (int g = 0; g < c->ngrp; g++) {
    const int rc = c->var_cls[c->grp_lo[g]]->launch_update(c->d, c->grid_grp[g], c->stream, c->grp_lo[g], c->grp_hi[g]);
    if (rc) return rc;
  }
  return DSP_OK;
}

// Only class k's update kernel (the autotuner's timing runs).
int launch_update_class(dsp_ctx *c, int k) {
  return c->var_cls[k]->launch_update(c->d, c->grid_cls[k], c->stream, k, k + 1);
}

// Launch groups and grids from the classes' variants.
void make_groups(dsp_ctx *c) {
  c->ngrp = 0;
  for (int k = 0; k < c->ncls; k++) {
    if (c->ngrp > 0 && c->var_cls[c->grp_lo[c->ngrp - 1]] == c->var_cls[k]) {
      c->grp_hi[c->ngrp - 1] = k + 1;
    } else {
      c->grp_lo[c->ngrp] = k;
      c->grp_hi[c->ngrp] = k + 1;
      c->ngrp++;
    }
  }
  for (int k = 0; k < c->ncls; k++) c->grid_cls[k] = c->var_cls[k]->grid(c->d, k, k + 1);
  for (int g = 0; g < c->ngrp; g++) c->grid_grp[g] = c->var_cls[c->grp_lo[g]]->grid(c->d, c->grp_lo[g], c->grp_hi[g]);
}

// One dispatcher step: publish the previous sweep, then (unless
// publish_only) find the next ready list and its steps.
int launch_plan(dsp_ctx *c, double t_end, int global_mode, int publish_only) {
  const int np = c->d.np;
  plan_publish_kernel<<<(np + EVAL_NT - 1) / EVAL_NT, EVAL_NT, 0, c->stream>>>(c->d);
  if (!publish_only) plan_ready_kernel<<<(np + EVAL_NT - 1) / EVAL_NT, EVAL_NT, 0, c->stream>>>(c->d, t_end);
  plan_compact_kernel<<<1, PLAN_NT, 0, c->stream>>>(c->d, global_mode, publish_only);
  return cudaGetLastError() == cudaSuccess ? DSP_OK : DSP_ERR_CUDA;
}

// Cross-level guard values of the ready patches that have some (two levels
// only), after the plan kernel and before the update kernel of a sweep.
int launch_xlevel(dsp_ctx *c) {
  if (c->d.nlev < 2) return DSP_OK;
  const int grid = std::max(1, std::min(c->n_xlevel * XL_PARTS, 8192));
  if (c->precision == 1) xlevel_kernel<float><<<grid, 256, 0, c->stream>>>(c->d);
  else xlevel_kernel<double><<<grid, 256, 0, c->stream>>>(c->d);
  return cudaGetLastError() == cudaSuccess ? DSP_OK : DSP_ERR_CUDA;
}

#define DSP_VARIANT_ENTRY(id, T, TX, TY, NT, MB, PREC, RS, NI) variant_##id,
const KernelVariant *(*const kVariants[])() = {DSP_VARIANT_LIST(DSP_VARIANT_ENTRY)};
#undef DSP_VARIANT_ENTRY
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

// Per-patch tiles and offsets, each patch tiled by its class's tile shape
// tx[k] x ty[k] and z run tz[k]; false if some tile's owner table would not
// fit the kernel's table.
bool make_geometry(const std::vector<dsp_patch_desc> &patches, const std::vector<int> &cls, const int *tx,
                   const int *ty, const int *tz, const int bszl[2][3], std::vector<PatchGeo> &geo, long long &off,
                   long long &total_tiles, long long *cls_tiles) {
  const int npatch = (int)patches.size();
  geo.assign((size_t)npatch, PatchGeo());
  off = 0;
  total_tiles = 0;
  for (int k = 0; k < MAXCLS; k++) cls_tiles[k] = 0;
  auto fdiv = [](long long a, long long b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
  for (int i = 0; i < npatch; i++) {
    PatchGeo &g = geo[(size_t)i];
    const int k = cls[(size_t)i];
    const int TX = tx[k], TY = ty[k];
    for (int d = 0; d < 3; d++) {
      g.n[d] = patches[(size_t)i].n[d];
      g.lo[d] = (int)patches[(size_t)i].lo[d];
    }
    g.level = patches[(size_t)i].level;
    g.cls = k;
    g.tz = std::min(tz[k], g.n[2]);
    const int *bsz = bszl[g.level];
    g.nt[0] = (g.n[0] + TX - 1) / TX;
    g.nt[1] = (g.n[1] + TY - 1) / TY;
    g.nt[2] = (g.n[2] + g.tz - 1) / g.tz;
    g.tiles = g.nt[0] * g.nt[1] * g.nt[2];
    g.off = off;
    const long long nc = (long long)g.n[0] * g.n[1] * g.n[2];
    off += 5 * nc + (long long)(g.n[0] + 1) * g.n[1] * g.n[2] + (long long)g.n[0] * (g.n[1] + 1) * g.n[2] +
           (long long)g.n[0] * g.n[1] * (g.n[2] + 1);
    total_tiles += g.tiles;
    cls_tiles[k] += g.tiles;
    for (int kz = 0; kz < g.nt[2]; kz++)
      for (int ky = 0; ky < g.nt[1]; ky++)
        for (int kx = 0; kx < g.nt[0]; kx++) {
          const int org[3] = {kx * TX, ky * TY, kz * g.tz};
          const int ext[3] = {std::min(TX, g.n[0] - org[0]), std::min(TY, g.n[1] - org[1]),
                              std::min(g.tz, g.n[2] - org[2])};
          long long ne = 1;
          for (int d = 0; d < 3; d++)
            ne *= fdiv(g.lo[d] + org[d] + ext[d] + 2, bsz[d]) - fdiv(g.lo[d] + org[d] - 2, bsz[d]) + 1;
          if (ne > TABMAX) return false;
        }
  }
  return true;
}

// Install the context's per-class variants and z runs: geometry, device
// copy, grids.  False if some class's tiles do not fit.
bool install_tuning(dsp_ctx *c) {
  int tx[MAXCLS], ty[MAXCLS];
  for (int k = 0; k < MAXCLS; k++) {
    const KernelVariant *v = c->var_cls[k < c->ncls ? k : 0];
    tx[k] = v->tx;
    ty[k] = v->ty;
  }
  std::vector<PatchGeo> geo;
  long long off = 0, tt = 0;
  if (!make_geometry(c->patches, c->cls, tx, ty, c->tz_cls, c->d.bsz, geo, off, tt, c->d.cls_tiles)) return false;
  c->geo = geo;
  c->d.total_tiles = tt;
  c->var = c->var_cls[0];
  if (cudaMemcpyAsync(c->geo_d, geo.data(), sizeof(PatchGeo) * geo.size(), cudaMemcpyHostToDevice, c->stream) !=
      cudaSuccess)
    return false;
  make_groups(c);
  c->grid_update = c->var->grid(c->d, 0, 1);
  return true;
}

int read_status(dsp_ctx *c) {
  CK(cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(int) * CTL_COUNT, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DSP_OK;
}

int ensure_staging(dsp_ctx *c, size_t bytes) {
  if (c->staging_bytes >= bytes) return DSP_OK;
  if (c->staging) cudaFree(c->staging);
  c->staging = nullptr;
  c->staging_bytes = 0;
  if (cudaMalloc(&c->staging, bytes) != cudaSuccess) return fail(c, DSP_ERR_OOM, "staging buffer of %zu bytes", bytes);
  c->staging_bytes = bytes;
  return DSP_OK;
}

template <typename TS>
int run_xfer(dsp_ctx *c, int first, int count, void *U, void *bx, void *by, void *bz, int dtype, int dir) {
  const int grid = std::min(count, 4096);
  if (dtype == 0)
    xfer_kernel<TS, double><<<grid, 256, 0, c->stream>>>(c->d, first, count, (double *)U, (double *)bx, (double *)by,
                                                       (double *)bz, dir);
  else
    xfer_kernel<TS, float><<<grid, 256, 0, c->stream>>>(c->d, first, count, (float *)U, (float *)bx, (float *)by,
                                                      (float *)bz, dir);
  CK(cudaGetLastError());
  return DSP_OK;
}

int transfer(dsp_ctx *c, int first, int count, const void *U, const void *bx, const void *by, const void *bz, int dtype,
             int on_device, int dir) {
  const size_t es = dtype == 0 ? 8 : 4;
  const int np1 = c->d.np + 1;
  auto span = [&](int f) { return (size_t)(c->coff[f * np1 + first + count] - c->coff[f * np1 + first]); };
  const size_t nU = span(0), nX = span(1), nY = span(2), nZ = span(3);
  void *dU = (void *)U, *dX = (void *)bx, *dY = (void *)by, *dZ = (void *)bz;
  if (!on_device) {
    int rc = ensure_staging(c, es * (nU + nX + nY + nZ));
    if (rc) return rc;
    char *s = (char *)c->staging;
    dU = s;
    dX = s + es * nU;
    dY = s + es * (nU + nX);
    dZ = s + es * (nU + nX + nY);
    if (dir == 0) {
      CK(cudaMemcpyAsync(dU, U, es * nU, cudaMemcpyHostToDevice, c->stream));
      CK(cudaMemcpyAsync(dX, bx, es * nX, cudaMemcpyHostToDevice, c->stream));
      CK(cudaMemcpyAsync(dY, by, es * nY, cudaMemcpyHostToDevice, c->stream));
      CK(cudaMemcpyAsync(dZ, bz, es * nZ, cudaMemcpyHostToDevice, c->stream));
    }
  }
  int rc = c->precision != 1 ? run_xfer<double>(c, first, count, dU, dX, dY, dZ, dtype, dir)
                             : run_xfer<float>(c, first, count, dU, dX, dY, dZ, dtype, dir);
  if (rc) return rc;
  if (!on_device && dir == 1) {
    CK(cudaMemcpyAsync((void *)U, dU, es * nU, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync((void *)bx, dX, es * nX, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync((void *)by, dY, es * nY, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync((void *)bz, dZ, es * nZ, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return DSP_OK;
}

void free_all(dsp_ctx *c) {
  void *ptrs[] = {c->slab,    c->t_slot,  c->smax_slot, c->dt_last, c->dtR,     c->latest,  c->omap_d[0],
                  c->omap_d[1], c->gmap0_d, c->gofs_d, c->gbuf, c->rflag, c->rdt,
                  c->work_off_d, c->geo_d, c->coff_d,
                  c->nbl_off_d, c->nbl_d, c->R,       c->ctl,     c->smax_new, c->cnt,    c->sched,
                  c->staging, c->q_patch, c->q_tile, c->p_state, c->tiles_done, c->q_dt, c->q_seq,
                  c->q_free,  c->q_ctl, c->owned_d, c->pk_ids, c->pk_off, c->pk_meta, c->Rk};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" int dsp_create(const dsp_patch_desc *patches, int32_t npatch, const dsp_params *prm, void *stream,
                          dsp_ctx **out) {
  if (!out) return DSP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!patches || !prm || npatch <= 0) return DSP_ERR_INVALID_ARG;
  if (prm->dt_pow2 != 1) return DSP_ERR_UNSUPPORTED;
  // grace (Eq. 1) in [0, 1); with g > 0 only the sweep dispatcher (whose
  // result does not depend on the order of updates); time order 1 or 2
  // (0 = 1); quadratic extrapolation needs four slices; at most 16 slices
  if (!(prm->grace >= 0.0) || !(prm->grace < 1.0)) return DSP_ERR_INVALID_ARG;
  if (prm->grace > 0.0 && prm->dispatcher == 0) return DSP_ERR_UNSUPPORTED;
  if (prm->time_order < 0 || prm->time_order > 2 || prm->nslices > 16) return DSP_ERR_INVALID_ARG;
  if (prm->grace > 0.0 && prm->time_order == 2 && prm->nslices < 4) return DSP_ERR_INVALID_ARG;
  if (prm->dispatcher != 0 && prm->dispatcher != 1) return DSP_ERR_INVALID_ARG;
  if (prm->dispatcher == 0 && prm->time_mode != 1) return DSP_ERR_UNSUPPORTED;  // a global step needs sweeps
  if (prm->riemann != 0 && prm->riemann != 1) return DSP_ERR_INVALID_ARG;
  // non-ideal MHD: coefficients >= 0 (0 = off), an ion density with the
  // ambipolar term, Courant-like factors > 0 (0 = the paper's 0.1)
  if (!(prm->eta >= 0.0) || !(prm->gamma_ad >= 0.0) || !(prm->eta < INFINITY) || !(prm->gamma_ad < INFINITY) ||
      !(prm->c_ohm >= 0.0) || !(prm->c_ad >= 0.0) || (prm->gamma_ad > 0.0 && !(prm->rho_i > 0.0)))
    return DSP_ERR_INVALID_ARG;
  const int nonideal = prm->eta > 0.0 || prm->gamma_ad > 0.0;
  if (prm->nguard < 2 || prm->nslices < 3 || prm->precision < 0 || prm->precision > 2 ||
      (prm->time_mode != 0 && prm->time_mode != 1) || !(prm->cfl > 0.0) || !(prm->gamma > 1.0))
    return DSP_ERR_INVALID_ARG;
  for (int d = 0; d < 3; d++)
    if (prm->base_cells[d] <= 0 || !(prm->box_len[d] > 0.0)) return DSP_ERR_INVALID_ARG;
  const double dx = prm->box_len[0] / prm->base_cells[0];
  for (int d = 1; d < 3; d++)
    if (std::fabs(prm->box_len[d] / prm->base_cells[d] - dx) > 1e-12 * dx) return DSP_ERR_INVALID_ARG;
  // Geometry.  Level 0: patches wider than their guard depth that tile the
  // periodic box exactly.  Level 1 (optional, half the cell size): disjoint
  // patches inside the level-1 box, each covering whole level-0 cells (even
  // origin and size).  The map of level l cuts its box into blocks of
  // bsz[l] cells: the gcd of the box and every patch size and origin of that
  // level; level 0's is reduced further until every block is either wholly
  // covered by level 1 or not at all.
  auto gcd = [](long long a, long long b) {
    while (b) {
      const long long t = a % b;
      a = b;
      b = t;
    }
    return a;
  };
  int nlev = 1;
  long long Lv[2][3];
  int bsz[2][3];
  for (int d = 0; d < 3; d++) {
    Lv[0][d] = prm->base_cells[d];
    Lv[1][d] = 2ll * prm->base_cells[d];
    bsz[0][d] = prm->base_cells[d];
    bsz[1][d] = 2 * prm->base_cells[d];
  }
  for (int i = 0; i < npatch; i++) {
    const dsp_patch_desc &p = patches[i];
    if (p.level < 0 || p.level > 1) return DSP_ERR_UNSUPPORTED;
    if (p.level == 1) nlev = 2;
    for (int d = 0; d < 3; d++) {
      if (p.n[d] <= prm->nguard || p.lo[d] < 0 || p.lo[d] + p.n[d] > Lv[p.level][d]) return DSP_ERR_INVALID_ARG;
      if (p.level == 1 && ((p.n[d] & 1) || (p.lo[d] & 1))) return DSP_ERR_INVALID_ARG;
      bsz[p.level][d] = (int)gcd(bsz[p.level][d], gcd(p.n[d], p.lo[d]));
    }
  }
  for (int pass = 0; nlev == 2; pass++) {
    // level-1 cells over each level-0 block (level-1 patches are disjoint)
    int md[3];
    long long nb = 1;
    for (int d = 0; d < 3; d++) {
      md[d] = (int)(Lv[0][d] / bsz[0][d]);
      nb *= md[d];
    }
    if (nb > (1ll << 28)) return DSP_ERR_UNSUPPORTED;
    std::vector<long long> cov((size_t)nb, 0);
    for (int i = 0; i < npatch; i++) {
      const dsp_patch_desc &p = patches[i];
      if (p.level != 1) continue;
      long long a[3], b[3];
      for (int d = 0; d < 3; d++) {
        a[d] = p.lo[d] / 2;
        b[d] = (p.lo[d] + p.n[d]) / 2;
      }
      for (long long bz = a[2] / bsz[0][2]; bz <= (b[2] - 1) / bsz[0][2]; bz++)
        for (long long by = a[1] / bsz[0][1]; by <= (b[1] - 1) / bsz[0][1]; by++)
          for (long long bx = a[0] / bsz[0][0]; bx <= (b[0] - 1) / bsz[0][0]; bx++) {
            const long long bb[3] = {bx, by, bz};
            long long v = 1;
            for (int d = 0; d < 3; d++)
              v *= std::min(b[d], (bb[d] + 1) * bsz[0][d]) - std::max(a[d], bb[d] * bsz[0][d]);
            cov[(size_t)((bz * md[1] + by) * md[0] + bx)] += v;
          }
    }
    const long long full = (long long)bsz[0][0] * bsz[0][1] * bsz[0][2];
    bool partial = false;
    for (long long k = 0; k < nb && !partial; k++)
      if (cov[(size_t)k] != 0 && cov[(size_t)k] != full) partial = true;
    if (!partial) break;
    if (bsz[0][0] == 1 && bsz[0][1] == 1 && bsz[0][2] == 1) return DSP_ERR_INVALID_ARG;
    for (int d = 0; d < 3; d++) bsz[0][d] = bsz[0][d] % 2 == 0 ? bsz[0][d] / 2 : 1;
  }
  if (nlev == 2 && prm->dispatcher == 0) return DSP_ERR_UNSUPPORTED;  // the ready queue runs one level
  // several processes (Sec. 3 C): with virtual patches the layout is one
  // process's share -- its own patches and copies of their neighbours --,
  // advanced by local steps with g = 0 by sweeps, on one level
  int nvirt = 0;
  if (prm->owned)
    for (int i = 0; i < npatch; i++) nvirt += prm->owned[i] ? 0 : 1;
  const bool partial = nvirt > 0;
  if (partial && (nlev == 2 || prm->time_mode != 1 || prm->grace > 0.0 || prm->dispatcher != 1))
    return DSP_ERR_UNSUPPORTED;
  int mapd[2][3];
  long long nmap[2] = {1, 1};
  std::vector<int> omap[2], gmap0;
  for (int l = 0; l < nlev; l++) {
    for (int d = 0; d < 3; d++) {
      mapd[l][d] = (int)(Lv[l][d] / bsz[l][d]);
      // the kernels divide level coordinates by bsz through a float product
      if (Lv[l][d] + 8 > (1 << 20) / std::max(bsz[l][d], 1)) return DSP_ERR_UNSUPPORTED;
      nmap[l] *= mapd[l][d];
    }
    if (nmap[l] > (1ll << 28)) return DSP_ERR_UNSUPPORTED;
    omap[l].assign((size_t)nmap[l], -1);
  }
  for (int i = 0; i < npatch; i++) {
    const dsp_patch_desc &p = patches[i];
    const int l = p.level;
    const int *bs = bsz[l], *md = mapd[l];
    for (long long bz = p.lo[2] / bs[2]; bz < (p.lo[2] + p.n[2]) / bs[2]; bz++)
      for (long long by = p.lo[1] / bs[1]; by < (p.lo[1] + p.n[1]) / bs[1]; by++)
        for (long long bx = p.lo[0] / bs[0]; bx < (p.lo[0] + p.n[0]) / bs[0]; bx++) {
          int &m = omap[l][(size_t)((bz * md[1] + by) * md[0] + bx)];
          if (m >= 0) return DSP_ERR_INVALID_ARG;  // overlap
          m = i;
        }
  }
  if (!partial) {
    for (long long k = 0; k < nmap[0]; k++)
      if (omap[0][(size_t)k] < 0) return DSP_ERR_INVALID_ARG;  // level 0 is not a tiling
  } else {
    // a share need not tile the box, but every guard cell of an owned patch
    // must lie in a patch of the share
    const int g = prm->nguard;
    for (int i = 0; i < npatch; i++) {
      if (!prm->owned[i]) continue;
      const dsp_patch_desc &p = patches[i];
      long long b0[3], b1[3];
      for (int k = 0; k < 3; k++) {
        const long long a = p.lo[k] - g, b = p.lo[k] + p.n[k] + g;
        b0[k] = a >= 0 ? a / bsz[0][k] : -((-a + bsz[0][k] - 1) / bsz[0][k]);
        b1[k] = (b - 1) >= 0 ? (b - 1) / bsz[0][k] : -((-(b - 1) + bsz[0][k] - 1) / bsz[0][k]);
      }
      for (long long bz = b0[2]; bz <= b1[2]; bz++)
        for (long long by = b0[1]; by <= b1[1]; by++)
          for (long long bx = b0[0]; bx <= b1[0]; bx++) {
            const long long wx = ((bx % mapd[0][0]) + mapd[0][0]) % mapd[0][0];
            const long long wy = ((by % mapd[0][1]) + mapd[0][1]) % mapd[0][1];
            const long long wz = ((bz % mapd[0][2]) + mapd[0][2]) % mapd[0][2];
            if (omap[0][(size_t)((wz * mapd[0][1] + wy) * mapd[0][0] + wx)] < 0) return DSP_ERR_INVALID_ARG;
          }
    }
  }
  // the gather map of level 0: blocks covered by level 1 come from there
  gmap0 = omap[0];
  for (int i = 0; i < npatch; i++) {
    const dsp_patch_desc &p = patches[i];
    if (p.level != 1) continue;
    // every block a level-1 patch touches is wholly covered (see above)
    for (long long bz = p.lo[2] / 2 / bsz[0][2]; bz <= ((p.lo[2] + p.n[2]) / 2 - 1) / bsz[0][2]; bz++)
      for (long long by = p.lo[1] / 2 / bsz[0][1]; by <= ((p.lo[1] + p.n[1]) / 2 - 1) / bsz[0][1]; by++)
        for (long long bx = p.lo[0] / 2 / bsz[0][0]; bx <= ((p.lo[0] + p.n[0]) / 2 - 1) / bsz[0][0]; bx++)
          gmap0[(size_t)((bz * mapd[0][1] + by) * mapd[0][0] + bx)] = -1;
  }
  // the update-kernel variant: the requested one, else the first of this precision
  const KernelVariant *var = nullptr;
  for (int k = 0; k < kNumVariants; k++) {
    const KernelVariant *v = kVariants[k]();
    if (v->precision != prm->precision || v->riemann != prm->riemann || v->nonideal != nonideal) continue;
    if (prm->variant >= 0 ? v->id == prm->variant : !var) var = v;
  }
  if (!var) return DSP_ERR_INVALID_ARG;
  // size classes: one per distinct patch size (sweep dispatcher, at most
  // MAXCLS sizes), else one for all; each starts with the default variant
  // and a z run of its patches' whole height (or tile_z)
  std::vector<int> cls((size_t)npatch, 0);
  int ncls = 1, cls_n[MAXCLS][3] = {};
  {
    std::vector<std::array<int, 3>> sizes;
    for (int i = 0; i < npatch; i++) {
      const std::array<int, 3> s3 = {patches[i].n[0], patches[i].n[1], patches[i].n[2]};
      if (std::find(sizes.begin(), sizes.end(), s3) == sizes.end()) sizes.push_back(s3);
    }
    std::sort(sizes.begin(), sizes.end());
    if (prm->dispatcher == 1 && sizes.size() <= (size_t)MAXCLS) {
      ncls = (int)sizes.size();
      for (int i = 0; i < npatch; i++) {
        const std::array<int, 3> s3 = {patches[i].n[0], patches[i].n[1], patches[i].n[2]};
        cls[(size_t)i] = (int)(std::find(sizes.begin(), sizes.end(), s3) - sizes.begin());
      }
      for (int k = 0; k < ncls; k++)
        for (int d = 0; d < 3; d++) cls_n[k][d] = sizes[(size_t)k][(size_t)d];
    } else {
      for (int d = 0; d < 3; d++) cls_n[0][d] = sizes.back()[(size_t)d];
    }
  }
  int tzc[MAXCLS], txc[MAXCLS], tyc[MAXCLS];
  for (int k = 0; k < MAXCLS; k++) {
    txc[k] = var->tx;
    tyc[k] = var->ty;
    tzc[k] = 0;
  }
  for (int i = 0; i < npatch; i++) tzc[cls[(size_t)i]] = std::max(tzc[cls[(size_t)i]], patches[i].n[2]);
  if (prm->tile_z > 0)
    for (int k = 0; k < MAXCLS; k++) tzc[k] = prm->tile_z;
  std::vector<dsp_patch_desc> pvec(patches, patches + npatch);
  std::vector<PatchGeo> geo;
  long long off = 0, total_tiles = 0, cls_tiles[MAXCLS];
  if (!make_geometry(pvec, cls, txc, tyc, tzc, bsz, geo, off, total_tiles, cls_tiles))
    return DSP_ERR_UNSUPPORTED;
  dsp_ctx *c = new dsp_ctx();
  memset(&c->d, 0, sizeof c->d);
  c->prm = *prm;
  c->stream = (cudaStream_t)stream;
  if (!c->stream && prm->graph) {
    // the legacy default stream cannot be captured: use a blocking stream of
    // our own, which the legacy stream orders with the caller's work
    if (cudaStreamCreate(&c->stream) != cudaSuccess) {
      (void)cudaGetLastError();
      delete c;
      return DSP_ERR_CUDA;
    }
    c->own_stream = 1;
  }
  c->precision = prm->precision;
  c->esize = prm->precision == 1 ? 4 : 8;
  c->poisoned = 0;
  c->nev = 0;
  c->geo = geo;
  c->var = var;
  c->patches = pvec;
  c->n_xlevel = 0;
  c->cls = cls;
  c->ncls = ncls;
  for (int k = 0; k < MAXCLS; k++) {
    c->var_cls[k] = var;
    c->tz_cls[k] = tzc[k];
    for (int dd = 0; dd < 3; dd++) c->cls_n[k][dd] = cls_n[k][dd];
  }
  DevCtx &d = c->d;
  d.np = npatch;
  d.ns = prm->nslices;
  d.ncls = ncls;
  for (int k = 0; k < MAXCLS; k++) d.cls_tiles[k] = cls_tiles[k];
  d.total_tiles = total_tiles;
  d.slot_stride = off;
  d.nlev = nlev;
  for (int l = 0; l < 2; l++)
    for (int k = 0; k < 3; k++) {
      d.bsz[l][k] = bsz[l][k];
      d.mapd[l][k] = l < nlev ? mapd[l][k] : 1;
      d.L[l][k] = (int)Lv[l][k];
      d.binv[l][k] = 1.0f / (float)bsz[l][k];
    }
  d.gamma = prm->gamma;
  d.cfl = prm->cfl;
  d.dx = dx;
  d.dt_max = prm->dt_max;
  d.eta = prm->eta;
  d.gad = prm->gamma_ad;
  d.rhoi = prm->gamma_ad > 0.0 ? prm->rho_i : 1.0;
  d.cohm = prm->c_ohm > 0.0 ? prm->c_ohm : 0.1;
  d.cad = prm->c_ad > 0.0 ? prm->c_ad : 0.1;
  d.grace = prm->grace;
  d.torder = prm->time_order == 2 ? 2 : 1;
  // Neighbours (symmetric).  Same level: every patch owning a block of the
  // padded box (periodic images), the patch itself excluded.  Other level:
  // every patch owning a block of the cells this patch may read there -- a
  // level-1 patch reads the level-0 parents of its padded cells and one
  // more level-0 cell on each side (limited slopes); a level-0 patch reads
  // the level-1 children of its padded cells and of the cell above its top
  // guard face -- and every patch that may read this one.
  const int g = prm->nguard;
  auto fdivl = [](long long a, long long b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
  std::vector<std::vector<int>> nbs((size_t)npatch);
  {
    std::vector<int> seen((size_t)npatch, -1);
    for (int i = 0; i < npatch; i++) {
      const dsp_patch_desc &p = patches[i];
      for (int l = 0; l < nlev; l++) {
        long long a[3], b[3];  // half-open cell interval on level l
        for (int k = 0; k < 3; k++) {
          if (l == p.level) {
            a[k] = p.lo[k] - g;
            b[k] = p.lo[k] + p.n[k] + g;
          } else if (p.level == 1) {
            a[k] = fdivl(p.lo[k] - g, 2) - 1;
            b[k] = fdivl(p.lo[k] + p.n[k] + g - 1, 2) + 2;
          } else {
            a[k] = 2 * (p.lo[k] - g);
            b[k] = 2 * (p.lo[k] + p.n[k] + g) + 2;
          }
        }
        long long b0[3], b1[3];
        for (int k = 0; k < 3; k++) {
          b0[k] = fdivl(a[k], bsz[l][k]);
          b1[k] = fdivl(b[k] - 1, bsz[l][k]);
        }
        for (long long bz = b0[2]; bz <= b1[2]; bz++)
          for (long long by = b0[1]; by <= b1[1]; by++)
            for (long long bx = b0[0]; bx <= b1[0]; bx++) {
              const long long wx = ((bx % mapd[l][0]) + mapd[l][0]) % mapd[l][0];
              const long long wy = ((by % mapd[l][1]) + mapd[l][1]) % mapd[l][1];
              const long long wz = ((bz % mapd[l][2]) + mapd[l][2]) % mapd[l][2];
              const int q = omap[l][(size_t)((wz * mapd[l][1] + wy) * mapd[l][0] + wx)];
              if (q >= 0 && q != i && seen[(size_t)q] != i) {
                seen[(size_t)q] = i;
                nbs[(size_t)i].push_back(q);
              }
            }
      }
    }
    for (int i = 0; i < npatch; i++)
      for (int q : std::vector<int>(nbs[(size_t)i]))
        if (patches[q].level != patches[i].level) nbs[(size_t)q].push_back(i);
  }
  c->nbl_off.assign((size_t)npatch + 1, 0);
  for (int i = 0; i < npatch; i++) {
    std::vector<int> &u = nbs[(size_t)i];
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
    c->nbl_off[i + 1] = c->nbl_off[i] + (int)u.size();
    c->nbl.insert(c->nbl.end(), u.begin(), u.end());
  }
  // cross-level guard buffers: every patch whose radius-2 padded box (and
  // the cells above its top faces) meets a block its gather takes from the
  // other level
  std::vector<long long> gofs((size_t)npatch, -1);
  long long gtotal = 0;
  if (nlev == 2) {
    for (int i = 0; i < npatch; i++) {
      const dsp_patch_desc &p = patches[i];
      const int l = p.level;
      const std::vector<int> &gm = l == 0 ? gmap0 : omap[1];
      long long b0[3], b1[3];
      for (int k = 0; k < 3; k++) {
        b0[k] = fdivl(p.lo[k] - 2, bsz[l][k]);
        b1[k] = fdivl(p.lo[k] + p.n[k] + 2, bsz[l][k]);
      }
      bool need = false;
      for (long long bz = b0[2]; bz <= b1[2] && !need; bz++)
        for (long long by = b0[1]; by <= b1[1] && !need; by++)
          for (long long bx = b0[0]; bx <= b1[0] && !need; bx++) {
            const long long wx = ((bx % mapd[l][0]) + mapd[l][0]) % mapd[l][0];
            const long long wy = ((by % mapd[l][1]) + mapd[l][1]) % mapd[l][1];
            const long long wz = ((bz % mapd[l][2]) + mapd[l][2]) % mapd[l][2];
            if (gm[(size_t)((wz * mapd[l][1] + wy) * mapd[l][0] + wx)] < 0) need = true;
          }
      if (!need) continue;
      const long long m0 = p.n[0] + 4, m1 = p.n[1] + 4, m2 = p.n[2] + 4;
      gofs[(size_t)i] = gtotal;
      c->n_xlevel++;
      gtotal += 5 * m0 * m1 * m2 + (m0 + 1) * m1 * m2 + m0 * (m1 + 1) * m2 + m0 * m1 * (m2 + 1);
    }
  }
  // offsets of each patch in the caller's four arrays
  c->coff.assign(4 * ((size_t)npatch + 1), 0);
  for (int i = 0; i < npatch; i++) {
    const PatchGeo &gg = geo[(size_t)i];
    const long long nc = (long long)gg.n[0] * gg.n[1] * gg.n[2];
    const long long per[4] = {5 * nc, (long long)(gg.n[0] + 1) * gg.n[1] * gg.n[2],
                              (long long)gg.n[0] * (gg.n[1] + 1) * gg.n[2], (long long)gg.n[0] * gg.n[1] * (gg.n[2] + 1)};
    for (int f = 0; f < 4; f++) c->coff[(size_t)f * (npatch + 1) + i + 1] = c->coff[(size_t)f * (npatch + 1) + i] + per[f];
  }
  auto alloc = [&](void **p, size_t bytes) {
    if (cudaMalloc(p, bytes ? bytes : 1) != cudaSuccess) return false;
    return true;
  };
  const size_t slab_bytes = c->esize * (size_t)d.slot_stride * d.ns;
  const long long cap = prm->sched_capacity > 0 ? prm->sched_capacity : 0;
  bool ok = alloc(&c->slab, slab_bytes) && alloc((void **)&c->t_slot, sizeof(double) * npatch * d.ns) &&
            alloc((void **)&c->smax_slot, sizeof(double) * npatch * d.ns) &&
            alloc((void **)&c->dt_last, sizeof(double) * npatch) && alloc((void **)&c->dtR, sizeof(double) * npatch) &&
            alloc((void **)&c->latest, sizeof(int) * npatch) && alloc((void **)&c->omap_d[0], sizeof(int) * nmap[0]) &&
            (nlev < 2 || alloc((void **)&c->omap_d[1], sizeof(int) * nmap[1])) &&
            (nlev < 2 || alloc((void **)&c->gmap0_d, sizeof(int) * nmap[0])) &&
            alloc((void **)&c->gofs_d, sizeof(long long) * npatch) &&
            (gtotal == 0 || alloc(&c->gbuf, c->esize * (size_t)gtotal)) &&
            alloc((void **)&c->geo_d, sizeof(PatchGeo) * npatch) &&
            alloc((void **)&c->coff_d, sizeof(long long) * c->coff.size()) &&
            alloc((void **)&c->work_off_d, sizeof(int) * (npatch + 1)) &&
            alloc((void **)&c->nbl_off_d, sizeof(int) * (npatch + 1)) &&
            alloc((void **)&c->nbl_d, sizeof(int) * std::max<size_t>(1, c->nbl.size())) &&
            alloc((void **)&c->R, sizeof(int) * npatch) && alloc((void **)&c->Rk, sizeof(int) * npatch) &&
            alloc((void **)&c->ctl, sizeof(int) * CTL_COUNT) &&
            alloc((void **)&c->rflag, sizeof(int) * npatch) && alloc((void **)&c->rdt, sizeof(double) * npatch) &&
            alloc((void **)&c->smax_new, sizeof(unsigned long long) * npatch) &&
            alloc((void **)&c->cnt, sizeof(long long) * CNT_COUNT) &&
            alloc((void **)&c->sched, sizeof(dsp_sched_entry) * std::max<long long>(1, cap)) &&
            alloc((void **)&c->pk_ids, sizeof(int) * npatch) &&
            alloc((void **)&c->pk_off, sizeof(long long) * (npatch + 1)) &&
            alloc((void **)&c->pk_meta, sizeof(double) * 3 * npatch) &&
            (!prm->owned || alloc((void **)&c->owned_d, sizeof(int) * npatch));
  if (ok && prm->dispatcher == 0) {
    // the ring itself is sized by the tiling in force at each advance
    ok = alloc((void **)&c->q_ctl, sizeof(unsigned long long) * 4) && alloc((void **)&c->p_state, sizeof(int) * npatch) &&
         alloc((void **)&c->tiles_done, sizeof(int) * npatch);
  }
  if (ok && cudaMallocHost((void **)&c->h_ctl, sizeof(int) * CTL_COUNT) != cudaSuccess) ok = false;
  if (!ok) {
    (void)cudaGetLastError();
    free_all(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return DSP_ERR_OOM;
  }
  d.slab = c->slab;
  d.t_slot = c->t_slot;
  d.smax_slot = c->smax_slot;
  d.latest = c->latest;
  d.dt_last = c->dt_last;
  d.geo = c->geo_d;
  d.omap[0] = c->omap_d[0];
  d.omap[1] = nlev == 2 ? c->omap_d[1] : c->omap_d[0];
  d.gmap[0] = nlev == 2 ? c->gmap0_d : c->omap_d[0];
  d.gmap[1] = d.omap[1];
  d.gofs = c->gofs_d;
  d.gbuf = c->gbuf;
  d.gbuf_len = gtotal;
  d.coff = c->coff_d;
  d.work_off = c->work_off_d;
  d.nbl_off = c->nbl_off_d;
  d.nbl = c->nbl_d;
  d.R = c->R;
  d.Rk = c->Rk;
  d.rflag = c->rflag;
  d.rdt = c->rdt;
  d.dtR = c->dtR;
  d.smax_new = c->smax_new;
  d.ctl = c->ctl;
  d.cnt = c->cnt;
  d.sched = c->sched;
  d.sched_cap = cap;
  d.q_patch = c->q_patch;
  d.q_dt = c->q_dt;
  d.q_seq = c->q_seq;
  d.q_free = c->q_free;
  d.q_tile = c->q_tile;
  d.q_cap = 0;
  d.q_ctl = c->q_ctl;
  d.p_state = c->p_state;
  d.tiles_done = c->tiles_done;
  d.wait_budget = prm->wait_budget > 0 ? prm->wait_budget : 4000000000ll;  // ~2 s of SM clock
  c->owned.assign((size_t)npatch, 1);
  if (prm->owned)
    for (int i = 0; i < npatch; i++) c->owned[(size_t)i] = prm->owned[i] ? 1 : 0;
  d.owned = prm->owned ? c->owned_d : nullptr;
  d.partial = partial ? 1 : 0;
  c->prm.owned = nullptr;  // the caller's array is not kept
  cudaError_t e = cudaMemcpyAsync(c->omap_d[0], omap[0].data(), sizeof(int) * omap[0].size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && nlev == 2)
    e = cudaMemcpyAsync(c->omap_d[1], omap[1].data(), sizeof(int) * omap[1].size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && nlev == 2)
    e = cudaMemcpyAsync(c->gmap0_d, gmap0.data(), sizeof(int) * gmap0.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->gofs_d, gofs.data(), sizeof(long long) * gofs.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && prm->owned)
    e = cudaMemcpyAsync(c->owned_d, c->owned.data(), sizeof(int) * npatch, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && gtotal > 0) e = cudaMemsetAsync(c->gbuf, 0, c->esize * (size_t)gtotal, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->geo_d, geo.data(), sizeof(PatchGeo) * geo.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->coff_d, c->coff.data(), sizeof(long long) * c->coff.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->nbl_off_d, c->nbl_off.data(), sizeof(int) * c->nbl_off.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && !c->nbl.empty())
    e = cudaMemcpyAsync(c->nbl_d, c->nbl.data(), sizeof(int) * c->nbl.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->work_off_d, 0, sizeof(int) * (npatch + 1), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ctl, 0, sizeof(int) * CTL_COUNT, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->cnt, 0, sizeof(long long) * CNT_COUNT, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->slab, 0, slab_bytes, c->stream);
  if (e == cudaSuccess) {
    reset_times_kernel<<<(npatch + 255) / 256, 256, 0, c->stream>>>(d, 0, npatch, prm->t0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    free_all(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return DSP_ERR_CUDA;
  }
  c->grid_update = var->grid(d, 0, 1);
  make_groups(c);
  *out = c;
  return DSP_OK;
}

extern "C" int dsp_set_state(dsp_ctx *c, int32_t first, int32_t count, const void *U, const void *bx, const void *by,
                             const void *bz, int32_t dtype, int32_t on_device) {
  if (!c) return DSP_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, DSP_ERR_INVALID_ARG, "context is poisoned by an earlier error");
  if (first < 0 || count <= 0 || first + count > c->d.np || !U || !bx || !by || !bz || (dtype != 0 && dtype != 1))
    return fail(c, DSP_ERR_INVALID_ARG, "bad arguments to dsp_set_state");
  int rc = transfer(c, first, count, U, bx, by, bz, dtype, on_device, 0);
  if (rc) return rc;
  reset_times_kernel<<<(count + 255) / 256, 256, 0, c->stream>>>(c->d, first, count, c->prm.t0);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(c->ctl, 0, sizeof(int) * CTL_COUNT, c->stream));
  CK(cudaMemsetAsync(c->cnt, 0, sizeof(long long) * CNT_COUNT, c->stream));
  if (c->precision != 1) smax_kernel<double><<<count, 256, 0, c->stream>>>(c->d, 0, first, count);
  else smax_kernel<float><<<count, 256, 0, c->stream>>>(c->d, 0, first, count);
  CK(cudaGetLastError());
  rc = read_status(c);
  if (rc) return rc;
  if (c->h_ctl[CTL_STATUS] != 0)
    return fail(c, c->h_ctl[CTL_STATUS], "initial state has rho <= 0 or p <= 0 in patch %d", c->h_ctl[CTL_ERRP]);
  return DSP_OK;
}

// Persistent ready-queue dispatcher: one plan step seeds the queue with the
// patches ready now, then one persistent launch runs every update until all
// patches reach t_end; each finishing patch publishes its new slice and
// queues itself and any neighbour it made ready.
int advance_queue(dsp_ctx *c, double t_end, const long long *c0, dsp_stats *out) {
  if (!(t_end < INFINITY)) return fail(c, DSP_ERR_INVALID_ARG, "the ready-queue dispatcher needs a finite t_end");
  const bool timing = c->prm.timing != 0;
  if (timing && c->nev == 0) {
    for (int i = 0; i < 2; i++) CK(cudaEventCreate(&c->ev[i]));
    c->nev = 2;
  }
  // the ring: every queued patch's tiles (each patch is queued at most once
  // at a time) twice over, plus a ticket per block claimed ahead of a push
  const long long cap = 2 * c->d.total_tiles + 4096;
  if (cap > c->q_alloc) {
    CK(cudaStreamSynchronize(c->stream));
    void *old[] = {c->q_patch, c->q_tile, c->q_dt, c->q_seq, c->q_free};
    for (void *p : old)
      if (p) cudaFree(p);
    c->q_patch = c->q_tile = nullptr;
    c->q_dt = nullptr;
    c->q_seq = c->q_free = nullptr;
    c->q_alloc = 0;
    auto alloc = [](void **q, size_t bytes) { return cudaMalloc(q, bytes) == cudaSuccess; };
    if (!(alloc((void **)&c->q_patch, sizeof(int) * cap) && alloc((void **)&c->q_tile, sizeof(int) * cap) &&
          alloc((void **)&c->q_dt, sizeof(double) * cap) && alloc((void **)&c->q_seq, sizeof(unsigned long long) * cap) &&
          alloc((void **)&c->q_free, sizeof(unsigned long long) * cap)))
      return fail(c, DSP_ERR_OOM, "cannot allocate the ready queue's ring of %lld tiles", cap);
    c->q_alloc = cap;
    c->d.q_patch = c->q_patch;
    c->d.q_tile = c->q_tile;
    c->d.q_dt = c->q_dt;
    c->d.q_seq = c->q_seq;
    c->d.q_free = c->q_free;
  }
  c->d.q_cap = cap;
  if (launch_plan(c, t_end, 0, 0)) return fail(c, DSP_ERR_CUDA, "dispatcher kernel launch failed");
  queue_ring_kernel<<<(int)std::min<long long>((cap + 255) / 256, 1024), 256, 0, c->stream>>>(c->d);
  queue_init_kernel<<<1, 1024, 0, c->stream>>>(c->d, t_end);
  CK(cudaGetLastError());
  if (timing) CK(cudaEventRecord(c->ev[0], c->stream));
  int rc = launch_queue(c, t_end);
  if (rc) return fail(c, rc, "queue kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  if (timing) CK(cudaEventRecord(c->ev[1], c->stream));
  rc = read_status(c);
  if (rc) return rc;
  float ms = 0.f;
  if (timing) CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
  long long c1[CNT_COUNT];
  CK(cudaMemcpyAsync(c1, c->cnt, sizeof c1, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const int st = c->h_ctl[CTL_STATUS];
  if (out) {
    out->patch_updates = c1[CNT_PATCH_UPDATES] - c0[CNT_PATCH_UPDATES];
    out->cell_updates = c1[CNT_CELL_UPDATES] - c0[CNT_CELL_UPDATES];
    out->sweeps = 0;
    out->fallbacks = c1[CNT_FALLBACKS] - c0[CNT_FALLBACKS];
    out->floors = c1[CNT_FLOORS] - c0[CNT_FLOORS];
    out->status = st;
    out->kernel_ms = timing ? ms : 0.0;
    out->kernel_launches = 1;
    out->plan_launches = 4;  // the three dispatcher kernels and the queue set-up
    std::vector<double> t((size_t)c->d.np);
    if (dsp_get_times(c, t.data(), nullptr) == DSP_OK) {
      out->t_min = *std::min_element(t.begin(), t.end());
      out->t_max = *std::max_element(t.begin(), t.end());
    }
  }
  if (st != 0) {
    const char *what = st == DSP_ERR_UNPHYSICAL ? "rho <= 0 or p <= 0 in a new state"
                       : st == DSP_ERR_TIMEOUT   ? "a ready-queue wait ran out of its budget"
                       : st == DSP_ERR_DEADLOCK  ? "no patch is ready but some are behind t_end"
                       : st == DSP_ERR_BRACKET   ? "neighbour slices do not bracket a guard-zone time"
                       : st == DSP_ERR_BOUNDS    ? "a global address outside every buffer (bounds-checked build)"
                                                 : "device error";
    return fail(c, st, "%s (patch %d, cell %d)", what, c->h_ctl[CTL_ERRP], c->h_ctl[CTL_ERRC]);
  }
  return DSP_OK;
}

extern "C" int dsp_advance(dsp_ctx *c, double t_end, int64_t max_sweeps, dsp_stats *out) {
  if (!c) return DSP_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, DSP_ERR_INVALID_ARG, "context is poisoned by an earlier error");
  if (std::isnan(t_end) || (!(t_end < INFINITY) && max_sweeps <= 0))
    return fail(c, DSP_ERR_INVALID_ARG, "an unbounded advance needs a finite t_end or a sweep limit");
  long long c0[CNT_COUNT];
  CK(cudaMemcpyAsync(c0, c->cnt, sizeof c0, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemsetAsync(c->ctl + CTL_DONE, 0, sizeof(int), c->stream));
  const int global_mode = c->prm.time_mode == 0;
  if (c->prm.dispatcher == 0) return advance_queue(c, t_end, c0, out);
  const int batch = 32;
  long long done_sweeps = 0, plans = 0, kl = 0;
  double kms = 0.0;
  int rc = DSP_OK;
  const bool timing = c->prm.timing != 0;
  if (timing && c->nev == 0) {
    for (int i = 0; i < 2 * batch; i++) CK(cudaEventCreate(&c->ev[i]));
    c->nev = 2 * batch;
  }
  // one batch of sweeps: plan + update kernels, optionally replayed from a
  // CUDA graph captured once per (t_end, timing) setting
  // per-launch events are recorded only outside graphs; a replayed graph is
  // timed as a whole (its plan kernels are a few microseconds each)
  auto issue_batch = [&](long long nb, bool events) -> int {
    for (long long s = 0; s < nb; s++) {
      if (launch_plan(c, t_end, global_mode, 0)) return fail(c, DSP_ERR_CUDA, "dispatcher kernel launch failed");
      if (launch_xlevel(c)) return fail(c, DSP_ERR_CUDA, "cross-level guard kernel launch failed");
      if (events) CK(cudaEventRecord(c->ev[2 * s], c->stream));
      const int r2 = launch_update(c);
      if (r2) return fail(c, r2, "update kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
      if (events) CK(cudaEventRecord(c->ev[2 * s + 1], c->stream));
    }
    return DSP_OK;
  };
  for (;;) {
    long long nb = batch;
    if (max_sweeps > 0) nb = std::min<long long>(nb, max_sweeps - done_sweeps);
    if (c->prm.graph && nb == batch) {
      if (c->graph_exec && (c->graph_t_end != t_end || c->graph_timing != (int)timing)) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
      }
      if (!c->graph_exec) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        const int r1 = issue_batch(nb, false);
        cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
        if (r1) return r1;
        if (ee != cudaSuccess) return fail(c, DSP_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ee));
        ee = cudaGraphInstantiate(&c->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (ee != cudaSuccess) return fail(c, DSP_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ee));
        c->graph_t_end = t_end;
        c->graph_timing = (int)timing;
      }
      if (timing) CK(cudaEventRecord(c->ev[0], c->stream));
      CK(cudaGraphLaunch(c->graph_exec, c->stream));
      if (timing) CK(cudaEventRecord(c->ev[1], c->stream));
    } else {
      rc = issue_batch(nb, timing);
      if (rc) return rc;
    }
    const bool graphed = c->prm.graph && nb == batch;
    plans += nb * (c->d.nlev > 1 ? 4 : 3);  // publish, readiness, compaction (+ cross-level guards)
    done_sweeps += nb;
    rc = read_status(c);
    if (rc) return rc;
    if (timing && graphed) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
      kms += ms;
    } else if (timing) {
      for (long long s = 0; s < nb; s++) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev[2 * s], c->ev[2 * s + 1]));
        kms += ms;
      }
    }
    kl += nb;
    if (c->h_ctl[CTL_STATUS] != 0 || c->h_ctl[CTL_DONE]) break;
    if (max_sweeps > 0 && done_sweeps >= max_sweeps) break;
  }
  if (launch_plan(c, t_end, global_mode, 1)) return fail(c, DSP_ERR_CUDA, "dispatcher kernel launch failed");
  plans += 2;  // publish and compaction
  rc = read_status(c);
  if (rc) return rc;
  long long c1[CNT_COUNT];
  CK(cudaMemcpyAsync(c1, c->cnt, sizeof c1, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const int st = c->h_ctl[CTL_STATUS];
  if (out) {
    out->patch_updates = c1[CNT_PATCH_UPDATES] - c0[CNT_PATCH_UPDATES];
    out->cell_updates = c1[CNT_CELL_UPDATES] - c0[CNT_CELL_UPDATES];
    out->sweeps = c1[CNT_SWEEPS] - c0[CNT_SWEEPS];
    out->fallbacks = c1[CNT_FALLBACKS] - c0[CNT_FALLBACKS];
    out->floors = c1[CNT_FLOORS] - c0[CNT_FLOORS];
    out->status = st;
    out->kernel_ms = timing ? kms : 0.0;
    out->kernel_launches = kl;
    out->plan_launches = plans;
    std::vector<double> t((size_t)c->d.np);
    if (dsp_get_times(c, t.data(), nullptr) == DSP_OK) {
      out->t_min = *std::min_element(t.begin(), t.end());
      out->t_max = *std::max_element(t.begin(), t.end());
    } else {
      out->t_min = out->t_max = NAN;
    }
  }
  if (st != 0) {
    const char *what = st == DSP_ERR_UNPHYSICAL ? "rho <= 0 or p <= 0 in a new state"
                       : st == DSP_ERR_DEADLOCK  ? "no patch is ready but some are behind t_end"
                       : st == DSP_ERR_BRACKET   ? "neighbour slices do not bracket a guard-zone time"
                       : st == DSP_ERR_BOUNDS    ? "a global address outside every buffer (bounds-checked build)"
                                                 : "device error";
    return fail(c, st, "%s (patch %d, cell %d)", what, c->h_ctl[CTL_ERRP], c->h_ctl[CTL_ERRC]);
  }
  return DSP_OK;
}

extern "C" int dsp_get_state(dsp_ctx *c, int32_t first, int32_t count, void *U, void *bx, void *by, void *bz,
                             int32_t dtype, int32_t on_device) {
  if (!c) return DSP_ERR_INVALID_ARG;
  if (first < 0 || count <= 0 || first + count > c->d.np || !U || !bx || !by || !bz || (dtype != 0 && dtype != 1))
    return fail(c, DSP_ERR_INVALID_ARG, "bad arguments to dsp_get_state");
  return transfer(c, first, count, U, bx, by, bz, dtype, on_device, 1);
}

extern "C" int dsp_get_times(dsp_ctx *c, double *t, double *dt_last) {
  if (!c || !t) return DSP_ERR_INVALID_ARG;
  const int np = c->d.np, ns = c->d.ns;
  std::vector<double> ts((size_t)np * ns);
  std::vector<int> lat((size_t)np);
  CK(cudaMemcpyAsync(ts.data(), c->t_slot, sizeof(double) * ts.size(), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(lat.data(), c->latest, sizeof(int) * np, cudaMemcpyDeviceToHost, c->stream));
  if (dt_last) CK(cudaMemcpyAsync(dt_last, c->dt_last, sizeof(double) * np, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < np; i++) t[i] = ts[(size_t)i * ns + lat[i]];
  return DSP_OK;
}

extern "C" int dsp_get_schedule(dsp_ctx *c, dsp_sched_entry *buf, int64_t cap, int64_t *n) {
  if (!c || !n) return DSP_ERR_INVALID_ARG;
  long long cnt[CNT_COUNT];
  CK(cudaMemcpyAsync(cnt, c->cnt, sizeof cnt, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const long long total = cnt[CNT_NSCHED];
  *n = total;
  const long long have = std::min<long long>(total, c->d.sched_cap);
  const long long k = std::min<long long>(have, cap);
  if (buf && k > 0) {
    CK(cudaMemcpyAsync(buf, c->sched, sizeof(dsp_sched_entry) * k, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  if (total > c->d.sched_cap) return fail(c, DSP_ERR_SCHEDULE_OVERFLOW, "schedule log holds %lld of %lld entries", (long long)c->d.sched_cap, total);
  return DSP_OK;
}

extern "C" int dsp_diagnostics(dsp_ctx *c, dsp_diag *out) {
  if (!c || !out) return DSP_ERR_INVALID_ARG;
  const int np = c->d.np;
  double *dd = nullptr;
  CK(cudaMalloc(&dd, sizeof(double) * DIAG_PER * np));
  if (c->precision != 1) diag_kernel<double><<<np, DIAG_NT, 0, c->stream>>>(c->d, dd);
  else diag_kernel<float><<<np, DIAG_NT, 0, c->stream>>>(c->d, dd);
  cudaError_t e = cudaGetLastError();
  std::vector<double> h((size_t)DIAG_PER * np);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), dd, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(dd);
  if (e != cudaSuccess) return fail(c, DSP_ERR_CUDA, "diagnostics: %s", cudaGetErrorString(e));
  double r[DIAG_PER];
  diag_combine(h.data(), np, r);
  out->mass = r[0];
  for (int d = 0; d < 3; d++) out->mom[d] = r[1 + d];
  out->energy = r[4];
  for (int d = 0; d < 3; d++) out->bmean[d] = r[5 + d];
  out->max_divb = r[8];
  out->max_b = r[9];
  return DSP_OK;
}

namespace {
struct SaveHeader {
  char magic[8];
  int32_t version, np, ns, precision;
  int64_t patch_len, slot_stride;
};
}  // namespace

extern "C" int dsp_save(dsp_ctx *c, void *buf, size_t cap, size_t *used) {
  if (!c || !used) return DSP_ERR_INVALID_ARG;
  const int np = c->d.np, ns = c->d.ns;
  const size_t slab = c->esize * (size_t)c->d.slot_stride * ns;
  const size_t need = sizeof(SaveHeader) + sizeof(double) * 2 * np * ns + sizeof(int) * np + sizeof(double) * np + slab;
  *used = need;
  if (!buf) return DSP_OK;
  if (cap < need) return fail(c, DSP_ERR_INVALID_ARG, "save buffer too small (%zu < %zu)", cap, need);
  char *p = (char *)buf;
  SaveHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, "DSPSAVE", 8);
  h.version = 1;
  h.np = np;
  h.ns = ns;
  h.precision = c->precision;
  h.patch_len = 0;
  h.slot_stride = c->d.slot_stride;
  memcpy(p, &h, sizeof h);
  p += sizeof h;
  CK(cudaMemcpyAsync(p, c->t_slot, sizeof(double) * np * ns, cudaMemcpyDeviceToHost, c->stream));
  p += sizeof(double) * np * ns;
  CK(cudaMemcpyAsync(p, c->smax_slot, sizeof(double) * np * ns, cudaMemcpyDeviceToHost, c->stream));
  p += sizeof(double) * np * ns;
  CK(cudaMemcpyAsync(p, c->latest, sizeof(int) * np, cudaMemcpyDeviceToHost, c->stream));
  p += sizeof(int) * np;
  CK(cudaMemcpyAsync(p, c->dt_last, sizeof(double) * np, cudaMemcpyDeviceToHost, c->stream));
  p += sizeof(double) * np;
  CK(cudaMemcpyAsync(p, c->slab, slab, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DSP_OK;
}

extern "C" int dsp_load(dsp_ctx *c, const void *buf, size_t size) {
  if (!c || !buf) return DSP_ERR_INVALID_ARG;
  const int np = c->d.np, ns = c->d.ns;
  const size_t slab = c->esize * (size_t)c->d.slot_stride * ns;
  const size_t need = sizeof(SaveHeader) + sizeof(double) * 2 * np * ns + sizeof(int) * np + sizeof(double) * np + slab;
  if (size < need) return fail(c, DSP_ERR_INVALID_ARG, "saved state too small");
  SaveHeader h;
  memcpy(&h, buf, sizeof h);
  if (memcmp(h.magic, "DSPSAVE", 8) || h.version != 1 || h.np != np || h.ns != ns || h.precision != c->precision ||
      h.slot_stride != c->d.slot_stride)
    return fail(c, DSP_ERR_INVALID_ARG, "saved state does not match this context");
  const char *p = (const char *)buf + sizeof h;
  CK(cudaMemcpyAsync(c->t_slot, p, sizeof(double) * np * ns, cudaMemcpyHostToDevice, c->stream));
  p += sizeof(double) * np * ns;
  CK(cudaMemcpyAsync(c->smax_slot, p, sizeof(double) * np * ns, cudaMemcpyHostToDevice, c->stream));
  p += sizeof(double) * np * ns;
  CK(cudaMemcpyAsync(c->latest, p, sizeof(int) * np, cudaMemcpyHostToDevice, c->stream));
  p += sizeof(int) * np;
  CK(cudaMemcpyAsync(c->dt_last, p, sizeof(double) * np, cudaMemcpyHostToDevice, c->stream));
  p += sizeof(double) * np;
  CK(cudaMemcpyAsync(c->slab, p, slab, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(c->ctl, 0, sizeof(int) * CTL_COUNT, c->stream));
  CK(cudaMemsetAsync(c->cnt, 0, sizeof(long long) * CNT_COUNT, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->poisoned = 0;
  c->err.clear();
  return DSP_OK;
}

extern "C" int dsp_autotune(dsp_ctx *c, int32_t reps, int32_t *chosen, double *ms, int32_t *ids, int32_t cap,
                            int32_t *n) {
  if (!c || reps < 1) return DSP_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, DSP_ERR_INVALID_ARG, "context is poisoned by an earlier error");
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const KernelVariant *orig_var[MAXCLS];
  int orig_tz[MAXCLS];
  for (int k = 0; k < MAXCLS; k++) {
    orig_var[k] = c->var_cls[k];
    orig_tz[k] = c->tz_cls[k];
  }
  int rc = DSP_OK, count = 0;
  const int nonideal = c->var->nonideal;
  // one class at a time: every fitting (variant, z run) pair, the others
  // classes keeping their current choice
  for (int k = 0; k < c->ncls && rc == DSP_OK; k++) {
    const KernelVariant *best = nullptr;
    int best_tz = 0;
    double best_ms = 0.0;
    const int nz = c->cls_n[k][2];
    // z runs: the patches' whole height and half of it, or the caller's
    const int tzs[2] = {c->prm.tile_z > 0 ? c->prm.tile_z : nz, c->prm.tile_z > 0 ? 0 : nz / 2};
    for (int vi = 0; vi < kNumVariants && rc == DSP_OK; vi++) {
      const KernelVariant *v = kVariants[vi]();
      if (v->precision != c->precision || v->riemann != c->prm.riemann || v->nonideal != nonideal) continue;
      for (int ti = 0; ti < 2 && rc == DSP_OK; ti++) {
        const int tz = tzs[ti];
        if (tz < 4 || (ti == 1 && tz == tzs[0])) continue;
        c->var_cls[k] = v;
        c->tz_cls[k] = tz;
        if (!install_tuning(c)) continue;  // tiles do not fit this variant's tables
        // plan the next sweep (nothing is published: the ready list is
        // dropped afterwards, and the update kernel only writes the patches'
        // next slot)
        CK(cudaMemsetAsync(c->ctl + CTL_NREADY, 0, sizeof(int), c->stream));
        if (launch_plan(c, INFINITY, c->prm.time_mode == 0, 0)) {
          rc = fail(c, DSP_ERR_CUDA, "dispatcher kernel launch failed");
          break;
        }
        rc = launch_xlevel(c);
        if (rc) break;
        rc = launch_update_class(c, k);
        if (rc) break;
        CK(cudaEventRecord(e0, c->stream));
        for (int r = 0; r < reps && rc == DSP_OK; r++) rc = launch_update_class(c, k);
        CK(cudaEventRecord(e1, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        const double per = t / reps;
        if (count < cap) {
          if (ms) ms[count] = per;
          if (ids) ids[count] = k * 1000000 + tz * 1000 + v->id;
        }
        count++;
        if (!best || per < best_ms) {
          best = v;
          best_tz = tz;
          best_ms = per;
        }
      }
    }
    if (rc == DSP_OK && !best) rc = fail(c, DSP_ERR_UNSUPPORTED, "no kernel variant fits size class %d", k);
    if (rc == DSP_OK) {
      c->var_cls[k] = best;
      c->tz_cls[k] = best_tz;
    }
  }
  CK(cudaMemsetAsync(c->ctl + CTL_NREADY, 0, sizeof(int), c->stream));
  for (int k = 0; k <= MAXCLS; k++) CK(cudaMemsetAsync(c->ctl + CTL_CLS + k, 0, sizeof(int), c->stream));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != DSP_OK) {
    for (int k = 0; k < MAXCLS; k++) {
      c->var_cls[k] = orig_var[k];
      c->tz_cls[k] = orig_tz[k];
    }
    install_tuning(c);
    return rc;
  }
  if (!install_tuning(c)) return fail(c, DSP_ERR_CUDA, "installing the tuned variants failed");
  CK(cudaStreamSynchronize(c->stream));
  if (c->graph_exec) {  // a captured batch holds the old launches
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  if (chosen) *chosen = c->var_cls[0]->id;
  if (n) *n = count;
  return DSP_OK;
}

extern "C" int dsp_get_tuning(dsp_ctx *c, int32_t cap, int32_t *ncls, int32_t *sizes, int32_t *variant,
                              int32_t *tile_z) {
  if (!c || !ncls) return DSP_ERR_INVALID_ARG;
  *ncls = c->ncls;
  for (int k = 0; k < c->ncls && k < cap; k++) {
    if (sizes)
      for (int d = 0; d < 3; d++) sizes[3 * k + d] = c->cls_n[k][d];
    if (variant) variant[k] = c->var_cls[k]->id;
    if (tile_z) tile_z[k] = c->tz_cls[k];
  }
  return DSP_OK;
}

namespace {
// Values of one patch's slice (and package).
long long patch_len(const PatchGeo &g) {
  const long long nc = (long long)g.n[0] * g.n[1] * g.n[2];
  return 5 * nc + (long long)(g.n[0] + 1) * g.n[1] * g.n[2] + (long long)g.n[0] * (g.n[1] + 1) * g.n[2] +
         (long long)g.n[0] * g.n[1] * (g.n[2] + 1);
}

// Validate a patch list and build its package offsets; virtual_only: every
// listed patch must be virtual.
int package_plan(dsp_ctx *c, const int32_t *ids, int32_t count, bool virtual_only, std::vector<long long> &off) {
  if (!ids || count < 0 || count > c->d.np) return fail(c, DSP_ERR_INVALID_ARG, "bad patch list");
  std::vector<char> seen((size_t)c->d.np, 0);
  off.assign((size_t)count + 1, 0);
  for (int k = 0; k < count; k++) {
    const int P = ids[k];
    if (P < 0 || P >= c->d.np || seen[(size_t)P]) return fail(c, DSP_ERR_INVALID_ARG, "patch list entry %d: %d", k, P);
    if (virtual_only && c->owned[(size_t)P]) return fail(c, DSP_ERR_INVALID_ARG, "patch %d is owned, not virtual", P);
    seen[(size_t)P] = 1;
    off[(size_t)k + 1] = off[(size_t)k] + patch_len(c->geo[(size_t)P]);
  }
  return DSP_OK;
}

int run_package(dsp_ctx *c, const int32_t *ids, int32_t count, void *buf, double *meta, int on_device, int dir) {
  std::vector<long long> off;
  int rc = package_plan(c, ids, count, dir == 1, off);
  if (rc) return rc;
  if (count == 0) return DSP_OK;
  const size_t bytes = c->esize * (size_t)off[(size_t)count];
  void *dbuf = buf;
  double *dmeta = meta;
  if (!on_device) {
    rc = ensure_staging(c, bytes);
    if (rc) return rc;
    dbuf = c->staging;
    dmeta = c->pk_meta;
  }
  CK(cudaMemcpyAsync(c->pk_ids, ids, sizeof(int) * count, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->pk_off, off.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice, c->stream));
  if (!on_device && dir == 1) {
    CK(cudaMemcpyAsync(dbuf, buf, bytes, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(dmeta, meta, sizeof(double) * 3 * count, cudaMemcpyHostToDevice, c->stream));
  }
  if (c->precision == 1)
    package_kernel<float><<<count, 256, 0, c->stream>>>(c->d, c->pk_ids, c->pk_off, count, (float *)dbuf, dmeta, dir);
  else
    package_kernel<double><<<count, 256, 0, c->stream>>>(c->d, c->pk_ids, c->pk_off, count, (double *)dbuf, dmeta, dir);
  CK(cudaGetLastError());
  if (!on_device && dir == 0) {
    CK(cudaMemcpyAsync(buf, dbuf, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(meta, dmeta, sizeof(double) * 3 * count, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return DSP_OK;
}
}  // namespace

extern "C" int dsp_package_len(dsp_ctx *c, const int32_t *ids, int32_t count, int64_t *values) {
  if (!c || !values) return DSP_ERR_INVALID_ARG;
  std::vector<long long> off;
  const int rc = package_plan(c, ids, count, false, off);
  if (rc) return rc;
  *values = off[(size_t)count];
  return DSP_OK;
}

extern "C" int dsp_pack(dsp_ctx *c, const int32_t *ids, int32_t count, void *buf, double *meta, int32_t on_device) {
  if (!c || !buf || !meta) return DSP_ERR_INVALID_ARG;
  return run_package(c, ids, count, buf, meta, on_device, 0);
}

extern "C" int dsp_unpack(dsp_ctx *c, const int32_t *ids, int32_t count, const void *buf, const double *meta,
                          int32_t on_device) {
  if (!c || !buf || !meta) return DSP_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, DSP_ERR_INVALID_ARG, "context is poisoned by an earlier error");
  return run_package(c, ids, count, const_cast<void *>(buf), const_cast<double *>(meta), on_device, 1);
}

extern "C" const char *dsp_last_error(dsp_ctx *c) { return c ? c->err.c_str() : "null context"; }

extern "C" void dsp_destroy(dsp_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  for (int i = 0; i < c->nev; i++) cudaEventDestroy(c->ev[i]);
  free_all(c);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

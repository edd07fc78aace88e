// dsp_update.cuh -- the fused per-patch update kernel.
//
// One work item is a tile of one ready patch: TX x TY columns of cells and a
// run of tz planes along z.  The block marches through the planes; for each
// plane it
//   A  takes the next plane of the padded tile (radius 2) from the patch's
//      own newest slice and its neighbours' slices, inter- or extrapolating
//      in time where a neighbour is not at the patch's time (DISPATCH I,
//      Sec. 3 A and B), and converts to
//      primitive variables (the plane's copies were started asynchronously
//      one plane earlier, so only the time blends remain to compute);
//   B  computes MC-limited slopes and the Hancock half-step predictor;
//   C  computes HLL (or HLLD) fluxes through the x- and y-faces of the
//      plane and the z-faces below it;
//   D  computes the upwind edge EMFs on the x- and y-edges below the plane and
//      the in-plane part of the flux divergence;
//   E  writes the conservative update of the plane below and the
//      constrained-transport update of its faces into the patch's next slice
//      (the oldest slice is overwritten, Sec. 3 A);
//   F  computes the z-edge EMFs of the plane, the signal speed of the freshly
//      written cells, and the values carried to the next plane.
// With the non-ideal terms (NI) phases D and F add the Ohmic and ambipolar
// EMFs to the edges, and the Poynting flux of those EMFs joins the energy
// flux before the update of the plane below (DISPATCH I, Sec. 4.3).
// Every intermediate lives in shared memory; HBM sees the gathered input and
// the written output only.  The arithmetic per cell, face and edge is the
// same sequence of operations as the oracle's, so the FP64 build (no FMA
// contraction) reproduces it bit for bit.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "dsp_dispatch.cuh"
#include "dsp_internal.h"
#include "dsp_physics.cuh"

namespace dsp {

template <int TX, int TY, int NI = 0>
struct Lay {
  static constexpr int H2N = (TX + 4) * (TY + 4);
  static constexpr int H1N = (TX + 2) * (TY + 2);
  static constexpr int FPN = (TX + 5) * (TY + 5);
  static constexpr int NFB = NI ? 3 : 2;       // face planes held (three for the non-ideal currents)
  static constexpr int oW = 0;                 // [3 planes][8][H2N] primitive ring
  static constexpr int oFB = oW + 24 * H2N;    // [NFB planes][4][FPN] faces: x-low, y-low, z-low, z-high
  static constexpr int oWS = oFB + NFB * 4 * FPN;  // [8][H1N] predicted state W*
  static constexpr int oDX = oWS + 8 * H1N;    // [8][H1N] slopes along x
  static constexpr int oDY = oDX + 8 * H1N;
  static constexpr int oDZ = oDY + 8 * H1N;
  static constexpr int oZP = oDZ + 8 * H1N;    // [8][H1N] upper z-face state of the previous plane
  static constexpr int oCX = oZP + 8 * H1N;    // [6][H1N] previous plane's +z corners for x-edges
  static constexpr int oCY = oCX + 6 * H1N;    // [6][H1N] previous plane's +z corners for y-edges
  static constexpr int oSX = oCY + 6 * H1N;    // [2 parity][2][H1N] x-face speeds
  static constexpr int oSY = oSX + 4 * H1N;    // [2 parity][2][H1N] y-face speeds
  static constexpr int oSZ = oSY + 4 * H1N;    // [2][H1N] z-face speeds
  static constexpr int oFX = oSZ + 2 * H1N;    // [5][H1N] x-face fluxes of the plane
  static constexpr int oFY = oFX + 5 * H1N;    // [5][H1N]
  static constexpr int oDU = oFY + 5 * H1N;    // [2 parity][5][H1N] in-plane flux divergence
  static constexpr int oFZ = oDU + 10 * H1N;   // [2 parity][5][H1N] z-face fluxes
  static constexpr int oEX = oFZ + 10 * H1N;   // [2 parity][H1N] x-edge EMFs
  static constexpr int oEY = oEX + 2 * H1N;    // [2 parity][H1N] y-edge EMFs
  static constexpr int oEZ = oEY + 2 * H1N;    // [H1N] z-edge EMFs of the previous plane
  static constexpr int oNBX = oEZ + H1N;       // [H1N] new x-faces of the updated plane
  static constexpr int oNBY = oNBX + H1N;      // [H1N] new y-faces
  static constexpr int oNBZ = oNBY + H1N;      // [2 parity][H1N] new z-faces
  // the old values phase E updates, copied in ahead of time: U of the tile's
  // cells, their x- and y-faces, the z-faces below them
  static constexpr int oOLD = oNBZ + 2 * H1N;
  static constexpr int OLDU = 0, OLDX = 5 * TX * TY, OLDY = OLDX + (TX + 1) * TY, OLDZ = OLDY + TX * (TY + 1);
  // non-ideal terms only: the non-ideal EMFs of the x- and y-edges (two
  // levels, by parity), of the z-edges of the previous plane, and the ideal
  // energy fluxes of the x- and y-faces of the last two planes (by parity)
  static constexpr int oENX = oOLD + OLDZ + TX * TY;
  static constexpr int oENY = oENX + (NI ? 2 * H1N : 0);
  static constexpr int oENZ = oENY + (NI ? 2 * H1N : 0);
  static constexpr int oFXE = oENZ + (NI ? H1N : 0);
  static constexpr int oFYE = oFXE + (NI ? 2 * H1N : 0);
  // and the edge currents: x- and y-edges of the level below each of two
  // planes, z-edges of two planes (rings by plane parity)
  static constexpr int oJX = oFYE + (NI ? 2 * H1N : 0);
  static constexpr int oJY = oJX + (NI ? 2 * H1N : 0);
  static constexpr int oJZ = oJY + (NI ? 2 * H1N : 0);
  static constexpr int total = oJZ + (NI ? 2 * H1N : 0);
};


// Asynchronous global-to-shared copies of single elements (cp.async, no
// registers held while in flight): one per gathered value, committed as a
// group per plane and waited for before the plane is used.
enum { GATHER_NOW = 0, GATHER_ISSUE = 1, GATHER_BLEND = 2 };
template <int M>
using GatherMode = std::integral_constant<int, M>;

template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void set_error(const DevCtx &c, int code, int P, long long cell) {
  if (atomicCAS(&c.ctl[CTL_STATUS], 0, code) == 0) {
    c.ctl[CTL_ERRP] = P;
    c.ctl[CTL_ERRC] = (int)cell;
  }
}

// Small per-block scratch shared by all tiles a block processes: the owner
// table of the work item's padded tile (one entry per map block it touches:
// the owning patch's slice(s) at the tile's time -- the first slice's
// address, the others as slot offsets from it packed in `blend` (0: a copy;
// else n | (dB + 16) << 2 | (dC + 16) << 8 for n = 2 or 3 slices) -- their
// weights, the periodic image of its first cell, its size), and reduction
// space.
template <typename T, int NT>
struct TileShared {
  const T *srcA[TABMAX];
  int blend[TABMAX];
  T wgt[3][TABMAX];
  int lo[3][TABMAX];
  int n[3][TABMAX];
  double red[NT / 32];
  int fallback;
  int floors;  // new cells whose pressure recovery took the floor
};

// An axis known at run time (int) or at compile time (AxisC<V>): bodies
// written once over `axis_value(d)` fold to constants in the second case.
template <int V>
struct AxisC {};
__device__ __forceinline__ int axis_value(int d) { return d; }
template <int V>
__device__ __forceinline__ int axis_value(AxisC<V>) { return V; }

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int posmod(int a, int b) { const int r = a % b; return r < 0 ? r + b : r; }

// Advance one tile of patch P by dt (all threads of the block take part).
// On return the tile's new cells, faces and signal speed are written.  CONC:
// other blocks publish patch times concurrently (ready-queue dispatcher).
// RS: Riemann solver of the face fluxes (0 HLL, 1 HLLD).  NI: add the
// non-ideal Ohmic and ambipolar EMFs (DISPATCH I, Sec. 4.3) and their
// Poynting flux; these variants gather each plane synchronously (no copies
// in flight) and hold three planes of faces.
template <typename T, int TX, int TY, int NT, bool CONC, int RS, int NI>
__device__ __forceinline__ void process_tile(const DevCtx &c, const int P, const double dt, const int tile, T *sm,
                                             TileShared<T, NT> &S) {
  static_assert(TX * TY <= NT, "one updated cell per thread");
  using L = Lay<TX, TY, NI>;
  // asynchronous copies of the next plane and of the old values (sweep
  // dispatcher, ideal MHD)
  constexpr bool ASYNC = !CONC && !NI;
  // phases C and D as pools of work items over the whole block (FP64), or
  // one loop per axis (FP32)
  constexpr bool POOL = sizeof(T) == 8;
  constexpr int H2N = L::H2N, H1N = L::H1N, FPN = L::FPN;
  T *const Wr = sm + L::oW;
  T *const FB = sm + L::oFB;
  T *const Sws = sm + L::oWS;
  T *const SdX = sm + L::oDX;
  T *const SdY = sm + L::oDY;
  T *const SdZ = sm + L::oDZ;
  T *const ZP = sm + L::oZP;
  T *const CX = sm + L::oCX;
  T *const CY = sm + L::oCY;
  T *const SX = sm + L::oSX;
  T *const SY = sm + L::oSY;
  T *const SZ = sm + L::oSZ;
  T *const FX = sm + L::oFX;
  T *const FY = sm + L::oFY;
  T *const DU = sm + L::oDU;
  T *const FZ = sm + L::oFZ;
  T *const EX = sm + L::oEX;
  T *const EY = sm + L::oEY;
  T *const EZ = sm + L::oEZ;
  T *const NBX = sm + L::oNBX;
  T *const NBY = sm + L::oNBY;
  T *const NBZ = sm + L::oNBZ;

  const T **srcA = S.srcA;
  double *red = S.red;
  int &s_fallback = S.fallback;

  const int tid = threadIdx.x;
  // threads renumbered from the first warp after the TX*TY that update the
  // tile's cells: pools of items that those warps need not take first
  const int rot = (tid + NT - TX * TY) % NT;
  const PatchGeo &gp = c.geo[P];
  const int nx = gp.n[0], ny = gp.n[1], nz = gp.n[2];
  const int lox = gp.lo[0], loy = gp.lo[1], loz = gp.lo[2];
  const long long nc = (long long)nx * ny * nz;
  const long long ofx = 5 * nc, ofy = ofx + (long long)(nx + 1) * ny * nz, ofz = ofy + (long long)nx * (ny + 1) * nz;
  const T gamma = (T)c.gamma;
  const T igm1 = (T)(1.0 / (c.gamma - 1.0));
  const T half = T(0.5);

#define H2(i, j) (((j) + 2) * (TX + 4) + ((i) + 2))
#define H1(i, j) (((j) + 1) * (TX + 2) + ((i) + 1))
#define F5(i, j) (((j) + 2) * (TX + 5) + ((i) + 2))

  const int lev = gp.level;
  const double dxl = ldexp(c.dx, -lev);
  const T hdt = (T)(0.5 * dt / dxl);
  const T dtdx = (T)(dt / dxl);
  const int tix = tile % gp.nt[0], tiy = (tile / gp.nt[0]) % gp.nt[1], tiz = tile / (gp.nt[0] * gp.nt[1]);
  const int x0 = tix * TX, y0 = tiy * TY, z0 = tiz * gp.tz;
  const int tx = min(TX, nx - x0), ty = min(TY, ny - y0), tz = min(gp.tz, nz - z0);
  const int Lp = newest<CONC>(c, P);
  const double tP = slot_time<CONC>(c, (long long)P * c.ns + Lp);
  const T *const own = (const T *)c.slab + (long long)Lp * c.slot_stride + gp.off;
  T *const dst = (T *)c.slab + (long long)((Lp + 1) % c.ns) * c.slot_stride + gp.off;

  // Owner table of the padded tile: every block of the level's map that
  // cells in [x0-2, x0+tx+2] x [y0-2, y0+ty+2] x [z0-2, z0+tz+2] fall in, with
  // the slices of its owning patch that supply time tP (pick_slices: a slice
  // at exactly tP is copied, else two or three are inter- or extrapolated in
  // time).  A block whose values
  // come from the other level points at the patch's cross-level guard
  // buffer, filled for time tP just before this update.
  const int *const gmap = c.gmap[lev];
  const int *const bsz = c.bsz[lev];
  const int *const mapd = c.mapd[lev];
  const float *const binv = c.binv[lev];
  const int bx0 = floordiv(lox + x0 - 2, bsz[0]), by0 = floordiv(loy + y0 - 2, bsz[1]),
            bz0 = floordiv(loz + z0 - 2, bsz[2]);
  const int nbx = floordiv(lox + x0 + tx + 2, bsz[0]) - bx0 + 1;
  const int nby = floordiv(loy + y0 + ty + 2, bsz[1]) - by0 + 1;
  const int nbz = floordiv(loz + z0 + tz + 2, bsz[2]) - bz0 + 1;
  int my_blend = 0;
  for (int e = tid; e < nbx * nby * nbz; e += NT) {
    const int bx = bx0 + e % nbx, by = by0 + (e / nbx) % nby, bz = bz0 + e / (nbx * nby);
    const int wx = posmod(bx, mapd[0]), wy = posmod(by, mapd[1]), wz = posmod(bz, mapd[2]);
    const int Q = gmap[((long long)wz * mapd[1] + wy) * mapd[0] + wx];
    if (Q < 0) {
      // the cross-level guard buffer: a patch of n+4 cells at lo-2, in P's
      // own (unwrapped) coordinates
      for (int d = 0; d < 3; d++) {
        S.lo[d][e] = gp.lo[d] - 2;
        S.n[d][e] = gp.n[d] + 4;
      }
      srcA[e] = (const T *)c.gbuf + c.gofs[P];
      S.blend[e] = 0;
      continue;
    }
    const PatchGeo &gq = c.geo[Q];
    S.lo[0][e] = gq.lo[0] + (bx - wx) * bsz[0];
    S.lo[1][e] = gq.lo[1] + (by - wy) * bsz[1];
    S.lo[2][e] = gq.lo[2] + (bz - wz) * bsz[2];
    S.n[0][e] = gq.n[0];
    S.n[1][e] = gq.n[1];
    S.n[2][e] = gq.n[2];
    const T *base = (const T *)c.slab + gq.off;
    SlicePick pk;
    if (pick_slices<CONC>(c, Q, tP, pk) != DSP_OK) {
      pk.n = 1;
      pk.s[0] = newest<CONC>(c, Q);
      set_error(c, DSP_ERR_BRACKET, P, -1);
    }
    srcA[e] = base + (long long)pk.s[0] * c.slot_stride;
    int bl = 0;
    if (pk.n >= 2) {
      bl = pk.n | ((pk.s[1] - pk.s[0] + 16) << 2) | ((pk.n == 3 ? pk.s[2] - pk.s[0] + 16 : 16) << 8);
      my_blend = 1;
    }
    S.blend[e] = bl;
#pragma unroll
    for (int q = 0; q < 3; q++) S.wgt[q][e] = q < pk.n ? (T)pk.w[q] : T(0);
  }
  if (tid == 0) {
    s_fallback = 0;
    S.floors = 0;
  }
  const int any_blend = __syncthreads_or(my_blend);

  // Where a gathered value lives: its address in the source slice (the
  // patch's own newest slice, a neighbour's slice, or the cross-level guard
  // buffer) and its owner-table entry (-1 on the patch's own interior).  An
  // entry with a second slice B blends A[idx] + w (B[idx] - A[idx]).
  struct Loc {
    const T *p;
    int e;
  };
  auto blended = [&](const Loc &l) -> bool { return l.e >= 0 && S.blend[l.e] != 0; };
  // Bounds-checked build: every global address of the update is tested
  // against the slab of slices and the cross-level guard buffers; an address
  // outside both records DSP_ERR_BOUNDS and the access is redirected to the
  // slab's first element (a load) or dropped (a store), so the run ends with
  // that status and nothing faults.
#ifdef DSP_BOUNDS_CHECK
  auto inside = [&](const T *q) -> bool {
    const T *s0 = (const T *)c.slab, *g0 = (const T *)c.gbuf;
    return (q >= s0 && q < s0 + c.slot_stride * c.ns) || (g0 && q >= g0 && q < g0 + c.gbuf_len);
  };
  auto src = [&](const T *q) -> const T * {
    if (inside(q)) return q;
    set_error(c, DSP_ERR_BOUNDS, P, -1);
    return (const T *)c.slab;
  };
  auto put_global = [&](T *q, T v) {
    const T *s0 = (const T *)c.slab;
    if ((const T *)q >= s0 && (const T *)q < s0 + c.slot_stride * c.ns) *q = v;
    else set_error(c, DSP_ERR_BOUNDS, P, -1);
  };
#else
  auto src = [&](const T *q) -> const T * { return q; };
  auto put_global = [&](T *q, T v) { *q = v; };
#endif
  auto fetch = [&](const Loc &l) -> T {
    T a = *src(l.p);
    if (l.e >= 0) {
      const int bl = S.blend[l.e];
      if (bl) {
        const T b = *src(l.p + (long long)(((bl >> 2) & 63) - 16) * c.slot_stride);
        if ((bl & 3) == 2) {
          a = a + S.wgt[0][l.e] * (b - a);
        } else {
          const T cc = *src(l.p + (long long)(((bl >> 8) & 63) - 16) * c.slot_stride);
          a = (S.wgt[0][l.e] * a + S.wgt[1][l.e] * b) + S.wgt[2][l.e] * cc;
        }
      }
    }
    return a;
  };
  // Table entry of the level cell (gx, gy, gz) of the padded tile (floor of
  // a small integer quotient through a rounded-up float product: exact for
  // level extents far below 2^20 cells).
  auto entry = [&](int gx, int gy, int gz) -> int {
    const int ex = __float2int_rd(((float)gx + 0.5f) * binv[0]) - bx0;
    const int ey = __float2int_rd(((float)gy + 0.5f) * binv[1]) - by0;
    const int ez = __float2int_rd(((float)gz + 0.5f) * binv[2]) - bz0;
    return (ez * nby + ey) * nbx + ex;
  };
  // Cell-centred component q of patch-local cell (x,y,z) (radius <= 2
  // outside the patch).
  auto cell_loc = [&](int x, int y, int z, long long q) -> Loc {
    if (x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz)
      return {own + q * nc + ((long long)z * ny + y) * nx + x, -1};
    const int gx = lox + x, gy = loy + y, gz = loz + z;
    const int e = entry(gx, gy, gz);
    const int mx = S.n[0][e], my = S.n[1][e], mz = S.n[2][e];
    const int lx = gx - S.lo[0][e], ly = gy - S.lo[1][e], lz = gz - S.lo[2][e];
    return {srcA[e] + q * ((long long)mx * my * mz) + ((long long)lz * my + ly) * mx + lx, e};
  };
  // Face below cell (x,y,z) along each axis: the patch's own face when it
  // lies on one of its interior cells, else the face of the patch that owns
  // cell (x,y,z).
  auto facex_loc = [&](int x, int y, int z) -> Loc {
    if (x >= 0 && x <= nx && y >= 0 && y < ny && z >= 0 && z < nz)
      return {own + ofx + ((long long)z * ny + y) * (nx + 1) + x, -1};
    const int gx = lox + x, gy = loy + y, gz = loz + z;
    const int e = entry(gx, gy, gz);
    const int mx = S.n[0][e], my = S.n[1][e], mz = S.n[2][e];
    const int lx = gx - S.lo[0][e], ly = gy - S.lo[1][e], lz = gz - S.lo[2][e];
    return {srcA[e] + 5 * ((long long)mx * my * mz) + ((long long)lz * my + ly) * (mx + 1) + lx, e};
  };
  auto facey_loc = [&](int x, int y, int z) -> Loc {
    if (x >= 0 && x < nx && y >= 0 && y <= ny && z >= 0 && z < nz)
      return {own + ofy + ((long long)z * (ny + 1) + y) * nx + x, -1};
    const int gx = lox + x, gy = loy + y, gz = loz + z;
    const int e = entry(gx, gy, gz);
    const int mx = S.n[0][e], my = S.n[1][e], mz = S.n[2][e];
    const int lx = gx - S.lo[0][e], ly = gy - S.lo[1][e], lz = gz - S.lo[2][e];
    const long long m = (long long)mx * my * mz;
    return {srcA[e] + 5 * m + (long long)(mx + 1) * my * mz + ((long long)lz * (my + 1) + ly) * mx + lx, e};
  };
  auto facez_loc = [&](int x, int y, int z) -> Loc {
    if (x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z <= nz)
      return {own + ofz + ((long long)z * ny + y) * nx + x, -1};
    const int gx = lox + x, gy = loy + y, gz = loz + z;
    const int e = entry(gx, gy, gz);
    const int mx = S.n[0][e], my = S.n[1][e], mz = S.n[2][e];
    const int lx = gx - S.lo[0][e], ly = gy - S.lo[1][e], lz = gz - S.lo[2][e];
    const long long m = (long long)mx * my * mz;
    return {srcA[e] + 5 * m + (long long)(mx + 1) * my * mz + (long long)mx * (my + 1) * mz +
                ((long long)lz * my + ly) * mx + lx,
            e};
  };

  // ---- A: gather plane q of the radius-2 padded tile: the raw conserved
  // values and the faces (x- and y-faces below each cell, both z-faces).
  // Mode GATHER_NOW loads every value; GATHER_ISSUE starts an asynchronous
  // copy (cp.async) of every value that is a plain copy and leaves the
  // blended ones; GATHER_BLEND computes only the blended ones (after the
  // copies have landed).
  // ring slot of plane q's faces: two planes, or three with non-ideal terms
  auto fslot = [&](int q) -> int { return NI ? (q - z0 + 3) % 3 : (q - z0 + 2) & 1; };
  auto gather_plane = [&](int q, auto mode) {
    constexpr int M = decltype(mode)::value;
    const int rs = (q - z0 + 3) % 3, fs = fslot(q);
    T *Wq = Wr + rs * 8 * H2N;
    T *Fq = FB + fs * 4 * FPN;
    auto put = [&](T *dst, const Loc &l) {
      if constexpr (M == GATHER_NOW) {
        *dst = fetch(l);
      } else if constexpr (M == GATHER_ISSUE) {
        if (!blended(l)) cp_async_elem(dst, src(l.p));
      } else {
        if (blended(l)) *dst = fetch(l);
      }
    };
    for (int ci = tid; ci < (TX + 5) * (TY + 5); ci += NT) {
      const int i = ci % (TX + 5) - 2, j = ci / (TX + 5) - 2;
      if (i > tx + 2 || j > ty + 2) continue;
      const int x = x0 + i, y = y0 + j;
      const int f = F5(i, j);
      const bool inside = x >= 0 && x < nx && y >= 0 && y < ny && q >= 0 && q < nz;
      if (M == GATHER_BLEND && inside) continue;  // every value of this column is the patch's own
      if (j <= ty + 1) put(Fq + f, facex_loc(x, y, q));
      if (i <= tx + 1) put(Fq + FPN + f, facey_loc(x, y, q));
      if (i <= tx + 1 && j <= ty + 1) {
        put(Fq + 2 * FPN + f, facez_loc(x, y, q));
        put(Fq + 3 * FPN + f, facez_loc(x, y, q + 1));
        const int h = H2(i, j);
#pragma unroll
        for (int k = 0; k < 5; k++) put(Wq + k * H2N + h, cell_loc(x, y, q, k));
      }
    }
    if constexpr (M == GATHER_ISSUE) cp_async_commit();
  };
  // The face updates of phase E as one pool of items: the x-faces of plane
  // p-1 ([0, NBXF)), its y-faces, the z-faces at p-1/2.  eface gives an
  // item's face (i, j) and kind (0 x, 1 y, 2 z; -1 outside a partial tile);
  // the item's old value sits at OLD[OLDX + item].
  constexpr int NBXF = (TX + 1) * TY, NBYF = TX * (TY + 1), NBF = NBXF + NBYF + TX * TY;
  auto eface = [&](int e, int &i, int &j) -> int {
    if (e < NBXF) {
      i = e % (TX + 1);
      j = e / (TX + 1);
      return i <= tx && j < ty ? 0 : -1;
    }
    e -= NBXF;
    if (e < NBYF) {
      i = e % TX;
      j = e / TX;
      return i < tx && j <= ty ? 1 : -1;
    }
    e -= NBYF;
    i = e % TX;
    j = e / TX;
    return i < tx && j < ty ? 2 : -1;
  };
  // Visit the face-update items this thread owns, x- and y-faces if xy,
  // z-faces if zf: fn(item, kind, i, j), the kind an int in FP64's pool
  // (dealt from the first warp after the cell-updating ones) and an AxisC<>
  // constant in FP32's loops, one per kind from thread 0.
  auto each_eface = [&](bool xy, bool zf, auto fn) {
    if constexpr (POOL) {
      for (int e = rot; e < NBF; e += NT) {
        int i, j;
        const int kd = eface(e, i, j);
        if (kd < 0 || (kd < 2 ? !xy : !zf)) continue;
        fn(e, kd, i, j);
      }
    } else {
      if (xy) {
        for (int e = tid; e < NBXF; e += NT) {
          const int i = e % (TX + 1), j = e / (TX + 1);
          if (i <= tx && j < ty) fn(e, AxisC<0>{}, i, j);
        }
        for (int e = tid; e < NBYF; e += NT) {
          const int i = e % TX, j = e / TX;
          if (i < tx && j <= ty) fn(NBXF + e, AxisC<1>{}, i, j);
        }
      }
      if (zf) {
        for (int e = tid; e < TX * TY; e += NT) {
          const int i = e % TX, j = e / TX;
          if (i < tx && j < ty) fn(NBXF + NBYF + e, AxisC<2>{}, i, j);
        }
      }
    }
  };
  // Start the copies of the old values phase E reads in iteration `it`
  // (plane p-1's U and x-/y-faces once it >= 2, the z-faces at p-1/2 once
  // it >= 1); each thread copies exactly the values it will update.
  T *const OLD = sm + L::oOLD;
  auto prefetch_old = [&](int it, int p) {
    if (it >= 2) {
      for (int ci = tid; ci < TX * TY; ci += NT) {
        const int i = ci % TX, j = ci / TX;
        if (i >= tx || j >= ty) continue;
        const long long id = ((long long)(p - 1) * ny + (y0 + j)) * nx + (x0 + i);
#pragma unroll
        for (int k = 0; k < 5; k++) cp_async_elem(OLD + L::OLDU + k * TX * TY + ci, src(own + k * nc + id));
      }
    }
    if (it >= 1) {
      each_eface(it >= 2, true, [&](int e, auto kdd, int i, int j) {
        const int kd = axis_value(kdd);
        const T *g = kd == 0   ? own + ofx + ((long long)(p - 1) * ny + (y0 + j)) * (nx + 1) + (x0 + i)
                     : kd == 1 ? own + ofy + ((long long)(p - 1) * (ny + 1) + (y0 + j)) * nx + (x0 + i)
                               : own + ofz + ((long long)p * ny + (y0 + j)) * nx + (x0 + i);
        cp_async_elem(OLD + L::OLDX + e, src(g));
      });
    }
    cp_async_commit();
  };
  auto prim_plane = [&](int q) {
    const int rs = (q - z0 + 3) % 3, fs = fslot(q);
    T *Wq = Wr + rs * 8 * H2N;
    const T *Fq = FB + fs * 4 * FPN;
    for (int ci = tid; ci < (TX + 4) * (TY + 4); ci += NT) {
      const int i = ci % (TX + 4) - 2, j = ci / (TX + 4) - 2;
      if (i > tx + 1 || j > ty + 1) continue;
      const int h = H2(i, j), f = F5(i, j);
      T Wt[8];
      prim(Wq[h], Wq[H2N + h], Wq[2 * H2N + h], Wq[3 * H2N + h], Wq[4 * H2N + h], Fq[f], Fq[F5(i + 1, j)],
           Fq[FPN + f], Fq[FPN + F5(i, j + 1)], Fq[2 * FPN + f], Fq[3 * FPN + f], gamma, Wt);
#pragma unroll
      for (int k = 0; k < 8; k++) Wq[k * H2N + h] = Wt[k];
    }
  };

  gather_plane(z0 - 2, GatherMode<GATHER_NOW>{});
  gather_plane(z0 - 1, GatherMode<GATHER_NOW>{});
  __syncthreads();
  prim_plane(z0 - 2);
  prim_plane(z0 - 1);
  __syncthreads();

  // ---- Non-ideal MHD (Sec. 4.3), from the state at the start of the step,
  // in the FP64 oracle's operation order.  Currents live on the edges: J_e
  // at the edge on the low corner of cell (i,j,q) is the discrete curl of the
  // four faces around it over dx.  E_Ohm = eta J (Eq. 2); E_AD = (J B^2 -
  // B (B.J)) / (gamma_AD rho rho_i) = -v_D x B (Eqs. 5-6) with the edge's
  // two face-normal B components the means of the faces on the edge, B_e and
  // rho the means over the four cells around it, and the other two current
  // components the means of the four nearest edges of their own axes.
  const T idx = (T)(1.0 / dxl);
  const T eta_t = (T)c.eta, gad_t = (T)c.gad, rhoi_t = (T)c.rhoi;
  auto fpl = [&](int q) -> const T * { return FB + fslot(q) * 4 * FPN; };
  auto wpl = [&](int q) -> const T * { return Wr + ((q - z0 + 3) % 3) * 8 * H2N; };
  auto fxq = [&](int i, int j, int q) -> T { return fpl(q)[F5(i, j)]; };
  auto fyq = [&](int i, int j, int q) -> T { return fpl(q)[FPN + F5(i, j)]; };
  auto fzq = [&](int i, int j, int q) -> T { return fpl(q)[2 * FPN + F5(i, j)]; };
  auto wc = [&](int k, int i, int j, int q) -> T { return wpl(q)[k * H2N + H2(i, j)]; };
  // currents from faces (computed once per plane into rings, read by Jx/Jy/Jz)
  auto Jx_f = [&](int i, int j, int q) -> T { return ((fzq(i, j, q) - fzq(i, j - 1, q)) - (fyq(i, j, q) - fyq(i, j, q - 1))) * idx; };
  auto Jy_f = [&](int i, int j, int q) -> T { return ((fxq(i, j, q) - fxq(i, j, q - 1)) - (fzq(i, j, q) - fzq(i - 1, j, q))) * idx; };
  auto Jz_f = [&](int i, int j, int q) -> T { return ((fyq(i, j, q) - fyq(i - 1, j, q)) - (fxq(i, j, q) - fxq(i, j - 1, q))) * idx; };
  T *const JXr = sm + L::oJX;
  T *const JYr = sm + L::oJY;
  T *const JZr = sm + L::oJZ;
  auto jring = [&](int q) -> int { return ((q - z0 + 2) & 1) * H1N; };
  auto Jx = [&](int i, int j, int q) -> T { return JXr[jring(q) + H1(i, j)]; };
  auto Jy = [&](int i, int j, int q) -> T { return JYr[jring(q) + H1(i, j)]; };
  auto Jz = [&](int i, int j, int q) -> T { return JZr[jring(q) + H1(i, j)]; };
  // x- and y-edge currents of the level below plane q and z-edge currents of
  // plane q-1, over the H1 region (faces of planes q-1 and q)
  auto currents = [&](int q) {
    for (int ci = tid; ci < (TX + 2) * (TY + 2); ci += NT) {
      const int i = ci % (TX + 2) - 1, j = ci / (TX + 2) - 1, h = H1(i, j);
      if (i > tx || j > ty) continue;
      JXr[jring(q) + h] = Jx_f(i, j, q);
      JYr[jring(q) + h] = Jy_f(i, j, q);
      JZr[jring(q - 1) + h] = Jz_f(i, j, q - 1);
    }
  };
  auto ni_law = [&](T Je, T Ba, T Bb, T Be, T re, T Ja, T Jb) -> T {
    T en = T(0);
    if (c.eta > 0.0) en = eta_t * Je;
    if (c.gad > 0.0) {
      const T B2 = (Be * Be + Ba * Ba) + Bb * Bb;
      const T BJ = (Be * Je + Ba * Ja) + Bb * Jb;
      en = en + (Je * B2 - Be * BJ) / ((gad_t * re) * rhoi_t);
    }
    return en;
  };
  // x-edge (i, j-1/2, q-1/2): e = x, a = y, b = z
  auto eni_x = [&](int i, int j, int q) -> T {
    const T Je = Jx(i, j, q);
    if (!(c.gad > 0.0)) return ni_law(Je, T(0), T(0), T(0), T(0), T(0), T(0));
    const T Ba = half * (fyq(i, j, q) + fyq(i, j, q - 1));
    const T Bb = half * (fzq(i, j, q) + fzq(i, j - 1, q));
    const T Be = T(0.25) * ((wc(BX, i, j, q) + wc(BX, i, j - 1, q)) + (wc(BX, i, j, q - 1) + wc(BX, i, j - 1, q - 1)));
    const T re = T(0.25) * ((wc(RHO, i, j, q) + wc(RHO, i, j - 1, q)) + (wc(RHO, i, j, q - 1) + wc(RHO, i, j - 1, q - 1)));
    const T Ja = T(0.25) * ((Jy(i, j, q) + Jy(i, j - 1, q)) + (Jy(i + 1, j, q) + Jy(i + 1, j - 1, q)));
    const T Jb = T(0.25) * ((Jz(i, j, q) + Jz(i, j, q - 1)) + (Jz(i + 1, j, q) + Jz(i + 1, j, q - 1)));
    return ni_law(Je, Ba, Bb, Be, re, Ja, Jb);
  };
  // y-edge (i-1/2, j, q-1/2): e = y, a = z, b = x
  auto eni_y = [&](int i, int j, int q) -> T {
    const T Je = Jy(i, j, q);
    if (!(c.gad > 0.0)) return ni_law(Je, T(0), T(0), T(0), T(0), T(0), T(0));
    const T Ba = half * (fzq(i, j, q) + fzq(i - 1, j, q));
    const T Bb = half * (fxq(i, j, q) + fxq(i, j, q - 1));
    const T Be = T(0.25) * ((wc(BY, i, j, q) + wc(BY, i, j, q - 1)) + (wc(BY, i - 1, j, q) + wc(BY, i - 1, j, q - 1)));
    const T re = T(0.25) * ((wc(RHO, i, j, q) + wc(RHO, i, j, q - 1)) + (wc(RHO, i - 1, j, q) + wc(RHO, i - 1, j, q - 1)));
    const T Ja = T(0.25) * ((Jz(i, j, q) + Jz(i, j, q - 1)) + (Jz(i, j + 1, q) + Jz(i, j + 1, q - 1)));
    const T Jb = T(0.25) * ((Jx(i, j, q) + Jx(i - 1, j, q)) + (Jx(i, j + 1, q) + Jx(i - 1, j + 1, q)));
    return ni_law(Je, Ba, Bb, Be, re, Ja, Jb);
  };
  // z-edge (i-1/2, j-1/2, q): e = z, a = x, b = y
  auto eni_z = [&](int i, int j, int q) -> T {
    const T Je = Jz(i, j, q);
    if (!(c.gad > 0.0)) return ni_law(Je, T(0), T(0), T(0), T(0), T(0), T(0));
    const T Ba = half * (fxq(i, j, q) + fxq(i, j - 1, q));
    const T Bb = half * (fyq(i, j, q) + fyq(i - 1, j, q));
    const T Be = T(0.25) * ((wc(BZ, i, j, q) + wc(BZ, i - 1, j, q)) + (wc(BZ, i, j - 1, q) + wc(BZ, i - 1, j - 1, q)));
    const T re = T(0.25) * ((wc(RHO, i, j, q) + wc(RHO, i - 1, j, q)) + (wc(RHO, i, j - 1, q) + wc(RHO, i - 1, j - 1, q)));
    const T Ja = T(0.25) * ((Jx(i, j, q) + Jx(i - 1, j, q)) + (Jx(i, j, q + 1) + Jx(i - 1, j, q + 1)));
    const T Jb = T(0.25) * ((Jy(i, j, q) + Jy(i, j - 1, q)) + (Jy(i, j, q + 1) + Jy(i, j - 1, q + 1)));
    return ni_law(Je, Ba, Bb, Be, re, Ja, Jb);
  };
  T *const ENX = sm + L::oENX;
  T *const ENY = sm + L::oENY;
  T *const ENZ = sm + L::oENZ;
  T *const FXE = sm + L::oFXE;
  T *const FYE = sm + L::oFYE;

  T smax_t = T(0);
  T unew[5];
  for (int it = 0; it <= tz + 1; it++) {
    const int p = z0 - 1 + it;
    const int par = it & 1;
    T *const SXc = SX + par * 2 * H1N, *const SXp = SX + (par ^ 1) * 2 * H1N;
    T *const SYc = SY + par * 2 * H1N, *const SYp = SY + (par ^ 1) * 2 * H1N;
    T *const FZc = FZ + par * 5 * H1N, *const FZp = FZ + (par ^ 1) * 5 * H1N;
    T *const DUc = DU + par * 5 * H1N, *const DUp = DU + (par ^ 1) * 5 * H1N;
    T *const EXc = EX + par * H1N, *const EXp = EX + (par ^ 1) * H1N;
    T *const EYc = EY + par * H1N, *const EYp = EY + (par ^ 1) * H1N;
    T *const NBZc = NBZ + par * H1N, *const NBZp = NBZ + (par ^ 1) * H1N;

    // ---- A: plane p+1 -- gathered now (first plane, or with concurrent
    // publishers), else its copies were started one iteration earlier and
    // only the blended values remain
    if (ASYNC) prefetch_old(it, p);
    if (!ASYNC || it == 0) {
      gather_plane(p + 1, GatherMode<GATHER_NOW>{});
    } else {
      cp_async_wait<1>();  // every copy but the old values just started
      if (any_blend) gather_plane(p + 1, GatherMode<GATHER_BLEND>{});
    }
    __syncthreads();
    prim_plane(p + 1);
    if constexpr (NI != 0) currents(p + 1);
    __syncthreads();

    // ---- B: slopes and predictor on the H1 region of plane p
    {
      const int rm = (p - 1 - z0 + 3) % 3, r0 = (p - z0 + 3) % 3, rp = (p + 1 - z0 + 3) % 3;
      const T *Wm = Wr + rm * 8 * H2N, *W0 = Wr + r0 * 8 * H2N, *Wp = Wr + rp * 8 * H2N;
      const T *F0 = FB + fslot(p) * 4 * FPN;
      for (int ci = tid; ci < (TX + 2) * (TY + 2); ci += NT) {
        const int i = ci % (TX + 2) - 1, j = ci / (TX + 2) - 1;
        if (i > tx || j > ty) continue;
        const int h = H2(i, j);
        T w8[8], dX[8], dY[8], dZ[8], ws[8];
#pragma unroll
        for (int k = 0; k < 8; k++) w8[k] = W0[k * H2N + h];
#pragma unroll
        for (int k = 0; k < 8; k++) {
          if (k == BX) dX[k] = F0[F5(i + 1, j)] - F0[F5(i, j)];
          else dX[k] = mc(w8[k] - W0[k * H2N + H2(i - 1, j)], W0[k * H2N + H2(i + 1, j)] - w8[k]);
          if (k == BY) dY[k] = F0[FPN + F5(i, j + 1)] - F0[FPN + F5(i, j)];
          else dY[k] = mc(w8[k] - W0[k * H2N + H2(i, j - 1)], W0[k * H2N + H2(i, j + 1)] - w8[k]);
          if (k == BZ) dZ[k] = F0[3 * FPN + F5(i, j)] - F0[2 * FPN + F5(i, j)];
          else dZ[k] = mc(w8[k] - Wm[k * H2N + h], Wp[k * H2N + h] - w8[k]);
        }
        predict(w8, dX, dY, dZ, gamma, hdt, ws);
        bool bad = false;
#pragma unroll
        for (int d = 0; d < 3; d++) {
          const T *d3 = d == 0 ? dX : d == 1 ? dY : dZ;
          const T rp_ = ws[RHO] + half * d3[RHO], rm_ = ws[RHO] - half * d3[RHO];
          const T pp_ = ws[PR] + half * d3[PR], pm_ = ws[PR] - half * d3[PR];
          if (!tpos(rp_) || !tpos(rm_) || !tpos(pp_) || !tpos(pm_)) bad = true;
        }
        if (bad) {
          atomicAdd(&s_fallback, 1);
#pragma unroll
          for (int k = 0; k < 8; k++) { dX[k] = T(0); dY[k] = T(0); dZ[k] = T(0); ws[k] = w8[k]; }
        }
        const int g = H1(i, j);
#pragma unroll
        for (int k = 0; k < 8; k++) {
          Sws[k * H1N + g] = ws[k];
          SdX[k * H1N + g] = dX[k];
          SdY[k * H1N + g] = dY[k];
          SdZ[k * H1N + g] = dZ[k];
        }
      }
    }
    __syncthreads();
    // plane p-1's primitive ring slot and plane p's faces are dead now: start
    // the copies of plane p+2 into them, to land while C..F run
    if (ASYNC) {
      if (p + 2 <= z0 + tz + 1) gather_plane(p + 2, GatherMode<GATHER_ISSUE>{});
      else cp_async_commit();  // an empty group keeps the wait counts in step
    }

    // ---- C: face fluxes: the x-, y- and z-faces whose fluxes are needed and
    // those whose signal speeds alone are (the halo rows and columns around
    // the tile).  A face's two states are loaded in the frame of its axis
    // (normal component first, then the two tangential ones in cyclic
    // order), the order in which the solvers of axis D read them, so one body
    // serves every axis.  FP64 (POOL) deals all faces of the plane to the
    // block as one pool, every axis running the same instructions in shared
    // warps (an FP64 warp instruction costs its pipe slot whatever its
    // active lanes, and the one block per SM has no other block's warps to
    // fill its idle ones); FP32 runs one loop per axis with the axis a
    // compile-time constant (fewer instructions: its two blocks per SM fill
    // each other's idle warps).
    {
      constexpr int NXF = (TX + 1) * TY, NYF = TX * (TY + 1), NZF = TX * TY;
      constexpr int NXS = 2 * (TX + 1), NYS = 2 * (TY + 1), NZS = 2 * (TX + 2) + 2 * TY;
      auto face_item = [&](auto dd, int i, int j, bool full) {
        const int d = axis_value(dd);
        // the face's cells: left hl, right hr (a z-face's left state is the
        // upper z-face state of plane p-1, carried in ZP)
        const int hr = H1(i, j), hl = hr - (d == 0 ? 1 : d == 1 ? TX + 2 : 0);
        const T *const Sd = d == 0 ? SdX : d == 1 ? SdY : SdZ;
        const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
        const int cmp[8] = {RHO, VX + d, VX + t1, VX + t2, PR, BX + d, BX + t1, BX + t2};
        T WL[8], WR[8], F[5], SL, SR;
#pragma unroll
        for (int k = 0; k < 8; k++) {
          const int o = cmp[k] * H1N;
          WL[k] = d == 2 ? ZP[o + hr] : Sws[o + hl] + half * Sd[o + hl];
          WR[k] = Sws[o + hr] - half * Sd[o + hr];
        }
        if (full) {
          face_flux<T, 0, RS>(WL, WR, gamma, igm1, F, SL, SR);
          T *const Fd = d == 0 ? FX : d == 1 ? FY : FZc;
          Fd[hr] = F[0];
          Fd[(1 + d) * H1N + hr] = F[1];
          Fd[(1 + t1) * H1N + hr] = F[2];
          Fd[(1 + t2) * H1N + hr] = F[3];
          Fd[4 * H1N + hr] = F[4];
        } else {
          hll_speeds<T, 0>(WL, WR, gamma, SL, SR);
        }
        T *const Sp = d == 0 ? SXc : d == 1 ? SYc : SZ;
        Sp[hr] = SL;
        Sp[H1N + hr] = SR;
      };
      // item k of axis d: its face (i, j), whether its flux is needed; false
      // if the face lies outside a partial tile.  Per axis the faces with
      // fluxes come first: x-faces (i-1/2, j), i in [0,tx], j in [0,ty),
      // then the halo rows j = -1 and ty; y-faces (i, j-1/2), i in [0,tx),
      // j in [0,ty], then the halo columns i = -1 and tx; z-faces (i, j,
      // p-1/2) of the tile's cells, then the ring around them.
      auto axis_item = [&](int d, int k, int &i, int &j, bool &full) -> bool {
        if (d == 0) {
          full = k < NXF;
          if (full) {
            i = k % (TX + 1);
            j = k / (TX + 1);
            return i <= tx && j < ty;
          }
          k -= NXF;
          i = k % (TX + 1);
          j = k / (TX + 1) == 0 ? -1 : ty;
          return i <= tx;
        }
        if (d == 1) {
          full = k < NYF;
          if (full) {
            i = k % TX;
            j = k / TX;
            return i < tx && j <= ty;
          }
          k -= NYF;
          i = k / (TY + 1) == 0 ? -1 : tx;
          j = k % (TY + 1);
          return j <= ty;
        }
        full = k < NZF;
        if (full) {
          i = k % TX;
          j = k / TX;
          return i < tx && j < ty;
        }
        k -= NZF;
        if (k < 2 * (TX + 2)) {
          i = k % (TX + 2) - 1;
          j = k / (TX + 2) == 0 ? -1 : ty;
          return i <= tx;
        }
        k -= 2 * (TX + 2);
        i = k / TY == 0 ? -1 : tx;
        j = k % TY;
        return j < ty;
      };
      if constexpr (POOL) {
        // the pool: every face with a flux (x, y, z), then every face with
        // speeds only; one call site, the axis a run-time value
        const int nfull = NXF + NYF + (it > 0 ? NZF : 0);
        const int nitems = nfull + NXS + NYS + (it > 0 ? NZS : 0);
        for (int ci = tid; ci < nitems; ci += NT) {
          int d, k;
          if (ci < nfull) {
            d = ci < NXF ? 0 : ci < NXF + NYF ? 1 : 2;
            k = ci - (d == 0 ? 0 : d == 1 ? NXF : NXF + NYF);
          } else {
            const int s = ci - nfull;
            d = s < NXS ? 0 : s < NXS + NYS ? 1 : 2;
            k = s - (d == 0 ? 0 : d == 1 ? NXS : NXS + NYS) + (d == 0 ? NXF : d == 1 ? NYF : NZF);
          }
          int i, j;
          bool full;
          if (axis_item(d, k, i, j, full)) face_item(d, i, j, full);
        }
      } else {
        for (int ci = tid; ci < NXF + NXS; ci += NT) {
          int i, j;
          bool full;
          if (axis_item(0, ci, i, j, full)) face_item(AxisC<0>{}, i, j, full);
        }
        for (int ci = tid; ci < NYF + NYS; ci += NT) {
          int i, j;
          bool full;
          if (axis_item(1, ci, i, j, full)) face_item(AxisC<1>{}, i, j, full);
        }
        if (it > 0) {
          for (int ci = tid; ci < NZF + NZS; ci += NT) {
            int i, j;
            bool full;
            if (axis_item(2, ci, i, j, full)) face_item(AxisC<2>{}, i, j, full);
          }
        }
      }
    }
    __syncthreads();

    // ---- D: x- and y-edge EMFs at p-1/2, in-plane divergence of plane p.
    // An edge along axis e has the two other axes a and b (x-edge: a = y,
    // b = z; y-edge: a = z, b = x); its corner states at the plane below come
    // carried in CX / CY, the two at plane p are extrapolated here, and one
    // body serves both axes.  FP64 (POOL) deals the x- and y-edges and then,
    // from the next warp boundary on, the cells' divergences to the block as
    // one pool; FP32 runs one loop each with the axis a compile-time constant.
    if (it > 0) {
      constexpr int NXE = TX * (TY + 1), NYE = (TX + 1) * TY, NE = NXE + NYE;
      // with non-ideal terms the energy part waits for the Poynting flux,
      // which needs the edges above this plane: keep the ideal energy
      // fluxes of the plane's x- and y-faces instead
      constexpr int KD = NI ? 4 : 5;
      const bool div = p < z0 + tz;
      auto div_item = [&](int k) {
        const int i = k % TX, j = k / TX;
        if (i >= tx || j >= ty) return;
        const int h = H1(i, j), hx = H1(i + 1, j), hy = H1(i, j + 1);
#pragma unroll
        for (int q = 0; q < KD; q++)
          DUc[q * H1N + h] = (FX[q * H1N + hx] - FX[q * H1N + h]) + (FY[q * H1N + hy] - FY[q * H1N + h]);
      };
      // edge k of axis d (x-edges (i, j-1/2, p-1/2): i in [0,tx), j in
      // [0,ty]; y-edges (i-1/2, j, p-1/2): i in [0,tx], j in [0,ty))
      auto edge_item = [&](auto dd, int k) {
        const int d = axis_value(dd);
        const int i = d == 0 ? k % TX : k % (TX + 1), j = d == 0 ? k / TX : k / (TX + 1);
        if (d == 0 ? (i >= tx || j > ty) : (i > tx || j >= ty)) return;
        // h0: the cell on the edge's high side along its in-plane normal (y
        // for an x-edge, x for a y-edge), hm the one below it
        const int h0 = H1(i, j), hm = h0 - (d == 0 ? TX + 2 : 1);
        const T *const C6 = d == 0 ? CX : CY;
        const T *const SdA = d == 0 ? SdY : SdZ;
        const T *const SdB = d == 0 ? SdZ : SdX;
        const int va = d == 0 ? VY : VZ, vb = d == 0 ? VZ : VX, ba = d == 0 ? BY : BZ, bb = d == 0 ? BZ : BX;
        // the corner at hm: (+a,-b) of an x-edge's low-y cell, (-a,+b) of a
        // y-edge's low-x cell; the corner at h0: (-a,-b)
        const T sA = d == 0 ? half : -half, sB = -sA;
        auto corner = [&](int c, int h, T s1, T s2) -> T {
          return (Sws[c * H1N + h] + s1 * SdA[c * H1N + h]) + s2 * SdB[c * H1N + h];
        };
        const T vam = corner(va, hm, sA, sB), vbm = corner(vb, hm, sA, sB);
        const T bam = corner(ba, hm, sA, sB), bbm = corner(bb, hm, sA, sB);
        const T va0 = corner(va, h0, -half, -half), vb0 = corner(vb, h0, -half, -half);
        const T ba0 = corner(ba, h0, -half, -half), bb0 = corner(bb, h0, -half, -half);
        const T Em = vbm * bam - vam * bbm;
        const T E0 = vb0 * ba0 - va0 * bb0;
        // the two corners carried from the plane below: (-a,-b) at hm and the
        // other one at h0
        const T Ell = C6[hm], Ba_ll = C6[H1N + hm], Bb_ll = C6[2 * H1N + hm];
        const T Ec = C6[3 * H1N + h0], Bac = C6[4 * H1N + h0], Bbc = C6[5 * H1N + h0];
        const T Erl = d == 0 ? Ec : Em, Elr = d == 0 ? Em : Ec;
        const T Ba_rl = d == 0 ? Bac : bam, Ba_lr = d == 0 ? bam : Bac;
        const T Bb_rl = d == 0 ? Bbc : bbm, Bb_lr = d == 0 ? bbm : Bbc;
        // weights: the faces normal to the in-plane normal (y-faces for an
        // x-edge, x-faces for a y-edge) of planes p-1 and p at h0, and the
        // z-faces at p-1/2 of hm and h0
        const T *const Pp = d == 0 ? SYp : SXp;
        const T *const Pc = d == 0 ? SYc : SXc;
        const T ap2 = pmax0(Pp[H1N + h0], Pc[H1N + h0]), am2 = nmax0(Pp[h0], Pc[h0]);
        const T apz = pmax0(SZ[H1N + hm], SZ[H1N + h0]), amz = nmax0(SZ[hm], SZ[h0]);
        const T apa = d == 0 ? ap2 : apz, ama = d == 0 ? am2 : amz;
        const T apb = d == 0 ? apz : ap2, amb = d == 0 ? amz : am2;
        T e = emf(Ell, Erl, Elr, E0, Ba_ll, Ba_rl, Ba_lr, ba0, Bb_ll, Bb_rl, Bb_lr, bb0, apa, ama, apb, amb);
        if constexpr (NI != 0) {
          const T en = d == 0 ? eni_x(i, j, p) : eni_y(i, j, p);
          (d == 0 ? ENX : ENY)[par * H1N + h0] = en;
          e = e + en;
        }
        (d == 0 ? EXc : EYc)[h0] = e;
      };
      if constexpr (POOL) {
        constexpr int DU0 = (NE + 31) / 32 * 32;
        const int nitems = div ? DU0 + TX * TY : NE;
        for (int ci = tid; ci < nitems; ci += NT) {
          if (ci < NE) edge_item(ci < NXE ? 0 : 1, ci < NXE ? ci : ci - NXE);
          else if (ci >= DU0) div_item(ci - DU0);
        }
      } else {
        for (int ci = tid; ci < NXE; ci += NT) edge_item(AxisC<0>{}, ci);
        for (int ci = tid; ci < NYE; ci += NT) edge_item(AxisC<1>{}, ci);
        if (div)
          for (int ci = tid; ci < TX * TY; ci += NT) div_item(ci);
      }
      if constexpr (NI != 0) {
        if (div) {
          for (int ci = tid; ci < (TX + 1) * (TY + 1); ci += NT) {
            const int i = ci % (TX + 1), j = ci / (TX + 1), h = H1(i, j);
            if (i <= tx && j < ty) FXE[par * H1N + h] = FX[4 * H1N + h];
            if (i < tx && j <= ty) FYE[par * H1N + h] = FY[4 * H1N + h];
          }
        }
      }
    }
    __syncthreads();

    // ---- Non-ideal energy flux: the Poynting flux (E_Ohm + E_AD) x B
    // through the z-faces at p-1/2 joins their energy flux, and plane p-1's
    // energy divergence is formed from its x- and y-faces' ideal fluxes plus
    // theirs (edge EMFs averaged to the face, cell-centred B averaged over
    // the two cells of the face)
    if constexpr (NI != 0) {
      if (it >= 1) {
        // z-faces (i, j, p-1/2): d = z, a = x, b = y
        for (int ci = tid; ci < TX * TY; ci += NT) {
          const int i = ci % TX, j = ci / TX;
          if (i >= tx || j >= ty) continue;
          const int h = H1(i, j);
          const T Ea = half * (ENX[par * H1N + h] + ENX[par * H1N + H1(i, j + 1)]);
          const T Eb = half * (ENY[par * H1N + h] + ENY[par * H1N + H1(i + 1, j)]);
          const T Ba = half * (wc(BX, i, j, p - 1) + wc(BX, i, j, p));
          const T Bb = half * (wc(BY, i, j, p - 1) + wc(BY, i, j, p));
          FZc[4 * H1N + h] = FZc[4 * H1N + h] + (Ea * Bb - Eb * Ba);
        }
      }
      if (it >= 2) {
        const int q = p - 1, pr = par ^ 1;
        // x-face (i-1/2, j, q): d = x, a = y (levels q-1/2, q+1/2), b = z
        auto ftx = [&](int i, int j) -> T {
          const T Ea = half * (ENY[pr * H1N + H1(i, j)] + ENY[par * H1N + H1(i, j)]);
          const T Eb = half * (ENZ[H1(i, j)] + ENZ[H1(i, j + 1)]);
          const T Ba = half * (wc(BY, i - 1, j, q) + wc(BY, i, j, q));
          const T Bb = half * (wc(BZ, i - 1, j, q) + wc(BZ, i, j, q));
          return FXE[pr * H1N + H1(i, j)] + (Ea * Bb - Eb * Ba);
        };
        // y-face (i, j-1/2, q): d = y, a = z, b = x (levels q-1/2, q+1/2)
        auto fty = [&](int i, int j) -> T {
          const T Ea = half * (ENZ[H1(i, j)] + ENZ[H1(i + 1, j)]);
          const T Eb = half * (ENX[pr * H1N + H1(i, j)] + ENX[par * H1N + H1(i, j)]);
          const T Ba = half * (wc(BZ, i, j - 1, q) + wc(BZ, i, j, q));
          const T Bb = half * (wc(BX, i, j - 1, q) + wc(BX, i, j, q));
          return FYE[pr * H1N + H1(i, j)] + (Ea * Bb - Eb * Ba);
        };
        for (int ci = tid; ci < TX * TY; ci += NT) {
          const int i = ci % TX, j = ci / TX;
          if (i >= tx || j >= ty) continue;
          DUp[4 * H1N + H1(i, j)] = (ftx(i + 1, j) - ftx(i, j)) + (fty(i, j + 1) - fty(i, j));
        }
      }
      __syncthreads();
    }

    // ---- E: update plane p-1 and the z-faces at p-1/2
    const bool upd = it >= 2;
    const int ui = tid % TX, uj = tid / TX;
    const bool mine = tid < TX * TY && ui < tx && uj < ty;
    if (ASYNC) cp_async_wait<1>();  // this thread's old values (not plane p+2's copies)
    auto old_u = [&](int k, long long ci) -> T { return !ASYNC ? *src(own + k * nc + ci) : OLD[L::OLDU + k * TX * TY + tid]; };
    if (upd && mine) {
      const int i = ui, j = uj, h = H1(i, j);
      const long long ci = ((long long)(p - 1) * ny + (y0 + j)) * nx + (x0 + i);
#pragma unroll
      for (int k = 0; k < 5; k++) {
        const T fz = FZc[k * H1N + h] - FZp[k * H1N + h];
        unew[k] = old_u(k, ci) - dtdx * (DUp[k * H1N + h] + fz);
        put_global(dst + k * nc + ci, unew[k]);
      }
    }
    if (it >= 1) {
      each_eface(upd, true, [&](int e, auto kdd, int i, int j) {
        const int kd = axis_value(kdd);
        const int h = H1(i, j);
        if (kd == 0) {
          const long long id = ((long long)(p - 1) * ny + (y0 + j)) * (nx + 1) + (x0 + i);
          const T b = (!ASYNC ? *src(own + ofx + id) : OLD[L::OLDX + e]) - dtdx * ((EZ[H1(i, j + 1)] - EZ[h]) - (EYc[h] - EYp[h]));
          NBX[h] = b;
          put_global(dst + ofx + id, b);
        } else if (kd == 1) {
          const long long id = ((long long)(p - 1) * (ny + 1) + (y0 + j)) * nx + (x0 + i);
          const T b = (!ASYNC ? *src(own + ofy + id) : OLD[L::OLDX + e]) - dtdx * ((EXc[h] - EXp[h]) - (EZ[H1(i + 1, j)] - EZ[h]));
          NBY[h] = b;
          put_global(dst + ofy + id, b);
        } else {
          const long long id = ((long long)p * ny + (y0 + j)) * nx + (x0 + i);
          const T b = (!ASYNC ? *src(own + ofz + id) : OLD[L::OLDX + e]) - dtdx * ((EYc[H1(i + 1, j)] - EYc[h]) - (EXc[H1(i, j + 1)] - EXc[h]));
          NBZc[h] = b;
          put_global(dst + ofz + id, b);
        }
      });
    }
    __syncthreads();

    // ---- F: signal speed of plane p-1, z-edge EMFs of plane p, carried values
    if (upd && mine) {
      const int i = ui, j = uj, h = H1(i, j);
      T Wn[8];
      int floored = 0;
      prim(unew[0], unew[1], unew[2], unew[3], unew[4], NBX[h], NBX[H1(i + 1, j)], NBY[h], NBY[H1(i, j + 1)],
           NBZp[h], NBZc[h], gamma, Wn, &floored);
      if (floored) atomicAdd(&S.floors, 1);
      if (!(Wn[RHO] > T(0)) || !(Wn[PR] > T(0)))
        set_error(c, DSP_ERR_UNPHYSICAL, P, ((long long)(p - 1) * ny + (y0 + j)) * nx + (x0 + i));
      if constexpr (NI != 0)
        smax_t = tmax(smax_t, tmax(signal_sum(Wn, gamma), nonideal_speed(Wn, c.cfl, c.eta, c.gad, c.rhoi, c.cohm, c.cad, dxl)));
      else smax_t = tmax(smax_t, signal_sum(Wn, gamma));
    }
    {
      // the z-edge EMFs of plane p and the values of plane p carried to the
      // next plane (its upper z-face state and its +z corner values for the
      // x- and y-edges above it).  FP64 deals them as one pool of items,
      // the carried values from the next warp boundary on, from the first
      // warp after the cell-updating ones (which have the new cells' signal
      // speeds to compute); FP32 runs one loop each from thread 0.
      constexpr int NZE = (TX + 1) * (TY + 1), CA0 = (NZE + 31) / 32 * 32, NCA = (TX + 2) * (TY + 2);
      const bool zedges = p >= z0 && p < z0 + tz;
      // z-edges (i-1/2, j-1/2, p): i in [0,tx], j in [0,ty]; a = x, b = y
      auto zedge_item = [&](int k) {
        const int i = k % (TX + 1), j = k / (TX + 1);
        if (i > tx || j > ty) return;
        const int hll_ = H1(i - 1, j - 1), hrl = H1(i, j - 1), hlr = H1(i - 1, j), hrr = H1(i, j);
        const T ll_vx = (Sws[VX * H1N + hll_] + half * SdX[VX * H1N + hll_]) + half * SdY[VX * H1N + hll_];
        const T ll_vy = (Sws[VY * H1N + hll_] + half * SdX[VY * H1N + hll_]) + half * SdY[VY * H1N + hll_];
        const T ll_bx = (Sws[BX * H1N + hll_] + half * SdX[BX * H1N + hll_]) + half * SdY[BX * H1N + hll_];
        const T ll_by = (Sws[BY * H1N + hll_] + half * SdX[BY * H1N + hll_]) + half * SdY[BY * H1N + hll_];
        const T rl_vx = (Sws[VX * H1N + hrl] - half * SdX[VX * H1N + hrl]) + half * SdY[VX * H1N + hrl];
        const T rl_vy = (Sws[VY * H1N + hrl] - half * SdX[VY * H1N + hrl]) + half * SdY[VY * H1N + hrl];
        const T rl_bx = (Sws[BX * H1N + hrl] - half * SdX[BX * H1N + hrl]) + half * SdY[BX * H1N + hrl];
        const T rl_by = (Sws[BY * H1N + hrl] - half * SdX[BY * H1N + hrl]) + half * SdY[BY * H1N + hrl];
        const T lr_vx = (Sws[VX * H1N + hlr] + half * SdX[VX * H1N + hlr]) - half * SdY[VX * H1N + hlr];
        const T lr_vy = (Sws[VY * H1N + hlr] + half * SdX[VY * H1N + hlr]) - half * SdY[VY * H1N + hlr];
        const T lr_bx = (Sws[BX * H1N + hlr] + half * SdX[BX * H1N + hlr]) - half * SdY[BX * H1N + hlr];
        const T lr_by = (Sws[BY * H1N + hlr] + half * SdX[BY * H1N + hlr]) - half * SdY[BY * H1N + hlr];
        const T rr_vx = (Sws[VX * H1N + hrr] - half * SdX[VX * H1N + hrr]) - half * SdY[VX * H1N + hrr];
        const T rr_vy = (Sws[VY * H1N + hrr] - half * SdX[VY * H1N + hrr]) - half * SdY[VY * H1N + hrr];
        const T rr_bx = (Sws[BX * H1N + hrr] - half * SdX[BX * H1N + hrr]) - half * SdY[BX * H1N + hrr];
        const T rr_by = (Sws[BY * H1N + hrr] - half * SdX[BY * H1N + hrr]) - half * SdY[BY * H1N + hrr];
        const T Ell = ll_vy * ll_bx - ll_vx * ll_by;
        const T Erl = rl_vy * rl_bx - rl_vx * rl_by;
        const T Elr = lr_vy * lr_bx - lr_vx * lr_by;
        const T Err = rr_vy * rr_bx - rr_vx * rr_by;
        const T apa = pmax0(SXc[H1N + hrl], SXc[H1N + hrr]);
        const T ama = nmax0(SXc[hrl], SXc[hrr]);
        const T apb = pmax0(SYc[H1N + hlr], SYc[H1N + hrr]);
        const T amb = nmax0(SYc[hlr], SYc[hrr]);
        T ez = emf(Ell, Erl, Elr, Err, ll_bx, rl_bx, lr_bx, rr_bx, ll_by, rl_by, lr_by, rr_by, apa, ama, apb, amb);
        if constexpr (NI != 0) {
          const T en = eni_z(i, j, p);
          ENZ[hrr] = en;
          ez = ez + en;
        }
        EZ[hrr] = ez;
      };
      auto carry_item = [&](int c) {
        const int i = c % (TX + 2) - 1, j = c / (TX + 2) - 1, h = H1(i, j);
        if (i > tx || j > ty) return;
#pragma unroll
        for (int k = 0; k < 8; k++) ZP[k * H1N + h] = Sws[k * H1N + h] + half * SdZ[k * H1N + h];
        {  // x-edges: a = y, b = z; corners (+y,+z) and (-y,+z)
          const T py_vy = (Sws[VY * H1N + h] + half * SdY[VY * H1N + h]) + half * SdZ[VY * H1N + h];
          const T py_vz = (Sws[VZ * H1N + h] + half * SdY[VZ * H1N + h]) + half * SdZ[VZ * H1N + h];
          const T py_by = (Sws[BY * H1N + h] + half * SdY[BY * H1N + h]) + half * SdZ[BY * H1N + h];
          const T py_bz = (Sws[BZ * H1N + h] + half * SdY[BZ * H1N + h]) + half * SdZ[BZ * H1N + h];
          const T my_vy = (Sws[VY * H1N + h] - half * SdY[VY * H1N + h]) + half * SdZ[VY * H1N + h];
          const T my_vz = (Sws[VZ * H1N + h] - half * SdY[VZ * H1N + h]) + half * SdZ[VZ * H1N + h];
          const T my_by = (Sws[BY * H1N + h] - half * SdY[BY * H1N + h]) + half * SdZ[BY * H1N + h];
          const T my_bz = (Sws[BZ * H1N + h] - half * SdY[BZ * H1N + h]) + half * SdZ[BZ * H1N + h];
          CX[0 * H1N + h] = py_vz * py_by - py_vy * py_bz;
          CX[1 * H1N + h] = py_by;
          CX[2 * H1N + h] = py_bz;
          CX[3 * H1N + h] = my_vz * my_by - my_vy * my_bz;
          CX[4 * H1N + h] = my_by;
          CX[5 * H1N + h] = my_bz;
        }
        {  // y-edges: a = z, b = x; corners (+z,+x) and (+z,-x)
          const T px_vz = (Sws[VZ * H1N + h] + half * SdZ[VZ * H1N + h]) + half * SdX[VZ * H1N + h];
          const T px_vx = (Sws[VX * H1N + h] + half * SdZ[VX * H1N + h]) + half * SdX[VX * H1N + h];
          const T px_bz = (Sws[BZ * H1N + h] + half * SdZ[BZ * H1N + h]) + half * SdX[BZ * H1N + h];
          const T px_bx = (Sws[BX * H1N + h] + half * SdZ[BX * H1N + h]) + half * SdX[BX * H1N + h];
          const T mx_vz = (Sws[VZ * H1N + h] + half * SdZ[VZ * H1N + h]) - half * SdX[VZ * H1N + h];
          const T mx_vx = (Sws[VX * H1N + h] + half * SdZ[VX * H1N + h]) - half * SdX[VX * H1N + h];
          const T mx_bz = (Sws[BZ * H1N + h] + half * SdZ[BZ * H1N + h]) - half * SdX[BZ * H1N + h];
          const T mx_bx = (Sws[BX * H1N + h] + half * SdZ[BX * H1N + h]) - half * SdX[BX * H1N + h];
          CY[0 * H1N + h] = px_vx * px_bz - px_vz * px_bx;
          CY[1 * H1N + h] = px_bz;
          CY[2 * H1N + h] = px_bx;
          CY[3 * H1N + h] = mx_vx * mx_bz - mx_vz * mx_bx;
          CY[4 * H1N + h] = mx_bz;
          CY[5 * H1N + h] = mx_bx;
        }
      };
      if constexpr (POOL) {
        for (int ci = rot; ci < CA0 + NCA; ci += NT) {
          if (ci < CA0) {
            if (zedges && ci < NZE) zedge_item(ci);
          } else {
            carry_item(ci - CA0);
          }
        }
      } else {
        if (zedges)
          for (int ci = tid; ci < NZE; ci += NT) zedge_item(ci);
        for (int ci = tid; ci < NCA; ci += NT) carry_item(ci);
      }
    }
    __syncthreads();
  }

  // signal speed of the new slice: block max, then the patch max
  {
    double v = (double)smax_t;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
      double u = tid < NT / 32 ? red[tid] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) u = fmax(u, __shfl_xor_sync(0xffffffffu, u, o));
      if (tid == 0) {
        atomicMax(&c.smax_new[P], (unsigned long long)__double_as_longlong(u));
        if (s_fallback) atomicAdd((unsigned long long *)&c.cnt[CNT_FALLBACKS], (unsigned long long)s_fallback);
        if (S.floors) atomicAdd((unsigned long long *)&c.cnt[CNT_FLOORS], (unsigned long long)S.floors);
      }
    }
    __syncthreads();
  }
#undef H2
#undef H1
#undef F5
}

// Sweep dispatcher: every (ready patch, tile) work item of size classes
// [cls, cls_end) in the current work list (grouped by class), grid-strided
// over a persistent grid.
// VARIANT only tells apart instantiations compiled with different
// floating-point contraction flags (FP64 with and without FMA); RS is the
// Riemann solver of the face fluxes (0 HLL, 1 HLLD).
template <typename T, int TX, int TY, int NT, int MINB, int VARIANT, int RS, int NI>
__global__ void __launch_bounds__(NT, MINB) update_kernel(DevCtx c, int cls, int cls_end) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ TileShared<T, NT> S;
  const int rb = c.ctl[CTL_CLS + cls], re = c.ctl[CTL_CLS + cls_end];
  const int wb = c.work_off[rb], we = c.work_off[re];
  for (int w = wb + blockIdx.x; w < we; w += gridDim.x) {
    // ready patch r owns work items [work_off[r], work_off[r+1])
    int lo = rb, hi = re - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (c.work_off[mid] <= w) lo = mid;
      else hi = mid - 1;
    }
    const int r = c.Rk[lo];
    process_tile<T, TX, TY, NT, false, RS, NI>(c, c.R[r], c.dtR[r], w - c.work_off[lo], reinterpret_cast<T *>(smraw),
                                               S);
  }
}

// ---------------------------------------------------------------- ready queue
// The queue is a ring of c.q_cap tile tickets: pushing patch Q takes the
// next T_Q tickets (one atomic add on q_ctl[1]) and publishes one slot per
// tile; a block claims the next ticket (one atomic add on q_ctl[0]) and
// waits until its slot carries that ticket.  Ticket t lives in slot
// t % q_cap; a producer may fill the slot once q_free == t, a consumer read
// it once q_seq == t.  Patches of different sizes simply take different
// numbers of tickets.  Every wait is bounded by c.wait_budget clock cycles,
// after which the waiter records DSP_ERR_TIMEOUT and the kernel winds down.

static __device__ __forceinline__ void queue_push(const DevCtx &c, int Q, double dt) {
  const unsigned long long C = (unsigned long long)c.q_cap;
  const int T = c.geo[Q].tiles;
  const unsigned long long t0 = atomicAdd(&c.q_ctl[1], (unsigned long long)T);
  for (int k = 0; k < T; k++) {
    const unsigned long long t = t0 + k;
    const long long slot = (long long)(t % C);
    const long long c0 = clock64();
    while (ld_acquire(&c.q_free[slot]) != t) {
      if (clock64() - c0 > c.wait_budget || ld_acquire(&c.ctl[CTL_STATUS]) != 0) {
        set_error(c, DSP_ERR_TIMEOUT, Q, -1);
        return;
      }
      __nanosleep(100);
    }
    c.q_patch[slot] = Q;
    c.q_tile[slot] = k;
    c.q_dt[slot] = dt;
    st_release(&c.q_seq[slot], t);
  }
}

// Queue Q if it is idle and ready; the claim (p_state 0 -> 1) makes sure only
// one of the patches that finish around the same time queues it.
static __device__ void try_queue(const DevCtx &c, int Q, double t_end) {
  for (int attempt = 0; attempt < 8; attempt++) {
    if (ld_acquire(&c.p_state[Q]) != 0) return;
    double tq;
    if (!is_ready<true>(c, Q, t_end, &tq)) return;
    if (atomicCAS(&c.p_state[Q], 0, 1) != 0) return;
    __threadfence();
    if (is_ready<true>(c, Q, t_end, &tq)) {
      double dt;
      const int rc = patch_dt<true>(c, Q, tq, t_end, &dt);
      if (rc != DSP_OK) {
        set_error(c, rc, Q, -1);
        return;
      }
      atomicExch(&c.smax_new[Q], 0ull);
      __threadfence();
      queue_push(c, Q, dt);
      return;
    }
    // Q moved on between the test and the claim: release and look again
    atomicExch(&c.p_state[Q], 0);
    __threadfence();
  }
}

// The last tile of P is done: publish P's new slice (time, signal speed,
// schedule entry, newest index with release).  One thread; the block then
// tests P and its neighbours for readiness, one patch per thread.
static __device__ void publish_patch(const DevCtx &c, int P, double dt, double t_end) {
  const int ns = c.ns;
  const int L = ld_acquire(c.latest + P), Ln = (L + 1) % ns;
  const double t = __ldcg(c.t_slot + (long long)P * ns + L);
  const double tn = t + dt;
  c.t_slot[(long long)P * ns + Ln] = tn;
  c.smax_slot[(long long)P * ns + Ln] = __longlong_as_double((long long)atomicAdd(&c.smax_new[P], 0ull));
  c.dt_last[P] = dt;
  const unsigned long long e = atomicAdd((unsigned long long *)&c.cnt[CNT_NSCHED], 1ull);
  if ((long long)e < c.sched_cap) {
    c.sched[e].patch = P;
    c.sched[e].t_start = t;
    c.sched[e].dt = dt;
  }
  atomicAdd((unsigned long long *)&c.cnt[CNT_PATCH_UPDATES], 1ull);
  atomicAdd((unsigned long long *)&c.cnt[CNT_CELL_UPDATES],
            (unsigned long long)c.geo[P].n[0] * c.geo[P].n[1] * c.geo[P].n[2]);
  __threadfence();
  st_release(c.latest + P, Ln);
  __threadfence();
  if (!(tn < t_end)) atomicAdd(&c.q_ctl[2], 1ull);
  st_release(&c.p_state[P], 0);
  __threadfence();
}

// Persistent ready-queue dispatcher (one block per resident slot): claim the
// next (entry, tile) work item, wait for the entry, update the tile; the block
// that finishes a patch's last tile publishes it and queues what became ready.
template <typename T, int TX, int TY, int NT, int MINB, int VARIANT, int RS, int NI>
__global__ void __launch_bounds__(NT, MINB) queue_kernel(DevCtx c, double t_end) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ TileShared<T, NT> S;
  __shared__ int s_P, s_tile, s_exit, s_last;
  __shared__ double s_dt;
  const int tid = threadIdx.x;
  const unsigned long long C = (unsigned long long)c.q_cap;
  for (;;) {
    if (tid == 0) {
      s_exit = 0;
      const unsigned long long t = atomicAdd(&c.q_ctl[0], 1ull);
      const long long slot = (long long)(t % C);
      const long long t0 = clock64();
      while (ld_acquire(&c.q_seq[slot]) != t) {
        if (ld_acquire(&c.q_ctl[2]) >= (unsigned long long)c.np || ld_acquire(&c.ctl[CTL_STATUS]) != 0) {
          s_exit = 1;
          break;
        }
        if (clock64() - t0 > c.wait_budget) {
          set_error(c, DSP_ERR_TIMEOUT, -1, -1);
          s_exit = 1;
          break;
        }
        __nanosleep(200);
      }
      if (!s_exit) {
        s_P = __ldcg(c.q_patch + slot);
        s_tile = __ldcg(c.q_tile + slot);
        s_dt = __ldcg(c.q_dt + slot);
        st_release(&c.q_free[slot], t + C);
      }
    }
    __syncthreads();
    if (s_exit) return;
    const int P = s_P, tile = s_tile;
    const double dt = s_dt;
    process_tile<T, TX, TY, NT, true, RS, NI>(c, P, dt, tile, reinterpret_cast<T *>(smraw), S);
    if (tid == 0) {
      __threadfence();
      const int k = atomicAdd(&c.tiles_done[P], 1);
      s_last = k == c.geo[P].tiles - 1;
      if (s_last) {
        __threadfence();
        c.tiles_done[P] = 0;
        publish_patch(c, P, dt, t_end);
      }
    }
    __syncthreads();
    if (s_last) {
      // P and each neighbour tested (and queued if it became ready) by its
      // own thread: the tests are independent (the queue claim is a CAS), and
      // one thread doing all of them in turn took longer than the update
      const int nb0 = c.nbl_off[P], nnb = c.nbl_off[P + 1] - nb0;
      for (int i = tid; i <= nnb; i += NT) try_queue(c, i == 0 ? P : c.nbl[nb0 + i - 1], t_end);
    }
    __syncthreads();
  }
}
template <typename T, int TX, int TY, int NT, int MINB, int VARIANT, int RS, int NI>
int launch_update(const DevCtx &c, int grid, void *stream, int cls, int cls_end) {
  // the shared-memory attribute was set by update_grid when the context was
  // created (a launch may be inside a stream capture)
  const size_t smem = sizeof(T) * (size_t)Lay<TX, TY, NI>::total;
  update_kernel<T, TX, TY, NT, MINB, VARIANT, RS, NI><<<grid, NT, smem, (cudaStream_t)stream>>>(c, cls, cls_end);
  return cudaGetLastError() == cudaSuccess ? DSP_OK : DSP_ERR_CUDA;
}

template <typename T, int TX, int TY, int NT, int MINB, int VARIANT, int RS, int NI>
int launch_queue(const DevCtx &c, int grid, double t_end, void *stream) {
  const size_t smem = sizeof(T) * (size_t)Lay<TX, TY, NI>::total;
  static bool configured = false;
  if (!configured) {
    if (cudaFuncSetAttribute(queue_kernel<T, TX, TY, NT, MINB, VARIANT, RS, NI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return DSP_ERR_CUDA;
    configured = true;
  }
  // one block per resident slot, so that every waiting block is co-resident
  // with the blocks it waits for
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, queue_kernel<T, TX, TY, NT, MINB, VARIANT, RS, NI>, NT, smem);
  if (per < 1) return DSP_ERR_CUDA;
  const int g = nsm * per < grid ? nsm * per : grid;
  queue_kernel<T, TX, TY, NT, MINB, VARIANT, RS, NI><<<g, NT, smem, (cudaStream_t)stream>>>(c, t_end);
  return cudaGetLastError() == cudaSuccess ? DSP_OK : DSP_ERR_CUDA;
}

template <typename T, int TX, int TY, int NT, int MINB, int VARIANT, int RS, int NI>
int update_grid(const DevCtx &c, int cls, int cls_end) {
  const size_t smem = sizeof(T) * (size_t)Lay<TX, TY, NI>::total;
  cudaFuncSetAttribute(update_kernel<T, TX, TY, NT, MINB, VARIANT, RS, NI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, update_kernel<T, TX, TY, NT, MINB, VARIANT, RS, NI>, NT, smem);
  if (per < 1) per = 1;
  long long maxwork = 0;  // every patch of the classes ready
  for (int k = cls; k < cls_end; k++) maxwork += c.cls_tiles[k];
  long long g = (long long)nsm * per;
  return (int)(g < maxwork ? g : maxwork);
}

}  // namespace dsp

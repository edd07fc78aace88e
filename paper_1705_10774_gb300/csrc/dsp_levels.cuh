// dsp_levels.cuh -- guard values across a resolution jump (DISPATCH I,
// Sec. 3 A: guard zones are interpolated in space as well as in time when
// neighbours differ in resolution; prolongation by conservative
// interpolation, restriction by averaging).
//
// Before a patch with such guards is updated, one block fills the patch's
// cross-level guard buffer for the patch's time: a level-1 patch gets, for
// every padded cell that no level-1 patch owns, its level-0 parent plus a
// quarter of the parent's MC-limited slopes (signed by the child's side), and
// for every such face the level-0 face it lies on or the mean of the parent's
// two faces along its axis; a level-0 patch gets, for every guard cell
// covered by level 1, the mean of its 8 children (summed z-, y-, x-child in
// that order), and for every such face the mean of the 4 level-1 faces on it.
// Level-0 values are read as stored, also under the refined region.  The
// operation order is the oracle's, so the FP64 build reproduces it exactly.
#pragma once
#include <cuda_runtime.h>

#include "dsp_dispatch.cuh"
#include "dsp_internal.h"
#include "dsp_physics.cuh"

namespace dsp {

__device__ __forceinline__ void xl_status(const DevCtx &c, int code, int P) {
  if (atomicCAS(&c.ctl[CTL_STATUS], 0, code) == 0) c.ctl[CTL_ERRP] = P;
}

__device__ __forceinline__ int xl_floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int xl_posmod(int a, int b) {
  const int r = a % b;
  return r < 0 ? r + b : r;
}

// Map block of a wrapped level-lev cell (floor of a small integer quotient
// through a float product, exact for level extents far below 2^20 cells).
__device__ __forceinline__ long long xl_block(const DevCtx &c, int lev, const int w[3]) {
  int b[3];
  for (int d = 0; d < 3; d++) b[d] = __float2int_rd(((float)w[d] + 0.5f) * c.binv[lev][d]);
  return ((long long)b[2] * c.mapd[lev][1] + b[1]) * c.mapd[lev][0] + b[0];
}

// The slices of patch Q that supply time t (pick_slices): A alone (a copy),
// A + w0 (B - A), or (w0 A + w1 B) + w2 C.
template <typename T>
struct XSrc {
  const T *A, *B, *C;
  T w[3];
  int Q, loc[3];
};

// Owner on level lev of the (unwrapped) level-lev cell g, its local cell
// index, and the slices for time t.  Returns 0, or an error code.
template <typename T>
__device__ int xl_source(const DevCtx &c, int lev, const int g[3], double t, XSrc<T> &s) {
  int w[3];
  for (int d = 0; d < 3; d++) w[d] = xl_posmod(g[d], c.L[lev][d]);
  const int Q = c.omap[lev][xl_block(c, lev, w)];
  if (Q < 0) return DSP_ERR_INVALID_ARG;
  const PatchGeo &gq = c.geo[Q];
  for (int d = 0; d < 3; d++) s.loc[d] = w[d] - gq.lo[d];
  s.Q = Q;
  const T *base = (const T *)c.slab + gq.off;
  SlicePick pk;
  if (pick_slices<false>(c, Q, t, pk) != DSP_OK) return DSP_ERR_BRACKET;
  s.A = base + (long long)pk.s[0] * c.slot_stride;
  s.B = pk.n >= 2 ? base + (long long)pk.s[1] * c.slot_stride : nullptr;
  s.C = pk.n == 3 ? base + (long long)pk.s[2] * c.slot_stride : nullptr;
  for (int q = 0; q < 3; q++) s.w[q] = q < pk.n ? (T)pk.w[q] : T(0);
  return DSP_OK;
}

template <typename T>
__device__ __forceinline__ T xl_val(const XSrc<T> &s, long long idx) {
  T a = s.A[idx];
  if (s.C) a = (s.w[0] * a + s.w[1] * s.B[idx]) + s.w[2] * s.C[idx];
  else if (s.B) a = a + s.w[0] * (s.B[idx] - a);
  return a;
}

// Conserved values of level-lev cell g at time t.
template <typename T>
__device__ int xl_cell(const DevCtx &c, int lev, const int g[3], double t, T u[5]) {
  XSrc<T> s;
  const int rc = xl_source<T>(c, lev, g, t, s);
  if (rc) return rc;
  const PatchGeo &gq = c.geo[s.Q];
  const long long nc = (long long)gq.n[0] * gq.n[1] * gq.n[2];
  const long long id = ((long long)s.loc[2] * gq.n[1] + s.loc[1]) * gq.n[0] + s.loc[0];
  for (int q = 0; q < 5; q++) u[q] = xl_val(s, q * nc + id);
  return DSP_OK;
}

// Face along ax on the low side of level-lev cell g (up = 1: its high side,
// owned by the same patch) at time t.
template <typename T>
__device__ int xl_face(const DevCtx &c, int lev, int ax, const int g[3], int up, double t, T *out) {
  XSrc<T> s;
  const int rc = xl_source<T>(c, lev, g, t, s);
  if (rc) return rc;
  const PatchGeo &gq = c.geo[s.Q];
  const int qx = gq.n[0], qy = gq.n[1], qz = gq.n[2];
  s.loc[ax] += up;
  const long long nc = (long long)qx * qy * qz;
  long long idx;
  if (ax == 0) idx = 5 * nc + ((long long)s.loc[2] * qy + s.loc[1]) * (qx + 1) + s.loc[0];
  else if (ax == 1)
    idx = 5 * nc + (long long)(qx + 1) * qy * qz + ((long long)s.loc[2] * (qy + 1) + s.loc[1]) * qx + s.loc[0];
  else
    idx = 5 * nc + (long long)(qx + 1) * qy * qz + (long long)qx * (qy + 1) * qz + ((long long)s.loc[2] * qy + s.loc[1]) * qx +
          s.loc[0];
  *out = xl_val(s, idx);
  return DSP_OK;
}

// Level-0 cell C (covered by level 1) restricted from its 8 children (one
// level-1 patch holds all of them: level-1 patches cover whole level-0
// cells).
template <typename T>
__device__ int xl_restrict_cell(const DevCtx &c, const int C[3], double t, T u[5]) {
  const int f0[3] = {2 * C[0], 2 * C[1], 2 * C[2]};
  XSrc<T> s;
  const int rc = xl_source<T>(c, 1, f0, t, s);
  if (rc) return rc;
  const PatchGeo &gq = c.geo[s.Q];
  const long long nc = (long long)gq.n[0] * gq.n[1] * gq.n[2];
  T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
  for (int kz = 0; kz < 2; kz++)
    for (int ky = 0; ky < 2; ky++)
      for (int kx = 0; kx < 2; kx++) {
        const long long id = ((long long)(s.loc[2] + kz) * gq.n[1] + s.loc[1] + ky) * gq.n[0] + s.loc[0] + kx;
        for (int q = 0; q < 5; q++) acc[q] = acc[q] + xl_val(s, q * nc + id);
      }
  for (int q = 0; q < 5; q++) u[q] = T(0.125) * acc[q];
  return DSP_OK;
}

// Face along ax on the low side of level-0 cell C, the mean of the 4 level-1
// faces on it (the children's low faces, in one level-1 patch).
template <typename T>
__device__ int xl_restrict_face(const DevCtx &c, int ax, const int C[3], double t, T *out) {
  const int f0[3] = {2 * C[0], 2 * C[1], 2 * C[2]};
  XSrc<T> s;
  const int rc = xl_source<T>(c, 1, f0, t, s);
  if (rc) return rc;
  const PatchGeo &gq = c.geo[s.Q];
  const int qx = gq.n[0], qy = gq.n[1], qz = gq.n[2];
  const long long nc = (long long)qx * qy * qz;
  T acc = T(0);
  for (int kz = 0; kz < 2; kz++)
    for (int ky = 0; ky < 2; ky++)
      for (int kx = 0; kx < 2; kx++) {
        const int k3[3] = {kx, ky, kz};
        if (k3[ax]) continue;
        const int l0 = s.loc[0] + kx, l1 = s.loc[1] + ky, l2 = s.loc[2] + kz;
        long long idx;
        if (ax == 0) idx = 5 * nc + ((long long)l2 * qy + l1) * (qx + 1) + l0;
        else if (ax == 1) idx = 5 * nc + (long long)(qx + 1) * qy * qz + ((long long)l2 * (qy + 1) + l1) * qx + l0;
        else
          idx = 5 * nc + (long long)(qx + 1) * qy * qz + (long long)qx * (qy + 1) * qz + ((long long)l2 * qy + l1) * qx + l0;
        acc = acc + xl_val(s, idx);
      }
  *out = T(0.25) * acc;
  return DSP_OK;
}

// Does the guard gather of a level-lev patch take level-lev cell g from the
// other level?
__device__ __forceinline__ bool xl_cross(const DevCtx &c, int lev, const int g[3]) {
  int w[3];
  for (int d = 0; d < 3; d++) w[d] = xl_posmod(g[d], c.L[lev][d]);
  return c.gmap[lev][xl_block(c, lev, w)] < 0;
}

// Position x (box coordinates, each in [0, b_d)) of shell item s of a box
// of b0 x b1 x b2 points around an inner box [2, b_d - 2) per axis: the 2-deep
// shell, enumerated as the four outer z-planes, then the four outer y-rows
// of the inner z-range, then the four outer x-points of the inner y- and
// z-range.  The shell has b0 b1 b2 - (b0-4)(b1-4)(b2-4) items.
__device__ __forceinline__ void xl_shell(long long s, const int b[3], int x[3]) {
  const long long pz = (long long)b[0] * b[1];
  if (s < 4 * pz) {
    const int k = (int)(s / pz);
    const long long r = s - k * pz;
    x[2] = k < 2 ? k : b[2] - 4 + k;
    x[1] = (int)(r / b[0]);
    x[0] = (int)(r % b[0]);
    return;
  }
  s -= 4 * pz;
  const long long py = 4ll * b[0];
  if (s < py * (b[2] - 4)) {
    x[2] = 2 + (int)(s / py);
    const long long r = s % py;
    const int k = (int)(r / b[0]);
    x[1] = k < 2 ? k : b[1] - 4 + k;
    x[0] = (int)(r % b[0]);
    return;
  }
  s -= py * (b[2] - 4);
  const long long px = 4ll * (b[1] - 4);
  x[2] = 2 + (int)(s / px);
  const long long r = s % px;
  x[1] = 2 + (int)(r / 4);
  const int k = (int)(r % 4);
  x[0] = k < 2 ? k : b[0] - 4 + k;
}
__device__ __forceinline__ long long xl_shell_count(const int b[3]) {
  return (long long)b[0] * b[1] * b[2] - (long long)(b[0] - 4) * (b[1] - 4) * (b[2] - 4);
}

// Fill patch P's cross-level guard buffer for its current time (block part
// `part` of `parts`: its items are part*blockDim.x + threadIdx.x, step
// parts*blockDim.x).  The buffer is laid out like a slice of a patch of m = n+4
// cells per axis whose first cell is P's cell lo-2: cells x in [-2, n+2),
// faces along an axis at x in [-2, n+2] (relative to lo).
template <typename T>
__device__ void fill_cross_level(const DevCtx &c, int P, int part, int parts) {
  const long long i0 = (long long)part * blockDim.x + threadIdx.x, istep = (long long)parts * blockDim.x;
  const PatchGeo &gp = c.geo[P];
  const int lev = gp.level;
  const int n[3] = {gp.n[0], gp.n[1], gp.n[2]};
  const int m[3] = {n[0] + 4, n[1] + 4, n[2] + 4};
  const double t = c.t_slot[(long long)P * c.ns + c.latest[P]];
  T *const buf = (T *)c.gbuf + c.gofs[P];
  const long long mc3 = (long long)m[0] * m[1] * m[2];
  const long long fofs[3] = {5 * mc3, 5 * mc3 + (long long)(m[0] + 1) * m[1] * m[2],
                             5 * mc3 + (long long)(m[0] + 1) * m[1] * m[2] + (long long)m[0] * (m[1] + 1) * m[2]};
  auto interior = [&](const int x[3]) {
    return x[0] >= 0 && x[0] < n[0] && x[1] >= 0 && x[1] < n[1] && x[2] >= 0 && x[2] < n[2];
  };
  // a face along ax at the low side of patch cell x: P's own, and is it in the buffer?
  auto own_face = [&](int ax, const int x[3]) {
    for (int d = 0; d < 3; d++)
      if (x[d] < 0 || x[d] > n[d] - (d != ax)) return false;
    return true;
  };
  auto face_in_buf = [&](int ax, const int x[3]) {
    for (int d = 0; d < 3; d++)
      if (x[d] < -2 || x[d] > n[d] + 1 + (d == ax)) return false;
    return true;
  };
  auto face_index = [&](int ax, const int x[3]) -> long long {
    const int f0 = m[0] + (ax == 0), f1 = m[1] + (ax == 1);
    return fofs[ax] + ((long long)(x[2] + 2) * f1 + (x[1] + 2)) * f0 + (x[0] + 2);
  };
  if (lev == 0) {
    // restriction: guard cells and faces whose cell is covered by level 1
    // (the guard cells are the 2-deep shell of the (n+4)^3 box)
    const long long ncs = xl_shell_count(m);
    for (long long si = i0; si < ncs; si += istep) {
      int b[3];
      xl_shell(si, m, b);
      const int x[3] = {b[0] - 2, b[1] - 2, b[2] - 2};
      const long long id = ((long long)b[2] * m[1] + b[1]) * m[0] + b[0];
      const int g[3] = {gp.lo[0] + x[0], gp.lo[1] + x[1], gp.lo[2] + x[2]};
      if (!xl_cross(c, 0, g)) continue;
      T u[5];
      const int rc = xl_restrict_cell<T>(c, g, t, u);
      if (rc) {
        xl_status(c, rc, P);
        return;
      }
      for (int q = 0; q < 5; q++) buf[q * mc3 + id] = u[q];
    }
    for (int ax = 0; ax < 3; ax++) {
      // the faces along ax not P's own: the 2-deep shell of the face box
      const int fb[3] = {m[0] + (ax == 0), m[1] + (ax == 1), m[2] + (ax == 2)};
      const long long nfs = xl_shell_count(fb);
      for (long long si = i0; si < nfs; si += istep) {
        int b[3];
        xl_shell(si, fb, b);
        const int x[3] = {b[0] - 2, b[1] - 2, b[2] - 2};
        const long long id = ((long long)b[2] * fb[1] + b[1]) * fb[0] + b[0];
        const int g[3] = {gp.lo[0] + x[0], gp.lo[1] + x[1], gp.lo[2] + x[2]};
        if (!xl_cross(c, 0, g)) continue;
        T v;
        const int rc = xl_restrict_face<T>(c, ax, g, t, &v);
        if (rc) {
          xl_status(c, rc, P);
          return;
        }
        buf[fofs[ax] + id] = v;
      }
    }
    return;
  }
  // prolongation: one thread per level-0 parent of the buffer's cells and
  // faces; the parent's slopes and faces serve all its children
  int c0[3], cn[3];
  for (int d = 0; d < 3; d++) {
    c0[d] = xl_floordiv(gp.lo[d] - 2, 2);
    cn[d] = xl_floordiv(gp.lo[d] + n[d] + 2, 2) - c0[d] + 1;
  }
  const long long npar = (long long)cn[0] * cn[1] * cn[2];
  for (long long id = i0; id < npar; id += istep) {
    const int C[3] = {c0[0] + (int)(id % cn[0]), c0[1] + (int)((id / cn[0]) % cn[1]),
                      c0[2] + (int)(id / ((long long)cn[0] * cn[1]))};
    const int f0[3] = {2 * C[0], 2 * C[1], 2 * C[2]};
    // children in patch coordinates; all 8 share one level-1 block
    const int xb[3] = {f0[0] - gp.lo[0], f0[1] - gp.lo[1], f0[2] - gp.lo[2]};
    bool all_inside = true;
    for (int d = 0; d < 3; d++)
      if (xb[d] < 0 || xb[d] + 1 >= n[d]) all_inside = false;
    if (all_inside || !xl_cross(c, 1, f0)) continue;
    // cells: the parent and its slopes, once
    bool any_cell = false;
    for (int k = 0; k < 8; k++) {
      const int x[3] = {xb[0] + (k & 1), xb[1] + ((k >> 1) & 1), xb[2] + (k >> 2)};
      if (x[0] >= -2 && x[0] < n[0] + 2 && x[1] >= -2 && x[1] < n[1] + 2 && x[2] >= -2 && x[2] < n[2] + 2 &&
          !interior(x))
        any_cell = true;
    }
    int rc = DSP_OK;
    if (any_cell) {
      T uc[5], ul[5], ur[5], sl[3][5];
      rc = xl_cell<T>(c, 0, C, t, uc);
      for (int d = 0; d < 3 && rc == DSP_OK; d++) {
        int Cm[3] = {C[0], C[1], C[2]}, Cp[3] = {C[0], C[1], C[2]};
        Cm[d] -= 1;
        Cp[d] += 1;
        rc = xl_cell<T>(c, 0, Cm, t, ul);
        if (rc == DSP_OK) rc = xl_cell<T>(c, 0, Cp, t, ur);
        if (rc == DSP_OK)
          for (int q = 0; q < 5; q++) sl[d][q] = mc(uc[q] - ul[q], ur[q] - uc[q]);
      }
      if (rc) {
        xl_status(c, rc, P);
        return;
      }
      for (int k = 0; k < 8; k++) {
        const int x[3] = {xb[0] + (k & 1), xb[1] + ((k >> 1) & 1), xb[2] + (k >> 2)};
        if (x[0] < -2 || x[0] >= n[0] + 2 || x[1] < -2 || x[1] >= n[1] + 2 || x[2] < -2 || x[2] >= n[2] + 2 ||
            interior(x))
          continue;
        const long long bi = ((long long)(x[2] + 2) * m[1] + (x[1] + 2)) * m[0] + (x[0] + 2);
        for (int q = 0; q < 5; q++) {
          const T a = (k & 1) ? sl[0][q] : -sl[0][q];
          const T b = ((k >> 1) & 1) ? sl[1][q] : -sl[1][q];
          const T e = (k >> 2) ? sl[2][q] : -sl[2][q];
          buf[q * mc3 + bi] = uc[q] + T(0.25) * ((a + b) + e);
        }
      }
    }
    // faces: the parent's two faces per axis (one owner patch), once
    for (int ax = 0; ax < 3; ax++) {
      bool any_face = false;
      for (int k = 0; k < 8; k++) {
        const int x[3] = {xb[0] + (k & 1), xb[1] + ((k >> 1) & 1), xb[2] + (k >> 2)};
        if (face_in_buf(ax, x) && !own_face(ax, x)) any_face = true;
      }
      if (!any_face) continue;
      T lo, hi;
      rc = xl_face<T>(c, 0, ax, C, 0, t, &lo);
      if (rc == DSP_OK) rc = xl_face<T>(c, 0, ax, C, 1, t, &hi);
      if (rc) {
        xl_status(c, rc, P);
        return;
      }
      for (int k = 0; k < 8; k++) {
        const int kk[3] = {k & 1, (k >> 1) & 1, k >> 2};
        const int x[3] = {xb[0] + kk[0], xb[1] + kk[1], xb[2] + kk[2]};
        if (!face_in_buf(ax, x) || own_face(ax, x)) continue;
        buf[face_index(ax, x)] = kk[ax] ? T(0.5) * (lo + hi) : lo;
      }
    }
  }
}

// XL_PARTS blocks per ready patch that has a cross-level guard buffer.
constexpr int XL_PARTS = 8;
template <typename T>
__global__ void __launch_bounds__(256) xlevel_kernel(DevCtx c) {
  const int nr = c.ctl[CTL_NREADY];
  for (long long w = blockIdx.x; w < (long long)nr * XL_PARTS; w += gridDim.x) {
    const int P = c.R[w / XL_PARTS];
    if (c.gofs[P] < 0) continue;
    fill_cross_level<T>(c, P, (int)(w % XL_PARTS), XL_PARTS);
  }
}

}  // namespace dsp

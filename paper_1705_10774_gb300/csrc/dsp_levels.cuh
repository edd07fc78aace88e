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

// The slices of patch Q that supply time t: a slice at exactly t is copied;
// otherwise the newest two must bracket t and are blended with weight w.
template <typename T>
struct XSrc {
  const T *A, *B;
  T w;
  int Q, loc[3];
};

// Owner on level lev of the (unwrapped) level-lev cell g, its local cell
// index, and the slices for time t.  Returns 0, or an error code.
template <typename T>
__device__ int xl_source(const DevCtx &c, int lev, const int g[3], double t, XSrc<T> &s) {
  int w[3];
  for (int d = 0; d < 3; d++) w[d] = xl_posmod(g[d], c.L[lev][d]);
  const long long b = ((long long)(w[2] / c.bsz[lev][2]) * c.mapd[lev][1] + w[1] / c.bsz[lev][1]) * c.mapd[lev][0] +
                      w[0] / c.bsz[lev][0];
  const int Q = c.omap[lev][b];
  if (Q < 0) return DSP_ERR_INVALID_ARG;
  const PatchGeo &gq = c.geo[Q];
  for (int d = 0; d < 3; d++) s.loc[d] = w[d] - gq.lo[d];
  s.Q = Q;
  const T *base = (const T *)c.slab + gq.off;
  const int ns = c.ns, L = c.latest[Q];
  const double tq = c.t_slot[(long long)Q * ns + L];
  s.B = nullptr;
  s.w = T(0);
  if (tq == t) {
    s.A = base + (long long)L * c.slot_stride;
    return DSP_OK;
  }
  const int Pv = (L + ns - 1) % ns;
  const double ta = c.t_slot[(long long)Q * ns + Pv];
  if (ta == t) {
    s.A = base + (long long)Pv * c.slot_stride;
    return DSP_OK;
  }
  if (ta < t && t < tq) {
    s.A = base + (long long)Pv * c.slot_stride;
    s.B = base + (long long)L * c.slot_stride;
    s.w = (T)((t - ta) / (tq - ta));
    return DSP_OK;
  }
  return DSP_ERR_BRACKET;
}

template <typename T>
__device__ __forceinline__ T xl_val(const XSrc<T> &s, long long idx) {
  T a = s.A[idx];
  if (s.B) a = a + s.w * (s.B[idx] - a);
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

// Level-1 cell f (not owned on level 1) prolonged from its level-0 parent.
template <typename T>
__device__ int xl_prolong_cell(const DevCtx &c, const int f[3], double t, T u[5]) {
  const int C[3] = {xl_floordiv(f[0], 2), xl_floordiv(f[1], 2), xl_floordiv(f[2], 2)};
  T uc[5], ul[5], ur[5], sl[3][5];
  int rc = xl_cell<T>(c, 0, C, t, uc);
  if (rc) return rc;
  for (int d = 0; d < 3; d++) {
    int Cm[3] = {C[0], C[1], C[2]}, Cp[3] = {C[0], C[1], C[2]};
    Cm[d] -= 1;
    Cp[d] += 1;
    if ((rc = xl_cell<T>(c, 0, Cm, t, ul))) return rc;
    if ((rc = xl_cell<T>(c, 0, Cp, t, ur))) return rc;
    for (int q = 0; q < 5; q++) sl[d][q] = mc(uc[q] - ul[q], ur[q] - uc[q]);
  }
  for (int q = 0; q < 5; q++) {
    const T a = (f[0] - 2 * C[0]) ? sl[0][q] : -sl[0][q];
    const T b = (f[1] - 2 * C[1]) ? sl[1][q] : -sl[1][q];
    const T e = (f[2] - 2 * C[2]) ? sl[2][q] : -sl[2][q];
    u[q] = uc[q] + T(0.25) * ((a + b) + e);
  }
  return DSP_OK;
}

// Face along ax on the low side of level-1 cell f, from level 0.
template <typename T>
__device__ int xl_prolong_face(const DevCtx &c, int ax, const int f[3], double t, T *out) {
  const int C[3] = {xl_floordiv(f[0], 2), xl_floordiv(f[1], 2), xl_floordiv(f[2], 2)};
  T lo, hi;
  int rc = xl_face<T>(c, 0, ax, C, 0, t, &lo);
  if (rc) return rc;
  if (f[ax] == 2 * C[ax]) {
    *out = lo;
    return DSP_OK;
  }
  if ((rc = xl_face<T>(c, 0, ax, C, 1, t, &hi))) return rc;
  *out = T(0.5) * (lo + hi);
  return DSP_OK;
}

// Level-0 cell C (covered by level 1) restricted from its 8 children.
template <typename T>
__device__ int xl_restrict_cell(const DevCtx &c, const int C[3], double t, T u[5]) {
  T s[5] = {T(0), T(0), T(0), T(0), T(0)}, v[5];
  for (int kz = 0; kz < 2; kz++)
    for (int ky = 0; ky < 2; ky++)
      for (int kx = 0; kx < 2; kx++) {
        const int f[3] = {2 * C[0] + kx, 2 * C[1] + ky, 2 * C[2] + kz};
        const int rc = xl_cell<T>(c, 1, f, t, v);
        if (rc) return rc;
        for (int q = 0; q < 5; q++) s[q] = s[q] + v[q];
      }
  for (int q = 0; q < 5; q++) u[q] = T(0.125) * s[q];
  return DSP_OK;
}

// Face along ax on the low side of level-0 cell C, the mean of the 4 level-1
// faces on it.
template <typename T>
__device__ int xl_restrict_face(const DevCtx &c, int ax, const int C[3], double t, T *out) {
  T s = T(0), v;
  for (int kz = 0; kz < 2; kz++)
    for (int ky = 0; ky < 2; ky++)
      for (int kx = 0; kx < 2; kx++) {
        const int k3[3] = {kx, ky, kz};
        if (k3[ax]) continue;
        const int f[3] = {2 * C[0] + kx, 2 * C[1] + ky, 2 * C[2] + kz};
        const int rc = xl_face<T>(c, 1, ax, f, 0, t, &v);
        if (rc) return rc;
        s = s + v;
      }
  *out = T(0.25) * s;
  return DSP_OK;
}

// Does the guard gather of a level-lev patch take level-lev cell g from the
// other level?
__device__ __forceinline__ bool xl_cross(const DevCtx &c, int lev, const int g[3]) {
  int b[3];
  for (int d = 0; d < 3; d++) b[d] = xl_posmod(g[d], c.L[lev][d]) / c.bsz[lev][d];
  return c.gmap[lev][((long long)b[2] * c.mapd[lev][1] + b[1]) * c.mapd[lev][0] + b[0]] < 0;
}

// Fill patch P's cross-level guard buffer for its current time (all threads
// of the block).  The buffer is laid out like a slice of a patch of m = n+4
// cells per axis whose first cell is P's cell lo-2.
template <typename T>
__device__ void fill_cross_level(const DevCtx &c, int P) {
  const PatchGeo &gp = c.geo[P];
  const int lev = gp.level;
  const int n[3] = {gp.n[0], gp.n[1], gp.n[2]};
  const int m[3] = {n[0] + 4, n[1] + 4, n[2] + 4};
  const double t = c.t_slot[(long long)P * c.ns + c.latest[P]];
  T *const buf = (T *)c.gbuf + c.gofs[P];
  const long long mc3 = (long long)m[0] * m[1] * m[2];
  for (long long id = threadIdx.x; id < mc3; id += blockDim.x) {
    const int x = (int)(id % m[0]) - 2, y = (int)((id / m[0]) % m[1]) - 2, z = (int)(id / ((long long)m[0] * m[1])) - 2;
    if (x >= 0 && x < n[0] && y >= 0 && y < n[1] && z >= 0 && z < n[2]) continue;
    const int g[3] = {gp.lo[0] + x, gp.lo[1] + y, gp.lo[2] + z};
    if (!xl_cross(c, lev, g)) continue;
    T u[5];
    const int rc = lev == 1 ? xl_prolong_cell<T>(c, g, t, u) : xl_restrict_cell<T>(c, g, t, u);
    if (rc) {
      xl_status(c, rc, P);
      return;
    }
    for (int q = 0; q < 5; q++) buf[q * mc3 + id] = u[q];
  }
  long long base = 5 * mc3;
  for (int ax = 0; ax < 3; ax++) {
    const int f0 = m[0] + (ax == 0), f1 = m[1] + (ax == 1), f2 = m[2] + (ax == 2);
    const long long nf = (long long)f0 * f1 * f2;
    for (long long id = threadIdx.x; id < nf; id += blockDim.x) {
      const int x = (int)(id % f0) - 2, y = (int)((id / f0) % f1) - 2, z = (int)(id / ((long long)f0 * f1)) - 2;
      // P's own faces: every face of its interior cells
      const int xy[3] = {x, y, z};
      bool own = true;
      for (int d = 0; d < 3; d++)
        if (xy[d] < 0 || xy[d] > n[d] - (d != ax)) own = false;
      if (own) continue;
      const int g[3] = {gp.lo[0] + x, gp.lo[1] + y, gp.lo[2] + z};
      if (!xl_cross(c, lev, g)) continue;
      T v;
      const int rc = lev == 1 ? xl_prolong_face<T>(c, ax, g, t, &v) : xl_restrict_face<T>(c, ax, g, t, &v);
      if (rc) {
        xl_status(c, rc, P);
        return;
      }
      buf[base + id] = v;
    }
    base += nf;
  }
}

// One block per ready patch that has a cross-level guard buffer.
template <typename T>
__global__ void __launch_bounds__(256) xlevel_kernel(DevCtx c) {
  const int nr = c.ctl[CTL_NREADY];
  for (int r = blockIdx.x; r < nr; r += gridDim.x) {
    const int P = c.R[r];
    if (c.gofs[P] < 0) continue;
    fill_cross_level<T>(c, P);
  }
}

}  // namespace dsp

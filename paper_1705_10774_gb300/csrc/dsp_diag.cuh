// dsp_diag.cuh -- the diagnostics reduction shared by dsp_diagnostics and
// dsp_diagnostics_noalloc: per-patch FP64 Neumaier-compensated volume
// integrals of rho, m, E and of the face fields (the low face of every cell,
// so each face of a periodic tiling counts once), max |sum_d Delta_d b| over
// cells and max |b| over those faces; then the patches combined in patch
// order.  Both orders are fixed, so the result is deterministic.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

namespace dsp {

constexpr int DIAG_NT = 256;  // threads of a per-patch diagnostics block
constexpr int DIAG_PER = 10;  // values per patch: 8 integrals, max |div b|, max |b|

struct NSum {
  double s, c;
};
__host__ __device__ __forceinline__ void nadd(NSum &a, double x) {
  const double t = a.s + x;
  if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x;
  else a.c += (x - t) + a.s;
  a.s = t;
}

// One block of DIAG_NT threads reduces one patch: interior U[5][nz][ny][nx],
// faces bx[nz][ny][nx+1], by[nz][ny+1][nx], bz[nz+1][ny][nx], cell volume dV.
// Thread-strided compensated sums, then thread 0 combines the threads'
// partials in thread order and writes DIAG_PER values to out.
template <typename T>
__device__ void diag_patch(const T *u, const T *fx, const T *fy, const T *fz, int nx, int ny, int nz, double dV,
                           double *out) {
  const long long nc = (long long)nx * ny * nz;
  NSum acc[8];
  for (int q = 0; q < 8; q++) acc[q].s = acc[q].c = 0.0;
  double mdiv = 0.0, mb = 0.0;
  for (long long id = threadIdx.x; id < nc; id += blockDim.x) {
    const int i = (int)(id % nx), j = (int)((id / nx) % ny), k = (int)(id / ((long long)nx * ny));
    for (int q = 0; q < 5; q++) nadd(acc[q], (double)u[q * nc + id] * dV);
    const double bxl = fx[((long long)k * ny + j) * (nx + 1) + i], bxr = fx[((long long)k * ny + j) * (nx + 1) + i + 1];
    const double byl = fy[((long long)k * (ny + 1) + j) * nx + i], byr = fy[((long long)k * (ny + 1) + j + 1) * nx + i];
    const double bzl = fz[((long long)k * ny + j) * nx + i], bzr = fz[((long long)(k + 1) * ny + j) * nx + i];
    nadd(acc[5], bxl * dV);
    nadd(acc[6], byl * dV);
    nadd(acc[7], bzl * dV);
    mdiv = fmax(mdiv, fabs((bxr - bxl) + (byr - byl) + (bzr - bzl)));
    mb = fmax(mb, fmax(fabs(bxl), fmax(fabs(byl), fabs(bzl))));
  }
  __shared__ double sh[DIAG_NT][18];
  for (int q = 0; q < 8; q++) {
    sh[threadIdx.x][2 * q] = acc[q].s;
    sh[threadIdx.x][2 * q + 1] = acc[q].c;
  }
  sh[threadIdx.x][16] = mdiv;
  sh[threadIdx.x][17] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    NSum tot[8];
    for (int q = 0; q < 8; q++) tot[q].s = tot[q].c = 0.0;
    double md = 0.0, mm = 0.0;
    for (int t = 0; t < (int)blockDim.x; t++) {
      for (int q = 0; q < 8; q++) {
        nadd(tot[q], sh[t][2 * q]);
        nadd(tot[q], sh[t][2 * q + 1]);
      }
      md = fmax(md, sh[t][16]);
      mm = fmax(mm, sh[t][17]);
    }
    for (int q = 0; q < 8; q++) out[q] = tot[q].s + tot[q].c;
    out[8] = md;
    out[9] = mm;
  }
}

// The patches' DIAG_PER values combined in patch order (compensated sums of
// the integrals, maxima of the rest) into out[DIAG_PER].
__host__ __device__ inline void diag_combine(const double *part, int np, double *out) {
  NSum s[8];
  for (int q = 0; q < 8; q++) s[q].s = s[q].c = 0.0;
  double md = 0.0, mb = 0.0;
  for (int P = 0; P < np; P++) {
    for (int q = 0; q < 8; q++) nadd(s[q], part[(long long)P * DIAG_PER + q]);
    md = fmax(md, part[(long long)P * DIAG_PER + 8]);
    mb = fmax(mb, part[(long long)P * DIAG_PER + 9]);
  }
  for (int q = 0; q < 8; q++) out[q] = s[q].s + s[q].c;
  out[8] = md;
  out[9] = mb;
}

}  // namespace dsp

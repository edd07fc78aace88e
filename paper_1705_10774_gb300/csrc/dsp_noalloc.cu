// dsp_noalloc.cu -- dsp_diagnostics_noalloc: the diagnostics reduction over
// a state held in caller-owned device arrays, using no device allocation.
//
// The per-patch partial results live in one file-scope __device__ array of
// fixed size (DSP_NOALLOC_MAX_PATCHES patches).  Every GPU that loads this
// library holds that array (about 1.3 MB) until the process exits.  Host
// code must not pass the array's name to a kernel: on the host it is only a
// stand-in symbol, so its device address is looked up once per device with
// cudaGetSymbolAddress and cached.  All calls share the array: two calls
// whose kernels overlap on a GPU (different streams, or different host
// threads on the same device) overwrite each other's partial results.
#include <cuda_runtime.h>

#include <mutex>

#include "dsp_internal.h"

namespace {

constexpr int kMax = DSP_NOALLOC_MAX_PATCHES;
constexpr int kPer = 10;  // per patch: 8 compensated sums, max |div b|, max |b|

static __device__ __align__(256) double g_noalloc_scratch[kMax * kPer + kPer];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_addr[kMaxDevices];

// Device address of the scratch array on the current device.  The first call
// on a device looks it up (that device must be current); later calls reuse it.
int scratch_address(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return DSP_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return DSP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DSP_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return DSP_OK;
}

struct NSum {
  double s, c;
};
__device__ __forceinline__ void nadd(NSum &a, double x) {
  const double t = a.s + x;
  if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x;
  else a.c += (x - t) + a.s;
  a.s = t;
}

// One block per patch: compensated sums of the patch's cells in a fixed
// order (thread-strided, then thread 0 over the threads' partials).  Every
// element of the patch's slot in `part` is written, nothing is read first.
template <typename T>
__global__ void noalloc_patch_kernel(const T *U, const T *bx, const T *by, const T *bz, int nx, int ny, int nz,
                                     double dx, double *part) {
  const int P = blockIdx.x;
  const long long nc = (long long)nx * ny * nz;
  const long long nfx = (long long)(nx + 1) * ny * nz, nfy = (long long)nx * (ny + 1) * nz,
                  nfz = (long long)nx * ny * (nz + 1);
  const T *u = U + (long long)P * 5 * nc;
  const T *fx = bx + (long long)P * nfx, *fy = by + (long long)P * nfy, *fz = bz + (long long)P * nfz;
  const double dV = dx * dx * dx;
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
  __shared__ double sh[256][18];
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
    for (int q = 0; q < 8; q++) part[(long long)P * kPer + q] = tot[q].s + tot[q].c;
    part[(long long)P * kPer + 8] = md;
    part[(long long)P * kPer + 9] = mm;
  }
}

// One thread combines the patches in patch order (compensated) into the ten
// values after the per-patch block of the scratch array.
__global__ void noalloc_final_kernel(const double *part, int np, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[8], c[8];
  for (int q = 0; q < 8; q++) s[q] = c[q] = 0.0;
  double md = 0.0, mb = 0.0;
  for (int P = 0; P < np; P++) {
    for (int q = 0; q < 8; q++) {
      const double x = part[(long long)P * kPer + q];
      const double t = s[q] + x;
      if (fabs(s[q]) >= fabs(x)) c[q] += (s[q] - t) + x;
      else c[q] += (x - t) + s[q];
      s[q] = t;
    }
    md = fmax(md, part[(long long)P * kPer + 8]);
    mb = fmax(mb, part[(long long)P * kPer + 9]);
  }
  for (int q = 0; q < 8; q++) out[q] = s[q] + c[q];
  out[8] = md;
  out[9] = mb;
}

}  // namespace

extern "C" int dsp_diagnostics_noalloc(const void *U, const void *bx, const void *by, const void *bz, int32_t dtype,
                                       int32_t npatch, const int32_t *n, double dx, void *stream, dsp_diag *out) {
  if (!U || !bx || !by || !bz || !n || !out || (dtype != 0 && dtype != 1) || !(dx > 0.0))
    return DSP_ERR_INVALID_ARG;
  if (npatch < 1 || npatch > kMax) return DSP_ERR_INVALID_ARG;
  if (n[0] < 1 || n[1] < 1 || n[2] < 1) return DSP_ERR_INVALID_ARG;
  double *scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == 0)
    noalloc_patch_kernel<double><<<npatch, 256, 0, s>>>((const double *)U, (const double *)bx, (const double *)by,
                                                        (const double *)bz, n[0], n[1], n[2], dx, scratch);
  else
    noalloc_patch_kernel<float><<<npatch, 256, 0, s>>>((const float *)U, (const float *)bx, (const float *)by,
                                                       (const float *)bz, n[0], n[1], n[2], dx, scratch);
  if (cudaGetLastError() != cudaSuccess) return DSP_ERR_CUDA;
  double *result = scratch + (long long)kMax * kPer;
  noalloc_final_kernel<<<1, 32, 0, s>>>(scratch, npatch, result);
  if (cudaGetLastError() != cudaSuccess) return DSP_ERR_CUDA;
  double h[kPer];
  if (cudaMemcpyAsync(h, result, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess) return DSP_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DSP_ERR_CUDA;
  out->mass = h[0];
  for (int d = 0; d < 3; d++) out->mom[d] = h[1 + d];
  out->energy = h[4];
  for (int d = 0; d < 3; d++) out->bmean[d] = h[5 + d];
  out->max_divb = h[8];
  out->max_b = h[9];
  return DSP_OK;
}

// dsp_noalloc.cu -- dsp_diagnostics_noalloc: the diagnostics reduction over
// a state held in caller-owned device arrays, using no device allocation.
//
// The per-patch partial results live in one file-scope __device__ array of
// fixed size (DSP_NOALLOC_MAX_PATCHES patches).  Every GPU that loads this
// library holds that array (about 1.3 MB) until the process exits.  Host
// code must not pass the array's name to a kernel: on the host it is only a
// stand-in symbol, so its device address is looked up once per device with
// cudaGetSymbolAddress and cached for the life of the process (so the
// library must not be used on a device after cudaDeviceReset, which would
// leave the cached address stale).  All calls share the array: two calls
// whose kernels overlap on a GPU (different streams, or different host
// threads on the same device) overwrite each other's partial results.
#include <cuda_runtime.h>

#include <mutex>

#include "dsp_diag.cuh"
#include "dsp_internal.h"

using namespace dsp;

namespace {

constexpr int kMax = DSP_NOALLOC_MAX_PATCHES;
constexpr int kPer = DIAG_PER;  // per patch: 8 compensated sums, max |div b|, max |b|

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

// One block per patch (all patches of n[0] x n[1] x n[2] cells, cell size
// dx): the per-patch reduction of dsp_diagnostics.  Every element of the
// patch's slot in `part` is written, nothing is read first.
template <typename T>
__global__ void __launch_bounds__(DIAG_NT) noalloc_patch_kernel(const T *U, const T *bx, const T *by, const T *bz,
                                                                int nx, int ny, int nz, double dx, double *part) {
  const int P = blockIdx.x;
  const long long nc = (long long)nx * ny * nz;
  const long long nfx = (long long)(nx + 1) * ny * nz, nfy = (long long)nx * (ny + 1) * nz,
                  nfz = (long long)nx * ny * (nz + 1);
  diag_patch<T>(U + (long long)P * 5 * nc, bx + (long long)P * nfx, by + (long long)P * nfy, bz + (long long)P * nfz,
                nx, ny, nz, dx * dx * dx, part + (long long)P * kPer);
}

// One thread combines the patches in patch order into the ten values after
// the per-patch block of the scratch array.
__global__ void noalloc_final_kernel(const double *part, int np, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) diag_combine(part, np, out);
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
    noalloc_patch_kernel<double><<<npatch, DIAG_NT, 0, s>>>((const double *)U, (const double *)bx, (const double *)by,
                                                        (const double *)bz, n[0], n[1], n[2], dx, scratch);
  else
    noalloc_patch_kernel<float><<<npatch, DIAG_NT, 0, s>>>((const float *)U, (const float *)bx, (const float *)by,
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

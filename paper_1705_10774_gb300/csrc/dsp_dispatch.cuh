// dsp_dispatch.cuh -- device-side dispatcher pieces shared by the sweep
// kernels and the persistent ready-queue kernel: memory-ordering helpers, the
// readiness test of Eq. (1) with grace 0, and the local Courant step.
#pragma once
#include <cuda_runtime.h>

#include "dsp_internal.h"

namespace dsp {

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Reads of another patch's newest-slice index, slice times and signal speeds.
// With CONC (several blocks publish concurrently) the index is read with
// acquire semantics and the values it guards bypass L1.
template <bool CONC>
__device__ __forceinline__ int newest(const DevCtx &c, int P) {
  return CONC ? ld_acquire(c.latest + P) : c.latest[P];
}
template <bool CONC>
__device__ __forceinline__ double slot_time(const DevCtx &c, long long i) {
  return CONC ? __ldcg(c.t_slot + i) : c.t_slot[i];
}
template <bool CONC>
__device__ __forceinline__ double slot_smax(const DevCtx &c, long long i) {
  return CONC ? __ldcg(c.smax_slot + i) : c.smax_slot[i];
}

// Local Courant step of patch P at time t (all FP64): the signal speed is the
// largest over P's newest slice and every neighbour slice its guard fill
// reads; the step is the power of two not above C dx / s (dx of P's level),
// capped by dt_max,
// halved until it divides t, and clipped to t_end.
template <bool CONC>
__device__ int patch_dt(const DevCtx &c, int P, double t, double t_end, double *out) {
  const int ns = c.ns;
  double M = slot_smax<CONC>(c, (long long)P * ns + newest<CONC>(c, P));
  for (int k = c.nbl_off[P]; k < c.nbl_off[P + 1]; k++) {
    const int N = c.nbl[k];
    const int L = newest<CONC>(c, N);
    const double tq = slot_time<CONC>(c, (long long)N * ns + L);
    if (tq == t) {
      M = fmax(M, slot_smax<CONC>(c, (long long)N * ns + L));
    } else {
      const int Pv = (L + ns - 1) % ns;
      const double ta = slot_time<CONC>(c, (long long)N * ns + Pv);
      if (ta == t) {
        M = fmax(M, slot_smax<CONC>(c, (long long)N * ns + Pv));
      } else if (ta < t && t < tq) {
        M = fmax(M, slot_smax<CONC>(c, (long long)N * ns + Pv));
        M = fmax(M, slot_smax<CONC>(c, (long long)N * ns + L));
      } else {
        return DSP_ERR_BRACKET;
      }
    }
  }
  const double dtc = c.cfl * ldexp(c.dx, -c.geo[P].level) / M;
  int e;
  frexp(dtc, &e);
  double dt = ldexp(1.0, e - 1);
  if (c.dt_max > 0.0 && dt > c.dt_max) dt = c.dt_max;
  int guard = 0;
  while (fmod(t, dt) != 0.0) {
    dt = dt * 0.5;
    if (++guard > 1200 || !(dt > 0.0)) return DSP_ERR_INVALID_ARG;
  }
  if (dt > t_end - t) dt = t_end - t;
  *out = dt;
  return DSP_OK;
}

// Eq. (1) with grace 0: P is ready when t_P < t_end and t_P <= t_N for every
// neighbour N.  Writes t_P.
template <bool CONC>
__device__ __forceinline__ bool is_ready(const DevCtx &c, int P, double t_end, double *tP) {
  const int ns = c.ns;
  const double t = slot_time<CONC>(c, (long long)P * ns + newest<CONC>(c, P));
  *tP = t;
  if (!(t < t_end)) return false;
  for (int k = c.nbl_off[P]; k < c.nbl_off[P + 1]; k++) {
    const int N = c.nbl[k];
    if (!(t <= slot_time<CONC>(c, (long long)N * ns + newest<CONC>(c, N)))) return false;
  }
  return true;
}

}  // namespace dsp

// dsp_dispatch.cuh -- device-side dispatcher pieces shared by the sweep
// kernels and the persistent ready-queue kernel: memory-ordering helpers, the
// choice of stored slices that supply a time, the readiness test of Eq. (1)
// with grace g, and the local Courant step.
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

// The stored slices of patch Q that supply time t (DISPATCH I, Sec. 3 A and
// B), older first, with their weights: n = 1, the slice at exactly t
// (copied); n = 2, linear inter- or extrapolation A + w0 (B - A) with
// w0 = (t - t_A)/(t_B - t_A); n = 3, quadratic (Lagrange) inter- or
// extrapolation (w0 A + w1 B) + w2 C.  Stored slices, newest first, have
// strictly decreasing times (the scan stops at an empty or out-of-order
// slot).  Past the newest slice (allowed by the grace of Eq. 1) the newest
// two (three) are extrapolated; otherwise the two slices around t are
// interpolated, the quadratic form adding the next older slice, or the next
// newer one where there is no older one, and staying linear with two.
struct SlicePick {
  int n;
  int s[3];
  double w[3];
};

template <bool CONC>
__device__ __forceinline__ int pick_slices(const DevCtx &c, int Q, double t, SlicePick &pk) {
  const int ns = c.ns, L = newest<CONC>(c, Q);
  auto slot = [&](int k) { return (L - k + ns) % ns; };
  auto tk = [&](int k) { return slot_time<CONC>(c, (long long)Q * ns + slot(k)); };
  int cnt = 1;
  for (double prev = tk(0); cnt < ns; cnt++) {
    const double tt = tk(cnt);
    if (!(tt < prev)) break;  // empty (NaN) or not older
    prev = tt;
  }
  for (int k = 0; k < cnt; k++)
    if (tk(k) == t) {
      pk.n = 1;
      pk.s[0] = slot(k);
      pk.w[0] = 1.0;
      return DSP_OK;
    }
  int ka, kb, kc = -1;
  if (t > tk(0)) {
    if (cnt < 2) return DSP_ERR_BRACKET;
    ka = 1;
    kb = 0;
    if (c.torder == 2 && cnt >= 3) { ka = 2; kb = 1; kc = 0; }
  } else {
    int k = 1;
    while (k < cnt && !(tk(k) < t)) k++;
    if (k >= cnt) return DSP_ERR_BRACKET;
    ka = k;
    kb = k - 1;
    if (c.torder == 2) {
      if (k + 1 < cnt) { kc = k - 1; kb = k; ka = k + 1; }
      else if (k - 2 >= 0) kc = k - 2;
    }
  }
  const double ta = tk(ka), tb = tk(kb);
  if (kc < 0) {
    pk.n = 2;
    pk.s[0] = slot(ka);
    pk.s[1] = slot(kb);
    pk.w[0] = (t - ta) / (tb - ta);
    return DSP_OK;
  }
  const double tc = tk(kc);
  pk.n = 3;
  pk.s[0] = slot(ka);
  pk.s[1] = slot(kb);
  pk.s[2] = slot(kc);
  pk.w[0] = ((t - tb) * (t - tc)) / ((ta - tb) * (ta - tc));
  pk.w[1] = ((t - ta) * (t - tc)) / ((tb - ta) * (tb - tc));
  pk.w[2] = ((t - ta) * (t - tb)) / ((tc - ta) * (tc - tb));
  return DSP_OK;
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
    SlicePick pk;
    if (pick_slices<CONC>(c, N, t, pk) != DSP_OK) return DSP_ERR_BRACKET;
    for (int q = 0; q < pk.n; q++) M = fmax(M, slot_smax<CONC>(c, (long long)N * ns + pk.s[q]));
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

// May P overwrite its oldest slice?  Not while a neighbour that may be
// updated before P's next slice exists (its time at most P's time plus g
// times P's last step) still takes values from that slice.  With g = 0 this
// never binds, so it is only asked with g > 0.  An empty slot is free.
template <bool CONC>
__device__ bool slot_free(const DevCtx &c, int P) {
  const int ns = c.ns, L = newest<CONC>(c, P), oldest = (L + 1) % ns;
  const double to = slot_time<CONC>(c, (long long)P * ns + oldest);
  if (to != to) return true;
  const double lim = slot_time<CONC>(c, (long long)P * ns + L) + c.grace * c.dt_last[P];
  for (int k = c.nbl_off[P]; k < c.nbl_off[P + 1]; k++) {
    const int N = c.nbl[k];
    const double tq = slot_time<CONC>(c, (long long)N * ns + newest<CONC>(c, N));
    if (!(tq <= lim)) continue;
    SlicePick pk;
    if (pick_slices<CONC>(c, P, tq, pk) != DSP_OK) continue;
    for (int q = 0; q < pk.n; q++)
      if (pk.s[q] == oldest) return false;
  }
  return true;
}

// Eq. (1): P is ready when t_P < t_end and t_P <= t_N + g dt_N for every
// neighbour N (dt_N its last step, 0 before the first), and, with g > 0,
// its oldest slice is free.  Writes t_P.
template <bool CONC>
__device__ __forceinline__ bool is_ready(const DevCtx &c, int P, double t_end, double *tP) {
  const int ns = c.ns;
  const double t = slot_time<CONC>(c, (long long)P * ns + newest<CONC>(c, P));
  *tP = t;
  if (!(t < t_end)) return false;
  for (int k = c.nbl_off[P]; k < c.nbl_off[P + 1]; k++) {
    const int N = c.nbl[k];
    if (!(t <= slot_time<CONC>(c, (long long)N * ns + newest<CONC>(c, N)) + c.grace * c.dt_last[N])) return false;
  }
  if (c.grace > 0.0 && !slot_free<CONC>(c, P)) return false;
  return true;
}

}  // namespace dsp

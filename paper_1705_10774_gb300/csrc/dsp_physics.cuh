// dsp_physics.cuh -- cell- and face-level arithmetic of the MHD step.
//
// Every expression has a fixed evaluation order; the FP64 translation units
// are compiled with -fmad=false so that each result is a pure function of its
// inputs (IEEE division and square root, no contraction).  Heaviside-Lorentz
// units: E = -v x B, total energy E = p/(gamma-1) + rho v^2/2 + B^2/2.
#pragma once
#include <cuda_runtime.h>

namespace dsp {

enum { RHO = 0, VX = 1, VY = 2, VZ = 3, PR = 4, BX = 5, BY = 6, BZ = 7 };

// Pressure floor of the primitive recovery, p >= PFLOOR * rho (a sound-speed
// floor of 1e-10), as in RAMSES-type solvers; the conserved energy is never
// modified.
constexpr double PFLOOR = 1e-20;

template <typename T> __device__ __forceinline__ T tmin(T a, T b);
template <typename T> __device__ __forceinline__ T tmax(T a, T b);
template <> __device__ __forceinline__ double tmin<double>(double a, double b) { return fmin(a, b); }
template <> __device__ __forceinline__ double tmax<double>(double a, double b) { return fmax(a, b); }
template <> __device__ __forceinline__ float tmin<float>(float a, float b) { return fminf(a, b); }
template <> __device__ __forceinline__ float tmax<float>(float a, float b) { return fmaxf(a, b); }
// Sign-bit and ordering tests on the bit patterns of floating-point values,
// done with integer instructions: on GB300 every FP64 compare, min or max
// takes a slot of the (narrow) FP64 pipe, while these run on the integer
// units.  Each gives exactly the result of the floating-point form it
// replaces, for every input stated beside it.
template <typename T>
struct FBits;
template <>
struct FBits<double> {
  using I = long long;
  static __device__ __forceinline__ I of(double x) { return __double_as_longlong(x); }
  static __device__ __forceinline__ double to(I i) { return __longlong_as_double(i); }
  static constexpr I MAG = 0x7fffffffffffffffll, INF = 0x7ff0000000000000ll;
};
template <>
struct FBits<float> {
  using I = int;
  static __device__ __forceinline__ I of(float x) { return __float_as_int(x); }
  static __device__ __forceinline__ float to(I i) { return __int_as_float(i); }
  static constexpr I MAG = 0x7fffffff, INF = 0x7f800000;
};
// |a| (as fabs: the sign bit cleared, for every input); in FP32 the native
// form, which the FP32 pipe folds into the operation that uses it
template <typename T>
__device__ __forceinline__ T tabs(T a) {
  if constexpr (sizeof(T) == 4) {
    return fabsf(a);
  } else {
    using B = FBits<T>;
    return B::to(B::of(a) & B::MAG);
  }
}
// a > 0 (for every input, NaN included)
template <typename T>
__device__ __forceinline__ bool tpos(T a) {
  using B = FBits<T>;
  const typename B::I i = B::of(a);
  return i > 0 && i <= B::INF;
}
// a < 0 (for every input, NaN included)
template <typename T>
__device__ __forceinline__ bool tneg(T a) {
  using B = FBits<T>;
  const typename B::I i = B::of(a), m = i & B::MAG;
  return i < 0 && m != 0 && m <= B::INF;
}
// min(a, b) for a, b >= +0 or NaN (as fmin: a NaN operand yields the other)
template <typename T>
__device__ __forceinline__ T tmin_nonneg(T a, T b) {
  using B = FBits<T>;
  return B::of(a) <= B::of(b) ? a : b;
}
// Evaluation order of the update's arithmetic.  kFast = false: the FP64
// oracle's order, operation for operation (the FMA-free FP64 build).  kFast =
// true in the builds held to a tolerance rather than bit equality; every
// kFast form below applies to FP64 only (the FP64 build with fused
// multiply-adds), where the FP64 pipe is the kernel's bottleneck and the
// integer units are idle: FP64 comparisons, minima, maxima and power-of-two
// scalings as integer operations on the bit patterns, one division per edge
// EMF instead of three, reciprocals and square roots by Newton steps from the
// hardware approximations.  The FP32 build keeps the plain forms.  Each
// translation unit of an update-kernel variant defines DSP_FAST_ORDER from
// its precision.
#ifndef DSP_FAST_ORDER
#define DSP_FAST_ORDER 0
#endif
constexpr bool kFast = DSP_FAST_ORDER != 0;

// Ordered integer key of an FP64 value: keys compare as the values do, for
// every non-NaN input (-0 orders just below +0).
__device__ __forceinline__ long long okey(double a) {
  const long long i = __double_as_longlong(a);
  return i ^ ((i >> 63) & 0x7fffffffffffffffll);
}
// min / max of two values (FP64 through ordered keys under kFast)
template <typename T>
__device__ __forceinline__ T fmin_k(T a, T b) {
  if constexpr (kFast && sizeof(T) == 8) return okey(a) <= okey(b) ? a : b;
  else return tmin(a, b);
}
template <typename T>
__device__ __forceinline__ T fmax_k(T a, T b) {
  if constexpr (kFast && sizeof(T) == 8) return okey(a) >= okey(b) ? a : b;
  else return tmax(a, b);
}
// max(0, a, b): a negative value's bit pattern is a negative integer, a
// positive value's orders as the value does
template <typename T>
__device__ __forceinline__ T pmax0(T a, T b) {
  if constexpr (kFast && sizeof(T) == 8) {
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    return __longlong_as_double(max(max(ia, 0ll), ib));
  } else {
    return tmax(T(0), tmax(a, b));
  }
}
// max(0, -a, -b)
template <typename T>
__device__ __forceinline__ T nmax0(T a, T b) {
  if constexpr (kFast && sizeof(T) == 8) {
    const long long s = (long long)0x8000000000000000ull;
    const long long ia = __double_as_longlong(a) ^ s, ib = __double_as_longlong(b) ^ s;
    return __longlong_as_double(max(max(ia, 0ll), ib));
  } else {
    return tmax(T(0), tmax(-a, -b));
  }
}
// a >= 0 and a <= 0 (non-NaN a)
template <typename T>
__device__ __forceinline__ bool ge0(T a) {
  if constexpr (kFast && sizeof(T) == 8) {
    const long long i = __double_as_longlong(a);
    return i >= 0 || i == (long long)0x8000000000000000ull;
  } else {
    return a >= T(0);
  }
}
template <typename T>
__device__ __forceinline__ bool le0(T a) {
  if constexpr (kFast && sizeof(T) == 8) return __double_as_longlong(a) <= 0;
  else return a <= T(0);
}

__device__ __forceinline__ double tsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float tsqrt(float a) { return sqrtf(a); }

// 1/x and sqrt(x) under kFast in FP64: the hardware approximations
// (rcp.approx / rsqrt.approx, relative error about 1e-6) refined by two
// Newton-Raphson steps, r <- r + r (1 - x r) and s <- s + (y/2)(x - s^2)
// with y ~ 1/sqrt(x), which square the error twice (below 3e-16 relative,
// measured against IEEE division and sqrt) in about 3.8 and 6.7 FP64-pipe
// slots instead of the IEEE forms' 4.6 and 7.6.  Normal positive x (a
// density, a sum of speeds squared); sqrt(0) = 0.  Elsewhere, and in FP32
// (whose build divides and takes roots approximately already), the plain
// operators.
template <typename T>
__device__ __forceinline__ T rcp_k(T x) {
  if constexpr (kFast && sizeof(T) == 8) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"((double)x));
    double e = fma(-(double)x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-(double)x, r, 1.0);
    return fma(r, e, r);
  } else {
    return T(1) / x;
  }
}
template <typename T>
__device__ __forceinline__ T sqrt_k(T x) {
  if constexpr (kFast && sizeof(T) == 8) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"((double)x));
    double s = (double)x * y;
    const double h = 0.5 * y;
    s = fma(h, fma(-s, s, (double)x), s);
    s = fma(h, fma(-s, s, (double)x), s);
    // x == +-0 tested on the bit pattern (an FP64 compare takes an FP64-pipe slot)
    return (__double_as_longlong((double)x) << 1) == 0 ? T(0) : s;
  } else {
    return tsqrt(x);
  }
}

// Primitive state (rho, v, p, B) from conserved (rho, m, E) and the six faces.
// With `floored`, *floored tells whether the pressure floor was taken.
template <typename T>
__device__ __forceinline__ void prim(T rho, T mx, T my, T mz, T E, T bxl, T bxr, T byl, T byr, T bzl, T bzr,
                                     T gamma, T W[8], int *floored = nullptr) {
  T irho = rcp_k(rho);
  const T h = T(0.5);
  T Bx = h * (bxl + bxr);
  T By = h * (byl + byr);
  T Bz = h * (bzl + bzr);
  T vx = mx * irho;
  T vy = my * irho;
  T vz = mz * irho;
  T ke = h * rho * (vx * vx + vy * vy + vz * vz);
  T me = h * (Bx * Bx + By * By + Bz * Bz);
  T p = (gamma - T(1)) * (E - ke - me);
  const T pf = T(PFLOOR) * rho;
  if constexpr (kFast && sizeof(T) == 8) {
    // pf > 0: p's bit pattern orders below pf's exactly when p < pf
    const bool fl = __double_as_longlong(p) < __double_as_longlong(pf);
    if (floored) *floored = fl;
    p = fl ? pf : p;
  } else {
    if (floored) *floored = p < pf;
    p = tmax(p, pf);
  }
  W[RHO] = rho; W[VX] = vx; W[VY] = vy; W[VZ] = vz; W[PR] = p;
  W[BX] = Bx; W[BY] = By; W[BZ] = Bz;
}

// Fast magnetosonic speed along the axis whose field component is bn
// (irho = 1/rho).
template <typename T>
__device__ __forceinline__ T cfast(T gamma, T irho, T p, T bn, T bt1, T bt2) {
  T a2 = gamma * p * irho;
  T bb = (bn * bn + bt1 * bt1 + bt2 * bt2) * irho;
  T ca2 = bn * bn * irho;
  T s = a2 + bb;
  T disc = s * s - T(4) * a2 * ca2;
  if (tneg(disc)) disc = T(0);
  return sqrt_k(T(0.5) * (s + sqrt_k(disc)));
}

// The non-ideal step limits of DISPATCH I, Sec. 4.3, as a signal speed s of
// a cell state W, so that cfl dx / s is the limit: C_Ohm dx^2 / eta (Eq. 4)
// for s = cfl eta / (C_Ohm dx), and C_AD gamma_AD rho_i rho dx^2 / B^2 (Eq. 8)
// for s = cfl B^2 / (C_AD gamma_AD rho_i rho dx); the larger of the terms
// that are on (eta > 0, gad > 0), else 0.
template <typename T>
__device__ __forceinline__ T nonideal_speed(const T W[8], double cfl, double eta, double gad, double rhoi, double cohm,
                                            double cad, double dxl) {
  T sp = T(0);
  if (eta > 0.0) sp = (T)cfl * (T)eta / ((T)cohm * (T)dxl);
  if (gad > 0.0) {
    const T B2 = W[BX] * W[BX] + W[BY] * W[BY] + W[BZ] * W[BZ];
    sp = tmax(sp, (T)cfl * B2 / (((((T)cad * (T)gad) * (T)rhoi) * W[RHO]) * (T)dxl));
  }
  return sp;
}

// Sum over axes of |v_d| + c_f,d: the signal speed that sets the Courant step.
template <typename T>
__device__ __forceinline__ T signal_sum(const T W[8], T gamma) {
  T ir = rcp_k(W[RHO]);
  T cx = cfast(gamma, ir, W[PR], W[BX], W[BY], W[BZ]);
  T cy = cfast(gamma, ir, W[PR], W[BY], W[BZ], W[BX]);
  T cz = cfast(gamma, ir, W[PR], W[BZ], W[BX], W[BY]);
  return (tabs(W[VX]) + cx) + (tabs(W[VY]) + cy) + (tabs(W[VZ]) + cz);
}

// Monotonised-central limited slope: zero when the one-sided differences
// have opposite signs or one is zero, else the smallest of twice either and
// their mean, with their sign.  The tests are on sign bits (the same result
// as comparisons for every non-NaN input).
template <typename T>
__device__ __forceinline__ T mc(T dl, T dr) {
  using B = FBits<T>;
  const typename B::I a = B::of(dl), b = B::of(dr);
  if ((a & B::MAG) == 0 || (b & B::MAG) == 0 || (a ^ b) < 0) return T(0);
  if constexpr (kFast && sizeof(T) == 8) {
    // the same value as 2 min(|dl|, |dr|, |dl + dr| / 4): the power-of-two
    // scalings are exact, so they are done on the bit patterns with integer
    // operations, leaving one FP64 operation, dl + dr.  Both arms of each
    // select are integer: near the ends of the exponent range, x/4 of a
    // result below the normal range is the significand shifted right and
    // rounded to nearest even (as the multiply would round it), 2x of a
    // subnormal x is its pattern shifted left, 2x of the largest binade is
    // infinity, and an infinity or NaN stays as it is.
    const long long m = min(a & B::MAG, b & B::MAG);
    const long long iq0 = __double_as_longlong(dl + dr) & B::MAG;
    const long long one = 1ll << 52;
    const int eq = (int)(iq0 >> 52);
    long long iq;
    if (eq == 2047) {
      iq = iq0;  // the sum overflowed: infinity / 4 is infinity
    } else if (eq > 2) {
      iq = iq0 - 2 * one;
    } else {
      // |dl + dr| / 4 below the normal range: significand (with its leading
      // bit for a normal input) times 2^(eq - 3), eq - 3 in [-3, -1]
      const long long sig = eq > 0 ? one | (iq0 & (one - 1)) : iq0;
      const int sh = eq > 0 ? 3 - eq : 2;
      const long long r = sig >> sh, rem = sig & ((1ll << sh) - 1), hf = 1ll << (sh - 1);
      iq = r + ((rem > hf || (rem == hf && (r & 1))) ? 1 : 0);
    }
    const long long is = min(m, iq);
    const int es = (int)(is >> 52);
    const long long i2 = es == 0 ? is << 1 : es < 2046 ? is + one : es == 2046 ? 0x7ff0000000000000ll : is;
    return __longlong_as_double(a < 0 ? i2 | (long long)0x8000000000000000ull : i2);
  } else if constexpr (sizeof(T) == 4) {
    // FP32: the FP32 pipe's own minimum (the same value as the bit-pattern
    // minimum of non-negative values) and absolute-value modifiers
    const T s = fminf(fminf(T(2) * fabsf(dl), T(2) * fabsf(dr)), T(0.5) * fabsf(dl + dr));
    return a < 0 ? B::to(B::of(s) ^ ~B::MAG) : s;
  } else {
    const T s = tmin_nonneg(tmin_nonneg(T(2) * tabs(dl), T(2) * tabs(dr)), T(0.5) * tabs(dl + dr));
    return a < 0 ? B::to(B::of(s) ^ ~B::MAG) : s;
  }
}

// Hancock half-step predictor in primitive form with d/dx_d -> dW_d, h = dt/(2dx).
template <typename T>
__device__ __forceinline__ void predict(const T W[8], const T dX[8], const T dY[8], const T dZ[8], T gamma, T h,
                                        T Ws[8]) {
  T rho = W[RHO], vx = W[VX], vy = W[VY], vz = W[VZ], p = W[PR];
  T Bx = W[BX], By = W[BY], Bz = W[BZ];
  T irho = rcp_k(rho);
  T divv = dX[VX] + dY[VY] + dZ[VZ];
  T r_rho = -(vx * dX[RHO] + vy * dY[RHO] + vz * dZ[RHO]) - rho * divv;
  T gpx = dX[PR] + (Bx * dX[BX] + By * dX[BY] + Bz * dX[BZ]);
  T gpy = dY[PR] + (Bx * dY[BX] + By * dY[BY] + Bz * dY[BZ]);
  T gpz = dZ[PR] + (Bx * dZ[BX] + By * dZ[BY] + Bz * dZ[BZ]);
  T tx = Bx * dX[BX] + By * dY[BX] + Bz * dZ[BX];
  T ty = Bx * dX[BY] + By * dY[BY] + Bz * dZ[BY];
  T tz = Bx * dX[BZ] + By * dY[BZ] + Bz * dZ[BZ];
  T r_vx = -(vx * dX[VX] + vy * dY[VX] + vz * dZ[VX]) - (gpx - tx) * irho;
  T r_vy = -(vx * dX[VY] + vy * dY[VY] + vz * dZ[VY]) - (gpy - ty) * irho;
  T r_vz = -(vx * dX[VZ] + vy * dY[VZ] + vz * dZ[VZ]) - (gpz - tz) * irho;
  T r_p = -(vx * dX[PR] + vy * dY[PR] + vz * dZ[PR]) - gamma * p * divv;
  T r_bx = (Bx * dX[VX] + By * dY[VX] + Bz * dZ[VX]) - (vx * dX[BX] + vy * dY[BX] + vz * dZ[BX]) - Bx * divv;
  T r_by = (Bx * dX[VY] + By * dY[VY] + Bz * dZ[VY]) - (vx * dX[BY] + vy * dY[BY] + vz * dZ[BY]) - By * divv;
  T r_bz = (Bx * dX[VZ] + By * dY[VZ] + Bz * dZ[VZ]) - (vx * dX[BZ] + vy * dY[BZ] + vz * dZ[BZ]) - Bz * divv;
  Ws[RHO] = rho + h * r_rho;
  Ws[VX] = vx + h * r_vx;
  Ws[VY] = vy + h * r_vy;
  Ws[VZ] = vz + h * r_vz;
  Ws[PR] = p + h * r_p;
  Ws[BX] = Bx + h * r_bx;
  Ws[BY] = By + h * r_by;
  Ws[BZ] = Bz + h * r_bz;
}

// HLL flux through a face with normal axis D (compile-time), Davis speeds;
// igm1 = 1/(gamma-1).
// WL/WR: lab-frame primitive states.  F[0..4]: lab-frame mass, momentum
// x,y,z, energy fluxes.  SL, SR: the two signal speeds.
template <typename T, int D>
__device__ __forceinline__ void hll(const T WL[8], const T WR[8], T gamma, T igm1, T F[5], T &SL, T &SR) {
  constexpr int t1 = (D + 1) % 3, t2 = (D + 2) % 3;
  const T h = T(0.5);
  T bn = h * (WL[BX + D] + WR[BX + D]);
  T FL[5], FR[5], UL[5], UR[5], cL, cR, vnL, vnR;
#pragma unroll
  for (int side = 0; side < 2; side++) {
    const T *W = side ? WR : WL;
    T rho = W[RHO], p = W[PR];
    T vn = W[VX + D], vt1 = W[VX + t1], vt2 = W[VX + t2];
    T bt1 = W[BX + t1], bt2 = W[BX + t2];
    T v2 = vn * vn + vt1 * vt1 + vt2 * vt2;
    T B2 = bn * bn + bt1 * bt1 + bt2 * bt2;
    T E = p * igm1 + h * rho * v2 + h * B2;
    T PT = p + h * B2;
    T vB = vn * bn + vt1 * bt1 + vt2 * bt2;
    T cf = cfast(gamma, rcp_k(rho), p, bn, bt1, bt2);
    T *Us = side ? UR : UL;
    T *Fs = side ? FR : FL;
    Us[0] = rho; Us[1] = rho * vn; Us[2] = rho * vt1; Us[3] = rho * vt2; Us[4] = E;
    Fs[0] = rho * vn;
    Fs[1] = rho * vn * vn + PT - bn * bn;
    Fs[2] = rho * vn * vt1 - bn * bt1;
    Fs[3] = rho * vn * vt2 - bn * bt2;
    Fs[4] = (E + PT) * vn - bn * vB;
    if (side) { cR = cf; vnR = vn; } else { cL = cf; vnL = vn; }
  }
  SL = fmin_k(vnL - cL, vnR - cR);
  SR = fmax_k(vnL + cL, vnR + cR);
  T Fr[5];
  const T inv = rcp_k(SR - SL);
  const bool left = ge0(SL), right = le0(SR);
#pragma unroll
  for (int q = 0; q < 5; q++) {
    if (left) Fr[q] = FL[q];
    else if (right) Fr[q] = FR[q];
    else Fr[q] = (SR * FL[q] - SL * FR[q] + SL * SR * (UR[q] - UL[q])) * inv;
  }
  F[0] = Fr[0];
  F[1 + D] = Fr[1];
  F[1 + t1] = Fr[2];
  F[1 + t2] = Fr[3];
  F[4] = Fr[4];
}

// HLLD flux (Miyoshi & Kusano 2005) through a face with normal axis D: the
// HLL outer speeds (Davis estimates from the fast speeds), a contact at S_M
// with one total pressure pT* across the fan, two rotational (Alfven) waves
// at S_M -+ |Bn|/sqrt(rho*), and the flux of the region of the fan holding
// x/t = 0.  In the normal frame a state is (rho, u, v, w, p) with tangential
// field (By, Bz) and the common normal field Bn.  Where
// rho (S - u)(S - S_M) - Bn^2 vanishes (to 1e-12 of rho (S - u)^2 + Bn^2) the
// star state keeps the tangential velocity and field of its side.  Outputs
// and speeds as hll; the same operation order as the FP64 oracle's HLLD.
template <typename T, int D>
__device__ __forceinline__ void hlld(const T WL[8], const T WR[8], T gamma, T igm1, T F[5], T &SL, T &SR) {
  constexpr int t1 = (D + 1) % 3, t2 = (D + 2) % 3;
  const T h = T(0.5);
  const T bx = h * (WL[BX + D] + WR[BX + D]);
  T rho[2], u[2], v[2], w[2], by[2], bz[2], E[2], PT[2], vB[2], c[2], Us[2][5], Fs[2][5];
#pragma unroll
  for (int a = 0; a < 2; a++) {
    const T *W = a ? WR : WL;
    rho[a] = W[RHO]; u[a] = W[VX + D]; v[a] = W[VX + t1]; w[a] = W[VX + t2];
    by[a] = W[BX + t1]; bz[a] = W[BX + t2];
    const T p = W[PR];
    const T v2 = u[a] * u[a] + v[a] * v[a] + w[a] * w[a];
    const T B2 = bx * bx + by[a] * by[a] + bz[a] * bz[a];
    E[a] = p * igm1 + h * rho[a] * v2 + h * B2;
    PT[a] = p + h * B2;
    vB[a] = u[a] * bx + v[a] * by[a] + w[a] * bz[a];
    c[a] = cfast(gamma, T(1) / rho[a], p, bx, by[a], bz[a]);
    Us[a][0] = rho[a]; Us[a][1] = rho[a] * u[a]; Us[a][2] = rho[a] * v[a]; Us[a][3] = rho[a] * w[a];
    Us[a][4] = E[a];
    Fs[a][0] = rho[a] * u[a];
    Fs[a][1] = rho[a] * u[a] * u[a] + PT[a] - bx * bx;
    Fs[a][2] = rho[a] * u[a] * v[a] - bx * by[a];
    Fs[a][3] = rho[a] * u[a] * w[a] - bx * bz[a];
    Fs[a][4] = (E[a] + PT[a]) * u[a] - bx * vB[a];
  }
  SL = tmin(u[0] - c[0], u[1] - c[1]);
  SR = tmax(u[0] + c[0], u[1] + c[1]);
  T Fr[5];
  if (SL >= T(0)) {
#pragma unroll
    for (int k = 0; k < 5; k++) Fr[k] = Fs[0][k];
  } else if (SR <= T(0)) {
#pragma unroll
    for (int k = 0; k < 5; k++) Fr[k] = Fs[1][k];
  } else {
    const T Sa[2] = {SL, SR};
    const T dl = (SL - u[0]) * rho[0], dr = (SR - u[1]) * rho[1];
    const T iden = T(1) / (dr - dl);
    const T SM = ((dr * u[1] - dl * u[0]) - PT[1] + PT[0]) * iden;
    const T PTs = ((dr * PT[0] - dl * PT[1]) + dl * dr * (u[1] - u[0])) * iden;
    T rs[2], vs[2], ws[2], bys[2], bzs[2], Es[2], sr[2];
#pragma unroll
    for (int a = 0; a < 2; a++) {
      const T su = Sa[a] - u[a];
      rs[a] = rho[a] * su / (Sa[a] - SM);
      const T den = rho[a] * su * (Sa[a] - SM) - bx * bx;
      const T ref = rho[a] * su * su + bx * bx;
      if (tabs(den) <= T(1e-12) * ref) {
        vs[a] = v[a]; ws[a] = w[a]; bys[a] = by[a]; bzs[a] = bz[a];
      } else {
        const T iv = T(1) / den;
        const T fv = bx * (SM - u[a]) * iv;
        const T fb = (rho[a] * su * su - bx * bx) * iv;
        vs[a] = v[a] - by[a] * fv;
        ws[a] = w[a] - bz[a] * fv;
        bys[a] = by[a] * fb;
        bzs[a] = bz[a] * fb;
      }
      const T vBs = SM * bx + vs[a] * bys[a] + ws[a] * bzs[a];
      Es[a] = ((su * E[a] - PT[a] * u[a] + PTs * SM) + bx * (vB[a] - vBs)) / (Sa[a] - SM);
      sr[a] = tsqrt(rs[a]);
    }
    const T aB = tabs(bx);
    const T SsL = SM - aB / sr[0], SsR = SM + aB / sr[1];
    if (SsL >= T(0)) {
      const T Ust[5] = {rs[0], rs[0] * SM, rs[0] * vs[0], rs[0] * ws[0], Es[0]};
#pragma unroll
      for (int k = 0; k < 5; k++) Fr[k] = Fs[0][k] + SL * (Ust[k] - Us[0][k]);
    } else if (SsR <= T(0)) {
      const T Ust[5] = {rs[1], rs[1] * SM, rs[1] * vs[1], rs[1] * ws[1], Es[1]};
#pragma unroll
      for (int k = 0; k < 5; k++) Fr[k] = Fs[1][k] + SR * (Ust[k] - Us[1][k]);
    } else {
      const T sg = bx > T(0) ? T(1) : bx < T(0) ? T(-1) : T(0);
      const T isum = T(1) / (sr[0] + sr[1]);
      const T vss = ((sr[0] * vs[0] + sr[1] * vs[1]) + (bys[1] - bys[0]) * sg) * isum;
      const T wss = ((sr[0] * ws[0] + sr[1] * ws[1]) + (bzs[1] - bzs[0]) * sg) * isum;
      const T byss = ((sr[0] * bys[1] + sr[1] * bys[0]) + sr[0] * sr[1] * (vs[1] - vs[0]) * sg) * isum;
      const T bzss = ((sr[0] * bzs[1] + sr[1] * bzs[0]) + sr[0] * sr[1] * (ws[1] - ws[0]) * sg) * isum;
      const T vBss = SM * bx + vss * byss + wss * bzss;
      // the side of the contact that holds x/t = 0 (selects, no indexing by
      // a run-time side)
      const bool left = SM >= T(0);
      const T rsa = left ? rs[0] : rs[1], vsa = left ? vs[0] : vs[1], wsa = left ? ws[0] : ws[1];
      const T bysa = left ? bys[0] : bys[1], bzsa = left ? bzs[0] : bzs[1];
      const T vBsa = SM * bx + vsa * bysa + wsa * bzsa;
      const T Ess = left ? Es[0] - sr[0] * (vBsa - vBss) * sg : Es[1] + sr[1] * (vBsa - vBss) * sg;
      const T Ust[5] = {rsa, rsa * SM, rsa * vsa, rsa * wsa, left ? Es[0] : Es[1]};
      const T Uss[5] = {rsa, rsa * SM, rsa * vss, rsa * wss, Ess};
      const T Sst = left ? SsL : SsR, Saa = left ? SL : SR;
#pragma unroll
      for (int k = 0; k < 5; k++) {
        const T Fa = left ? Fs[0][k] : Fs[1][k], Ua = left ? Us[0][k] : Us[1][k];
        Fr[k] = ((Fa + Sst * Uss[k]) - (Sst - Saa) * Ust[k]) - Saa * Ua;
      }
    }
  }
  F[0] = Fr[0];
  F[1 + D] = Fr[1];
  F[1 + t1] = Fr[2];
  F[1 + t2] = Fr[3];
  F[4] = Fr[4];
}

// The face flux of Riemann solver RS (0 HLL, 1 HLLD).
template <typename T, int D, int RS>
__device__ __forceinline__ void face_flux(const T WL[8], const T WR[8], T gamma, T igm1, T F[5], T &SL, T &SR) {
  if constexpr (RS == 1) hlld<T, D>(WL, WR, gamma, igm1, F, SL, SR);
  else hll<T, D>(WL, WR, gamma, igm1, F, SL, SR);
}

// The two HLL signal speeds of a face alone (same arithmetic as in hll), for
// faces whose flux is not needed.
template <typename T, int D>
__device__ __forceinline__ void hll_speeds(const T WL[8], const T WR[8], T gamma, T &SL, T &SR) {
  constexpr int t1 = (D + 1) % 3, t2 = (D + 2) % 3;
  const T h = T(0.5);
  T bn = h * (WL[BX + D] + WR[BX + D]);
  T cL = cfast(gamma, rcp_k(WL[RHO]), WL[PR], bn, WL[BX + t1], WL[BX + t2]);
  T cR = cfast(gamma, rcp_k(WR[RHO]), WR[PR], bn, WR[BX + t1], WR[BX + t2]);
  SL = fmin_k(WL[VX + D] - cL, WR[VX + D] - cR);
  SR = fmax_k(WL[VX + D] + cL, WR[VX + D] + cR);
}

// Upwind HLL edge EMF from the four corner values around an edge (LL: low
// a and low b side, RL: high a / low b, LR: low a / high b, RR: high/high),
// with ap/am = max(0, +-S) over the faces touching the edge.
template <typename T>
__device__ __forceinline__ T emf(T Ell, T Erl, T Elr, T Err, T Ba_ll, T Ba_rl, T Ba_lr, T Ba_rr, T Bb_ll, T Bb_rl,
                                 T Bb_lr, T Bb_rr, T apa, T ama, T apb, T amb) {
  const T h = T(0.5);
  T BbL = h * (Bb_ll + Bb_lr);
  T BbR = h * (Bb_rl + Bb_rr);
  T BaL = h * (Ba_ll + Ba_rl);
  T BaR = h * (Ba_lr + Ba_rr);
  T num = apa * apb * Ell + ama * apb * Erl + apa * amb * Elr + ama * amb * Err;
  if constexpr (kFast && sizeof(T) == 8) {
    // one reciprocal of the product of the two weight sums serves all three
    // quotients (FP64: a division costs about five FP64-pipe slots; the FP32
    // build divides approximately, at the cost of a multiply)
    const T sa = apa + ama, sb = apb + amb;
    const T r = rcp_k(sa * sb);
    return num * r + (apa * ama * sb * r) * (BbR - BbL) - (apb * amb * sa * r) * (BaR - BaL);
  } else {
    T den = (apa + ama) * (apb + amb);
    return num / den + apa * ama / (apa + ama) * (BbR - BbL) - apb * amb / (apb + amb) * (BaR - BaL);
  }
}

}  // namespace dsp

// dsp_variants.h -- the compiled variants of the update kernel.
//
// Each row is compiled from dsp_variant.cu into its own object (the build
// reads this list): id, element type, tile TX x TY, threads per block,
// minimum resident blocks per SM, precision code of dsp_params (0 FP64
// without FMA, 1 FP32, 2 FP64 with FMA), Riemann solver of the face fluxes
// (0 HLL, 1 HLLD), non-ideal terms (1: the Ohmic and ambipolar EMFs; these
// hold a third plane of faces, so the FP64 rows use a smaller tile).  All
// variants of one precision, solver and physics compute bit-identical
// results; they differ only in how the work is spread over threads, so
// dsp_autotune may pick any of them.  The bounds-checked build
// (DSP_BOUNDS_CHECK) compiles the three rows of DSP_VARIANT_LIST_CHECKED only.
#pragma once

#define DSP_VARIANT_LIST_ALL(X)        \
  X(0, double, 16, 8, 256, 1, 0, 0, 0)    \
  X(1, double, 16, 8, 384, 1, 0, 0, 0)    \
  X(2, double, 16, 8, 256, 1, 2, 0, 0)    \
  X(3, double, 16, 8, 384, 1, 2, 0, 0)    \
  X(4, double, 16, 8, 512, 1, 2, 0, 0)    \
  X(5, float, 16, 8, 256, 2, 1, 0, 0)     \
  X(6, float, 16, 8, 512, 1, 1, 0, 0)     \
  X(7, float, 32, 8, 256, 1, 1, 0, 0)     \
  X(8, float, 16, 16, 256, 1, 1, 0, 0)    \
  X(9, double, 16, 8, 256, 1, 0, 1, 0)    \
  X(10, double, 16, 8, 256, 1, 2, 1, 0)   \
  X(11, float, 16, 8, 256, 2, 1, 1, 0)  \
  X(12, double, 16, 4, 128, 1, 0, 0, 1) \
  X(13, double, 16, 4, 128, 1, 2, 0, 1) \
  X(14, float, 16, 8, 256, 1, 1, 0, 1) \
  X(15, double, 16, 4, 256, 1, 2, 0, 1) \
  X(16, float, 16, 4, 128, 2, 1, 0, 1) \
  X(17, double, 16, 4, 256, 1, 0, 0, 1) \
  X(18, double, 16, 4, 256, 1, 0, 1, 1) \
  X(19, double, 16, 4, 256, 1, 2, 1, 1) \
  X(20, float, 16, 8, 256, 1, 1, 1, 1)   \
  X(21, float, 24, 8, 256, 1, 1, 0, 0)

#define DSP_VARIANT_LIST_CHECKED(X)    \
  X(0, double, 16, 8, 256, 1, 0, 0, 0)    \
  X(2, double, 16, 8, 256, 1, 2, 0, 0)    \
  X(5, float, 16, 8, 256, 2, 1, 0, 0)

#ifdef DSP_BOUNDS_CHECK
#define DSP_VARIANT_LIST(X) DSP_VARIANT_LIST_CHECKED(X)
#else
#define DSP_VARIANT_LIST(X) DSP_VARIANT_LIST_ALL(X)
#endif

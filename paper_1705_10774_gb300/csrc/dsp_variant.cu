// dsp_variant.cu -- one compiled variant of the update and ready-queue
// kernels.  The build compiles this file once per row of dsp_variants.h,
// defining V_ID, V_T, V_TX, V_TY, V_NT, V_MB, V_PREC, V_RS and V_NI (and the
// floating-point flags of the precision: no FMA for FP64 parity, fast
// division and square root for FP32).
// FP64 without FMA keeps the oracle's evaluation order; the other builds
// take the faster one (dsp_physics.cuh, kFast)
#define DSP_FAST_ORDER (V_PREC != 0)
#include "dsp_update.cuh"

#define DSP_STR2(x) #x
#define DSP_STR(x) DSP_STR2(x)
#define DSP_CAT2(a, b) a##b
#define DSP_CAT(a, b) DSP_CAT2(a, b)

namespace dsp {
namespace {
int lu(const DevCtx &c, int grid, void *s, int cls, int cls_end) {
  return launch_update<V_T, V_TX, V_TY, V_NT, V_MB, V_ID, V_RS, V_NI>(c, grid, s, cls, cls_end);
}
int lq(const DevCtx &c, int grid, double t, void *s) {
  return launch_queue<V_T, V_TX, V_TY, V_NT, V_MB, V_ID, V_RS, V_NI>(c, grid, t, s);
}
int gr(const DevCtx &c, int cls, int cls_end) {
  return update_grid<V_T, V_TX, V_TY, V_NT, V_MB, V_ID, V_RS, V_NI>(c, cls, cls_end);
}
const KernelVariant kv = {V_ID, V_PREC, V_RS, V_NI, V_TX, V_TY, V_NT,
                          DSP_STR(V_T) " " DSP_STR(V_TX) "x" DSP_STR(V_TY) " " DSP_STR(V_NT) "t", lu, lq, gr};
}  // namespace
const KernelVariant *DSP_CAT(variant_, V_ID)() { return &kv; }
}  // namespace dsp

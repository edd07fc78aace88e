// FP64 instantiation compiled with fused multiply-adds (the fast FP64 form).
// Results differ from the FMA-free build only by rounding; they are checked
// against the FP64 oracle with a relative tolerance of 1e-11.
#include "dsp_update.cuh"

namespace dsp {
constexpr int TXF = 16, TYF = 8, NTF = 256, MBF = 1;
int launch_update_f64f(const DevCtx &c, int grid, void *stream) {
  return launch_update<double, TXF, TYF, NTF, MBF, 1>(c, grid, stream);
}
int update_grid_f64f(const DevCtx &c) { return update_grid<double, TXF, TYF, NTF, MBF, 1>(c); }
int launch_queue_f64f(const DevCtx &c, int grid, double t_end, void *stream) {
  return launch_queue<double, TXF, TYF, NTF, MBF, 1>(c, grid, t_end, stream);
}
}  // namespace dsp

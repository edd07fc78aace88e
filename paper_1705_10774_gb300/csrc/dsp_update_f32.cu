// FP32 instantiation of the update kernel (FP32 state and stencil
// arithmetic; times, steps and interpolation weights stay FP64).
#include "dsp_update.cuh"

namespace dsp {
constexpr int TX32 = 16, TY32 = 8, NT32 = 256, MB32 = 2;
int launch_update_f32(const DevCtx &c, int grid, void *stream) {
  return launch_update<float, TX32, TY32, NT32, MB32, 0>(c, grid, stream);
}
int update_grid_f32(const DevCtx &c) { return update_grid<float, TX32, TY32, NT32, MB32, 0>(c); }
void update_tile_f32(int *tx, int *ty) {
  *tx = TX32;
  *ty = TY32;
}
int launch_queue_f32(const DevCtx &c, int grid, double t_end, void *stream) {
  return launch_queue<float, TX32, TY32, NT32, MB32, 0>(c, grid, t_end, stream);
}
}  // namespace dsp

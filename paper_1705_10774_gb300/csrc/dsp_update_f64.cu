// FP64 instantiation of the update kernel.  Compiled with -fmad=false so that
// every product and sum is rounded separately, exactly as in the FP64 oracle.
#include "dsp_update.cuh"

namespace dsp {
constexpr int TX64 = 16, TY64 = 8, NT64 = 256, MB64 = 1;
int launch_update_f64(const DevCtx &c, int grid, void *stream) {
  return launch_update<double, TX64, TY64, NT64, MB64, 0>(c, grid, stream);
}
int update_grid_f64(const DevCtx &c) { return update_grid<double, TX64, TY64, NT64, MB64, 0>(c); }
void update_tile_f64(int *tx, int *ty) {
  *tx = TX64;
  *ty = TY64;
}
int launch_queue_f64(const DevCtx &c, int grid, double t_end, void *stream) {
  return launch_queue<double, TX64, TY64, NT64, MB64, 0>(c, grid, t_end, stream);
}
}  // namespace dsp

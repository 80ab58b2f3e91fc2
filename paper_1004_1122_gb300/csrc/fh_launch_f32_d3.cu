// Pass kernels for 3-D grids, float.
#include "fh_launch_impl.cuh"

namespace fh {
LaunchTable<float> launch_table_f32_d3(int nl) {
  if (nl == 1) return Launchers<float, 3, 1>::table();
  if (nl == 3) return Launchers<float, 3, 3>::table();
  return LaunchTable<float>();
}
}  // namespace fh

// Pass kernels for 2-D grids, float.
#include "fh_launch_impl.cuh"

namespace fh {
LaunchTable<float> launch_table_f32_d2(int nl) {
  if (nl == 1) return Launchers<float, 2, 1>::table();
  if (nl == 2) return Launchers<float, 2, 2>::table();
  return LaunchTable<float>();
}
}  // namespace fh

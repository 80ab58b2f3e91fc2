// Pass kernels for 3-D grids, double.
#include "fh_launch_impl.cuh"

namespace fh {
LaunchTable<double> launch_table_f64_d3(int nl) {
  if (nl == 1) return Launchers<double, 3, 1>::table();
  if (nl == 3) return Launchers<double, 3, 3>::table();
  return LaunchTable<double>();
}
}  // namespace fh

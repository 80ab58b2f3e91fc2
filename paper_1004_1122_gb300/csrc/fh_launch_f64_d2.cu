// Pass kernels for 2-D grids, double.
#include "fh_launch_impl.cuh"

namespace fh {
LaunchTable<double> launch_table_f64_d2(int nl) {
  if (nl == 1) return Launchers<double, 2, 1>::table();
  if (nl == 2) return Launchers<double, 2, 2>::table();
  return LaunchTable<double>();
}
}  // namespace fh

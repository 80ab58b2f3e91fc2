// fh_launch.cuh -- per (precision, dimension, load count) launch table.
// The pass kernels are templates over D (2 or 3) and NL (loads per launch);
// each combination is compiled in its own translation unit and reached
// through a table of host function pointers.
#pragma once

#include "fh_kernels.cuh"

namespace fh {

struct Launch {
  int grid = 0, block = 0;
  size_t smem = 0;
};

template <typename T>
struct LaunchTable {
  int D = 0, NL = 0;
  cudaError_t (*set_smem)(size_t row_smem, size_t col0_smem, size_t col1_smem) = nullptr;
  cudaError_t (*row_fwd)(int pro, const Launch&, const RowArgs<T>&, cudaStream_t) = nullptr;
  cudaError_t (*row_inv)(int epi, const Launch&, const RowArgs<T>&, cudaStream_t) = nullptr;
  cudaError_t (*col)(int mode, const Launch&, const ColArgs<T>&, cudaStream_t) = nullptr;
  // persistent bulk-copy Green pass (2-D only; nullptr otherwise)
  cudaError_t (*col_pipe)(const Launch&, const ColArgs<T>&, cudaStream_t) = nullptr;
  cudaError_t (*set_smem_pipe)(size_t bytes) = nullptr;
  cudaError_t (*occupancy_pipe)(int block, size_t smem, int* per_sm) = nullptr;
  // 2-D float64 Green pass in double-float arithmetic (the refinement
  // residual); tw_df is the axis-0 twiddle table as complex double-floats.
  // nullptr for float and for 3-D.
  cudaError_t (*col_df)(const Launch&, const ColArgs<T>&, const void* tw_df, cudaStream_t) = nullptr;
  cudaError_t (*cg_update)(const Launch&, const VecArgs<T>&, cudaStream_t) = nullptr;
  cudaError_t (*cg_flush)(const Launch&, const VecArgs<T>&, cudaStream_t) = nullptr;
  cudaError_t (*bicg_update)(const Launch&, const VecArgs<T>&, cudaStream_t) = nullptr;
  cudaError_t (*current_sum)(const Launch&, const T*, const uint8_t*, const double*, long long nodes,
                             int ncell, long long cell_nodes, int tab_stride, double*,
                             cudaStream_t) = nullptr;
  cudaError_t (*matnorm2)(const Launch&, const T*, long long nodes, int ncell, long long cell_nodes,
                          const Mat3&, double*, cudaStream_t) = nullptr;
  // Length of the compile-time FFT plan that every pass kernel of a CG
  // iteration (direction pass, A p pass, Green pass and, in 3-D, the
  // middle-axis passes) runs for these plans and launch shapes, or 0 when at
  // least one of them runs a run-time-plan kernel.
  int (*ct_plan)(const FFTPlan& prow, const Launch& row, const FFTPlan& pc0, const Launch& col0,
                 const FFTPlan& pc1, const Launch& col1) = nullptr;
};

// Supported (D, NL): (2, 1), (2, 2), (3, 1), (3, 3).
LaunchTable<float> launch_table_f32_d2(int nl);
LaunchTable<float> launch_table_f32_d3(int nl);
LaunchTable<double> launch_table_f64_d2(int nl);
LaunchTable<double> launch_table_f64_d3(int nl);

template <typename T> LaunchTable<T> launch_table(int d, int nl);
template <> inline LaunchTable<float> launch_table<float>(int d, int nl) {
  return d == 2 ? launch_table_f32_d2(nl) : launch_table_f32_d3(nl);
}
template <> inline LaunchTable<double> launch_table<double>(int d, int nl) {
  return d == 2 ? launch_table_f64_d2(nl) : launch_table_f64_d3(nl);
}

}  // namespace fh

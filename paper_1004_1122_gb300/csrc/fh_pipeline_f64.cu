// Explicit instantiation of the float64 pass pipeline.
#include "fh_pipeline_impl.cuh"

namespace fh {
template struct Pipeline<double>;
}  // namespace fh

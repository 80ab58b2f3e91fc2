// Explicit instantiation of the float32 pass pipeline.
#include "fh_pipeline_impl.cuh"

namespace fh {
template struct Pipeline<float>;
}  // namespace fh

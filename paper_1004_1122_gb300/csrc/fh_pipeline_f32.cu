// Explicit instantiation of the float32 pass pipeline.
#include "fh_pipeline_impl.cuh"

namespace fh {
template struct Pipeline<float>;
template int run_loops<float>(Pipeline<float>* const*, int, cudaStream_t, LoopCache&, std::string&);
}  // namespace fh

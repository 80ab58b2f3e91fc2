// Explicit instantiation of the float64 pass pipeline.
#include "fh_pipeline_impl.cuh"

namespace fh {
template struct Pipeline<double>;
template int run_loops<double>(Pipeline<double>* const*, int, cudaStream_t, LoopCache&, std::string&);
}  // namespace fh

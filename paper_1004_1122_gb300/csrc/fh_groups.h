// fh_groups.h -- internal entry into the concurrent group solver of
// fh_batch.cu for one context's problem with all d unit loads batched into
// every launch (the full effective tensor in one solve).
#pragma once

#include <string>

#include "fh_pipeline.cuh"

namespace fh {

struct LoadsResult {
  int status[kMaxLoads];   // fh_status per load
  int iters[kMaxLoads];
  double rel[kMaxLoads];   // float64 true relative residual per load
  int outer = 0;
  long long launches = 0;
  int ct_plans = 0;        // fh_info.ct_plans bits of the float32 CG iterations
};

// Solves (I + B) e = e_b for b = 1..d with the loads batched (NL = d).  The
// first call allocates a persistent group (pipelines and float64 iterates)
// stored in *cache; free it with release_loads_group.  Leff is row-major d x d,
// column b from load b.  Returns 0 or an fh_status code (err set).
int solve_all_loads(const Problem& pb, int precision, double tol, int method, int max_iter,
                    double* Leff, LoadsResult& res, void** cache, std::string& err);
void release_loads_group(void* cache);

// The launch shapes recorded in the tuning cache (FH_TUNE_CACHE) for this
// problem with nloads loads per launch, if any.
bool tuning_from_cache(const Problem& pb, int nloads, bool f64, Tuning& t);

}  // namespace fh

// fh_pipeline.cuh -- per-precision pass pipeline: plans, tilings, device
// buffers, kernel launches, and the Krylov solvers, whose iterations run on
// the device in one graph launch (a while node over chunks of iterations).
//
// Pipeline<T> is explicitly instantiated for float and double in
// fh_pipeline_f32.cu / fh_pipeline_f64.cu.
#pragma once

#include <atomic>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "fh_launch.cuh"
#include "fh_plan.h"

namespace fh {

// Host copy of one problem (Section 2.1 / 2.2 inputs) shared by both pipelines.
struct Problem {
  int d = 2;
  int N[3] = {1, 1, 1};
  double Y[3] = {1.0, 1.0, 1.0};
  long long nodes = 0;      // all cells together (ncell * prod N)
  int nphase = 0;
  int ncell = 1;            // same-size cells solved together (2-D batches)
  std::vector<double> L;    // [ncell][nphase][d][d]
  std::vector<double> L0;   // d * d (common reference medium)
  std::vector<double> L0cell;  // [ncell][3][3] per-cell reference media, or empty
  std::vector<double> dL;   // [ncell][nphase][d][d], L - L0 of the cell
  const uint8_t* d_phase = nullptr;  // device [ncell][N...], owned by the caller of init
};

// Krylov methods (mirror fh_method)
enum : int { kCG = 0, kBiCG = 1, kFixed = 2 };

// How the solve starts.
enum : int {
  kX0Const = 0,   // x = E (cold start, e^0)
  kX0Field = 1,   // x = given field (same precision, device)
  kX0Zero = 2,    // x = 0 (inner refinement solve on A d = r)
  kX0Rhs = 3,     // x = rhs field (inner fixed point starts at e^0 = rhs)
  kX0Keep = 4     // x already holds the start (restart from the current iterate)
};

// Launch-shape choices of one pipeline.  Zero means "heuristic default".
struct Tuning {
  int C = 0;     // half-spectrum tile width
  int lpc = 0;   // lines per CTA in the row passes
  int tpl = 0;   // threads per line FFT (selects the radix plan)
  int tpc0 = 0;  // threads per column FFT along axis 0
  int tpc1 = 0;  // threads per column FFT along axis 1 (3-D)
  int pipe = 0;  // 2-D Green pass: 1 = persistent double-buffered bulk-copy kernel
  bool operator==(const Tuning& o) const {
    return C == o.C && lpc == o.lpc && tpl == o.tpl && tpc0 == o.tpc0 && tpc1 == o.tpc1 && pipe == o.pipe;
  }
};

struct SolveResult {
  int status = 0;      // kConverged / kBreakdown / kCap
  int iters = 0;
  double rel = 0.0;    // last recursive relative residual
  double alpha = 0.0;
};

// A number unique to each initialised pipeline in the process (graph caches
// key on it: a pipeline rebuilt in place gets a new one).
inline unsigned long long next_pipeline_uid() {
  static std::atomic<unsigned long long> n{0};
  return ++n;
}

// Instantiated graphs of device-side iteration loops (run_loops), keyed by
// the pipelines, method and chunk they were captured for.
struct LoopCache {
  std::map<std::string, cudaGraphExec_t> exec;
  std::map<std::string, std::vector<long long>> kernels;  // kernels per loop body, per pipeline
  void clear() {
    for (auto& kv : exec) cudaGraphExecDestroy(kv.second);
    exec.clear();
    kernels.clear();
  }
};

template <typename T>
struct Pipeline {
  using C = cplx<T>;
  Geom g{};
  FFTPlan prow{}, pcol0{}, pcol1{};
  int lpc = 0, tpl = 0, nseq = 0;
  Launch row{}, col0{}, col1{};
  Launch colp{};              // persistent bulk-copy Green pass (when green_pipe)
  bool green_pipe = false;
  int* dev_err = nullptr;     // set by kernels whose bounded waits expired
  int* h_err = nullptr;       // pinned host mirror, refreshed with the scalars
  ColArgsBase cb0{}, cb1{};
  C* tw_last = nullptr;
  C* tw0 = nullptr;
  C* tw1 = nullptr;
  dfc* tw0_df = nullptr;     // 2-D float64: axis-0 twiddles as double-floats (lt.col_df)
  dfc* tw_last_df = nullptr; // 2-D float64: line twiddles as double-floats
  bool df_green = false;     // route the next Green passes through lt.col_df
  C* S = nullptr;
  T* dtab = nullptr;   // dL per phase
  T* qtab = nullptr;   // L0 for every phase: the passes then apply Q = Gamma0 L0
  T* ltab = nullptr;   // L per phase
  double* ltab64 = nullptr;
  const uint8_t* phase = nullptr;
  int nphase = 0;
  Scal* scal = nullptr;      // [nloads] Krylov scalars
  Scal* scal_aux = nullptr;  // [nloads] scratch scalars for residual / norms
  Scal* h_scal = nullptr;    // pinned host mirror
  double* part = nullptr;
  double* h_red = nullptr;   // pinned host mirror of small reductions
  double* d_red = nullptr;
  int part_stride = 0;       // max grid over all partial producers
  int nloads = 1;
  int ncell = 1;
  int items = 1;             // ncell * nloads
  double* L0cell_dev = nullptr;
  long long vlen = 0;        // d * nodes
  T* x[kMaxLoads] = {};
  T* r[kMaxLoads] = {};
  T* p[kMaxLoads] = {};
  T* p2[kMaxLoads] = {};     // CG with deferred x steps: the second direction buffer
  T* ap[kMaxLoads] = {};
  T* rs[kMaxLoads] = {};
  T* ps[kMaxLoads] = {};
  T* atps[kMaxLoads] = {};
  T* rhs[kMaxLoads] = {};
  double* hist = nullptr;
  int hist_cap = 0;
  // per-iteration Section 3 norms (single-load, single-cell solves): device
  // arrays of hist_cap entries, or nullptr
  double* hist_eta_r = nullptr;
  double* hist_eta_e = nullptr;
  double l0iso = 0.0;          // L0 = l0iso I, or 0 when L0 is not isotropic
  double* eta_bufs[2] = {};    // allocations behind hist_eta_e / hist_eta_r
  cudaStream_t st = nullptr;
  std::vector<void*> allocs;
  Launch vec{};
  LaunchTable<T> lt{};
  int sms = 0;
  bool rhs_active_ = false;
  long long launches = 0;                    // kernels enqueued (graph replays included)

  Tuning tuning{};   // the shape actually in use
  int ct_plan = 0;   // compile-time plan length of the CG-iteration passes (0: run-time plans)
  unsigned long long uid = 0;  // next_pipeline_uid() of the last init
  int init(const Problem& pb, int nloads_, bool krylov, cudaStream_t stream, std::string& err,
           const Tuning* want = nullptr);
  // Time the CG-iteration pass kernels for candidate tunings (temporary
  // pipelines) and return the fastest; `ms` receives its time per iteration.
  static int autotune(const Problem& pb, int nloads, cudaStream_t stream, Tuning& best, double& ms,
                      std::string& err, int max_candidates = 256);
  void release();
  bool device_error() const { return h_err != nullptr && *h_err != 0; }
  void set_phase(const uint8_t* d_phase) { phase = d_phase; }

  // ---- one application of the operator passes --------------------------
  RowArgs<T> row_args() const;
  cudaError_t launch_row_fwd(int pro, const RowArgs<T>& a);
  cudaError_t launch_row_inv(int epi, const RowArgs<T>& a);
  cudaError_t launch_green(int mode, Scal* sc, double* pt);
  cudaError_t passes(int pro, int epi, const RowArgs<T>& af, const RowArgs<T>& ai, Scal* sc);

  // e_out = (I + B) e_in  or (I + B^T) e_in, single load, no scalars
  cudaError_t apply(const T* in, T* out, bool transpose);

  // ---- Krylov solve ------------------------------------------------------
  // Solves A x = rhs for every load.  rhs is the constant E[l] when
  // rhs_field is false, else the field in this->rhs[l].  x0 per kX0*.
  // tol_item (optional, [ncell * nloads]) overrides tol per (cell, load).
  // stall_window > 0 ends an item as kStalled once its recursive residual has
  // not halved for that many iterations.
  int solve(int method, const double (*E)[kMaxD], bool rhs_field, int x0, const T* const* x_init,
            double tol, int max_iter, SolveResult* res, std::string& err,
            const double* tol_item = nullptr, int stall_window = 0);
  // The same solve in pieces, for drivers that run several pipelines at once:
  // solve_begin (asynchronous set-up), then run_loops over the pipelines (all
  // iterations on the device, one graph launch), solve_done and
  // solve_results.
  int solve_begin(int method, const double (*E)[kMaxD], bool rhs_field, int x0,
                  const T* const* x_init, double tol, int max_iter, std::string& err,
                  const double* tol_item = nullptr, int stall_window = 0);
  bool solve_done() const;
  void solve_results(SolveResult* res) const;
  int run_method_ = 0, run_K_ = 8;
  // CG defers every other x step (x is read and written once per two
  // iterations); off while the eta_e history needs the iterate every iteration
  bool defer_x_ = false;
  long long run_guard_max_ = 0;
  int* d_loop = nullptr;     // device [2]: rounds run by the device-side loop, round limit
  int* h_loop = nullptr;     // pinned host mirror
  LoopCache loops;           // this pipeline's own device-side loop graphs (solve)
  // Capture `K` iterations of `method` followed by the loop condition into
  // `body`, the body graph of a while node with handle h (on this pipeline's
  // stream).  *kernels receives the kernels one body launches.
  cudaError_t capture_loop_body(cudaGraph_t body, cudaGraphConditionalHandle h, int method, int K,
                                long long* kernels);
  // j: parity of the iteration within the captured body (CG with deferred x
  // steps alternates the two direction buffers and settles x every second
  // iteration)
  cudaError_t enqueue_iter(int method, int j = 0);
  // CG items that stopped with an x step owed receive it (after the loop)
  cudaError_t enqueue_x_flush();
  // eta_e (Eq. errE_def) of the current iterate x[0] into hist_eta_e[iter]
  cudaError_t enqueue_eta_record();
  int chunk_size(int method) const;

  // ---- reductions ---------------------------------------------------------
  // out[l] = ||x_l||^2 (sum over the vector), synchronous
  int norm2(T* const* v, double* out, std::string& err);
  // ||rhs - A x||^2 per load into out (synchronous), residual field into r.
  // df: run the FFTs of the three passes in double-float arithmetic where the
  // pipeline has those kernels (2-D float64); the pointwise work stays in T.
  int residual(const T* const* xin, T* const* rout, bool rhs_field, const double (*E)[kMaxD],
               double* out, std::string& err, bool df = false);
  // column of <tab e> (tab = L) in float64
  int current_mean(const T* e, double* col, std::string& err);
  int eta_e(const T* e, double* eta, std::string& err);
  int matnorm2(const T* e, const double* M, double* out, std::string& err);
  // out_l = (I - Q) r_l with Q = F^-1 Gamma0 F L0 (asynchronous).  Q projects
  // onto the compatible (gradient) fields along the complement on which
  // I + B is the identity, so for A d = r the complement part of d is exactly
  // (I - Q) r; starting a Krylov solve there leaves its residual compatible.
  int project_complement(T* const* r, T* const* out, std::string& err);

  // ---- measurement --------------------------------------------------------
  // Average device time (ms, CUDA events on the pipeline stream) of `reps`
  // back-to-back launches of one piece of the CG iteration:
  // 0 row_fwd (direction update + dL + FFT), 1 column passes (Green),
  // 2 row_inv (inverse FFT + A p + dot), 3 CG vector update, 5 operator apply.
  int profile(int what, int reps, double* ms, std::string& err);
};

// fh_info.ct_plans bit of a compile-time plan length (FH_CT_2187, FH_CT_729, FH_CT_243).
inline int ct_plan_bit(int n) { return n == 2187 ? 1 : n == 729 ? 2 : n == 243 ? 4 : 0; }

// Runs the iteration loops of np pipelines, each prepared by solve_begin, in
// ONE graph launch on `launch`: a CUDA graph with one while node per
// pipeline, whose body is K iterations and a condition kernel; a body runs
// again while an item of its pipeline is running and its round guard
// (max_iter / K + 4 rounds) has not run out, so every loop ends.  Waits for
// the pipelines' streams before the launch and makes them wait for it after;
// synchronises `launch` and refreshes each pipeline's host scalars and error
// word.  Returns 0, 5 (FH_ERR_CUDA) or 8 (FH_ERR_TIMEOUT: a bounded device
// wait expired).
template <typename T>
int run_loops(Pipeline<T>* const* ps, int np, cudaStream_t launch, LoopCache& cache, std::string& err);

extern template struct Pipeline<float>;
extern template struct Pipeline<double>;
extern template int run_loops<float>(Pipeline<float>* const*, int, cudaStream_t, LoopCache&, std::string&);
extern template int run_loops<double>(Pipeline<double>* const*, int, cudaStream_t, LoopCache&, std::string&);

}  // namespace fh

// fh_capi.cu -- the C ABI of include/fh.h: context creation and validation,
// the matrix-free product, and the solve drivers (float64, float32, and
// float32 inner solves with float64 refinement).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/fh.h"
#include "fh_groups.h"
#include "fh_pipeline.cuh"

using fh::Pipeline;
using fh::Problem;
using fh::SolveResult;
using fh::Tuning;

struct fh_ctx {
  Problem pb;
  int precision = FH_FP64;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  uint8_t* d_phase = nullptr;
  Pipeline<float>* p32 = nullptr;
  Pipeline<double>* p64 = nullptr;
  double* d_x64 = nullptr;   // float64 solution (refinement iterate / output staging)
  double* d_r64 = nullptr;   // float64 residual
  long long own_launches = 0;  // kernels launched directly by this file
  void* loads_group = nullptr; // persistent all-loads group of fh_solve_all
  std::string err;
};

namespace {

const char* kStatusNames[] = {"FH_OK",          "FH_ERR_ARG",           "FH_ERR_EVEN_N",
                              "FH_ERR_NOT_SPD", "FH_ERR_OOM",           "FH_ERR_CUDA",
                              "FH_ERR_NOT_CONVERGED", "FH_ERR_BREAKDOWN", "FH_ERR_TIMEOUT",
                              "FH_ERR_UNSUPPORTED"};

fh_status fail(fh_ctx* c, fh_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

// Cholesky test of a symmetric matrix (row-major, n x n).
bool is_spd(const double* A, int n) {
  double scale = 0.0;
  for (int i = 0; i < n * n; ++i) scale = std::fmax(scale, std::fabs(A[i]));
  if (!(scale > 0.0) || !std::isfinite(scale)) return false;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j)
      if (std::fabs(A[i * n + j] - A[j * n + i]) > 1e-12 * scale) return false;
  std::vector<double> Lc(n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= Lc[j * n + k] * Lc[j * n + k];
    if (!(s > 1e-14 * scale)) return false;
    Lc[j * n + j] = std::sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= Lc[i * n + k] * Lc[j * n + k];
      Lc[i * n + j] = t / Lc[j * n + j];
    }
  }
  return true;
}

// Symmetric eigenvalue extremes by Jacobi rotations (n <= 3).
void sym_eig_range(const double* A, int n, double& lo, double& hi) {
  double a[9];
  for (int i = 0; i < n * n; ++i) a[i] = A[i];
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += a[i * n + j] * a[i * n + j];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
      }
  }
  lo = hi = a[0];
  for (int i = 1; i < n; ++i) {
    lo = std::fmin(lo, a[i * n + i]);
    hi = std::fmax(hi, a[i * n + i]);
  }
}

template <typename T>
__global__ void k_convert_vec(const double* in, T* out, long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = T(in[i]);
}
template <typename T>
__global__ void k_widen_vec(const T* in, double* out, long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}
__global__ void k_to_float(const double* in, float* out, float* zero1, long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    out[i] = (float)in[i];
    zero1[i] = 0.0f;
  }
}
__global__ void k_sub_from(const double* a, double* b, long long len) {  // b = a - b
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = a[i] - b[i];
}
__global__ void k_add_float(double* x, const float* d, long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}
__global__ void k_fill_vec(double* x, long long nodes, int d, double e0, double e1, double e2) {
  const long long len = nodes * d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / nodes;
    x[i] = c == 0 ? e0 : (c == 1 ? e1 : e2);
  }
}

int vec_grid(long long len) {
  long long g = (len + 255) / 256;
  return (int)(g < 1184 ? (g < 1 ? 1 : g) : 1184);
}

fh_status from_rc(fh_ctx* c, int rc, const std::string& err) {
  if (rc == 0) return FH_OK;
  c->err = err;
  return (fh_status)rc;
}

fh_status cuda_fail(fh_ctx* c, cudaError_t e, const char* what) {
  c->err = std::string(what) + ": " + cudaGetErrorString(e);
  return FH_ERR_CUDA;
}

int to_status(int done) {
  switch (done) {
    case fh::kConverged: return FH_OK;
    case fh::kBreakdown: return FH_ERR_BREAKDOWN;
    default: return FH_ERR_NOT_CONVERGED;
  }
}

// ---- autotuning cache ---------------------------------------------------
// A plain text file named by the environment variable FH_TUNE_CACHE, one line
// per problem shape:  <key> C lpc tpl tpc0 tpc1 pipe ms_per_iteration
// (lines without the pipe field read as pipe = 0).
std::mutex g_cache_mu;

std::string tune_key(const Problem& pb, int nloads, bool f64) {
  std::ostringstream k;
  k << (f64 ? "f64" : "f32") << "_d" << pb.d << "_L" << nloads << "_";
  for (int a = 0; a < pb.d; ++a) k << (a ? "x" : "") << pb.N[a];
  return k.str();
}

bool cache_lookup(const std::string& key, Tuning& t) {
  const char* path = std::getenv("FH_TUNE_CACHE");
  if (!path || !*path) return false;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  std::ifstream f(path);
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream ls(line);
    std::string k;
    std::vector<double> v;
    double x;
    if (!(ls >> k) || k != key) continue;
    while (ls >> x) v.push_back(x);
    if (v.size() != 6 && v.size() != 7) continue;
    Tuning c;
    c.C = (int)v[0];
    c.lpc = (int)v[1];
    c.tpl = (int)v[2];
    c.tpc0 = (int)v[3];
    c.tpc1 = (int)v[4];
    c.pipe = v.size() == 7 ? (int)v[5] : 0;
    t = c;
    found = true;  // the last entry for a key wins
  }
  return found;
}

void cache_store(const std::string& key, const Tuning& t, double ms) {
  const char* path = std::getenv("FH_TUNE_CACHE");
  if (!path || !*path) return;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  std::ofstream f(path, std::ios::app);
  f << key << " " << t.C << " " << t.lpc << " " << t.tpl << " " << t.tpc0 << " " << t.tpc1 << " " << t.pipe
    << " " << ms << "\n";
}

}  // namespace

namespace fh {
bool tuning_from_cache(const Problem& pb, int nloads, bool f64, Tuning& t) {
  return cache_lookup(tune_key(pb, nloads, f64), t);
}
}  // namespace fh

namespace {

template <typename T>
int init_tuned(Pipeline<T>* P, const Problem& pb, bool krylov, cudaStream_t st, std::string& err) {
  Tuning t;
  if (cache_lookup(tune_key(pb, 1, sizeof(T) == 8), t)) {
    if (P->init(pb, 1, krylov, st, err, &t) == 0) return 0;
    P->release();
    *P = Pipeline<T>();
  }
  return P->init(pb, 1, krylov, st, err);
}

// An inner float32 solve whose recursive residual has not halved for this many
// iterations has reached float32's noise floor for its right-hand side; the
// float64 outer residual then decides whether another refinement step helps.
constexpr int kInnerStallWindow = 100;

// Relative residual at which the first float32 solve of a refined solve hands
// over to the float64 outer residual.
constexpr double kFirstEta = 1e-3;

bool l0_isotropic(const Problem& pb, double& l0) {
  const int d = pb.d;
  l0 = pb.L0[0];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (std::fabs(pb.L0[i * d + j] - (i == j ? l0 : 0.0)) > 1e-15 * std::fabs(l0)) return false;
  return true;
}

}  // namespace

// ---- bounded device waits ------------------------------------------------
namespace {
std::atomic<unsigned long long> g_wait_limit_ns{0};

// Word written by the wait self-test: 1 when its wait gave up.
__device__ int g_selftest_word;

// One CTA: an mbarrier that expects one arrival which nothing makes; thread 0
// waits on it with the given limit, then records whether the wait gave up.
// Nothing is in flight, so the kernel ends cleanly either way.
__global__ void k_wait_selftest(unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    fh::tma::mbar_init(&bar, 1);
    fh::tma::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) g_selftest_word = fh::tma::mbar_wait(&bar, 0, limit_ns) ? 0 : 1;
}
}  // namespace

namespace fh {
namespace tma {
unsigned long long wait_limit_ns() { return g_wait_limit_ns.load(); }
}  // namespace tma
}  // namespace fh

extern "C" {

fh_status fh_set_wait_limit(double seconds) {
  if (!(seconds >= 0.0) || seconds > 3600.0) return FH_ERR_ARG;
  g_wait_limit_ns.store((unsigned long long)(seconds * 1e9));
  return FH_OK;
}

fh_status fh_wait_selftest(double seconds, void* stream) {
  if (!(seconds > 0.0) || seconds > 60.0) return FH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int zero = 0;
  cudaError_t e = cudaMemcpyToSymbolAsync(g_selftest_word, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, st>>>((unsigned long long)(seconds * 1e9));
    e = cudaGetLastError();
  }
  int word = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyFromSymbolAsync(&word, g_selftest_word, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return FH_ERR_CUDA;
  return word ? FH_ERR_TIMEOUT : FH_OK;
}

const char* fh_version(void) { return "fh 0.1.0 (sm_103a)"; }

const char* fh_status_string(int s) {
  if (s < 0 || s > 9) return "FH_UNKNOWN";
  return kStatusNames[s];
}

const char* fh_last_error(const fh_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

void fh_destroy(fh_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->p32) {
    c->p32->release();
    delete c->p32;
  }
  if (c->p64) {
    c->p64->release();
    delete c->p64;
  }
  fh::release_loads_group(c->loads_group);
  if (c->d_phase) cudaFree(c->d_phase);
  if (c->d_x64) cudaFree(c->d_x64);
  if (c->d_r64) cudaFree(c->d_r64);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
  delete c;
}

fh_status fh_create(fh_ctx** out, int d, const int* N, const double* Y, const uint8_t* phase,
                    int phase_on_device, int nphase, const double* L, const double* L0,
                    int precision, void* stream) {
  if (!out) return FH_ERR_ARG;
  *out = nullptr;
  if (d != 2 && d != 3) return FH_ERR_ARG;
  if (!N || !phase || !L || nphase < 1 || nphase > 256) return FH_ERR_ARG;
  if (precision < FH_FP64 || precision > FH_FP32_REFINED) return FH_ERR_ARG;
  for (int a = 0; a < d; ++a) {
    if (N[a] < 3) return FH_ERR_ARG;
    if (Y && !(Y[a] > 0.0 && std::isfinite(Y[a]))) return FH_ERR_ARG;
  }
  fh_ctx* c = new (std::nothrow) fh_ctx();
  if (!c) return FH_ERR_OOM;
  Problem& pb = c->pb;
  pb.d = d;
  pb.nodes = 1;
  for (int a = 0; a < d; ++a) {
    pb.N[a] = N[a];
    pb.Y[a] = Y ? Y[a] : 1.0;
    pb.nodes *= N[a];
  }
  pb.nphase = nphase;
  pb.L.assign(L, L + (size_t)nphase * d * d);
  for (int p = 0; p < nphase; ++p) {
    if (!is_spd(&pb.L[(size_t)p * d * d], d)) {
      fh_destroy(c);
      return FH_ERR_NOT_SPD;
    }
  }
  if (L0) {
    pb.L0.assign(L0, L0 + d * d);
    if (!is_spd(pb.L0.data(), d)) {
      fh_destroy(c);
      return FH_ERR_NOT_SPD;
    }
  } else {
    // Eq. (opt_ref): (lambda_min + lambda_max) / 2 I over every phase eigenvalue
    double lo = 1e300, hi = -1e300;
    for (int p = 0; p < nphase; ++p) {
      double a, b;
      sym_eig_range(&pb.L[(size_t)p * d * d], d, a, b);
      lo = std::fmin(lo, a);
      hi = std::fmax(hi, b);
    }
    pb.L0.assign(d * d, 0.0);
    for (int i = 0; i < d; ++i) pb.L0[i * d + i] = 0.5 * (lo + hi);
  }
  pb.dL.resize(pb.L.size());
  for (int p = 0; p < nphase; ++p)
    for (int i = 0; i < d * d; ++i) pb.dL[(size_t)p * d * d + i] = pb.L[(size_t)p * d * d + i] - pb.L0[i];
  c->precision = precision;

  if (stream) {
    c->st = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreate(&c->st) != cudaSuccess) {
      fh_destroy(c);
      return FH_ERR_CUDA;
    }
    c->own_stream = true;
  }
  if (cudaMalloc(&c->d_phase, pb.nodes) != cudaSuccess) {
    fh_destroy(c);
    return FH_ERR_OOM;
  }
  pb.d_phase = c->d_phase;
  fh_status s = fh_set_phase(c, phase, phase_on_device);
  if (s != FH_OK) {
    fh_destroy(c);
    return s;
  }
  std::string err;
  int rc = 0;
  if (precision == FH_FP64 || precision == FH_FP32_REFINED) {
    c->p64 = new (std::nothrow) Pipeline<double>();
    if (!c->p64) rc = FH_ERR_OOM;
    if (!rc) rc = init_tuned(c->p64, pb, precision == FH_FP64, c->st, err);
  }
  if (!rc && (precision == FH_FP32 || precision == FH_FP32_REFINED)) {
    c->p32 = new (std::nothrow) Pipeline<float>();
    if (!c->p32) rc = FH_ERR_OOM;
    if (!rc) rc = init_tuned(c->p32, pb, true, c->st, err);
  }
  const size_t vbytes = (size_t)d * pb.nodes * sizeof(double);
  if (!rc && cudaMalloc(&c->d_x64, vbytes) != cudaSuccess) rc = FH_ERR_OOM;
  if (!rc && cudaMalloc(&c->d_r64, vbytes) != cudaSuccess) rc = FH_ERR_OOM;
  if (rc) {
    fh_destroy(c);
    return (fh_status)rc;
  }
  *out = c;
  return FH_OK;
}

fh_status fh_set_phase(fh_ctx* c, const uint8_t* phase, int phase_on_device) {
  if (!c || !phase) return FH_ERR_ARG;
  const size_t n = (size_t)c->pb.nodes;
  std::vector<uint8_t> h(n);
  cudaError_t e;
  if (phase_on_device) {
    e = cudaMemcpyAsync(h.data(), phase, n, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  } else {
    std::memcpy(h.data(), phase, n);
    e = cudaSuccess;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "phase copy");
  for (size_t i = 0; i < n; ++i)
    if (h[i] >= c->pb.nphase) return fail(c, FH_ERR_ARG, "phase id out of range");
  e = cudaMemcpyAsync(c->d_phase, h.data(), n, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "phase upload");
  return FH_OK;
}

fh_status fh_apply(fh_ctx* c, const void* in, void* out, int transpose, int dtype) {
  if (!c || !in || !out) return FH_ERR_ARG;
  cudaError_t e;
  if (dtype == FH_FP64) {
    if (!c->p64) return fail(c, FH_ERR_ARG, "context has no float64 pipeline");
    e = c->p64->apply(static_cast<const double*>(in), static_cast<double*>(out), transpose != 0);
  } else if (dtype == FH_FP32) {
    if (!c->p32) return fail(c, FH_ERR_ARG, "context has no float32 pipeline");
    e = c->p32->apply(static_cast<const float*>(in), static_cast<float*>(out), transpose != 0);
  } else {
    return fail(c, FH_ERR_ARG, "dtype must be FH_FP64 or FH_FP32");
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "fh_apply");
  return FH_OK;
}

}  // extern "C"

namespace {

template <typename T>
fh_status finish_info(fh_ctx* c, Pipeline<T>* P, fh_info* info, int hist_len) {
  if (!info || info->history_cap <= 0 || hist_len <= 0) return FH_OK;
  const int n = hist_len < info->history_cap ? hist_len : info->history_cap;
  auto copy = [&](double* dst, const double* src, int len, int* out_len) -> fh_status {
    if (!dst || !src || len <= 0) return FH_OK;
    cudaError_t e = cudaMemcpyAsync(dst, src, len * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "history copy");
    *out_len = len;
    return FH_OK;
  };
  fh_status s = copy(info->history, P->hist, n, &info->history_len);
  if (s == FH_OK) s = copy(info->eta_e_history, P->hist_eta_e, n, &info->eta_e_len);
  if (s == FH_OK) s = copy(info->eta_r_history, P->hist_eta_r, n - 1, &info->eta_r_len);
  P->hist_eta_e = nullptr;  // the next solve asks again
  P->hist_eta_r = nullptr;
  return s;
}

// Device history buffers of the pipeline sized for info->history_cap: the
// residual history, and (norms = true) the eta_e / eta_r histories the
// caller asked for.
template <typename T>
int ensure_hist(Pipeline<T>* P, fh_info* info, std::string& err, bool norms = false) {
  P->hist_eta_e = nullptr;
  P->hist_eta_r = nullptr;
  const int cap = info ? info->history_cap : 0;
  const bool want_h = info && info->history && cap > 0;
  const bool want_e = norms && info && info->eta_e_history && cap > 0;
  const bool want_r = norms && info && info->eta_r_history && cap > 0;
  if (!want_h && !want_e && !want_r) {
    P->hist = nullptr;
    P->hist_cap = 0;
    return 0;
  }
  auto get = [&](double** dst) -> int {
    double* h = nullptr;
    if (cudaMalloc(&h, cap * sizeof(double)) != cudaSuccess) {
      err = "history allocation";
      return FH_ERR_OOM;
    }
    P->allocs.push_back(h);
    *dst = h;
    return 0;
  };
  if (P->hist_cap < cap || P->hist == nullptr) {
    if (int rc = get(&P->hist)) return rc;
    P->hist_cap = cap;
    P->eta_bufs[0] = P->eta_bufs[1] = nullptr;  // sized for the old capacity
  }
  P->hist_cap = cap;
  if (want_e) {
    if (!P->eta_bufs[0] && get(&P->eta_bufs[0])) return FH_ERR_OOM;
    P->hist_eta_e = P->eta_bufs[0];
  }
  if (want_r) {
    if (!P->eta_bufs[1] && get(&P->eta_bufs[1])) return FH_ERR_OOM;
    P->hist_eta_r = P->eta_bufs[1];
  }
  return 0;
}

// Direct solve in one precision (FH_FP64 or FH_FP32): the Krylov loop runs in
// P; x0 = E or e_init.  Restarts from the current iterate if the true residual
// (same precision) misses the tolerance while the recursive one met it.
template <typename T>
fh_status solve_direct(fh_ctx* c, Pipeline<T>* P, const double* E, double tol, int method,
                       int max_iter, const double* e_init, fh_info* info, double& rel_true,
                       double& eta_r) {
  std::string err;
  const long long len = (long long)c->pb.d * c->pb.nodes;
  double Ev[fh::kMaxLoads][fh::kMaxD] = {};
  for (int a = 0; a < c->pb.d; ++a) Ev[0][a] = E[a];
  int rc = ensure_hist(P, info, err, true);
  if (rc) return from_rc(c, rc, err);
  int x0 = fh::kX0Const;
  if (e_init) {
    ++c->own_launches;
    k_convert_vec<T><<<vec_grid(len), 256, 0, c->st>>>(e_init, P->x[0], len);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "initial field");
    x0 = fh::kX0Keep;
  }
  int total = 0, status = fh::kCap;
  SolveResult res;
  const double e2 = [&] {
    double s = 0.0;
    for (int a = 0; a < c->pb.d; ++a) s += E[a] * E[a];
    return s * (double)c->pb.nodes;
  }();
  rel_true = NAN;
  for (int attempt = 0; attempt < 4; ++attempt) {
    const int budget = max_iter - total;
    rc = P->solve(method, Ev, false, x0, nullptr, tol, budget > 0 ? budget : 0, &res, err);
    if (rc) return from_rc(c, rc, err);
    total += res.iters;
    status = res.status;
    // true residual of the iterate (into the ap buffer as scratch)
    double rr;
    const T* xin[fh::kMaxLoads] = {P->x[0]};
    T* rout[fh::kMaxLoads] = {P->ap[0]};
    rc = P->residual(xin, rout, false, Ev, &rr, err);
    if (rc) return from_rc(c, rc, err);
    rel_true = std::sqrt(rr / (e2 > 0 ? e2 : 1.0));
    if (status != fh::kConverged || rel_true <= tol || total >= max_iter) break;
    x0 = fh::kX0Keep;  // restart CG from the current iterate
  }
  if (status == fh::kConverged && !(rel_true <= tol)) status = fh::kCap;
  if (info) {
    info->iters = total;
    info->outer_iters = 0;
    info->rel_res = res.rel;
  }
  // eta_r (Eq. errR_def as printed)
  eta_r = NAN;
  if (method == fh::kFixed) {
    double l0;
    if (l0_isotropic(c->pb, l0)) eta_r = l0 * res.rel;
  } else {
    double M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < c->pb.d; ++i)
      for (int j = 0; j < c->pb.d; ++j) M[i * 3 + j] = c->pb.L0[i * c->pb.d + j];
    double n2;
    rc = P->matnorm2(P->p[0], M, &n2, err);
    if (rc) return from_rc(c, rc, err);
    eta_r = std::fabs(res.alpha) * std::sqrt(n2 / (e2 > 0 ? e2 : 1.0));
  }
  fh_status fs = finish_info(c, P, info, res.iters + 1);
  if (fs != FH_OK) return fs;
  return (fh_status)to_status(status);
}

}  // namespace

extern "C" {

fh_status fh_solve(fh_ctx* c, const double* E, double tol, int method, int max_iter,
                   const double* e_init, double* e_out, double* Leff_col, fh_info* info) {
  if (!c || !E) return FH_ERR_ARG;
  if (!(tol > 0.0) || max_iter < 0) return fail(c, FH_ERR_ARG, "tol must be > 0, max_iter >= 0");
  if (method < FH_CG || method > FH_FIXED_POINT) return fail(c, FH_ERR_ARG, "unknown method");
  for (int a = 0; a < c->pb.d; ++a)
    if (!std::isfinite(E[a])) return fail(c, FH_ERR_ARG, "E not finite");
  const int d = c->pb.d;
  const long long len = (long long)d * c->pb.nodes;
  const size_t vbytes = (size_t)len * sizeof(double);
  if (info) {
    info->iters = info->outer_iters = info->matvecs = 0;
    info->history_len = 0;
    info->launches = 0;
    info->ct_plans = 0;
    info->eta_e_len = info->eta_r_len = 0;
    info->rel_res_true = info->rel_res = info->eta_r = info->eta_e = NAN;
  }
  const long long launches0 = c->own_launches + (c->p32 ? c->p32->launches : 0) +
                              (c->p64 ? c->p64->launches : 0);
  std::string err;
  int rc;
  cudaError_t e;
  fh_status st = FH_OK;
  double rel_true = NAN, eta_r = NAN;
  const double* xfinal = nullptr;  // float64 device field of the result

  if (c->precision == FH_FP64) {
    st = solve_direct<double>(c, c->p64, E, tol, method, max_iter, e_init, info, rel_true, eta_r);
    if (st == FH_ERR_CUDA || st == FH_ERR_OOM || st == FH_ERR_ARG || st == FH_ERR_TIMEOUT) return st;
    xfinal = c->p64->x[0];
  } else if (c->precision == FH_FP32) {
    st = solve_direct<float>(c, c->p32, E, tol, method, max_iter, e_init, info, rel_true, eta_r);
    if (st == FH_ERR_CUDA || st == FH_ERR_OOM || st == FH_ERR_ARG || st == FH_ERR_TIMEOUT) return st;
    ++c->own_launches;
    k_widen_vec<float><<<vec_grid(len), 256, 0, c->st>>>(c->p32->x[0], c->d_x64, len);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "widen");
    xfinal = c->d_x64;
  } else {
    // FP32 inner solves on A d = r with a float64 outer residual r = e0 - A x
    Pipeline<float>* P = c->p32;
    Pipeline<double>* Q = c->p64;
    rc = ensure_hist(P, info, err);
    if (rc) return from_rc(c, rc, err);
    double Ev[fh::kMaxLoads][fh::kMaxD] = {};
    for (int a = 0; a < d; ++a) Ev[0][a] = E[a];
    double e2 = 0.0;
    for (int a = 0; a < d; ++a) e2 += E[a] * E[a];
    e2 *= (double)c->pb.nodes;
    if (e2 <= 0.0) e2 = 1.0;
    if (e_init) {
      e = cudaMemcpyAsync(c->d_x64, e_init, vbytes, cudaMemcpyDeviceToDevice, c->st);
    } else {
      ++c->own_launches;
      k_fill_vec<<<vec_grid(len), 256, 0, c->st>>>(c->d_x64, c->pb.nodes, d, E[0], E[1], d > 2 ? E[2] : 0.0);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "initial field");
    int total = 0, outer = 0, status = fh::kCap, hist_len = 0;
    double prev_rel = INFINITY;
    SolveResult res;
    double last_alpha = 0.0;
    bool done_first = false;
    if (!e_init) {
      // From e = E the first correction solves A d = -B E, whose complement
      // part is zero (B maps into the compatible fields): that is the float32
      // solve of A x = E from x = E itself, with no float64 residual before it.
      // It stops at kFirstEta (or 0.3 tol if that is looser): float32 CG
      // tracks float64 CG closely that far, and restarting from the float64
      // residual there took fewer iterations in total than pushing float32 to
      // its limit first (2187^2, contrast 1e4: 395 instead of 446).
      double eta = std::max(0.3 * tol, kFirstEta);
      if (eta > 0.1) eta = 0.1;
      rc = P->solve(method, Ev, false, fh::kX0Const, nullptr, eta, max_iter, &res, err, nullptr,
                    kInnerStallWindow);
      if (rc) return from_rc(c, rc, err);
      total = res.iters;
      hist_len = res.iters + 1;
      last_alpha = res.alpha;
      ++c->own_launches;
      k_widen_vec<float><<<vec_grid(len), 256, 0, c->st>>>(P->x[0], c->d_x64, len);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "widen");
      outer = 1;
      if (res.status == fh::kBreakdown && res.iters == 0) {
        status = fh::kBreakdown;
        done_first = true;
      }
    }
    for (; !done_first;) {
      double rr;
      const double* xin[fh::kMaxLoads] = {c->d_x64};
      double* rout[fh::kMaxLoads] = {c->d_r64};
      // float64-accuracy residual; its Green pass runs in double-float
      rc = Q->residual(xin, rout, false, Ev, &rr, err, true);
      if (rc) return from_rc(c, rc, err);
      rel_true = std::sqrt(rr / e2);
      if (!std::isfinite(rel_true)) { status = fh::kBreakdown; break; }
      if (rel_true <= tol) { status = fh::kConverged; break; }
      if (total >= max_iter) { status = fh::kCap; break; }
      if (outer > 0 && !(rel_true < 0.9 * prev_rel)) {
        // the float64 residual stopped improving: float32 accuracy exhausted
        status = res.status == fh::kBreakdown ? fh::kBreakdown : fh::kCap;
        break;
      }
      prev_rel = rel_true;
      // inner tolerance relative to the current residual: aim a little past
      // the target, never below what float32 can resolve
      double eta = 0.3 * tol / rel_true;
      // a first step from a given initial field far from the solution hands
      // over at kFirstEta |E| too, as the direct first step from e = E does
      if (outer == 0 && rel_true > 10.0 * kFirstEta) eta = std::max(eta, kFirstEta / rel_true);
      if (eta < 2e-6) eta = 2e-6;
      if (eta > 0.1) eta = 0.1;
      ++c->own_launches;
      k_to_float<<<vec_grid(len), 256, 0, c->st>>>(c->d_r64, P->rhs[0], P->x[0], len);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "refine init");
      int x0 = fh::kX0Rhs;
      if (method != fh::kFixed) {
        // start at the exact complement part of the correction, d0 = (I - Q) r
        float* rr_[fh::kMaxLoads] = {P->rhs[0]};
        float* xx_[fh::kMaxLoads] = {P->x[0]};
        rc = P->project_complement(rr_, xx_, err);
        if (rc) return from_rc(c, rc, err);
        x0 = fh::kX0Keep;
      }
      rc = P->solve(method, Ev, true, x0, nullptr, eta, max_iter - total, &res, err, nullptr,
                    kInnerStallWindow);
      if (rc) return from_rc(c, rc, err);
      total += res.iters;
      hist_len = res.iters + 1;
      last_alpha = res.alpha;
      ++c->own_launches;
      k_add_float<<<vec_grid(len), 256, 0, c->st>>>(c->d_x64, P->x[0], len);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "refine add");
      ++outer;
      if (res.status == fh::kBreakdown && res.iters == 0) { status = fh::kBreakdown; break; }
    }
    if (info) {
      info->iters = total;
      info->outer_iters = outer;
      info->rel_res = res.rel;
    }
    eta_r = NAN;
    if (method == fh::kFixed) {
      double l0;
      if (l0_isotropic(c->pb, l0)) eta_r = l0 * rel_true;
    } else if (outer > 0) {
      double M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) M[i * 3 + j] = c->pb.L0[i * d + j];
      double n2;
      rc = P->matnorm2(P->p[0], M, &n2, err);
      if (rc) return from_rc(c, rc, err);
      eta_r = std::fabs(last_alpha) * std::sqrt(n2 / e2);
    }
    fh_status fs = finish_info(c, P, info, hist_len);
    if (fs != FH_OK) return fs;
    st = (fh_status)to_status(status);
    xfinal = c->d_x64;
  }

  if (e_out) {
    e = cudaMemcpyAsync(e_out, xfinal, vbytes, cudaMemcpyDeviceToDevice, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "output copy");
  }
  if (Leff_col) {
    fh_status s2 = fh_effective_column(c, xfinal, Leff_col);
    if (s2 != FH_OK) return s2;
  }
  if (info) {
    info->rel_res_true = rel_true;
    info->eta_r = eta_r;
    info->status = st;
    double eta;
    if ((info->flags & FH_INFO_ETA_E) && fh_eta_e(c, xfinal, &eta) == FH_OK) info->eta_e = eta;
    info->matvecs = info->iters * (method == FH_BICG ? 2 : 1) + 1 + info->outer_iters;
    info->launches = c->own_launches + (c->p32 ? c->p32->launches : 0) +
                     (c->p64 ? c->p64->launches : 0) - launches0;
    info->ct_plans = (method == FH_CG && c->precision != FH_FP64 && c->p32) ? fh::ct_plan_bit(c->p32->ct_plan) : 0;
  }
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return cuda_fail(c, e, "fh_solve");
  return st;
}

fh_status fh_solve_all(fh_ctx* c, double tol, int method, int max_iter, double* Leff,
                       fh_info* infos) {
  if (!c || !Leff) return FH_ERR_ARG;
  if (!(tol > 0.0) || max_iter < 0) return fail(c, FH_ERR_ARG, "tol must be > 0, max_iter >= 0");
  if (method < FH_CG || method > FH_FIXED_POINT) return fail(c, FH_ERR_ARG, "unknown method");
  const int d = c->pb.d;
  bool ext = false;
  for (int a = 0; a < d; ++a) {
    bool e;
    fh::factorable(c->pb.N[a], e);
    ext = ext || e;
  }
  if (c->precision == FH_FP32 || ext) {
    // no float64 pipeline to check the loads against (FH_FP32), or an axis
    // whose plan runs one load per launch only: solve the loads one by one
    fh_status first = FH_OK;
    for (int b = 0; b < d; ++b) {
      double E[3] = {0, 0, 0};
      E[b] = 1.0;
      double col[3];
      fh_status s = fh_solve(c, E, tol, method, max_iter, nullptr, nullptr, col, infos ? &infos[b] : nullptr);
      if (s == FH_ERR_CUDA || s == FH_ERR_OOM || s == FH_ERR_ARG || s == FH_ERR_TIMEOUT) return s;
      if (first == FH_OK && s != FH_OK) first = s;
      for (int a = 0; a < d; ++a) Leff[a * d + b] = col[a];
    }
    return first;
  }
  // all d loads batched into every launch
  fh::LoadsResult r;
  std::string err;
  int rc = fh::solve_all_loads(c->pb, c->precision, tol, method, max_iter, Leff, r, &c->loads_group, err);
  if (rc) return fail(c, (fh_status)rc, err);
  fh_status first = FH_OK;
  for (int b = 0; b < d; ++b) {
    if (first == FH_OK && r.status[b] != FH_OK) first = (fh_status)r.status[b];
    if (infos) {
      fh_info& inf = infos[b];
      inf.iters = r.iters[b];
      inf.outer_iters = r.outer;
      inf.matvecs = 0;
      inf.status = r.status[b];
      inf.rel_res_true = r.rel[b];
      inf.rel_res = NAN;
      inf.eta_r = NAN;
      inf.eta_e = NAN;
      inf.history_len = 0;
      inf.launches = r.launches;
      inf.ct_plans = r.ct_plans;
    }
  }
  return first;
}

fh_status fh_project_compatible(fh_ctx* c, const double* in, double* out) {
  if (!c || !in || !out) return FH_ERR_ARG;
  const long long len = (long long)c->pb.d * c->pb.nodes;
  std::string err;
  cudaError_t e;
  if (c->p64) {
    // scratch = (I - Q) in, then scratch = in - scratch = Q in, copied to out
    double* rin[fh::kMaxLoads] = {const_cast<double*>(in)};
    double* rout[fh::kMaxLoads] = {c->d_r64};
    int rc = c->p64->project_complement(rin, rout, err);
    if (rc) return from_rc(c, rc, err);
    ++c->own_launches;
    k_sub_from<<<vec_grid(len), 256, 0, c->st>>>(in, c->d_r64, len);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "project");
    if ((e = cudaMemcpyAsync(out, c->d_r64, len * sizeof(double), cudaMemcpyDeviceToDevice, c->st)) != cudaSuccess)
      return cuda_fail(c, e, "copy");
    return FH_OK;
  }
  // float32 context
  ++c->own_launches;
  k_convert_vec<float><<<vec_grid(len), 256, 0, c->st>>>(in, c->p32->rhs[0], len);
  float* rin[fh::kMaxLoads] = {c->p32->rhs[0]};
  float* rout[fh::kMaxLoads] = {c->p32->ap[0]};
  int rc = c->p32->project_complement(rin, rout, err);
  if (rc) return from_rc(c, rc, err);
  ++c->own_launches;
  k_widen_vec<float><<<vec_grid(len), 256, 0, c->st>>>(c->p32->ap[0], c->d_r64, len);
  ++c->own_launches;
  k_sub_from<<<vec_grid(len), 256, 0, c->st>>>(in, c->d_r64, len);
  if ((e = cudaMemcpyAsync(out, c->d_r64, len * sizeof(double), cudaMemcpyDeviceToDevice, c->st)) != cudaSuccess)
    return cuda_fail(c, e, "copy");
  return FH_OK;
}

fh_status fh_profile(fh_ctx* c, int dtype, int what, int reps, double* ms) {
  if (!c || !ms || reps < 1) return FH_ERR_ARG;
  std::string err;
  int rc;
  if (dtype == FH_FP64 && c->p64 && c->p64->x[0]) {
    rc = c->p64->profile(what, reps, ms, err);
  } else if (dtype == FH_FP32 && c->p32) {
    rc = c->p32->profile(what, reps, ms, err);
  } else {
    return fail(c, FH_ERR_ARG, "no Krylov pipeline of that precision in this context");
  }
  return from_rc(c, rc, err);
}

}  // extern "C"

namespace {
template <typename T>
fh_status autotune_one(fh_ctx* c, Pipeline<T>*& P, bool krylov, double* ms_before, double* ms_after) {
  std::string err;
  double before = 0.0, t;
  for (int what = 0; what < 4; ++what) {
    int rc = P->profile(what, 10, &t, err);
    if (rc) return from_rc(c, rc, err);
    before += t;
  }
  Tuning best;
  double best_ms;
  int rc = Pipeline<T>::autotune(c->pb, 1, c->st, best, best_ms, err);
  if (rc) return from_rc(c, rc, err);
  if (ms_before) *ms_before = before;
  if (best_ms < before && !(best == P->tuning)) {
    Pipeline<T>* Q = new (std::nothrow) Pipeline<T>();
    if (!Q) return FH_ERR_OOM;
    cudaStreamSynchronize(c->st);
    P->release();
    delete P;
    P = Q;
    rc = P->init(c->pb, 1, krylov, c->st, err, &best);
    if (rc) return from_rc(c, rc, err);
  } else {
    best = P->tuning;
    best_ms = before;
  }
  cache_store(tune_key(c->pb, 1, sizeof(T) == 8), best, best_ms);
  if (ms_after) *ms_after = best_ms;
  return FH_OK;
}
}  // namespace

extern "C" {

fh_status fh_autotune(fh_ctx* c, int dtype, double* ms_before, double* ms_after) {
  if (!c) return FH_ERR_ARG;
  if (dtype == FH_FP32 && c->p32) return autotune_one<float>(c, c->p32, true, ms_before, ms_after);
  if (dtype == FH_FP64 && c->p64 && c->p64->x[0])
    return autotune_one<double>(c, c->p64, true, ms_before, ms_after);
  return fail(c, FH_ERR_ARG, "no Krylov pipeline of that precision in this context");
}

fh_status fh_autotune_loads(fh_ctx* c, double* ms_before, double* ms_after) {
  if (!c) return FH_ERR_ARG;
  if (c->precision == FH_FP64) return fail(c, FH_ERR_ARG, "the all-loads float32 pipeline needs FH_FP32 or FH_FP32_REFINED");
  const int d = c->pb.d;
  std::string err;
  // the default shapes' time, from a temporary pipeline
  double before = 0.0, t;
  {
    fh::Pipeline<float> P;
    int rc = P.init(c->pb, d, true, c->st, err);
    for (int what = 0; what < 4 && !rc; ++what) {
      rc = P.profile(what, 10, &t, err);
      before += t;
    }
    P.release();
    if (rc) return from_rc(c, rc, err);
  }
  Tuning best;
  double best_ms;
  int rc = fh::Pipeline<float>::autotune(c->pb, d, c->st, best, best_ms, err);
  if (rc) return from_rc(c, rc, err);
  cache_store(tune_key(c->pb, d, false), best, best_ms);
  // the next fh_solve_all rebuilds its pipelines with the tuned shapes
  fh::release_loads_group(c->loads_group);
  c->loads_group = nullptr;
  if (ms_before) *ms_before = before;
  if (ms_after) *ms_after = best_ms;
  return FH_OK;
}

fh_status fh_effective_column(fh_ctx* c, const double* e, double* col) {
  if (!c || !e || !col) return FH_ERR_ARG;
  std::string err;
  int rc;
  if (c->p64) {
    rc = c->p64->current_mean(e, col, err);
  } else {
    const long long len = (long long)c->pb.d * c->pb.nodes;
    ++c->own_launches;
    k_convert_vec<float><<<vec_grid(len), 256, 0, c->st>>>(e, c->p32->ap[0], len);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(c, ce, "convert");
    rc = c->p32->current_mean(c->p32->ap[0], col, err);
  }
  return from_rc(c, rc, err);
}

fh_status fh_eta_e(fh_ctx* c, const double* e, double* eta) {
  if (!c || !e || !eta) return FH_ERR_ARG;
  std::string err;
  int rc;
  if (c->p64) {
    rc = c->p64->eta_e(e, eta, err);
  } else {
    const long long len = (long long)c->pb.d * c->pb.nodes;
    ++c->own_launches;
    k_convert_vec<float><<<vec_grid(len), 256, 0, c->st>>>(e, c->p32->ap[0], len);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(c, ce, "convert");
    rc = c->p32->eta_e(c->p32->ap[0], eta, err);
  }
  return from_rc(c, rc, err);
}

}  // extern "C"

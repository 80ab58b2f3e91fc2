// fh_batch.cu -- many independent 2-D cells of uneven sizes solved together.
//
// Cells are grouped by grid size.  Every group is one pipeline whose kernels
// treat the group's cells as extra lines of one launch (per-cell dL tables,
// per-cell reference media, per-(cell, load) Krylov scalars; a cell whose
// loads have converged is skipped inside the kernels).  Each group iterates in
// its own CUDA-graph chunks on its own stream, so the groups run concurrently;
// the host polls every group's small scalar block once per round.
// Float32 inner solves with a float64 outer residual per (cell, load) follow
// the single-cell refinement of fh_solve.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/fh.h"
#include "fh_groups.h"
#include "fh_pipeline.cuh"

using fh::Pipeline;
using fh::Problem;
using fh::SolveResult;

namespace {

__global__ void kb_fill(double* x, long long nodes, int d, double e0, double e1, double e2) {
  const long long len = nodes * d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / nodes;
    x[i] = c == 0 ? e0 : (c == 1 ? e1 : e2);
  }
}
__global__ void kb_to_float(const double* in, float* out, long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void kb_add(double* x, const float* dx, long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    x[i] += (double)dx[i];
}
// Candidate launch shapes timed per size group by fh_batch_autotune (each
// candidate builds a full pipeline for the group, so the search is bounded).
constexpr int kBatchTuneCandidates = 48;

// Inner float32 solves stop as stalled after this many iterations without
// halving their residual (see the single-cell driver).
constexpr int kInnerStallWindow = 100;
// absolute residual (relative to |E|) at which the first float32 step hands
// over to the float64 outer residual
constexpr double kFirstEta = 1e-3;

int grid_for(long long len) {
  const long long g = (len + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(g, 2048));
}

struct Group {
  int N[2] = {0, 0};
  std::vector<int> cells;  // global cell ids, in batch order
  Problem pb;
  uint8_t* d_phase = nullptr;
  bool own_phase = true;
  cudaStream_t st = nullptr;
  Pipeline<float>* p32 = nullptr;
  Pipeline<double>* p64 = nullptr;
  double* x64[fh::kMaxLoads] = {};  // refinement iterate per load
  double* r64[fh::kMaxLoads] = {};
  long long launches0 = 0;
  fh::LoopCache loops32, loops64;  // device-side iteration loops of this group alone
};

bool spd2(const double* A) {
  const double s = std::fmax(std::fabs(A[0]), std::fmax(std::fabs(A[1]), std::fabs(A[3])));
  if (!(s > 0.0) || !std::isfinite(s)) return false;
  if (std::fabs(A[1] - A[2]) > 1e-12 * s) return false;
  return A[0] > 0.0 && A[0] * A[3] - A[1] * A[2] > 1e-14 * s * s;
}

void eig2(const double* A, double& lo, double& hi) {
  const double tr = A[0] + A[3], det = A[0] * A[3] - A[1] * A[2];
  const double disc = std::sqrt(std::fmax(0.0, 0.25 * tr * tr - det));
  lo = 0.5 * tr - disc;
  hi = 0.5 * tr + disc;
}

}  // namespace

struct fh_batch {
  int ncells = 0;
  int nloads = 0;
  int precision = FH_FP32_REFINED;
  std::vector<Group> groups;
  std::string err;
  long long own_launches = 0;
  fh::LoopCache loops32, loops64;  // device-side iteration loops over all groups
};

extern "C" {

void fh_batch_destroy(fh_batch* b) {
  if (!b) return;
  for (Group& g : b->groups)
    if (g.st) cudaStreamSynchronize(g.st);
  b->loops32.clear();
  b->loops64.clear();
  for (Group& g : b->groups) {
    g.loops32.clear();
    g.loops64.clear();
    if (g.p32) {
      g.p32->release();
      delete g.p32;
    }
    if (g.p64) {
      g.p64->release();
      delete g.p64;
    }
    for (int l = 0; l < fh::kMaxLoads; ++l) {
      if (g.x64[l]) cudaFree(g.x64[l]);
      if (g.r64[l]) cudaFree(g.r64[l]);
    }
    if (g.d_phase && g.own_phase) cudaFree(g.d_phase);
    if (g.st) cudaStreamDestroy(g.st);
  }
  delete b;
}

fh_status fh_batch_create(fh_batch** out, int ncells, const int* N, const uint8_t* const* phase,
                          const int* nphase, const double* const* L, int nloads, int precision) {
  if (!out) return FH_ERR_ARG;
  *out = nullptr;
  if (ncells < 1 || !N || !phase || !nphase || !L || nloads < 1 || nloads > 2) return FH_ERR_ARG;
  if (precision != FH_FP64 && precision != FH_FP32_REFINED) return FH_ERR_ARG;
  std::map<std::pair<int, int>, int> gid;
  fh_batch* b = new (std::nothrow) fh_batch();
  if (!b) return FH_ERR_OOM;
  b->ncells = ncells;
  b->nloads = nloads;
  b->precision = precision;
  for (int c = 0; c < ncells; ++c) {
    const int n0 = N[2 * c], n1 = N[2 * c + 1];
    if (n0 < 3 || n1 < 3 || !phase[c] || !L[c] || nphase[c] < 1 || nphase[c] > 256) {
      fh_batch_destroy(b);
      return FH_ERR_ARG;
    }
    for (int p = 0; p < nphase[c]; ++p)
      if (!spd2(L[c] + 4 * p)) {
        fh_batch_destroy(b);
        return FH_ERR_NOT_SPD;
      }
    auto key = std::make_pair(n0, n1);
    auto it = gid.find(key);
    if (it == gid.end()) {
      gid[key] = (int)b->groups.size();
      b->groups.emplace_back();
      b->groups.back().N[0] = n0;
      b->groups.back().N[1] = n1;
      it = gid.find(key);
    }
    b->groups[it->second].cells.push_back(c);
  }
  for (Group& g : b->groups) {
    const int nc = (int)g.cells.size();
    const long long cn = (long long)g.N[0] * g.N[1];
    int np = 1;
    for (int c : g.cells) np = std::max(np, nphase[c]);
    Problem& pb = g.pb;
    pb.d = 2;
    pb.N[0] = g.N[0];
    pb.N[1] = g.N[1];
    pb.nodes = cn * nc;
    pb.nphase = np;
    pb.ncell = nc;
    pb.L.assign((size_t)nc * np * 4, 0.0);
    pb.dL.assign((size_t)nc * np * 4, 0.0);
    pb.L0cell.assign((size_t)nc * 9, 0.0);
    for (int k = 0; k < nc; ++k) {
      const int c = g.cells[k];
      double lo = 1e300, hi = -1e300;
      for (int p = 0; p < nphase[c]; ++p) {
        double a, bb;
        eig2(L[c] + 4 * p, a, bb);
        lo = std::fmin(lo, a);
        hi = std::fmax(hi, bb);
      }
      const double l0 = 0.5 * (lo + hi);  // Eq. (opt_ref) per cell
      pb.L0cell[9 * k + 0] = l0;
      pb.L0cell[9 * k + 4] = l0;
      for (int p = 0; p < np; ++p) {
        const double* src = L[c] + 4 * std::min(p, nphase[c] - 1);
        for (int i = 0; i < 4; ++i) {
          pb.L[((size_t)k * np + p) * 4 + i] = src[i];
          pb.dL[((size_t)k * np + p) * 4 + i] = src[i] - (i == 0 || i == 3 ? l0 : 0.0);
        }
      }
    }
    pb.L0 = {pb.L0cell[0], 0.0, 0.0, pb.L0cell[4]};
    cudaError_t e = cudaStreamCreate(&g.st);
    if (e == cudaSuccess) e = cudaMalloc(&g.d_phase, pb.nodes);
    if (e != cudaSuccess) {
      fh_batch_destroy(b);
      return FH_ERR_OOM;
    }
    for (int k = 0; k < nc; ++k) {
      const uint8_t* src = phase[g.cells[k]];
      for (long long i = 0; i < cn; ++i)
        if (src[i] >= nphase[g.cells[k]]) {
          fh_batch_destroy(b);
          return FH_ERR_ARG;
        }
      e = cudaMemcpy(g.d_phase + (size_t)k * cn, src, cn, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        fh_batch_destroy(b);
        return FH_ERR_CUDA;
      }
    }
    pb.d_phase = g.d_phase;
    std::string err;
    int rc = 0;
    g.p64 = new (std::nothrow) Pipeline<double>();
    if (!g.p64) rc = FH_ERR_OOM;
    if (!rc) rc = g.p64->init(pb, nloads, precision == FH_FP64, g.st, err);
    if (!rc && precision == FH_FP32_REFINED) {
      g.p32 = new (std::nothrow) Pipeline<float>();
      if (!g.p32) rc = FH_ERR_OOM;
      if (!rc) rc = g.p32->init(pb, nloads, true, g.st, err);
    }
    for (int l = 0; l < nloads && !rc; ++l) {
      if (cudaMalloc(&g.x64[l], 2 * pb.nodes * sizeof(double)) != cudaSuccess ||
          cudaMalloc(&g.r64[l], 2 * pb.nodes * sizeof(double)) != cudaSuccess)
        rc = FH_ERR_OOM;
    }
    if (rc) {
      b->err = err;
      fh_batch_destroy(b);
      return (fh_status)rc;
    }
  }
  *out = b;
  return FH_OK;
}

fh_status fh_batch_autotune(fh_batch* b, double* ms_before, double* ms_after) {
  if (!b) return FH_ERR_ARG;
  double before = 0.0, after = 0.0;
  for (Group& g : b->groups) {
    if (!g.p32) continue;  // float64 batches keep their default shapes
    std::string err;
    double t, cur = 0.0;
    for (int what = 0; what < 4; ++what) {
      int rc = g.p32->profile(what, 10, &t, err);
      if (rc) {
        b->err = err;
        return (fh_status)rc;
      }
      cur += t;
    }
    fh::Tuning best;
    double best_ms;
    int rc = Pipeline<float>::autotune(g.pb, b->nloads, g.st, best, best_ms, err, kBatchTuneCandidates);
    if (rc) {
      b->err = err;
      return (fh_status)rc;
    }
    before += cur;
    if (best_ms < cur && !(best == g.p32->tuning)) {
      cudaStreamSynchronize(g.st);
      g.p32->release();
      *g.p32 = Pipeline<float>();
      rc = g.p32->init(g.pb, b->nloads, true, g.st, err, &best);
      if (rc) {
        // fall back to the default shapes
        g.p32->release();
        *g.p32 = Pipeline<float>();
        rc = g.p32->init(g.pb, b->nloads, true, g.st, err);
        if (rc) {
          b->err = err;
          return (fh_status)rc;
        }
        best_ms = cur;
      }
      after += best_ms;
    } else {
      after += cur;
    }
  }
  if (ms_before) *ms_before = before;
  if (ms_after) *ms_after = after;
  return FH_OK;
}

const char* fh_batch_last_error(const fh_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"

namespace {

// Solve every (cell, load) of every group (any dimension; groups of several
// cells are 2-D).  Ev[l] is load l.  Results per group gi, item = k * nl + l:
// st (kConverged / kBreakdown / kCap), its (inner iterations), rel (float64
// true relative residual); x64[l] of each group holds the solution fields.
fh_status solve_groups(std::vector<Group*>& groups, int d, int nl, const double (*Ev)[fh::kMaxD],
                       double tol, int method, int max_iter, int precision,
                       std::vector<std::vector<int>>& st, std::vector<std::vector<int>>& its,
                       std::vector<std::vector<double>>& rel, int& outer, long long& own_launches,
                       fh::LoopCache& loops32, fh::LoopCache& loops64, std::string& err) {
  double e2[fh::kMaxLoads] = {};
  for (int l = 0; l < nl; ++l)
    for (int a = 0; a < d; ++a) e2[l] += Ev[l][a] * Ev[l][a];
  auto fail = [&](int rc) { return (fh_status)rc; };
  const int ng = (int)groups.size();
  st.assign(ng, {});
  its.assign(ng, {});
  rel.assign(ng, {});
  for (int gi = 0; gi < ng; ++gi) {
    const int items = (int)(*groups[gi]).cells.size() * nl;
    st[gi].assign(items, fh::kRunning);
    its[gi].assign(items, 0);
    rel[gi].assign(items, INFINITY);
  }
  outer = 0;

  if (precision == FH_FP64) {
    for (Group* gp : groups) {
      Group& g = *gp;
      int rc = g.p64->solve_begin(method, Ev, false, fh::kX0Const, nullptr, tol, max_iter, err);
      if (rc) return fail(rc);
    }
    // every group's iterations in one graph launch (a while node per group)
    std::vector<Pipeline<double>*> ps;
    for (Group* gp : groups) ps.push_back(gp->p64);
    int rc = fh::run_loops<double>(ps.data(), ng, groups[0]->st, loops64, err);
    if (rc) return fail(rc);
    for (int gi = 0; gi < ng; ++gi) {
      Group& g = *groups[gi];
      std::vector<SolveResult> res(g.cells.size() * nl);
      g.p64->solve_results(res.data());
      // true residual per item
      std::vector<double> rr(res.size());
      const double* xin[fh::kMaxLoads];
      double* rout[fh::kMaxLoads];
      for (int l = 0; l < nl; ++l) {
        xin[l] = g.p64->x[l];
        rout[l] = g.r64[l];
      }
      int rc = g.p64->residual(xin, rout, false, Ev, rr.data(), err);
      if (rc) return fail(rc);
      const long long cn = g.pb.nodes / g.pb.ncell;
      for (size_t it = 0; it < res.size(); ++it) {
        const int l = (int)(it % nl);
        rel[gi][it] = std::sqrt(rr[it] / std::max(e2[l] * cn, 1e-300));
        its[gi][it] = res[it].iters;
        st[gi][it] = (res[it].status == fh::kConverged && rel[gi][it] <= tol) ? fh::kConverged
                     : res[it].status == fh::kBreakdown                       ? fh::kBreakdown
                                                                              : fh::kCap;
      }
      for (int l = 0; l < nl; ++l)
        cudaMemcpyAsync(g.x64[l], g.p64->x[l], (long long)d * g.pb.nodes * sizeof(double), cudaMemcpyDeviceToDevice,
                        g.st);
    }
  } else {
    // float32 inner solves, float64 outer residual per (cell, load)
    for (Group* gp : groups)
      for (int l = 0; l < nl; ++l) {
        Group& g = *gp;
        ++own_launches;
        kb_fill<<<grid_for((long long)d * g.pb.nodes), 256, 0, g.st>>>(g.x64[l], g.pb.nodes, d, Ev[l][0], Ev[l][1], Ev[l][2]);
      }
    std::vector<std::vector<double>> prev(ng);
    for (int gi = 0; gi < ng; ++gi) prev[gi].assign(st[gi].size(), INFINITY);
    for (;;) {
      bool any = false;
      std::vector<std::vector<double>> eta(ng);
      for (int gi = 0; gi < ng; ++gi) {
        Group& g = *groups[gi];
        std::vector<double> rr(st[gi].size());
        const double* xin[fh::kMaxLoads];
        double* rout[fh::kMaxLoads];
        for (int l = 0; l < nl; ++l) {
          xin[l] = g.x64[l];
          rout[l] = g.r64[l];
        }
        // float64-accuracy residual; its Green pass runs in double-float
        int rc = g.p64->residual(xin, rout, false, Ev, rr.data(), err, true);
        if (rc) return fail(rc);
        const long long cn = g.pb.nodes / g.pb.ncell;
        eta[gi].assign(st[gi].size(), 1.0);
        for (size_t it = 0; it < rr.size(); ++it) {
          const int l = (int)(it % nl);
          if (st[gi][it] != fh::kRunning) continue;
          const double r = std::sqrt(rr[it] / std::max(e2[l] * cn, 1e-300));
          rel[gi][it] = r;
          if (!std::isfinite(r)) {
            st[gi][it] = fh::kBreakdown;
          } else if (r <= tol) {
            st[gi][it] = fh::kConverged;
          } else if (its[gi][it] >= max_iter || (outer > 0 && !(r < 0.9 * prev[gi][it]))) {
            st[gi][it] = fh::kCap;
          } else {
            // the first step stops at an absolute residual of kFirstEta |E|
            // (float32 CG tracks float64 CG that far), later steps aim a little
            // past tol
            double e = 0.3 * tol / r;
            if (outer == 0) e = std::max(e, kFirstEta / r);
            eta[gi][it] = std::min(0.1, std::max(2e-6, e));
            any = true;
          }
          prev[gi][it] = r;
        }
      }
      if (!any) break;
      int budget = 0;
      for (int gi = 0; gi < ng; ++gi)
        for (size_t it = 0; it < its[gi].size(); ++it)
          if (st[gi][it] == fh::kRunning) budget = std::max(budget, max_iter - its[gi][it]);
      // inner solves of every group, all iterations in one graph launch
      std::vector<bool> active(ng, false);
      for (int gi = 0; gi < ng; ++gi) {
        Group& g = *groups[gi];
        bool need = false;
        for (size_t it = 0; it < st[gi].size(); ++it) need = need || st[gi][it] == fh::kRunning;
        if (!need) continue;
        active[gi] = true;
        for (int l = 0; l < nl; ++l) {
          ++own_launches;
          kb_to_float<<<grid_for((long long)d * g.pb.nodes), 256, 0, g.st>>>(g.r64[l], g.p32->rhs[l], (long long)d * g.pb.nodes);
        }
        int x0 = fh::kX0Rhs;
        if (method != FH_FIXED_POINT) {
          // start at the exact complement part of the correction, d0 = (I - Q) r
          int rc0 = g.p32->project_complement(g.p32->rhs, g.p32->x, err);
          if (rc0) return fail(rc0);
          x0 = fh::kX0Keep;
        }
        int rc = g.p32->solve_begin(method, Ev, true, x0, nullptr, 1.0, budget, err, eta[gi].data(),
                                    kInnerStallWindow);
        if (rc) return fail(rc);
      }
      {
        std::vector<Pipeline<float>*> ps;
        for (int gi = 0; gi < ng; ++gi)
          if (active[gi]) ps.push_back(groups[gi]->p32);
        if (!ps.empty()) {
          int rc = fh::run_loops<float>(ps.data(), (int)ps.size(), ps[0]->st, loops32, err);
          if (rc) return fail(rc);
        }
      }
      for (int gi = 0; gi < ng; ++gi) {
        Group& g = *groups[gi];
        std::vector<SolveResult> res(st[gi].size());
        g.p32->solve_results(res.data());
        for (size_t it = 0; it < res.size(); ++it)
          if (st[gi][it] == fh::kRunning) its[gi][it] += res[it].iters;
        for (int l = 0; l < nl; ++l) {
          ++own_launches;
          kb_add<<<grid_for((long long)d * g.pb.nodes), 256, 0, g.st>>>(g.x64[l], g.p32->x[l], (long long)d * g.pb.nodes);
        }
      }
      ++outer;
    }
  }
  return FH_OK;
}

}  // namespace

extern "C" {

fh_status fh_batch_solve(fh_batch* b, const double* E, double tol, int method, int max_iter,
                         double* Leff, int* status, int* iters, fh_info* summary) {
  if (!b || !E || !Leff || !(tol > 0.0) || max_iter < 0 || method < FH_CG || method > FH_FIXED_POINT)
    return FH_ERR_ARG;
  const int nl = b->nloads;
  double Ev[fh::kMaxLoads][fh::kMaxD] = {};
  for (int l = 0; l < nl; ++l) {
    Ev[l][0] = E[2 * l];
    Ev[l][1] = E[2 * l + 1];
    if (!std::isfinite(Ev[l][0]) || !std::isfinite(Ev[l][1])) return FH_ERR_ARG;
  }
  std::vector<Group*> groups;
  for (Group& g : b->groups) groups.push_back(&g);
  const int ng = (int)groups.size();
  long long launches0 = b->own_launches;
  for (Group* g : groups) launches0 += g->p64->launches + (g->p32 ? g->p32->launches : 0);
  std::vector<std::vector<int>> st, its;
  std::vector<std::vector<double>> rel;
  int outer = 0;
  std::string err;
  fh_status rs = solve_groups(groups, 2, nl, Ev, tol, method, max_iter, b->precision, st, its, rel, outer,
                              b->own_launches, b->loops32, b->loops64, err);
  if (rs != FH_OK) {
    b->err = err;
    return rs;
  }
  double worst = 0.0;
  // effective tensor columns per cell and load (float64)
  for (int gi = 0; gi < ng; ++gi) {
    Group& g = b->groups[gi];
    const int nc = (int)g.cells.size();
    std::vector<double> col((size_t)nc * 2);
    for (int l = 0; l < nl; ++l) {
      int rc = g.p64->current_mean(g.x64[l], col.data(), err);
      if (rc) {
        b->err = err;
        return (fh_status)rc;
      }
      for (int k = 0; k < nc; ++k) {
        const int c = g.cells[k];
        for (int a = 0; a < 2; ++a) Leff[((size_t)c * 2 + a) * nl + l] = col[2 * k + a];
        const int it = k * nl + l;
        if (status) status[(size_t)c * nl + l] = st[gi][it] == fh::kConverged ? FH_OK
                                                : st[gi][it] == fh::kBreakdown  ? FH_ERR_BREAKDOWN
                                                                                : FH_ERR_NOT_CONVERGED;
        if (iters) iters[(size_t)c * nl + l] = its[gi][it];
        worst = std::max(worst, rel[gi][it]);
      }
    }
  }
  fh_status first = FH_OK;
  for (int gi = 0; gi < ng; ++gi)
    for (int s2 : st[gi])
      if (first == FH_OK && s2 != fh::kConverged)
        first = s2 == fh::kBreakdown ? FH_ERR_BREAKDOWN : FH_ERR_NOT_CONVERGED;
  if (summary) {
    long long total = 0;
    for (auto& v : its)
      for (int x : v) total += x;
    long long launches = b->own_launches;
    for (Group& g : b->groups) launches += g.p64->launches + (g.p32 ? g.p32->launches : 0);
    summary->iters = (int)std::min<long long>(total, 2147483647LL);
    summary->outer_iters = outer;
    summary->matvecs = 0;
    summary->status = first;
    summary->rel_res_true = worst;
    summary->rel_res = NAN;
    summary->eta_r = NAN;
    summary->eta_e = NAN;
    summary->history_len = 0;
    summary->launches = launches - launches0;
    summary->ct_plans = 0;
    if (method == FH_CG)
      for (Group& g : b->groups)
        if (g.p32) summary->ct_plans |= fh::ct_plan_bit(g.p32->ct_plan);
  }
  for (Group& g : b->groups)
    if (cudaStreamSynchronize(g.st) != cudaSuccess) return FH_ERR_CUDA;
  return first;
}

}  // extern "C"

namespace fh {

void release_loads_group(void* cache) {
  Group* g = static_cast<Group*>(cache);
  if (!g) return;
  if (g->st) cudaStreamSynchronize(g->st);
  g->loops32.clear();
  g->loops64.clear();
  if (g->p32) {
    g->p32->release();
    delete g->p32;
  }
  if (g->p64) {
    g->p64->release();
    delete g->p64;
  }
  for (int l = 0; l < kMaxLoads; ++l) {
    if (g->x64[l]) cudaFree(g->x64[l]);
    if (g->r64[l]) cudaFree(g->r64[l]);
  }
  if (g->st) cudaStreamDestroy(g->st);
  delete g;
}

int solve_all_loads(const Problem& pb, int precision, double tol, int method, int max_iter,
                    double* Leff, LoadsResult& res, void** cache, std::string& err) {
  const int d = pb.d;
  Group* g = static_cast<Group*>(*cache);
  if (!g) {
    g = new (std::nothrow) Group();
    if (!g) return FH_ERR_OOM;
    g->pb = pb;
    g->d_phase = const_cast<uint8_t*>(pb.d_phase);
    g->own_phase = false;
    g->cells = {0};
    int rc = 0;
    if (cudaStreamCreate(&g->st) != cudaSuccess) rc = FH_ERR_CUDA;
    if (!rc) {
      g->p64 = new (std::nothrow) Pipeline<double>();
      rc = g->p64 ? g->p64->init(pb, d, precision == FH_FP64, g->st, err) : FH_ERR_OOM;
    }
    if (!rc && precision != FH_FP64) {
      g->p32 = new (std::nothrow) Pipeline<float>();
      if (!g->p32) {
        rc = FH_ERR_OOM;
      } else {
        // launch shapes tuned for d loads per launch (fh_autotune_loads), else the defaults
        Tuning t;
        rc = -1;
        if (tuning_from_cache(pb, d, false, t)) {
          rc = g->p32->init(pb, d, true, g->st, err, &t);
          if (rc) {
            g->p32->release();
            *g->p32 = Pipeline<float>();
          }
        }
        if (rc) rc = g->p32->init(pb, d, true, g->st, err);
      }
    }
    for (int l = 0; l < d && !rc; ++l)
      if (cudaMalloc(&g->x64[l], (size_t)d * pb.nodes * sizeof(double)) != cudaSuccess ||
          cudaMalloc(&g->r64[l], (size_t)d * pb.nodes * sizeof(double)) != cudaSuccess)
        rc = FH_ERR_OOM;
    if (rc) {
      release_loads_group(g);
      return rc;
    }
    *cache = g;
  }
  double Ev[kMaxLoads][kMaxD] = {};
  for (int l = 0; l < d; ++l) Ev[l][l] = 1.0;
  std::vector<Group*> groups = {g};
  std::vector<std::vector<int>> st, its;
  std::vector<std::vector<double>> rel;
  long long own = 0;
  const long long l0 = g->p64->launches + (g->p32 ? g->p32->launches : 0);
  fh_status rs = solve_groups(groups, d, d, Ev, tol, method, max_iter,
                              precision == FH_FP64 ? FH_FP64 : FH_FP32_REFINED, st, its, rel, res.outer,
                              own, g->loops32, g->loops64, err);
  if (rs != FH_OK) return rs;
  std::vector<double> col(d);
  for (int l = 0; l < d; ++l) {
    int rc = g->p64->current_mean(g->x64[l], col.data(), err);
    if (rc) return rc;
    for (int a = 0; a < d; ++a) Leff[a * d + l] = col[a];
    res.status[l] = st[0][l] == kConverged ? FH_OK : st[0][l] == kBreakdown ? FH_ERR_BREAKDOWN
                                                                           : FH_ERR_NOT_CONVERGED;
    res.iters[l] = its[0][l];
    res.rel[l] = rel[0][l];
  }
  res.launches = own + g->p64->launches + (g->p32 ? g->p32->launches : 0) - l0;
  res.ct_plans = (method == FH_CG && g->p32) ? ct_plan_bit(g->p32->ct_plan) : 0;
  if (cudaStreamSynchronize(g->st) != cudaSuccess) return FH_ERR_CUDA;
  return 0;
}

}  // namespace fh

// fh_plan.h -- host-side planning: FFT radix schedules, pass tilings and
// float64 twiddle tables.  Pure host code (no CUDA calls).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "fh_fft.cuh"

namespace fh {

// Radices compiled into the stage dispatchers (must match FH_FOR_EACH_RADIX
// and FH_FOR_EACH_RADIX_X).  The extended radices (powers of 2 up to 16, and
// the primes 11, 13 and 17) are used only by lengths that have one of 2, 11,
// 13, 17 as a factor; those plans run the DynPlanX kernels with the register
// budget RegBudgetX.
inline const std::vector<int>& compiled_radices() {
  static const std::vector<int> r = {27, 25, 17, 16, 15, 13, 11, 9, 8, 7, 5, 4, 3, 2};
  return r;
}

inline int reg_budget(bool fp64) { return fp64 ? RegBudget<double>::value : RegBudget<float>::value; }
inline int reg_budget_x(bool fp64) { return fp64 ? RegBudgetX<double>::value : RegBudgetX<float>::value; }

// Does n factor into the supported primes 2, 3, 5, 7, 11, 13, 17?  ext is
// set when one of 2, 11, 13, 17 divides n (the extended radix set).
inline bool factorable(int n, bool& ext) {
  ext = false;
  if (n < 1) return false;
  for (int p : {2, 3, 5, 7, 11, 13, 17}) {
    while (n % p == 0) {
      n /= p;
      if (p == 2 || p > 7) ext = true;
    }
  }
  return n == 1;
}

// Minimum-stage radix schedule for length n when each sequence is worked on
// by tpl threads: a stage of radix R is allowed iff every thread holds at most
// floor(budget / R) butterflies, i.e. ceil(n / R / tpl) * R <= budget.
// Returns the stage list (empty if impossible).  Radices are emitted largest
// first.  Dynamic programme over the divisors m of n: best[m] is a shortest
// list of allowed radices whose product is m.
inline std::vector<int> plan_radices(int n, int tpl, int budget) {
  bool ext;
  if (!factorable(n, ext)) return {};
  std::vector<int> allowed;
  for (int R : compiled_radices()) {
    if (n % R) continue;
    const int bmax = budget / R;
    if (bmax < 1) continue;
    const int need = (n / R + tpl - 1) / tpl;
    if (need > bmax) continue;
    allowed.push_back(R);
  }
  std::vector<int> divs;
  for (int m = 1; m <= n; ++m)
    if (n % m == 0) divs.push_back(m);  // ascending
  std::map<int, std::vector<int>> best;
  best[1] = {};
  for (int m : divs) {
    if (m == 1) continue;
    bool found = false;
    std::vector<int> cand;
    for (int R : allowed) {
      if (m % R) continue;
      auto it = best.find(m / R);
      if (it == best.end()) continue;
      if (!found || it->second.size() + 1 < cand.size()) {
        cand = it->second;
        cand.push_back(R);
        found = true;
      }
    }
    if (found) best[m] = cand;
  }
  auto it = best.find(n);
  if (it == best.end()) return {};
  std::vector<int> r = it->second;
  std::sort(r.begin(), r.end(), [](int u, int v) { return u > v; });
  return r;
}

// Choose (tpl, radices): fewest stages first, then the fewest threads per
// sequence (more butterflies per thread, more independent work in flight).
// Even lengths and lengths with a prime factor 11, 13 or 17 get an extended
// plan (pl.ext = 1).
inline bool make_fft_plan(int n, bool fp64, int max_tpl, FFTPlan& pl, int& tpl,
                          int force_tpl = 0) {
  bool ext;
  if (!factorable(n, ext)) return false;
  const int budget = ext ? reg_budget_x(fp64) : reg_budget(fp64);
  int best_stages = 1 << 30, best_tpl = 0;
  std::vector<int> best_r;
  for (int t = 1; t <= max_tpl; ++t) {
    if (force_tpl && t != force_tpl) continue;
    std::vector<int> r = plan_radices(n, t, budget);
    if (r.empty()) continue;
    if ((int)r.size() < best_stages) {
      best_stages = (int)r.size();
      best_tpl = t;
      best_r = r;
    }
  }
  if (best_r.empty() || (int)best_r.size() > kMaxStages) return false;
  pl.n = n;
  pl.nstages = (int)best_r.size();
  for (int s = 0; s < kMaxStages; ++s) pl.radix[s] = s < pl.nstages ? best_r[s] : 0;
  pl.ext = ext ? 1 : 0;
  tpl = best_tpl;
  return true;
}

// exp(-2 pi i m / n) for m in [0, n), float64.  The angle is reduced exactly
// on the rational m / n (octant symmetry) before calling the C library, so
// every entry is within an ulp or two of the true value.
inline void twiddles(int n, std::vector<double>& re, std::vector<double>& im) {
  re.resize(n);
  im.resize(n);
  for (int m = 0; m < n; ++m) {
    ct::cs v;
    // reuse the exact rational reduction, then evaluate with std::cos/sin
    long long num = 8LL * m, den = n;
    double sgn_s = 1.0, sgn_c = 1.0;
    bool swap = false;
    if (2 * num >= 8 * den) { num = 8 * den - num; sgn_s = -1.0; }
    if (2 * num > 4 * den) { num = 4 * den - num; sgn_c = -1.0; }
    if (num > den) { num = 2 * den - num; swap = true; }
    const double x = (ct::kPi / 4.0) * (double)num / (double)den;
    v.c = std::cos(x);
    v.s = std::sin(x);
    if (swap) std::swap(v.c, v.s);
    re[m] = sgn_c * v.c;
    im[m] = -(sgn_s * v.s);  // forward sign
  }
}

}  // namespace fh

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

// Radices compiled into the stage dispatcher (must match FH_FOR_EACH_RADIX).
inline const std::vector<int>& compiled_radices() {
  static const std::vector<int> r = {27, 25, 15, 9, 7, 5, 3};
  return r;
}

inline int reg_budget(bool fp64) { return fp64 ? RegBudget<double>::value : RegBudget<float>::value; }

// Factor n = 3^a 5^b 7^c; returns false if another prime divides n.
inline bool factor357(int n, int& a, int& b, int& c) {
  a = b = c = 0;
  if (n < 1) return false;
  while (n % 3 == 0) { n /= 3; ++a; }
  while (n % 5 == 0) { n /= 5; ++b; }
  while (n % 7 == 0) { n /= 7; ++c; }
  return n == 1;
}

// Minimum-stage radix schedule for length n when each sequence is worked on
// by tpl threads: a stage of radix R is allowed iff every thread holds at most
// floor(budget / R) butterflies, i.e. ceil(n / R / tpl) * R <= budget.
// Returns the stage list (empty if impossible).  Radices are emitted largest
// first.
inline std::vector<int> plan_radices(int n, int tpl, int budget) {
  int a, b, c;
  if (!factor357(n, a, b, c)) return {};
  std::vector<std::tuple<int, int, int, int>> allowed;  // (R, i, j, k)
  for (int R : compiled_radices()) {
    if (n % R) continue;
    const int bmax = budget / R;
    if (bmax < 1) continue;
    const int need = (n / R + tpl - 1) / tpl;
    if (need > bmax) continue;
    int i, j, k;
    factor357(R, i, j, k);
    allowed.emplace_back(R, i, j, k);
  }
  // DP over exponent vectors
  std::map<std::tuple<int, int, int>, std::vector<int>> best;
  best[{0, 0, 0}] = {};
  for (int x = 0; x <= a; ++x)
    for (int y = 0; y <= b; ++y)
      for (int z = 0; z <= c; ++z) {
        if (x == 0 && y == 0 && z == 0) continue;
        std::vector<int> cand;
        bool found = false;
        for (auto& t : allowed) {
          int R, i, j, k;
          std::tie(R, i, j, k) = t;
          if (i > x || j > y || k > z) continue;
          auto it = best.find({x - i, y - j, z - k});
          if (it == best.end()) continue;
          if (!found || it->second.size() + 1 < cand.size()) {
            cand = it->second;
            cand.push_back(R);
            found = true;
          }
        }
        if (found) best[{x, y, z}] = cand;
      }
  auto it = best.find({a, b, c});
  if (it == best.end()) return {};
  std::vector<int> r = it->second;
  std::sort(r.begin(), r.end(), [](int u, int v) { return u > v; });
  return r;
}

// Choose (tpl, radices): fewest stages first, then the fewest threads per
// sequence (more butterflies per thread, more independent work in flight).
inline bool make_fft_plan(int n, bool fp64, int max_tpl, FFTPlan& pl, int& tpl,
                          int force_tpl = 0) {
  const int budget = reg_budget(fp64);
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

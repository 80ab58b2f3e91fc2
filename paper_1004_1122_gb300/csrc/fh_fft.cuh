// fh_fft.cuh -- device FFT building blocks (radix 3, 5, 7 and their products;
// 2, 4, 8, 16, 11, 13 and 17 in the extended set for even lengths and the
// larger primes), float32, float64 and double-float (fh_dfloat.cuh).
//
// The discrete Fourier transform is the one of Eq. (DFT_def): forward
// X[k] = sum_m x[m] exp(-2 pi i k m / n), inverse with +i and no 1/n (the
// 1/|N| factor is applied once, in the Green-operator step).
//
// Structure:
//  * Butterfly constants cos/sin(2 pi a / b) are compile-time values computed
//    by an exact rational octant reduction followed by a Taylor series on
//    |x| <= pi/4 (our own constexpr routine; no math library involved).
//  * dft<R>() is an R-point DFT held entirely in registers.  Odd primes use
//    the symmetric form  X_k = x_0 + sum_j (x_j + x_{R-j}) cos - i (x_j - x_{R-j}) sin;
//    radix 2 the sum and difference; composite R = P*Q is the textbook
//    Cooley-Tukey split with inner twiddles.
//  * stage<R>() is one Stockham autosort pass over a sequence held in shared
//    memory: butterfly j reads x[j + r n/R], applies the twiddles
//    W_{Ns R}^{r (j mod Ns)}, transforms, and writes x[(j - j mod Ns) R + j mod Ns + r Ns]
//    (Ns = product of the radices already applied).  Stage twiddles come from
//    a per-length table tw[m] = exp(-2 pi i m / n) built on the host in
//    float64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "fh_dfloat.cuh"

namespace fh {

// ----------------------------------------------------------------------------
// complex helpers
// ----------------------------------------------------------------------------
template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<dfl> { using type = dfc; };
template <typename T> using cplx = typename cplx_t<T>::type;

// Read-only load of one stage twiddle.
template <typename C>
__device__ __forceinline__ C ld_tw(const C* p) { return __ldg(p); }
__device__ __forceinline__ dfc ld_tw(const dfc* p) {
  const float4 w = __ldg(reinterpret_cast<const float4*>(p));
  dfc r;
  r.x = dfl(w.x, w.y);
  r.y = dfl(w.z, w.w);
  return r;
}

template <typename T>
__device__ __forceinline__ cplx<T> cmk(T x, T y) { cplx<T> r; r.x = x; r.y = y; return r; }
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}

// ----------------------------------------------------------------------------
// compile-time trigonometry: cos / sin of 2 pi a / b for integers a, b > 0
// ----------------------------------------------------------------------------
namespace ct {
constexpr double kPi = 3.14159265358979323846264338327950288;

// Taylor series, valid for |x| <= pi/4 where 24 terms are far below 1e-17.
__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 24; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 24; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}

struct cs { double c, s; };

// Exact reduction of the angle 2 pi a / b to [0, pi/4] using the rational
// representation, then the series.  Symmetries used: 2 pi periodicity,
// theta -> 2pi - theta (sin flips), theta -> pi - theta (cos flips),
// theta -> pi/2 - theta (swap).
__host__ __device__ constexpr cs cossin2pi(long long a, long long b) {
  a %= b;
  if (a < 0) a += b;
  // angle = 2 pi a / b = (pi/4) * (8 a / b); work in units of pi/4: u = 8a / b
  long long num = 8 * a, den = b;  // u = num / den in [0, 8)
  double sgn_s = 1.0;
  if (2 * num >= 8 * den) { num = 8 * den - num; sgn_s = -1.0; }  // theta > pi: use 2pi - theta
  // now u in [0, 4] (theta in [0, pi])
  double sgn_c = 1.0;
  if (2 * num > 4 * den) { num = 4 * den - num; sgn_c = -1.0; }   // theta > pi/2: use pi - theta
  // now u in [0, 2] (theta in [0, pi/2])
  bool swap = false;
  if (num > den) { num = 2 * den - num; swap = true; }             // theta > pi/4: use pi/2 - theta
  double x = (kPi / 4.0) * (double)num / (double)den;
  double c = taylor_cos(x), s = taylor_sin(x);
  if (swap) { double t = c; c = s; s = t; }
  return cs{sgn_c * c, sgn_s * s};
}
__host__ __device__ constexpr double cos2pi(long long a, long long b) { return cossin2pi(a, b).c; }
__host__ __device__ constexpr double sin2pi(long long a, long long b) { return cossin2pi(a, b).s; }

__host__ __device__ constexpr int smallest_factor(int r) {
  for (int p = 2; p * p <= r; ++p)
    if (r % p == 0) return p;
  return r;
}
__host__ __device__ constexpr bool is_prime(int r) { return r > 1 && smallest_factor(r) == r; }
}  // namespace ct

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0 .. N-1, so
// that values derived from I inside f are constant expressions.
template <typename F, int... Is>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ----------------------------------------------------------------------------
// register DFTs
// ----------------------------------------------------------------------------
// R-point DFT on v[0], v[S], ..., v[(R-1)S]; natural order in and out.
// INV selects exp(+2 pi i ...).
template <int R, int S, bool INV, typename T> struct RegDFT;

template <int S, bool INV, typename T> struct RegDFT<1, S, INV, T> {
  static __device__ __forceinline__ void run(cplx<T>*) {}
};

template <int P, int S, bool INV, typename T, bool PRIME> struct RegDFTImpl;

// odd prime P: symmetric form
template <int P, int S, bool INV, typename T> struct RegDFTImpl<P, S, INV, T, true> {
  static __device__ __forceinline__ void run(cplx<T>* v) {
    static_assert(P % 2 == 1, "odd primes only");
    constexpr int h = (P - 1) / 2;
    using C = cplx<T>;
    C a[h + 1], b[h + 1];
#pragma unroll
    for (int j = 1; j <= h; ++j) {
      a[j] = cadd(v[j * S], v[(P - j) * S]);
      b[j] = csub(v[j * S], v[(P - j) * S]);
    }
    const C x0 = v[0];
    C sum = x0;
#pragma unroll
    for (int j = 1; j <= h; ++j) sum = cadd(sum, a[j]);
    static_for<h>([&](auto K) {
      constexpr int k = decltype(K)::value + 1;
      C re = x0, im;
      im.x = T(0);
      im.y = T(0);
      static_for<h>([&](auto J) {
        constexpr int j = decltype(J)::value + 1;
        constexpr double c = ct::cos2pi((long long)j * k, P);
        constexpr double s = ct::sin2pi((long long)j * k, P);
        re.x += a[j].x * T(c); re.y += a[j].y * T(c);
        im.x += b[j].x * T(s); im.y += b[j].y * T(s);
      });
      // forward: X_k = re - i im, X_{P-k} = re + i im; inverse swaps the signs
      C m1, p1;
      m1.x = re.x + im.y; m1.y = re.y - im.x;  // re - i*im
      p1.x = re.x - im.y; p1.y = re.y + im.x;  // re + i*im
      if (INV) { v[k * S] = p1; v[(P - k) * S] = m1; }
      else     { v[k * S] = m1; v[(P - k) * S] = p1; }
    });
    v[0] = sum;
  }
};

// radix 2 (even lengths): X_0 = x_0 + x_1, X_1 = x_0 - x_1 in either direction
template <int S, bool INV, typename T> struct RegDFTImpl<2, S, INV, T, true> {
  static __device__ __forceinline__ void run(cplx<T>* v) {
    const cplx<T> a = v[0], b = v[S];
    v[0] = cadd(a, b);
    v[S] = csub(a, b);
  }
};

// composite R = P * Q, P the smallest prime factor (decimation in time):
//   n = P n2 + n1, k = k1 + Q k2:
//   X[k1 + Q k2] = sum_n1 W_P^{n1 k2} W_R^{n1 k1} sum_n2 x[P n2 + n1] W_Q^{n2 k1}
template <int R, int S, bool INV, typename T> struct RegDFTImpl<R, S, INV, T, false> {
  static __device__ __forceinline__ void run(cplx<T>* v) {
    constexpr int P = ct::smallest_factor(R);
    constexpr int Q = R / P;
    using C = cplx<T>;
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) RegDFT<Q, P * S, INV, T>::run(v + n1 * S);
    static_for<P - 1>([&](auto N1) {
      constexpr int n1 = decltype(N1)::value + 1;
      static_for<Q - 1>([&](auto K1) {
        constexpr int k1 = decltype(K1)::value + 1;
        constexpr double c = ct::cos2pi((long long)n1 * k1, R);
        constexpr double s = ct::sin2pi((long long)n1 * k1, R);
        C w;
        w.x = T(c);
        w.y = T(INV ? s : -s);
        v[(n1 + P * k1) * S] = cmul(v[(n1 + P * k1) * S], w);
      });
    });
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) RegDFT<P, S, INV, T>::run(v + P * k1 * S);
    C tmp[R];
#pragma unroll
    for (int i = 0; i < R; ++i) tmp[i] = v[i * S];
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) {
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) v[(k1 + Q * k2) * S] = tmp[P * k1 + k2];
    }
  }
};

template <int R, int S, bool INV, typename T> struct RegDFT {
  static __device__ __forceinline__ void run(cplx<T>* v) {
    RegDFTImpl<R, S, INV, T, ct::is_prime(R)>::run(v);
  }
};

// ----------------------------------------------------------------------------
// Stockham stage in shared memory
// ----------------------------------------------------------------------------
// Per-thread register budget in complex elements, per precision.
template <typename T> struct RegBudget;
template <> struct RegBudget<float> { static constexpr int value = 27; };
template <> struct RegBudget<double> { static constexpr int value = 9; };
template <> struct RegBudget<dfl> { static constexpr int value = 9; };

// Sequence element i of the sequence this thread works on lives at
// sm[i * is].  u in [0, nthr) is the thread's rank within the sequence's
// thread group.  Every thread of the CTA must call this (it contains
// __syncthreads), with identical n / Ns across the CTA.  The register array v
// is shared by every radix variant of the caller's stage loop (one array,
// EM complex values), which keeps it in registers.
template <int R, bool INV, typename T, int EM>
__device__ __forceinline__ void stockham_stage(cplx<T> (&v)[EM], cplx<T>* sm, int is, int n, int Ns,
                                               int u, int nthr, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int BM = EM / R;
  static_assert(BM >= 1, "radix exceeds the register budget");
  const int nb = n / R;
  const int S = nb / Ns;
  const int in_step = nb * is, out_step = Ns * is;
  // j = u + b * nthr = q * Ns + k, advanced without divisions
  const int dq = nthr / Ns, dk = nthr - dq * Ns;
  int q0 = u / Ns;
  int k0 = u - q0 * Ns;
  int kb[BM], ob[BM];
  {
    int q = q0, k = k0;
#pragma unroll
    for (int b = 0; b < BM; ++b) {
      kb[b] = k;
      ob[b] = (q * R * Ns + k) * is;
      q += dq;
      k += dk;
      if (k >= Ns) { k -= Ns; ++q; }
    }
  }
#pragma unroll
  for (int b = 0; b < BM; ++b) {
    const int j = u + b * nthr;
    if (j < nb) {
      const C* src = sm + j * is;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b * R + r] = src[r * in_step];
      if (Ns > 1) {
        const int ks = kb[b] * S;
        int ti = ks;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const C w = ld_tw(tw + ti);
          ti += ks;
          v[b * R + r] = INV ? cmulc(v[b * R + r], w) : cmul(v[b * R + r], w);
        }
      }
      RegDFT<R, 1, INV, T>::run(&v[b * R]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BM; ++b) {
    const int j = u + b * nthr;
    if (j < nb) {
      C* dst = sm + ob[b];
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * out_step] = v[b * R + r];
    }
  }
  __syncthreads();
}

// Supported stage radices.  The plan stores them as small integers.
#define FH_FOR_EACH_RADIX(X) X(3) X(5) X(7) X(9) X(15) X(25) X(27)
// The extended set of the DynPlanX kernels: lengths with a factor 2 (even
// axes) or a prime factor 11, 13 or 17 (for example the 255 = 3 * 5 * 17 grid
// of the paper's Section 3).
#define FH_FOR_EACH_RADIX_X(X) \
  X(2) X(3) X(4) X(5) X(7) X(8) X(9) X(11) X(13) X(15) X(16) X(17) X(25) X(27)

// Largest prime radix of the extended set; every extended plan's register
// array holds at least one butterfly of it.
constexpr int kMaxPrimeX = 17;
template <typename T> struct RegBudgetX {
  static constexpr int value = RegBudget<T>::value > kMaxPrimeX ? RegBudget<T>::value : kMaxPrimeX;
};

// Maximum number of stages in a plan.
constexpr int kMaxStages = 12;

struct FFTPlan {
  int n;                    // sequence length
  int nstages;
  int radix[kMaxStages];
  int ext;                  // 1: uses a radix of the extended set (DynPlanX kernels)
};

// Run all stages of the plan on one sequence layout.  X selects the extended
// radix set (and its register budget).
template <bool INV, typename T, bool X = false>
__device__ __forceinline__ void run_fft(cplx<T>* sm, int is, const FFTPlan& pl, int u, int nthr,
                                        const cplx<T>* __restrict__ tw) {
  constexpr int EM = X ? RegBudgetX<T>::value : RegBudget<T>::value;
  cplx<T> v[EM];
  int Ns = 1;
  for (int s = 0; s < pl.nstages; ++s) {
    const int R = pl.radix[s];
#define FH_STAGE_CASE(RR)                                                      \
  case RR:                                                                     \
    if constexpr (RR <= EM) stockham_stage<RR, INV, T, EM>(v, sm, is, pl.n, Ns, u, nthr, tw); \
    break;
    if constexpr (X) {
      switch (R) {
        FH_FOR_EACH_RADIX_X(FH_STAGE_CASE)
        default: break;
      }
    } else {
      switch (R) {
        FH_FOR_EACH_RADIX(FH_STAGE_CASE)
        default: break;
      }
    }
#undef FH_STAGE_CASE
    Ns *= R;
  }
}

// Forward FFT, a pointwise operation in the frequency domain, and the inverse
// FFT, with the last forward stage and the first inverse stage fused in
// registers.  The inverse runs the forward radices in reverse order, so its
// first stage (Ns = 1) reads exactly the positions j + r n/R the last forward
// stage produced (Ns = n/R) and no shared-memory round trip or barrier pair is
// needed in between.  mid(v, i, active) maps the spectrum value at row i; it
// is called by every thread of the CTA for the same (b, r) sequence, so it may
// use warp shuffles (inactive threads pass active = false and garbage values).
template <int R, typename T, int EM, typename F>
__device__ __forceinline__ void fused_middle(cplx<T> (&v)[EM], cplx<T>* sm, int is, int n, int u, int nthr,
                                             const cplx<T>* __restrict__ tw, F& mid) {
  using C = cplx<T>;
  constexpr int BM = EM / R;
  const int nb = n / R;  // = Ns of the last forward stage
  const int in_step = nb * is;
#pragma unroll
  for (int b = 0; b < BM; ++b) {
    const int j = u + b * nthr;
    if (j < nb) {
      const C* src = sm + j * is;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b * R + r] = src[r * in_step];
      if (nb > 1) {
        int ti = j;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          v[b * R + r] = cmul(v[b * R + r], ld_tw(tw + ti));
          ti += j;
        }
      }
      RegDFT<R, 1, false, T>::run(&v[b * R]);
    }
  }
#pragma unroll
  for (int b = 0; b < BM; ++b) {
    const int j = u + b * nthr;
    const bool act = j < nb;
#pragma unroll
    for (int r = 0; r < R; ++r) v[b * R + r] = mid(v[b * R + r], j + r * nb, act);
    if (act) RegDFT<R, 1, true, T>::run(&v[b * R]);
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BM; ++b) {
    const int j = u + b * nthr;
    if (j < nb) {
      C* dst = sm + j * R * is;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * is] = v[b * R + r];
    }
  }
  __syncthreads();
}

template <typename T, typename F, bool X = false>
__device__ __forceinline__ void run_fft_fused(cplx<T>* sm, int is, const FFTPlan& pl, int u, int nthr,
                                              const cplx<T>* __restrict__ tw, F& mid) {
  constexpr int EM = X ? RegBudgetX<T>::value : RegBudget<T>::value;
  cplx<T> v[EM];
  const int S = pl.nstages;
  int Ns = 1;
#define FH_SWITCH(R, CASE)             \
  if constexpr (X) {                   \
    switch (R) {                       \
      FH_FOR_EACH_RADIX_X(CASE)        \
      default: break;                  \
    }                                  \
  } else {                             \
    switch (R) {                       \
      FH_FOR_EACH_RADIX(CASE)          \
      default: break;                  \
    }                                  \
  }
  for (int s = 0; s + 1 < S; ++s) {
#define FH_STAGE_CASE(RR)                                                                          \
  case RR:                                                                                         \
    if constexpr (RR <= EM) stockham_stage<RR, false, T, EM>(v, sm, is, pl.n, Ns, u, nthr, tw); \
    break;
    FH_SWITCH(pl.radix[s], FH_STAGE_CASE)
#undef FH_STAGE_CASE
    Ns *= pl.radix[s];
  }
#define FH_MID_CASE(RR)                                                              \
  case RR:                                                                           \
    if constexpr (RR <= EM) fused_middle<RR, T, EM>(v, sm, is, pl.n, u, nthr, tw, mid); \
    break;
  FH_SWITCH(pl.radix[S - 1], FH_MID_CASE)
#undef FH_MID_CASE
  Ns = pl.radix[S - 1];
  for (int s = S - 2; s >= 0; --s) {
#define FH_STAGE_CASE(RR)                                                                         \
  case RR:                                                                                        \
    if constexpr (RR <= EM) stockham_stage<RR, true, T, EM>(v, sm, is, pl.n, Ns, u, nthr, tw); \
    break;
    FH_SWITCH(pl.radix[s], FH_STAGE_CASE)
#undef FH_STAGE_CASE
    Ns *= pl.radix[s];
  }
#undef FH_SWITCH
}

// ----------------------------------------------------------------------------
// compile-time plans
// ----------------------------------------------------------------------------
// A plan fixed at compile time: the stage loop is unrolled, every stage size
// (n, Ns, n/R) is a constant, and only the radices of this plan are compiled
// into the kernel (the run-time dispatcher above instantiates every radix for
// both directions, which overflows the instruction cache of a busy SM).
struct DynPlan {};
// Run-time plan over the extended radix set (primes 11, 13, 17 as well).
struct DynPlanX {};

template <int... Rs> struct CPlan {
  static constexpr int S = sizeof...(Rs);
  static constexpr int r[S] = {Rs...};
  static constexpr int n = (Rs * ... * 1);
};

template <typename P> __host__ __device__ constexpr int cplan_prefix(int s) {
  int p = 1;
  for (int i = 0; i < s; ++i) p *= P::r[i];
  return p;
}
template <typename P> __host__ __device__ constexpr int cplan_suffix(int s) {
  int p = 1;
  for (int i = s; i < P::S; ++i) p *= P::r[i];
  return p;
}

// Does the run-time plan pl equal the compile-time plan P?
template <typename P> inline bool cplan_is(const FFTPlan& pl) {
  if (pl.n != P::n || pl.nstages != P::S) return false;
  for (int i = 0; i < P::S; ++i)
    if (pl.radix[i] != P::r[i]) return false;
  return true;
}

template <bool INV, typename T, typename P>
__device__ __forceinline__ void run_fft_ct(cplx<T>* sm, int is, int u, int nthr, const cplx<T>* __restrict__ tw) {
  constexpr int EM = RegBudget<T>::value;
  cplx<T> v[EM];
  static_for<P::S>([&](auto I) {
    constexpr int st = decltype(I)::value;
    constexpr int R = P::r[st];
    static_assert(R <= EM, "radix exceeds the register budget");
    stockham_stage<R, INV, T, EM>(v, sm, is, P::n, cplan_prefix<P>(st), u, nthr, tw);
  });
}

template <typename T, typename P, typename F>
__device__ __forceinline__ void run_fft_fused_ct(cplx<T>* sm, int is, int u, int nthr,
                                                 const cplx<T>* __restrict__ tw, F& mid) {
  constexpr int EM = RegBudget<T>::value;
  cplx<T> v[EM];
  static_for<P::S - 1>([&](auto I) {
    constexpr int st = decltype(I)::value;
    stockham_stage<P::r[st], false, T, EM>(v, sm, is, P::n, cplan_prefix<P>(st), u, nthr, tw);
  });
  fused_middle<P::r[P::S - 1], T, EM>(v, sm, is, P::n, u, nthr, tw, mid);
  static_for<P::S - 1>([&](auto I) {
    constexpr int st = P::S - 2 - decltype(I)::value;
    stockham_stage<P::r[st], true, T, EM>(v, sm, is, P::n, cplan_suffix<P>(st + 1), u, nthr, tw);
  });
}

// Dispatch on the plan kind: DynPlan uses the run-time plan pl.
template <bool INV, typename T, typename P>
__device__ __forceinline__ void fft_plan(cplx<T>* sm, int is, const FFTPlan& pl, int u, int nthr,
                                         const cplx<T>* __restrict__ tw) {
  if constexpr (std::is_same<P, DynPlan>::value)
    run_fft<INV, T, false>(sm, is, pl, u, nthr, tw);
  else if constexpr (std::is_same<P, DynPlanX>::value)
    run_fft<INV, T, true>(sm, is, pl, u, nthr, tw);
  else
    run_fft_ct<INV, T, P>(sm, is, u, nthr, tw);
}

template <typename T, typename P, typename F>
__device__ __forceinline__ void fft_fused_plan(cplx<T>* sm, int is, const FFTPlan& pl, int u, int nthr,
                                               const cplx<T>* __restrict__ tw, F& mid) {
  if constexpr (std::is_same<P, DynPlan>::value)
    run_fft_fused<T, F, false>(sm, is, pl, u, nthr, tw, mid);
  else if constexpr (std::is_same<P, DynPlanX>::value)
    run_fft_fused<T, F, true>(sm, is, pl, u, nthr, tw, mid);
  else
    run_fft_fused_ct<T, P>(sm, is, u, nthr, tw, mid);
}

// The plans the planner picks for the 3^7 = 2187 axis (81 threads), the
// 3^5 = 243 axis (9 threads) and the 3^6 = 729 axis (27 threads).
using Plan2187 = CPlan<27, 27, 3>;
using Plan243 = CPlan<27, 9>;
using Plan729 = CPlan<27, 27>;

}  // namespace fh

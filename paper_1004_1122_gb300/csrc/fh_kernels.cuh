// fh_kernels.cuh -- the fused memory passes of the collocation operator
//   A e = e + F^-1 [ Gamma0(k) . F(dL . e) ]         (Eq. linear_system, Eq. mtrx_B)
// and the Krylov vector work around it (Section 2.3, Section 3).
//
// One application of B on a d-dimensional grid is 2d-1 passes over HBM:
//
//   row_fwd   lines along the contiguous last axis: gather dL[phase] (d x d),
//             tau = dL e (optionally fused with the CG direction update
//             p = r + beta p), pack two real channels per complex sequence,
//             forward FFT, unpack to the half spectrum k_last in [0, (n+1)/2)
//             and store it in the tiled spectrum layout below.
//   col(mid)  3-D only: forward FFT along axis 1 on contiguous tiles.
//   col(last) forward FFT along axis 0, Green projection
//             y^(k) = xi (xi . tau^(k)) / (xi . L0 . xi) / |N|, zero at k = 0
//             (Section 2.1), inverse FFT along axis 0.
//   col(mid)  3-D only: inverse FFT along axis 1.
//   row_inv   inverse FFT of each line (rebuilding the Hermitian spectrum of
//             two real channels at once), then a fused epilogue: e + y,
//             e + dL y (transpose), A p with (p, A p), the fixed-point update
//             e <- e0 - y, or the residual e0 - e - y, with float64 dot
//             partials per CTA.
//
// Spectrum layout (complex, element type T):
//   S[((t * nlines + line) * C + c) * M + m]
// line = i0 * n1 + i1 is the index of a line along the last axis (2-D: n1 = 1),
// k_last = t * C + c is the half-spectrum frequency (tiles of C, padded),
// m in [0, M) is the real channel (load l = m / d, component a = m % d).
// For a fixed tile t, the Green pass reads the whole axis-0 column of C
// frequencies x M channels as one contiguous block (2-D) or as contiguous
// chunks of G * C * M (3-D), and the row passes touch contiguous runs of
// lines_per_cta * C * M elements.
#pragma once

#include "fh_fft.cuh"
#include "fh_tma.cuh"

namespace fh {

constexpr int kMaxLoads = 3;
constexpr int kMaxD = 3;
constexpr int kMaxChannels = kMaxLoads * kMaxD;
constexpr int kRedThreads = 256;
constexpr int kRowMaxThreads = 512;   // row passes: <= 128 registers per thread
constexpr int kColMaxThreads = 768;   // column passes: <= 85 registers per thread
// Row kernels with a compile-time plan run one line per 96-thread CTA; their
// register cap is set for kRowCtBlocks resident CTAs per SM (measured on
// 2187^2: 7 CTAs beat 6, 8 and 10 -- 49.7 / 43.2 us for the direction and
// A p passes against 59.6 / 49.6 us at 6 and spills at 10).
constexpr int kRowCtThreads = 96;
constexpr int kRowCtBlocks = 7;
template <typename PS> struct RowBounds {
  static constexpr int threads = kRowMaxThreads, blocks = 1;
};
template <> struct RowBounds<Plan2187> {
  static constexpr int threads = kRowCtThreads, blocks = kRowCtBlocks;
};
// Row-pass launch shape fixed at compile time: one line per CTA of NT
// threads, TPL threads per line FFT (0: from the launch arguments), spectrum
// tiles of CC frequencies.  The loop bounds, the thread-to-butterfly mapping
// and the tiled-spectrum index then fold into constants.  RowShape<0, 0, 0>
// takes all of it from the launch arguments.
template <int NT, int TPL, int CC> struct RowShape {
  static constexpr int nt = NT, tpl = TPL, cc = CC;
  static constexpr int csh = CC <= 1 ? 0 : CC <= 2 ? 1 : CC <= 4 ? 2 : CC <= 8 ? 3 : 4;
  static_assert(CC == 0 || (1 << csh) == CC, "tile width must be a power of two");
};
using RowDyn = RowShape<0, 0, 0>;
// Axis length of a compile-time plan (0 for run-time plans).
template <typename PS> struct PlanLen {
  static constexpr int value = PS::n;
};
template <> struct PlanLen<DynPlan> {
  static constexpr int value = 0;
};
template <> struct PlanLen<DynPlanX> {
  static constexpr int value = 0;
};
// Axis length of a plan: a constant for compile-time plans.
template <typename PS> __device__ __forceinline__ int plan_len(const FFTPlan& pl) {
  if constexpr (std::is_same<PS, DynPlan>::value || std::is_same<PS, DynPlanX>::value)
    return pl.n;
  else
    return PS::n;
}
// Green-pass kernels with a compile-time plan: kColCtBlocks resident CTAs of
// at most kColCtThreads threads (measured on 2187^2: a cap for 2 x 352 threads
// or 3 x 352 threads is slower than the 80-register cap of 768 threads).
constexpr int kColCtThreads = 768;
constexpr int kColCtBlocks = 1;
template <typename PS> struct ColBounds {
  static constexpr int threads = kColCtThreads, blocks = kColCtBlocks;
};
template <> struct ColBounds<DynPlan> {
  static constexpr int threads = kColMaxThreads, blocks = 1;
};
constexpr int kColPipeMaxThreads = 512;  // persistent Green pass: <= 128 registers per thread

// ----------------------------------------------------------------------------
// device scalars of one Krylov solve (one per load)
// ----------------------------------------------------------------------------
struct Scal {
  double rr;       // (r, r)
  double rho;      // BiCG (r, r*)
  double den;      // (A p, p) or (A p, p*)
  double alpha;
  double beta;
  double b2;       // ||rhs||^2, denominator of the relative residual
  double tol2;     // tol^2
  double rel;      // last relative residual
  double rel_true; // last true residual (set by residual kernels)
  int iter;
  int max_iter;
  int done;        // 0 running, 1 converged, 2 breakdown, 3 iteration cap
  int hist_cap;
  double* hist;    // device history array or nullptr
  double E[3];     // constant right-hand side (macroscopic field) when no rhs field
  double best_rel; // smallest relative residual so far
  int best_iter;   // iteration at which best_rel last halved
  int stall_window;// > 0: stop as kStalled after this many iterations without halving
  // Per-iteration norms of Section 3 (device arrays of hist_cap entries, or nullptr):
  // hist_eta_r[m] = Eq. (errR_def) ||L0 (e_{m+1} - e_m)|| / ||e0|| for an
  // isotropic L0 = l0iso I (NaN when l0iso == 0); hist_eta_e[m] = Eq. (errE_def)
  // of the iterate e_m (written by k_eta_record).
  double* hist_eta_r;
  double* hist_eta_e;
  double l0iso;
  // CG with the x step deferred to every second iteration: alpha_x is the
  // step length whose update of x is still owed (direction in the first p
  // buffer) while xpend is 1.
  double alpha_x;
  int xpend;
};

// kStalled: the recursive residual stopped decreasing (the working precision's
// noise floor); refinement drivers continue from it with a float64 residual.
enum : int { kRunning = 0, kConverged = 1, kBreakdown = 2, kCap = 3, kStalled = 4 };

__device__ __forceinline__ bool stalled(Scal& s) {
  if (!(s.rel < 0.5 * s.best_rel) && s.best_rel > 0.0) {
    return s.stall_window > 0 && s.iter - s.best_iter >= s.stall_window;
  }
  s.best_rel = s.rel;
  s.best_iter = s.iter;
  return false;
}

struct Mat3 {
  double v[9];
};

// ----------------------------------------------------------------------------
// launch descriptors (plain structs passed by value)
// ----------------------------------------------------------------------------
struct Geom {
  int d;
  int n[3];
  int nlast, H, C, Tt;
  int nlines;     // |N| / nlast
  int n1;         // 3-D: n[1]; 2-D: 1
  long long nodes;
  int M;          // channels = d * nloads
  int nloads;
  int cshift;     // log2(C): tile widths are powers of two
  double invY[3];
  double L0[9];
  double inv_nodes;
  // batches of same-size cells: cell b owns lines [b*lines_cell, (b+1)*lines_cell)
  // and nodes [b*cell_nodes, (b+1)*cell_nodes) of every component plane
  int ncell;
  int lines_cell;
  long long cell_nodes;
  int tab_stride;   // table entries per cell (nphase * d * d)
};

template <typename T> struct RowArgs {
  Geom g;
  FFTPlan plan;
  int lpc;        // lines per CTA
  int tpl;        // threads per sequence
  int nseq;       // complex sequences per CTA
  const cplx<T>* tw;
  const dfc* twdf;          // line twiddles as double-floats: run the line FFT in double-float
  cplx<T>* S;
  const uint8_t* phase;
  const T* tab;   // per-phase d x d table (dL, or L for the equilibrium norm), T
  int nphase;
  // per-load vectors (meaning depends on the mode)
  const T* in[kMaxLoads];
  T* out[kMaxLoads];
  const T* aux[kMaxLoads];
  T* aux2[kMaxLoads];
  const T* rhs[kMaxLoads];   // field right-hand side or nullptr for constant scal[l].E
  Scal* scal;               // [ncell][NL] entries
  double* part;             // partials [NL][gridDim.x]
};

struct ColArgsBase {
  Geom g;
  FFTPlan plan;
  int Q;          // columns per CTA
  int tpc;        // threads per column
  int G;          // 3-D: lines along axis 1 grouped per CTA in the last pass
  long long stride_i;
  int nb_inner;
  long long base_outer, base_inner;
  int axis;       // FFT axis of this pass (0 = Green axis, 1 = middle axis)
};

template <typename T> struct ColArgs {
  ColArgsBase b;
  const cplx<T>* tw;
  cplx<T>* S;
  Scal* scal;
  double* part;
  const double* L0cell;  // per-cell reference medium [ncell][9], or nullptr for g.L0
  int* err;              // device error word (bounded waits that expired), or nullptr
  unsigned long long wait_ns;  // limit of the bounded waits (0: tma::kWaitLimitNs)
};

// ----------------------------------------------------------------------------
// small helpers
// ----------------------------------------------------------------------------
__device__ __forceinline__ bool all_done(const Scal* s, int nloads) {
  if (s == nullptr) return false;
  for (int l = 0; l < nloads; ++l)
    if (s[l].done == kRunning) return false;
  return true;
}

// Signed frequency of FFT bin j on an axis of n nodes: the set Z^N of
// Section 2.2, -n/2 < k <= n/2.
__device__ __forceinline__ int signed_freq(int j, int n) { return j <= n / 2 ? j : j - n; }
// Bin j is the Nyquist frequency of an even axis.  The Green operator is zero
// at every frequency with a Nyquist component (the reading for even grids;
// the paper's grids are odd), and the equilibrium norm leaves them out.
__device__ __forceinline__ bool nyquist_bin(int j, int n) { return (n & 1) == 0 && 2 * j == n; }

// Dot-product accumulator.  float64 work accumulates directly; float32 work
// uses compensated (Kahan) summation in float32, whose error is a few float32
// ulps of the sum of |terms| whatever the count, and converts to float64 once
// at the end.  Keeping float64 arithmetic and float32->float64 conversions out
// of the per-element loop matters on this part: a float64 fold every 32 terms
// cost the row-inverse pass 35 % and the CG update 25 % (measured, 2187^2).
template <typename T> struct DotAcc {
  double total = 0.0;
  __device__ __forceinline__ void add(T x) { total += (double)x; }
  __device__ __forceinline__ double get() const { return total; }
};
template <> struct DotAcc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

// Block-wide float64 sum of up to kMaxLoads values; thread 0 writes
// part[l * gridDim.x + blockIdx.x].
template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], int nv, double* part,
                                                   int nblocks, int blk) {
  __shared__ double red[32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][i] = x;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double x = lane < nw ? red[lane][i] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0 && i < nv) part[(long long)i * nblocks + blk] = x;
    }
  }
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
// Prefetch [p, p + bytes) into L2, one request per 128-byte line, spread over the CTA.
__device__ __forceinline__ void prefetch_range(const void* p, long long bytes) {
  const char* b = reinterpret_cast<const char*>((reinterpret_cast<uintptr_t>(p)) & ~(uintptr_t)127);
  const long long nl = (reinterpret_cast<const char*>(p) + bytes - b + 127) / 128;
  for (long long i = threadIdx.x; i < nl; i += blockDim.x) prefetch_l2(b + i * 128);
}

// Line FFTs of float64 sequences in double-float arithmetic: the packed
// sequences are split in place into hi + lo float32 parts (a complex
// double-float takes the 16 bytes of a double2), transformed on the float32
// pipes and recombined in place.  Used by the float64 residual passes, whose
// pointwise work stays float64.  Every thread of the CTA calls it.
template <bool INV>
__device__ __forceinline__ void line_fft_df(double2* sm, int nseq, int n, const FFTPlan& plan, int tpl,
                                            const dfc* __restrict__ twdf) {
  dfc* smd = reinterpret_cast<dfc*>(sm);
  const int tot = nseq * n;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) smd[i] = dfc_from(sm[i]);
  __syncthreads();
  const int s = threadIdx.x / tpl;
  const int u = s < nseq ? threadIdx.x - s * tpl : n;  // idle threads never touch smem
  fft_plan<INV, dfl, DynPlan>(smd + (size_t)(s < nseq ? s : 0) * n, 1, plan, u, tpl, twdf);
  for (int i = threadIdx.x; i < tot; i += blockDim.x) sm[i] = dfc_to(smd[i]);
  __syncthreads();
}

// ----------------------------------------------------------------------------
// row forward pass
// ----------------------------------------------------------------------------
enum : int {
  kProApply = 0,     // tau = tab . in
  kProPlain = 1,     // tau = in
  kProDir = 2,       // p = r + beta p (in = r, out = p); tau = tab . p
  kProDirPlain = 3   // p = r + beta p; tau = p
};

// DF (float64 only): the line FFT runs in double-float arithmetic (line_fft_df).
// RS: compile-time launch shape (RowShape) or RowDyn.
template <typename T, int D, int NL, int PRO, typename PS = DynPlan, bool DF = false, typename RS = RowDyn>
__global__ void __launch_bounds__(RowBounds<PS>::threads, RowBounds<PS>::blocks) k_row_fwd(RowArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const Geom& g = a.g;
  constexpr int d = D, M = D * NL;
  constexpr bool kFix = RS::nt > 0;
  const int n = plan_len<PS>(a.plan);
  const int nthr = kFix ? RS::nt : (int)blockDim.x;
  const int tpl = (kFix && RS::tpl > 0) ? RS::tpl : a.tpl;
  const int lpc = kFix ? 1 : a.lpc;
  const int nseq = kFix ? (M + 1) / 2 : a.nseq;
  const int Cc = kFix ? RS::cc : g.C, csh = kFix ? RS::csh : g.cshift;
  const int H = kFix ? n / 2 + 1 : g.H;
  T* stab = reinterpret_cast<T*>(sm + (size_t)nseq * n);
  const int line0 = blockIdx.x * lpc;
  const int cell = g.ncell > 1 ? line0 / g.lines_cell : 0;
  Scal* const sc = a.scal ? a.scal + cell * NL : nullptr;
  const T* const tabc = a.tab + (size_t)cell * g.tab_stride;
  if (all_done(sc, NL)) return;

  constexpr bool kUseTab = (PRO == kProApply || PRO == kProDir);
  constexpr bool kDir = (PRO == kProDir || PRO == kProDirPlain);
  bool lact[NL];
  T lbeta[NL];
  const T* pin[NL];
  T* pout[NL];
  const T* pold[NL];  // direction modes: the previous p (a.aux when it is kept apart, else read in place)
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    lact[l] = !kDir || sc[l].done == kRunning;
    lbeta[l] = kDir ? T(sc[l].beta) : T(0);
    pin[l] = a.in[l];
    pout[l] = a.out[l];
    pold[l] = a.aux[l] ? a.aux[l] : a.out[l];
  }
  // ask L2 for the CTA's input lines before the table load and the barrier:
  // the gather below then waits on L2 rather than on HBM (direction pass on
  // 2187^2: 50.0 -> 47.2 us; the same hint in the A p pass measured slower)
  for (int ll = 0; ll < lpc; ++ll) {
    const int line = line0 + ll;
    if (line >= g.nlines) break;
    const long long lo = (long long)line * n;
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        prefetch_range(pin[l] + c * g.nodes + lo, (long long)n * sizeof(T));
        if (kDir) prefetch_range(pold[l] + c * g.nodes + lo, (long long)n * sizeof(T));
      }
    if (kUseTab) prefetch_range(a.phase + lo, n);
  }
  if (kUseTab) {
    for (int i = threadIdx.x; i < a.nphase * d * d; i += nthr) stab[i] = tabc[i];
  }
  __syncthreads();

  // 1. gather + polarisation into the packed sequences.  Loads of kUnroll
  // elements per thread are issued before any of them is used, so each thread
  // keeps several global loads in flight (the row pass is latency-bound
  // otherwise).
  constexpr int kUnroll = 4;
  for (int ll = 0; ll < lpc; ++ll) {
    const int line = line0 + ll;
    const bool valid = line < g.nlines;
    const long long lo = (long long)line * n;
    for (int i0 = threadIdx.x; i0 < n; i0 += kUnroll * nthr) {
      T v[kUnroll][NL][D];
      T pv[kUnroll][NL][D];
      int ph[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int i = i0 + u * nthr;
        const bool ok = valid && i < n;
        ph[u] = (kUseTab && ok) ? a.phase[lo + i] : 0;
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
          for (int c = 0; c < D; ++c) {
            v[u][l][c] = ok ? __ldg(pin[l] + c * g.nodes + lo + i) : T(0);
            if (kDir) pv[u][l][c] = ok ? pold[l][c * g.nodes + lo + i] : T(0);
          }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int i = i0 + u * nthr;
        if (i >= n) continue;
        const bool ok = valid;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
          T x[D];
#pragma unroll
          for (int c = 0; c < D; ++c) {
            x[c] = kDir ? v[u][l][c] + lbeta[l] * pv[u][l][c] : v[u][l][c];
            if (kDir && ok && lact[l]) pout[l][c * g.nodes + lo + i] = x[c];
          }
#pragma unroll
          for (int c = 0; c < D; ++c) {
            T t = x[c];
            if (kUseTab) {
              t = T(0);
              const T* row = stab + (ph[u] * D + c) * D;
#pragma unroll
              for (int b2 = 0; b2 < D; ++b2) t += row[b2] * x[b2];
            }
            const int gch = ll * M + l * D + c;
            T* dst = reinterpret_cast<T*>(&sm[(size_t)(gch >> 1) * n + i]);
            dst[gch & 1] = t;
          }
        }
      }
    }
  }
  // zero the imaginary half of a trailing unpaired channel
  if ((lpc * M) & 1) {
    const int s = nseq - 1;
    for (int i = threadIdx.x; i < n; i += nthr) sm[(size_t)s * n + i].y = T(0);
  }
  __syncthreads();

  // 2. forward FFT of every sequence
  if constexpr (DF) {
    static_assert(std::is_same<T, double>::value, "double-float line FFTs are for float64 rows");
    line_fft_df<false>(sm, nseq, n, a.plan, tpl, a.twdf);
  } else {
    const int s = threadIdx.x / tpl;
    const int u = s < nseq ? threadIdx.x - s * tpl : n;  // idle threads never touch smem
    fft_plan<false, T, PS>(sm + (size_t)(s < nseq ? s : 0) * n, 1, a.plan, u, tpl, a.tw);
  }

  // 3. unpack two real spectra per sequence and store the half spectrum:
  // one thread per (line, frequency kx), all M channels of that frequency
  // (contiguous in the tiled layout) written together.
  const int TC = kFix ? (H + Cc - 1) / Cc * Cc : g.Tt * g.C;
  for (int ll = 0; ll < lpc; ++ll) {
    const int line = line0 + ll;
    if (line >= g.nlines) break;
    for (int kx = threadIdx.x; kx < TC; kx += nthr) {
      const int t = kx >> csh, c = kx & (Cc - 1);
      const int kneg = kx == 0 ? 0 : n - kx;
      C val[M];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        val[m].x = T(0);
        val[m].y = T(0);
        if (kx < H) {
          const int gch = ll * M + m;
          const C* seq = sm + (size_t)(gch >> 1) * n;
          const C z1 = seq[kx];
          const C z2 = seq[kneg];
          if ((gch & 1) == 0) {
            val[m].x = T(0.5) * (z1.x + z2.x);
            val[m].y = T(0.5) * (z1.y - z2.y);
          } else {
            val[m].x = T(0.5) * (z1.y + z2.y);
            val[m].y = T(0.5) * (z2.x - z1.x);
          }
        }
      }
      C* dst = a.S + (((long long)t * g.nlines + line) * Cc + c) * M;
      if constexpr (sizeof(C) == 8 && M % 2 == 0) {
        // float32: two complex values per 16-byte store
#pragma unroll
        for (int m = 0; m < M; m += 2)
          reinterpret_cast<float4*>(dst)[m / 2] =
              make_float4((float)val[m].x, (float)val[m].y, (float)val[m + 1].x, (float)val[m + 1].y);
      } else {
#pragma unroll
        for (int m = 0; m < M; ++m) dst[m] = val[m];
      }
    }
  }
}

// ----------------------------------------------------------------------------
// column passes
// ----------------------------------------------------------------------------
enum : int { kColFwd = 0, kColInv = 1, kColGreen = 2, kColEta = 3 };

// Green projection of one value of a 2-D spectrum in registers:
// y_a = xi_a (xi . v) / (xi . L0 . xi) / |N| at (k0, k_last), zero at k = 0 and
// on padded frequencies.  The caller holds component a = q % 2 of the value;
// the other component comes from the neighbouring lane (q ^ 1).
// NC > 0: the column length n is the compile-time constant NC.
template <typename T, int NC = 0>
struct GreenPoint2 {
  T invY0, invY1, L00, L01, L10, L11, inv_nodes, xi1;
  int n_rt, a;
  bool pad, kl0;
  __device__ __forceinline__ void init(const Geom& g, const double* L0src, int t, int q, int n_) {
    const int c = (q / g.M) % g.C;
    const int kl = t * g.C + c;
    invY0 = T(g.invY[0]);
    invY1 = T(g.invY[1]);
    L00 = T(L0src[0]);
    L01 = T(L0src[1]);
    L10 = T(L0src[3]);
    L11 = T(L0src[4]);
    inv_nodes = T(g.inv_nodes);
    xi1 = T(kl) * invY1;
    n_rt = n_;
    a = q & 1;
    pad = kl >= g.H || nyquist_bin(kl, g.nlast);  // padding, or the last axis's Nyquist column
    kl0 = kl == 0;
  }
  __device__ __forceinline__ cplx<T> operator()(cplx<T> v, int i, bool act) const {
    const int n = NC > 0 ? NC : n_rt;
    cplx<T> o;
    o.x = __shfl_xor_sync(0xffffffffu, v.x, 1);
    o.y = __shfl_xor_sync(0xffffffffu, v.y, 1);
    const int k0 = i <= n / 2 ? i : i - n;
    const T xi0 = T(k0) * invY0;
    const cplx<T> v0 = a == 0 ? v : o;
    const cplx<T> v1 = a == 0 ? o : v;
    const T den = xi0 * (L00 * xi0 + L01 * xi1) + xi1 * (L10 * xi0 + L11 * xi1);
    const bool zero = !act || pad || (k0 == 0 && kl0) || nyquist_bin(i, n);
    const T f = zero ? T(0) : inv_nodes / den;
    const T sre = xi0 * v0.x + xi1 * v1.x;
    const T sim = xi0 * v0.y + xi1 * v1.y;
    const T xa = a == 0 ? xi0 : xi1;
    cplx<T> y;
    y.x = xa * sre * f;
    y.y = xa * sim * f;
    return y;
  }
};

// Green projection of one column tile held in shared memory (after the
// forward FFT along axis 0): y^(k) = xi (xi . tau^(k)) / (xi . L0 . xi) / |N|,
// zero at k = 0 and on padded frequencies (kColGreen), or the equilibrium-norm
// sums of Eq. (errE_def) (kColEta, into acc).
template <typename T, int D, int CM_, int QC = 0, int NC = 0>
__device__ __forceinline__ void green_tile(const ColArgs<T>& a, cplx<T>* sm, int t, int blk_inner, int cell_idx,
                                           double (&acc)[2]) {
  using C = cplx<T>;
  const ColArgsBase& b = a.b;
  const Geom& g = b.g;
  const int n = NC ? NC : b.plan.n, Q = QC ? QC : b.Q;
  const int M = g.M;
  const int ngrp = Q / D;  // groups of D components sharing one frequency
  T invY[D], L0[D * D];
#pragma unroll
  for (int p = 0; p < D; ++p) invY[p] = T(g.invY[p]);
  const double* L0src = a.L0cell ? a.L0cell + 9 * cell_idx : g.L0;
#pragma unroll
  for (int p = 0; p < D; ++p)
#pragma unroll
    for (int r = 0; r < D; ++r) L0[p * D + r] = T(L0src[p * 3 + r]);
  const T inv_nodes = T(g.inv_nodes);
  for (int idx = threadIdx.x; idx < n * ngrp; idx += blockDim.x) {
    const int i = idx / ngrp, grp = idx - i * ngrp;
    const int q0 = grp * D;
    const int gl = q0 / (g.C * M);
    const int c = (q0 / M) % g.C;
    const int kl = t * g.C + c;
    const int k0 = signed_freq(i, n);
    const int k1 = D == 2 ? kl : signed_freq(blk_inner * b.G + gl, g.n[1]);
    T xi[D];
    xi[0] = T(k0) * invY[0];
    xi[1] = T(k1) * invY[1];
    if (D == 3) xi[D - 1] = T(kl) * invY[D - 1];
    C* v = sm + (size_t)i * Q + q0;
    const bool pad = kl >= g.H;
    // even axes: no Green operator and no equilibrium term at a Nyquist frequency
    const bool nyq = nyquist_bin(i, n) || nyquist_bin(kl, g.nlast) ||
                     (D == 3 && nyquist_bin(blk_inner * b.G + gl, g.n[1]));
    if (CM_ == kColGreen) {
      T den = T(0);
#pragma unroll
      for (int p = 0; p < D; ++p) {
        T row = T(0);
#pragma unroll
        for (int r = 0; r < D; ++r) row += L0[p * D + r] * xi[r];
        den += xi[p] * row;
      }
      T sre = T(0), sim = T(0);
#pragma unroll
      for (int p = 0; p < D; ++p) {
        sre += xi[p] * v[p].x;
        sim += xi[p] * v[p].y;
      }
      const bool zero = pad || nyq || (k0 == 0 && k1 == 0 && kl == 0);
      const T f = zero ? T(0) : inv_nodes / den;
#pragma unroll
      for (int p = 0; p < D; ++p) {
        v[p].x = xi[p] * sre * f;
        v[p].y = xi[p] * sim * f;
      }
    } else {
      if (!pad && !nyq) {
        double dre = 0.0, dim = 0.0;
#pragma unroll
        for (int p = 0; p < D; ++p) {
          dre += (double)xi[p] * (double)v[p].x;
          dim += (double)xi[p] * (double)v[p].y;
        }
        const double w = kl == 0 ? 1.0 : 2.0;  // half spectrum: k and -k
        acc[0] += w * (dre * dre + dim * dim);
        if (k0 == 0 && k1 == 0 && kl == 0) {
#pragma unroll
          for (int p = 0; p < D; ++p)
            acc[1] += (double)v[p].x * v[p].x + (double)v[p].y * v[p].y;
        }
      }
    }
  }
}

// QC, TC > 0: the tile's column count Q and the threads per column FFT are
// compile-time constants (they must equal a.b.Q and a.b.tpc); the column
// stride and the thread-to-butterfly mapping then fold into immediate
// offsets instead of run-time index arithmetic.
template <typename T, int D, int CM_, typename PS = DynPlan, int QC = 0, int TC = 0>
__global__ void __launch_bounds__(ColBounds<PS>::threads, ColBounds<PS>::blocks) k_col(ColArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const ColArgsBase& b = a.b;
  const Geom& g = b.g;
  constexpr int d = D;
  const int n = plan_len<PS>(b.plan), Q = QC ? QC : b.Q;
  const int tpc = TC ? TC : b.tpc;
  // 2-D tiles are contiguous: row i of the tile starts Q values after row i - 1
  const long long stride_i = (QC && D == 2) ? (long long)QC : b.stride_i;
  const int blk_outer = blockIdx.x / b.nb_inner;
  const int blk_inner = blockIdx.x - blk_outer * b.nb_inner;
  // 2-D batches: the inner block index is the cell
  const int cell = (D == 2 && g.ncell > 1) ? blk_inner : 0;
  if (all_done(a.scal ? a.scal + cell * g.nloads : nullptr, g.nloads)) return;
  const long long base = blk_outer * b.base_outer + blk_inner * b.base_inner;
  // columns that fall outside the grid (partial G group in 3-D) are zero
  int qvalid = Q;
  if (b.axis == 0 && D == 3) {
    const int lines_left = g.n1 - blk_inner * b.G;
    const int gv = lines_left < b.G ? lines_left : b.G;
    qvalid = gv * g.C * g.M;
  }

  // Each row i of the tile is Q contiguous complex values at base + i * stride_i.
  // When rows are 16-byte multiples (and aligned) they move as float4 / double2
  // words, kUnroll per thread in flight.
  constexpr int kUnroll = 4;
  const int wpr = (int)(Q * sizeof(C) / 16);  // 16-byte words per row
  const bool vec = qvalid == Q && (Q * sizeof(C)) % 16 == 0 && (base * sizeof(C)) % 16 == 0 &&
                   (stride_i * sizeof(C)) % 16 == 0;
  if (vec) {
    const int nw = n * wpr;
    for (int w0 = threadIdx.x; w0 < nw; w0 += kUnroll * blockDim.x) {
      float4 buf[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int w = w0 + u * blockDim.x;
        if (w < nw) {
          const int i = w / wpr, j = w - i * wpr;
          buf[u] = __ldg(reinterpret_cast<const float4*>(a.S + base + i * stride_i) + j);
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int w = w0 + u * blockDim.x;
        if (w < nw) reinterpret_cast<float4*>(sm)[w] = buf[u];
      }
    }
  } else {
    for (int idx = threadIdx.x; idx < n * Q; idx += blockDim.x) {
      const int i = idx / Q, q = idx - i * Q;
      C v;
      v.x = T(0);
      v.y = T(0);
      if (q < qvalid) v = a.S[base + i * stride_i + q];
      sm[idx] = v;
    }
  }
  __syncthreads();

  const int q = threadIdx.x % Q;
  const int u0 = threadIdx.x / Q;
  const int u = u0 < tpc ? u0 : n;
  if constexpr (CM_ == kColGreen && D == 2) {
    // 2-D: the Green projection runs in registers between the forward and
    // inverse FFTs.  Q = C * M is even and the two components of a frequency
    // sit in columns q and q ^ 1, i.e. adjacent lanes of one warp.
    const int t = blk_outer;
    const double* L0src = a.L0cell ? a.L0cell + 9 * cell : g.L0;
    GreenPoint2<T, QC ? PlanLen<PS>::value : 0> gp;
    gp.init(g, L0src, t, q, n);
    fft_fused_plan<T, PS>(sm + q, Q, b.plan, u, tpc, a.tw, gp);
  } else {
  if (CM_ == kColFwd || CM_ == kColGreen || CM_ == kColEta)
    fft_plan<false, T, PS>(sm + q, Q, b.plan, u, tpc, a.tw);
  else
    fft_plan<true, T, PS>(sm + q, Q, b.plan, u, tpc, a.tw);

  if (CM_ == kColGreen || CM_ == kColEta) {
    double acc[2] = {0.0, 0.0};
    green_tile<T, D, CM_, QC, PlanLen<PS>::value>(a, sm, blk_outer, blk_inner, cell, acc);
    if (CM_ == kColEta) {
      block_reduce_store<2>(acc, 2, a.part, gridDim.x, blockIdx.x);
      return;
    }
    __syncthreads();
    fft_plan<true, T, PS>(sm + q, Q, b.plan, u, tpc, a.tw);
  }
  }

  if (vec) {
    const int nw = n * wpr;
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
      const int i = w / wpr, j = w - i * wpr;
      reinterpret_cast<float4*>(a.S + base + i * stride_i)[j] = reinterpret_cast<const float4*>(sm)[w];
    }
  } else {
    for (int idx = threadIdx.x; idx < n * Q; idx += blockDim.x) {
      const int i = idx / Q, qq = idx - i * Q;
      if (qq < qvalid) a.S[base + i * stride_i + qq] = sm[idx];
    }
  }
}

// Green projection of one value of a 2-D float64 spectrum held in double-float
// registers (the refinement residual's Green pass, k_col_green_df): the same
// map as GreenPoint2, y_a = xi_a (xi . v) / (xi . L0 . xi) / |N|, with every
// product, sum and the quotient in double-float arithmetic.
struct GreenPointDF {
  dfl invY0, xi1, L00, L01, L10, L11, inv_nodes;
  int n, a;
  bool pad, kl0;
  __device__ __forceinline__ void init(const Geom& g, const double* L0src, int t, int q, int n_) {
    const int c = (q / g.M) % g.C;
    const int kl = t * g.C + c;
    invY0 = df_from(g.invY[0]);
    xi1 = df_mul_f(df_from(g.invY[1]), (float)kl);  // |kl| < 2^24: exact in float32
    L00 = df_from(L0src[0]);
    L01 = df_from(L0src[1]);
    L10 = df_from(L0src[3]);
    L11 = df_from(L0src[4]);
    inv_nodes = df_from(g.inv_nodes);
    n = n_;
    a = q & 1;
    pad = kl >= g.H || nyquist_bin(kl, g.nlast);
    kl0 = kl == 0;
  }
  __device__ __forceinline__ dfc operator()(dfc v, int i, bool act) const {
    dfc o;
    o.x = df_shfl_xor(v.x, 1);
    o.y = df_shfl_xor(v.y, 1);
    const int k0 = i <= n / 2 ? i : i - n;
    const dfl xi0 = df_mul_f(invY0, (float)k0);
    const dfc v0 = a == 0 ? v : o;
    const dfc v1 = a == 0 ? o : v;
    const bool zero = !act || pad || (k0 == 0 && kl0) || nyquist_bin(i, n);
    const dfl den = xi0 * (L00 * xi0 + L01 * xi1) + xi1 * (L10 * xi0 + L11 * xi1);
    const dfl f = zero ? dfl(0.0f, 0.0f) : df_div(inv_nodes, zero ? dfl(1.0f, 0.0f) : den);
    const dfl sre = xi0 * v0.x + xi1 * v1.x;
    const dfl sim = xi0 * v0.y + xi1 * v1.y;
    const dfl xaf = (a == 0 ? xi0 : xi1) * f;
    dfc y;
    y.x = xaf * sre;
    y.y = xaf * sim;
    return y;
  }
};

// Green pass of a 2-D float64 spectrum in double-float arithmetic: the same
// forward FFT along axis 0, projection and inverse FFT as k_col<double, 2,
// kColGreen>, on the same launch shape and shared memory (a complex
// double-float is 16 bytes, like a double2).  Each value is split into
// hi + lo float32 parts when the tile is read and recombined when it is
// written; in between, every operation runs on the float32 pipes.  Used for
// the float64 residual of the refined solves, where the result must be
// accurate far below the float32 rounding level but not to the last float64
// bit (relative error ~1e-14 against ~1e-16).  In 2-D every tile row is Q
// whole double2 values (16-byte aligned), so the tile moves as 16-byte words.
template <typename PS = DynPlan>
__global__ void __launch_bounds__(kColMaxThreads) k_col_green_df(ColArgs<double> a, const dfc* __restrict__ twdf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dfc* sm = reinterpret_cast<dfc*>(smem_raw);
  const ColArgsBase& b = a.b;
  const Geom& g = b.g;
  const int n = b.plan.n, Q = b.Q;
  const int blk_outer = blockIdx.x / b.nb_inner;
  const int blk_inner = blockIdx.x - blk_outer * b.nb_inner;
  const int cell = g.ncell > 1 ? blk_inner : 0;  // 2-D batches: the inner block index is the cell
  if (all_done(a.scal ? a.scal + cell * g.nloads : nullptr, g.nloads)) return;
  const long long base = blk_outer * b.base_outer + blk_inner * b.base_inner;
  const int nq = n * Q;
  constexpr int kUnroll = 4;
  for (int w0 = threadIdx.x; w0 < nq; w0 += kUnroll * blockDim.x) {
    double2 buf[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int w = w0 + u * blockDim.x;
      if (w < nq) {
        const int i = w / Q, j = w - i * Q;
        buf[u] = __ldg(a.S + base + i * b.stride_i + j);
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int w = w0 + u * blockDim.x;
      if (w < nq) sm[w] = dfc_from(buf[u]);
    }
  }
  __syncthreads();

  const int q = threadIdx.x % Q;
  const int u0 = threadIdx.x / Q;
  const int u = u0 < b.tpc ? u0 : n;
  const double* L0src = a.L0cell ? a.L0cell + 9 * cell : g.L0;
  GreenPointDF gp;
  gp.init(g, L0src, blk_outer, q, n);
  fft_fused_plan<dfl, PS>(sm + q, Q, b.plan, u, b.tpc, twdf, gp);

  for (int w = threadIdx.x; w < nq; w += blockDim.x) {
    const int i = w / Q, j = w - i * Q;
    a.S[base + i * b.stride_i + j] = dfc_to(sm[w]);
  }
}

// Persistent, double-buffered Green pass for 2-D grids.  A work item is the
// spectrum block of one (tile, cell): n rows of Q = C*M complex values, one
// contiguous, 16-byte aligned range.  One thread moves each block into shared
// memory with a bulk copy while the CTA transforms the previous block, and
// writes the result back with a bulk store, so HBM traffic overlaps the FFTs
// and the grid (one CTA per SM) has no wave tail.
template <typename T, int D, typename PS = DynPlan>
__global__ void __launch_bounds__(kColPipeMaxThreads) k_col_pipe(ColArgs<T> a) {
  static_assert(D == 2, "the persistent Green pass is 2-D only");
  using C = cplx<T>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_fail;
  const ColArgsBase& b = a.b;
  const Geom& g = b.g;
  const int n = b.plan.n, Q = b.Q;
  const uint32_t bytes = (uint32_t)((size_t)n * Q * sizeof(C));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* const buf0 = reinterpret_cast<C*>(smem_raw + 128);
  const size_t bstride = (size_t)n * Q;  // buffer j starts at buf0 + j * bstride
  const int nitems = g.Tt * b.nb_inner;
  const int tid = threadIdx.x;
  if (tid == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::fence_barrier_init();
    s_fail = 0;
  }
  __syncthreads();
  auto base_of = [&](int w) -> long long {
    const int t = w / b.nb_inner;
    return (long long)t * b.base_outer + (long long)(w - t * b.nb_inner) * b.base_inner;
  };
  auto issue = [&](int w, int k) {
    tma::mbar_arrive_expect_tx(&bar[k & 1], bytes);
    tma::bulk_load(buf0 + (k & 1) * bstride, a.S + base_of(w), bytes, &bar[k & 1]);
  };
  const int q = tid % Q;
  const int u0 = tid / Q;
  const int u = u0 < b.tpc ? u0 : n;
  int w = blockIdx.x;
  if (tid == 0 && w < nitems) issue(w, 0);
  int k = 0;
  for (; w < nitems; ++k, w += gridDim.x) {
    const int wn = w + gridDim.x;
    if (tid == 0 && wn < nitems) {
      tma::bulk_wait_read();  // the store of item k-1 has read buffer (k+1)&1
      issue(wn, k + 1);
    }
    if (!tma::mbar_wait(&bar[k & 1], (k >> 1) & 1, a.wait_ns)) s_fail = 1;
    __syncthreads();
    if (s_fail) break;
    C* sm = buf0 + (k & 1) * bstride;
    const int t = w / b.nb_inner, blk_inner = w - t * b.nb_inner;
    const int cell = g.ncell > 1 ? blk_inner : 0;
    if (all_done(a.scal ? a.scal + cell * g.nloads : nullptr, g.nloads)) continue;
    GreenPoint2<T> gp;
    gp.init(g, a.L0cell ? a.L0cell + 9 * cell : g.L0, t, q, n);
    fft_fused_plan<T, PS>(sm + q, Q, b.plan, u, b.tpc, a.tw, gp);
    tma::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tma::bulk_store(a.S + base_of(w), sm, bytes);
      tma::bulk_commit();
    }
  }
  if (tid == 0) {
    if (s_fail) {
      // drain (default limit) the load whose wait gave up, and the load owed
      // to the other buffer when the next item existed, before leaving
      tma::mbar_wait(&bar[k & 1], (k >> 1) & 1);
      if (w + gridDim.x < nitems) tma::mbar_wait(&bar[(k + 1) & 1], ((k + 1) >> 1) & 1);
      if (a.err) atomicExch(a.err, 1);
    }
    tma::bulk_wait_all();
  }
}

// ----------------------------------------------------------------------------
// row inverse pass with fused epilogues
// ----------------------------------------------------------------------------
enum : int {
  kEpiApply = 0,    // out = in + y
  kEpiApplyT = 1,   // out = in + tab . y
  kEpiDir = 2,      // out = in + y (A p), dot (in, out)
  kEpiDirShadow = 3,// out = in + y (A p), dot (out, aux)  [BiCG: (A p, p*)]
  kEpiFixed = 4,    // out = rhs - y, dot |out - in|^2     [FFTH]
  kEpiResid = 5     // out = rhs - in - y, dot |out|^2     [residual]
};

// DF (float64 only): the line FFT runs in double-float arithmetic (line_fft_df).
// RS: compile-time launch shape (RowShape) or RowDyn.
template <typename T, int D, int NL, int EPI, typename PS = DynPlan, bool DF = false, typename RS = RowDyn>
__global__ void __launch_bounds__(RowBounds<PS>::threads, RowBounds<PS>::blocks) k_row_inv(RowArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const Geom& g = a.g;
  constexpr int d = D, M = D * NL;
  constexpr bool kFix = RS::nt > 0;
  const int n = plan_len<PS>(a.plan);
  const int nthr = kFix ? RS::nt : (int)blockDim.x;
  const int tpl = (kFix && RS::tpl > 0) ? RS::tpl : a.tpl;
  const int lpc = kFix ? 1 : a.lpc;
  const int nseq = kFix ? (M + 1) / 2 : a.nseq;
  const int Cc = kFix ? RS::cc : g.C, csh = kFix ? RS::csh : g.cshift;
  const int H = kFix ? n / 2 + 1 : g.H;
  T* stab = reinterpret_cast<T*>(sm + (size_t)nseq * n);
  const int line0 = blockIdx.x * lpc;
  const int nch = lpc * M;
  const int cell = g.ncell > 1 ? line0 / g.lines_cell : 0;
  Scal* const sc = a.scal ? a.scal + cell * NL : nullptr;
  const T* const tabc = a.tab + (size_t)cell * g.tab_stride;
  if (all_done(sc, NL)) return;

  if (EPI == kEpiApplyT) {
    for (int i = threadIdx.x; i < a.nphase * D * D; i += nthr) stab[i] = tabc[i];
  }

  // 1. rebuild the full spectrum of each packed sequence from the half spectra
  // (one thread per (sequence, kx); kUnroll frequencies' loads in flight)
  constexpr int kUnroll = 8;
  for (int s = 0; s < nseq; ++s) {
    const int g0 = 2 * s, g1 = 2 * s + 1;
    const int ll0 = g0 / M, m0 = g0 - ll0 * M;
    const int ll1 = g1 / M, m1 = g1 - ll1 * M;
    const bool has0 = line0 + ll0 < g.nlines;
    const bool has1 = g1 < nch && line0 + ll1 < g.nlines;
    C* seq = sm + (size_t)s * n;
    for (int kb = threadIdx.x; kb < H; kb += kUnroll * nthr) {
      C y0[kUnroll], y1[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int kx = kb + u * nthr;
        y0[u].x = y0[u].y = y1[u].x = y1[u].y = T(0);
        if (kx >= H) continue;
        const int t = kx >> csh, c = kx & (Cc - 1);
        const long long tb = ((long long)t * g.nlines + line0) * Cc + c;
        if (has0) y0[u] = a.S[(tb + (long long)ll0 * Cc) * M + m0];
        if (has1) y1[u] = a.S[(tb + (long long)ll1 * Cc) * M + m1];
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int kx = kb + u * nthr;
        if (kx >= H) continue;
        if (kx == 0 || 2 * kx == n) {  // bins that are their own Hermitian partner
          C w;
          w.x = y0[u].x;
          w.y = y1[u].x;
          seq[kx] = w;
        } else {
          C w, wm;
          w.x = y0[u].x - y1[u].y;
          w.y = y0[u].y + y1[u].x;
          wm.x = y0[u].x + y1[u].y;
          wm.y = y1[u].x - y0[u].y;
          seq[kx] = w;
          seq[n - kx] = wm;
        }
      }
    }
  }
  __syncthreads();

  // 2. inverse FFT
  if constexpr (DF) {
    static_assert(std::is_same<T, double>::value, "double-float line FFTs are for float64 rows");
    line_fft_df<true>(sm, nseq, n, a.plan, tpl, a.twdf);
  } else {
    const int s = threadIdx.x / tpl;
    const int u = s < nseq ? threadIdx.x - s * tpl : n;
    fft_plan<true, T, PS>(sm + (size_t)(s < nseq ? s : 0) * n, 1, a.plan, u, tpl, a.tw);
  }

  // 3. epilogue
  constexpr bool kDot = (EPI == kEpiDir || EPI == kEpiDirShadow || EPI == kEpiFixed || EPI == kEpiResid);
  DotAcc<T> acc[NL];
  bool lact[NL];
  const T* pin[NL];
  T* pout[NL];
  const T* paux[NL];
  const T* prhs[NL];
  T Ec[NL][D];
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    lact[l] = !kDot || sc == nullptr || sc[l].done == kRunning;
    pin[l] = a.in[l];
    pout[l] = a.out[l];
    paux[l] = a.aux[l];
    prhs[l] = a.rhs[l];
#pragma unroll
    for (int c = 0; c < D; ++c)
      Ec[l][c] = (sc != nullptr && (EPI == kEpiFixed || EPI == kEpiResid)) ? T(sc[l].E[c]) : T(0);
  }
  constexpr bool kReadIn = true;
  constexpr bool kReadAux = (EPI == kEpiDirShadow);
  for (int ll = 0; ll < lpc; ++ll) {
    const int line = line0 + ll;
    if (line >= g.nlines) break;
    const long long lo = (long long)line * n;
    for (int i0 = threadIdx.x; i0 < n; i0 += kUnroll * nthr) {
      T vin[kUnroll][NL][D];
      T vaux[kUnroll][NL][D];
      T vrhs[kUnroll][NL][D];
      int ph[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int i = i0 + u * nthr;
        const bool ok = i < n;
        ph[u] = (EPI == kEpiApplyT && ok) ? a.phase[lo + i] : 0;
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
          for (int c = 0; c < D; ++c) {
            const long long o = c * g.nodes + lo + i;
            vin[u][l][c] = (kReadIn && ok && lact[l]) ? pin[l][o] : T(0);
            vaux[u][l][c] = (kReadAux && ok && lact[l]) ? __ldg(paux[l] + o) : T(0);
            vrhs[u][l][c] = ((EPI == kEpiFixed || EPI == kEpiResid) && ok && lact[l])
                                ? (prhs[l] ? __ldg(prhs[l] + o) : Ec[l][c]) : T(0);
          }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int i = i0 + u * nthr;
        if (i >= n) continue;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
          if (!lact[l]) continue;
          T y[D];
#pragma unroll
          for (int c = 0; c < D; ++c) {
            const int gch = ll * M + l * D + c;
            const T* src = reinterpret_cast<const T*>(&sm[(size_t)(gch >> 1) * n + i]);
            y[c] = src[gch & 1];
          }
#pragma unroll
          for (int c = 0; c < D; ++c) {
            const long long o = c * g.nodes + lo + i;
            const T e = vin[u][l][c];
            if (EPI == kEpiApply) {
              pout[l][o] = e + y[c];
            } else if (EPI == kEpiApplyT) {
              const T* row = stab + (ph[u] * D + c) * D;
              T t = T(0);
#pragma unroll
              for (int b2 = 0; b2 < D; ++b2) t += row[b2] * y[b2];
              pout[l][o] = e + t;
            } else if (EPI == kEpiDir) {
              const T ap = e + y[c];
              pout[l][o] = ap;
              acc[l].add(e * ap);
            } else if (EPI == kEpiDirShadow) {
              const T ap = e + y[c];
              pout[l][o] = ap;
              acc[l].add(ap * vaux[u][l][c]);
            } else if (EPI == kEpiFixed) {
              const T en = vrhs[u][l][c] - y[c];
              pout[l][o] = en;
              const T df = en - e;
              acc[l].add(df * df);
            } else {  // kEpiResid
              const T r = vrhs[u][l][c] - e - y[c];
              pout[l][o] = r;
              acc[l].add(r * r);
            }
          }
        }
      }
    }
  }
  if (kDot) {
    double tot[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) tot[l] = acc[l].get();
    block_reduce_store<NL>(tot, NL, a.part, gridDim.x, blockIdx.x);
  }
}

// ----------------------------------------------------------------------------
// vector kernels (grid-stride, float64 dot partials)
// ----------------------------------------------------------------------------
struct VecArgsBase {
  long long len;   // elements per load vector (d * |N|)
  int nloads;
  int ncell;       // cells in the batch (blocks are split evenly between cells)
  int d;
  long long nodes;       // nodes per component plane (all cells)
  long long cell_nodes;  // nodes per cell
};

template <typename T> struct VecArgs {
  VecArgsBase b;
  int want_pp;             // CG: also reduce (p, p) (eta_r history)
  int xmode;               // CG: 1 x += alpha p; 0 x untouched (step deferred); 2 x += alpha_x p2 + alpha p
  T* x[kMaxLoads];
  T* r[kMaxLoads];
  const T* p[kMaxLoads];
  const T* p2[kMaxLoads];  // CG, xmode 2: the previous iteration's direction
  const T* ap[kMaxLoads];
  T* rs[kMaxLoads];        // BiCG shadow residual
  const T* atps[kMaxLoads];// BiCG A^T p*
  Scal* scal;
  double* part;            // [2][nloads][grid]
};

// 16-byte vector of T (4 floats or 2 doubles)
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <> struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};
template <typename V, typename T>
__device__ __forceinline__ T& vlane(V& v, int k) { return reinterpret_cast<T*>(&v)[k]; }

// Range helpers for the vector updates: [b, e) processed by thread t of
// `stride` threads, 16-byte vectors on the aligned interior, scalar head/tail.
template <typename T, typename F>
__device__ __forceinline__ void for_range(long long b, long long e, long long t, long long stride, F&& f) {
  constexpr int W = Vec16<T>::n;
  long long hb = (b + W - 1) / W * W;  // first aligned index
  if (hb > e) hb = e;
  for (long long i = b + t; i < hb; i += stride) f.scalar(i);
  const long long nv = (e - hb) / W;
  for (long long k = t; k < nv; k += 2 * stride) {
    f.vec2(hb / W + k, k + stride < nv ? hb / W + k + stride : -1);
  }
  for (long long i = hb + nv * W + t; i < e; i += stride) f.scalar(i);
}

// PP: also accumulate (p, p) into *dpp (the eta_r history of Section 3).
// XM: the x step.  1: x += al p.  0: x is not touched (its step is owed).
// 2: x += ax p2, then x += al p -- the owed step of the previous iteration
// and this one's, in that order, so x receives exactly the float32 sums of two
// single updates while it is read and written once instead of twice.
template <typename T, bool PP = false, int XM = 1>
struct CgUpd {
  using V = typename Vec16<T>::type;
  static constexpr int W = Vec16<T>::n;
  T* __restrict__ x;
  T* __restrict__ r;
  const T* __restrict__ p;
  const T* __restrict__ ap;
  const T* __restrict__ p2;
  T al, ax;
  DotAcc<T>* dot;
  DotAcc<T>* dpp;
  __device__ __forceinline__ void scalar(long long i) {
    if (XM != 0 || PP) {
      const T pi = p[i];
      if (XM == 1) {
        x[i] += al * pi;
      } else if (XM == 2) {
        T xv = x[i];
        xv += ax * p2[i];
        xv += al * pi;
        x[i] = xv;
      }
      if (PP) dpp->add(pi * pi);
    }
    const T rn = r[i] - al * ap[i];
    r[i] = rn;
    dot->add(rn * rn);
  }
  __device__ __forceinline__ void vec2(long long k0, long long k1) {
    constexpr bool kP = XM != 0 || PP;
    V xv[2], rv[2], pv[2], qv[2], av[2];
    const long long kk[2] = {k0, k1};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (kk[u] < 0) continue;
      if (XM != 0) xv[u] = reinterpret_cast<const V*>(x)[kk[u]];
      rv[u] = reinterpret_cast<const V*>(r)[kk[u]];
      if (kP) pv[u] = __ldg(reinterpret_cast<const V*>(p) + kk[u]);
      if (XM == 2) qv[u] = __ldg(reinterpret_cast<const V*>(p2) + kk[u]);
      av[u] = __ldg(reinterpret_cast<const V*>(ap) + kk[u]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (kk[u] < 0) continue;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        if (XM == 2) vlane<V, T>(xv[u], w) += ax * vlane<V, T>(qv[u], w);
        if (XM != 0) vlane<V, T>(xv[u], w) += al * vlane<V, T>(pv[u], w);
        const T rn = vlane<V, T>(rv[u], w) - al * vlane<V, T>(av[u], w);
        vlane<V, T>(rv[u], w) = rn;
        dot->add(rn * rn);
        if (PP) dpp->add(vlane<V, T>(pv[u], w) * vlane<V, T>(pv[u], w));
      }
      if (XM != 0) reinterpret_cast<V*>(x)[kk[u]] = xv[u];
      reinterpret_cast<V*>(r)[kk[u]] = rv[u];
    }
  }
};

// The owed x step of CG items that stopped after an iteration whose x update
// was deferred: x += alpha_x p (p = the first direction buffer).
template <typename T>
struct XFlush {
  using V = typename Vec16<T>::type;
  static constexpr int W = Vec16<T>::n;
  T* __restrict__ x;
  const T* __restrict__ p;
  T ax;
  __device__ __forceinline__ void scalar(long long i) { x[i] += ax * p[i]; }
  __device__ __forceinline__ void vec2(long long k0, long long k1) {
    const long long kk[2] = {k0, k1};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (kk[u] < 0) continue;
      V xv = reinterpret_cast<const V*>(x)[kk[u]];
      V pv = __ldg(reinterpret_cast<const V*>(p) + kk[u]);
#pragma unroll
      for (int w = 0; w < W; ++w) vlane<V, T>(xv, w) += ax * vlane<V, T>(pv, w);
      reinterpret_cast<V*>(x)[kk[u]] = xv;
    }
  }
};

template <typename T>
struct BicgUpd {
  T* __restrict__ x;
  T* __restrict__ r;
  T* __restrict__ rs;
  const T* __restrict__ p;
  const T* __restrict__ ap;
  const T* __restrict__ atps;
  T al;
  DotAcc<T>* d1;
  DotAcc<T>* d2;
  DotAcc<T>* d3;  // (p, p)
  __device__ __forceinline__ void scalar(long long i) {
    const T pi = p[i];
    x[i] += al * pi;
    const T rn = r[i] - al * ap[i];
    const T sn = rs[i] - al * atps[i];
    r[i] = rn;
    rs[i] = sn;
    d1->add(rn * sn);
    d2->add(rn * rn);
    d3->add(pi * pi);
  }
  __device__ __forceinline__ void vec2(long long k0, long long k1) {
    constexpr int W = Vec16<T>::n;
    scalar_block(k0 * W, W);
    if (k1 >= 0) scalar_block(k1 * W, W);
  }
  __device__ __forceinline__ void scalar_block(long long i0, int w) {
    for (int k = 0; k < w; ++k) scalar(i0 + k);
  }
};

// Block b of the launch belongs to cell b / (gridDim / ncell); a cell's data
// is one contiguous range per component plane (the whole vector when there is
// a single cell).  Partials: slot l of block b.
template <typename T, int NL, typename Mk>
__device__ __forceinline__ void cell_ranges(const VecArgs<T>& a, Mk&& mk) {
  const int ncell = a.b.ncell;
  const int bpc = gridDim.x / ncell;
  const int cell = blockIdx.x / bpc;
  const long long t = (long long)(blockIdx.x - cell * bpc) * blockDim.x + threadIdx.x;
  const long long stride = (long long)bpc * blockDim.x;
  if (ncell == 1) {
    mk(0, a.b.len, t, stride, cell);
  } else {
    for (int c = 0; c < a.b.d; ++c) {
      const long long b0 = c * a.b.nodes + cell * a.b.cell_nodes;
      mk(b0, b0 + a.b.cell_nodes, t, stride, cell);
    }
  }
}

// CG: x += alpha p (as selected by XM, see CgUpd); r -= alpha A p; partial
// (r, r) at slot l, and with PP (p, p) at slot kMaxLoads + l (for the eta_r
// history)
template <typename T, int NL, bool PP = false, int XM = 1>
__global__ void k_cg_update(VecArgs<T> a) {
  const int bpc = gridDim.x / a.b.ncell;
  const int cell = blockIdx.x / bpc;
  Scal* const sc = a.scal + cell * NL;
  if (all_done(sc, NL)) return;
  constexpr int NV = PP ? kMaxLoads + NL : NL;
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    if (sc[l].done != kRunning) continue;
    DotAcc<T> dot, dpp;
    CgUpd<T, PP, XM> f{a.x[l], a.r[l], a.p[l], a.ap[l], a.p2[l], T(sc[l].alpha), T(sc[l].alpha_x), &dot, &dpp};
    cell_ranges<T, NL>(a, [&](long long b0, long long e0, long long t, long long stride, int) {
      for_range<T>(b0, e0, t, stride, f);
    });
    acc[l] = dot.get();
    if (PP) acc[PP ? kMaxLoads + l : 0] = dpp.get();
  }
  block_reduce_store<NV>(acc, NV, a.part, gridDim.x, blockIdx.x);
}

// After the iteration loop: items whose last x step is still owed (xpend)
// receive it, x += alpha_x p.
template <typename T, int NL>
__global__ void k_cg_flush(VecArgs<T> a) {
  const int bpc = gridDim.x / a.b.ncell;
  const int cell = blockIdx.x / bpc;
  const Scal* const sc = a.scal + cell * NL;
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    if (!sc[l].xpend) continue;
    XFlush<T> f{a.x[l], a.p[l], T(sc[l].alpha_x)};
    cell_ranges<T, NL>(a, [&](long long b0, long long e0, long long t, long long stride, int) {
      for_range<T>(b0, e0, t, stride, f);
    });
  }
}

// BiCG: x += alpha p; r -= alpha A p; r* -= alpha A^T p*; partials (r, r*), (r, r), (p, p)
// partial layout: (r, r*) of load l at slot l, (r, r) at slot kMaxLoads + l,
// (p, p) at slot 2 kMaxLoads + l.
template <typename T, int NL>
__global__ void k_bicg_update(VecArgs<T> a) {
  const int bpc = gridDim.x / a.b.ncell;
  const int cell = blockIdx.x / bpc;
  Scal* const sc = a.scal + cell * NL;
  if (all_done(sc, NL)) return;
  double acc[3 * kMaxLoads];
#pragma unroll
  for (int i = 0; i < 3 * kMaxLoads; ++i) acc[i] = 0.0;
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    if (sc[l].done != kRunning) continue;
    DotAcc<T> d1, d2, d3;
    BicgUpd<T> f{a.x[l], a.r[l], a.rs[l], a.p[l], a.ap[l], a.atps[l], T(sc[l].alpha), &d1, &d2, &d3};
    cell_ranges<T, NL>(a, [&](long long b0, long long e0, long long t, long long stride, int) {
      for (long long i = b0 + t; i < e0; i += stride) f.scalar(i);
    });
    acc[l] = d1.get();
    acc[kMaxLoads + l] = d2.get();
    acc[2 * kMaxLoads + l] = d3.get();
  }
  block_reduce_store<3 * kMaxLoads>(acc, 3 * kMaxLoads, a.part, gridDim.x, blockIdx.x);
}

// ----------------------------------------------------------------------------
// scalar control kernels: one CTA of kRedThreads threads per item
// ----------------------------------------------------------------------------
// One CTA of kRedThreads threads per item (cell, load): the item's partials are
// the bpc = np / ncell consecutive slots of its cell in row l of the partial
// array.  Four independent accumulators per thread keep several L2 loads in
// flight (a single-cell 2187^2 CG item has 2187 slots; one warp walking them in
// a dependent chain took ~10 us per scalar launch).
__device__ __forceinline__ double block_sum(const double* p, int n) {
  __shared__ double red[kRedThreads / 32];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int i = threadIdx.x;
  for (; i + 3 * kRedThreads < n; i += 4 * kRedThreads) {
    a0 += p[i];
    a1 += p[i + kRedThreads];
    a2 += p[i + 2 * kRedThreads];
    a3 += p[i + 3 * kRedThreads];
  }
  for (; i < n; i += kRedThreads) a0 += p[i];
  double x = (a0 + a1) + (a2 + a3);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    x = lane < kRedThreads / 32 ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  }
  __syncthreads();  // red[] may be reused by a second sum in the same kernel
  return x;         // valid in thread 0
}

struct ItemRef {
  int item, cell, l, bpc;
  bool valid;
};

__device__ __forceinline__ ItemRef item_ref(int np, int ncell, int nl) {
  ItemRef r;
  r.item = (int)blockIdx.x;
  r.valid = r.item < ncell * nl;
  r.cell = r.item / nl;
  r.l = r.item - r.cell * nl;
  r.bpc = np / ncell;
  return r;
}

__device__ __forceinline__ const double* item_part(const double* part, int row, int np, const ItemRef& r) {
  return part + (long long)row * np + (long long)r.cell * r.bpc;
}

__device__ __forceinline__ bool finite_d(double x) { return x == x && x - x == 0.0; }

__device__ __forceinline__ void record_hist(Scal& s) {
  if (s.hist != nullptr && s.iter < s.hist_cap) s.hist[s.iter] = s.rel;
}

// After the initial residual (kEpiResid partials or a copied rhs):
// rr = sum, rel = sqrt(rr / b2), beta = 0, iter = 0.
static __global__ void k_scal_start(Scal* scal, const double* part, int np, int ncell, int nl) {
  const ItemRef r = item_ref(np, ncell, nl);
  if (!r.valid) return;
  const double rr = block_sum(item_part(part, r.l, np, r), r.bpc);
  if (threadIdx.x == 0) {
    Scal& s = scal[r.item];
    s.rr = rr;
    s.rho = rr;  // r0* = r0
    s.beta = 0.0;
    s.alpha = 0.0;
    s.iter = 0;
    s.rel = sqrt(rr / s.b2);
    s.rel_true = s.rel;
    s.best_rel = s.rel;
    s.best_iter = 0;
    record_hist(s);
    if (!finite_d(rr)) s.done = kBreakdown;
    else if (rr <= s.tol2 * s.b2) s.done = kConverged;
    else if (s.max_iter <= 0) s.done = kCap;
    else s.done = kRunning;
  }
}

// alpha = (r, r) / (A p, p) for CG; alpha = (r, r*) / (A p, p*) for BiCG
static __global__ void k_scal_alpha(Scal* scal, const double* part, int np, int ncell, int nl, int bicg) {
  const ItemRef r = item_ref(np, ncell, nl);
  if (!r.valid) return;
  const double den = block_sum(item_part(part, r.l, np, r), r.bpc);
  if (threadIdx.x == 0) {
    Scal& s = scal[r.item];
    if (s.done != kRunning) return;
    s.den = den;
    const double num = bicg ? s.rho : s.rr;
    if (!finite_d(den) || (!bicg && den <= 0.0) || den == 0.0) s.done = kBreakdown;
    else s.alpha = num / den;
  }
}

// CG: beta = (r+, r+) / (r, r); convergence on the recursive residual.
// BiCG: beta = (r+, r*+) / (r, r*); convergence on (r+, r+).
// xpar (CG with the x step deferred): 0 after an iteration that left its x
// step owed, 1 after one that settled it, -1 when x moves every iteration.
static __global__ void k_scal_beta(Scal* scal, const double* part, int np, int ncell, int nl, int bicg,
                                   int xpar) {
  const ItemRef r = item_ref(np, ncell, nl);
  if (!r.valid) return;
  double rho_new = 0.0, rr_new, pp = 0.0;
  const bool want_pp = scal[r.item].hist_eta_r != nullptr;
  if (bicg) {
    rho_new = block_sum(item_part(part, r.l, np, r), r.bpc);
    rr_new = block_sum(item_part(part, kMaxLoads + r.l, np, r), r.bpc);
    if (want_pp) pp = block_sum(item_part(part, 2 * kMaxLoads + r.l, np, r), r.bpc);
  } else {
    rr_new = block_sum(item_part(part, r.l, np, r), r.bpc);
    if (want_pp) pp = block_sum(item_part(part, kMaxLoads + r.l, np, r), r.bpc);
  }
  if (threadIdx.x == 0) {
    Scal& s = scal[r.item];
    if (s.done != kRunning) return;
    if (xpar == 0) {
      s.alpha_x = s.alpha;
      s.xpend = 1;
    } else if (xpar == 1) {
      s.xpend = 0;
    }
    // eta_r of this step: ||L0 alpha p|| / ||e0|| (Eq. errR_def), index = step
    if (s.hist_eta_r != nullptr && s.iter < s.hist_cap)
      s.hist_eta_r[s.iter] = s.l0iso > 0.0 ? s.l0iso * fabs(s.alpha) * sqrt(pp / s.b2) : NAN;
    s.iter += 1;
    s.rel = sqrt(rr_new / s.b2);
    record_hist(s);
    if (!finite_d(rr_new)) { s.done = kBreakdown; return; }
    if (rr_new <= s.tol2 * s.b2) { s.rr = rr_new; s.done = kConverged; return; }
    if (s.iter >= s.max_iter) { s.rr = rr_new; s.done = kCap; return; }
    if (stalled(s)) { s.rr = rr_new; s.done = kStalled; return; }
    if (bicg) {
      if (!finite_d(rho_new) || rho_new == 0.0) { s.done = kBreakdown; return; }
      s.beta = rho_new / s.rho;
      s.rho = rho_new;
      s.rr = rr_new;
    } else {
      s.beta = rr_new / s.rr;
      s.rr = rr_new;
    }
  }
}

// Fixed point: the epilogue produced ||e_new - e||^2 = ||r(e)||^2.
static __global__ void k_scal_fixed(Scal* scal, const double* part, int np, int ncell, int nl) {
  const ItemRef r = item_ref(np, ncell, nl);
  if (!r.valid) return;
  const double rr = block_sum(item_part(part, r.l, np, r), r.bpc);
  if (threadIdx.x == 0) {
    Scal& s = scal[r.item];
    if (s.done != kRunning) return;
    s.rr = rr;
    s.rel = sqrt(rr / s.b2);
    record_hist(s);
    // the step e_{m+1} - e_m of the fixed point is the residual of e_m
    if (s.hist_eta_r != nullptr && s.iter < s.hist_cap)
      s.hist_eta_r[s.iter] = s.l0iso > 0.0 ? s.l0iso * s.rel : NAN;
    if (!finite_d(rr)) { s.done = kBreakdown; return; }
    s.iter += 1;
    if (rr <= s.tol2 * s.b2) { s.done = kConverged; return; }
    if (s.iter >= s.max_iter) { s.done = kCap; return; }
    if (stalled(s)) { s.done = kStalled; return; }
  }
}

// eta_e history (Eq. errE_def): after the equilibrium-norm passes on the
// current iterate, hist_eta_e[iter] = sqrt(sum_k |xi . j^(k)|^2 / |j^(0)|^2)
// from the two partial rows of the kColEta pass (single item).
static __global__ void k_eta_record(const double* part, int np, const Scal* scal) {
  const double num = block_sum(part, np);
  const double den = block_sum(part + np, np);
  if (threadIdx.x == 0) {
    const Scal& s = scal[0];
    if (s.hist_eta_e != nullptr && s.iter < s.hist_cap) s.hist_eta_e[s.iter] = den > 0.0 ? sqrt(num / den) : 0.0;
  }
}

// out[cell * nv + v] = sum of row v of the partials over the cell's slots.
static __global__ void k_reduce_items(const double* part, int np, int ncell, int nv, double* out) {
  const ItemRef r = item_ref(np, ncell, nv);
  if (!r.valid) return;
  const double x = block_sum(item_part(part, r.l, np, r), r.bpc);
  if (threadIdx.x == 0) out[r.item] = x;
}

inline int item_blocks(int items) { return items; }

// Condition of a device-side iteration loop (a while node of a CUDA graph):
// one more body of iterations while an item is running and fewer than
// loop[1] bodies have run (loop[0] counts them).  One CTA; every loop ends.
static __global__ void k_loop_cond(cudaGraphConditionalHandle h, const Scal* scal, int items, int* loop) {
  int run = 0;
  for (int i = threadIdx.x; i < items; i += blockDim.x) run |= scal[i].done == kRunning;
  run = __syncthreads_or(run);
  if (threadIdx.x == 0) {
    const int rounds = ++loop[0];
    cudaGraphSetConditional(h, (run && rounds < loop[1]) ? 1u : 0u);
  }
}

// ----------------------------------------------------------------------------
// misc elementwise kernels
// ----------------------------------------------------------------------------
// x[c * nodes + i] = E[c]
template <typename T>
__global__ void k_fill_const(T* x, long long nodes, int d, double E0, double E1, double E2) {
  const double E[3] = {E0, E1, E2};
  const long long len = nodes * d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = T(E[i / nodes]);
}

// Per-cell partial sums of (Tab[phase] e)_c over the cell's nodes (effective
// tensor column); blocks are split evenly between cells, slot c of block b.
template <typename T, int D>
__global__ void k_current_sum(const T* e, const uint8_t* phase, const double* tab, long long nodes,
                              int ncell, long long cell_nodes, int tab_stride, double* part) {
  const int bpc = gridDim.x / ncell;
  const int cell = blockIdx.x / bpc;
  const long long t = (long long)(blockIdx.x - cell * bpc) * blockDim.x + threadIdx.x;
  const long long stride = (long long)bpc * blockDim.x;
  const double* tb = tab + (size_t)cell * tab_stride;
  double acc[D];
#pragma unroll
  for (int c = 0; c < D; ++c) acc[c] = 0.0;
  const long long base = (long long)cell * cell_nodes;
  for (long long i = t; i < cell_nodes; i += stride) {
    const int ph = phase[base + i];
    double v[D];
#pragma unroll
    for (int c = 0; c < D; ++c) v[c] = (double)e[c * nodes + base + i];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double s = 0.0;
#pragma unroll
      for (int b2 = 0; b2 < D; ++b2) s += tb[(ph * D + c) * D + b2] * v[b2];
      acc[c] += s;
    }
  }
  block_reduce_store<D>(acc, D, part, gridDim.x, blockIdx.x);
}

// Per-cell partial sums of |M e|^2 with a constant D x D matrix (norms, eta_r numerator)
template <typename T, int D>
__global__ void k_matnorm2(const T* e, long long nodes, int ncell, long long cell_nodes, Mat3 m,
                           double* part) {
  const int bpc = gridDim.x / ncell;
  const int cell = blockIdx.x / bpc;
  const long long t = (long long)(blockIdx.x - cell * bpc) * blockDim.x + threadIdx.x;
  const long long stride = (long long)bpc * blockDim.x;
  T Mx[D * D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) Mx[i * D + j] = T(m.v[i * 3 + j]);
  DotAcc<T> dot;
  const long long base = (long long)cell * cell_nodes;
  for (long long i = t; i < cell_nodes; i += stride) {
    T v[D];
#pragma unroll
    for (int c = 0; c < D; ++c) v[c] = e[c * nodes + base + i];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T s = T(0);
#pragma unroll
      for (int b2 = 0; b2 < D; ++b2) s += Mx[c * D + b2] * v[b2];
      dot.add(s * s);
    }
  }
  double acc[1] = {dot.get()};
  block_reduce_store<1>(acc, 1, part, gridDim.x, blockIdx.x);
}

}  // namespace fh

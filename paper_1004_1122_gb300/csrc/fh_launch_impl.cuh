// fh_launch_impl.cuh -- launcher templates behind LaunchTable; included by the
// four fh_launch_*.cu translation units only.
#pragma once

#include <type_traits>

#include "fh_launch.cuh"

namespace fh {

// Raise the dynamic shared-memory limit of a kernel to everything the device
// allows (minus its static shared memory), so contexts of different sizes in
// one process never lower each other's limit.  `bytes` is the size this
// context needs; it must fit.
template <typename K>
static cudaError_t opt_in_smem(K kernel, size_t bytes) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const size_t cap = (size_t)optin - fa.sharedSizeBytes;
  if (bytes > cap) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
}

// Kernels with a compile-time FFT plan are built for float: 2-D with one load
// per launch and the 2187-point plan, 3-D (one or three loads) with the
// 243-point plan.  They are the hot kernels of one CG iteration (direction
// pass, A p pass, Green pass and, in 3-D, the middle-axis passes).  Launches
// whose run-time plan matches use them; everything else runs the
// run-time-plan kernels.
template <typename T, int D, int NL>
constexpr bool kHasCt = std::is_same<T, float>::value && (D == 2 || D == 3);
// 2-D one load: the 2187-point plan; 2-D two loads (the batched sweep's
// largest cells): the 729-point plan; 3-D: the 243-point plan.
template <int D, int NL>
using CtPlan = typename std::conditional<D == 2, typename std::conditional<NL == 1, Plan2187, Plan729>::type,
                                         Plan243>::type;

// The double-float passes of the float64 residual (Green pass, and the A x and
// residual row passes with double-float line FFTs) exist for the 2-D float64
// pipelines.
template <typename T, int D>
constexpr bool kHasDf = std::is_same<T, double>::value && D == 2;

// The 2187^2 Green pass also exists with its tuned tile shape compiled in:
// tiles of 2 frequencies x 2 components (Q = 4 columns), 81 threads per
// 2187-point column FFT.
constexpr int kGreenQ = 4;
constexpr int kGreenT = 81;
// The 3-D column passes (axis-1 forward and inverse, Green pass along axis 0)
// also exist with the tuned 243^3 three-load tile shape compiled in: tiles of
// 2 frequencies x 9 channels (Q = 18 columns), 9 threads per 243-point column
// FFT.
constexpr int kCol3Q = 18;
constexpr int kCol3T = 9;
// The 3-D three-load direction and A p passes with their tuned launch shape:
// one line per 64-thread CTA (five packed sequences of nine channels), tiles
// of 2 frequencies.
using RowShape243x3 = RowShape<64, 0, 2>;
// The two-load 729^2 Green pass (the batched sweep's largest cells) with
// tiles of 1 or 2 frequencies x 4 channels and 27 threads per column FFT.
constexpr int kGreen729T = 27;
// Likewise the 2187^2 A p pass: one line per 96-thread CTA, spectrum tiles of
// 2 frequencies; the threads per line FFT stay a launch argument (compiled in,
// they cost registers and the pass spilled: 44.0 against 41.7 us; the
// direction pass measured no gain from either form: 47.3 / 48.8 against 47.1).
using RowShape2187 = RowShape<96, 0, 2>;
template <typename RS, int M, typename T>
inline bool row_shape_is(const Launch& L, const RowArgs<T>& a) {
  return L.block == RS::nt && a.lpc == 1 && (RS::tpl == 0 || a.tpl == RS::tpl) && a.g.C == RS::cc &&
         a.nseq == (M + 1) / 2;
}
template <typename T>
inline bool row_shape_is_2187(const Launch& L, const RowArgs<T>& a) {
  return row_shape_is<RowShape2187, 2>(L, a);
}

template <typename T, int D, int NL>
struct Launchers {
  static cudaError_t set_smem(size_t rs, size_t c0, size_t c1) {
    cudaError_t e;
    if constexpr (kHasCt<T, D, NL>) {
      using P = CtPlan<D, NL>;
      if ((e = opt_in_smem(k_row_fwd<T, D, NL, kProDir, P>, rs)) != cudaSuccess) return e;
      if ((e = opt_in_smem(k_row_inv<T, D, NL, kEpiDir, P>, rs)) != cudaSuccess) return e;
      if constexpr (D == 2 && NL == 1)
        if ((e = opt_in_smem(k_row_inv<T, D, NL, kEpiDir, P, false, RowShape2187>, rs)) != cudaSuccess) return e;
      if constexpr (D == 3 && NL == 3) {
        if ((e = opt_in_smem(k_row_fwd<T, D, NL, kProDir, P, false, RowShape243x3>, rs)) != cudaSuccess) return e;
        if ((e = opt_in_smem(k_row_inv<T, D, NL, kEpiDir, P, false, RowShape243x3>, rs)) != cudaSuccess) return e;
      }
      if constexpr (D == 2 && NL == 2) {
        if ((e = opt_in_smem(k_col<T, D, kColGreen, P, 4, kGreen729T>, c0)) != cudaSuccess) return e;
        if ((e = opt_in_smem(k_col<T, D, kColGreen, P, 8, kGreen729T>, c0)) != cudaSuccess) return e;
      }
      if ((e = opt_in_smem(k_col<T, D, kColGreen, P>, c0)) != cudaSuccess) return e;
      if constexpr (D == 2 && NL == 1)
        if ((e = opt_in_smem(k_col<T, D, kColGreen, P, kGreenQ, kGreenT>, c0)) != cudaSuccess) return e;
      if constexpr (D == 3) {
        if ((e = opt_in_smem(k_col<T, D, kColFwd, P>, c1)) != cudaSuccess) return e;
        if ((e = opt_in_smem(k_col<T, D, kColInv, P>, c1)) != cudaSuccess) return e;
        if constexpr (NL == 3) {
          if ((e = opt_in_smem(k_col<T, D, kColFwd, P, kCol3Q, kCol3T>, c1)) != cudaSuccess) return e;
          if ((e = opt_in_smem(k_col<T, D, kColInv, P, kCol3Q, kCol3T>, c1)) != cudaSuccess) return e;
          if ((e = opt_in_smem(k_col<T, D, kColGreen, P, kCol3Q, kCol3T>, c0)) != cudaSuccess) return e;
        }
      }
    }
#define FH_SM(K, B) \
  if ((e = opt_in_smem(K, B)) != cudaSuccess) return e;
    FH_SM((k_row_fwd<T, D, NL, kProApply>), rs)
    FH_SM((k_row_fwd<T, D, NL, kProPlain>), rs)
    FH_SM((k_row_fwd<T, D, NL, kProDir>), rs)
    FH_SM((k_row_fwd<T, D, NL, kProDirPlain>), rs)
    FH_SM((k_row_inv<T, D, NL, kEpiApply>), rs)
    FH_SM((k_row_inv<T, D, NL, kEpiApplyT>), rs)
    FH_SM((k_row_inv<T, D, NL, kEpiDir>), rs)
    FH_SM((k_row_inv<T, D, NL, kEpiDirShadow>), rs)
    FH_SM((k_row_inv<T, D, NL, kEpiFixed>), rs)
    FH_SM((k_row_inv<T, D, NL, kEpiResid>), rs)
    FH_SM((k_col<T, D, kColGreen>), c0)
    FH_SM((k_col<T, D, kColEta>), c0)
    FH_SM((k_col<T, D, kColFwd>), c1)
    FH_SM((k_col<T, D, kColInv>), c1)
    if constexpr (NL == 1) {
      FH_SM((k_row_fwd<T, D, NL, kProApply, DynPlanX>), rs)
      FH_SM((k_row_fwd<T, D, NL, kProPlain, DynPlanX>), rs)
      FH_SM((k_row_fwd<T, D, NL, kProDir, DynPlanX>), rs)
      FH_SM((k_row_fwd<T, D, NL, kProDirPlain, DynPlanX>), rs)
      FH_SM((k_row_inv<T, D, NL, kEpiApply, DynPlanX>), rs)
      FH_SM((k_row_inv<T, D, NL, kEpiApplyT, DynPlanX>), rs)
      FH_SM((k_row_inv<T, D, NL, kEpiDir, DynPlanX>), rs)
      FH_SM((k_row_inv<T, D, NL, kEpiDirShadow, DynPlanX>), rs)
      FH_SM((k_row_inv<T, D, NL, kEpiFixed, DynPlanX>), rs)
      FH_SM((k_row_inv<T, D, NL, kEpiResid, DynPlanX>), rs)
      FH_SM((k_col<T, D, kColGreen, DynPlanX>), c0)
      FH_SM((k_col<T, D, kColEta, DynPlanX>), c0)
      FH_SM((k_col<T, D, kColFwd, DynPlanX>), c1)
      FH_SM((k_col<T, D, kColInv, DynPlanX>), c1)
    }
    if constexpr (kHasDf<T, D>) {
      FH_SM((k_col_green_df<>), c0)
      FH_SM((k_row_fwd<T, D, NL, kProApply, DynPlan, true>), rs)
      FH_SM((k_row_inv<T, D, NL, kEpiResid, DynPlan, true>), rs)
    }
#undef FH_SM
    return cudaSuccess;
  }
  static cudaError_t row_fwd(int pro, const Launch& L, const RowArgs<T>& a, cudaStream_t st) {
    if constexpr (kHasDf<T, D>) {
      if (a.twdf != nullptr) {  // float64 residual: double-float line FFTs
        if (pro != kProApply) return cudaErrorInvalidValue;
        k_row_fwd<T, D, NL, kProApply, DynPlan, true><<<L.grid, L.block, L.smem, st>>>(a);
        return cudaGetLastError();
      }
    }
    if constexpr (kHasCt<T, D, NL>) {
      using P = CtPlan<D, NL>;
      if (pro == kProDir && L.block <= RowBounds<P>::threads && cplan_is<P>(a.plan)) {
        if constexpr (D == 3 && NL == 3) {
          if (row_shape_is<RowShape243x3, D * NL>(L, a)) {
            k_row_fwd<T, D, NL, kProDir, P, false, RowShape243x3><<<L.grid, L.block, L.smem, st>>>(a);
            return cudaGetLastError();
          }
        }
        k_row_fwd<T, D, NL, kProDir, P><<<L.grid, L.block, L.smem, st>>>(a);
        return cudaGetLastError();
      }
    }
    if (a.plan.ext) {  // a length with a prime factor 11, 13 or 17
      if constexpr (NL == 1) {
        switch (pro) {
          case kProApply: k_row_fwd<T, D, NL, kProApply, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a); break;
          case kProPlain: k_row_fwd<T, D, NL, kProPlain, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a); break;
          case kProDir: k_row_fwd<T, D, NL, kProDir, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a); break;
          case kProDirPlain: k_row_fwd<T, D, NL, kProDirPlain, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a); break;
          default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
      }
      return cudaErrorInvalidValue;
    }
    switch (pro) {
      case kProApply: k_row_fwd<T, D, NL, kProApply><<<L.grid, L.block, L.smem, st>>>(a); break;
      case kProPlain: k_row_fwd<T, D, NL, kProPlain><<<L.grid, L.block, L.smem, st>>>(a); break;
      case kProDir: k_row_fwd<T, D, NL, kProDir><<<L.grid, L.block, L.smem, st>>>(a); break;
      case kProDirPlain: k_row_fwd<T, D, NL, kProDirPlain><<<L.grid, L.block, L.smem, st>>>(a); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  static cudaError_t row_inv(int epi, const Launch& L, const RowArgs<T>& a, cudaStream_t st) {
    if constexpr (kHasDf<T, D>) {
      if (a.twdf != nullptr) {  // float64 residual: double-float line FFTs
        if (epi != kEpiResid) return cudaErrorInvalidValue;
        k_row_inv<T, D, NL, kEpiResid, DynPlan, true><<<L.grid, L.block, L.smem, st>>>(a);
        return cudaGetLastError();
      }
    }
    if constexpr (kHasCt<T, D, NL>) {
      using P = CtPlan<D, NL>;
      if (epi == kEpiDir && L.block <= RowBounds<P>::threads && cplan_is<P>(a.plan)) {
        if constexpr (D == 3 && NL == 3) {
          if (row_shape_is<RowShape243x3, D * NL>(L, a)) {
            k_row_inv<T, D, NL, kEpiDir, P, false, RowShape243x3><<<L.grid, L.block, L.smem, st>>>(a);
            return cudaGetLastError();
          }
        }
        if constexpr (D == 2 && NL == 1) {
          if (row_shape_is_2187(L, a)) {
            k_row_inv<T, D, NL, kEpiDir, P, false, RowShape2187><<<L.grid, L.block, L.smem, st>>>(a);
            return cudaGetLastError();
          }
        }
        k_row_inv<T, D, NL, kEpiDir, P><<<L.grid, L.block, L.smem, st>>>(a);
        return cudaGetLastError();
      }
    }
    if (a.plan.ext) {  // a length with a prime factor 11, 13 or 17
      if constexpr (NL == 1) {
        switch (epi) {
          case kEpiApply: k_row_inv<T, D, NL, kEpiApply, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a); break;
          case kEpiApplyT: k_row_inv<T, D, NL, kEpiApplyT, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a); break;
          case kEpiDir: k_row_inv<T, D, NL, kEpiDir, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a); break;
          case kEpiDirShadow:
            k_row_inv<T, D, NL, kEpiDirShadow, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a);
            break;
          case kEpiFixed: k_row_inv<T, D, NL, kEpiFixed, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a); break;
          case kEpiResid: k_row_inv<T, D, NL, kEpiResid, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a); break;
          default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
      }
      return cudaErrorInvalidValue;
    }
    switch (epi) {
      case kEpiApply: k_row_inv<T, D, NL, kEpiApply><<<L.grid, L.block, L.smem, st>>>(a); break;
      case kEpiApplyT: k_row_inv<T, D, NL, kEpiApplyT><<<L.grid, L.block, L.smem, st>>>(a); break;
      case kEpiDir: k_row_inv<T, D, NL, kEpiDir><<<L.grid, L.block, L.smem, st>>>(a); break;
      case kEpiDirShadow: k_row_inv<T, D, NL, kEpiDirShadow><<<L.grid, L.block, L.smem, st>>>(a); break;
      case kEpiFixed: k_row_inv<T, D, NL, kEpiFixed><<<L.grid, L.block, L.smem, st>>>(a); break;
      case kEpiResid: k_row_inv<T, D, NL, kEpiResid><<<L.grid, L.block, L.smem, st>>>(a); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  static cudaError_t col(int mode, const Launch& L, const ColArgs<T>& a, cudaStream_t st) {
    if constexpr (kHasCt<T, D, NL>) {
      using P = CtPlan<D, NL>;
      if (L.block <= ColBounds<P>::threads && cplan_is<P>(a.b.plan)) {
        if constexpr (D == 3 && NL == 3) {
          if (a.b.Q == kCol3Q && a.b.tpc == kCol3T) {  // the tuned 243^3 three-load tile shape
            switch (mode) {
              case kColFwd: k_col<T, D, kColFwd, P, kCol3Q, kCol3T><<<L.grid, L.block, L.smem, st>>>(a); break;
              case kColInv: k_col<T, D, kColInv, P, kCol3Q, kCol3T><<<L.grid, L.block, L.smem, st>>>(a); break;
              case kColGreen: k_col<T, D, kColGreen, P, kCol3Q, kCol3T><<<L.grid, L.block, L.smem, st>>>(a); break;
              default: return cudaErrorInvalidValue;
            }
            return cudaGetLastError();
          }
        }
        if (mode == kColGreen) {
          if constexpr (D == 2 && NL == 2) {
            if (a.b.tpc == kGreen729T && a.b.stride_i == a.b.Q) {  // the 729^2 two-load tiles
              if (a.b.Q == 4) {
                k_col<T, D, kColGreen, P, 4, kGreen729T><<<L.grid, L.block, L.smem, st>>>(a);
                return cudaGetLastError();
              }
              if (a.b.Q == 8) {
                k_col<T, D, kColGreen, P, 8, kGreen729T><<<L.grid, L.block, L.smem, st>>>(a);
                return cudaGetLastError();
              }
            }
          }
          if constexpr (D == 2 && NL == 1) {
            if (a.b.Q == kGreenQ && a.b.tpc == kGreenT && a.b.stride_i == kGreenQ) {  // the tuned 2187^2 tile shape
              k_col<T, D, kColGreen, P, kGreenQ, kGreenT><<<L.grid, L.block, L.smem, st>>>(a);
              return cudaGetLastError();
            }
          }
          k_col<T, D, kColGreen, P><<<L.grid, L.block, L.smem, st>>>(a);
          return cudaGetLastError();
        }
        if constexpr (D == 3) {
          if (mode == kColFwd) {
            k_col<T, D, kColFwd, P><<<L.grid, L.block, L.smem, st>>>(a);
            return cudaGetLastError();
          }
          if (mode == kColInv) {
            k_col<T, D, kColInv, P><<<L.grid, L.block, L.smem, st>>>(a);
            return cudaGetLastError();
          }
        }
      }
    }
    if (a.b.plan.ext) {  // a length with a prime factor 11, 13 or 17
      if constexpr (NL == 1) {
        switch (mode) {
          case kColFwd: k_col<T, D, kColFwd, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a); break;
          case kColInv: k_col<T, D, kColInv, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a); break;
          case kColGreen: k_col<T, D, kColGreen, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a); break;
          case kColEta: k_col<T, D, kColEta, DynPlanX><<<L.grid, L.block, L.smem, st>>>(a); break;
          default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
      }
      return cudaErrorInvalidValue;
    }
    switch (mode) {
      case kColFwd: k_col<T, D, kColFwd><<<L.grid, L.block, L.smem, st>>>(a); break;
      case kColInv: k_col<T, D, kColInv><<<L.grid, L.block, L.smem, st>>>(a); break;
      case kColGreen: k_col<T, D, kColGreen><<<L.grid, L.block, L.smem, st>>>(a); break;
      case kColEta: k_col<T, D, kColEta><<<L.grid, L.block, L.smem, st>>>(a); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  static cudaError_t col_pipe(const Launch& L, const ColArgs<T>& a, cudaStream_t st) {
    if constexpr (kHasCt<T, D, NL> && D == 2 && NL == 1) {
      if (cplan_is<Plan2187>(a.b.plan)) {
        k_col_pipe<T, D, Plan2187><<<L.grid, L.block, L.smem, st>>>(a);
        return cudaGetLastError();
      }
    }
    if constexpr (D == 2) {
      k_col_pipe<T, D><<<L.grid, L.block, L.smem, st>>>(a);
      return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
  }
  static cudaError_t col_df(const Launch& L, const ColArgs<T>& a, const void* tw, cudaStream_t st) {
    if constexpr (kHasDf<T, D>) {
      k_col_green_df<><<<L.grid, L.block, L.smem, st>>>(a, static_cast<const dfc*>(tw));
      return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
  }
  static cudaError_t set_smem_pipe(size_t bytes) {
    if constexpr (kHasCt<T, D, NL> && D == 2 && NL == 1) {
      cudaError_t e = opt_in_smem(k_col_pipe<T, D, Plan2187>, bytes);
      if (e != cudaSuccess) return e;
    }
    if constexpr (D == 2) return opt_in_smem(k_col_pipe<T, D>, bytes);
    return cudaErrorInvalidValue;
  }
  static cudaError_t occupancy_pipe(int block, size_t smem, int* per_sm) {
    if constexpr (D == 2) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_col_pipe<T, D>, block, smem);
    return cudaErrorInvalidValue;
  }
  static cudaError_t cg_update(const Launch& L, const VecArgs<T>& v, cudaStream_t st) {
#define FH_CGU(PP, XM) k_cg_update<T, NL, PP, XM><<<L.grid, L.block, 0, st>>>(v)
    switch (v.xmode * 2 + (v.want_pp ? 1 : 0)) {
      case 0: FH_CGU(false, 0); break;
      case 1: FH_CGU(true, 0); break;
      case 2: FH_CGU(false, 1); break;
      case 3: FH_CGU(true, 1); break;
      case 4: FH_CGU(false, 2); break;
      case 5: FH_CGU(true, 2); break;
      default: return cudaErrorInvalidValue;
    }
#undef FH_CGU
    return cudaGetLastError();
  }
  static cudaError_t cg_flush(const Launch& L, const VecArgs<T>& v, cudaStream_t st) {
    k_cg_flush<T, NL><<<L.grid, L.block, 0, st>>>(v);
    return cudaGetLastError();
  }
  static cudaError_t bicg_update(const Launch& L, const VecArgs<T>& v, cudaStream_t st) {
    k_bicg_update<T, NL><<<L.grid, L.block, 0, st>>>(v);
    return cudaGetLastError();
  }
  static cudaError_t current_sum(const Launch& L, const T* e, const uint8_t* ph, const double* tab,
                                 long long nodes, int ncell, long long cell_nodes, int tab_stride,
                                 double* part, cudaStream_t st) {
    k_current_sum<T, D><<<L.grid, L.block, 0, st>>>(e, ph, tab, nodes, ncell, cell_nodes, tab_stride, part);
    return cudaGetLastError();
  }
  static cudaError_t matnorm2(const Launch& L, const T* e, long long nodes, int ncell,
                              long long cell_nodes, const Mat3& m, double* part, cudaStream_t st) {
    k_matnorm2<T, D><<<L.grid, L.block, 0, st>>>(e, nodes, ncell, cell_nodes, m, part);
    return cudaGetLastError();
  }
  static int ct_plan(const FFTPlan& prow, const Launch& row, const FFTPlan& pc0, const Launch& col0,
                     const FFTPlan& pc1, const Launch& col1) {
    if constexpr (kHasCt<T, D, NL>) {
      using P = CtPlan<D, NL>;
      bool ok = row.block <= RowBounds<P>::threads && cplan_is<P>(prow) &&
                col0.block <= ColBounds<P>::threads && cplan_is<P>(pc0);
      if (D == 3) ok = ok && col1.block <= ColBounds<P>::threads && cplan_is<P>(pc1);
      return ok ? P::n : 0;
    }
    return 0;
  }
  static LaunchTable<T> table() {
    LaunchTable<T> t;
    t.D = D;
    t.NL = NL;
    t.set_smem = &set_smem;
    t.row_fwd = &row_fwd;
    t.row_inv = &row_inv;
    t.col = &col;
    if (D == 2) {
      t.col_pipe = &col_pipe;
      t.set_smem_pipe = &set_smem_pipe;
      t.occupancy_pipe = &occupancy_pipe;
    }
    if (kHasDf<T, D>) t.col_df = &col_df;
    t.cg_update = &cg_update;
    t.cg_flush = &cg_flush;
    t.bicg_update = &bicg_update;
    t.current_sum = &current_sum;
    t.matnorm2 = &matnorm2;
    t.ct_plan = &ct_plan;
    return t;
  }
};

}  // namespace fh

// fh_noalloc.cu -- fh_apply_noalloc: one float64 operator application that
// allocates no device memory.
//
// Who needs this: callers that cannot call cudaMalloc -- code running inside a
// host framework that owns all device memory through its own pool and forbids
// outside allocations, latency-critical loops where cudaMalloc's implicit
// device synchronisation is unacceptable, or embedded users with a fixed
// device-memory budget decided at load time.  They pass inputs and outputs
// they already own; the spectrum scratch, the twiddle tables and the dL table
// of this call live in the file-scope arrays below, which every GPU that loads
// the library holds until the process exits (kScratchBytes + tables, about
// 16.1 MiB per device).
//
// Sharing: every call on a device uses the same arrays and leaves its contents
// behind.  Each call writes every scratch element before reading it (the
// forward row pass stores the whole tiled half spectrum, padding included), so
// nothing needs clearing between calls.  Calls whose GPU work overlaps (two
// streams, or two host threads) race on the arrays and give wrong results; the
// caller must order them.
//
// Set-up: the first call on each device, with that device current, looks up
// the device addresses of the arrays (cudaGetSymbolAddress) and raises the
// pass kernels' shared-memory limit; both are kept for the life of the
// process.  That first call should come before any stream capture on the
// device.  A cudaDeviceReset (or any other teardown of the device's primary
// context) after it is not supported: the kept addresses would be stale.
//
// Tables: every call fills the twiddle and dL arrays with a small kernel on
// the caller's stream (the dL values travel as a by-value kernel argument), so
// after the set-up every operation of a call is a kernel launch on that stream
// and nothing is staged from host memory.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/fh.h"
#include "fh_launch.cuh"
#include "fh_plan.h"

namespace {

constexpr size_t kScratchBytes = 16u << 20;  // 16 MiB: the float64 half spectrum
constexpr int kMaxAxis = 2187;               // longest axis accepted
constexpr int kMaxDevices = 64;
constexpr int kTabEntries = 256 * 9;         // every uint8 phase id, d <= 3

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) double2 g_tw[3 * kMaxAxis];
static __device__ __align__(256) double g_tab[kTabEntries];

struct DeviceSymbols {
  bool ready = false;
  unsigned char* scratch = nullptr;
  double2* tw = nullptr;
  double* tab = nullptr;
};

// The dL table of one call, passed by value (18 KB of kernel parameters).
struct DLTable {
  double v[kTabEntries];
};

// g_tw[off_k + m] = exp(-2 pi i m / n_k) for the (up to) three axis lengths,
// back to back; g_tab[i] = dL entry i for i < nt and 0 beyond (phase ids that
// have no tensor act as L = L0).
__global__ void k_fill_tables(int n0, int n1, int n2, DLTable dl, int nt) {
  const int total = n0 + n1 + n2;
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    int m = i, n = n0;
    if (m >= n0) {
      m -= n0;
      n = n1;
      if (m >= n1) {
        m -= n1;
        n = n2;
      }
    }
    double sn, cs;
    sincospi(2.0 * (double)m / (double)n, &sn, &cs);
    g_tw[i] = make_double2(cs, -sn);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kTabEntries; i += stride)
    g_tab[i] = i < nt ? dl.v[i] : 0.0;
}

DeviceSymbols g_dev[kMaxDevices];
std::mutex g_mu;

void set_err(char* buf, size_t len, const char* msg) {
  if (buf && len > 0) {
    std::snprintf(buf, len, "%s", msg);
  }
}

bool spd_small(const double* A, int n) {
  double a[9];
  for (int i = 0; i < n * n; ++i) a[i] = A[i];
  double scale = 0.0;
  for (int i = 0; i < n * n; ++i) scale = std::fmax(scale, std::fabs(a[i]));
  if (!(scale > 0.0) || !std::isfinite(scale)) return false;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j)
      if (std::fabs(a[i * n + j] - a[j * n + i]) > 1e-12 * scale) return false;
  for (int j = 0; j < n; ++j) {  // in-place Cholesky
    double s = a[j * n + j];
    for (int k = 0; k < j; ++k) s -= a[j * n + k] * a[j * n + k];
    if (!(s > 1e-14 * scale)) return false;
    a[j * n + j] = std::sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = a[i * n + j];
      for (int k = 0; k < j; ++k) t -= a[i * n + k] * a[j * n + k];
      a[i * n + j] = t / a[j * n + j];
    }
  }
  return true;
}

fh_status device_setup(DeviceSymbols& s, char* errbuf, size_t errlen) {
  cudaError_t e = cudaGetSymbolAddress((void**)&s.scratch, g_scratch);
  if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&s.tw, g_tw);
  if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&s.tab, g_tab);
  // raise the pass kernels' dynamic shared-memory limit to the device maximum
  // once (the limit does not depend on the grid)
  if (e == cudaSuccess) e = fh::launch_table<double>(2, 1).set_smem(0, 0, 0);
  if (e == cudaSuccess) e = fh::launch_table<double>(3, 1).set_smem(0, 0, 0);
  if (e != cudaSuccess) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "device set-up: %s", cudaGetErrorString(e));
    set_err(errbuf, errlen, msg);
    return FH_ERR_CUDA;
  }
  s.ready = true;
  return FH_OK;
}

inline int round_up32(int x) { return (x + 31) / 32 * 32; }

}  // namespace

extern "C" fh_status fh_apply_noalloc(int d, const int* N, const double* Y, const uint8_t* phase,
                                      int nphase, const double* L, const double* L0,
                                      const double* e_in, double* e_out, int transpose,
                                      void* stream, char* errbuf, size_t errlen) {
  using namespace fh;
  if (d != 2 && d != 3) { set_err(errbuf, errlen, "d must be 2 or 3"); return FH_ERR_ARG; }
  if (!N || !phase || !L || !L0 || !e_in || !e_out || nphase < 1 || nphase > 256) {
    set_err(errbuf, errlen, "null pointer or nphase outside 1..256");
    return FH_ERR_ARG;
  }
  long long nodes = 1;
  for (int a = 0; a < d; ++a) {
    if (N[a] < 3) { set_err(errbuf, errlen, "axis length < 3"); return FH_ERR_ARG; }
    if (N[a] > kMaxAxis) { set_err(errbuf, errlen, "axis length > 2187"); return FH_ERR_UNSUPPORTED; }
    if (Y && !(Y[a] > 0.0 && std::isfinite(Y[a]))) { set_err(errbuf, errlen, "bad Y"); return FH_ERR_ARG; }
    nodes *= N[a];
  }
  for (int p = 0; p < nphase; ++p)
    if (!spd_small(L + (size_t)p * d * d, d)) { set_err(errbuf, errlen, "phase tensor not SPD"); return FH_ERR_NOT_SPD; }
  if (!spd_small(L0, d)) { set_err(errbuf, errlen, "L0 not SPD"); return FH_ERR_NOT_SPD; }

  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_err(errbuf, errlen, "no usable current device");
    return FH_ERR_CUDA;
  }
  DeviceSymbols sym;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev[dev].ready) {
      fh_status st = device_setup(g_dev[dev], errbuf, errlen);
      if (st != FH_OK) return st;
    }
    sym = g_dev[dev];
  }
  int sms = 0, optin = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    set_err(errbuf, errlen, "device attribute query failed");
    return FH_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;

  // ---- geometry and tiling (float64, one load) -------------------------
  Geom g;
  std::memset(&g, 0, sizeof g);
  g.d = d;
  for (int a = 0; a < 3; ++a) g.n[a] = a < d ? N[a] : 1;
  g.nlast = N[d - 1];
  g.H = g.nlast / 2 + 1;  // half spectrum: 0 .. floor(n / 2) (the Nyquist bin of an even axis)
  g.nodes = nodes;
  g.nlines = (int)(nodes / g.nlast);
  g.n1 = d == 3 ? N[1] : 1;
  g.M = d;
  g.nloads = 1;
  for (int a = 0; a < 3; ++a) g.invY[a] = a < d ? 1.0 / (Y ? Y[a] : 1.0) : 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) g.L0[i * 3 + j] = L0[i * d + j];
  g.inv_nodes = 1.0 / (double)nodes;

  FFTPlan prow, pc0, pc1;
  int tpl = 0, tpc0 = 0, tpc1 = 0;
  if (!make_fft_plan(g.nlast, true, kRowMaxThreads, prow, tpl) ||
      !make_fft_plan(N[0], true, kColMaxThreads, pc0, tpc0) ||
      (d == 3 && !make_fft_plan(N[1], true, kColMaxThreads, pc1, tpc1))) {
    set_err(errbuf, errlen, "axis lengths must factor into 2, 3, 5, 7, 11, 13 and 17");
    return FH_ERR_UNSUPPORTED;
  }
  const size_t esz = sizeof(double2);
  const int M = d;
  const size_t smem_green = std::min<size_t>(150 * 1024, (size_t)optin - 4096);
  int C = 0;
  for (int cand : {16, 8, 4, 2, 1}) {
    const int Tt = (g.H + cand - 1) / cand;
    if (cand > 1 && double(Tt * cand - g.H) / g.H > 0.15) continue;
    if ((size_t)N[0] * cand * M * esz > smem_green || round_up32(cand * M * tpc0) > kColMaxThreads) continue;
    if (d == 3 && ((size_t)N[1] * cand * M * esz > smem_green || round_up32(cand * M * tpc1) > kColMaxThreads))
      continue;
    C = cand;
    break;
  }
  if (C == 0) { set_err(errbuf, errlen, "no column tiling fits"); return FH_ERR_UNSUPPORTED; }
  g.C = C;
  g.Tt = (g.H + C - 1) / C;
  g.cshift = 0;
  while ((1 << g.cshift) < C) ++g.cshift;
  g.ncell = 1;
  g.lines_cell = g.nlines;
  g.cell_nodes = nodes;
  g.tab_stride = 256 * d * d;
  const size_t spec_bytes = (size_t)g.Tt * C * g.nlines * M * esz;
  if (spec_bytes > kScratchBytes) {
    char msg[200];
    std::snprintf(msg, sizeof msg, "grid needs %zu bytes of spectrum scratch; the static limit is %zu",
                  spec_bytes, kScratchBytes);
    set_err(errbuf, errlen, msg);
    return FH_ERR_UNSUPPORTED;
  }
  const long long CM = (long long)C * M;

  int lpc = std::max(1, 256 / std::max(1, tpl * M / 2));
  lpc = std::min(lpc, std::max(1, (g.nlines + 2 * sms - 1) / (2 * sms)));
  while (lpc > 1 && (size_t)((lpc * M + 1) / 2) * g.nlast * esz > 96 * 1024) --lpc;
  if ((lpc * M) % 2 && lpc > 1) --lpc;
  while (lpc > 1 && round_up32(((lpc * M + 1) / 2) * tpl) > kRowMaxThreads) --lpc;
  const int nseq = (lpc * M + 1) / 2;
  Launch row;
  row.block = round_up32(nseq * tpl);
  row.grid = (g.nlines + lpc - 1) / lpc;
  row.smem = (size_t)nseq * g.nlast * esz + (size_t)kTabEntries / 9 * d * d * sizeof(double);
  if (row.block > kRowMaxThreads || row.smem > (size_t)optin) {
    set_err(errbuf, errlen, "row pass does not fit one CTA");
    return FH_ERR_UNSUPPORTED;
  }
  ColArgsBase cb0, cb1;
  std::memset(&cb0, 0, sizeof cb0);
  std::memset(&cb1, 0, sizeof cb1);
  int G = 1;
  if (d == 3) {
    for (int cand = g.n1; cand >= 1; --cand) {
      if (g.n1 % cand) continue;
      if ((size_t)N[0] * cand * CM * esz > std::min<size_t>(100 * 1024, smem_green)) continue;
      if (round_up32((int)(cand * CM) * tpc0) > kColMaxThreads) continue;
      G = cand;
      break;
    }
  }
  cb0.g = g;
  cb0.plan = pc0;
  cb0.Q = (int)(G * CM);
  cb0.tpc = tpc0;
  cb0.G = G;
  cb0.axis = 0;
  cb0.base_outer = (long long)g.nlines * CM;
  cb0.stride_i = d == 2 ? CM : (long long)g.n1 * CM;
  cb0.nb_inner = d == 2 ? 1 : (g.n1 + G - 1) / G;
  cb0.base_inner = d == 2 ? 0 : G * CM;
  Launch col0, col1;
  col0.block = round_up32(cb0.Q * tpc0);
  col0.grid = g.Tt * cb0.nb_inner;
  col0.smem = (size_t)N[0] * cb0.Q * esz;
  if (d == 3) {
    cb1.g = g;
    cb1.plan = pc1;
    cb1.Q = (int)CM;
    cb1.tpc = tpc1;
    cb1.G = 1;
    cb1.axis = 1;
    cb1.stride_i = CM;
    cb1.nb_inner = N[0];
    cb1.base_outer = (long long)g.nlines * CM;
    cb1.base_inner = (long long)g.n1 * CM;
    col1.block = round_up32(cb1.Q * tpc1);
    col1.grid = g.Tt * N[0];
    col1.smem = (size_t)N[1] * cb1.Q * esz;
  }
  LaunchTable<double> lt = launch_table<double>(d, 1);
  if (col0.smem > (size_t)optin || (d == 3 && col1.smem > (size_t)optin)) {
    set_err(errbuf, errlen, "column pass does not fit one CTA");
    return FH_ERR_UNSUPPORTED;
  }

  // ---- tables into the static arrays, filled on the device --------------
  const int lens[3] = {g.nlast, N[0], d == 3 ? N[1] : 0};
  const int offs[3] = {0, lens[0], lens[0] + lens[1]};
  {
    DLTable dl;
    const int nt = nphase * d * d;
    for (int p = 0; p < nphase; ++p)
      for (int i = 0; i < d * d; ++i) dl.v[p * d * d + i] = L[(size_t)p * d * d + i] - L0[i];
    for (int i = nt; i < kTabEntries; ++i) dl.v[i] = 0.0;
    k_fill_tables<<<8, 256, 0, st>>>(lens[0], lens[1], lens[2], dl, nt);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { set_err(errbuf, errlen, cudaGetErrorString(ce)); return FH_ERR_CUDA; }
  }

  // ---- the three (2-D) or five (3-D) passes ------------------------------
  RowArgs<double> a;
  std::memset(&a, 0, sizeof a);
  a.g = g;
  a.plan = prow;
  a.lpc = lpc;
  a.tpl = tpl;
  a.nseq = nseq;
  a.tw = sym.tw + offs[0];
  a.S = reinterpret_cast<double2*>(sym.scratch);
  a.phase = phase;
  a.tab = sym.tab;
  a.nphase = 256;
  for (int l = 0; l < kMaxLoads; ++l) {
    a.in[l] = e_in;
    a.out[l] = e_out;
  }
  ColArgs<double> c0{}, c1{};
  c0.b = cb0;
  c0.tw = sym.tw + offs[1];
  c0.S = a.S;
  c0.scal = nullptr;
  c0.part = nullptr;
  c1.b = cb1;
  c1.tw = sym.tw + offs[2];
  c1.S = a.S;
  c1.scal = nullptr;
  c1.part = nullptr;
  ce = lt.row_fwd(transpose ? kProPlain : kProApply, row, a, st);
  if (ce == cudaSuccess && d == 3) ce = lt.col(kColFwd, col1, c1, st);
  if (ce == cudaSuccess) ce = lt.col(kColGreen, col0, c0, st);
  if (ce == cudaSuccess && d == 3) ce = lt.col(kColInv, col1, c1, st);
  if (ce == cudaSuccess) ce = lt.row_inv(transpose ? kEpiApplyT : kEpiApply, row, a, st);
  if (ce != cudaSuccess) { set_err(errbuf, errlen, cudaGetErrorString(ce)); return FH_ERR_CUDA; }
  set_err(errbuf, errlen, "");
  return FH_OK;
}

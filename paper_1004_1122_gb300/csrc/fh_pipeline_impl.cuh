// fh_pipeline_impl.cuh -- member definitions of Pipeline<T>; included only by
// the two explicit-instantiation translation units.
#pragma once

#include <cstdlib>

#include <algorithm>
#include <cmath>

#include "fh_pipeline.cuh"

namespace fh {

#define FH_CK(call)                               \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return e_;             \
  } while (0)

#define FH_CKS(call)                                                          \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      err = std::string(#call) + ": " + cudaGetErrorString(e_);               \
      return 5; /* FH_ERR_CUDA */                                             \
    }                                                                         \
  } while (0)

static inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

template <typename T>
static int dev_alloc(std::vector<void*>& allocs, T** ptr, size_t count, std::string& err) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T) + 16);
  if (e != cudaSuccess) {
    err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return 4;  // FH_ERR_OOM
  }
  allocs.push_back(p);
  *ptr = static_cast<T*>(p);
  return 0;
}

template <typename T>
int Pipeline<T>::init(const Problem& pb, int nloads_, bool krylov, cudaStream_t stream,
                      std::string& err, const Tuning* want) {
  Tuning w;
  if (want) w = *want;
  uid = next_pipeline_uid();
  st = stream;
  nloads = nloads_;
  const bool f64 = sizeof(T) == 8;
  const size_t esz = sizeof(C);
  int dev = 0;
  FH_CKS(cudaGetDevice(&dev));
  FH_CKS(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int optin = 0;
  FH_CKS(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));

  const int d = pb.d;
  g.d = d;
  for (int a = 0; a < 3; ++a) g.n[a] = a < d ? pb.N[a] : 1;
  g.nlast = pb.N[d - 1];
  g.H = g.nlast / 2 + 1;  // half spectrum: 0 .. floor(n / 2) (the Nyquist bin of an even axis)
  g.nodes = pb.nodes;
  g.nlines = (int)(pb.nodes / g.nlast);
  g.n1 = d == 3 ? pb.N[1] : 1;
  g.M = d * nloads;
  g.nloads = nloads;
  ncell = pb.ncell < 1 ? 1 : pb.ncell;
  items = ncell * nloads;
  if (ncell > 1 && d != 2) {
    err = "batches of cells are 2-D only";
    return 1;
  }
  g.ncell = ncell;
  g.cell_nodes = pb.nodes / ncell;
  g.lines_cell = (int)(g.cell_nodes / pb.N[d - 1]);
  g.tab_stride = pb.nphase * d * d;
  for (int a = 0; a < 3; ++a) g.invY[a] = a < d ? 1.0 / pb.Y[a] : 0.0;
  for (int i = 0; i < 9; ++i) g.L0[i] = 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) g.L0[i * 3 + j] = pb.L0[i * d + j];
  g.inv_nodes = 1.0 / (double)g.cell_nodes;
  l0iso = g.L0[0];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (g.L0[i * 3 + j] != (i == j ? g.L0[0] : 0.0)) l0iso = 0.0;
  vlen = (long long)d * pb.nodes;
  phase = pb.d_phase;
  nphase = pb.nphase;
  lt = launch_table<T>(d, nloads);
  if (lt.row_fwd == nullptr) {
    err = "unsupported number of loads per launch for this dimension";
    return 9;
  }

  // FFT plans
  int tpc0 = 0, tpc1 = 0;
  if (!make_fft_plan(g.nlast, f64, kRowMaxThreads, prow, tpl, w.tpl) ||
      !make_fft_plan(pb.N[0], f64, kColMaxThreads, pcol0, tpc0, w.tpc0) ||
      (d == 3 && !make_fft_plan(pb.N[1], f64, kColMaxThreads, pcol1, tpc1, w.tpc1))) {
    err = "no FFT plan for this grid (axis lengths must factor into 2, 3, 5, 7, 11, 13 and 17)";
    return 9;  // FH_ERR_UNSUPPORTED
  }
  const bool ext = prow.ext || pcol0.ext || (d == 3 && pcol1.ext);
  if (ext && nloads != 1) {
    err = "even axis lengths and lengths with a prime factor 11, 13 or 17 run one load per launch only";
    return 9;
  }
  const int M = g.M;
  const size_t smem_green = std::min<size_t>(150 * 1024, (size_t)optin - 4096);
  // tile width C of the half spectrum
  int Cc = 0;
  for (int cand : {16, 8, 4, 2, 1}) {
    if (w.C && cand != w.C) continue;
    const int Tt = (g.H + cand - 1) / cand;
    const double pad = double(Tt * cand - g.H) / g.H;
    if (cand > 1 && pad > 0.15 && !w.C) continue;
    if (d == 2) {
      if ((size_t)pb.N[0] * cand * M * esz > smem_green) continue;
      if (round_up(cand * M * tpc0, 32) > kColMaxThreads) continue;
    } else {
      if ((size_t)pb.N[1] * cand * M * esz > smem_green) continue;
      if (round_up(cand * M * tpc1, 32) > kColMaxThreads) continue;
      if ((size_t)pb.N[0] * cand * M * esz > smem_green) continue;
      if (round_up(cand * M * tpc0, 32) > kColMaxThreads) continue;
    }
    Cc = cand;
    break;
  }
  if (Cc == 0) {
    err = "grid too large for the column tiling";
    return 9;
  }
  g.C = Cc;
  g.Tt = (g.H + Cc - 1) / Cc;
  g.cshift = 0;
  while ((1 << g.cshift) < Cc) ++g.cshift;
  const long long CM = (long long)Cc * M;

  // row passes
  {
    const int per_line_thr = std::max(1, tpl * M / 2);
    int l = std::max(1, 256 / per_line_thr);
    const int cap = std::max(1, (g.nlines + 2 * sms - 1) / (2 * sms));
    l = std::min(l, cap);
    while (l > 1 && ((size_t)((l * M + 1) / 2) * g.nlast * esz > 96 * 1024)) --l;
    if ((l * M) % 2 && l > 1) --l;
    if (w.lpc) l = w.lpc;
    while (ncell > 1 && l > 1 && g.lines_cell % l) --l;
    lpc = l;
    nseq = (lpc * M + 1) / 2;
    while (lpc > 1 && round_up(((lpc * M + 1) / 2) * tpl, 32) > kRowMaxThreads) --lpc;
    nseq = (lpc * M + 1) / 2;
    row.block = round_up(nseq * tpl, 32);
    row.grid = (g.nlines + lpc - 1) / lpc;
    row.smem = (size_t)nseq * g.nlast * esz + (size_t)std::max(1, nphase) * d * d * sizeof(T);
    if (row.block > kRowMaxThreads || row.smem > (size_t)optin || (w.lpc && lpc != w.lpc) ||
        (ncell > 1 && g.lines_cell % lpc)) {
      err = "row pass does not fit one CTA";
      return 9;
    }
  }
  // Green pass along axis 0
  {
    int G = 1;
    if (d == 3) {
      for (int cand = g.n1; cand >= 1; --cand) {
        if (g.n1 % cand) continue;
        if ((size_t)pb.N[0] * cand * CM * esz > std::min<size_t>(100 * 1024, smem_green)) continue;
        if (round_up((int)(cand * CM) * tpc0, 32) > kColMaxThreads) continue;
        G = cand;
        break;
      }
    }
    cb0.g = g;
    cb0.plan = pcol0;
    cb0.Q = (int)(G * CM);
    cb0.tpc = tpc0;
    cb0.G = G;
    cb0.axis = 0;
    cb0.base_outer = (long long)g.nlines * CM;
    if (d == 2) {
      cb0.stride_i = CM;
      cb0.nb_inner = ncell;
      cb0.base_inner = (long long)g.lines_cell * CM;
    } else {
      cb0.stride_i = (long long)g.n1 * CM;
      cb0.nb_inner = (g.n1 + G - 1) / G;
      cb0.base_inner = G * CM;
    }
    col0.block = round_up(cb0.Q * tpc0, 32);
    col0.grid = g.Tt * cb0.nb_inner;
    col0.smem = (size_t)pb.N[0] * cb0.Q * esz;
  }
  if (d == 3) {
    cb1.g = g;
    cb1.plan = pcol1;
    cb1.Q = (int)CM;
    cb1.tpc = tpc1;
    cb1.G = 1;
    cb1.axis = 1;
    cb1.stride_i = CM;
    cb1.nb_inner = pb.N[0];
    cb1.base_outer = (long long)g.nlines * CM;
    cb1.base_inner = (long long)g.n1 * CM;
    col1.block = round_up(cb1.Q * tpc1, 32);
    col1.grid = g.Tt * pb.N[0];
    col1.smem = (size_t)pb.N[1] * cb1.Q * esz;
  }
  tuning.C = g.C;
  tuning.lpc = lpc;
  tuning.tpl = tpl;
  tuning.tpc0 = tpc0;
  tuning.tpc1 = tpc1;
  vec.block = 256;
  {
    const long long cell_len = (long long)d * g.cell_nodes;
    const long long want = std::max<long long>(1, ((long long)sms * 4 + ncell - 1) / ncell);
    const long long bpc = std::max<long long>(1, std::min<long long>(want, (cell_len + 255) / 256));
    vec.grid = (int)(bpc * ncell);
  }
  part_stride = std::max(std::max(row.grid, col0.grid), vec.grid);

  FH_CKS(lt.set_smem(row.smem, col0.smem, d == 3 ? col1.smem : 0));

  // Persistent bulk-copy Green pass (2-D): two tile buffers per CTA, CTAs
  // sized to the SMs.  Needs 16-byte aligned, 16-byte multiple blocks.  It is
  // a tuning choice (Tuning::pipe, picked by the autotuner); without a
  // requested tuning the environment variable FH_GREEN_PIPE=1 selects it.
  green_pipe = false;
  {
    const char* env = std::getenv("FH_GREEN_PIPE");
    const bool allow = want ? want->pipe != 0 : (env && env[0] == '1');
    const size_t bytes = (size_t)pb.N[0] * cb0.Q * esz;
    const size_t smem = 128 + 2 * bytes;
    const bool aligned = bytes % 16 == 0 && (cb0.base_outer * esz) % 16 == 0 && (cb0.base_inner * esz) % 16 == 0;
    if (allow && d == 2 && !pcol0.ext && lt.col_pipe && aligned && col0.block <= kColPipeMaxThreads &&
        smem + 1024 <= (size_t)optin &&
        lt.set_smem_pipe(smem) == cudaSuccess) {
      int per_sm = 0;
      if (lt.occupancy_pipe(col0.block, smem, &per_sm) == cudaSuccess && per_sm > 0) {
        colp = col0;
        colp.smem = smem;
        colp.grid = std::min(col0.grid, sms * per_sm);
        green_pipe = true;
      }
    }
    cudaGetLastError();  // clear a refused opt-in
  }
  tuning.pipe = green_pipe ? 1 : 0;
  ct_plan = lt.ct_plan(prow, row, pcol0, green_pipe ? colp : col0, pcol1, col1);
  if (green_pipe && nloads != 1) ct_plan = 0;  // the persistent Green pass has no two-load plan

  // device buffers
  int rc;
  const size_t spec = (size_t)g.Tt * g.C * g.nlines * M;
  if ((rc = dev_alloc(allocs, &S, spec, err))) return rc;
  auto upload_tw = [&](int n, C** dst) -> int {
    std::vector<double> re, im;
    twiddles(n, re, im);
    std::vector<C> h(n);
    for (int m = 0; m < n; ++m) {
      h[m].x = T(re[m]);
      h[m].y = T(im[m]);
    }
    int r2 = dev_alloc(allocs, dst, n, err);
    if (r2) return r2;
    FH_CKS(cudaMemcpy(*dst, h.data(), n * sizeof(C), cudaMemcpyHostToDevice));
    return 0;
  };
  if ((rc = upload_tw(g.nlast, &tw_last))) return rc;
  if ((rc = upload_tw(pb.N[0], &tw0))) return rc;
  if (d == 3 && (rc = upload_tw(pb.N[1], &tw1))) return rc;
  if (d == 2 && lt.col_df) {
    // twiddles as complex double-floats: hi = fl32(w), lo = fl32(w - hi)
    auto upload_tw_df = [&](int n, dfc** dst) -> int {
      std::vector<double> re, im;
      twiddles(n, re, im);
      std::vector<dfc> h(n);
      for (int m = 0; m < n; ++m) {
        h[m].x = dfl(re[m]);
        h[m].y = dfl(im[m]);
      }
      int r2 = dev_alloc(allocs, dst, n, err);
      if (r2) return r2;
      FH_CKS(cudaMemcpy(*dst, h.data(), n * sizeof(dfc), cudaMemcpyHostToDevice));
      return 0;
    };
    if ((rc = upload_tw_df(pb.N[0], &tw0_df))) return rc;
    if ((rc = upload_tw_df(g.nlast, &tw_last_df))) return rc;
  }
  {
    const int nt = std::max(1, nphase) * d * d * ncell;
    std::vector<T> hd(nt), hl(nt);
    for (int i = 0; i < nphase * d * d * ncell; ++i) {
      hd[i] = T(pb.dL[i]);
      hl[i] = T(pb.L[i]);
    }
    if ((rc = dev_alloc(allocs, &dtab, nt, err))) return rc;
    {
      std::vector<T> hq(nt);
      for (int c = 0; c < ncell; ++c)
        for (int ph = 0; ph < std::max(1, nphase); ++ph)
          for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
              const double v = pb.L0cell.empty() ? pb.L0[i * d + j] : pb.L0cell[9 * c + i * 3 + j];
              hq[((size_t)c * std::max(1, nphase) + ph) * d * d + i * d + j] = T(v);
            }
      if ((rc = dev_alloc(allocs, &qtab, nt, err))) return rc;
      FH_CKS(cudaMemcpy(qtab, hq.data(), nt * sizeof(T), cudaMemcpyHostToDevice));
    }
    if ((rc = dev_alloc(allocs, &ltab, nt, err))) return rc;
    if ((rc = dev_alloc(allocs, &ltab64, nt, err))) return rc;
    FH_CKS(cudaMemcpy(dtab, hd.data(), nt * sizeof(T), cudaMemcpyHostToDevice));
    FH_CKS(cudaMemcpy(ltab, hl.data(), nt * sizeof(T), cudaMemcpyHostToDevice));
    FH_CKS(cudaMemcpy(ltab64, pb.L.data(), (size_t)nphase * d * d * ncell * sizeof(double),
                      cudaMemcpyHostToDevice));
  }
  if ((rc = dev_alloc(allocs, &d_loop, 2, err))) return rc;
  FH_CKS(cudaMallocHost(&h_loop, 2 * sizeof(int)));
  if ((rc = dev_alloc(allocs, &dev_err, 1, err))) return rc;
  FH_CKS(cudaMemset(dev_err, 0, sizeof(int)));
  FH_CKS(cudaMallocHost(&h_err, sizeof(int)));
  *h_err = 0;
  const int nscal = std::max(items, kMaxLoads);
  const int nred = std::max(std::max(items, ncell * d), 16);
  if ((rc = dev_alloc(allocs, &scal, nscal, err))) return rc;
  if ((rc = dev_alloc(allocs, &scal_aux, nscal, err))) return rc;
  if ((rc = dev_alloc(allocs, &part, (size_t)3 * kMaxLoads * part_stride, err))) return rc;
  if ((rc = dev_alloc(allocs, &d_red, nred, err))) return rc;
  FH_CKS(cudaMallocHost(&h_scal, 2 * nscal * sizeof(Scal)));
  FH_CKS(cudaMallocHost(&h_red, nred * sizeof(double)));
  std::memset(h_scal, 0, 2 * nscal * sizeof(Scal));
  if (!pb.L0cell.empty()) {
    if ((rc = dev_alloc(allocs, &L0cell_dev, (size_t)9 * ncell, err))) return rc;
    FH_CKS(cudaMemcpy(L0cell_dev, pb.L0cell.data(), 9 * ncell * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (krylov) {
    for (int l = 0; l < nloads; ++l) {
      if ((rc = dev_alloc(allocs, &x[l], vlen, err))) return rc;
      if ((rc = dev_alloc(allocs, &r[l], vlen, err))) return rc;
      if ((rc = dev_alloc(allocs, &p[l], vlen, err))) return rc;
      if ((rc = dev_alloc(allocs, &ap[l], vlen, err))) return rc;
      if ((rc = dev_alloc(allocs, &rhs[l], vlen, err))) return rc;
    }
  }
  return 0;
}

template <typename T>
void Pipeline<T>::release() {
  for (void* q : allocs) cudaFree(q);
  allocs.clear();
  if (h_scal) cudaFreeHost(h_scal);
  if (h_red) cudaFreeHost(h_red);
  if (h_err) cudaFreeHost(h_err);
  if (h_loop) cudaFreeHost(h_loop);
  loops.clear();
  h_scal = nullptr;
  h_red = nullptr;
  h_err = nullptr;
  h_loop = nullptr;
}

template <typename T>
RowArgs<T> Pipeline<T>::row_args() const {
  RowArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.g = g;
  a.plan = prow;
  a.lpc = lpc;
  a.tpl = tpl;
  a.nseq = nseq;
  a.tw = tw_last;
  a.S = S;
  a.phase = phase;
  a.tab = dtab;
  a.nphase = nphase;
  a.part = part;
  return a;
}

template <typename T>
cudaError_t Pipeline<T>::launch_row_fwd(int pro, const RowArgs<T>& a) {
  ++launches;
  return lt.row_fwd(pro, row, a, st);
}

template <typename T>
cudaError_t Pipeline<T>::launch_row_inv(int epi, const RowArgs<T>& a) {
  ++launches;
  return lt.row_inv(epi, row, a, st);
}

template <typename T>
cudaError_t Pipeline<T>::launch_green(int mode, Scal* sc, double* pt) {
  ColArgs<T> m;
  m.b = cb1;
  m.tw = tw1;
  m.S = S;
  m.scal = sc;
  m.part = pt;
  m.L0cell = L0cell_dev;
  ColArgs<T> a;
  a.b = cb0;
  a.tw = tw0;
  a.S = S;
  a.scal = sc;
  a.part = pt;
  a.L0cell = L0cell_dev;
  a.err = dev_err;
  m.err = dev_err;
  a.wait_ns = m.wait_ns = tma::wait_limit_ns();
  if (g.d == 3) {
    ++launches;
    FH_CK(lt.col(kColFwd, col1, m, st));
  }
  ++launches;
  if (mode == kColEta) return lt.col(kColEta, col0, a, st);
  if (df_green && g.d == 2) return lt.col_df(col0, a, tw0_df, st);
  if (green_pipe) {
    FH_CK(lt.col_pipe(colp, a, st));
  } else {
    FH_CK(lt.col(kColGreen, col0, a, st));
  }
  if (g.d == 3) {
    ++launches;
    FH_CK(lt.col(kColInv, col1, m, st));
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t Pipeline<T>::passes(int pro, int epi, const RowArgs<T>& af, const RowArgs<T>& ai,
                                Scal* sc) {
  FH_CK(launch_row_fwd(pro, af));
  FH_CK(launch_green(kColGreen, sc, nullptr));
  FH_CK(launch_row_inv(epi, ai));
  return cudaSuccess;
}

template <typename T>
cudaError_t Pipeline<T>::apply(const T* in, T* out, bool transpose) {
  RowArgs<T> a = row_args();
  for (int l = 0; l < kMaxLoads; ++l) {
    a.in[l] = in;
    a.out[l] = out;
  }
  a.scal = nullptr;
  if (nloads != 1) return cudaErrorInvalidValue;
  return passes(transpose ? kProPlain : kProApply, transpose ? kEpiApplyT : kEpiApply, a, a, nullptr);
}

template <typename T>
int Pipeline<T>::chunk_size(int method) const {
  int K = g.nodes >= 1000000 ? 8 : (g.nodes >= 100000 ? 16 : 32);
  if (method == kFixed) K *= 4;
  return K;
}

template <typename T>
cudaError_t Pipeline<T>::enqueue_iter(int method, int j) {
  RowArgs<T> a = row_args();
  a.scal = scal;
  if (method == kCG) {
    // With deferred x steps the direction alternates between p (even j) and
    // p2 (odd j): the direction pass reads the previous p from the other
    // buffer, and the odd iteration's update settles both x steps.
    const bool odd = defer_x_ && (j & 1);
    T* const* pcur = odd ? p2 : p;
    T* const* pprev = odd ? p : p2;
    RowArgs<T> f = a, i = a;
    for (int l = 0; l < nloads; ++l) {
      f.in[l] = r[l];
      f.out[l] = pcur[l];
      f.aux[l] = defer_x_ ? pprev[l] : nullptr;
      i.in[l] = pcur[l];
      i.out[l] = ap[l];
    }
    FH_CK(passes(kProDir, kEpiDir, f, i, scal));
    ++launches;
    k_scal_alpha<<<item_blocks(items), kRedThreads, 0, st>>>(scal, part, row.grid, ncell, nloads, 0);
    FH_CK(cudaGetLastError());
    VecArgs<T> v;
    std::memset(&v, 0, sizeof(v));
    v.b.len = vlen;
    v.b.nloads = nloads;
    v.b.ncell = ncell;
    v.b.d = g.d;
    v.b.nodes = g.nodes;
    v.b.cell_nodes = g.cell_nodes;
    for (int l = 0; l < nloads; ++l) {
      v.x[l] = x[l];
      v.r[l] = r[l];
      v.p[l] = pcur[l];
      v.p2[l] = pprev[l];
      v.ap[l] = ap[l];
    }
    v.scal = scal;
    v.part = part;
    v.want_pp = hist_eta_r != nullptr && items == 1;
    v.xmode = !defer_x_ ? 1 : (odd ? 2 : 0);
    ++launches;
    FH_CK(lt.cg_update(vec, v, st));
    ++launches;
    k_scal_beta<<<item_blocks(items), kRedThreads, 0, st>>>(scal, part, vec.grid, ncell, nloads, 0,
                                                            !defer_x_ ? -1 : (odd ? 1 : 0));
    FH_CK(cudaGetLastError());
    return hist_eta_e != nullptr && items == 1 ? enqueue_eta_record() : cudaSuccess;
  }
  if (method == kBiCG) {
    // A^T p* with p* = r* + beta p*
    RowArgs<T> ft = a, it = a, f = a, i = a;
    for (int l = 0; l < nloads; ++l) {
      ft.in[l] = rs[l];
      ft.out[l] = ps[l];
      it.in[l] = ps[l];
      it.out[l] = atps[l];
      f.in[l] = r[l];
      f.out[l] = p[l];
      i.in[l] = p[l];
      i.out[l] = ap[l];
      i.aux[l] = ps[l];
    }
    FH_CK(passes(kProDirPlain, kEpiApplyT, ft, it, scal));
    FH_CK(passes(kProDir, kEpiDirShadow, f, i, scal));
    ++launches;
    k_scal_alpha<<<item_blocks(items), kRedThreads, 0, st>>>(scal, part, row.grid, ncell, nloads, 1);
    FH_CK(cudaGetLastError());
    VecArgs<T> v;
    std::memset(&v, 0, sizeof(v));
    v.b.len = vlen;
    v.b.nloads = nloads;
    v.b.ncell = ncell;
    v.b.d = g.d;
    v.b.nodes = g.nodes;
    v.b.cell_nodes = g.cell_nodes;
    for (int l = 0; l < nloads; ++l) {
      v.x[l] = x[l];
      v.r[l] = r[l];
      v.p[l] = p[l];
      v.ap[l] = ap[l];
      v.rs[l] = rs[l];
      v.atps[l] = atps[l];
    }
    v.scal = scal;
    v.part = part;
    ++launches;
    FH_CK(lt.bicg_update(vec, v, st));
    ++launches;
    k_scal_beta<<<item_blocks(items), kRedThreads, 0, st>>>(scal, part, vec.grid, ncell, nloads, 1, -1);
    FH_CK(cudaGetLastError());
    return hist_eta_e != nullptr && items == 1 ? enqueue_eta_record() : cudaSuccess;
  }
  // fixed point: e <- rhs - B e
  RowArgs<T> f = a, i = a;
  for (int l = 0; l < nloads; ++l) {
    f.in[l] = x[l];
    i.in[l] = x[l];
    i.out[l] = x[l];
    i.rhs[l] = rhs_active_ ? rhs[l] : nullptr;
  }
  FH_CK(passes(kProApply, kEpiFixed, f, i, scal));
  ++launches;
  k_scal_fixed<<<item_blocks(items), kRedThreads, 0, st>>>(scal, part, row.grid, ncell, nloads);
  FH_CK(cudaGetLastError());
  return hist_eta_e != nullptr && items == 1 ? enqueue_eta_record() : cudaSuccess;
}

template <typename T>
cudaError_t Pipeline<T>::enqueue_eta_record() {
  // j = L x (the passes of eta_e with the L table), then the equilibrium sums
  RowArgs<T> a = row_args();
  a.tab = ltab;
  for (int l = 0; l < kMaxLoads; ++l) a.in[l] = x[0];
  FH_CK(launch_row_fwd(kProApply, a));
  FH_CK(launch_green(kColEta, nullptr, part));
  ++launches;
  k_eta_record<<<1, kRedThreads, 0, st>>>(part, col0.grid, scal);
  return cudaGetLastError();
}

template <typename T>
int Pipeline<T>::norm2(T* const* v, double* out, std::string& err) {
  const Mat3 I = {{1, 0, 0, 0, 1, 0, 0, 0, 1}};
  for (int l = 0; l < nloads; ++l) {
    ++launches;
    FH_CKS(lt.matnorm2(vec, v[l], g.nodes, ncell, g.cell_nodes, I, part + (long long)l * vec.grid, st));
  }
  ++launches;
  k_reduce_items<<<item_blocks(items), kRedThreads, 0, st>>>(part, vec.grid, ncell, nloads, d_red);
  FH_CKS(cudaGetLastError());
  FH_CKS(cudaMemcpyAsync(h_red, d_red, items * sizeof(double), cudaMemcpyDeviceToHost, st));
  FH_CKS(cudaStreamSynchronize(st));
  for (int i = 0; i < items; ++i) out[i] = h_red[i];
  return 0;
}

template <typename T>
int Pipeline<T>::matnorm2(const T* e, const double* Mx, double* out, std::string& err) {
  Mat3 m;
  for (int i = 0; i < 9; ++i) m.v[i] = Mx[i];
  ++launches;
  FH_CKS(lt.matnorm2(vec, e, g.nodes, ncell, g.cell_nodes, m, part, st));
  ++launches;
  k_reduce_items<<<item_blocks(ncell), kRedThreads, 0, st>>>(part, vec.grid, ncell, 1, d_red);
  FH_CKS(cudaGetLastError());
  FH_CKS(cudaMemcpyAsync(h_red, d_red, ncell * sizeof(double), cudaMemcpyDeviceToHost, st));
  FH_CKS(cudaStreamSynchronize(st));
  for (int i = 0; i < ncell; ++i) out[i] = h_red[i];
  return 0;
}

template <typename T>
int Pipeline<T>::residual(const T* const* xin, T* const* rout, bool rhs_field,
                          const double (*E)[kMaxD], double* out, std::string& err, bool df) {
  const int nscal = std::max(items, kMaxLoads);
  for (int it = 0; it < items; ++it) {
    const int l = it % nloads;
    Scal& s = h_scal[nscal + it];
    std::memset(&s, 0, sizeof(Scal));
    s.done = kRunning;
    s.b2 = 1.0;
    for (int c = 0; c < kMaxD; ++c) s.E[c] = c < g.d ? E[l][c] : 0.0;
  }
  FH_CKS(cudaMemcpyAsync(scal_aux, h_scal + nscal, items * sizeof(Scal), cudaMemcpyHostToDevice, st));
  RowArgs<T> a = row_args();
  a.scal = scal_aux;
  for (int l = 0; l < nloads; ++l) {
    a.in[l] = xin[l];
    a.out[l] = rout[l];
    a.rhs[l] = rhs_field ? rhs[l] : nullptr;
  }
  df_green = df && lt.col_df != nullptr && tw0_df != nullptr && tw_last_df != nullptr && !prow.ext &&
             !pcol0.ext;  // the double-float kernels run the standard radix set only
  if (df_green) a.twdf = tw_last_df;
  const cudaError_t pe = passes(kProApply, kEpiResid, a, a, scal_aux);
  df_green = false;
  FH_CKS(pe);
  ++launches;
  k_reduce_items<<<item_blocks(items), kRedThreads, 0, st>>>(part, row.grid, ncell, nloads, d_red);
  FH_CKS(cudaGetLastError());
  FH_CKS(cudaMemcpyAsync(h_red, d_red, items * sizeof(double), cudaMemcpyDeviceToHost, st));
  FH_CKS(cudaStreamSynchronize(st));
  for (int i = 0; i < items; ++i) out[i] = h_red[i];
  return 0;
}

template <typename T>
int Pipeline<T>::project_complement(T* const* r, T* const* out, std::string& err) {
  const int nscal = std::max(items, kMaxLoads);
  for (int it = 0; it < items; ++it) {
    Scal& s = h_scal[nscal + it];
    std::memset(&s, 0, sizeof(Scal));
    s.done = kRunning;
    s.b2 = 1.0;
  }
  FH_CKS(cudaMemcpyAsync(scal_aux, h_scal + nscal, items * sizeof(Scal), cudaMemcpyHostToDevice, st));
  RowArgs<T> a = row_args();
  a.tab = qtab;
  a.scal = scal_aux;
  for (int l = 0; l < nloads; ++l) {
    a.in[l] = r[l];
    a.out[l] = out[l];
    a.rhs[l] = r[l];
  }
  // y = Q r;  out = r - y  (the fixed-point epilogue with right-hand side r)
  FH_CKS(passes(kProApply, kEpiFixed, a, a, scal_aux));
  return 0;
}

template <typename T>
int Pipeline<T>::current_mean(const T* e, double* col, std::string& err) {
  ++launches;
  FH_CKS(lt.current_sum(vec, e, phase, ltab64, g.nodes, ncell, g.cell_nodes, g.tab_stride, part, st));
  ++launches;
  k_reduce_items<<<item_blocks(ncell * g.d), kRedThreads, 0, st>>>(part, vec.grid, ncell, g.d, d_red);
  FH_CKS(cudaGetLastError());
  FH_CKS(cudaMemcpyAsync(h_red, d_red, ncell * g.d * sizeof(double), cudaMemcpyDeviceToHost, st));
  FH_CKS(cudaStreamSynchronize(st));
  for (int c = 0; c < ncell * g.d; ++c) col[c] = h_red[c] / (double)g.cell_nodes;
  return 0;
}

template <typename T>
int Pipeline<T>::eta_e(const T* e, double* eta, std::string& err) {
  if (nloads != 1 || ncell != 1) {
    err = "eta_e needs a single-load, single-cell pipeline";
    return 1;
  }
  RowArgs<T> a = row_args();
  a.tab = ltab;  // j = L e
  for (int l = 0; l < kMaxLoads; ++l) a.in[l] = e;
  FH_CKS(launch_row_fwd(kProApply, a));
  FH_CKS(launch_green(kColEta, nullptr, part));
  ++launches;
  k_reduce_items<<<item_blocks(2), kRedThreads, 0, st>>>(part, col0.grid, 1, 2, d_red);
  FH_CKS(cudaGetLastError());
  FH_CKS(cudaMemcpyAsync(h_red, d_red, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  FH_CKS(cudaStreamSynchronize(st));
  *eta = h_red[1] > 0.0 ? std::sqrt(h_red[0] / h_red[1]) : 0.0;
  return 0;
}

template <typename T>
int Pipeline<T>::solve(int method, const double (*E)[kMaxD], bool rhs_field, int x0,
                       const T* const* x_init, double tol, int max_iter, SolveResult* res,
                       std::string& err, const double* tol_item, int stall_window) {
  int rc = solve_begin(method, E, rhs_field, x0, x_init, tol, max_iter, err, tol_item, stall_window);
  if (rc) return rc;
  // every iteration runs on the device: one graph launch whose while node
  // repeats chunks of iterations until the items stop or the guard runs out
  Pipeline<T>* self = this;
  rc = run_loops<T>(&self, 1, st, loops, err);
  if (rc) return rc;
  if (!solve_done()) {
    err = "iteration guard exceeded without a device status";
    return 6;  // FH_ERR_NOT_CONVERGED: the round guard, not an expired device wait
  }
  solve_results(res);
  return 0;
}

template <typename T>
cudaError_t Pipeline<T>::enqueue_x_flush() {
  VecArgs<T> v;
  std::memset(&v, 0, sizeof(v));
  v.b.len = vlen;
  v.b.nloads = nloads;
  v.b.ncell = ncell;
  v.b.d = g.d;
  v.b.nodes = g.nodes;
  v.b.cell_nodes = g.cell_nodes;
  for (int l = 0; l < nloads; ++l) {
    v.x[l] = x[l];
    v.p[l] = p[l];
  }
  v.scal = scal;
  ++launches;
  return lt.cg_flush(vec, v, st);
}

template <typename T>
cudaError_t Pipeline<T>::capture_loop_body(cudaGraph_t body, cudaGraphConditionalHandle h, int method, int K,
                                           long long* kernels) {
  const long long before = launches;
  FH_CK(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < K && e == cudaSuccess; ++k) e = enqueue_iter(method, k);
  if (e == cudaSuccess) {
    ++launches;
    k_loop_cond<<<1, 128, 0, st>>>(h, scal, items, d_loop);
    e = cudaGetLastError();
  }
  cudaGraph_t out = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(st, &out);
  *kernels = launches - before;
  launches = before;
  return e != cudaSuccess ? e : e2;
}

// FH_HOST_LOOP set (and not "0"): run_loops drives the iterations from the
// host instead (run_loops_host).
static bool host_loop_mode() {
  static const bool on = [] {
    const char* v = std::getenv("FH_HOST_LOOP");
    return v != nullptr && v[0] != '\0' && !(v[0] == '0' && v[1] == '\0');
  }();
  return on;
}

// The same iterations as ordinary stream launches, K at a time per pipeline
// on its own stream, with the host reading the scalars after every chunk and
// stopping at the same conditions as the graph's while node (all items
// stopped, or the round guard).  For profilers, which cannot profile the
// kernel nodes of a graph that holds conditional nodes; the kernels and their
// arguments are those of the graph.
template <typename T>
static int run_loops_host(Pipeline<T>* const* ps, int np, std::string& err) {
  std::vector<long long> rounds(np, 0);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < np && e == cudaSuccess; ++i) {
    Pipeline<T>& P = *ps[i];
    e = cudaMemcpyAsync(P.h_scal, P.scal, P.items * sizeof(Scal), cudaMemcpyDeviceToHost, P.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P.st);
  }
  while (e == cudaSuccess) {
    bool any = false;
    for (int i = 0; i < np && e == cudaSuccess; ++i) {
      Pipeline<T>& P = *ps[i];
      if (P.solve_done() || rounds[i] >= P.run_guard_max_) continue;
      for (int k = 0; k < P.run_K_ && e == cudaSuccess; ++k) e = P.enqueue_iter(P.run_method_, k);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.h_scal, P.scal, P.items * sizeof(Scal), cudaMemcpyDeviceToHost, P.st);
      ++rounds[i];
      any = true;
    }
    if (!any) break;
    for (int i = 0; i < np && e == cudaSuccess; ++i) e = cudaStreamSynchronize(ps[i]->st);
  }
  for (int i = 0; i < np && e == cudaSuccess; ++i) {
    Pipeline<T>& P = *ps[i];
    if (P.defer_x_) e = P.enqueue_x_flush();
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.h_err, P.dev_err, sizeof(int), cudaMemcpyDeviceToHost, P.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P.st);
  }
  if (e != cudaSuccess) {
    err = std::string("host-driven iteration loop: ") + cudaGetErrorString(e);
    return 5;
  }
  for (int i = 0; i < np; ++i) {
    if (ps[i]->device_error()) {
      err = "a bounded device wait expired";
      return 8;
    }
  }
  return 0;
}

template <typename T>
int run_loops(Pipeline<T>* const* ps, int np, cudaStream_t launch, LoopCache& cache, std::string& err) {
  if (host_loop_mode()) return run_loops_host(ps, np, err);
  std::string key;
  for (int i = 0; i < np; ++i) {
    const Pipeline<T>& P = *ps[i];
    key += std::to_string(P.uid) + ":" + std::to_string(P.run_method_) + ":" +
           std::to_string(P.run_K_) + ":" + (P.rhs_active_ ? "r" : "c") +
           (P.hist_eta_e || P.hist_eta_r ? "h" : "-") + ";";
  }
  auto it = cache.exec.find(key);
  if (it == cache.exec.end()) {
    cudaGraph_t g = nullptr;
    FH_CKS(cudaGraphCreate(&g, 0));
    std::vector<long long> kern(2 * np, 0);  // per pipeline: kernels per loop round, then after the loop
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < np && e == cudaSuccess; ++i) {
      cudaGraphConditionalHandle h;
      e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
      if (e != cudaSuccess) break;
      cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node;
      e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
      if (e != cudaSuccess) break;
      e = ps[i]->capture_loop_body(cp.conditional.phGraph_out[0], h, ps[i]->run_method_, ps[i]->run_K_, &kern[i]);
      if (e == cudaSuccess && ps[i]->defer_x_) {
        // after the loop: the x step owed by items that stopped on an even iteration
        Pipeline<T>& P = *ps[i];
        e = cudaStreamBeginCaptureToGraph(P.st, g, &node, nullptr, 1, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        const long long before = P.launches;
        e = P.enqueue_x_flush();
        P.launches = before;
        cudaGraph_t out = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(P.st, &out);
        if (e == cudaSuccess) e = e2;
        kern[np + i] = 1;
      }
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      err = std::string("device-side iteration loop: ") + cudaGetErrorString(e);
      return 5;
    }
    it = cache.exec.emplace(key, exec).first;
    cache.kernels[key] = kern;
  }
  // round guard per pipeline, then start after every pipeline's preparation
  std::vector<cudaEvent_t> evs;
  auto cleanup = [&]() {
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
  };
  for (int i = 0; i < np; ++i) {
    Pipeline<T>& P = *ps[i];
    P.h_loop[0] = 0;
    P.h_loop[1] = (int)std::min<long long>(P.run_guard_max_, 1 << 30);
    FH_CKS(cudaMemcpyAsync(P.d_loop, P.h_loop, 2 * sizeof(int), cudaMemcpyHostToDevice, P.st));
    if (P.st != launch) {
      cudaEvent_t ev;
      FH_CKS(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      evs.push_back(ev);
      FH_CKS(cudaEventRecord(ev, P.st));
      FH_CKS(cudaStreamWaitEvent(launch, ev, 0));
    }
  }
  cudaError_t e = cudaGraphLaunch(it->second, launch);
  for (int i = 0; i < np && e == cudaSuccess; ++i) {
    Pipeline<T>& P = *ps[i];
    e = cudaMemcpyAsync(P.h_scal, P.scal, P.items * sizeof(Scal), cudaMemcpyDeviceToHost, launch);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.h_err, P.dev_err, sizeof(int), cudaMemcpyDeviceToHost, launch);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.h_loop, P.d_loop, 2 * sizeof(int), cudaMemcpyDeviceToHost, launch);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(launch);
  cleanup();
  if (e != cudaSuccess) {
    err = std::string("device-side iteration loop: ") + cudaGetErrorString(e);
    return 5;
  }
  const std::vector<long long>& kern = cache.kernels[key];
  for (int i = 0; i < np; ++i) {
    ps[i]->launches += (long long)ps[i]->h_loop[0] * kern[i] + kern[np + i];
    if (ps[i]->device_error()) {
      err = "a bounded device wait expired";
      return 8;
    }
  }
  return 0;
}

template <typename T>
bool Pipeline<T>::solve_done() const {
  for (int it = 0; it < items; ++it)
    if (h_scal[it].done == kRunning) return false;
  return true;
}

template <typename T>
void Pipeline<T>::solve_results(SolveResult* res) const {
  for (int it = 0; it < items; ++it) {
    res[it].status = h_scal[it].done;
    res[it].iters = h_scal[it].iter;
    res[it].rel = h_scal[it].rel;
    res[it].alpha = h_scal[it].alpha;
  }
}

template <typename T>
int Pipeline<T>::solve_begin(int method, const double (*E)[kMaxD], bool rhs_field, int x0,
                             const T* const* x_init, double tol, int max_iter, std::string& err,
                             const double* tol_item, int stall_window) {
  int rc;
  if (method == kBiCG && rs[0] == nullptr) {
    for (int l = 0; l < nloads; ++l) {
      if ((rc = dev_alloc(allocs, &rs[l], vlen, err))) return rc;
      if ((rc = dev_alloc(allocs, &ps[l], vlen, err))) return rc;
      if ((rc = dev_alloc(allocs, &atps[l], vlen, err))) return rc;
    }
  }
  defer_x_ = method == kCG && !(hist_eta_e != nullptr && items == 1);
  if (defer_x_ && p2[0] == nullptr) {
    for (int l = 0; l < nloads; ++l)
      if ((rc = dev_alloc(allocs, &p2[l], vlen, err))) return rc;
  }
  rhs_active_ = rhs_field;
  // a wait that expired in an earlier solve has been reported; start clean
  FH_CKS(cudaMemsetAsync(dev_err, 0, sizeof(int), st));
  *h_err = 0;
  std::vector<double> b2(items);
  if (rhs_field) {
    if ((rc = norm2(rhs, b2.data(), err))) return rc;
  } else {
    for (int it = 0; it < items; ++it) {
      const int l = it % nloads;
      double e2 = 0.0;
      for (int c = 0; c < g.d; ++c) e2 += E[l][c] * E[l][c];
      b2[it] = e2 * (double)g.cell_nodes;
    }
  }
  for (int it = 0; it < items; ++it) {
    const int l = it % nloads;
    Scal& s = h_scal[it];
    std::memset(&s, 0, sizeof(Scal));
    s.b2 = b2[it] > 0.0 ? b2[it] : 1.0;
    const double tl = tol_item ? tol_item[it] : tol;
    s.tol2 = tl * tl;
    s.max_iter = max_iter;
    s.done = kRunning;
    s.stall_window = stall_window;
    s.hist = items == 1 ? hist : nullptr;
    s.hist_cap = items == 1 ? hist_cap : 0;
    s.hist_eta_r = items == 1 ? hist_eta_r : nullptr;
    s.hist_eta_e = items == 1 ? hist_eta_e : nullptr;
    s.l0iso = l0iso;
    for (int c = 0; c < kMaxD; ++c) s.E[c] = (!rhs_field && c < g.d) ? E[l][c] : 0.0;
  }
  FH_CKS(cudaMemcpyAsync(scal, h_scal, items * sizeof(Scal), cudaMemcpyHostToDevice, st));
  const size_t vbytes = (size_t)vlen * sizeof(T);
  for (int l = 0; l < nloads; ++l) {
    switch (x0) {
      case kX0Const:
        ++launches;
        k_fill_const<T><<<vec.grid, vec.block, 0, st>>>(x[l], g.nodes, g.d, E[l][0], E[l][1],
                                                        g.d > 2 ? E[l][2] : 0.0);
        FH_CKS(cudaGetLastError());
        break;
      case kX0Field:
        FH_CKS(cudaMemcpyAsync(x[l], x_init[l], vbytes, cudaMemcpyDeviceToDevice, st));
        break;
      case kX0Zero:
        FH_CKS(cudaMemsetAsync(x[l], 0, vbytes, st));
        break;
      case kX0Keep:
        break;
      default:
        FH_CKS(cudaMemcpyAsync(x[l], rhs[l], vbytes, cudaMemcpyDeviceToDevice, st));
        break;
    }
  }
  if (method != kFixed) {
    if (x0 == kX0Zero) {
      const Mat3 I = {{1, 0, 0, 0, 1, 0, 0, 0, 1}};
      for (int l = 0; l < nloads; ++l) {
        FH_CKS(cudaMemcpyAsync(r[l], rhs[l], vbytes, cudaMemcpyDeviceToDevice, st));
        ++launches;
        FH_CKS(lt.matnorm2(vec, r[l], g.nodes, ncell, g.cell_nodes, I, part + (long long)l * vec.grid, st));
      }
      ++launches;
      k_scal_start<<<item_blocks(items), kRedThreads, 0, st>>>(scal, part, vec.grid, ncell, nloads);
    } else {
      RowArgs<T> a = row_args();
      a.scal = scal;
      for (int l = 0; l < nloads; ++l) {
        a.in[l] = x[l];
        a.out[l] = r[l];
        a.rhs[l] = rhs_field ? rhs[l] : nullptr;
      }
      FH_CKS(passes(kProApply, kEpiResid, a, a, scal));
      ++launches;
      k_scal_start<<<item_blocks(items), kRedThreads, 0, st>>>(scal, part, row.grid, ncell, nloads);
    }
    FH_CKS(cudaGetLastError());
    for (int l = 0; l < nloads; ++l) {
      FH_CKS(cudaMemsetAsync(p[l], 0, vbytes, st));
      if (defer_x_) FH_CKS(cudaMemsetAsync(p2[l], 0, vbytes, st));  // the first iteration's previous p
      if (method == kBiCG) {
        FH_CKS(cudaMemcpyAsync(rs[l], r[l], vbytes, cudaMemcpyDeviceToDevice, st));
        FH_CKS(cudaMemsetAsync(ps[l], 0, vbytes, st));
      }
    }
  }
  if (hist_eta_e != nullptr && items == 1) FH_CKS(enqueue_eta_record());  // iterate 0
  run_method_ = method;
  run_K_ = chunk_size(method);
  run_guard_max_ = (long long)max_iter / run_K_ + 4;
  return 0;
}

template <typename T>
int Pipeline<T>::autotune(const Problem& pb, int nloads_, cudaStream_t stream, Tuning& best,
                          double& best_ms, std::string& err, int max_candidates) {
  const bool f64 = sizeof(T) == 8;
  const int d = pb.d;
  const int nlast = pb.N[d - 1];
  // candidate plans: every thread count that reaches the minimum stage count
  // of its axis, plus the next stage count (fewer registers per thread)
  auto plan_tpls = [&](int n, int maxthr) {
    std::vector<int> out;
    int best_st = 1 << 30;
    std::vector<std::pair<int, int>> all;  // (stages, tpl)
    for (int t = 1; t <= maxthr; ++t) {
      bool ext;
      factorable(n, ext);
      std::vector<int> r = plan_radices(n, t, ext ? reg_budget_x(f64) : reg_budget(f64));
      if (r.empty()) continue;
      const int st = (int)r.size();
      if (st < best_st) best_st = st;
      if (all.empty() || all.back().first != st) all.emplace_back(st, t);
    }
    for (auto& sv : all)
      if (sv.first <= best_st + 1) out.push_back(sv.second);
    return out;
  };
  std::vector<int> tpls = plan_tpls(nlast, kRowMaxThreads);
  std::vector<int> tpc0s = plan_tpls(pb.N[0], kColMaxThreads);
  std::vector<int> tpc1s = d == 3 ? plan_tpls(pb.N[1], kColMaxThreads) : std::vector<int>{0};
  std::vector<Tuning> cands;
  const std::vector<int> pipes = d == 2 ? std::vector<int>{0, 1} : std::vector<int>{0};
  for (int C : {16, 8, 4, 2, 1})
    for (int lpc : {1, 2, 3, 4, 6, 8})
      for (int tp : tpls)
        for (int t0 : tpc0s)
          for (int t1 : tpc1s)
            for (int pp : pipes) {
              Tuning c;
              c.C = C;
              c.lpc = lpc;
              c.tpl = tp;
              c.tpc0 = t0;
              c.tpc1 = t1;
              c.pipe = pp;
              cands.push_back(c);
            }
  best_ms = 1e30;
  int tried = 0;
  std::string e2;
  for (const Tuning& c : cands) {
    if (tried >= max_candidates) break;
    Pipeline<T> trial;
    if (trial.init(pb, nloads_, true, stream, e2, &c) != 0) {
      trial.release();
      continue;
    }
    if (!(trial.tuning == c)) {  // the constraints changed a requested value
      trial.release();
      continue;
    }
    ++tried;
    double total = 0.0, t;
    bool ok = true;
    for (int what = 0; what < 4 && ok; ++what) {
      if (trial.profile(what, 10, &t, e2) != 0) ok = false;
      total += t;
    }
    trial.release();
    if (ok && total < best_ms) {
      best_ms = total;
      best = c;
    }
  }
  if (best_ms >= 1e30) {
    err = "autotune: no candidate could be timed";
    return 9;
  }
  return 0;
}

template <typename T>
int Pipeline<T>::profile(int what, int reps, double* ms, std::string& err) {
  if (x[0] == nullptr) {
    err = "profiling needs a context with Krylov buffers";
    return 1;
  }
  for (int it = 0; it < items; ++it) {
    Scal& s = h_scal[it];
    std::memset(&s, 0, sizeof(Scal));
    s.done = kRunning;
    s.alpha = 1e-3;
    s.beta = 0.5;
    s.b2 = 1.0;
    s.max_iter = 1 << 30;
  }
  FH_CKS(cudaMemcpyAsync(scal, h_scal, items * sizeof(Scal), cudaMemcpyHostToDevice, st));
  const size_t vbytes = (size_t)vlen * sizeof(T);
  for (int l = 0; l < nloads; ++l) {
    FH_CKS(cudaMemsetAsync(x[l], 0, vbytes, st));
    FH_CKS(cudaMemsetAsync(r[l], 0, vbytes, st));
    FH_CKS(cudaMemsetAsync(p[l], 0, vbytes, st));
    FH_CKS(cudaMemsetAsync(ap[l], 0, vbytes, st));
  }
  RowArgs<T> a = row_args();
  a.scal = scal;
  RowArgs<T> f = a, i = a, app = a;
  for (int l = 0; l < nloads; ++l) {
    f.in[l] = r[l];
    f.out[l] = p[l];
    i.in[l] = p[l];
    i.out[l] = ap[l];
    app.in[l] = x[l];
    app.out[l] = ap[l];
  }
  app.scal = nullptr;
  VecArgs<T> v;
  std::memset(&v, 0, sizeof(v));
  v.b.len = vlen;
  v.b.nloads = nloads;
  v.b.ncell = ncell;
  v.b.d = g.d;
  v.b.nodes = g.nodes;
  v.b.cell_nodes = g.cell_nodes;
  for (int l = 0; l < nloads; ++l) {
    v.x[l] = x[l];
    v.r[l] = r[l];
    v.p[l] = p[l];
    v.ap[l] = ap[l];
  }
  v.scal = scal;
  v.part = part;
  v.xmode = 1;
  auto one = [&]() -> cudaError_t {
    switch (what) {
      case 0: return launch_row_fwd(kProDir, f);
      case 1: return launch_green(kColGreen, scal, nullptr);
      case 2: return launch_row_inv(kEpiDir, i);
      case 3: ++launches; return lt.cg_update(vec, v, st);
      case 5: return passes(kProApply, kEpiApply, app, app, nullptr);
      default: return cudaErrorInvalidValue;
    }
  };
  for (int w = 0; w < 3; ++w) FH_CKS(one());
  cudaEvent_t e0, e1;
  FH_CKS(cudaEventCreate(&e0));
  FH_CKS(cudaEventCreate(&e1));
  FH_CKS(cudaEventRecord(e0, st));
  for (int k = 0; k < reps; ++k) FH_CKS(one());
  FH_CKS(cudaEventRecord(e1, st));
  FH_CKS(cudaEventSynchronize(e1));
  float t = 0.f;
  FH_CKS(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = (double)t / reps;
  return 0;
}

}  // namespace fh

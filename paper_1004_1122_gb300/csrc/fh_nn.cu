// fh_nn.cu -- the learned warm start's 3-D convolutional network: forward,
// backward and Adam, all in hand-written kernels.
//
// Activations are float32 [channels][N0][N1][N2]; weights are kept as float32
// masters for Adam and rounded to bfloat16 (round to nearest even) for every
// product; products accumulate in float32.  Architecture (levels N, N/3,
// N/9, N/27; channels c0..c3; layers 0..10 in parameter order):
//   a0 = leaky(conv0(x))            a1 = leaky(conv1(pool(a0)))
//   a2 = leaky(conv2(pool(a1)))     a3 = leaky(conv3(pool(a2)))
//   v2 = up(leaky(conv4(a3))) + a2  u2 = leaky(conv5(v2))
//   v1 = up(leaky(conv6(u2))) + a1  u1 = leaky(conv7(v1))
//   v0 = up(leaky(conv8(u1))) + a0  u0 = leaky(conv9(v0))
//   y  = conv10(u0)
// conv = 3x3x3 with periodic padding (the unit cell is periodic), pool = mean
// over 3x3x3 blocks, up = nearest-neighbour upsampling by 3.
// The forward convolutions run on the tensor cores (fh_conv_tc.cuh: tcgen05
// implicit GEMM, bfloat16 weights, float32 activations split into two
// bfloat16 halves); the backward ones (data and weight gradients) on the
// CUDA cores in float32.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/fh_nn.h"
#include "fh_conv_tc.cuh"

namespace {

constexpr float kSlope = 0.1f;
constexpr int kThreads = 256;

struct Dims {
  int n0, n1, n2;
  __host__ __device__ long long v() const { return (long long)n0 * n1 * n2; }
};

// dW[o][c][t] = sum_z gy[o](z) x[c](z + t);  db[o] = sum_z gy[o](z).
// CTA (o, c, s) sums the 27 taps and the bias over voxel slice s of S; the
// partials go to part[((s * O + o) * C + c) * 28 + t] and k_wgrad_reduce adds
// the slices in a fixed order (no atomics, deterministic).
__global__ void __launch_bounds__(kThreads) k_conv_wgrad(const float* __restrict__ x, int C,
                                                         const float* __restrict__ gy, int O, int S,
                                                         float* __restrict__ part, Dims dm) {
  const int pair = blockIdx.x % (O * C), sl = blockIdx.x / (O * C);
  const int o = pair / C, c = pair - (pair / C) * C;
  const long long V = dm.v();
  const long long v0 = V * sl / S, v1 = V * (sl + 1) / S;
  const float* xc = x + (long long)c * V;
  const float* go = gy + (long long)o * V;
  const int plane = dm.n1 * dm.n2;
  float acc[27];
#pragma unroll
  for (int t = 0; t < 27; ++t) acc[t] = 0.0f;
  float accb = 0.0f;
  for (long long vox = v0 + threadIdx.x; vox < v1; vox += blockDim.x) {
    const int z = (int)(vox / plane);
    const int rem = (int)(vox - (long long)z * plane);
    const int yy = rem / dm.n2, xx = rem - yy * dm.n2;
    const float g = __ldg(go + vox);
    accb += g;
    int xs[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      int x2 = xx + k - 1;
      x2 += x2 < 0 ? dm.n2 : (x2 >= dm.n2 ? -dm.n2 : 0);
      xs[k] = x2;
    }
#pragma unroll
    for (int dz = 0; dz < 3; ++dz) {
      int zz = z + dz - 1;
      zz += zz < 0 ? dm.n0 : (zz >= dm.n0 ? -dm.n0 : 0);
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        int y2 = yy + dy - 1;
        y2 += y2 < 0 ? dm.n1 : (y2 >= dm.n1 ? -dm.n1 : 0);
        const float* row = xc + (long long)(zz * dm.n1 + y2) * dm.n2;
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[dz * 9 + dy * 3 + k] = fmaf(g, __ldg(row + xs[k]), acc[dz * 9 + dy * 3 + k]);
      }
    }
  }
  __shared__ float red[kThreads / 32][28];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < 28; ++t) {
    float v = t < 27 ? acc[t] : accb;
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) v += __shfl_down_sync(0xffffffffu, v, k);
    if (lane == 0) red[warp][t] = v;
  }
  __syncthreads();
  if (threadIdx.x < 28) {
    float v = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
    part[((long long)(sl * O + o) * C + c) * 28 + threadIdx.x] = v;
  }
}

// gW[o][c][t] = sum_s part[s][o][c][t];  gb[o] = sum_s part[s][o][0][27]
__global__ void k_wgrad_reduce(const float* __restrict__ part, int O, int C, int S, float* __restrict__ gW,
                               float* __restrict__ gb) {
  const long long n = (long long)O * C * 28;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i % 28);
    const long long oc = i / 28;
    float v = 0.0f;
    for (int sl = 0; sl < S; ++sl) v += part[((long long)sl * O * C + oc) * 28 + t];
    if (t < 27) {
      gW[oc * 27 + t] = v;
    } else if (oc % C == 0) {
      gb[oc / C] = v;
    }
  }
}

__global__ void k_leaky(const float* __restrict__ z, float* __restrict__ a, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = z[i];
    a[i] = v > 0.0f ? v : kSlope * v;
  }
}

// g <- g * leaky'(z)
__global__ void k_leaky_bwd(const float* __restrict__ z, float* __restrict__ g, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!(z[i] > 0.0f)) g[i] *= kSlope;
}

// coarse[c][Z][Y][X] = mean of the 3x3x3 fine block (fine dims = 3 * coarse dims)
__global__ void k_pool(const float* __restrict__ fine, float* __restrict__ coarse, int C, Dims cd) {
  const long long Vc = cd.v();
  const long long n = Vc * C;
  const int f1 = 3 * cd.n1, f2 = 3 * cd.n2;
  const long long Vf = 27 * Vc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / Vc);
    const long long v = i - (long long)c * Vc;
    const int Z = (int)(v / ((long long)cd.n1 * cd.n2));
    const int rem = (int)(v - (long long)Z * cd.n1 * cd.n2);
    const int Y = rem / cd.n2, X = rem - Y * cd.n2;
    const float* fc = fine + (long long)c * Vf;
    float s = 0.0f;
    for (int a = 0; a < 3; ++a)
      for (int bb = 0; bb < 3; ++bb)
        for (int e = 0; e < 3; ++e) s += fc[((long long)(3 * Z + a) * f1 + 3 * Y + bb) * f2 + 3 * X + e];
    coarse[i] = s * (1.0f / 27.0f);
  }
}

// fine[c][z][y][x] = scale * coarse[c][z/3][y/3][x/3] (+ add[c][z][y][x] if add, + fine if accumulate)
__global__ void k_up(const float* __restrict__ coarse, float* __restrict__ fine, const float* __restrict__ add,
                     int C, Dims fd, float scale, int accumulate) {
  const long long Vf = fd.v();
  const long long n = Vf * C;
  const int c1 = fd.n1 / 3, c2 = fd.n2 / 3;
  const long long Vc = Vf / 27;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / Vf);
    const long long v = i - (long long)c * Vf;
    const int z = (int)(v / ((long long)fd.n1 * fd.n2));
    const int rem = (int)(v - (long long)z * fd.n1 * fd.n2);
    const int y = rem / fd.n2, x = rem - y * fd.n2;
    float s = scale * coarse[(long long)c * Vc + ((long long)(z / 3) * c1 + y / 3) * c2 + x / 3];
    if (add) s += add[i];
    if (accumulate) s += fine[i];
    fine[i] = s;
  }
}

// coarse[c][Z][Y][X] = sum of the fine block (adjoint of nearest upsampling)
__global__ void k_up_bwd(const float* __restrict__ fine, float* __restrict__ coarse, int C, Dims cd) {
  const long long Vc = cd.v();
  const long long n = Vc * C;
  const int f1 = 3 * cd.n1, f2 = 3 * cd.n2;
  const long long Vf = 27 * Vc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / Vc);
    const long long v = i - (long long)c * Vc;
    const int Z = (int)(v / ((long long)cd.n1 * cd.n2));
    const int rem = (int)(v - (long long)Z * cd.n1 * cd.n2);
    const int Y = rem / cd.n2, X = rem - Y * cd.n2;
    const float* fc = fine + (long long)c * Vf;
    float s = 0.0f;
    for (int a = 0; a < 3; ++a)
      for (int bb = 0; bb < 3; ++bb)
        for (int e = 0; e < 3; ++e) s += fc[((long long)(3 * Z + a) * f1 + 3 * Y + bb) * f2 + 3 * X + e];
    coarse[i] = s;
  }
}

// g = 2 (y - t) / n; per-block partial sums of (y - t)^2 in float64
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ g,
                      long long n, double* part) {
  double acc = 0.0;
  const float sc = 2.0f / (float)n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float dlt = y[i] - t[i];
    g[i] = sc * dlt;
    acc += (double)dlt * (double)dlt;
  }
  __shared__ double red[kThreads];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Tensor-core weight layout of one layer: wt[o][t * Cp + c] = bf16(w[o][c][t]),
// zero for o >= O or c >= C (NT rows, 27 * Cp columns).
__global__ void k_to_bf16_tc(const float* __restrict__ w, int O, int C, int Cp, int NT,
                             __nv_bfloat16* __restrict__ wt) {
  const long long n = (long long)NT * 27 * Cp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int o = (int)(i / (27 * Cp));
    const int k = (int)(i - (long long)o * 27 * Cp);
    const int t = k / Cp, c = k - t * Cp;
    const float v = (o < O && c < C) ? w[((long long)o * C + c) * 27 + t] : 0.0f;
    wt[i] = __float2bfloat16_rn(v);
  }
}

// Transposed layout for the data gradient gx[c] = sum_o sum_t w[o][c][t] gy[o](. - t):
// wt[c][t * Op + o] = bf16(w[o][c][26 - t]), zero for c >= C or o >= O (NT rows
// = C padded to 16, 27 * Op columns).
__global__ void k_to_bf16_tc_t(const float* __restrict__ w, int O, int C, int Op, int NT,
                               __nv_bfloat16* __restrict__ wt) {
  const long long n = (long long)NT * 27 * Op;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / (27 * Op));
    const int k = (int)(i - (long long)c * 27 * Op);
    const int t = k / Op, o = k - t * Op;
    const float v = (o < O && c < C) ? w[((long long)o * C + c) * 27 + (26 - t)] : 0.0f;
    wt[i] = __float2bfloat16_rn(v);
  }
}

// x[0] = tab0[phase], x[1] = tab1[phase]  (input features from the phase image)
__global__ void k_features(const uint8_t* __restrict__ phase, const float* __restrict__ t0,
                           const float* __restrict__ t1, float* __restrict__ x, long long V) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    const int p = phase[i];
    x[i] = t0[p];
    x[V + i] = t1[p];
  }
}

// target[b * d + a] = e^(b)_a - delta_ab (+ base[b * d + a] if base)
// (fields: d loads, each [d][V] float64)
__global__ void k_targets(const double* __restrict__ f0, const double* __restrict__ f1,
                          const double* __restrict__ f2, int d, const float* __restrict__ base,
                          float* __restrict__ t, long long V) {
  const double* f[3] = {f0, f1, f2};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x)
    for (int b = 0; b < d; ++b)
      for (int a = 0; a < d; ++a) {
        const long long k = (long long)(b * d + a) * V + i;
        float v = (float)(f[b][(long long)a * V + i] - (a == b ? 1.0 : 0.0));
        if (base) v += base[k];
        t[k] = v;
      }
}

// g[a] = sum_b E_b (pred[b * d + a] - base[b * d + a])  (fluctuation of load E
// predicted by the network; base = the residual base the network was trained
// against, or null)
__global__ void k_combine(const float* __restrict__ pred, const float* __restrict__ base, int d, double E0,
                          double E1, double E2, double* __restrict__ g, long long V) {
  const double E[3] = {E0, E1, E2};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x)
    for (int a = 0; a < d; ++a) {
      double s = 0.0;
      for (int b = 0; b < d; ++b) {
        const long long k = (long long)(b * d + a) * V + i;
        s += E[b] * ((double)pred[k] - (base ? (double)base[k] : 0.0));
      }
      g[(long long)a * V + i] = s;
    }
}

// x = E + g  (g already projected)
__global__ void k_add_E(double* __restrict__ x, int d, double E0, double E1, double E2, long long V) {
  const double E[3] = {E0, E1, E2};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)d * V; i += (long long)gridDim.x * blockDim.x)
    x[i] += E[i / V];
}

// e[a][i] = delta_ab: the constant unit load b
template <typename T>
__global__ void k_unit_load(T* __restrict__ e, int b, int d, long long V) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)d * V; i += (long long)gridDim.x * blockDim.x)
    e[i] = (i / V == b) ? T(1) : T(0);
}

// x[a][i] = y[a][i] - delta_ab  (B e_b from y = (I + B) e_b), as float32
template <typename T>
__global__ void k_response(const T* __restrict__ y, int b, int d, float* __restrict__ x, long long V) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)d * V; i += (long long)gridDim.x * blockDim.x)
    x[i] = (float)(y[i] - ((i / V == b) ? T(1) : T(0)));
}

int grid1(long long n) {
  const long long g = (n + kThreads - 1) / kThreads;
  return (int)(g < 4096 ? (g < 1 ? 1 : g) : 4096);
}

}  // namespace

constexpr int kLayers = 11;

struct fh_nn {
  Dims lv[4];
  int cin = 0, cout = 0;
  int ch[4] = {16, 32, 48, 64};
  int lo[kLayers], li[kLayers], ll[kLayers];  // layer out / in channels, level
  long long woff[kLayers], boff[kLayers];      // offsets in the flat parameter vector
  long long nparam = 0;
  cudaStream_t st = nullptr;
  float *P = nullptr, *G = nullptr, *Mo = nullptr, *Ve = nullptr;
  __nv_bfloat16* Wtc = nullptr;                 // tensor-core weight layout, all layers
  __nv_bfloat16* WtcT = nullptr;                // transposed (data-gradient) layout
  long long wtc_off[kLayers], wtct_off[kLayers];// offsets (multiples of 8 elements)
  int cpad[kLayers], ntile[kLayers];             // forward: in channels padded to 8, N tile
  int opad[kLayers], ntile_t[kLayers];           // data gradient: out channels padded to 8, N tile
  int* dev_err = nullptr;                        // bounded waits that expired
  float* wpart = nullptr;                        // weight-gradient partials per voxel slice
  // forward: pre-activations z[k] (k < 10), encoder a[l], pooled pl[l],
  // decoder sums v[l] and activations u[l], output y; tmp = leaky(up conv)
  float *x = nullptr, *z[kLayers - 1] = {}, *a[4] = {}, *pl[3] = {}, *v[3] = {}, *u[3] = {}, *y = nullptr;
  float* tmp = nullptr;
  // backward
  float *gy = nullptr, *gu[3] = {}, *gv[3] = {}, *ga3 = nullptr, *gp[3] = {}, *gt = nullptr;
  double* part = nullptr;
  double* h_part = nullptr;
  int npart = 0;
  std::vector<void*> allocs;
  long long launches = 0;
};

namespace {

template <typename T>
int nn_alloc(fh_nn* n, T** p, long long count) {
  void* q = nullptr;
  if (cudaMalloc(&q, (size_t)count * sizeof(T) + 16) != cudaSuccess) return FH_ERR_OOM;
  n->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return 0;
}

cudaError_t conv(fh_nn* n, int layer, const float* in, float* out, bool trans) {
  const int O = trans ? n->li[layer] : n->lo[layer];
  const int C = trans ? n->lo[layer] : n->li[layer];
  const Dims d = n->lv[n->ll[layer]];
  ++n->launches;
  {
    // forward: y = conv(x; W) + b;  data gradient: gx = conv(gy; W^T, taps
    // reversed), the same implicit GEMM with the transposed weight layout
    fh::tc::ConvTcArgs ta;
    ta.x = in;
    ta.C = C;
    ta.Cp = trans ? n->opad[layer] : n->cpad[layer];
    ta.y = out;
    ta.O = O;
    ta.NT = trans ? n->ntile_t[layer] : n->ntile[layer];
    ta.w = trans ? n->WtcT + n->wtct_off[layer] : n->Wtc + n->wtc_off[layer];
    ta.b = trans ? nullptr : n->P + n->boff[layer];
    ta.n0 = d.n0;
    ta.n1 = d.n1;
    ta.n2 = d.n2;
    ta.err = n->dev_err;
    ta.wait_ns = fh::tma::wait_limit_ns();
    const unsigned g = (unsigned)((d.v() + fh::tc::kM - 1) / fh::tc::kM);
    fh::tc::k_conv_tc<<<g, fh::tc::kThreads, fh::tc::kSmemBytes, n->st>>>(ta);
  }
  return cudaGetLastError();
}

// voxel slices per (o, c) pair: enough CTAs for ~4 per SM, at least 2048 voxels a slice
int wgrad_slices(int O, int C, long long V) {
  long long s = (608 + (long long)O * C - 1) / ((long long)O * C);
  s = std::min<long long>(s, std::max<long long>(1, V / 2048));
  return (int)std::max<long long>(1, std::min<long long>(s, 64));
}

cudaError_t wgrad(fh_nn* n, int layer, const float* in, const float* gy) {
  const Dims d = n->lv[n->ll[layer]];
  const int O = n->lo[layer], C = n->li[layer];
  const int S = wgrad_slices(O, C, d.v());
  n->launches += 2;
  k_conv_wgrad<<<O * C * S, kThreads, 0, n->st>>>(in, C, gy, O, S, n->wpart, d);
  k_wgrad_reduce<<<grid1((long long)O * C * 28), kThreads, 0, n->st>>>(n->wpart, O, C, S, n->G + n->woff[layer],
                                                                       n->G + n->boff[layer]);
  return cudaGetLastError();
}

void leaky(fh_nn* n, const float* z, float* a, long long cnt) {
  ++n->launches;
  k_leaky<<<grid1(cnt), kThreads, 0, n->st>>>(z, a, cnt);
}
void leaky_bwd(fh_nn* n, const float* z, float* g, long long cnt) {
  ++n->launches;
  k_leaky_bwd<<<grid1(cnt), kThreads, 0, n->st>>>(z, g, cnt);
}
void pool(fh_nn* n, const float* f, float* c, int C, Dims cd) {
  ++n->launches;
  k_pool<<<grid1(cd.v() * C), kThreads, 0, n->st>>>(f, c, C, cd);
}
void up(fh_nn* n, const float* c, float* f, const float* add, int C, Dims fd, float scale, int accum) {
  ++n->launches;
  k_up<<<grid1(fd.v() * C), kThreads, 0, n->st>>>(c, f, add, C, fd, scale, accum);
}
void up_bwd(fh_nn* n, const float* f, float* c, int C, Dims cd) {
  ++n->launches;
  k_up_bwd<<<grid1(cd.v() * C), kThreads, 0, n->st>>>(f, c, C, cd);
}

// decoder level l: (up convolution, post convolution) layer indices
constexpr int kUp[3] = {8, 6, 4};
constexpr int kPost[3] = {9, 7, 5};

cudaError_t forward(fh_nn* n) {
  cudaError_t e;
  for (int k = 0; k < kLayers; ++k) {
    n->launches += 2;
    k_to_bf16_tc<<<grid1((long long)n->ntile[k] * 27 * n->cpad[k]), kThreads, 0, n->st>>>(
        n->P + n->woff[k], n->lo[k], n->li[k], n->cpad[k], n->ntile[k], n->Wtc + n->wtc_off[k]);
    k_to_bf16_tc_t<<<grid1((long long)n->ntile_t[k] * 27 * n->opad[k]), kThreads, 0, n->st>>>(
        n->P + n->woff[k], n->lo[k], n->li[k], n->opad[k], n->ntile_t[k], n->WtcT + n->wtct_off[k]);
  }
  if ((e = conv(n, 0, n->x, n->z[0], false))) return e;
  leaky(n, n->z[0], n->a[0], n->lv[0].v() * n->ch[0]);
  for (int l = 1; l < 4; ++l) {
    pool(n, n->a[l - 1], n->pl[l - 1], n->ch[l - 1], n->lv[l]);
    if ((e = conv(n, l, n->pl[l - 1], n->z[l], false))) return e;
    leaky(n, n->z[l], n->a[l], n->lv[l].v() * n->ch[l]);
  }
  const float* in = n->a[3];
  for (int l = 2; l >= 0; --l) {
    const int ku = kUp[l], kp = kPost[l];
    // v_l = up(leaky(conv_ku(in))) + a_l ; u_l = leaky(conv_kp(v_l))
    if ((e = conv(n, ku, in, n->z[ku], false))) return e;
    leaky(n, n->z[ku], n->tmp, n->lv[l + 1].v() * n->ch[l]);
    up(n, n->tmp, n->v[l], n->a[l], n->ch[l], n->lv[l], 1.0f, 0);
    if ((e = conv(n, kp, n->v[l], n->z[kp], false))) return e;
    leaky(n, n->z[kp], n->u[l], n->lv[l].v() * n->ch[l]);
    in = n->u[l];
  }
  if ((e = conv(n, 10, n->u[0], n->y, false))) return e;
  return cudaGetLastError();
}

// gradients of sum(gy * y) (gy already in n->gy)
cudaError_t backward(fh_nn* n) {
  cudaError_t e;
  if ((e = wgrad(n, 10, n->u[0], n->gy))) return e;
  if ((e = conv(n, 10, n->gy, n->gu[0], true))) return e;        // g_u0
  for (int l = 0; l < 3; ++l) {
    const int ku = kUp[l], kp = kPost[l];
    const long long Vl = n->lv[l].v(), Vc = n->lv[l + 1].v();
    leaky_bwd(n, n->z[kp], n->gu[l], Vl * n->ch[l]);               // -> g_z(post)
    if ((e = wgrad(n, kp, n->v[l], n->gu[l]))) return e;
    if ((e = conv(n, kp, n->gu[l], n->gv[l], true))) return e;     // g_v_l (= skip part of g_a_l)
    up_bwd(n, n->gv[l], n->gt, n->ch[l], n->lv[l + 1]);             // c_l at level l+1
    leaky_bwd(n, n->z[ku], n->gt, Vc * n->ch[l]);                   // -> g_z(up)
    const float* up_in = l < 2 ? n->u[l + 1] : n->a[3];
    if ((e = wgrad(n, ku, up_in, n->gt))) return e;
    float* g_in = l < 2 ? n->gu[l + 1] : n->ga3;
    if ((e = conv(n, ku, n->gt, g_in, true))) return e;            // g_u_{l+1} (or g_a3)
  }
  // encoder: g_a3 in ga3; g_a_l = g_v_l + poolT(g_p_l)
  float* g_a = n->ga3;
  for (int l = 3; l >= 1; --l) {
    leaky_bwd(n, n->z[l], g_a, n->lv[l].v() * n->ch[l]);          // -> g_z_l
    if ((e = wgrad(n, l, n->pl[l - 1], g_a))) return e;
    if ((e = conv(n, l, g_a, n->gp[l - 1], true))) return e;      // g_p_{l-1}
    up(n, n->gp[l - 1], n->gv[l - 1], nullptr, n->ch[l - 1], n->lv[l - 1], 1.0f / 27.0f, 1);
    g_a = n->gv[l - 1];
  }
  leaky_bwd(n, n->z[0], g_a, n->lv[0].v() * n->ch[0]);            // -> g_z0
  if ((e = wgrad(n, 0, n->x, g_a))) return e;
  return cudaGetLastError();
}

// true when a kernel's bounded wait expired (synchronises the stream)
bool device_error(fh_nn* n) {
  int h = 0;
  if (cudaMemcpyAsync(&h, n->dev_err, sizeof(int), cudaMemcpyDeviceToHost, n->st) != cudaSuccess ||
      cudaStreamSynchronize(n->st) != cudaSuccess)
    return true;
  return h != 0;
}

int loss_grad(fh_nn* n, const float* target, double* loss) {
  const long long cnt = n->lv[0].v() * n->cout;
  const int g = std::min(n->npart, grid1(cnt));
  ++n->launches;
  k_mse<<<g, kThreads, 0, n->st>>>(n->y, target, n->gy, cnt, n->part);
  if (cudaMemcpyAsync(n->h_part, n->part, g * sizeof(double), cudaMemcpyDeviceToHost, n->st) != cudaSuccess)
    return FH_ERR_CUDA;
  if (cudaStreamSynchronize(n->st) != cudaSuccess) return FH_ERR_CUDA;
  double s = 0.0;
  for (int i = 0; i < g; ++i) s += n->h_part[i];
  if (loss) *loss = s / (double)cnt;
  return device_error(n) ? FH_ERR_TIMEOUT : 0;
}

}  // namespace

extern "C" {

void fh_nn_destroy(fh_nn* n) {
  if (!n) return;
  if (n->st) cudaStreamSynchronize(n->st);
  for (void* p : n->allocs) cudaFree(p);
  if (n->h_part) cudaFreeHost(n->h_part);
  delete n;
}

fh_status fh_nn_create(fh_nn** out, const int* N, int cin, int cout, const int* channels, void* stream) {
  if (!out || !N || cin < 1 || cout < 1) return FH_ERR_ARG;
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (N[a] < 27 || N[a] % 27) return FH_ERR_ARG;
  fh_nn* n = new (std::nothrow) fh_nn();
  if (!n) return FH_ERR_OOM;
  n->cin = cin;
  n->cout = cout;
  if (channels)
    for (int k = 0; k < 4; ++k) {
      if (channels[k] < 1) {
        delete n;
        return FH_ERR_ARG;
      }
      n->ch[k] = channels[k];
    }
  for (int l = 0; l < 4; ++l) {
    int f = 1;
    for (int k = 0; k < l; ++k) f *= 3;
    n->lv[l] = Dims{N[0] / f, N[1] / f, N[2] / f};
  }
  const int c0 = n->ch[0], c1 = n->ch[1], c2 = n->ch[2], c3 = n->ch[3];
  const int io[kLayers][3] = {{cin, c0, 0}, {c0, c1, 1}, {c1, c2, 2}, {c2, c3, 3},
                              {c3, c2, 3},  {c2, c2, 2}, {c2, c1, 2}, {c1, c1, 1},
                              {c1, c0, 1},  {c0, c0, 0}, {c0, cout, 0}};
  long long off = 0;
  for (int k = 0; k < kLayers; ++k) {
    n->li[k] = io[k][0];
    n->lo[k] = io[k][1];
    n->ll[k] = io[k][2];
    n->woff[k] = off;
    off += (long long)n->lo[k] * n->li[k] * 27;
    n->boff[k] = off;
    off += n->lo[k];
  }
  n->nparam = off;
  long long toff = 0, ttoff = 0;
  for (int k = 0; k < kLayers; ++k) {
    n->cpad[k] = (n->li[k] + 7) / 8 * 8;
    n->ntile[k] = (n->lo[k] + 15) / 16 * 16;
    n->opad[k] = (n->lo[k] + 7) / 8 * 8;
    n->ntile_t[k] = (n->li[k] + 15) / 16 * 16;
    n->wtc_off[k] = toff;
    toff += (long long)n->ntile[k] * 27 * n->cpad[k];
    n->wtct_off[k] = ttoff;
    ttoff += (long long)n->ntile_t[k] * 27 * n->opad[k];
    if (n->ntile[k] > fh::tc::kNmax || n->ntile_t[k] > fh::tc::kNmax) {
      delete n;
      return FH_ERR_ARG;  // more than 64 channels on one side of a layer
    }
  }
  n->st = (cudaStream_t)stream;
  int rc = 0;
  const long long V[4] = {n->lv[0].v(), n->lv[1].v(), n->lv[2].v(), n->lv[3].v()};
  long long coarse_max = 0;  // largest c_l * |level l+1|
  for (int l = 0; l < 3; ++l) coarse_max = std::max(coarse_max, (long long)n->ch[l] * V[l + 1]);
  rc |= nn_alloc(n, &n->P, off);
  rc |= nn_alloc(n, &n->G, off);
  rc |= nn_alloc(n, &n->Mo, off);
  rc |= nn_alloc(n, &n->Ve, off);
  rc |= nn_alloc(n, &n->Wtc, toff);
  rc |= nn_alloc(n, &n->WtcT, ttoff);
  {
    long long wp = 0;
    for (int k = 0; k < kLayers; ++k)
      wp = std::max(wp, (long long)wgrad_slices(n->lo[k], n->li[k], V[n->ll[k]]) * n->lo[k] * n->li[k] * 28);
    rc |= nn_alloc(n, &n->wpart, wp);
  }
  rc |= nn_alloc(n, &n->dev_err, 1);
  rc |= nn_alloc(n, &n->x, V[0] * cin);
  for (int k = 0; k < kLayers - 1; ++k) rc |= nn_alloc(n, &n->z[k], V[n->ll[k]] * (long long)n->lo[k]);
  for (int k = 0; k < 4; ++k) rc |= nn_alloc(n, &n->a[k], V[k] * n->ch[k]);
  for (int k = 0; k < 3; ++k) rc |= nn_alloc(n, &n->pl[k], V[k + 1] * n->ch[k]);
  for (int k = 0; k < 3; ++k) rc |= nn_alloc(n, &n->v[k], V[k] * n->ch[k]);
  for (int k = 0; k < 3; ++k) rc |= nn_alloc(n, &n->u[k], V[k] * n->ch[k]);
  rc |= nn_alloc(n, &n->y, V[0] * cout);
  rc |= nn_alloc(n, &n->tmp, coarse_max);
  rc |= nn_alloc(n, &n->gy, V[0] * cout);
  for (int k = 0; k < 3; ++k) rc |= nn_alloc(n, &n->gu[k], V[k] * n->ch[k]);
  for (int k = 0; k < 3; ++k) rc |= nn_alloc(n, &n->gv[k], V[k] * n->ch[k]);
  rc |= nn_alloc(n, &n->ga3, V[3] * n->ch[3]);
  for (int k = 0; k < 3; ++k) rc |= nn_alloc(n, &n->gp[k], V[k + 1] * n->ch[k]);
  rc |= nn_alloc(n, &n->gt, coarse_max);
  n->npart = 4096;
  rc |= nn_alloc(n, &n->part, n->npart);
  if (!rc && cudaMallocHost(&n->h_part, n->npart * sizeof(double)) != cudaSuccess) rc = FH_ERR_OOM;
  if (!rc && (cudaMemsetAsync(n->dev_err, 0, sizeof(int), n->st) != cudaSuccess ||
              cudaMemsetAsync(n->Mo, 0, off * sizeof(float), n->st) != cudaSuccess ||
              cudaMemsetAsync(n->Ve, 0, off * sizeof(float), n->st) != cudaSuccess ||
              cudaMemsetAsync(n->P, 0, off * sizeof(float), n->st) != cudaSuccess))
    rc = FH_ERR_CUDA;
  if (rc) {
    fh_nn_destroy(n);
    return FH_ERR_OOM;
  }
  *out = n;
  return FH_OK;
}

long long fh_nn_param_count(const fh_nn* n) { return n ? n->nparam : 0; }

long long fh_nn_launches(const fh_nn* n) { return n ? n->launches : 0; }

fh_status fh_nn_set_params(fh_nn* n, const float* host, long long count) {
  if (!n || !host || count != n->nparam) return FH_ERR_ARG;
  if (cudaMemcpyAsync(n->P, host, count * sizeof(float), cudaMemcpyHostToDevice, n->st) != cudaSuccess ||
      cudaMemsetAsync(n->Mo, 0, count * sizeof(float), n->st) != cudaSuccess ||
      cudaMemsetAsync(n->Ve, 0, count * sizeof(float), n->st) != cudaSuccess ||
      cudaStreamSynchronize(n->st) != cudaSuccess)
    return FH_ERR_CUDA;
  return FH_OK;
}

fh_status fh_nn_get_params(fh_nn* n, float* host, long long count) {
  if (!n || !host || count != n->nparam) return FH_ERR_ARG;
  if (cudaMemcpyAsync(host, n->P, count * sizeof(float), cudaMemcpyDeviceToHost, n->st) != cudaSuccess ||
      cudaStreamSynchronize(n->st) != cudaSuccess)
    return FH_ERR_CUDA;
  return FH_OK;
}

fh_status fh_nn_forward(fh_nn* n, const float* x, float* y) {
  if (!n || !x || !y) return FH_ERR_ARG;
  const long long Vx = n->lv[0].v() * n->cin, Vy = n->lv[0].v() * n->cout;
  if (cudaMemcpyAsync(n->x, x, Vx * sizeof(float), cudaMemcpyDeviceToDevice, n->st) != cudaSuccess)
    return FH_ERR_CUDA;
  if (forward(n) != cudaSuccess) return FH_ERR_CUDA;
  if (cudaMemcpyAsync(y, n->y, Vy * sizeof(float), cudaMemcpyDeviceToDevice, n->st) != cudaSuccess)
    return FH_ERR_CUDA;
  return FH_OK;
}

fh_status fh_nn_gradients(fh_nn* n, const float* x, const float* target, double* loss, float* grad_host) {
  if (!n || !x || !target) return FH_ERR_ARG;
  const long long Vx = n->lv[0].v() * n->cin;
  if (cudaMemcpyAsync(n->x, x, Vx * sizeof(float), cudaMemcpyDeviceToDevice, n->st) != cudaSuccess)
    return FH_ERR_CUDA;
  if (forward(n) != cudaSuccess) return FH_ERR_CUDA;
  int rc = loss_grad(n, target, loss);
  if (rc) return (fh_status)rc;
  if (backward(n) != cudaSuccess) return FH_ERR_CUDA;
  if (grad_host) {
    if (cudaMemcpyAsync(grad_host, n->G, n->nparam * sizeof(float), cudaMemcpyDeviceToHost, n->st) != cudaSuccess ||
        cudaStreamSynchronize(n->st) != cudaSuccess)
      return FH_ERR_CUDA;
  }
  return FH_OK;
}

fh_status fh_nn_train_step(fh_nn* n, const float* x, const float* target, float lr, int step, double* loss) {
  if (!n || step < 1 || !(lr > 0.0f)) return FH_ERR_ARG;
  fh_status s = fh_nn_gradients(n, x, target, loss, nullptr);
  if (s != FH_OK) return s;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - (float)std::pow(0.9, step), c2 = 1.0f - (float)std::pow(0.999, step);
  ++n->launches;
  k_adam<<<grid1(n->nparam), kThreads, 0, n->st>>>(n->P, n->G, n->Mo, n->Ve, n->nparam, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError() == cudaSuccess ? FH_OK : FH_ERR_CUDA;
}

fh_status fh_nn_features(const uint8_t* phase, int nphase, const double* L, int d, long long nodes,
                         float* x, void* stream) {
  if (!phase || !L || !x || nphase < 1 || nphase > 256 || (d != 2 && d != 3)) return FH_ERR_ARG;
  // channel 0: log10(L_p / L_0) / 4 (isotropic phases, first diagonal entry), channel 1: indicator
  std::vector<float> h(512, 0.0f);
  const double l0 = L[0];
  if (!(l0 > 0.0)) return FH_ERR_NOT_SPD;
  for (int p = 0; p < nphase; ++p) {
    const double lp = L[(size_t)p * d * d];
    if (!(lp > 0.0)) return FH_ERR_NOT_SPD;
    h[p] = (float)(std::log10(lp / l0) / 4.0);
    h[256 + p] = p > 0 ? 1.0f : 0.0f;
  }
  float* dt = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMallocAsync((void**)&dt, 512 * sizeof(float), st) != cudaSuccess) return FH_ERR_OOM;
  cudaMemcpyAsync(dt, h.data(), 512 * sizeof(float), cudaMemcpyHostToDevice, st);
  k_features<<<grid1(nodes), kThreads, 0, st>>>(phase, dt, dt + 256, x, nodes);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(dt, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? FH_OK : FH_ERR_CUDA;
}

fh_status fh_nn_targets(const double* const* fields, int d, long long nodes, const float* base, float* target,
                        void* stream) {
  if (!fields || !target || (d != 2 && d != 3)) return FH_ERR_ARG;
  for (int b = 0; b < d; ++b)
    if (!fields[b]) return FH_ERR_ARG;
  k_targets<<<grid1(nodes), kThreads, 0, (cudaStream_t)stream>>>(fields[0], fields[1], d > 2 ? fields[2] : fields[0], d,
                                                                  base, target, nodes);
  return cudaGetLastError() == cudaSuccess ? FH_OK : FH_ERR_CUDA;
}

}  // extern "C"

namespace {

template <typename T>
fh_status response_features(fh_ctx* ctx, int dtype, int d, long long nodes, float* x) {
  const long long len = (long long)d * nodes;
  T* buf = nullptr;
  if (cudaMalloc((void**)&buf, 2 * len * sizeof(T)) != cudaSuccess) return FH_ERR_OOM;
  fh_status s = FH_OK;
  for (int b = 0; b < d && s == FH_OK; ++b) {
    k_unit_load<T><<<grid1(len), kThreads>>>(buf, b, d, len / d);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
      s = FH_ERR_CUDA;
      break;
    }
    s = fh_apply(ctx, buf, buf + len, 0, dtype);
    if (s != FH_OK) break;
    if (cudaDeviceSynchronize() != cudaSuccess) {
      s = FH_ERR_CUDA;
      break;
    }
    k_response<T><<<grid1(len), kThreads>>>(buf + len, b, d, x + (long long)b * len, len / d);
    if (cudaGetLastError() != cudaSuccess) s = FH_ERR_CUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess && s == FH_OK) s = FH_ERR_CUDA;
  cudaFree(buf);
  return s;
}

}  // namespace

extern "C" {

fh_status fh_nn_response_features(fh_ctx* ctx, int d, long long nodes, float* x) {
  if (!ctx || !x || (d != 2 && d != 3) || nodes < 1) return FH_ERR_ARG;
  // float32 products where the context has them (the features are float32),
  // else the float64 pipeline
  fh_status s = response_features<float>(ctx, FH_FP32, d, nodes, x);
  if (s == FH_ERR_ARG) s = response_features<double>(ctx, FH_FP64, d, nodes, x);
  return s;
}

fh_status fh_nn_warm_start(fh_ctx* ctx, const float* pred, const float* base, const double* E, int d,
                           long long nodes, double* x0, void* stream) {
  if (!ctx || !pred || !E || !x0 || (d != 2 && d != 3)) return FH_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  k_combine<<<grid1(nodes), kThreads, 0, st>>>(pred, base, d, E[0], E[1], d > 2 ? E[2] : 0.0, x0, nodes);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return FH_ERR_CUDA;
  fh_status s = fh_project_compatible(ctx, x0, x0);
  if (s != FH_OK) return s;
  if (cudaDeviceSynchronize() != cudaSuccess) return FH_ERR_CUDA;
  k_add_E<<<grid1((long long)d * nodes), kThreads, 0, st>>>(x0, d, E[0], E[1], d > 2 ? E[2] : 0.0, nodes);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return FH_ERR_CUDA;
  return FH_OK;
}

}  // extern "C"

// fh_conv_tc.cuh -- the forward 3x3x3 periodic convolution of the warm-start
// network as an implicit GEMM on the fifth-generation tensor cores.
//
//   Y[o][v] = b[o] + sum_k W[o][k] X_k[v],   k = (tap t, channel c)
//
// is D(M x N) = A(M x K) B(K x N) with M = voxels (tiles of 128), N = output
// channels (padded to a multiple of 16, <= 64) and K = 27 taps x channels.
// The weights are bfloat16 (the network's definition); the float32
// activations are split as x = hi + lo with hi = bf16(x), lo = bf16(x - hi),
// and both halves are multiplied into the same float32 accumulator, so the
// product keeps ~16 mantissa bits of x (the float32-activation definition to
// ~1e-5 relative) while both MMA operands are bfloat16.
//
// Per CTA (128 threads, one voxel row of A per thread): K is walked in chunks
// of kKC; each thread gathers its voxel's chunk (periodic neighbours, 8
// channels at one tap per 16-byte group), writes hi / lo / weights into
// shared memory in the no-swizzle K-major core-matrix layout, and one thread
// issues the tcgen05.mma instructions of the chunk and commits them to the
// chunk's mbarrier.  Two chunk buffers alternate, so gathering chunk i+1
// overlaps the MMAs of chunk i.  The accumulator lives in tensor memory and is
// read back with tcgen05.ld by the four warps (32 rows each).
//
// Shared-memory operand layout (no swizzle, K-major): an 8-row x 16-byte core
// matrix is 128 contiguous bytes; core matrices adjacent along K are kLBO =
// 128 bytes apart, 8-row groups kSBO = (kKC / 8) * 128 bytes apart.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "fh_tma.cuh"

namespace fh {
namespace tc {

constexpr int kM = 128;            // voxels per tile (MMA M)
constexpr int kKC = 32;            // K elements per chunk
constexpr int kKG = kKC / 8;       // 16-byte k-groups per chunk
constexpr int kLBO = 128;          // bytes between K-adjacent core matrices
constexpr int kSBO = kKG * 128;    // bytes between 8-row groups
constexpr int kThreads = 128;

// shared memory of one chunk buffer: A hi, A lo (kM rows) and B (kNmax rows)
constexpr int kNmax = 64;
constexpr int kABytes = kM * kKC * 2;
constexpr int kBBytes = kNmax * kKC * 2;
constexpr int kStageBytes = 2 * kABytes + kBBytes;
constexpr int kSmemBytes = 2 * kStageBytes + 64;  // two stages + barriers + TMEM slot

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);              // start address
  d |= (uint64_t)((kLBO >> 4) & 0x3FFF) << 16;         // leading (K) byte offset
  d |= (uint64_t)((kSBO >> 4) & 0x3FFF) << 32;         // stride (8-row group) byte offset
  d |= (uint64_t)1 << 46;                              // descriptor version
  return d;                                            // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D float32, A and B bfloat16, both
// K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t instr_desc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   tma::saddr(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 16 columns of float32 from tensor memory into r[0..15]
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(u[i]);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

struct ConvTcArgs {
  const float* x;            // [C][V] float32 activations
  int C, Cp;                 // channels, channels padded to a multiple of 8
  float* y;                  // [O][V]
  int O, NT;                 // output channels, N tile (multiple of 16, <= kNmax)
  const __nv_bfloat16* w;    // [NT][27 * Cp], k = t * Cp + c, zero padded
  const float* b;            // [O], or nullptr for no bias
  int n0, n1, n2;            // grid
  int* err;                  // device error word (bounded waits), or nullptr
  unsigned long long wait_ns;  // limit of the primary waits (0: tma::kWaitLimitNs)
};

// Byte offset of element (row, k) of a K-major no-swizzle operand chunk.
__device__ __forceinline__ uint32_t core_off(int row, int kg) {
  return (uint32_t)((row >> 3) * kSBO + kg * kLBO + (row & 7) * 16);
}

__global__ void __launch_bounds__(kThreads) k_conv_tc(ConvTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * kStageBytes);  // [0], [1]: chunk stages
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * kStageBytes + 32);
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long V = (long long)a.n0 * a.n1 * a.n2;
  const long long m0 = (long long)blockIdx.x * kM;
  const uint32_t ncols = a.NT <= 32 ? 32u : 64u;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tma::saddr(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::fence_barrier_init();
    s_fail = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  // this thread's voxel (row of A)
  const long long v = m0 + tid;
  const bool live = v < V;
  int z = 0, yy = 0, xx = 0;
  if (live) {
    z = (int)(v / ((long long)a.n1 * a.n2));
    const int rem = (int)(v - (long long)z * a.n1 * a.n2);
    yy = rem / a.n2;
    xx = rem - yy * a.n2;
  }
  const int cg_per_tap = a.Cp >> 3;             // 16-byte groups of channels per tap
  const int KG = 27 * cg_per_tap;               // k-groups in K
  const int nch = (KG + kKG - 1) / kKG;         // chunks
  const int Kp = 27 * a.Cp;
  const uint32_t idesc = instr_desc(a.NT);

  int ch = 0;
  for (; ch < nch; ++ch) {
    const int st = ch & 1;
    unsigned char* A_hi = smem + st * kStageBytes;
    unsigned char* A_lo = A_hi + kABytes;
    unsigned char* Bm = A_lo + kABytes;
    if (ch >= 2) {
      // the MMAs of chunk ch - 2 have finished reading this stage
      if (!tma::mbar_wait(&bar[st], ((ch - 2) >> 1) & 1, a.wait_ns)) s_fail = 1;
      __syncthreads();
      if (s_fail) break;
    }
    // A: this thread's voxel row, kKG k-groups of 8 channels at one tap
#pragma unroll
    for (int j = 0; j < kKG; ++j) {
      const int kg = ch * kKG + j;
      float val[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) val[i] = 0.0f;
      if (live && kg < KG) {
        const int t = kg / cg_per_tap;
        const int c0 = (kg - t * cg_per_tap) * 8;
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        int zz = z + dz, y2 = yy + dy, x2 = xx + dx;
        zz += zz < 0 ? a.n0 : (zz >= a.n0 ? -a.n0 : 0);
        y2 += y2 < 0 ? a.n1 : (y2 >= a.n1 ? -a.n1 : 0);
        x2 += x2 < 0 ? a.n2 : (x2 >= a.n2 ? -a.n2 : 0);
        const long long off = ((long long)zz * a.n1 + y2) * a.n2 + x2;
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (c0 + i < a.C) val[i] = __ldg(a.x + (long long)(c0 + i) * V + off);
      }
      uint32_t h[4], l[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(val[2 * i]);
        const __nv_bfloat16 h1 = __float2bfloat16_rn(val[2 * i + 1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(val[2 * i] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(val[2 * i + 1] - __bfloat162float(h1));
        h[i] = pack2(h0, h1);
        l[i] = pack2(l0, l1);
      }
      const uint32_t o = core_off(tid, j);
      *reinterpret_cast<uint4*>(A_hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(A_lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
    }
    // B: NT rows x kKG k-groups of the weights (16-byte loads, zero past K)
    for (int q = tid; q < a.NT * kKG; q += kThreads) {
      const int row = q / kKG, j = q - row * kKG;
      const int k0 = (ch * kKG + j) * 8;
      uint4 w = make_uint4(0u, 0u, 0u, 0u);
      if (k0 < Kp) w = __ldg(reinterpret_cast<const uint4*>(a.w + (long long)row * Kp + k0));
      *reinterpret_cast<uint4*>(Bm + core_off(row, j)) = w;
    }
    tma::fence_proxy_async();  // make these shared-memory writes visible to the tensor cores
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      const uint32_t sa_hi = tma::saddr(A_hi), sa_lo = tma::saddr(A_lo), sb = tma::saddr(Bm);
#pragma unroll
      for (int s = 0; s < kKC / 16; ++s) {
        const uint64_t bd = smem_desc(sb + s * 2 * kLBO);
        mma(tmem, smem_desc(sa_hi + s * 2 * kLBO), bd, idesc, (ch > 0 || s > 0) ? 1u : 0u);
        mma(tmem, smem_desc(sa_lo + s * 2 * kLBO), bd, idesc, 1u);
      }
      commit(&bar[st]);
    }
  }

  // wait for the last chunk's MMAs (a commit covers every earlier MMA)
  if (!s_fail && nch > 0) {
    const int lc = nch - 1;
    if (!tma::mbar_wait(&bar[lc & 1], (lc >> 1) & 1, a.wait_ns)) s_fail = 1;
  }
  __syncthreads();
  fence_after();
  if (!s_fail) {
    // epilogue: warp w holds rows 32 w .. 32 w + 31 (lanes of tensor memory)
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < a.NT; c0 += 16) {
      float r[16];
      tmem_ld16(lane_base + (uint32_t)c0, r);
      if (live) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int o = c0 + i;
          if (o < a.O) a.y[(long long)o * V + v] = r[i] + (a.b ? a.b[o] : 0.0f);
        }
      }
    }
  } else if (tid == 0) {
    // a wait gave up: chunks 0 .. ch-1 were committed; wait (bounded) for the
    // last commit of each stage before the accumulator is released, and report
    for (int s2 = 0; s2 < 2; ++s2) {
      const int last = (ch - 1) - (((ch - 1) & 1) != s2 ? 1 : 0);
      if (last >= 0) tma::mbar_wait(&bar[s2], (last >> 1) & 1);
    }
    if (a.err) atomicExch(a.err, 1);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

}  // namespace tc
}  // namespace fh

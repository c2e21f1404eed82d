// Kernels of the spectral neural operator used as a learned warm start
// (declared in include/rlbm_fno.h).
//
// The GEMM runs on the tensor cores with mma.sync m16n8k16 (BF16 inputs,
// FP32 accumulation): 64 x 64 block tiles, K slices of 32 staged in shared
// memory, four warps of 32 x 32.  Operand tiles are loaded element-wise so
// any transpose / stride / ragged size works; the FNO's GEMMs are small and
// far from compute-bound.
#include "rlbm.h"
#include "rlbm_fno.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rlbm {
namespace {

constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;
constexpr int kGemmThreads = 128;

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * __expf(-0.5f * x * x);
  return cdf + x * pdf;
}

__device__ __forceinline__ uint32_t pack2(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct GemmArgs {
  int transA, transB, M, N, K;
  float alpha, beta;
  const __nv_bfloat16* A;
  long long lda, strideA;
  const __nv_bfloat16* B;
  long long ldb, strideB;
  float* C;
  long long ldc, strideC;
  const float* bias;
  __nv_bfloat16* D;
  int epilogue;
};

__global__ void __launch_bounds__(kGemmThreads) k_gemm(GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const long long b = blockIdx.z;
  const __nv_bfloat16* A = g.A + b * g.strideA;
  const __nv_bfloat16* B = g.B + b * g.strideB;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);

  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

  for (int k0 = 0; k0 < g.K; k0 += BK) {
    // consecutive threads read consecutive addresses of the stored layout
    for (int i = tid; i < BM * BK; i += kGemmThreads) {
      int m, k;
      if (!g.transA) { m = i / BK; k = i % BK; } else { k = i / BM; m = i % BM; }
      const int gm = m0 + m, gk = k0 + k;
      __nv_bfloat16 v = zero;
      if (gm < g.M && gk < g.K) v = g.transA ? A[(long long)gk * g.lda + gm] : A[(long long)gm * g.lda + gk];
      As[m][k] = v;
    }
    for (int i = tid; i < BN * BK; i += kGemmThreads) {
      int n, k;
      if (!g.transB) { k = i / BN; n = i % BN; } else { n = i / BK; k = i % BK; }
      const int gn = n0 + n, gk = k0 + k;
      __nv_bfloat16 v = zero;
      if (gn < g.N && gk < g.K) v = g.transB ? B[(long long)gn * g.ldb + gk] : B[(long long)gk * g.ldb + gn];
      Bs[n][k] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      const int r = lane >> 2, c = kk + (lane & 3) * 2;
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int row = wm * 32 + mi * 16 + r;
        af[mi][0] = pack2(&As[row][c]);
        af[mi][1] = pack2(&As[row + 8][c]);
        af[mi][2] = pack2(&As[row][c + 8]);
        af[mi][3] = pack2(&As[row + 8][c + 8]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int col = wn * 32 + ni * 8 + r;
        bfr[ni][0] = pack2(&Bs[col][c]);
        bfr[ni][1] = pack2(&Bs[col][c + 8]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni]);
    }
    __syncthreads();
  }

  float* C = g.C ? g.C + b * g.strideC : nullptr;
  __nv_bfloat16* D = g.D ? g.D + b * g.strideC : nullptr;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = m0 + wm * 32 + mi * 16 + (lane >> 2) + (e >= 2 ? 8 : 0);
        const int col = n0 + wn * 32 + ni * 8 + (lane & 3) * 2 + (e & 1);
        if (row >= g.M || col >= g.N) continue;
        const long long o = (long long)row * g.ldc + col;
        float v = g.alpha * acc[mi][ni][e];
        if (g.epilogue == RLBM_EPI_ATOMIC) {
          atomicAdd(C + o, v);
          continue;
        }
        if (C && g.beta != 0.f) v += g.beta * C[o];
        if (g.bias) v += g.bias[col];
        if (C) C[o] = v;
        if (D) D[o] = __float2bfloat16_rn(g.epilogue == RLBM_EPI_GELU ? gelu(v) : v);
      }
}

// ---------------------------------------------------------------------------
// Fifth-generation tensor-core GEMM (tcgen05 / TMEM), one CTA per 128 x 64
// output tile.  Four warps stage K slabs of 64 into shared memory in the
// canonical no-swizzle K-major layout (8 x 16-byte core matrices: the two
// 8-element halves of a K16 step are LBO = 128 B apart, consecutive 8-row
// groups SBO = 1024 B apart); one thread issues four tcgen05.mma (M = 128,
// N = 64, K = 16, BF16 x BF16 -> FP32 in TMEM) per slab and commits them to
// an mbarrier; the accumulator is read back with tcgen05.ld (warp w owns TMEM
// lanes 32 w .. 32 w + 31 = output rows).  Every wait is bounded: on timeout
// the CTA raises the error flag, skips its tile, frees its TMEM and returns.
// ---------------------------------------------------------------------------
constexpr int TC_M = 128, TC_N = 64, TC_K = 64;
constexpr long long kTcSpinCycles = 4000000000LL;   // ~2 s at 2 GHz

__device__ unsigned g_tc_error = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Matrix descriptor: start >> 4 [0,14), LBO >> 4 [16,30), SBO >> 4 [32,46),
// version 1 [46,48), base offset 0, LBO mode 0, layout 0 (no swizzle) [61,64).
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ULL << 46);
}

// Instruction descriptor, kind::f16: D F32 (bit 4), A BF16 (bit 7), B BF16
// (bit 10), both K-major, N >> 3 at [17,23), M >> 4 at [24,29).
__host__ __device__ constexpr uint32_t tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
         ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
    if (clock64() - t0 > kTcSpinCycles) return false;
  }
}

__global__ void __launch_bounds__(128) k_gemm_tc(GemmArgs g) {
  __shared__ __align__(1024) uint8_t sA[TC_M * TC_K * 2];
  __shared__ __align__(1024) uint8_t sB[TC_N * TC_K * 2];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_tile;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;
  const long long b = blockIdx.z;
  const __nv_bfloat16* A = g.A + b * g.strideA;
  const __nv_bfloat16* B = g.B + b * g.strideB;
  const uint32_t bar = smem_u32(&mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 :: "r"(smem_u32(&tmem_slot)), "r"(TC_N) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_tile = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(sA);
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(sB);
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  const int nslab = (g.K + TC_K - 1) / TC_K;
  int issued = 0;   // slabs whose MMAs were committed (same value in every thread)
  for (int sl = 0; sl < nslab; ++sl) {
    if (sl > 0) {
      // the MMAs of the previous slab must have read shared memory
      if (!mbar_wait(bar, (sl - 1) & 1)) abort_tile = 1;
      __syncthreads();
      if (abort_tile) break;
    }
    const int k0 = sl * TC_K;
    // element (row, k) of a slab -> core matrix (row / 8, k / 8), 8 core matrices per row group
    for (int i = tid; i < TC_M * TC_K; i += 128) {
      int m, k;
      if (!g.transA) { m = i / TC_K; k = i % TC_K; } else { k = i / TC_M; m = i % TC_M; }
      const int gm = m0 + m, gk = k0 + k;
      __nv_bfloat16 v = zero;
      if (gm < g.M && gk < g.K) v = g.transA ? A[(long long)gk * g.lda + gm] : A[(long long)gm * g.lda + gk];
      As[((m >> 3) * 8 + (k >> 3)) * 64 + (m & 7) * 8 + (k & 7)] = v;
    }
    for (int i = tid; i < TC_N * TC_K; i += 128) {
      int n, k;
      if (!g.transB) { k = i / TC_N; n = i % TC_N; } else { n = i / TC_K; k = i % TC_K; }
      const int gn = n0 + n, gk = k0 + k;
      __nv_bfloat16 v = zero;
      if (gn < g.N && gk < g.K) v = g.transB ? B[(long long)gn * g.ldb + gk] : B[(long long)gk * g.ldb + gn];
      Bs[((n >> 3) * 8 + (k >> 3)) * 64 + (n & 7) * 8 + (k & 7)] = v;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < TC_K / 16; ++kk) {
        const uint64_t da = tc_desc(a_base + kk * 256, 128, 1024);
        const uint64_t db = tc_desc(b_base + kk * 256, 128, 1024);
        const uint32_t acc = (sl > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
            :: "r"(tmem), "l"(da), "l"(db), "r"(tc_idesc()), "r"(acc) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                   :: "r"(bar) : "memory");
    }
    issued = sl + 1;
  }
  if (!abort_tile) {
    if (!mbar_wait(bar, (nslab - 1) & 1)) abort_tile = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (!abort_tile) {
    float* C = g.C ? g.C + b * g.strideC : nullptr;
    __nv_bfloat16* D = g.D ? g.D + b * g.strideC : nullptr;
    const int row = m0 + warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < TC_N; c0 += 8) {
      uint32_t r[8];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (row < g.M) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int col = n0 + c0 + e;
          if (col >= g.N) continue;
          const long long o = (long long)row * g.ldc + col;
          float v = g.alpha * __uint_as_float(r[e]);
          if (g.epilogue == RLBM_EPI_ATOMIC) {
            atomicAdd(C + o, v);
            continue;
          }
          if (C && g.beta != 0.f) v += g.beta * C[o];
          if (g.bias) v += g.bias[col];
          if (C) C[o] = v;
          if (D) D[o] = __float2bfloat16_rn(g.epilogue == RLBM_EPI_GELU ? gelu(v) : v);
        }
      }
    }
  } else {
    if (tid == 0) atomicOr(&g_tc_error, 1u);
    // let the last committed MMAs finish (bounded) before the TMEM is freed
    if (issued > 0) mbar_wait(bar, (issued - 1) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tmem), "r"(TC_N)
                 : "memory");
}

// ---------------------------------------------------------------------------
// Spectral mixing.  S, U: [batch][KX][2][KY][C]; R: [KX][KY][C][C][2].
// ---------------------------------------------------------------------------
__global__ void k_mix_fwd(const float* __restrict__ S, const float* __restrict__ R,
                          float* __restrict__ U, int batch, int KX, int KY, int C) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)batch * KX * KY * C;
  if (t >= total) return;
  const int o = (int)(t % C);
  long long r = t / C;
  const int ky = (int)(r % KY);
  r /= KY;
  const int kx = (int)(r % KX);
  const int b = (int)(r / KX);
  const float* sre = S + (((long long)b * KX + kx) * 2 + 0) * KY * C + (long long)ky * C;
  const float* sim = S + (((long long)b * KX + kx) * 2 + 1) * KY * C + (long long)ky * C;
  const float* w = R + (((long long)kx * KY + ky) * C) * C * 2;
  float ure = 0.f, uim = 0.f;
  for (int i = 0; i < C; ++i) {
    const float a = sre[i], bb = sim[i];
    const float wr = w[((long long)i * C + o) * 2], wi = w[((long long)i * C + o) * 2 + 1];
    ure = fmaf(a, wr, fmaf(-bb, wi, ure));
    uim = fmaf(a, wi, fmaf(bb, wr, uim));
  }
  U[(((long long)b * KX + kx) * 2 + 0) * KY * C + (long long)ky * C + o] = ure;
  U[(((long long)b * KX + kx) * 2 + 1) * KY * C + (long long)ky * C + o] = uim;
}

// dS(b,kx,ky,i) = sum_o dU(b,kx,ky,o) conj(R(kx,ky,i,o))
__global__ void k_mix_bwd_s(const float* __restrict__ R, const float* __restrict__ dU,
                            float* __restrict__ dS, int batch, int KX, int KY, int C) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)batch * KX * KY * C;
  if (t >= total) return;
  const int i = (int)(t % C);
  long long r = t / C;
  const int ky = (int)(r % KY);
  r /= KY;
  const int kx = (int)(r % KX);
  const int b = (int)(r / KX);
  const float* gre = dU + (((long long)b * KX + kx) * 2 + 0) * KY * C + (long long)ky * C;
  const float* gim = dU + (((long long)b * KX + kx) * 2 + 1) * KY * C + (long long)ky * C;
  const float* w = R + ((((long long)kx * KY + ky) * C + i) * C) * 2;
  float sre = 0.f, sim = 0.f;
  for (int o = 0; o < C; ++o) {
    const float gr = gre[o], gi = gim[o], wr = w[2 * o], wi = w[2 * o + 1];
    sre = fmaf(gr, wr, fmaf(gi, wi, sre));
    sim = fmaf(gi, wr, fmaf(-gr, wi, sim));
  }
  dS[(((long long)b * KX + kx) * 2 + 0) * KY * C + (long long)ky * C + i] = sre;
  dS[(((long long)b * KX + kx) * 2 + 1) * KY * C + (long long)ky * C + i] = sim;
}

// dR(kx,ky,i,o) += sum_b conj(S(b,kx,ky,i)) dU(b,kx,ky,o)
__global__ void k_mix_bwd_r(const float* __restrict__ S, const float* __restrict__ dU,
                            float* __restrict__ dR, int batch, int KX, int KY, int C) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)KX * KY * C * C;
  if (t >= total) return;
  const int o = (int)(t % C);
  long long r = t / C;
  const int i = (int)(r % C);
  r /= C;
  const int ky = (int)(r % KY);
  const int kx = (int)(r / KY);
  float rre = 0.f, rim = 0.f;
  for (int b = 0; b < batch; ++b) {
    const long long base = ((long long)b * KX + kx) * 2 * KY * C + (long long)ky * C;
    const float sr = S[base + i], si = S[base + (long long)KY * C + i];
    const float gr = dU[base + o], gi = dU[base + (long long)KY * C + o];
    rre = fmaf(sr, gr, fmaf(si, gi, rre));
    rim = fmaf(sr, gi, fmaf(-si, gr, rim));
  }
  dR[t * 2] += rre;
  dR[t * 2 + 1] += rim;
}

__global__ void k_gelu_bwd(const float* __restrict__ Z, const float* __restrict__ dH,
                           float* __restrict__ dZ, __nv_bfloat16* __restrict__ dZ16, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = dH[i] * gelu_grad(Z[i]);
  dZ[i] = g;
  if (dZ16) dZ16[i] = __float2bfloat16_rn(g);
}

__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

__device__ __forceinline__ float block_sum(float v) {
  __shared__ float s[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  v = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.f;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;
}

// acc[0] += sum m, acc[1] += sum m (Y - t)^2
__global__ void k_mse_sums(const float* __restrict__ Y, const float* __restrict__ T,
                           const float* __restrict__ m, float* acc, long long rows, int ch) {
  float sm = 0.f, se = 0.f;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
       r += (long long)gridDim.x * blockDim.x) {
    const float w = m[r];
    sm += w;
    for (int c = 0; c < ch; ++c) {
      const float d = Y[r * ch + c] - T[r * ch + c];
      se += w * d * d;
    }
  }
  sm = block_sum(sm);
  se = block_sum(se);
  if (threadIdx.x == 0) {
    atomicAdd(acc, sm);
    atomicAdd(acc + 1, se);
  }
}

__global__ void k_mse_grad(const float* __restrict__ Y, const float* __restrict__ T,
                           const float* __restrict__ m, float* __restrict__ dY,
                           const float* acc, float* loss, long long rows, int ch) {
  const float inv = 1.0f / (fmaxf(acc[0], 1.0f) * ch);
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i == 0) *loss = acc[1] * inv;
  if (i >= rows * ch) return;
  const long long r = i / ch;
  dY[i] = 2.0f * m[r] * (Y[i] - T[i]) * inv;
}

__global__ void k_colsum(const float* __restrict__ X, float* out, long long rows, int cols) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  const long long chunk = (rows + gridDim.y - 1) / gridDim.y;
  const long long r0 = blockIdx.y * chunk, r1 = r0 + chunk < rows ? r0 + chunk : rows;
  float s = 0.f;
  for (long long r = r0; r < r1; ++r) s += X[r * cols + j];
  atomicAdd(out + j, s);
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                       float* __restrict__ V, __nv_bfloat16* __restrict__ P16, long long n,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = b1 * M[i] + (1.f - b1) * g;
  const float v = b2 * V[i] + (1.f - b2) * g * g;
  M[i] = m;
  V[i] = v;
  const float p = P[i] - lr * (m * c1) / (sqrtf(v * c2) + eps);
  P[i] = p;
  if (P16) P16[i] = __float2bfloat16_rn(p);
}

__global__ void k_resample(const float* __restrict__ src, int nch, int sh, int sw,
                           float* __restrict__ dst, int dh, int dw) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)nch * dh * dw;
  if (t >= total) return;
  const int j = (int)(t % dw);
  const int i = (int)((t / dw) % dh);
  const int c = (int)(t / ((long long)dw * dh));
  float y = (i + 0.5f) * sh / dh - 0.5f, x = (j + 0.5f) * sw / dw - 0.5f;
  y = fminf(fmaxf(y, 0.f), (float)(sh - 1));
  x = fminf(fmaxf(x, 0.f), (float)(sw - 1));
  const int y0 = (int)y, x0 = (int)x;
  const int y1 = y0 + 1 < sh ? y0 + 1 : y0, x1 = x0 + 1 < sw ? x0 + 1 : x0;
  const float fy = y - y0, fx = x - x0;
  const float* p = src + (long long)c * sh * sw;
  const float v = (1.f - fy) * ((1.f - fx) * p[(long long)y0 * sw + x0] + fx * p[(long long)y0 * sw + x1])
                + fy * ((1.f - fx) * p[(long long)y1 * sw + x0] + fx * p[(long long)y1 * sw + x1]);
  dst[t] = v;
}

inline int grid1(long long n, int bs) { return (int)((n + bs - 1) / bs); }

int status() { return cudaGetLastError() == cudaSuccess ? RLBM_OK : RLBM_ECUDA; }

}  // namespace
}  // namespace rlbm

using namespace rlbm;

extern "C" {

int rlbm_gemm_bf16(int transA, int transB, int M, int N, int K, float alpha, const void* A,
                   long long lda, long long strideA, const void* B, long long ldb,
                   long long strideB, float beta, float* C, long long ldc, long long strideC,
                   const float* bias, void* D, int epilogue, int batch, void* stream) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0 || !A || !B) return RLBM_EINVAL;
  if (!C && !D) return RLBM_EINVAL;
  if (epilogue == RLBM_EPI_ATOMIC && !C) return RLBM_EINVAL;
  if (epilogue < 0 || epilogue > 2 || batch > 65535) return RLBM_EINVAL;
  GemmArgs g;
  g.transA = transA; g.transB = transB; g.M = M; g.N = N; g.K = K;
  g.alpha = alpha; g.beta = C ? beta : 0.f;
  g.A = static_cast<const __nv_bfloat16*>(A); g.lda = lda; g.strideA = strideA;
  g.B = static_cast<const __nv_bfloat16*>(B); g.ldb = ldb; g.strideB = strideB;
  g.C = C; g.ldc = ldc; g.strideC = strideC;
  g.bias = bias; g.D = static_cast<__nv_bfloat16*>(D); g.epilogue = epilogue;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  if (grid.y > 65535) return RLBM_EINVAL;
  k_gemm<<<grid, kGemmThreads, 0, static_cast<cudaStream_t>(stream)>>>(g);
  return status();
}

int rlbm_gemm_bf16_tc(int transA, int transB, int M, int N, int K, float alpha, const void* A,
                      long long lda, long long strideA, const void* B, long long ldb,
                      long long strideB, float beta, float* C, long long ldc, long long strideC,
                      const float* bias, void* D, int epilogue, int batch, void* stream) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0 || !A || !B) return RLBM_EINVAL;
  if (!C && !D) return RLBM_EINVAL;
  if (epilogue == RLBM_EPI_ATOMIC && !C) return RLBM_EINVAL;
  if (epilogue < 0 || epilogue > 2 || batch > 65535) return RLBM_EINVAL;
  GemmArgs g;
  g.transA = transA; g.transB = transB; g.M = M; g.N = N; g.K = K;
  g.alpha = alpha; g.beta = C ? beta : 0.f;
  g.A = static_cast<const __nv_bfloat16*>(A); g.lda = lda; g.strideA = strideA;
  g.B = static_cast<const __nv_bfloat16*>(B); g.ldb = ldb; g.strideB = strideB;
  g.C = C; g.ldc = ldc; g.strideC = strideC;
  g.bias = bias; g.D = static_cast<__nv_bfloat16*>(D); g.epilogue = epilogue;
  dim3 grid((N + TC_N - 1) / TC_N, (M + TC_M - 1) / TC_M, batch);
  if (grid.y > 65535) return RLBM_EINVAL;
  k_gemm_tc<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(g);
  return status();
}

int rlbm_gemm_tc_error(int* flag) {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof v) != cudaSuccess) return RLBM_ECUDA;
  if (flag) *flag = (int)v;
  if (v) {
    const unsigned z = 0;
    cudaMemcpyToSymbol(g_tc_error, &z, sizeof z);
  }
  return RLBM_OK;
}

int rlbm_fno_mix_forward(const float* S, const float* R, float* U, int batch, int KX, int KY,
                         int C, void* stream) {
  const long long n = (long long)batch * KX * KY * C;
  if (n <= 0) return RLBM_EINVAL;
  k_mix_fwd<<<grid1(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(S, R, U, batch, KX, KY, C);
  return status();
}

int rlbm_fno_mix_backward(const float* S, const float* R, const float* dU, float* dS, float* dR,
                          int batch, int KX, int KY, int C, void* stream) {
  const long long n = (long long)batch * KX * KY * C;
  if (n <= 0) return RLBM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_mix_bwd_s<<<grid1(n, 256), 256, 0, st>>>(R, dU, dS, batch, KX, KY, C);
  const long long nr = (long long)KX * KY * C * C;
  k_mix_bwd_r<<<grid1(nr, 256), 256, 0, st>>>(S, dU, dR, batch, KX, KY, C);
  return status();
}

int rlbm_fno_gelu_backward(const float* Z, const float* dH, float* dZ, void* dZ16, long long n,
                           void* stream) {
  if (n <= 0) return RLBM_EINVAL;
  k_gelu_bwd<<<grid1(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      Z, dH, dZ, static_cast<__nv_bfloat16*>(dZ16), n);
  return status();
}

int rlbm_fno_to_bf16(const float* x, void* y, long long n, void* stream) {
  if (n <= 0) return RLBM_EINVAL;
  k_to_bf16<<<grid1(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      x, static_cast<__nv_bfloat16*>(y), n);
  return status();
}

int rlbm_fno_mse(const float* Y, const float* target, const float* mask, float* dY, float* loss,
                 long long rows, int ch, void* stream) {
  if (rows <= 0 || ch <= 0) return RLBM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // loss[1], loss[2]: sums of the mask and of the weighted squared error
  cudaMemsetAsync(loss + 1, 0, 2 * sizeof(float), st);
  k_mse_sums<<<256, 256, 0, st>>>(Y, target, mask, loss + 1, rows, ch);
  k_mse_grad<<<grid1(rows * ch, 256), 256, 0, st>>>(Y, target, mask, dY, loss + 1, loss, rows,
                                                     ch);
  return status();
}

int rlbm_fno_colsum(const float* X, float* out, long long rows, int cols, void* stream) {
  if (rows <= 0 || cols <= 0) return RLBM_EINVAL;
  dim3 grid((cols + 127) / 128, (unsigned)(rows < 512 ? rows : 512));
  k_colsum<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(X, out, rows, cols);
  return status();
}

int rlbm_fno_adam(float* P, const float* G, float* M, float* V, void* P16, long long n, float lr,
                  float beta1, float beta2, float eps, int t, void* stream) {
  if (n <= 0 || t < 1) return RLBM_EINVAL;
  const float c1 = 1.0f / (1.0f - powf(beta1, (float)t));
  const float c2 = 1.0f / (1.0f - powf(beta2, (float)t));
  k_adam<<<grid1(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      P, G, M, V, static_cast<__nv_bfloat16*>(P16), n, lr, beta1, beta2, eps, c1, c2);
  return status();
}

int rlbm_resample_bilinear(const float* src, int nch, int sh, int sw, float* dst, int dh, int dw,
                           void* stream) {
  if (nch <= 0 || sh <= 0 || sw <= 0 || dh <= 0 || dw <= 0) return RLBM_EINVAL;
  const long long n = (long long)nch * dh * dw;
  k_resample<<<grid1(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(src, nch, sh, sw, dst,
                                                                          dh, dw);
  return status();
}

}  // extern "C"

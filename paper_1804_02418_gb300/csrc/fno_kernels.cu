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
// FP32 GEMM on the FP32 units (the operator's FP32 mode, whose results are
// compared with the FP64 oracle at 1e-5): 64 x 64 block tiles, K slices of 16
// staged k-major in shared memory, 256 threads with 4 x 4 outputs each.  Same
// arguments, layouts and epilogues as k_gemm; D is FP32.
// ---------------------------------------------------------------------------
constexpr int FBM = 64, FBN = 64, FBK = 16, kF32Threads = 256;

struct GemmArgsF32 {
  int transA, transB, M, N, K;
  float alpha, beta;
  const float* A;
  long long lda, strideA;
  const float* B;
  long long ldb, strideB;
  float* C;
  long long ldc, strideC;
  const float* bias;
  float* D;
  int epilogue;
};

__global__ void __launch_bounds__(kF32Threads) k_gemm_f32(GemmArgsF32 g) {
  __shared__ float As[FBK][FBM + 4];
  __shared__ float Bs[FBK][FBN + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * FBM, n0 = blockIdx.x * FBN;
  const long long b = blockIdx.z;
  const float* A = g.A + b * g.strideA;
  const float* B = g.B + b * g.strideB;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < g.K; k0 += FBK) {
    // consecutive threads read consecutive addresses of the stored layout
    for (int i = tid; i < FBM * FBK; i += kF32Threads) {
      int m, k;
      if (!g.transA) { m = i / FBK; k = i % FBK; } else { k = i / FBM; m = i % FBM; }
      const int gm = m0 + m, gk = k0 + k;
      float v = 0.f;
      if (gm < g.M && gk < g.K) v = g.transA ? A[(long long)gk * g.lda + gm] : A[(long long)gm * g.lda + gk];
      As[k][m] = v;
    }
    for (int i = tid; i < FBN * FBK; i += kF32Threads) {
      int n, k;
      if (!g.transB) { k = i / FBN; n = i % FBN; } else { n = i / FBK; k = i % FBK; }
      const int gn = n0 + n, gk = k0 + k;
      float v = 0.f;
      if (gn < g.N && gk < g.K) v = g.transB ? B[(long long)gn * g.ldb + gk] : B[(long long)gk * g.ldb + gn];
      Bs[k][n] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < FBK; ++kk) {
      float a[4], c[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) c[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], c[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* C = g.C ? g.C + b * g.strideC : nullptr;
  float* D = g.D ? g.D + b * g.strideC : nullptr;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = m0 + ty * 4 + i, col = n0 + tx * 4 + j;
      if (row >= g.M || col >= g.N) continue;
      const long long o = (long long)row * g.ldc + col;
      float v = g.alpha * acc[i][j];
      if (g.epilogue == RLBM_EPI_ATOMIC) {
        atomicAdd(C + o, v);
        continue;
      }
      if (C && g.beta != 0.f) v += g.beta * C[o];
      if (g.bias) v += g.bias[col];
      if (C) C[o] = v;
      if (D) D[o] = g.epilogue == RLBM_EPI_GELU ? gelu(v) : v;
    }
}

// ---------------------------------------------------------------------------
// Fifth-generation tensor-core GEMM (tcgen05 / TMEM): one CTA of 4 warps per
// 128 x BN output tile (BN = 32 / 64 / 128 chosen per call), K in slabs of 64.
//
// Operands live in shared memory in the canonical no-swizzle K-major layout:
// 8 x 16-byte core matrices (8 rows, 8 consecutive k each), the two k-halves
// of a K16 step LBO = 128 B apart, consecutive 8-row groups SBO = 1040 B apart
// (1024 B of data plus 16 B of padding against bank conflicts).
// Staging moves 16-byte chunks: an operand whose rows are contiguous in k
// (A not transposed, B transposed) is copied chunk for chunk; an operand
// contiguous along M / N is read as 8 x 8 blocks (8 chunks along k) and
// transposed in registers (byte permutes) on the way.  Ragged or unaligned
// chunks fall back to element loads with zero fill.  Two slab buffers: the
// global loads of slab s + 1 are issued while the MMAs of slab s run; one
// thread issues four tcgen05.mma (M 128, N BN, K 16, BF16 -> FP32 in TMEM)
// per slab and commits them to that buffer's mbarrier, which frees the buffer
// again.  The epilogue reads the accumulator with tcgen05.ld (warp w owns
// TMEM lanes / output rows 32 w .. 32 w + 31) and stores 16-byte vectors where
// the output is aligned.  Every wait is bounded: on timeout the CTA raises the
// error flag, skips its tile, drains its MMAs, frees its TMEM and returns.
// ---------------------------------------------------------------------------
constexpr int TC_M = 128, TC_K = 64;
// Core matrices: k groups 128 B apart (LBO), 8-row groups kTcSbo apart (SBO,
// padded by 16 B so that stores of different row groups fall on different
// shared-memory banks).
constexpr int kTcLbo = 128, kTcSbo = 1040;
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
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
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

// One operand of the tile: `rows` rows (M or N) of one K slab.
struct TcOperand {
  const __nv_bfloat16* p;   // batch base
  long long ld;             // leading dimension (elements)
  int row0, nrows;          // first row of the tile, rows of the whole operand
  int K;
  bool kcontig;             // element (row, k) at p[row * ld + k] (else p[k * ld + row])
  bool vec;                 // 16-byte chunks allowed (aligned base, ld, batch stride)
};

__device__ __forceinline__ __nv_bfloat16 tc_elem(const TcOperand& o, int r, int k) {
  const int gr = o.row0 + r;
  if (gr >= o.nrows || k >= o.K) return __float2bfloat16(0.0f);
  return o.kcontig ? o.p[(long long)gr * o.ld + k] : o.p[(long long)k * o.ld + gr];
}

// Register copy of this thread's share of one slab of one operand: R rows.
// K-contiguous: chunk i (i = tid + 128 q) = row i % R, k group i / R.
// MN-contiguous: block i = (row group i % (R / 8), k group i / (R / 8)), 8 chunks.
template <int R>
struct TcStage {
  static constexpr int kChunks = R * 8 / 128;          // K-contiguous chunks per thread
  static constexpr int kBlocks = (R / 8) * 8;          // MN-contiguous 8x8 blocks per slab
  uint4 v[8];

  __device__ __forceinline__ void load(const TcOperand& o, int k0) {
    const int tid = threadIdx.x;
    if (o.kcontig) {
#pragma unroll
      for (int q = 0; q < kChunks; ++q) {
        const int i = tid + 128 * q, r = i % R, kg = i / R;
        const int gr = o.row0 + r, gk = k0 + 8 * kg;
        if (o.vec && gr < o.nrows && gk + 8 <= o.K) {
          v[q] = __ldg(reinterpret_cast<const uint4*>(o.p + (long long)gr * o.ld + gk));
        } else {
          __nv_bfloat16 e[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) e[j] = tc_elem(o, r, gk + j);
          memcpy(&v[q], e, 16);
        }
      }
    } else if (tid < kBlocks) {
      const int rg = tid % (R / 8), kg = tid / (R / 8);
      const int gr = o.row0 + 8 * rg;
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const int gk = k0 + 8 * kg + kk;
        if (o.vec && gr + 8 <= o.nrows && gk < o.K) {
          v[kk] = __ldg(reinterpret_cast<const uint4*>(o.p + (long long)gk * o.ld + gr));
        } else {
          __nv_bfloat16 e[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) e[j] = tc_elem(o, 8 * rg + j, gk);
          memcpy(&v[kk], e, 16);
        }
      }
    }
  }

  // Writes the registers into the K-major slab at shared address `base`.
  __device__ __forceinline__ void store(const TcOperand& o, uint32_t base) {
    const int tid = threadIdx.x;
    if (o.kcontig) {
#pragma unroll
      for (int q = 0; q < kChunks; ++q) {
        const int i = tid + 128 * q, r = i % R, kg = i / R;
        const uint32_t a = base + (uint32_t)((r >> 3) * kTcSbo + kg * kTcLbo + (r & 7) * 16);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n"
                     :: "r"(a), "r"(v[q].x), "r"(v[q].y), "r"(v[q].z), "r"(v[q].w) : "memory");
      }
    } else if (tid < kBlocks) {
      const int rg = tid % (R / 8), kg = tid / (R / 8);
      const uint32_t cm = base + (uint32_t)(rg * kTcSbo + kg * kTcLbo);
      // transpose: output row c (one M / N index) holds k = 0..7; word w of it
      // pairs k = 2w, 2w + 1, taken from word c / 2 of input chunks 2w, 2w + 1
      const uint32_t* in = reinterpret_cast<const uint32_t*>(v);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint32_t sel = (c & 1) ? 0x7632u : 0x5410u;
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t lo = in[(2 * q) * 4 + (c >> 1)], hi = in[(2 * q + 1) * 4 + (c >> 1)];
          w[q] = __byte_perm(lo, hi, sel);
        }
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n"
                     :: "r"(cm + c * 16), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]) : "memory");
      }
    }
  }
};

template <int BN>
__global__ void __launch_bounds__(128) k_gemm_tc(GemmArgs g, int vecA, int vecB) {
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  constexpr int A_BYTES = (TC_M / 8) * kTcSbo, B_BYTES = (BN / 8) * kTcSbo;
  constexpr int STAGE = A_BYTES + B_BYTES;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * BN;
  const long long b = blockIdx.z;
  TcOperand A{g.A + b * g.strideA, g.lda, m0, g.M, g.K, g.transA == 0, vecA != 0};
  TcOperand B{g.B + b * g.strideB, g.ldb, n0, g.N, g.K, g.transB != 0, vecB != 0};
  const uint32_t smem0 = smem_u32(tc_smem);
  const uint32_t bar0 = smem_u32(&mbar[0]), bar1 = smem_u32(&mbar[1]);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 :: "r"(smem_u32(&tmem_slot)), "r"(BN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;

  TcStage<TC_M> ra;
  TcStage<BN> rb;
  const int nslab = (g.K + TC_K - 1) / TC_K;
  int issued = 0;        // slabs whose MMAs were committed (same in every thread)
  bool abort_tile = false;
  ra.load(A, 0);
  rb.load(B, 0);
  for (int sl = 0; sl < nslab; ++sl) {
    const int buf = sl & 1;
    const uint32_t sa = smem0 + buf * STAGE, sb = sa + A_BYTES;
    bool ok = true;
    // buffer `buf` was last read by the MMAs of slab sl - 2
    if (sl >= 2) ok = mbar_wait(buf ? bar1 : bar0, ((sl - 2) >> 1) & 1);
    if (ok) {
      ra.store(A, sa);
      rb.store(B, sb);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (__syncthreads_or(!ok)) { abort_tile = true; break; }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < TC_K / 16; ++kk) {
        const uint64_t da = tc_desc(sa + kk * 2 * kTcLbo, kTcLbo, kTcSbo);
        const uint64_t db = tc_desc(sb + kk * 2 * kTcLbo, kTcLbo, kTcSbo);
        const uint32_t acc = (sl > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
            :: "r"(tmem), "l"(da), "l"(db), "r"(tc_idesc(BN)), "r"(acc) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                   :: "r"(buf ? bar1 : bar0) : "memory");
    }
    issued = sl + 1;
    // the next slab's global loads overlap these MMAs
    if (sl + 1 < nslab) {
      ra.load(A, (sl + 1) * TC_K);
      rb.load(B, (sl + 1) * TC_K);
    }
  }
  if (!abort_tile) {
    const int last = nslab - 1;
    const bool ok = mbar_wait((last & 1) ? bar1 : bar0, (last >> 1) & 1);
    abort_tile = __syncthreads_or(!ok);
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (!abort_tile) {
    float* C = g.C ? g.C + b * g.strideC : nullptr;
    __nv_bfloat16* D = g.D ? g.D + b * g.strideC : nullptr;
    const int row = m0 + warp * 32 + lane;
    // 16-byte stores need 4 (f32) / 8 (bf16) aligned columns, row pitch and base
    const bool vc = C && (g.ldc % 4 == 0) && (g.strideC % 4 == 0) &&
                    ((reinterpret_cast<uintptr_t>(g.C) & 15) == 0);
    const bool vd = D && (g.ldc % 8 == 0) && (g.strideC % 8 == 0) &&
                    ((reinterpret_cast<uintptr_t>(g.D) & 15) == 0);
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += 8) {
      uint32_t r[8];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      const int col0 = n0 + c0;
      if (row >= g.M || col0 >= g.N) continue;
      const long long o = (long long)row * g.ldc + col0;
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = g.alpha * __uint_as_float(r[e]);
      const bool full = col0 + 8 <= g.N;
      if (g.epilogue == RLBM_EPI_ATOMIC) {
        if (vc && full) {
          atomicAdd(reinterpret_cast<float4*>(C + o), make_float4(v[0], v[1], v[2], v[3]));
          atomicAdd(reinterpret_cast<float4*>(C + o + 4), make_float4(v[4], v[5], v[6], v[7]));
        } else {
          for (int e = 0; e < 8 && col0 + e < g.N; ++e) atomicAdd(C + o + e, v[e]);
        }
        continue;
      }
      if (C && g.beta != 0.f) {
        if (vc && full) {
          const float4 p = *reinterpret_cast<const float4*>(C + o);
          const float4 q = *reinterpret_cast<const float4*>(C + o + 4);
          v[0] += g.beta * p.x; v[1] += g.beta * p.y; v[2] += g.beta * p.z; v[3] += g.beta * p.w;
          v[4] += g.beta * q.x; v[5] += g.beta * q.y; v[6] += g.beta * q.z; v[7] += g.beta * q.w;
        } else {
          for (int e = 0; e < 8 && col0 + e < g.N; ++e) v[e] += g.beta * C[o + e];
        }
      }
      if (g.bias) {
#pragma unroll
        for (int e = 0; e < 8; ++e) if (col0 + e < g.N) v[e] += g.bias[col0 + e];
      }
      if (C) {
        if (vc && full) {
          *reinterpret_cast<float4*>(C + o) = make_float4(v[0], v[1], v[2], v[3]);
          *reinterpret_cast<float4*>(C + o + 4) = make_float4(v[4], v[5], v[6], v[7]);
        } else {
          for (int e = 0; e < 8 && col0 + e < g.N; ++e) C[o + e] = v[e];
        }
      }
      if (D) {
        __nv_bfloat16 h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e)
          h[e] = __float2bfloat16_rn(g.epilogue == RLBM_EPI_GELU ? gelu(v[e]) : v[e]);
        if (vd && full) {
          uint4 u;
          memcpy(&u, h, 16);
          *reinterpret_cast<uint4*>(D + o) = u;
        } else {
          for (int e = 0; e < 8 && col0 + e < g.N; ++e) D[o + e] = h[e];
        }
      }
    }
  } else {
    if (tid == 0) atomicOr(&g_tc_error, 1u);
    // let the last committed MMAs finish (bounded) before the TMEM is freed
    if (issued > 0) mbar_wait(((issued - 1) & 1) ? bar1 : bar0, ((issued - 1) >> 1) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tmem), "r"(BN)
                 : "memory");
}

template <int BN>
constexpr int tc_smem_bytes() { return 2 * ((TC_M / 8) * kTcSbo + (BN / 8) * kTcSbo); }

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

// Column sums of X [rows][cols] added to out.  With cols <= 256, a block of
// 256 threads covers 256 / cols rows per pass (thread t: column t % cols, row
// t / cols; coalesced), walks the rows with a grid stride, and reduces the
// per-thread partial sums of each column in shared memory before one atomic
// add per column.  Wider matrices: one column per thread, looped.
constexpr int kColsumThreads = 256;

__global__ void __launch_bounds__(kColsumThreads) k_colsum(const float* __restrict__ X, float* out,
                                                           long long rows, int cols) {
  __shared__ float part[kColsumThreads];
  const int t = threadIdx.x;
  if (cols <= kColsumThreads) {
    const int rpp = kColsumThreads / cols;             // rows per pass
    const int j = t % cols, rr = t / cols;
    float s = 0.f;
    if (rr < rpp)
      for (long long r = (long long)blockIdx.x * rpp + rr; r < rows; r += (long long)gridDim.x * rpp)
        s += X[r * cols + j];
    part[t] = rr < rpp ? s : 0.f;
    __syncthreads();
    if (t < cols) {
      float c = 0.f;
      for (int k = 0; k < rpp; ++k) c += part[k * cols + t];
      atomicAdd(out + t, c);
    }
  } else {
    for (int j = t; j < cols; j += kColsumThreads) {
      float s = 0.f;
      for (long long r = blockIdx.x; r < rows; r += gridDim.x) s += X[r * cols + j];
      atomicAdd(out + j, s);
    }
  }
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

int rlbm_gemm_f32(int transA, int transB, int M, int N, int K, float alpha, const float* A,
                  long long lda, long long strideA, const float* B, long long ldb,
                  long long strideB, float beta, float* C, long long ldc, long long strideC,
                  const float* bias, float* D, int epilogue, int batch, void* stream) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0 || !A || !B) return RLBM_EINVAL;
  if (!C && !D) return RLBM_EINVAL;
  if (epilogue == RLBM_EPI_ATOMIC && !C) return RLBM_EINVAL;
  if (epilogue < 0 || epilogue > 2 || batch > 65535) return RLBM_EINVAL;
  GemmArgsF32 g;
  g.transA = transA; g.transB = transB; g.M = M; g.N = N; g.K = K;
  g.alpha = alpha; g.beta = C ? beta : 0.f;
  g.A = A; g.lda = lda; g.strideA = strideA;
  g.B = B; g.ldb = ldb; g.strideB = strideB;
  g.C = C; g.ldc = ldc; g.strideC = strideC;
  g.bias = bias; g.D = D; g.epilogue = epilogue;
  dim3 grid((N + FBN - 1) / FBN, (M + FBM - 1) / FBM, batch);
  if (grid.y > 65535) return RLBM_EINVAL;
  k_gemm_f32<<<grid, kF32Threads, 0, static_cast<cudaStream_t>(stream)>>>(g);
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
  // 16-byte operand chunks need aligned bases, leading dimensions and strides
  const bool vecA = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && lda % 8 == 0 &&
                    strideA % 8 == 0;
  const bool vecB = ((reinterpret_cast<uintptr_t>(B) & 15) == 0) && ldb % 8 == 0 &&
                    strideB % 8 == 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned gy = (unsigned)((M + TC_M - 1) / TC_M);
  if (gy > 65535) return RLBM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RLBM_ECUDA;
  static bool smem_set[64][3] = {};
  auto launch = [&](auto kernel, int bn, int slot, int bytes) -> int {
    if (!smem_set[dev][slot]) {
      if (cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               bytes) != cudaSuccess)
        return RLBM_ECUDA;
      smem_set[dev][slot] = true;
    }
    dim3 grid((unsigned)((N + bn - 1) / bn), gy, (unsigned)batch);
    kernel<<<grid, 128, bytes, st>>>(g, (int)vecA, (int)vecB);
    return RLBM_OK;
  };
  int r;
  if (N <= 32) r = launch(k_gemm_tc<32>, 32, 0, tc_smem_bytes<32>());
  else if (N <= 64) r = launch(k_gemm_tc<64>, 64, 1, tc_smem_bytes<64>());
  else r = launch(k_gemm_tc<128>, 128, 2, tc_smem_bytes<128>());
  if (r != RLBM_OK) return r;
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
  const long long passes = cols <= kColsumThreads ? rows / (kColsumThreads / cols) + 1 : rows;
  const int grid = (int)(passes < 1216 ? passes : 1216);
  k_colsum<<<grid, kColsumThreads, 0, static_cast<cudaStream_t>(stream)>>>(X, out, rows, cols);
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

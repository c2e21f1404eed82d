/*
 * rlbm_fno.h - C ABI of the spectral neural operator kernels (learned warm
 * start of the relativistic LBM; no counterpart in the paper, whose method
 * this only initialises).
 *
 * A Fourier neural operator maps per-site input channels (geometry mask,
 * drive, relaxation time, coordinates) on an N x N canvas to the steady
 * macroscopic fields (n, u_x, u_y, T).  Every layer is expressed as batched
 * BF16 tensor-core GEMMs with FP32 accumulation (truncated DFTs as products
 * with DFT matrices, pointwise channel mixing), a per-mode complex channel
 * mixing in FP32, and elementwise kernels.  All pointers are device pointers
 * on the current device; the caller owns them.  Every call is asynchronous on
 * `stream` (NULL: default stream) and returns RLBM_OK (0) or a negative code
 * of rlbm.h (RLBM_EINVAL for bad sizes, RLBM_ECUDA for launch failures).
 *
 * Element types: "bf16" buffers hold IEEE bfloat16 (2 bytes), "f32" buffers
 * IEEE binary32.
 */
#ifndef RLBM_FNO_H
#define RLBM_FNO_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RLBM_EPI_NONE = 0,     /* C = alpha A B + beta C + bias */
  RLBM_EPI_GELU = 1,     /* as NONE, and D = gelu(C) (erf form) in bf16 */
  RLBM_EPI_ATOMIC = 2    /* C += alpha A B (atomic adds: split-K over the batch) */
};

/* Batched C_b = alpha * op(A_b) op(B_b) (+ beta C_b + bias) for b < batch.
 * op(A) is M x K: A is row-major M x K (lda >= K) if transA == 0, K x M
 * (lda >= M) otherwise; op(B) is K x N: B row-major K x N (ldb >= N) if
 * transB == 0, N x K (ldb >= K) otherwise.  A, B bf16; C f32 row-major
 * M x N with ldc >= N; bias (f32, length N) may be NULL; D (bf16, same
 * layout as C, used by RLBM_EPI_GELU) may be NULL.  Batch strides are in
 * elements and may be 0 (shared operand).  beta is ignored by
 * RLBM_EPI_ATOMIC.  Tensor cores: mma m16n8k16 BF16 -> FP32. */
int rlbm_gemm_bf16(int transA, int transB, int M, int N, int K, float alpha,
                   const void* A, long long lda, long long strideA,
                   const void* B, long long ldb, long long strideB,
                   float beta, float* C, long long ldc, long long strideC,
                   const float* bias, void* D, int epilogue, int batch, void* stream);

/* The same operation as rlbm_gemm_bf16 (same arguments, layouts and
 * epilogues) on the fifth-generation tensor cores: one CTA per 128 x 64
 * output tile, operands staged in shared memory, tcgen05.mma (M 128, N 64,
 * K 16, BF16 x BF16 -> FP32) accumulating in tensor memory, read back with
 * tcgen05.ld for the epilogue.  The summation order over K differs from
 * rlbm_gemm_bf16, so the two agree to FP32 rounding, not bit for bit.  Every
 * wait inside the kernel is bounded (about 2 s); a CTA that gives up skips
 * its tile and sets a device flag that rlbm_gemm_tc_error reports. */
int rlbm_gemm_bf16_tc(int transA, int transB, int M, int N, int K, float alpha,
                      const void* A, long long lda, long long strideA,
                      const void* B, long long ldb, long long strideB,
                      float beta, float* C, long long ldc, long long strideC,
                      const float* bias, void* D, int epilogue, int batch, void* stream);

/* The same operation as rlbm_gemm_bf16 on FP32 operands, on the FP32 units
 * (FP32 products and accumulation): A, B and D are f32 (D receives C's value,
 * or gelu of it with RLBM_EPI_GELU).  The operator's FP32 mode runs on it. */
int rlbm_gemm_f32(int transA, int transB, int M, int N, int K, float alpha,
                  const float* A, long long lda, long long strideA,
                  const float* B, long long ldb, long long strideB,
                  float beta, float* C, long long ldc, long long strideC,
                  const float* bias, float* D, int epilogue, int batch, void* stream);

/* Reads (and clears) the timeout flag of rlbm_gemm_bf16_tc on the current
 * device: *flag = 0 if no CTA gave up since the last call.  Synchronous with
 * respect to the device (the read waits for prior work). */
int rlbm_gemm_tc_error(int* flag);

/* Per-mode complex channel mixing of the spectral layer.
 * S, U: f32 [batch][KX][2][KY][C] (re / im planes per kx), R: f32
 * [KX][KY][C][C][2] (re, im), U(b, kx, ky, o) = sum_i S(b, kx, ky, i) R(kx, ky, i, o). */
int rlbm_fno_mix_forward(const float* S, const float* R, float* U, int batch, int KX, int KY,
                         int C, void* stream);

/* Gradients of the mixing: dS = dU conj(R) (written), dR += conj(S) dU
 * summed over the batch (accumulated). */
int rlbm_fno_mix_backward(const float* S, const float* R, const float* dU, float* dS,
                          float* dR, int batch, int KX, int KY, int C, void* stream);

/* dZ = dH * gelu'(Z) elementwise (Z: pre-activation); written as f32 and,
 * if dZ16 != NULL, as bf16. */
int rlbm_fno_gelu_backward(const float* Z, const float* dH, float* dZ, void* dZ16,
                           long long n, void* stream);

/* f32 -> bf16 (round to nearest even), n elements. */
int rlbm_fno_to_bf16(const float* x, void* y, long long n, void* stream);

/* Masked mean-squared error of Y (f32 [rows][ch]) against target (same
 * layout) with weights mask (f32 [rows], 0 or 1): loss[0] = sum m (Y - t)^2 /
 * (ch * sum m) and dY = d loss / d Y.  loss points at 3 device f32 values:
 * loss[1], loss[2] are the caller-provided scratch of the two sums. */
int rlbm_fno_mse(const float* Y, const float* target, const float* mask, float* dY,
                 float* loss, long long rows, int ch, void* stream);

/* Column sums: out[j] += sum_r X[r][j] (bias gradients), X f32 [rows][cols]. */
int rlbm_fno_colsum(const float* X, float* out, long long rows, int cols, void* stream);

/* Adam (with bias correction, step t >= 1) on f32 master weights P with
 * gradient G and moments M, V (all n); writes the bf16 copy P16 if non-NULL. */
int rlbm_fno_adam(float* P, const float* G, float* M, float* V, void* P16, long long n,
                  float lr, float beta1, float beta2, float eps, int t, void* stream);

/* Bilinear resampling of nch f32 planes: src [nch][sh][sw] (row-major) onto
 * dst [nch][dh][dw]; destination pixel (i, j) samples source point
 * ((i + 0.5) * sh / dh - 0.5, (j + 0.5) * sw / dw - 0.5) clamped to the edges. */
int rlbm_resample_bilinear(const float* src, int nch, int sh, int sw, float* dst, int dh, int dw,
                           void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RLBM_FNO_H */

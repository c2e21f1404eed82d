// Arithmetic peak probe (declared in include/rlbm.h as rlbm_fma_peak): the
// rate at which this GPU retires fused multiply-adds of one type, measured
// with a kernel that does nothing else.  It is the denominator of the
// arithmetic roofline of a kernel that is bound by its FP64 (or FP32)
// instructions rather than by memory, such as the FP64 fused step.
//
// Every thread runs kChains independent FMA chains for `iters` rounds (the
// chains hide the pipeline latency), one 256-thread block per 1/8 of an SM's
// thread slots, 8 blocks per SM; the chain values are summed and stored so
// that nothing is dead code.  One launch is timed with CUDA events after two
// warm-up launches; the result is the best of three.
#include "rlbm.h"

#include <cuda_runtime.h>

#include <cstdio>

namespace rlbm {

void set_global_error(const char* msg);   // api.cpp: text for rlbm_last_error(NULL)

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* out, T b, T c, int iters) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x) * T(1e-3) + T(k);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int fail(const char* what, cudaError_t e) {
  char b[200];
  snprintf(b, sizeof b, "rlbm_fma_peak: %s: %s", what, cudaGetErrorString(e));
  set_global_error(b);
  return RLBM_ECUDA;
}

template <typename T>
int measure(int iters, double* fma_per_s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail("device query", e);
  const int blocks = 8 * sms;
  T* out = nullptr;
  e = cudaMalloc(&out, sizeof(T) * (size_t)blocks * kThreads);
  if (e != cudaSuccess) return fail("cudaMalloc", e);
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0.0;
  if (e == cudaSuccess) {
    const T b = T(0.999), c = T(1e-3);
    for (int w = 0; w < 2; ++w) k_fma_chains<T><<<blocks, kThreads, 0, st>>>(out, b, c, iters);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
      cudaEventRecord(e0, st);
      k_fma_chains<T><<<blocks, kThreads, 0, st>>>(out, b, c, iters);
      cudaEventRecord(e1, st);
      e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      const double fmas = (double)blocks * kThreads * kChains * (double)iters;
      if (e == cudaSuccess && ms > 0.f && fmas / (ms * 1e-3) > best) best = fmas / (ms * 1e-3);
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  if (e != cudaSuccess) return fail("probe kernel", e);
  *fma_per_s = best;
  return RLBM_OK;
}

}  // namespace
}  // namespace rlbm

extern "C" int rlbm_fma_peak(int fp64, double* fma_per_s) {
  if (!fma_per_s) {
    rlbm::set_global_error("rlbm_fma_peak: fma_per_s is NULL");
    return RLBM_EINVAL;
  }
  // a few milliseconds per launch at GB300's rates (FP64 retires ~1/58 of FP32)
  return fp64 ? rlbm::measure<double>(512, fma_per_s) : rlbm::measure<float>(16384, fma_per_s);
}

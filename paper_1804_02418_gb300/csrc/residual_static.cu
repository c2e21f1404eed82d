// Convergence residual without any allocation (declared in include/rlbm.h as
// rlbm_velocity_residual_static).
//
// Some callers of this library cannot allocate device memory at the moment
// they want a convergence check: code that runs while another framework owns
// the whole device memory pool, real-time monitoring loops whose memory
// budget was fixed at start-up, or host callbacks in which cudaMalloc is not
// allowed.  For them this entry point computes the same quantity as the
// residual of rlbm_step,
//     r = ||u(t) - u(t-1)||_2 / ||u(t)||_2 ,
// from two velocity fields they already hold on the device, using only a
// fixed scratch array that is part of the library image itself.
//
// Scratch: one (sum |u - u_prev|^2, sum |u|^2) pair per block of 2048 sites,
// in a file-scope device array of kResMaxBlocks pairs (64 KiB).  Every GPU
// that loads the library holds this array until the process exits.  Each
// call rewrites every slot it later reads, so nothing has to be cleared
// between calls; slots beyond a call's block count are never read.  All calls
// share the array: calls that overlap on the GPU (for example on two streams)
// race on it and must be serialised by the caller.
//
// Host code must not pass the array's name to a kernel: on the host it is
// only a stand-in symbol.  Its device address belongs to the CUDA context
// that loaded the library's module, so every call made outside a stream
// capture looks it up again with cudaGetSymbolAddress (which allocates
// nothing) in the context current at that moment; a pointer kept from an
// earlier context (before cudaDeviceReset, or another context on the same
// device) is never used.  A call made while its stream is being captured
// cannot look it up and takes the address the last uncaptured call on the
// same device found: make one call outside capture first, and again after
// cudaDeviceReset or a change of context, before capturing.
#include "rlbm.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

namespace rlbm {

void set_global_error(const char* msg);   // api.cpp: text for rlbm_last_error(NULL)

namespace {

constexpr int kResThreads = 256;
constexpr int kResTile = 2048;                                   // sites per block
constexpr int kResMaxBlocks = 4096;
constexpr long long kResMaxSites = (long long)kResTile * kResMaxBlocks;   // 8,388,608
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_res_partials[2 * kResMaxBlocks];

__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[kResThreads / 32], sb[kResThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sa[warp] = a; sb[warp] = b; }
  __syncthreads();
  if (warp == 0) {
    a = lane < kResThreads / 32 ? sa[lane] : 0.0;
    b = lane < kResThreads / 32 ? sb[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
  }
}

// One block per tile of kResTile sites: writes its pair into partials[2 b].
__global__ void __launch_bounds__(kResThreads)
k_res_partial(const double* __restrict__ uxp, const double* __restrict__ uyp,
              const double* __restrict__ ux, const double* __restrict__ uy, long long n,
              double* __restrict__ partials) {
  double a = 0.0, b = 0.0;
  const long long base = (long long)blockIdx.x * kResTile;
  for (int k = threadIdx.x; k < kResTile; k += kResThreads) {
    const long long i = base + k;
    if (i >= n) break;
    const double x = ux[i], y = uy[i];
    const double dx = x - uxp[i], dy = y - uyp[i];
    a += dx * dx + dy * dy;
    b += x * x + y * y;
  }
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

// One block: sums the first nblocks pairs in a fixed order and writes r.
__global__ void __launch_bounds__(kResThreads)
k_res_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += kResThreads) {
    a += partials[2 * k];
    b += partials[2 * k + 1];
  }
  block_sum2(a, b);
  if (threadIdx.x == 0) *out = b > 0.0 ? sqrt(a / b) : (a == 0.0 ? 0.0 : INFINITY);
}

std::mutex g_setup_mutex;
double* g_scratch[kMaxDevices] = {};

int fail(int code, const char* msg) {
  set_global_error(msg);
  return code;
}

}  // namespace
}  // namespace rlbm

extern "C" int rlbm_velocity_residual_static(const double* ux_prev, const double* uy_prev,
                                             const double* ux, const double* uy,
                                             long long nsites, double* residual, void* stream) {
  using namespace rlbm;
  if (!ux_prev || !uy_prev || !ux || !uy || !residual)
    return fail(RLBM_EINVAL, "rlbm_velocity_residual_static: a pointer is NULL");
  if (nsites < 1 || nsites > kResMaxSites) {
    char b[160];
    snprintf(b, sizeof b,
             "rlbm_velocity_residual_static: nsites = %lld outside 1..%lld (scratch holds %d "
             "blocks of %d sites)", nsites, kResMaxSites, kResMaxBlocks, kResTile);
    return fail(RLBM_EINVAL, b);
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(RLBM_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(RLBM_EINVAL, "rlbm_velocity_residual_static: device index out of range");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Is the stream being captured?  An error (e.g. the legacy stream while
  // another stream captures globally) counts as capturing: no lookup then.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  bool capturing = false;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    (void)cudaGetLastError();
    capturing = true;
  } else {
    capturing = cs != cudaStreamCaptureStatusNone;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!capturing) {
      // the address in the context that is current now (never a kept one)
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_res_partials);
      if (e != cudaSuccess || !p) {
        char b[160];
        snprintf(b, sizeof b, "rlbm_velocity_residual_static: cudaGetSymbolAddress: %s",
                 cudaGetErrorString(e));
        return fail(RLBM_ECUDA, b);
      }
      g_scratch[dev] = static_cast<double*>(p);
    } else if (!g_scratch[dev]) {
      return fail(RLBM_ESTATE,
                  "rlbm_velocity_residual_static: first call on this device inside a stream "
                  "capture; make one call outside capture first");
    }
    scratch = g_scratch[dev];
  }
  const int nblocks = (int)((nsites + kResTile - 1) / kResTile);
  k_res_partial<<<nblocks, kResThreads, 0, st>>>(ux_prev, uy_prev, ux, uy, nsites, scratch);
  k_res_final<<<1, kResThreads, 0, st>>>(scratch, nblocks, residual);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(RLBM_ECUDA, cudaGetErrorString(e));
  return RLBM_OK;
}

// Kernel module for one storage type.  Included once per translation unit
// with RLBM_S (storage type) and RLBM_OPS (accessor name) defined; each unit
// owns its own copy of the quadrature constants in constant memory.
#include "kernels.cuh"
#include "ops.h"

#include <cmath>

namespace rlbm {
namespace {

using S = RLBM_S;
using R = typename Codec<S>::R;

__constant__ QuadConsts<R> c_qc;

// RLBM_STEP_MIN_BLOCKS: resident blocks of 128 threads per SM the register
// allocation aims for (measured per storage type, with the populations parked
// in shared memory and the paired FP32 collision: FP32 storage runs best at
// 6 blocks / 80 registers, 16-bit storage at 7 blocks / 72 registers; the
// FP64 kernels take all the registers they want).
#ifndef RLBM_STEP_MIN_BLOCKS
#define RLBM_STEP_MIN_BLOCKS 4
#endif
// Registers per thread of every step kernel of the module: one cap for all
// block widths (64 / 128 / 256 sites), so that every launch shape compiles the
// per-site arithmetic alike (the code generator's multiply-add contraction
// depends on the register budget) and all shapes give bit-identical states.
constexpr int kStepRegs = (65536 / (RLBM_STEP_MIN_BLOCKS * kBX)) > 255
                              ? 255 : ((65536 / (RLBM_STEP_MIN_BLOCKS * kBX)) & ~7);

// Dynamic shared memory of the direct step kernels: the parking area
// (park_bytes: 12 x threads x 16 B with FP32 arithmetic, none with FP64).
template <int FORCE, int RES>
__global__ void __maxnreg__(kStepRegs) k_step(const S* __restrict__ fin, S* __restrict__ fout,
                                              DevSample s, const R* __restrict__ ghost,
                                              StepAux<R> aux) {
  extern __shared__ __align__(128) unsigned char park_smem[];
  step_body<S, FORCE, RES>(fin, fout, s, ghost, aux, c_qc, park_smem);
}

template <int FORCE, int RES, int BX>
__global__ void __maxnreg__(kStepRegs)
k_step_batch(S* __restrict__ base, BatchArgs b, const R* __restrict__ ghost, StepAux<R> aux) {
  extern __shared__ __align__(128) unsigned char park_smem[];
  batch_body<S, FORCE, RES, BX>(base, b, ghost, aux, c_qc, park_smem);
}

// Staged pulls (persistent; dynamic shared memory: two slot-row buffers).
template <int FORCE, int RES, int BX>
__global__ void __maxnreg__(kStepRegs)
k_step_staged(S* __restrict__ base, BatchArgs b, const R* __restrict__ ghost, StepAux<R> aux) {
  extern __shared__ __align__(128) unsigned char stage_smem[];
  staged_batch_body<S, FORCE, RES, BX>(base, b, ghost, aux, c_qc, stage_smem);
}

// Shared-memory opt-in of the direct batched kernels: the parking area of a
// 256-thread block (12 x 256 x 16 B = 48 KiB with FP32 arithmetic) plus the
// residual reduction's static scratch exceed the default 48 KiB.
template <int BX>
cudaError_t allow_park_smem() {
  const int bytes = (int)park_bytes<R>(BX);
  cudaError_t e = cudaSuccess;
  if (bytes == 0) return e;
  auto set = [&](const void* fn) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  set((const void*)k_step_batch<0, 0, BX>);
  set((const void*)k_step_batch<0, 1, BX>);
  set((const void*)k_step_batch<0, 2, BX>);
  set((const void*)k_step_batch<1, 0, BX>);
  set((const void*)k_step_batch<1, 1, BX>);
  set((const void*)k_step_batch<1, 2, BX>);
  set((const void*)k_step_batch<2, 0, BX>);
  set((const void*)k_step_batch<2, 1, BX>);
  set((const void*)k_step_batch<2, 2, BX>);
  return e;
}

template <int BX>
cudaError_t allow_stage_smem() {
  const int bytes = (int)Stage<S>::template smem_bytes<BX>();
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* fn) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  set((const void*)k_step_staged<0, 0, BX>);
  set((const void*)k_step_staged<0, 1, BX>);
  set((const void*)k_step_staged<0, 2, BX>);
  set((const void*)k_step_staged<1, 0, BX>);
  set((const void*)k_step_staged<1, 1, BX>);
  set((const void*)k_step_staged<1, 2, BX>);
  set((const void*)k_step_staged<2, 0, BX>);
  set((const void*)k_step_staged<2, 1, BX>);
  set((const void*)k_step_staged<2, 2, BX>);
  return e;
}

__global__ void __launch_bounds__(kBX) k_moments(const S* __restrict__ fin, DevSample s,
                                                 const R* __restrict__ ghost, double* n,
                                                 double* ux, double* uy, double* T,
                                                 unsigned* err, R* dn_out) {
  moments_body<S>(fin, s, ghost, n, ux, uy, T, err, c_qc, dn_out);
}

__global__ void __launch_bounds__(kBX) k_init(S* __restrict__ fout, DevSample s, const double* n,
                                              const double* ux, const double* uy,
                                              const double* T, unsigned* err) {
  init_body<S>(fout, s, n, ux, uy, T, err, c_qc);
}

__global__ void __launch_bounds__(kBX) k_init_ce(S* __restrict__ fout, DevSample s,
                                                 const double* n, const double* ux,
                                                 const double* uy, const double* T,
                                                 unsigned* err) {
  init_ce_body<S>(fout, s, n, ux, uy, T, err, c_qc);
}

__global__ void __launch_bounds__(kBX) k_get(const S* __restrict__ fin, DevSample s, int q0,
                                             double* out) {
  get_state_body<S>(fin, s, q0, out, c_qc);
}

__global__ void __launch_bounds__(kBX) k_set(S* __restrict__ fout, DevSample s, int q0,
                                             const double* in) {
  set_state_body<S>(fout, s, q0, in, c_qc);
}

dim3 site_grid(const DevSample& s) { return dim3((s.nx + kBX - 1) / kBX, s.ny, 1); }

cudaError_t upload(const double p0[4], const double w[2][4], double scale) {
  QuadConsts<R> h;
  double K[4] = {0.0, 0.0, 0.0, 0.0};     // K_m = sum_j w_2j p0_j^m
  h.dec_s = R(1.0 / scale);
  h.enc_s = R(scale);
  for (int j = 0; j < kShells; ++j) {
    h.p0[j] = R(p0[j]);
    for (int k = 0; k < 2; ++k) {
      h.w[k][j] = R(w[k][j]);
      h.wd[k][j] = w[k][j];
      h.wp0[k][j] = R(w[k][j] * p0[j] / scale);
      h.wp0sq[k][j] = R(w[k][j] * p0[j] * p0[j] / scale);
    }
    for (int m = 1; m <= 3; ++m) K[m] += w[1][j] * std::pow(p0[j], m);
  }
  // operand pairs of the paired FP32 arithmetic (the values the kernels use)
  for (int q = 0; q < kDirs / 2; ++q) {
    const int d = 2 * q;
    const double vx = hop_x(d) / 5.0, vy = hop_y(d) / 5.0;
    for (int o = 0; o < kOddMonos; ++o)
      h.odd[q][o] = make_float2(float(odd_mono(d, o)), float(-odd_mono(d, o)));
    h.vxy[q] = make_float2(float(vx), float(vy));
    h.vsq[q] = make_float2(float(vx * vx), float(vx * vy));
  }
  for (int k = 0; k < 2; ++k) {
    for (int j = 0; j < kShells; ++j)
      h.wab[k][j] = make_float2(float(w[k][j] * p0[j] / scale),
                                float(w[k][j] * p0[j] * p0[j] / scale));
  }
  h.p01 = make_float2(float(p0[0]), float(p0[1]));
  h.p23 = make_float2(float(p0[2]), float(p0[3]));
  // Conservation projection on the four (5,0)-type directions:
  //   [4K1 4K2; 4K2 4K3] (l0, l1) = -(rN, rE),   2 K3 lx = -rX,  2 K3 ly = -rY.
  const double det = 16.0 * (K[1] * K[3] - K[2] * K[2]);
  h.P00 = R(-4.0 * K[3] / det);
  h.P01 = R(4.0 * K[2] / det);
  h.P10 = R(4.0 * K[2] / det);
  h.P11 = R(-4.0 * K[1] / det);
  h.px = R(-1.0 / (2.0 * K[3]));
  cudaError_t e = cudaMemcpyToSymbol(c_qc, &h, sizeof(h));
  // shared-memory opt-in of the staged kernels (current device)
  if (e == cudaSuccess) e = allow_stage_smem<64>();
  if (e == cudaSuccess) e = allow_stage_smem<128>();
  if (e == cudaSuccess) e = allow_stage_smem<256>();
  if (e == cudaSuccess) e = allow_park_smem<256>();
  return e;
}

template <int F>
void launch_single(const S* a, S* b, const DevSample& s, const R* g, int res, const StepAux<R>& aux,
                   cudaStream_t st) {
  const dim3 grid = site_grid(s);
  const size_t pk = park_bytes<R>(kBX);
  if (res == 0) k_step<F, 0><<<grid, kBX, pk, st>>>(a, b, s, g, aux);
  else if (res == 1) k_step<F, 1><<<grid, kBX, pk, st>>>(a, b, s, g, aux);
  else k_step<F, 2><<<grid, kBX, pk, st>>>(a, b, s, g, aux);
}

cudaError_t step(const void* fin, void* fout, const DevSample& s, const void* ghost, int force,
                 int res, void* uprev, double* acc, unsigned* err, cudaStream_t st) {
  StepAux<R> aux{static_cast<R*>(uprev), acc, err};
  const S* a = static_cast<const S*>(fin);
  S* b = static_cast<S*>(fout);
  const R* g = static_cast<const R*>(ghost);
  if (force == kForceLca) launch_single<kForceLca>(a, b, s, g, res, aux, st);
  else if (force == kForceUniform) launch_single<kForceUniform>(a, b, s, g, res, aux, st);
  else launch_single<kForceNone>(a, b, s, g, res, aux, st);
  return cudaGetLastError();
}

template <int F, int BX>
void launch_batch_f(S* base, const BatchArgs& b, const R* g, int res, int grid, int staged,
                    const StepAux<R>& aux, cudaStream_t st) {
  if (staged == 1) {
    const size_t sm = Stage<S>::template smem_bytes<BX>();
    if (res == 0) k_step_staged<F, 0, BX><<<grid, BX, sm, st>>>(base, b, g, aux);
    else if (res == 1) k_step_staged<F, 1, BX><<<grid, BX, sm, st>>>(base, b, g, aux);
    else k_step_staged<F, 2, BX><<<grid, BX, sm, st>>>(base, b, g, aux);
    return;
  }
  const size_t pk = park_bytes<R>(BX);
  if (res == 0) k_step_batch<F, 0, BX><<<grid, BX, pk, st>>>(base, b, g, aux);
  else if (res == 1) k_step_batch<F, 1, BX><<<grid, BX, pk, st>>>(base, b, g, aux);
  else k_step_batch<F, 2, BX><<<grid, BX, pk, st>>>(base, b, g, aux);
}

template <int BX>
void launch_batch(S* base, const BatchArgs& b, const R* g, int force, int res, int grid,
                  int staged, const StepAux<R>& aux, cudaStream_t st) {
  if (force == kForceLca) launch_batch_f<kForceLca, BX>(base, b, g, res, grid, staged, aux, st);
  else if (force == kForceUniform)
    launch_batch_f<kForceUniform, BX>(base, b, g, res, grid, staged, aux, st);
  else launch_batch_f<kForceNone, BX>(base, b, g, res, grid, staged, aux, st);
}

cudaError_t step_batch(void* base, const BatchArgs& b, const void* ghost, int force, int res,
                       int bx, int grid, int staged, void* uprev, double* acc, unsigned* err,
                       cudaStream_t st) {
  StepAux<R> aux{static_cast<R*>(uprev), acc, err};
  S* p = static_cast<S*>(base);
  const R* g = static_cast<const R*>(ghost);
  if (bx == 64) launch_batch<64>(p, b, g, force, res, grid, staged, aux, st);
  else if (bx == 256) launch_batch<256>(p, b, g, force, res, grid, staged, aux, st);
  else launch_batch<128>(p, b, g, force, res, grid, staged, aux, st);
  return cudaGetLastError();
}

cudaError_t moments(const void* fin, const DevSample& s, const void* ghost, double* n, double* ux,
                    double* uy, double* T, unsigned* err, void* dn_out, cudaStream_t st) {
  k_moments<<<site_grid(s), kBX, 0, st>>>(static_cast<const S*>(fin), s,
                                         static_cast<const R*>(ghost), n, ux, uy, T, err,
                                         static_cast<R*>(dn_out));
  return cudaGetLastError();
}

cudaError_t init(void* fout, const DevSample& s, const double* n, const double* ux,
                 const double* uy, const double* T, unsigned* err, cudaStream_t st) {
  k_init<<<site_grid(s), kBX, 0, st>>>(static_cast<S*>(fout), s, n, ux, uy, T, err);
  return cudaGetLastError();
}

cudaError_t init_ce(void* fout, const DevSample& s, const double* n, const double* ux,
                    const double* uy, const double* T, unsigned* err, cudaStream_t st) {
  k_init_ce<<<site_grid(s), kBX, 0, st>>>(static_cast<S*>(fout), s, n, ux, uy, T, err);
  return cudaGetLastError();
}

cudaError_t get_state(const void* fin, const DevSample& s, int q0, int nq, double* out,
                      cudaStream_t st) {
  dim3 grid = site_grid(s);
  grid.z = nq;
  k_get<<<grid, kBX, 0, st>>>(static_cast<const S*>(fin), s, q0, out);
  return cudaGetLastError();
}

cudaError_t set_state(void* fout, const DevSample& s, int q0, int nq, const double* in,
                      cudaStream_t st) {
  dim3 grid = site_grid(s);
  grid.z = nq;
  k_set<<<grid, kBX, 0, st>>>(static_cast<S*>(fout), s, q0, in);
  return cudaGetLastError();
}

const PrecOps kOps = {
    RLBM_NAME, sizeof(S), sizeof(R), upload, step, step_batch, moments, init, init_ce, get_state,
    set_state, 1,
};

}  // namespace

const PrecOps* RLBM_OPS() { return &kOps; }

}  // namespace rlbm

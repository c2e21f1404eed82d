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

// RLBM_STEP_MIN_BLOCKS: resident blocks per SM the register allocation aims
// for (measured per storage type: FP32 runs best at 4 blocks / 128
// registers, 16-bit storage at 5 blocks).
#ifndef RLBM_STEP_MIN_BLOCKS
#define RLBM_STEP_MIN_BLOCKS 4
#endif

template <bool FORCE, int RES>
__global__ void __launch_bounds__(kBX, RLBM_STEP_MIN_BLOCKS) k_step(const S* __restrict__ fin, S* __restrict__ fout,
                                              DevSample s, const R* __restrict__ ghost,
                                              StepAux<R> aux) {
  step_body<S, FORCE, RES>(fin, fout, s, ghost, aux, c_qc);
}

template <bool FORCE, int RES, int BX>
__global__ void __launch_bounds__(BX, RLBM_STEP_MIN_BLOCKS * kBX / BX)
k_step_batch(S* __restrict__ base, BatchArgs b, const R* __restrict__ ghost, StepAux<R> aux) {
  batch_body<S, FORCE, RES, BX>(base, b, ghost, aux, c_qc);
}

__global__ void __launch_bounds__(kBX) k_moments(const S* __restrict__ fin, DevSample s,
                                                 const R* __restrict__ ghost, double* n,
                                                 double* ux, double* uy, double* T,
                                                 unsigned* err) {
  moments_body<S>(fin, s, ghost, n, ux, uy, T, err, c_qc);
}

__global__ void __launch_bounds__(kBX) k_init(S* __restrict__ fout, DevSample s, const double* n,
                                              const double* ux, const double* uy,
                                              const double* T, unsigned* err) {
  init_body<S>(fout, s, n, ux, uy, T, err, c_qc);
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
  for (int j = 0; j < kShells; ++j) {
    h.p0[j] = R(p0[j]);
    h.p0sq[j] = R(p0[j] * p0[j]);
    for (int k = 0; k < 2; ++k) {
      h.w[k][j] = R(w[k][j]);
      h.dec[k][j] = R(w[k][j] / scale);
      h.enc[k][j] = R(scale / w[k][j]);
    }
    for (int m = 1; m <= 3; ++m) K[m] += w[1][j] * std::pow(p0[j], m);
  }
  // Conservation projection on the four (5,0)-type directions:
  //   [4K1 4K2; 4K2 4K3] (l0, l1) = -(rN, rE),   2 K3 lx = -rX,  2 K3 ly = -rY.
  const double det = 16.0 * (K[1] * K[3] - K[2] * K[2]);
  h.P00 = R(-4.0 * K[3] / det);
  h.P01 = R(4.0 * K[2] / det);
  h.P10 = R(4.0 * K[2] / det);
  h.P11 = R(-4.0 * K[1] / det);
  h.px = R(-1.0 / (2.0 * K[3]));
  return cudaMemcpyToSymbol(c_qc, &h, sizeof(h));
}

cudaError_t step(const void* fin, void* fout, const DevSample& s, const void* ghost, bool force,
                 int res, void* uprev, double* acc, unsigned* err, cudaStream_t st) {
  StepAux<R> aux{static_cast<R*>(uprev), acc, err};
  const S* a = static_cast<const S*>(fin);
  S* b = static_cast<S*>(fout);
  const R* g = static_cast<const R*>(ghost);
  const dim3 grid = site_grid(s);
  if (force) {
    if (res == 0) k_step<true, 0><<<grid, kBX, 0, st>>>(a, b, s, g, aux);
    else if (res == 1) k_step<true, 1><<<grid, kBX, 0, st>>>(a, b, s, g, aux);
    else k_step<true, 2><<<grid, kBX, 0, st>>>(a, b, s, g, aux);
  } else {
    if (res == 0) k_step<false, 0><<<grid, kBX, 0, st>>>(a, b, s, g, aux);
    else if (res == 1) k_step<false, 1><<<grid, kBX, 0, st>>>(a, b, s, g, aux);
    else k_step<false, 2><<<grid, kBX, 0, st>>>(a, b, s, g, aux);
  }
  return cudaGetLastError();
}

template <int BX>
void launch_batch(S* base, const BatchArgs& b, const R* g, bool force, int res, int grid,
                  const StepAux<R>& aux, cudaStream_t st) {
  if (force) {
    if (res == 0) k_step_batch<true, 0, BX><<<grid, BX, 0, st>>>(base, b, g, aux);
    else if (res == 1) k_step_batch<true, 1, BX><<<grid, BX, 0, st>>>(base, b, g, aux);
    else k_step_batch<true, 2, BX><<<grid, BX, 0, st>>>(base, b, g, aux);
  } else {
    if (res == 0) k_step_batch<false, 0, BX><<<grid, BX, 0, st>>>(base, b, g, aux);
    else if (res == 1) k_step_batch<false, 1, BX><<<grid, BX, 0, st>>>(base, b, g, aux);
    else k_step_batch<false, 2, BX><<<grid, BX, 0, st>>>(base, b, g, aux);
  }
}

cudaError_t step_batch(void* base, const BatchArgs& b, const void* ghost, bool force, int res,
                       int bx, int grid, void* uprev, double* acc, unsigned* err,
                       cudaStream_t st) {
  StepAux<R> aux{static_cast<R*>(uprev), acc, err};
  S* p = static_cast<S*>(base);
  const R* g = static_cast<const R*>(ghost);
  if (bx == 64) launch_batch<64>(p, b, g, force, res, grid, aux, st);
  else if (bx == 256) launch_batch<256>(p, b, g, force, res, grid, aux, st);
  else launch_batch<128>(p, b, g, force, res, grid, aux, st);
  return cudaGetLastError();
}

cudaError_t moments(const void* fin, const DevSample& s, const void* ghost, double* n, double* ux,
                    double* uy, double* T, unsigned* err, cudaStream_t st) {
  k_moments<<<site_grid(s), kBX, 0, st>>>(static_cast<const S*>(fin), s,
                                         static_cast<const R*>(ghost), n, ux, uy, T, err);
  return cudaGetLastError();
}

cudaError_t init(void* fout, const DevSample& s, const double* n, const double* ux,
                 const double* uy, const double* T, unsigned* err, cudaStream_t st) {
  k_init<<<site_grid(s), kBX, 0, st>>>(static_cast<S*>(fout), s, n, ux, uy, T, err);
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
    RLBM_NAME, sizeof(S), sizeof(R), upload, step, step_batch, moments, init, get_state,
    set_state, 1,
};

}  // namespace

const PrecOps* RLBM_OPS() { return &kOps; }

}  // namespace rlbm

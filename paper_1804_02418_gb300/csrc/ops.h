// Host-side interface between the C ABI and the per-precision kernel modules.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include "kernels.cuh"

namespace rlbm {

struct PrecOps {
  const char* name;
  size_t elem_bytes;   // bytes per stored population value
  size_t real_bytes;   // bytes of the arithmetic type (residual velocity plane)
  // Uploads the quadrature (p0_j, w_kj) and the 16-bit storage scale s.
  cudaError_t (*upload)(const double p0[4], const double w[2][4], double scale);
  // force: kForceNone / kForceUniform / kForceLca (kernels.cuh)
  cudaError_t (*step)(const void* fin, void* fout, const DevSample& s, const void* ghost,
                      int force, int res, void* uprev, double* acc, unsigned* err,
                      cudaStream_t st);
  // All samples in one launch over the tile list (bx: 64 / 128 / 256 sites per
  // tile and block; grid: number of blocks walking the list; staged: 0 pulls
  // straight from HBM, 1 the tile's row segments staged in shared memory by
  // bulk copies).
  cudaError_t (*step_batch)(void* base, const BatchArgs& b, const void* ghost, int force,
                            int res, int bx, int grid, int staged, void* uprev, double* acc,
                            unsigned* err, cudaStream_t st);
  // (n, u, T) of the streamed populations; dn_out (may be null): n - 1 into a
  // plane of the arithmetic type (the electric force's density)
  cudaError_t (*moments)(const void* fin, const DevSample& s, const void* ghost, double* n,
                         double* ux, double* uy, double* T, unsigned* err, void* dn_out,
                         cudaStream_t st);
  cudaError_t (*init)(void* fout, const DevSample& s, const double* n, const double* ux,
                      const double* uy, const double* T, unsigned* err, cudaStream_t st);
  // the Chapman-Enskog seed of the fields (kernels.cuh: init_ce_body)
  cudaError_t (*init_ce)(void* fout, const DevSample& s, const double* n, const double* ux,
                         const double* uy, const double* T, unsigned* err, cudaStream_t st);
  // planes q0 .. q0+nq-1 <-> dense FP64 [nq][ny][nx]
  cudaError_t (*get_state)(const void* fin, const DevSample& s, int q0, int nq, double* out,
                           cudaStream_t st);
  cudaError_t (*set_state)(void* fout, const DevSample& s, int q0, int nq, const double* in,
                           cudaStream_t st);
  int launches_per_step;
};

const PrecOps* ops_f64();
const PrecOps* ops_f32();
const PrecOps* ops_f16();
const PrecOps* ops_bf16();

bool refine_quadrature(double w1[4], double w2[4], double p0[4]);

}  // namespace rlbm

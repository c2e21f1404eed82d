/*
 * rlbm_massive.h - C ABI of the massive-particle variant of the relativistic
 * lattice Boltzmann method (Gabbana, Mendoza, Succi, Tripiccione,
 * arXiv:1804.02418, Sec. 2.3): particles of rest mass m = 5 T0 on the
 * 45-vector stencil of Fig. m5-stencil
 *     G = {(0,0), (1,0)_FS, (1,1)_FS, (2,0)_FS, (2,1)_FS, (2,2)_FS, (3,0)_FS,
 *          (3,2)_FS, (3,3)_FS, (4,0)_FS}   (FS: all signs and component swaps),
 * discrete momenta p_i = p0_i (1, v0 n_i), p0_i = m / sqrt(1 - v0^2 |n_i|^2)
 * (Eq. discrete-quadri-momentum, Eq. discrete-p0), weights making Eq.
 * orthonormal exact up to third order against the rest Maxwell-Juttner
 * distribution at T0 = 1.  One time step per site (Eq. discrete-rbe): pull
 * streaming f_i(x, t+1) = f*_i(x - n_i, t); moments N^a, T^ab; Landau frame
 * eps U^a = T^ab U_b, n = U_a N^a, T from the 2-D massive ideal gas
 *     eps = n (m^2 + 2 m T + 2 T^2) / (m + T),   P = n T;
 * equilibrium f^eq_i = w_i sum_k a^(k) J^(k)(p_i) (Eq. feq-expansion-discrete,
 * projection of the Maxwell-Juttner distribution on the polynomials of degree
 * <= 3); Anderson-Witting relaxation with omega_i = p_i.U / (p0_i tau); a
 * uniform force F per particle,
 *     F_i^ext = w_i [ (F.v_i) P(p_i) - F.grad_p P(p_i) ],  P = f^eq / omega
 * (grad_p along the mass shell); on-site bounce-back walls.
 *
 * v0 (Sec. 2.3 leaves it free): the weights are non-negative only on one
 * interval of v0 of width about 1.4e-5 near 0.2211; the library takes its
 * midpoint (rlbm_massive_quadrature reports it).
 *
 * Units: dt = 1, T0 = 1 (so m = 5), one site is v0 length units (c = 1 is
 * 1 / v0 sites per step); population i moves n_i sites per step.
 *
 * Population order (the state layout): 22 pairs of opposite vectors, pair p
 * holding populations 2p and 2p + 1 = the opposite vector; class by class in
 * the order (1,0) (1,1) (2,0) (2,1) (2,2) (3,0) (3,2) (3,3) (4,0); within a
 * class (a,0): (a,0) (-a,0) (0,a) (0,-a); (a,a): (a,a) (-a,-a) (-a,a) (a,-a);
 * (a,b): (a,b) (-a,-b) (-a,b) (a,-b) (b,a) (-b,-a) (-b,a) (b,-a); the rest
 * vector (0,0) is population 44.
 *
 * Fields exchanged with the caller are FP64, row-major [ny][nx], dense.
 * Pointers are host pointers when device_ptrs == 0 and device pointers on
 * the context's device otherwise; the caller owns them.  Return values and
 * error codes are those of rlbm.h (RLBM_OK or a negative RLBM_E* code);
 * rlbm_massive_last_error() then holds a message.  All device work runs on
 * the stream of the config; calls returning host data synchronise it.
 */
#ifndef RLBM_MASSIVE_H
#define RLBM_MASSIVE_H

#include "rlbm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RLBM_MASSIVE_Q 45
#define RLBM_MASSIVE_MASS 5

typedef struct {
  int nx, ny;                   /* 5 .. 131072 each */
  int periodic_x, periodic_y;   /* 1: periodic axis, 0: bounce-back walls at both ends */
  double tau;                   /* relaxation time, > 0.5 */
  double Fx, Fy;                /* uniform force per particle, |F| < 1e-2 */
  rlbm_prec prec;               /* RLBM_F64 or RLBM_F32 (storage = arithmetic) */
  void* stream;                 /* cudaStream_t, or NULL for the default stream */
} rlbm_massive_config;

typedef struct rlbm_massive_ctx rlbm_massive_ctx;

/* The quadrature the library uses (host only, no GPU): *v0, the interval
 * [window[0], window[1]] of v0 where every weight is non-negative, the class
 * weights w[10] and energies p0[10] in the class order above followed by the
 * rest class (0,0).  Any pointer may be NULL. */
int rlbm_massive_quadrature(double* v0, double window[2], double w[10], double p0[10]);

/* The stencil vectors n_i (x, y) of the 45 populations (host only). */
int rlbm_massive_stencil(int vx[45], int vy[45]);

/* Validates the config, uploads the tables (first call computes them, about
 * 0.5 s) and allocates two population buffers of 45 planes (FP64: 720 B,
 * FP32: 360 B per site in all).  On failure *out is NULL. */
int rlbm_massive_create(const rlbm_massive_config* cfg, rlbm_massive_ctx** out);

/* Stored (post-collision) state := f^eq of the given fields; all four NULL
 * means the rest state n = T = 1, u = 0.  |u| < 1, n, T > 0. */
int rlbm_massive_init(rlbm_massive_ctx* ctx, const double* n, const double* ux,
                      const double* uy, const double* T, int device_ptrs);

/* Advances by nsteps >= 0 time steps (one kernel launch each; asynchronous
 * when residual is NULL).  With residual != NULL (nsteps >= 1) the velocity
 * field before and after the last step (Landau frame of the streamed
 * populations, as rlbm_massive_moments) gives
 *     *residual = ||u(t) - u(t-1)||_2 / ||u(t)||_2   over all sites
 * (0 if both norms vanish, +inf if only ||u(t)|| does); the stream is then
 * synchronised and the error word checked (RLBM_ENAN).  The residual uses
 * 4 FP64 planes of context scratch, allocated on first use. */
int rlbm_massive_step(rlbm_massive_ctx* ctx, int nsteps, double* residual);

/* Landau-frame n, ux, uy, T of the streamed populations (the fields the next
 * collision uses).  Any output may be NULL. */
int rlbm_massive_moments(rlbm_massive_ctx* ctx, double* n, double* ux, double* uy,
                         double* T, int device_ptrs);

/* State as deviations f_i - f0_i from the rest populations f0_i = w_i / (m + 1),
 * layout [45][ny][nx] FP64.  The library stores relative deviations
 * (f_i - f0_i) / f0_i and converts in FP64. */
int rlbm_massive_get_state(rlbm_massive_ctx* ctx, double* delta, int device_ptrs);
int rlbm_massive_set_state(rlbm_massive_ctx* ctx, const double* delta, int device_ptrs);

/* Synchronises the stream; RLBM_ENAN if a step met a non-finite or
 * unphysical site (|u| >= 1, n <= 0, T <= 0) or an unconverged Landau solve
 * since the last check (the flag is then cleared). */
int rlbm_massive_check(rlbm_massive_ctx* ctx);

long long rlbm_massive_steps_done(const rlbm_massive_ctx* ctx);
long long rlbm_massive_launch_count(const rlbm_massive_ctx* ctx);

/* Frees the context (NULL: no-op). */
void rlbm_massive_destroy(rlbm_massive_ctx* ctx);

/* Message of the last failed call on ctx, or of the last failed call without
 * a context when ctx is NULL. */
const char* rlbm_massive_last_error(const rlbm_massive_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* RLBM_MASSIVE_H */

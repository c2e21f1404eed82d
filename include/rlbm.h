/*
 * rlbm.h - C ABI of the GB300 relativistic lattice Boltzmann library.
 *
 * The library advances the (2+1)-dimensional relativistic lattice Boltzmann
 * method for a massless fluid of Gabbana, Mendoza, Succi and Tripiccione
 * (arXiv:1804.02418) on one GPU:
 *   - discrete relativistic BGK update, Eq. discrete-rbe (Sec. 2.2):
 *       f_i(x + v_i dt, t + dt) - f_i(x, t)
 *         = -dt (p_i^m U_m / (p_i^0 tau)) (f_i - f_i^eq) + F_i^ext ;
 *   - per-site algorithm (end of Sec. 2): moments N^a, T^ab; Landau frame
 *     eps U^a = T^ab U_b; n = U_a N^a; massless equation of state
 *     eps = 2 n T; equilibrium f_i^eq = w_i (n/T) sum_k a^(k) J^(k)(p_i)
 *     (Eq. feq-expansion-discrete, App. A-B); forcing term (Sec. 2.4);
 *   - the 48-population stencil G = {(+-3,+-4)_FS, (+-5,0)_FS} with four
 *     energy shells (Sec. 2.3), weights refined onto Eq. orthonormal;
 *   - bounce-back walls and non-evolving injector / collector contacts
 *     (Sec. 3, Fig. geom caption).
 *
 * Units: dt = 1, one hop is 5 sites (c = 5 sites per step), a force is the
 * momentum given to one particle per step.
 *
 * Population index i = 4 d + j (direction d = 0..11, shell j = 0..3) with
 * directions (3,4) (-3,-4) (-3,4) (3,-4) (4,3) (-4,-3) (-4,3) (4,-3)
 * (5,0) (-5,0) (0,5) (0,-5); the opposite of direction d is d ^ 1.
 *
 * Fields exchanged with the caller are FP64, row-major [ny][nx] (x fastest),
 * dense (row stride nx).  Pointers are host pointers when device_ptrs == 0
 * and device pointers on the context's device when device_ptrs != 0.  The
 * caller owns every array it passes; the context owns (or borrows, see
 * rlbm_config.workspace) the population buffers.
 *
 * Errors: every int-returning call returns RLBM_OK (0) or a negative code;
 * rlbm_last_error() then holds a message.  A context is not thread-safe;
 * distinct contexts are independent.  All device work is issued on the
 * stream given in rlbm_config (default stream if NULL).  Calls that return
 * data to host memory synchronise that stream.
 */
#ifndef RLBM_H
#define RLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RLBM_Q 48
#define RLBM_MAX_CONTACTS 4
#define RLBM_HOP_RADIUS 5

enum {
  RLBM_OK = 0,
  RLBM_EINVAL = -1,    /* bad argument: dims < 11, tau <= 0.5, |F| >= 1e-2, bad contact, ... */
  RLBM_ENOMEM = -2,    /* device allocation failed or workspace too small */
  RLBM_ECUDA = -3,     /* a CUDA runtime call failed */
  RLBM_ENAN = -4,      /* device error word set: non-finite field, |u| >= 1 or
                          no convergence of the Landau solve */
  RLBM_ETIMEOUT = -5,  /* a bounded device wait gave up */
  RLBM_ESTATE = -6     /* call out of order (e.g. step before init) */
};

/* Storage / arithmetic precision of the populations.
 * RLBM_F64:    FP64 storage of f_i - w_i, FP64 arithmetic.
 * RLBM_F32:    FP32 storage of f_i - w_i, FP32 arithmetic.
 * RLBM_F16DEV: FP16 storage of the scaled relative deviation
 *              g_i = s (f_i - w_i) / w_i, FP32 arithmetic.
 * RLBM_BF16DEV: as RLBM_F16DEV with BF16 storage. */
typedef enum { RLBM_F64 = 0, RLBM_F32 = 1, RLBM_F16DEV = 2, RLBM_BF16DEV = 3 } rlbm_prec;

/* A contact (Sec. 3): `length` sites of edge `edge` starting at `x0`
 * (edge 0: y = 0, 1: y = ny-1, 2: x = 0, 3: x = nx-1; x0 runs along x for
 * edges 0/1 and along y for edges 2/3).  It is a ghost strip 5 sites deep
 * outside that edge whose populations stay at the equilibrium of
 * (n, u_n * inward normal, T).  A pull whose source lies in the strip reads
 * that value; every other pull from outside the rectangle bounces back. */
typedef struct {
  int edge;
  int x0;
  int length;
  double u_n;
  double n;
  double T;
} rlbm_contact;

/* One sample: an nx x ny rectangle, periodic or walled per axis, relaxation
 * time tau (> 0.5), uniform body force (Fx, Fy) per particle, contacts, and
 * the electric force of the local capacitance approximation (Sec. 3, Eq. lca:
 * phi = -e n / C_g): inv_cg = e^2 / C_g in lattice units (e = 1), 0 for none
 * (C_g infinite).  With inv_cg > 0 every site adds
 *     F_E = -inv_cg grad n
 * to (Fx, Fy), the gradient taken from the previous time step's density over
 * one hop (5 sites, the length unit of c = 1): (n(x+5) - n(x-5)) / 2, forward
 * or backward over 5 sites next to a walled edge, wrapped on periodic axes;
 * the first step uses the density given to rlbm_init.  0 <= inv_cg < 1e3;
 * the explicit force is stable up to about inv_cg = 0.3 at tau = 0.8
 * (measured; the paper's C_g = 10 is 0.1). */
typedef struct {
  int nx, ny;
  int periodic_x, periodic_y;
  double tau;
  double Fx, Fy;
  int ncontacts;
  rlbm_contact contacts[RLBM_MAX_CONTACTS];
  double inv_cg;
} rlbm_sample;

typedef struct {
  rlbm_prec prec;
  int nsamples;                 /* >= 1; all samples advance together */
  const rlbm_sample* samples;   /* array of nsamples, copied by rlbm_create */
  void* stream;                 /* cudaStream_t, or NULL for the default stream */
  void* workspace;              /* optional device buffer of >= rlbm_workspace_size()
                                   bytes, 256-byte aligned, borrowed (not freed);
                                   NULL: the context allocates its own */
  size_t workspace_bytes;
  int graph_steps;              /* > 0 (even): rlbm_step replays CUDA graphs of this many
                                   steps, captured on first use; needs a non-NULL
                                   stream.  0: plain launches */
  const char* tune_cache;       /* optional JSON file where rlbm_autotune keeps its choices
                                   (one entry per GPU / precision / workload), or NULL */
} rlbm_config;

typedef struct rlbm_ctx rlbm_ctx;

/* Bytes of device memory a context needs for cfg (populations: two buffers of
 * 48 planes per sample; plus residual and staging scratch).  Host only. */
int rlbm_workspace_size(const rlbm_config* cfg, size_t* bytes);

/* Validates cfg, derives the refined quadrature, uploads constants and binds
 * or allocates the workspace.  The populations are undefined until
 * rlbm_init / rlbm_set_state.  On failure *out is NULL. */
int rlbm_create(const rlbm_config* cfg, rlbm_ctx** out);

/* Sets the stored (post-collision) state of `sample` to f^eq of the given
 * fields (Eq. feq-expansion-discrete).  NULL field pointers mean the rest
 * state n = T = 1, u = 0 (all four must then be NULL).  |u| < 1, n, T > 0. */
int rlbm_init(rlbm_ctx* ctx, int sample, const double* n, const double* ux,
              const double* uy, const double* T, int device_ptrs);

/* Sets the stored state of `sample` to the Chapman-Enskog seed of the given
 * fields: the state whose first pull-stream yields, at every site x and
 * population i whose source x - n_i lies in the sample (or wraps on a
 * periodic axis), the equilibrium plus its first-order non-equilibrium part
 * of a steady flow,
 *     f_i(x) = f^eq_i(x) - (f^eq_i(x) - f^eq_i(x - n_i)) / omega_i(x),
 *     omega_i = gamma (1 - v_i.u) / tau,
 * i.e. Eq. discrete-rbe in steady state with f - f^eq small and slowly
 * varying (the paper states no seed; this is the library's reading).  The
 * stored value of population i at site s is f^eq_i(d) - (f^eq_i(d) -
 * f^eq_i(s)) / omega_i(d), d = s + n_i, or f^eq_i(s) where d is outside the
 * sample.  Its non-equilibrium shear stress is the first-order (Navier-
 * Stokes) stress of the relaxation-time model, eta = (3/4) n T tau.  Same
 * arguments, layout and checks as rlbm_init (NULL fields: the rest state);
 * with the electric force on, the first step's density is n. */
int rlbm_init_ce(rlbm_ctx* ctx, int sample, const double* n, const double* ux,
                 const double* uy, const double* T, int device_ptrs);

/* Advances every sample by nsteps >= 0 time steps (stream, then collide).
 * If residual != NULL, the last two steps also reduce
 *   r = ||u(t) - u(t-1)||_2 / ||u(t)||_2   over all sites of all samples
 * (u from the streamed populations of those steps), the stream is
 * synchronised, *residual is written and the device error word is checked
 * (RLBM_ENAN).  Needs nsteps >= 2 in that case.  Without residual the call
 * is asynchronous and checks nothing; use rlbm_check. */
int rlbm_step(rlbm_ctx* ctx, int nsteps, double* residual);

/* Residual of every sample, r_k = ||u_k(t) - u_k(t-1)|| / ||u_k(t)||, from the
 * last rlbm_step call that asked for a residual (out holds nsamples values). */
int rlbm_sample_residuals(const rlbm_ctx* ctx, double* out);

/* Chooses the launch shape of the step kernel by timing the candidates on
 * the current state (without advancing it): sites per block (64 / 128 / 256),
 * the number of blocks walking the work list of all samples (one per tile, or
 * 1..16 per SM, persistent) and whether the pulls are staged in shared memory
 * (0 none; 1 bulk asynchronous copies of the 12 shifted row segments of a
 * tile, the next tile in flight while the current one is computed).  With
 * rlbm_config.tune_cache the choice is read from / added to that file
 * (a JSON object {"<key>": {"bx": B, "grid": G, "staged": S}, ...}, the key
 * naming the GPU, the precision and the batch's geometry).  Needs an initialised state.  Writes the
 * choice to *bx, *grid and *staged (each may be NULL).  The staged kernels
 * bound every wait (about 1 s); a wait that gives up raises the error bit
 * that rlbm_check reports as RLBM_ETIMEOUT. */
int rlbm_autotune(rlbm_ctx* ctx, int* bx, int* grid, int* staged);

/* Sets the launch shape directly (same meaning as the rlbm_autotune outputs):
 * bx 0 (single-sample kernel, one launch per sample; grid and staged must be
 * 0) or 64 / 128 / 256 with grid >= 0 (0: one block per tile) and staged
 * 0 (pulls straight from HBM) or 1 (the 12 row segments of a tile staged in
 * shared memory by bulk asynchronous copies, next tile in flight).
 * RLBM_EINVAL for any other combination.
 * Every shape runs the same per-site arithmetic (results agree to the last
 * bits; the code generator may contract multiply-adds differently per kernel). */
int rlbm_set_launch_shape(rlbm_ctx* ctx, int bx, int grid, int staged);

/* Failure detection: the longest a bounded device wait of this context may
 * take, in GPU clock cycles (0, the default, means about one second).  It
 * applies to the staged-pull kernel's waits for a tile's bulk copies; a wait
 * that gives up sets the device error word's timeout bit (rlbm_check then
 * returns RLBM_ETIMEOUT), the block still waits, bounded by the default, for
 * the copies it has issued, and leaves the step incomplete: the state must be
 * set again (rlbm_init / rlbm_set_state) before stepping on.  cycles >= 0. */
int rlbm_set_wait_limit(rlbm_ctx* ctx, long long cycles);

/* Macroscopic fields (n, u_x, u_y, T) of `sample` at the current time: the
 * Landau-frame values of the streamed populations, i.e. those the next
 * collision uses.  Any output pointer may be NULL. */
int rlbm_moments(rlbm_ctx* ctx, int sample, double* n, double* ux, double* uy,
                 double* T, int device_ptrs);

/* Stored post-collision state of `sample` as deviations f_i - w_i, layout
 * [48][ny][nx] FP64 (checkpoint / restart and one-step checks).  The library
 * stores relative deviations (f_i - w_i) / w_i and converts in FP64: a
 * get / set round trip is exact for FP32 and 16-bit storage and within one
 * ulp for FP64 storage.  With the
 * electric force on, rlbm_set_state also sets the density the next step's
 * force uses, to the density of the restored state (the previous step's
 * density is not part of the checkpoint). */
int rlbm_get_state(rlbm_ctx* ctx, int sample, double* delta, int device_ptrs);
int rlbm_set_state(rlbm_ctx* ctx, int sample, const double* delta, int device_ptrs);

/* Raw stored values of rows y0 .. y0 + nrows - 1 of `sample`'s current state,
 * for exchanging the halo rows of a domain cut into slabs of rows (one
 * context per slab; halo rows hold a neighbour's rows).  The buffer `dev`
 * (device memory of the context's device, caller-owned) holds 12 direction
 * planes one after another, each nrows x ldx sites x 4 shells in the storage
 * type (ldx = nx rounded up to a multiple of 32); its size is
 * rlbm_rows_raw_bytes(ctx, sample, nrows).  A get from one context and a set
 * into another context of the same precision and nx moves the values bit for
 * bit.  Asynchronous on the context's stream; RLBM_EINVAL for rows outside
 * the sample.  (No counterpart in the paper: domain decomposition.) */
int rlbm_rows_raw_bytes(const rlbm_ctx* ctx, int sample, int nrows, size_t* bytes);
int rlbm_get_rows_raw(rlbm_ctx* ctx, int sample, int y0, int nrows, void* dev);
int rlbm_set_rows_raw(rlbm_ctx* ctx, int sample, int y0, int nrows, const void* dev);

/* Synchronises the stream and returns RLBM_ENAN if any kernel since the last
 * check flagged a non-finite or unphysical site (then clears the flag). */
int rlbm_check(rlbm_ctx* ctx);

/* Number of time steps taken since the last rlbm_init / rlbm_set_state. */
long long rlbm_steps_done(const rlbm_ctx* ctx);

/* Frees what the context allocated.  NULL is a no-op. */
void rlbm_destroy(rlbm_ctx* ctx);

/* Last error message of ctx (or of the last failed rlbm_create if ctx is
 * NULL).  Valid until the next call on ctx. */
const char* rlbm_last_error(const rlbm_ctx* ctx);

/* The refined quadrature the library uses: w1[j] for the (3,4)-type
 * directions, w2[j] for the (5,0)-type, p0[j] the shell energies (Sec. 2.3,
 * printed values moved onto the exact solutions of Eq. orthonormal by
 * minimum-norm Gauss-Newton steps).  Host only; needs no GPU. */
int rlbm_quadrature(double w1[4], double w2[4], double p0[4]);

/* Kernel launches issued by this context so far (all kinds). */
long long rlbm_launch_count(const rlbm_ctx* ctx);

int rlbm_version(void);

/* Measurement utility (no counterpart in the paper): the rate at which the
 * current device retires fused multiply-adds of one type, FP64 (fp64 != 0)
 * or FP32, from a kernel of independent FMA chains on every SM (best of three
 * timed launches, CUDA events, a few milliseconds each).  *fma_per_s receives
 * thread-level FMA instructions per second (flops / 2).  It is the peak the
 * FP64 step, which is bound by its FP64 instructions, is compared with.
 * Allocates a small output buffer and a stream; changes no device setting. */
int rlbm_fma_peak(int fp64, double* fma_per_s);

/* Convergence residual that allocates nothing (no counterpart in the paper).
 *
 * For callers that cannot allocate device memory when they check convergence
 * (another framework owns the whole memory pool, a real-time loop with a
 * memory budget fixed at start-up, a host callback where cudaMalloc is not
 * allowed).  Computes on `stream`
 *     *residual = ||u - u_prev||_2 / ||u||_2   (0 if both norms are 0,
 *                                              +inf if only ||u|| is 0)
 * over nsites sites from four caller-owned FP64 device arrays of nsites
 * values (ux_prev, uy_prev, ux, uy) into one caller-owned device double.
 * Scratch is a fixed 64 KiB array inside the library (one partial-sum pair
 * per 2048 sites); nsites must be 1 .. 8,388,608, larger sizes return
 * RLBM_EINVAL with a message in rlbm_last_error(NULL).  Calls no
 * cudaMalloc, cudaFree or allocating library routine.  Every call made
 * outside a stream capture looks the scratch address up in the context
 * current at that moment (cudaGetSymbolAddress); a call inside a capture
 * reuses the address the last uncaptured call on the same device found, so
 * make one call outside capture before capturing, and again after
 * cudaDeviceReset or a switch to another context on that device (a first
 * call inside a capture returns RLBM_ESTATE).  All calls share the scratch:
 * calls that overlap on the GPU race and must be serialised by the caller.
 * The result is the same quantity rlbm_step reports, summed in a fixed
 * order. */
int rlbm_velocity_residual_static(const double* ux_prev, const double* uy_prev,
                                  const double* ux, const double* uy, long long nsites,
                                  double* residual, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RLBM_H */

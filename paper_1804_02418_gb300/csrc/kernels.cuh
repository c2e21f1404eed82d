// Kernels of the fused relativistic LBM step, templated on the storage type.
//
// Stored values are relative deviations g = (f - w) / w from the rest weights
// (times s in 16-bit storage, where the kernels also compute on s g).
//
// Layout in HBM (per sample): two ping-pong buffers, each 12 direction planes
// of `plane` sites (row-major, row pitch ldx a multiple of 32, plane a
// multiple of 64 sites).  A site of direction plane d holds the four shells of
// direction d side by side:
//     element (d, site, j) = buffer[(d * plane + site) * 4 + j].
// The four shells share their pull offset n_d, so one aligned vector access
// moves them (the shift by n_d keeps the 16 / 32 / 8-byte alignment because
// it moves by whole sites).
//
// One thread updates one site.  Pull scheme: the thread gathers the 12 vectors
// arriving at its site (each warp reads 32 consecutive sites of a shifted row:
// coalesced), applies the boundary rules, collides in registers and writes 12
// vectors of its own site into the other buffer.
#pragma once
#include <type_traits>

#include "site.cuh"

namespace rlbm {

constexpr int kBX = 128;   // threads per block along x; one block row per y

// FORCE template argument of the step kernels: no force, a uniform force per
// particle, or a uniform force plus the electric force of the local
// capacitance approximation (its own instantiation, so that the others do not
// carry its registers).
constexpr int kForceNone = 0, kForceUniform = 1, kForceLca = 2;

template <typename R>
struct StepAux {
  R* uprev;              // [sites] x 2 velocity plane for the residual (or null)
  double* acc;           // [2] residual accumulators (sum |du|^2, sum |u|^2)
  unsigned* err;         // device error word
};

__device__ __forceinline__ long long vec_index(const DevSample& s, int d, long long site) {
  return ((long long)d * s.plane + site) * 4;
}

// Index of the contact whose ghost strip holds the (outside) source (sx, sy).
__device__ __forceinline__ int contact_of(const DevSample& s, int sx, int sy) {
#pragma unroll
  for (int k = 0; k < kMaxContacts; ++k) {
    if (k >= s.ncontacts) break;
    const int e = s.cedge[k];
    const int t = (e < 2) ? sx : sy;
    const bool side = e == 0 ? (sy < 0) : e == 1 ? (sy >= s.ny) : e == 2 ? (sx < 0) : (sx >= s.nx);
    if (side && t >= s.clo[k] && t < s.chi[k]) return k;
  }
  return -1;
}

// Gathers the 48 streamed deviations arriving at (x, y).
template <typename S, bool INTERIOR, class C>
__device__ __forceinline__ void pull(const S* __restrict__ fin, const DevSample& s, int x, int y,
                                     const typename Codec<S>::R* __restrict__ ghost, const C& qc,
                                     typename Codec<S>::R (&f)[kQ]) {
  const long long site = (long long)y * s.ldx + x;
#pragma unroll
  for (int d = 0; d < kDirs; ++d) {
    const int dx = hop_x(d), dy = hop_y(d);
    if (INTERIOR) {
      Codec<S>::load4(fin + vec_index(s, d, site - ((long long)dy * s.ldx + dx)), dir_kind(d),
                      qc, &f[4 * d]);
    } else {
      int sx = x - dx, sy = y - dy;
      if (s.periodic_x) sx = sx < 0 ? sx + s.nx : (sx >= s.nx ? sx - s.nx : sx);
      if (s.periodic_y) sy = sy < 0 ? sy + s.ny : (sy >= s.ny ? sy - s.ny : sy);
      const bool inside = (unsigned)sx < (unsigned)s.nx && (unsigned)sy < (unsigned)s.ny;
      if (inside) {
        Codec<S>::load4(fin + vec_index(s, d, (long long)sy * s.ldx + sx), dir_kind(d), qc,
                        &f[4 * d]);
      } else {
        const int owner = contact_of(s, sx, sy);
        if (owner >= 0) {
#pragma unroll
          for (int j = 0; j < kShells; ++j) f[4 * d + j] = ghost[owner * kQ + 4 * d + j];
        } else {
          // bounce-back: post-collision population of the opposite direction, same shell
          Codec<S>::load4(fin + vec_index(s, d ^ 1, site), dir_kind(d), qc, &f[4 * d]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Shared-memory staging of the pull.  For one tile (a row segment of BX sites
// starting at x0 in row y) the 12 arriving populations come from 12 row
// segments, one per direction plane: plane d, row y - dy_d, columns
// x0 - dx_d .. x0 - dx_d + BX - 1.  Each segment is contiguous in HBM (whole
// site vectors), so the persistent batched kernel moves it with one bulk
// asynchronous copy (cp.async.bulk, completion counted in bytes on an
// mbarrier) into a shared-memory slot row while the block still computes the
// previous tile.  Columns outside the sample are clipped (their sites take the
// boundary rules, as in pull()); a segment that wraps around a periodic x edge
// is not staged and read directly.  Copies move whole 16-byte granules:
// 16-bit storage (8-byte vectors) rounds a segment out to even sites, and the
// slot index of column c is c - (a & ~(G - 1)), a = x0 - dx_d, G sites per
// granule.
// ---------------------------------------------------------------------------
// Parking of the gathered populations (FP32 arithmetic).  After the moments
// are formed, the 48 values of a site leave the registers for a shared-memory
// area laid out [direction][thread] (16 bytes per entry: conflict-free) and
// come back one direction pair at a time for the relaxation.  This frees
// about 40 registers per thread, so more warps are resident to hide the
// latency of the long per-site arithmetic.  The accesses are volatile so that
// the compiler cannot keep the register copies alive instead.
template <typename R> struct Park { static constexpr bool kOn = false; };
template <> struct Park<float> { static constexpr bool kOn = true; };

// Bytes of the parking area of a block of `threads` threads.
template <typename R>
__host__ __device__ constexpr size_t park_bytes(int threads) {
  return Park<R>::kOn ? (size_t)kDirs * threads * 16 : 0;
}

__device__ __forceinline__ void park_store(uint32_t a, const float* v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n"
               :: "r"(a), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]) : "memory");
}
__device__ __forceinline__ void park_load(uint32_t a, float* v) {
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "r"(a) : "memory");
}

// Control block after the two buffers: full[2] (mbarriers, 8 B each),
// released[2] (+ pad), tiles[2] (int4), masks[2], abort flag (+ pad).
constexpr size_t kStageCtlBytes = 16 + 16 + 32 + 8 + 8;

template <typename S>
struct Stage {
  static constexpr int kVecBytes = 4 * (int)sizeof(S);
  static constexpr int kG = kVecBytes >= 16 ? 1 : 16 / kVecBytes;   // sites per granule
  template <int BX> __host__ __device__ static constexpr int slots() { return BX + 2 * (kG - 1); }
  // elements of one buffer (12 slot rows)
  template <int BX> __host__ __device__ static constexpr int buf_elems() { return kDirs * slots<BX>() * 4; }
  // dynamic shared memory of the kernel: two buffers, then the control block
  template <int BX> __host__ __device__ static constexpr size_t smem_bytes() {
    return 2 * (size_t)buf_elems<BX>() * sizeof(S) + kStageCtlBytes +
           park_bytes<typename Codec<S>::R>(BX);
  }
};

constexpr long long kStageSpinCycles = 2000000000LL;   // about 1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}


__device__ __forceinline__ void stage_bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(bar), "r"(count) : "memory");
}


// Bounded wait for the completion of the phase with the given parity: gives
// up (false) once more than `limit` clock cycles have passed.  The first probe
// does not block (test_wait), so a limit shorter than a copy's latency gives up
// at once; later probes may suspend the thread for a while (try_wait).
__device__ __forceinline__ bool stage_wait(uint32_t bar, uint32_t parity,
                                           long long limit = kStageSpinCycles) {
  const long long t0 = clock64();
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  while (!ok) {
    if (clock64() - t0 > limit) return false;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  }
  return true;
}

// Issued by the 32 lanes of one warp (lane d < 12 copies direction d): the
// segments of tile (x0, y) of sample s into `buf`; *mask gets bit d for every
// staged direction and *tile the tile (sample, x0, y).  One arrive with the
// expected byte count (release semantics: mask and tile become visible to the
// waiting threads) completes the phase together with the copies.
template <typename S, int BX>
__device__ __forceinline__ void stage_issue(const S* __restrict__ fin, const DevSample& s, int x0,
                                            int y, S* buf, uint32_t bar, unsigned* mask,
                                            int4* tile, int sample) {
  constexpr int G = Stage<S>::kG, VB = Stage<S>::kVecBytes, SL = Stage<S>::template slots<BX>();
  const int lane = threadIdx.x & 31;
  const int nv = min(BX, s.nx - x0);
  bool ok = false;
  uint32_t bytes = 0, dst = 0;
  const S* src = nullptr;
  if (lane < kDirs) {
    const int d = lane, dx = hop_x(d), dy = hop_y(d);
    int sy = y - dy;
    if (s.periodic_y) sy = sy < 0 ? sy + s.ny : (sy >= s.ny ? sy - s.ny : sy);
    if ((unsigned)sy < (unsigned)s.ny) {
      const int a = x0 - dx;
      int lo = a, hi = a + nv;
      const bool wraps = s.periodic_x && (lo < 0 || hi > s.nx);
      if (!s.periodic_x) { lo = max(lo, 0); hi = min(hi, s.nx); }
      if (!wraps && lo < hi) {
        const int lor = lo & ~(G - 1), hir = (hi + G - 1) & ~(G - 1);
        ok = true;
        bytes = (uint32_t)(hir - lor) * VB;
        src = fin + vec_index(s, d, (long long)sy * s.ldx + lor);
        dst = smem_addr(buf + ((long long)d * SL + (lor - (a & ~(G - 1)))) * 4);
      }
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, ok);
  uint32_t total = bytes;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
  if (lane == 0) {
    *mask = m;
    *tile = make_int4(sample, x0, y, 0);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                 :: "r"(bar), "r"(total) : "memory");
  }
  __syncwarp();
  if (ok)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
        :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Where the 48 arriving deviations of a site come from: straight from HBM, or
// from the staged slot rows of its tile.
struct DirectSrc {};
template <typename S, int BX>
struct StagedSrc {
  uint32_t buf;     // shared-window address of the tile's slot rows
  unsigned mask;    // bit d: direction d staged
  int x0;           // first column of the tile
};

// pull() with staged segments: a source inside the sample whose direction is
// staged is read from shared memory; everything else as in pull().
template <typename S, bool INTERIOR, int BX, class C>
__device__ __forceinline__ void pull_staged(const S* __restrict__ fin, const DevSample& s, int x,
                                            int y, const typename Codec<S>::R* __restrict__ ghost,
                                            const C& qc, const StagedSrc<S, BX>& st,
                                            typename Codec<S>::R (&f)[kQ]) {
  constexpr int G = Stage<S>::kG, SL = Stage<S>::template slots<BX>();
  constexpr int VB = Stage<S>::kVecBytes;
  const long long site = (long long)y * s.ldx + x;
  const int i = x - st.x0;
  if (INTERIOR && __builtin_expect(st.mask == (1u << kDirs) - 1u, 1)) {
#pragma unroll
    for (int d = 0; d < kDirs; ++d)
      Codec<S>::load4s(st.buf + (uint32_t)((d * SL + i + ((st.x0 - hop_x(d)) & (G - 1))) * VB),
                       dir_kind(d), qc, &f[4 * d]);
    return;
  }
#pragma unroll
  for (int d = 0; d < kDirs; ++d) {
    const int dx = hop_x(d), dy = hop_y(d);
    const bool staged = (st.mask >> d) & 1u;
    const uint32_t sp = st.buf + (uint32_t)((d * SL + i + ((st.x0 - dx) & (G - 1))) * VB);
    if (INTERIOR) {
      if (staged) Codec<S>::load4s(sp, dir_kind(d), qc, &f[4 * d]);
      else Codec<S>::load4(fin + vec_index(s, d, site - ((long long)dy * s.ldx + dx)), dir_kind(d),
                           qc, &f[4 * d]);
    } else {
      int sx = x - dx, sy = y - dy;
      if (s.periodic_x) sx = sx < 0 ? sx + s.nx : (sx >= s.nx ? sx - s.nx : sx);
      if (s.periodic_y) sy = sy < 0 ? sy + s.ny : (sy >= s.ny ? sy - s.ny : sy);
      const bool inside = (unsigned)sx < (unsigned)s.nx && (unsigned)sy < (unsigned)s.ny;
      if (inside) {
        if (staged) Codec<S>::load4s(sp, dir_kind(d), qc, &f[4 * d]);
        else Codec<S>::load4(fin + vec_index(s, d, (long long)sy * s.ldx + sx), dir_kind(d), qc,
                             &f[4 * d]);
      } else {
        const int owner = contact_of(s, sx, sy);
        if (owner >= 0) {
#pragma unroll
          for (int j = 0; j < kShells; ++j) f[4 * d + j] = ghost[owner * kQ + 4 * d + j];
        } else {
          Codec<S>::load4(fin + vec_index(s, d ^ 1, site), dir_kind(d), qc, &f[4 * d]);
        }
      }
    }
  }
}

template <typename R>
__device__ __forceinline__ void block_reduce_add2(double a, double b, double* acc) {
  __shared__ double sa[32], sb[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sa[warp] = a; sb[warp] = b; }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      atomicAdd(acc, a);
      atomicAdd(acc + 1, b);
    }
  }
}

// Warp sums of (a, b) added to acc[0], acc[1] by lane 0 (no block barrier).
__device__ __forceinline__ void warp_reduce_add2(double a, double b, double* acc) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc, a);
    atomicAdd(acc + 1, b);
  }
}

// New relative deviations of the four shells of a direction from its cubic:
// out_j = (1 - omega) g_j + R0 + R1 p0_j + R2 p0_j^2 + R3 p0_j^3
// (delta = w g: the weight w_j drops out of the update).
template <typename R, class C>
__device__ __forceinline__ void relax_shells(const R (&Rm)[4], R omega, int kind, const C& qc,
                                             R* f) {
  const R omc = R(1) - omega;
#pragma unroll
  for (int j = 0; j < kShells; ++j) {
    const R p = qc.p0[j];
    const R val = fma(fma(fma(Rm[3], p, Rm[2]), p, Rm[1]), p, Rm[0]);
    f[j] = fma(omc, f[j], val);
  }
}

// Adds sum_j w_j (out_j - in_j) p0_j and sum_j w_j (out_j - in_j) p0_j^2 of one
// direction (relative deviations in / out).
template <typename R, class C>
__device__ __forceinline__ void balance(const R* in, const R* out, int kind, const C& qc, R& aN,
                                        R& aE) {
#pragma unroll
  for (int j = 0; j < kShells; ++j) {
    const R dlt = out[j] - in[j];
    aN = fma(dlt, qc.wp0[kind][j], aN);
    aE = fma(dlt, qc.wp0sq[kind][j], aE);
  }
}

// Gradient of the previous step's n - 1 at (x, y) over one hop (5 sites, the
// length unit of c = 1): (a(x + 5) - a(x - 5)) / 2 where both exist, the
// forward or backward difference over 5 sites next to a walled edge, wrapped
// on periodic axes (Sec. 3, local capacitance approximation; a difference over
// neighbouring sites would drive density structure finer than a hop).
template <typename R>
__device__ __forceinline__ void lca_gradient(const DevSample& s, const R* __restrict__ p, int x,
                                             int y, R& gx, R& gy) {
  constexpr int h = kRadius;
  int xm = x - h, xp = x + h, ym = y - h, yp = y + h;
  R hx = R(0.5), hy = R(0.5);
  if (s.periodic_x) { xm = xm < 0 ? xm + s.nx : xm; xp = xp >= s.nx ? xp - s.nx : xp; }
  else if (xm < 0) { xm = x; hx = R(1); }
  else if (xp >= s.nx) { xp = x; hx = R(1); }
  if (s.periodic_y) { ym = ym < 0 ? ym + s.ny : ym; yp = yp >= s.ny ? yp - s.ny : yp; }
  else if (ym < 0) { ym = y; hy = R(1); }
  else if (yp >= s.ny) { yp = y; hy = R(1); }
  const long long row = (long long)y * s.ldx;
  gx = (p[row + xp] - p[row + xm]) * hx;
  gy = (p[(long long)yp * s.ldx + x] - p[(long long)ym * s.ldx + x]) * hy;
}

// Gathers the 48 deviations streamed into site (x < nx, y): from HBM or from
// the staged slot rows.  All 32 threads of a warp must hold consecutive x of
// the same row (the interior test is per warp).
template <typename S, class C, class SRC>
__device__ __forceinline__ void gather(const S* __restrict__ fin, const DevSample& s, int x, int y,
                                       const typename Codec<S>::R* __restrict__ ghost, const C& qc,
                                       const SRC& src, typename Codec<S>::R (&f)[kQ]) {
  // warp-uniform: the 32 sites of this warp pull only from inside the rectangle
  const int wx0 = x & ~31;
  const bool interior = wx0 >= kRadius && wx0 + 32 + kRadius <= s.nx &&
                        y >= kRadius && y + kRadius < s.ny;
  if constexpr (std::is_same<SRC, DirectSrc>::value) {
    if (interior) pull<S, true>(fin, s, x, y, ghost, qc, f);
    else          pull<S, false>(fin, s, x, y, ghost, qc, f);
  } else {
    if (interior) pull_staged<S, true>(fin, s, x, y, ghost, qc, src, f);
    else          pull_staged<S, false>(fin, s, x, y, ghost, qc, src, f);
  }
}

// Per-direction cubic coefficients of a direction pair, on lanes (d, d + 1):
// the quantities pair_cubics() computes, written on register pairs.  Every
// polynomial in v is split into even and odd parts, and the odd parts take
// the constant pairs (a, -a) of QuadConsts::odd, so each instruction serves
// both directions.  nT, nmT as in pair_cubics; FxT, FyT = (Fx, Fy) nT.
// Returns R0..R3 (lanes p, n) and om = (omega_p, omega_n).
template <bool FORCE, class C>
__device__ __forceinline__ void pair_cubics_paired(const int d, const EqCoeffs<float>& c,
                                                   float nT, float nmT, float gt, float gux,
                                                   float guy, float FxT, float FyT, const C& qc,
                                                   float2 (&R)[4], float2& om) {
  const int q = d / 2;
  const bool hx = hop_x(d) != 0, hy = hop_y(d) != 0;
  const float vx = float(hop_x(d)) / 5.f, vy = float(hop_y(d)) / 5.f;
  const float2* od = qc.odd[q];
  // omega = gamma (1 -+ v.u) / tau on the two lanes
  om = S2(gt);
  if (hx) om = fma2(S2(gux), od[kONVx], om);
  if (hy) om = fma2(S2(guy), od[kONVy], om);
  const float2 on = mul2(om, S2(nT));
  float2 q1 = S2(c.c1_0);
  if (hx) q1 = fma2(S2(c.c1_x), od[kOVx], q1);
  if (hy) q1 = fma2(S2(c.c1_y), od[kOVy], q1);
  float2 q2 = S2(c.c2_0);
  if (hx) q2 = fma2(S2(c.c2_xx), S2(vx * vx), q2);
  if (hx && hy) q2 = fma2(S2(c.c2_xy), S2(vx * vy), q2);
  if (hx) q2 = fma2(S2(c.c2_x), od[kOVx], q2);
  if (hy) q2 = fma2(S2(c.c2_y), od[kOVy], q2);
  float2 q3 = S2(c.c3_0);
  if (hx) q3 = fma2(S2(c.c3_xx), S2(vx * vx), q3);
  if (hx && hy) q3 = fma2(S2(c.c3_xy), S2(vx * vy), q3);
  if (hx) q3 = fma2(S2(c.c3_x), od[kOVx], q3);
  if (hy) q3 = fma2(S2(c.c3_y), od[kOVy], q3);
  if (hx) q3 = fma2(S2(c.c3_xxx), od[kOVx3], q3);
  if (hx && hy) q3 = fma2(S2(c.c3_xxy), od[kOVx2y], q3);
  R[0] = fma2(on, S2(c.q0m1), mul2(om, S2(nmT)));
  R[1] = mul2(on, q1);
  R[2] = mul2(on, q2);
  R[3] = mul2(on, q3);
  if (FORCE) {
    // lanes (F.v, -F.v) and (F.t, -F.t) times n/T, t = (-vy, vx)
    float2 Fv, Ft;
    if (hx && hy) {
      Fv = fma2(S2(FxT), od[kOVx], mul2(S2(FyT), od[kOVy]));
      Ft = fma2(S2(FyT), od[kOVx], mul2(S2(FxT), od[kONVy]));
    } else if (hx) {
      Fv = mul2(S2(FxT), od[kOVx]);
      Ft = mul2(S2(FyT), od[kOVx]);
    } else {
      Fv = mul2(S2(FyT), od[kOVy]);
      Ft = mul2(S2(FxT), od[kONVy]);
    }
    // minus the shell derivatives dq_m/dtheta on the two lanes
    float2 nD1;
    if (hx && hy) nD1 = fma2(S2(c.c1_x), od[kOVy], mul2(S2(c.c1_y), od[kONVx]));
    else if (hx) nD1 = mul2(S2(c.c1_y), od[kONVx]);
    else nD1 = mul2(S2(c.c1_x), od[kOVy]);
    // even part of -dq2/dtheta: 2 vx vy c2_xx + (vy^2 - vx^2) c2_xy
    float2 nD2 = mul2(S2(c.c2_xy), S2(vy * vy - vx * vx));
    if (hx && hy) nD2 = fma2(S2(c.c2_xx), S2(2.f * vx * vy), nD2);
    if (hy) nD2 = fma2(S2(c.c2_x), od[kOVy], nD2);
    if (hx) nD2 = fma2(S2(c.c2_y), od[kONVx], nD2);
    float2 nD3 = mul2(S2(c.c3_xy), S2(vy * vy - vx * vx));
    if (hx && hy) nD3 = fma2(S2(c.c3_xx), S2(2.f * vx * vy), nD3);
    if (hy) nD3 = fma2(S2(c.c3_x), od[kOVy], nD3);
    if (hx) nD3 = fma2(S2(c.c3_y), od[kONVx], nD3);
    if (hx && hy) nD3 = fma2(S2(c.c3_xxx), od[kO3x2y], nD3);
    if (hx) nD3 = fma2(S2(c.c3_xxy), od[kOX3m2xy2], nD3);
    const float q0 = 1.f + c.q0m1;
    // s_m = (F.v)(q_m - (m + 1) q_{m+1}) - (F.t) dq_{m+1}/dtheta
    R[0] = fma2(Fv, fma2(q1, S2(-1.f), S2(q0)), R[0]);
    R[0] = fma2(Ft, nD1, R[0]);
    R[1] = fma2(Fv, fma2(q2, S2(-2.f), q1), R[1]);
    R[1] = fma2(Ft, nD2, R[1]);
    R[2] = fma2(Fv, fma2(q3, S2(-3.f), q2), R[2]);
    R[2] = fma2(Ft, nD3, R[2]);
    R[3] = fma2(Fv, q3, R[3]);
  }
}

// New relative deviations of the four shells of one direction on shell pairs:
// out_j = (1 - omega) g_j + R0 + R1 p0_j + R2 p0_j^2 + R3 p0_j^3.  With BAL the
// direction's moment change (sum_j w p0_j (out_j - g_j), sum_j w p0_j^2
// (out_j - g_j)) is returned in bal (the conservation projection's input).
template <bool BAL, class C>
__device__ __forceinline__ void relax_shells_paired(float R0, float R1, float R2, float R3,
                                                    float omc, int kind, const C& qc, float* f,
                                                    float2& bal) {
  const float2 v01 = fma2(fma2(fma2(S2(R3), qc.p01, S2(R2)), qc.p01, S2(R1)), qc.p01, S2(R0));
  const float2 v23 = fma2(fma2(fma2(S2(R3), qc.p23, S2(R2)), qc.p23, S2(R1)), qc.p23, S2(R0));
  const float2 i01 = make_float2(f[0], f[1]), i23 = make_float2(f[2], f[3]);
  const float2 o01 = fma2(S2(omc), i01, v01);
  const float2 o23 = fma2(S2(omc), i23, v23);
  if (BAL) {
    const float2 d01 = fma2(i01, S2(-1.f), o01), d23 = fma2(i23, S2(-1.f), o23);
    bal = mul2(S2(d01.x), qc.wab[kind][0]);
    bal = fma2(S2(d01.y), qc.wab[kind][1], bal);
    bal = fma2(S2(d23.x), qc.wab[kind][2], bal);
    bal = fma2(S2(d23.y), qc.wab[kind][3], bal);
  }
  f[0] = o01.x; f[1] = o01.y; f[2] = o23.x; f[3] = o23.y;
}

// collide_store() with FP32 arithmetic (FP32 and 16-bit storage) on register
// pairs: the same quantities in the same order of operations per population,
// with each instruction serving two directions or two shells.
template <typename S, int FORCE, int RES, int BT, class C>
__device__ __forceinline__ void collide_store_paired(float (&f)[kQ], S* __restrict__ fout,
                                                     const DevSample& s, int x, int y,
                                                     const StepAux<float>& aux, const C& qc,
                                                     double& r_du2, double& r_u2, uint32_t park,
                                                     const float* dn_prev, float* dn_next) {
  constexpr bool kProject = sizeof(S) == sizeof(float);
  const bool lca = FORCE == kForceLca && s.inv_cg != 0.0;
  float egx = 0.f, egy = 0.f;
  if (lca) lca_gradient(s, dn_prev, x, y, egx, egy);
  const Moments<float> m = moments(f, qc);
  constexpr uint32_t park_stride = BT * 16u;
#pragma unroll
  for (int d = 0; d < kDirs; ++d) park_store(park + d * park_stride, &f[4 * d]);
  Macro<float> M;
  const bool conv = landau(m, M);
  unsigned bad = 0;
  if (!conv) bad |= kErrNoConvergence;
  if (!all_finite(M)) bad |= kErrNonFinite;
  else if (!macro_ok(M)) bad |= kErrUnphysical;
  if (bad) atomicOr(aux.err, bad);

  const EqCoeffs<float> c = eq_coeffs(M);
  const float scl = sizeof(S) == 2 ? qc.enc_s : 1.f;
  const float inv1T = qdiv(1.f, 1.f + M.dT);
  const float nT = (1.f + M.dn) * inv1T * scl;
  const float nmT = (M.dn - M.dT) * inv1T * scl;
  const float gt = M.gamma * float(s.inv_tau);
  const float gux = gt * M.ux, guy = gt * M.uy;
  const float Fx = lca ? float(s.Fx) + (-float(s.inv_cg) * egx) : float(s.Fx);
  const float Fy = lca ? float(s.Fy) + (-float(s.inv_cg) * egy) : float(s.Fy);
  const float FxT = Fx * nT, FyT = Fy * nT;
  const long long site = (long long)y * s.ldx + x;
  if (lca) dn_next[site] = M.dn;
  // conservation projection: sums of the moment changes (N^0, T^00) and
  // (T^0x, T^0y), started with minus the forcing's target
  float2 accNE = S2(0.f), accXY = S2(0.f);
  if (kProject && FORCE != 0) {
    // forcing changes T^0a by (F.N_E, F N_E^0), N_E = n gamma (1, u)
    const float nG = (1.f + M.dn) * M.gamma;
    accNE = make_float2(0.f, -(nG * (Fx * M.ux + Fy * M.uy)));
    accXY = make_float2(-(nG * Fx), -(nG * Fy));
  }
  // (5,0)-type pairs first: with FP32 storage they take the correction and
  // are stored last; the (3,4)-type pairs are stored as soon as done.
#pragma unroll
  for (int pi = 0; pi < kDirs / 2; ++pi) {
    const int d = (2 * pi + 8) % kDirs;
    const int kind = dir_kind(d);
    float2 R[4], om;
    pair_cubics_paired<FORCE != 0>(d, c, nT, nmT, gt, gux, guy, FxT, FyT, qc, R, om);
    park_load(park + d * park_stride, &f[4 * d]);
    park_load(park + (d + 1) * park_stride, &f[4 * d + 4]);
    const float2 omc = fma2(om, S2(-1.f), S2(1.f));
    float2 bp, bn;
    relax_shells_paired<kProject>(R[0].x, R[1].x, R[2].x, R[3].x, omc.x, kind, qc, &f[4 * d], bp);
    relax_shells_paired<kProject>(R[0].y, R[1].y, R[2].y, R[3].y, omc.y, kind, qc, &f[4 * d + 4],
                                  bn);
    if (kProject) {
      accNE = add2(accNE, add2(bp, bn));
      accXY = fma2(S2(bp.y - bn.y), qc.vxy[d / 2], accXY);
    }
    if (!kProject || kind == 0) {
      Codec<S>::store4(fout + vec_index(s, d, site), kind, qc, &f[4 * d]);
      Codec<S>::store4(fout + vec_index(s, d + 1, site), kind, qc, &f[4 * d + 4]);
    } else {
      // (5,0)-type: wait for the correction in the parking area, not in registers
      park_store(park + d * park_stride, &f[4 * d]);
      park_store(park + (d + 1) * park_stride, &f[4 * d + 4]);
    }
  }
  if (kProject) {
    const float rN = accNE.x, rE = accNE.y;
    const float l0 = qc.P00 * rN + qc.P01 * rE;
    const float l1 = qc.P10 * rN + qc.P11 * rE;
    const float lx = qc.px * accXY.x, ly = qc.px * accXY.y;
#pragma unroll
    for (int d = 8; d < kDirs; ++d) {
      const float cd = l1 + (hop_x(d) > 0 ? lx : hop_x(d) < 0 ? -lx : hop_y(d) > 0 ? ly : -ly);
      park_load(park + d * park_stride, &f[4 * d]);
      // delta += w (l0 + p0 cd)
      const float2 t01 = fma2(S2(cd), qc.p01, S2(l0));
      const float2 t23 = fma2(S2(cd), qc.p23, S2(l0));
      const float2 o01 = add2(make_float2(f[4 * d], f[4 * d + 1]), t01);
      const float2 o23 = add2(make_float2(f[4 * d + 2], f[4 * d + 3]), t23);
      f[4 * d] = o01.x; f[4 * d + 1] = o01.y; f[4 * d + 2] = o23.x; f[4 * d + 3] = o23.y;
      Codec<S>::store4(fout + vec_index(s, d, site), 1, qc, &f[4 * d]);
    }
  }
  if (RES == 1) {
    const long long k = s.site0 + (long long)y * s.nx + x;
    aux.uprev[2 * k] = M.ux;
    aux.uprev[2 * k + 1] = M.uy;
  } else if (RES == 2) {
    const long long k = s.site0 + (long long)y * s.nx + x;
    const double dx = double(M.ux) - double(aux.uprev[2 * k]);
    const double dy = double(M.uy) - double(aux.uprev[2 * k + 1]);
    r_du2 += dx * dx + dy * dy;
    r_u2 += double(M.ux) * double(M.ux) + double(M.uy) * double(M.uy);
  }
}

// Collision of the gathered deviations f of site (x < nx, y) and store of the
// 48 new deviations into fout.  RES: 0 nothing extra; 1 store u for the
// residual; 2 add |u - u_prev|^2 and |u|^2 to r_du2, r_u2 (the caller
// reduces them).  dn_prev / dn_next: the electric force's density planes of
// the previous and of this step (used when s.inv_cg != 0).
template <typename S, int FORCE, int RES, int BT, class C>
__device__ __forceinline__ void collide_store(typename Codec<S>::R (&f)[kQ], S* __restrict__ fout,
                                              const DevSample& s, int x, int y,
                                              const StepAux<typename Codec<S>::R>& aux,
                                              const C& qc, double& r_du2, double& r_u2,
                                              uint32_t park,
                                              const typename Codec<S>::R* dn_prev,
                                              typename Codec<S>::R* dn_next) {
  using R = typename Codec<S>::R;
  if constexpr (std::is_same<R, float>::value) {
    collide_store_paired<S, FORCE, RES, BT>(f, fout, s, x, y, aux, qc, r_du2, r_u2, park, dn_prev,
                                        dn_next);
    return;
  }
  // FP32 storage: the FP32 quadrature constants satisfy Eq. orthonormal only
  // to ~1e-7, which would break the exact conservation of N^0 and T^0a by the
  // collision at that level every step (a secular drift).  The update is
  // projected back onto the exact discrete balance
  //   sum_i p0 (f* - f) = 0,  sum_i p0 p^a (f* - f) = (F.N_E, F N_E^0)
  // by a correction on the (5,0)-type directions (solved with the constants P**, px).
  constexpr bool kProject = sizeof(S) == sizeof(float);
  {
    // electric force (local capacitance approximation): the neighbours'
    // density of the previous step, loaded before the long arithmetic
    const bool lca = FORCE == kForceLca && s.inv_cg != 0.0;
    R egx = R(0), egy = R(0);
    if (lca) lca_gradient(s, dn_prev, x, y, egx, egy);
    const Moments<R> m = moments(f, qc);
    // park: entry of direction d at park + d * BT * 16 (BT threads per block)
    constexpr uint32_t park_stride = BT * 16u;
    if constexpr (Park<R>::kOn) {
#pragma unroll
      for (int d = 0; d < kDirs; ++d) park_store(park + d * park_stride, &f[4 * d]);
    }
    Macro<R> M;
    const bool conv = landau(m, M);
    unsigned bad = 0;
    if (!conv) bad |= kErrNoConvergence;
    if (!all_finite(M)) bad |= kErrNonFinite;
    else if (!macro_ok(M)) bad |= kErrUnphysical;
    if (bad) atomicOr(aux.err, bad);

    const EqCoeffs<R> c = eq_coeffs(M);
    // every term of the update is proportional to n/T or (n - T)/T: the
    // 16-bit kernels, which work on the stored s g, scale those by s
    const R scl = sizeof(S) == 2 ? qc.enc_s : R(1);
    const R inv1T = qdiv(R(1), R(1) + M.dT);
    const R nT = (R(1) + M.dn) * inv1T * scl;
    const R nmT = (M.dn - M.dT) * inv1T * scl;
    const R gt = M.gamma * R(s.inv_tau);
    const R gux = gt * M.ux, guy = gt * M.uy;
    const R Fx = lca ? R(s.Fx) + (-R(s.inv_cg) * egx) : R(s.Fx);
    const R Fy = lca ? R(s.Fy) + (-R(s.inv_cg) * egy) : R(s.Fy);
    const long long site = (long long)y * s.ldx + x;
    if (lca) dn_next[site] = M.dn;
    R rN = R(0), rE = R(0), rX = R(0), rY = R(0);
    // (5,0)-type pairs first: in reduced precision they take the correction
    // and are stored last; the (3,4)-type pairs are stored as soon as done.
#pragma unroll
    for (int pi = 0; pi < kDirs / 2; ++pi) {
      const int d = (2 * pi + 8) % kDirs;
      R Rp[4], Rn[4], omp, omn;
      pair_cubics<R, FORCE != 0>(d, c, nT, nmT, gt, gux, guy, Fx, Fy, Rp, Rn, omp, omn);
      const int kind = dir_kind(d);
      if constexpr (Park<R>::kOn) {
        park_load(park + d * park_stride, &f[4 * d]);
        park_load(park + (d + 1) * park_stride, &f[4 * d + 4]);
      }
      if (kProject) {
        R in[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) in[j] = f[4 * d + j];
        relax_shells(Rp, omp, kind, qc, &f[4 * d]);
        relax_shells(Rn, omn, kind, qc, &f[4 * d + 4]);
        R aNp = R(0), aEp = R(0), aNn = R(0), aEn = R(0);
        balance(in, &f[4 * d], kind, qc, aNp, aEp);
        balance(in + 4, &f[4 * d + 4], kind, qc, aNn, aEn);
        rN += aNp + aNn;
        rE += aEp + aEn;
        const R vx = R(hop_x(d)) / R(5), vy = R(hop_y(d)) / R(5);
        if (hop_x(d) != 0) rX = fma(aEp - aEn, vx, rX);
        if (hop_y(d) != 0) rY = fma(aEp - aEn, vy, rY);
        if (kind == 0) {
          Codec<S>::store4(fout + vec_index(s, d, site), kind, qc, &f[4 * d]);
          Codec<S>::store4(fout + vec_index(s, d + 1, site), kind, qc, &f[4 * d + 4]);
        } else if constexpr (Park<R>::kOn) {
          // (5,0)-type: wait for the correction in the parking area, not in registers
          park_store(park + d * park_stride, &f[4 * d]);
          park_store(park + (d + 1) * park_stride, &f[4 * d + 4]);
        }
      } else {
        relax_shells(Rp, omp, kind, qc, &f[4 * d]);
        relax_shells(Rn, omn, kind, qc, &f[4 * d + 4]);
        Codec<S>::store4(fout + vec_index(s, d, site), kind, qc, &f[4 * d]);
        Codec<S>::store4(fout + vec_index(s, d + 1, site), kind, qc, &f[4 * d + 4]);
      }
    }
    if (kProject) {
      if (FORCE != 0) {
        // forcing changes T^0a by (F.N_E, F N_E^0), N_E = n gamma (1, u)
        const R nG = (R(1) + M.dn) * M.gamma;
        rE -= nG * (Fx * M.ux + Fy * M.uy);
        rX -= nG * Fx;
        rY -= nG * Fy;
      }
      const R l0 = qc.P00 * rN + qc.P01 * rE;
      const R l1 = qc.P10 * rN + qc.P11 * rE;
      const R lx = qc.px * rX, ly = qc.px * rY;
#pragma unroll
      for (int d = 8; d < kDirs; ++d) {
        const R cd = l1 + (hop_x(d) > 0 ? lx : hop_x(d) < 0 ? -lx : hop_y(d) > 0 ? ly : -ly);
        if constexpr (Park<R>::kOn) park_load(park + d * park_stride, &f[4 * d]);
#pragma unroll
        for (int j = 0; j < kShells; ++j)
          f[4 * d + j] = f[4 * d + j] + fma(qc.p0[j], cd, l0);   // delta += w (l0 + p0 cd)
        Codec<S>::store4(fout + vec_index(s, d, site), 1, qc, &f[4 * d]);
      }
    }
    if (RES == 1) {
      const long long k = s.site0 + (long long)y * s.nx + x;
      aux.uprev[2 * k] = M.ux;
      aux.uprev[2 * k + 1] = M.uy;
    } else if (RES == 2) {
      const long long k = s.site0 + (long long)y * s.nx + x;
      const double dx = double(M.ux) - double(aux.uprev[2 * k]);
      const double dy = double(M.uy) - double(aux.uprev[2 * k + 1]);
      r_du2 += dx * dx + dy * dy;
      r_u2 += double(M.ux) * double(M.ux) + double(M.uy) * double(M.uy);
    }
  }
}

// Fused stream + collide of site (x, y) (nothing if x >= nx).
template <typename S, int FORCE, int RES, int BT, class C>
__device__ __forceinline__ void site_step(const S* __restrict__ fin, S* __restrict__ fout,
                                          const DevSample& s, int x, int y,
                                          const typename Codec<S>::R* __restrict__ ghost,
                                          const StepAux<typename Codec<S>::R>& aux, const C& qc,
                                          double& r_du2, double& r_u2, uint32_t park, int cur) {
  using R = typename Codec<S>::R;
  if (x < s.nx) {
    R f[kQ];
    gather(fin, s, x, y, ghost, qc, DirectSrc(), f);
    // select, not s.dn[cur]: a runtime index would move the descriptor to local memory
    void* const prev = cur ? s.dn[1] : s.dn[0];
    void* const next = cur ? s.dn[0] : s.dn[1];
    collide_store<S, FORCE, RES, BT>(f, fout, s, x, y, aux, qc, r_du2, r_u2, park,
                                 static_cast<const R*>(prev), static_cast<R*>(next));
  }
}

// One sample, one block row of kBX sites.
template <typename S, int FORCE, int RES, class C>
__device__ __forceinline__ void step_body(const S* __restrict__ fin, S* __restrict__ fout,
                                          const DevSample& s,
                                          const typename Codec<S>::R* __restrict__ ghost,
                                          const StepAux<typename Codec<S>::R>& aux, const C& qc,
                                          unsigned char* park) {
  double r_du2 = 0.0, r_u2 = 0.0;
  site_step<S, FORCE, RES, kBX>(fin, fout, s, blockIdx.x * kBX + threadIdx.x, blockIdx.y, ghost, aux,
                           qc, r_du2, r_u2, smem_addr(park) + threadIdx.x * 16u, s.cur);
  if (RES == 2) block_reduce_add2<typename Codec<S>::R>(r_du2, r_u2, aux.acc);
}

// Many samples of uneven size in one launch.  The work list is every row
// segment of BX sites of every sample ("tile"), numbered sample by sample;
// tile_start[k] is the first tile of sample k (tile_start[nsamples] = total).
// Blocks walk the list with a grid stride (persistent when the grid is a
// multiple of the SM count).  Sample k's buffers are base + samples[k].off[cur]
// (input) and base + samples[k].off[1 - cur] (output).
struct BatchArgs {
  const DevSample* samples;
  const long long* tile_start;
  int nsamples;
  int cur;
  long long ntiles;
  long long wait_limit;   // clock cycles a wait for a staged tile may take before it gives up
};

template <typename S, int FORCE, int RES, int BX, class C>
__device__ __forceinline__ void batch_body(S* __restrict__ base, const BatchArgs& b,
                                           const typename Codec<S>::R* __restrict__ ghost,
                                           const StepAux<typename Codec<S>::R>& aux, const C& qc,
                                           unsigned char* park) {
  const uint32_t my_park = smem_addr(park) + threadIdx.x * 16u;
#pragma unroll 1
  for (long long t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
    int lo = 0, hi = b.nsamples;                 // tile_start[lo] <= t < tile_start[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(b.tile_start + mid) <= t) lo = mid; else hi = mid;
    }
    const DevSample s = b.samples[lo];
    const long long lt = t - __ldg(b.tile_start + lo);
    const int tpr = (s.nx + BX - 1) / BX;
    const int y = (int)(lt / tpr);
    const int x = (int)(lt - (long long)y * tpr) * BX + threadIdx.x;
    const long long oin = b.cur ? s.off[1] : s.off[0];
    const long long oout = b.cur ? s.off[0] : s.off[1];
    double r_du2 = 0.0, r_u2 = 0.0;
    site_step<S, FORCE, RES, BX>(base + oin, base + oout, s, x, y,
                             ghost + (long long)lo * kMaxContacts * kQ, aux, qc, r_du2, r_u2,
                             my_park, b.cur);
    // per-sample residual accumulators: acc[2 k], acc[2 k + 1]
    if (RES == 2) {
      block_reduce_add2<typename Codec<S>::R>(r_du2, r_u2, aux.acc + 2 * lo);
      __syncthreads();   // the reduction's shared scratch is reused by the next tile
    }
  }
}

// The batched step with staged pulls (persistent: gridDim.x blocks walk the
// tile list with a grid stride; the block's k-th tile is blockIdx.x + k G,
// G = gridDim.x).  Two slot-row buffers alternate: buffer b holds tiles
// k = b, b + 2, ... (use j = k / 2), and mbarrier full[b] completes phase j
// when tile 2 j + b has landed (one arrive with the byte count by the issuing
// warp, plus the copies' bytes).  Warp 0 fills both buffers up front; after
// that the last warp to finish gathering tile k (a shared counter per buffer)
// issues tile k + 2 into the buffer it just freed, so two tiles are always in
// flight or landed and no warp waits for another one.  Every wait is bounded
// (b.wait_limit cycles, about 1 s by default): a warp that gives up sets
// kErrTimeout and a shared abort flag, waits once more for the copies of both
// buffers (bounded by the full ~1 s whatever b.wait_limit is, so that no bulk
// copy into the block's shared memory is left in flight), and leaves the loop;
// the other warps leave at their next tile.
template <typename S, int FORCE, int RES, int BX, class C>
__device__ __forceinline__ void staged_batch_body(S* __restrict__ base, const BatchArgs& b,
                                                  const typename Codec<S>::R* __restrict__ ghost,
                                                  const StepAux<typename Codec<S>::R>& aux,
                                                  const C& qc, unsigned char* smem) {
  using R = typename Codec<S>::R;
  constexpr int BUF = Stage<S>::template buf_elems<BX>();
  constexpr int kWarps = BX / 32;
  S* stage = reinterpret_cast<S*>(smem);
  unsigned char* ctl = smem + 2 * (size_t)BUF * sizeof(S);
  uint64_t* full = reinterpret_cast<uint64_t*>(ctl);          // [2]
  unsigned* released = reinterpret_cast<unsigned*>(ctl + 16);  // [2] warps done gathering
  int4* tiles = reinterpret_cast<int4*>(ctl + 32);             // [2]: sample, x0, y
  unsigned* masks = reinterpret_cast<unsigned*>(ctl + 64);     // [2]
  volatile int* abort_flag = reinterpret_cast<volatile int*>(ctl + 72);
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t my_park = smem_addr(ctl + kStageCtlBytes) + tid * 16u;
  const uint32_t full0 = smem_addr(&full[0]), full1 = smem_addr(&full[1]);
  const uint32_t buf0 = smem_addr(stage), buf1 = smem_addr(stage + BUF);
  auto full_bar = [&](int k) { return k ? full1 : full0; };
  const long long G = gridDim.x;
  long long t = blockIdx.x;
  if (t >= b.ntiles) return;
  if (tid == 0) {
    stage_bar_init(full0, 1);
    stage_bar_init(full1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    released[0] = released[1] = 0;
    *abort_flag = 0;
  }
  __syncthreads();

  // fills buffer `buf` with tile tt (all lanes of the calling warp)
  auto issue = [&](long long tt, int buf) {
    int lo = 0, hi = b.nsamples;                 // tile_start[lo] <= tt < tile_start[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(b.tile_start + mid) <= tt) lo = mid; else hi = mid;
    }
    const DevSample& s = b.samples[lo];
    const long long lt = tt - __ldg(b.tile_start + lo);
    const int tpr = (s.nx + BX - 1) / BX;
    const int y = (int)(lt / tpr);
    const int x0 = (int)(lt - (long long)y * tpr) * BX;
    const S* fin = base + (b.cur ? s.off[1] : s.off[0]);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    stage_issue<S, BX>(fin, s, x0, y, stage + (size_t)buf * BUF, full_bar(buf), &masks[buf],
                       &tiles[buf], lo);
  };

  if (tid < 32) {
    issue(t, 0);
    if (t + G < b.ntiles) issue(t + G, 1);
  }
#pragma unroll 1
  for (int it = 0;; ++it) {
    const int cb = it & 1;
    bool ok = !*abort_flag && stage_wait(full_bar(cb), (it >> 1) & 1, b.wait_limit);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
      if (lane == 0 && !*abort_flag) {
        *abort_flag = 1;
        atomicOr(aux.err, kErrTimeout);
      }
      // copies that may still be in flight into either buffer
      stage_wait(full_bar(cb), (it >> 1) & 1);
      if (t + G < b.ntiles) stage_wait(full_bar(cb ^ 1), ((it + 1) >> 1) & 1);
      break;
    }
    const int4 tl = tiles[cb];
    const StagedSrc<S, BX> src{cb ? buf1 : buf0, masks[cb], tl.y};
    const DevSample s = b.samples[tl.x];
    const int x = tl.y + tid;
    R f[kQ];
    if (x < s.nx) gather(base + (b.cur ? s.off[1] : s.off[0]), s, x, tl.z,
                         ghost + (long long)tl.x * kMaxContacts * kQ, qc, src, f);
    __syncwarp();
    // the last warp done with this buffer refills it with tile k + 2
    if (t + 2 * G < b.ntiles) {
      unsigned last = 0;
      if (lane == 0) {
        // a compiler barrier too: this tile's shared reads stay before it
        unsigned prev;
        asm volatile("atom.shared.add.u32 %0, [%1], 1;\n"
                     : "=r"(prev) : "r"(smem_addr(&released[cb])) : "memory");
        last = prev == kWarps - 1;
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      if (last) {
        if (lane == 0) released[cb] = 0;
        issue(t + 2 * G, cb);
      }
    }
    double r_du2 = 0.0, r_u2 = 0.0;
    if (x < s.nx)
      collide_store<S, FORCE, RES, BX>(f, base + (b.cur ? s.off[0] : s.off[1]), s, x, tl.z, aux, qc,
                                   r_du2, r_u2, my_park,
                                   static_cast<const R*>(b.cur ? s.dn[1] : s.dn[0]),
                                   static_cast<R*>(b.cur ? s.dn[0] : s.dn[1]));
    if (RES == 2) warp_reduce_add2(r_du2, r_u2, aux.acc + 2 * tl.x);
    t += G;
    if (t >= b.ntiles) break;
  }
}

// Macroscopic fields of the streamed populations (no collision).
template <typename S, class C>
__device__ __forceinline__ void moments_body(const S* __restrict__ fin, const DevSample& s,
                                             const typename Codec<S>::R* __restrict__ ghost,
                                             double* n, double* ux, double* uy, double* T,
                                             unsigned* err, const C& qc,
                                             typename Codec<S>::R* dn_out) {
  using R = typename Codec<S>::R;
  const int bx0 = blockIdx.x * kBX;
  const int x = bx0 + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= s.nx) return;
  R f[kQ];
  pull<S, false>(fin, s, x, y, ghost, qc, f);
  const Moments<R> m = moments(f, qc);
  Macro<R> M;
  const bool conv = landau(m, M);
  unsigned bad = conv ? 0u : kErrNoConvergence;
  if (!all_finite(M)) bad |= kErrNonFinite;
  if (bad) atomicOr(err, bad);
  const long long k = (long long)y * s.nx + x;
  if (n) n[k] = 1.0 + double(M.dn);
  if (ux) ux[k] = double(M.ux);
  if (uy) uy[k] = double(M.uy);
  if (T) T[k] = 1.0 + double(M.dT);
  if (dn_out) dn_out[(long long)y * s.ldx + x] = M.dn;
}

// Macroscopic state of site k of dense FP64 fields (n, u, T).
template <typename R>
__device__ __forceinline__ Macro<R> field_macro(const double* n, const double* ux,
                                                const double* uy, const double* T, long long k,
                                                bool& ok) {
  Macro<R> M;
  const double vx = ux[k], vy = uy[k];
  const double u2 = vx * vx + vy * vy;
  const double sq = sqrt(1.0 - u2);
  M.ux = R(vx);
  M.uy = R(vy);
  M.gamma = R(1.0 / sq);
  M.gm1 = R(u2 / (sq * (1.0 + sq)));
  M.dn = R(n[k] - 1.0);
  M.dT = R(T[k] - 1.0);
  M.deps = R(0);
  ok = (u2 < 1.0) && (n[k] > 0.0) && (T[k] > 0.0) && isfinite(n[k]) && isfinite(T[k]);
  return M;
}

// Relative deviations (f^eq - w) / w of the two directions d (even), d + 1
// for the macroscopic state M (times s in 16-bit storage): vp, vn.
template <typename S, class C>
__device__ __forceinline__ void eq_pair(const Macro<typename Codec<S>::R>& M,
                                        const EqCoeffs<typename Codec<S>::R>& c, int d,
                                        const C& qc, typename Codec<S>::R* vp,
                                        typename Codec<S>::R* vn) {
  using R = typename Codec<S>::R;
  const R scl = sizeof(S) == 2 ? qc.enc_s : R(1);     // 16-bit storage holds s g
  const R inv1T = R(1) / (R(1) + M.dT);
  const R nT = (R(1) + M.dn) * inv1T * scl;
  const R nmT = (M.dn - M.dT) * inv1T * scl;
  R Rp[4], Rn[4], omp, omn;
  // omega = 1 and no force: out = w (f^eq - w) / w
  pair_cubics<R, false>(d, c, nT, nmT, R(1), R(0), R(0), R(0), R(0), Rp, Rn, omp, omn);
#pragma unroll
  for (int j = 0; j < kShells; ++j) vp[j] = vn[j] = R(0);
  relax_shells(Rp, R(1), dir_kind(d), qc, vp);
  relax_shells(Rn, R(1), dir_kind(d), qc, vn);
}

// Stored state := f^eq(n, u, T) - w (dense FP64 inputs).
template <typename S, class C>
__device__ __forceinline__ void init_body(S* __restrict__ fout, const DevSample& s,
                                          const double* n, const double* ux, const double* uy,
                                          const double* T, unsigned* err, const C& qc) {
  using R = typename Codec<S>::R;
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= s.nx) return;
  const long long k = (long long)y * s.nx + x;
  bool ok;
  const Macro<R> M = field_macro<R>(n, ux, uy, T, k, ok);
  if (!ok) atomicOr(err, kErrUnphysical);
  const EqCoeffs<R> c = eq_coeffs(M);
  const long long site = (long long)y * s.ldx + x;
  void* const dn0 = s.cur ? s.dn[1] : s.dn[0];
  if (dn0) static_cast<R*>(dn0)[site] = M.dn;     // the electric force's first step
#pragma unroll
  for (int d = 0; d < kDirs; d += 2) {
    R v[8];
    eq_pair<S>(M, c, d, qc, v, v + 4);
    Codec<S>::store4(fout + vec_index(s, d, site), dir_kind(d), qc, v);
    Codec<S>::store4(fout + vec_index(s, d + 1, site), dir_kind(d), qc, v + 4);
  }
}

// Stored state := the Chapman-Enskog seed of the fields (n, u, T): the state
// whose first pull-stream gives f^eq plus its first-order non-equilibrium part
// of a steady flow (steady Eq. discrete-rbe with f - f^eq small and slowly
// varying),
//     f_i(x) = f^eq_i(x) - (f^eq_i(x) - f^eq_i(x - n_i)) / omega_i(x),
// omega_i = gamma (1 - v_i.u) / tau, wherever the source x - n_i lies in the
// sample.  Stored per source site s with d = s + n_i (wrapped on periodic
// axes):  f*_i(s) = f^eq_i(d) - (f^eq_i(d) - f^eq_i(s)) / omega_i(d), and
// f^eq_i(s) where d lies outside (only the bounce-back at s reads it).  The
// relation is affine with unit weight on f^eq, so it holds for the stored
// relative deviations as well.  Each thread evaluates the equilibrium at its
// own site and, for each direction, at the arrival site.
template <typename S, class C>
__device__ __forceinline__ void init_ce_body(S* __restrict__ fout, const DevSample& s,
                                             const double* n, const double* ux,
                                             const double* uy, const double* T, unsigned* err,
                                             const C& qc) {
  using R = typename Codec<S>::R;
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= s.nx) return;
  const long long k = (long long)y * s.nx + x;
  bool ok;
  const Macro<R> M = field_macro<R>(n, ux, uy, T, k, ok);
  if (!ok) atomicOr(err, kErrUnphysical);
  const EqCoeffs<R> c = eq_coeffs(M);
  const long long site = (long long)y * s.ldx + x;
  void* const dn0 = s.cur ? s.dn[1] : s.dn[0];
  if (dn0) static_cast<R*>(dn0)[site] = M.dn;     // the electric force's first step
#pragma unroll 1
  for (int d = 0; d < kDirs; d += 2) {
    R v[8];
    eq_pair<S>(M, c, d, qc, v, v + 4);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int dd = d + h;
      int tx = x + hop_x(dd), ty = y + hop_y(dd);
      if (s.periodic_x) tx = tx < 0 ? tx + s.nx : (tx >= s.nx ? tx - s.nx : tx);
      if (s.periodic_y) ty = ty < 0 ? ty + s.ny : (ty >= s.ny ? ty - s.ny : ty);
      if ((unsigned)tx < (unsigned)s.nx && (unsigned)ty < (unsigned)s.ny) {
        bool okd;
        const Macro<R> Md = field_macro<R>(n, ux, uy, T, (long long)ty * s.nx + tx, okd);
        R ed[8];
        eq_pair<S>(Md, eq_coeffs(Md), d, qc, ed, ed + 4);
        const R vx = R(hop_x(dd)) / R(5), vy = R(hop_y(dd)) / R(5);
        const R om = Md.gamma * (R(1) - (vx * Md.ux + vy * Md.uy)) * R(s.inv_tau);
        const R iom = R(1) / om;
#pragma unroll
        for (int j = 0; j < kShells; ++j)
          v[4 * h + j] = ed[4 * h + j] - (ed[4 * h + j] - v[4 * h + j]) * iom;
      }
    }
    Codec<S>::store4(fout + vec_index(s, d, site), dir_kind(d), qc, v);
    Codec<S>::store4(fout + vec_index(s, d + 1, site), dir_kind(d), qc, v + 4);
  }
}

// Dense FP64 deviations [48][ny][nx]  <->  stored vectors.
// Populations q0 .. q0 + gridDim.z - 1; `out` / `in` point at population q0
// of the dense array.
template <typename S, class C>
__device__ __forceinline__ void get_state_body(const S* __restrict__ fin, const DevSample& s,
                                               int q0, double* out, const C& qc) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y;
  const int dq = blockIdx.z, q = q0 + dq;
  if (x >= s.nx) return;
  const int d = q >> 2, j = q & 3;
  const S v = fin[vec_index(s, d, (long long)y * s.ldx + x) + j];
  out[((long long)dq * s.ny + y) * s.nx + x] = Codec<S>::decode(v, dir_kind(d), j, qc);
}

template <typename S, class C>
__device__ __forceinline__ void set_state_body(S* __restrict__ fout, const DevSample& s, int q0,
                                               const double* in, const C& qc) {
  using R = typename Codec<S>::R;
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y;
  const int dq = blockIdx.z, q = q0 + dq;
  if (x >= s.nx) return;
  const int d = q >> 2, j = q & 3;
  const double v = in[((long long)dq * s.ny + y) * s.nx + x];
  fout[vec_index(s, d, (long long)y * s.ldx + x) + j] = Codec<S>::encode(v, dir_kind(d), j, qc);
}

}  // namespace rlbm

// Massive-particle variant, m = 5 T0 (Sec. 2.3, Fig. m5-stencil): the fused
// stream + collide kernel, its helpers and the C ABI of
// include/rlbm_massive.h.
//
// One thread per site.  Per step (Eq. discrete-rbe): pull the 45 post-
// collision populations (periodic wrap or on-site bounce-back), moments
// N^a, T^ab as deviations from the rest values, Landau frame with the
// massive equation of state, equilibrium, Anderson-Witting relaxation,
// uniform force, store.  Every stored value is the relative deviation
// g_i = (f_i - f0_i) / f0_i from the rest populations f0_i = w_i / (m + 1)
// (f^eq at n = T = 1, u = 0).
//
// Equilibrium.  g^eq_i = (m + 1) m(p_i)^T G^-1 M(n, U, T) - 1 (projection
// of the Maxwell-Juttner distribution onto the polynomials of degree <= 3,
// Eq. feq-expansion-discrete; m the 16 monomials, G their Gram matrix
// under the weight function, M their Maxwell-Juttner moments).  The
// entries of (m + 1) m^T G^-1 reach 3e4 (1 and p0 are nearly collinear on
// the nodes), so the kernel never applies them to rounded O(delta) moments:
// with delta = (n - 1, T - 1, ux, uy),
//   g^eq_i = dn + L_i . (dT, ux, uy) + W_i . (quadratic monomials of delta)
//          + B_i . R3(delta),
// L and W exact per-node tables, and R3 the moments minus their linear and
// quadratic parts, written out below without cancellation (each term is a
// product of small factors).  The Maxwell-Juttner moments are
//   M[1] = n / (m + T),   M[p^a] = n U^a,   M[p^a p^b] = h U^a U^b - P eta^ab,
//   M[p^a p^b p^c] = alpha U^a U^b U^c - T h (U^a eta^bc + U^b eta^ac + U^c eta^ab),
// with P = n T, h = eps + P = n (m^2 + 3 m T + 3 T^2) / (m + T) and
// alpha = n (m^3 + 6 m^2 T + 15 m T^2 + 15 T^3) / (m + T) (rest-frame
// integrals of exp(-p0 / T) on the mass shell).
#include "rlbm_massive.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "massive_tables.h"

namespace rlbm {
namespace massive {
namespace {

// physical constants at T0 = 1, m = 5
constexpr double kM = kMass;
constexpr double kM1 = kMass + 1;
constexpr double kE0 = (kM * kM + 2 * kM + 2) / kM1;            // eps at rest   37/6
constexpr double kH0 = (kM * kM + 3 * kM + 3) / kM1;            // eps + P       43/6
constexpr double kK1 = (2 * kM * kM + 6 * kM + 3) / (kM1 * kM1); // dh/dT          83/36
constexpr double kA0 = (kM * kM * kM + 6 * kM * kM + 15 * kM + 15) / kM1;   // alpha 365/6
constexpr double kC2 = kM * kM / (kM1 * kM1 * kM1);             // 25/216
constexpr double kSD0 = 2 * kM + 4 - kE0;                        // sqrt of the EOS discriminant at rest

constexpr unsigned kErrNonFinite = 1u, kErrUnphysical = 2u, kErrNoConvergence = 4u;

template <typename R>
struct MConsts {
  R vx[kPairs], vy[kPairs];
  R mN0[kPairs], mE[kPairs], mPxx[kPairs], mPxy[kPairs], mPyy[kPairs];
  R mNx[kPairs], mNy[kPairs], mMx[kPairs], mMy[kPairs];
  R LT[kPairs], LX[kPairs], LY[kPairs];
  R WE[kPairs][5], WO[kPairs][4];
  R BE[kPairs][8], BO[kPairs][8];
  R mvE[kPairs][8], mvO[kPairs][8];
  R gi[16][16];
  R restN0, restE, restLT, restWE[5], restBE[8];
  double f0[kQm];
};

__constant__ MConsts<float> c_f;
__constant__ MConsts<double> c_d;

template <typename R> __device__ __forceinline__ const MConsts<R>& mc();
template <> __device__ __forceinline__ const MConsts<float>& mc<float>() { return c_f; }
template <> __device__ __forceinline__ const MConsts<double>& mc<double>() { return c_d; }

__device__ __forceinline__ double mdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float mdiv(float a, float b) { return __fdividef(a, b); }

template <typename R> struct MTol;
template <> struct MTol<double> { static constexpr double v = 1e-15; };
template <> struct MTol<float> { static constexpr float v = 2e-7f; };

// library monomial order (massive_tables.h): exponents of p0, px, py
__host__ __device__ constexpr int mon_b(int k) {
  return k == 2 ? 2 : k == 3 ? 1 : k == 5 ? 2 : k == 6 ? 1 : k == 8 ? 1 : k == 10 ? 1 : k == 12 ? 3
       : k == 13 ? 2 : k == 14 ? 1 : 0;
}
__host__ __device__ constexpr int mon_c(int k) {
  return k == 3 ? 1 : k == 4 ? 2 : k == 6 ? 1 : k == 7 ? 2 : k == 9 ? 1 : k == 11 ? 1 : k == 13 ? 1
       : k == 14 ? 2 : k == 15 ? 3 : 0;
}
// G couples two monomials only if their px and py exponents have equal parities
__host__ __device__ constexpr bool same_block(int a, int b) {
  return ((mon_b(a) ^ mon_b(b)) & 1) == 0 && ((mon_c(a) ^ mon_c(b)) & 1) == 0;
}

struct MGeom {
  int nx, ny, ldx;
  int px, py;            // periodic axes
  long long plane;       // elements per population plane
};

template <typename R>
struct MMacro {
  R ux, uy, gamma, gm1, s;   // s = sqrt(1 - u^2), gm1 = gamma - 1
  R dn, dT;                  // n - 1, T - 1
};

template <typename R>
struct MMom {
  R dN0, dNx, dNy;           // N^a - (1, 0, 0)
  R dE, Mx, My;              // T^00 - eps0, T^0x, T^0y
  R dPxx, dPxy, dPyy;        // T^ij - delta_ij
};

// ---------------------------------------------------------------------------
// Pull streaming: f_i(x) = f*_i(x - n_i); a source outside a walled axis
// bounces back (the opposite population of the destination site).
// ---------------------------------------------------------------------------
template <typename S>
__device__ __forceinline__ void mpull(const S* __restrict__ src, const MGeom& g, int x, int y,
                                      S (&f)[kQm]) {
  const long long site = (long long)y * g.ldx + x;
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 2 * p + h;
      const int ex = h ? -pair_x(p) : pair_x(p);
      const int ey = h ? -pair_y(p) : pair_y(p);
      int sx = x - ex, sy = y - ey;
      bool in = true;
      if (ex != 0) {
        if (g.px) { sx += sx < 0 ? g.nx : 0; sx -= sx >= g.nx ? g.nx : 0; }
        else in = sx >= 0 && sx < g.nx;
      }
      if (ey != 0) {
        if (g.py) { sy += sy < 0 ? g.ny : 0; sy -= sy >= g.ny ? g.ny : 0; }
        else in = in && sy >= 0 && sy < g.ny;
      }
      const S* ptr = in ? src + (long long)i * g.plane + (long long)sy * g.ldx + sx
                        : src + (long long)(i ^ 1) * g.plane + site;
      f[i] = __ldg(ptr);
    }
  }
  f[kRestPop] = __ldg(src + (long long)kRestPop * g.plane + site);
}

// The same for a block lying at least kReach sites inside every edge: no
// wrap, no bounce-back; each offset is uniform across the block.
template <typename S>
__device__ __forceinline__ void mpull_interior(const S* __restrict__ src, const MGeom& g,
                                               long long site, S (&f)[kQm]) {
  const S* base = src + site;
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 2 * p + h;
      const int ex = h ? -pair_x(p) : pair_x(p);
      const int ey = h ? -pair_y(p) : pair_y(p);
      f[i] = __ldg(base + ((long long)i * g.plane - (long long)ey * g.ldx - ex));
    }
  }
  f[kRestPop] = __ldg(base + (long long)kRestPop * g.plane);
}

__device__ __forceinline__ bool block_interior(const MGeom& g) {
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 4;
  return x0 >= kReach && x0 + 31 < g.nx - kReach && y0 >= kReach && y0 + 3 < g.ny - kReach;
}

template <typename R>
__device__ __forceinline__ MMom<R> mmoments(const R (&g)[kQm]) {
  const MConsts<R>& c = mc<R>();
  MMom<R> m;
  m.dN0 = m.dNx = m.dNy = m.dE = m.Mx = m.My = m.dPxx = m.dPxy = m.dPyy = R(0);
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    const R se = g[2 * p] + g[2 * p + 1], so = g[2 * p] - g[2 * p + 1];
    m.dN0 = fma(c.mN0[p], se, m.dN0);
    m.dE = fma(c.mE[p], se, m.dE);
    if (pair_x(p) != 0) {
      m.dPxx = fma(c.mPxx[p], se, m.dPxx);
      m.dNx = fma(c.mNx[p], so, m.dNx);
      m.Mx = fma(c.mMx[p], so, m.Mx);
    }
    if (pair_y(p) != 0) {
      m.dPyy = fma(c.mPyy[p], se, m.dPyy);
      m.dNy = fma(c.mNy[p], so, m.dNy);
      m.My = fma(c.mMy[p], so, m.My);
    }
    if (pair_x(p) != 0 && pair_y(p) != 0) m.dPxy = fma(c.mPxy[p], se, m.dPxy);
  }
  m.dN0 = fma(c.restN0, g[kRestPop], m.dN0);
  m.dE = fma(c.restE, g[kRestPop], m.dE);
  return m;
}

// Landau frame eps U^a = T^ab U_b: u = (Pi + eps I)^-1 M, Newton on
// eps - E + M.u(eps) (derivative 1 - u.u) from eps = E; n = U_a N^a; T from
// eps / n = (m^2 + 2 m T + 2 T^2) / (m + T).
template <typename R>
__device__ __forceinline__ bool mlandau(const MMom<R>& M, MMacro<R>& o) {
  R deps = M.dE, ux = R(0), uy = R(0);
  bool conv = false;
#pragma unroll 1
  for (int it = 0; it < 16; ++it) {
    const R a = R(kH0) + M.dPxx + deps, c = R(kH0) + M.dPyy + deps;
    const R inv = mdiv(R(1), a * c - M.dPxy * M.dPxy);
    ux = (c * M.Mx - M.dPxy * M.My) * inv;
    uy = (a * M.My - M.dPxy * M.Mx) * inv;
    const R gf = deps - M.dE + M.Mx * ux + M.My * uy;
    const R step = mdiv(gf, R(1) - ux * ux - uy * uy);
    deps -= step;
    if (fabs(step) <= MTol<R>::v * (R(kE0) + fabs(deps))) { conv = true; break; }
  }
  {
    const R a = R(kH0) + M.dPxx + deps, c = R(kH0) + M.dPyy + deps;
    const R inv = mdiv(R(1), a * c - M.dPxy * M.dPxy);
    ux = (c * M.Mx - M.dPxy * M.My) * inv;
    uy = (a * M.My - M.dPxy * M.Mx) * inv;
  }
  const R u2 = ux * ux + uy * uy;
  const R s = sqrt(R(1) - u2);
  const R gamma = mdiv(R(1), s);
  const R gm1 = mdiv(u2 * gamma, R(1) + s);
  const R dNpar = M.dN0 - ux * M.dNx - uy * M.dNy;     // U_a N^a / gamma - 1
  const R dn = gm1 * (R(1) + dNpar) + dNpar;
  // T - 1 = (de + sqrt(D) - sqrt(D0)) / 4,  D = e^2 + 4 m e - 4 m^2,  e = eps / n
  const R de = mdiv(deps - R(kE0) * dn, R(1) + dn);
  const R e = R(kE0) + de;
  const R sD = sqrt(e * e + R(4 * kM) * e - R(4 * kM * kM));
  const R dT = R(0.25) * de * (R(1) + mdiv(e + R(kE0 + 4 * kM), sD + R(kSD0)));
  o.ux = ux; o.uy = uy; o.gamma = gamma; o.gm1 = gm1; o.s = s; o.dn = dn; o.dT = dT;
  return conv;
}

template <typename R>
__device__ __forceinline__ MMacro<R> macro_of(R n, R ux, R uy, R T) {
  MMacro<R> M;
  const R u2 = ux * ux + uy * uy;
  M.ux = ux; M.uy = uy;
  M.s = sqrt(R(1) - u2);
  M.gamma = mdiv(R(1), M.s);
  M.gm1 = mdiv(u2 * M.gamma, R(1) + M.s);
  M.dn = n - R(1);
  M.dT = T - R(1);
  return M;
}

// Per-site part of the equilibrium: delta, its quadratic monomials and the
// third-order remainder R3 of the 16 moments (library order).
template <typename R>
struct EqSite {
  R dn, dT, ux, uy;
  R qE[5];      // dn dT, dT^2, ux^2, ux uy, uy^2
  R qO[4];      // dn ux, dn uy, dT ux, dT uy
  R E[8], O[8];
};

template <typename R>
__device__ __forceinline__ EqSite<R> eq_site(const MMacro<R>& M) {
  const R m = R(kM), m1 = R(kM1), one = R(1);
  const R H0 = R(kH0), K1 = R(kK1), A0 = R(kA0);
  const R dn = M.dn, dT = M.dT, ux = M.ux, uy = M.uy;
  const R g = M.gamma, gm1 = M.gm1, s = M.s;
  const R u2 = ux * ux + uy * uy;
  const R T = one + dT;
  const R imT = mdiv(one, m + T);
  const R im1 = R(1.0 / kM1);
  const R gm1mh = u2 * (u2 * mdiv(one, one + s) + R(2) * gm1) * mdiv(R(0.5), one + s);   // gm1 - u^2/2
  const R phi = (m * m + R(3) * m * T + R(3) * T * T) * imT;                        // h / n
  const R kT = (R(3) * m1 * T + R(2) * m * m + R(3) * m) * imT * im1;               // (phi(T) - phi(1)) / dT
  const R aT = (m * m * m + R(6) * m * m * T + R(15) * m * T * T + R(15) * T * T * T) * imT;   // alpha / n
  const R kaT = R(5) * (R(3) * m1 * T * T + R(3) * m1 * m1 * T + m * (m * m + R(3) * m + R(3))) * imT * im1;
  const R dh = dn * phi + dT * kT;                                  // h - h0
  const R dT2 = dT * dT;
  const R dhq = dn * dT * kT + dT2 * (m * m) * imT * (im1 * im1);     // dh - h0 dn - k1 dT
  const R da = dn * aT + dT * kaT;                                  // alpha - alpha0
  const R g2 = g * g;
  const R g2m1 = g2 * u2;                                           // gamma^2 - 1
  const R g3m1 = gm1 * (g2 + g + one);                              // gamma^3 - 1
  const R hg2m = dh * g2 + H0 * g2m1;                               // h gamma^2 - h0
  const R hg2mq = dhq * g2 + (H0 * dn + K1 * dT) * g2m1 + H0 * g2m1;
  const R ag3m = da * g2 * g + A0 * g3m1;                           // alpha gamma^3 - alpha0
  const R ag3 = A0 + ag3m;                                          // alpha gamma^3
  const R Xlin = H0 * dn + (K1 + H0) * dT;
  const R XmXl = dhq + dT * dh;                                     // (T h - h0) - Xlin
  const R XmXl2 = dn * dT * (K1 + H0) + dT2 * (K1 + R(kC2));        // its quadratic part
  const R XmXl3 = dn * dT2 * (m * m) * imT * (im1 * im1) - dT2 * dT * (m * m) * imT * (im1 * im1 * im1)
                + dT * dhq;
  const R Rthg = XmXl * g + (Xlin + H0) * gm1;                      // T h gamma - h0 - Xlin
  const R Rthg3 = XmXl3 * g + XmXl2 * gm1 + Xlin * gm1 + H0 * gm1mh;
  EqSite<R> e;
  e.dn = dn; e.dT = dT; e.ux = ux; e.uy = uy;
  e.qE[0] = dn * dT; e.qE[1] = dT2; e.qE[2] = ux * ux; e.qE[3] = ux * uy; e.qE[4] = uy * uy;
  e.qO[0] = dn * ux; e.qO[1] = dn * uy; e.qO[2] = dT * ux; e.qO[3] = dT * uy;
  e.E[0] = (dn * m1 - dT) * dT2 * imT * (im1 * im1 * im1);
  e.E[1] = gm1mh + gm1 * dn;
  e.E[2] = hg2m * e.qE[2];
  e.E[3] = hg2m * e.qE[3];
  e.E[4] = hg2m * e.qE[4];
  e.E[5] = ag3m * e.qE[2] + Rthg3;
  e.E[6] = ag3m * e.qE[3];
  e.E[7] = ag3m * e.qE[4] + Rthg3;
  const R ngm = gm1 * (one + dn);
  e.O[0] = ngm * ux;
  e.O[1] = ngm * uy;
  e.O[2] = hg2mq * ux;
  e.O[3] = hg2mq * uy;
  e.O[4] = (ag3 * e.qE[2] + R(3) * Rthg) * ux;
  e.O[5] = ag3 * e.qE[2] * uy + Rthg * uy;
  e.O[6] = ag3 * e.qE[4] * ux + Rthg * ux;
  e.O[7] = (ag3 * e.qE[4] + R(3) * Rthg) * uy;
  return e;
}

// Parities in (ux, uy) / (px, py) of the table columns: a node on an axis
// is its own mirror image across that axis, so every entry odd in the other
// component vanishes there.  WE: dn dT, dT^2, ux^2, ux uy, uy^2; WO: dn ux,
// dn uy, dT ux, dT uy; BE / BO: the E / O monomials.
__host__ __device__ constexpr bool we_odd(int k) { return k == 3; }                 // in x and in y
__host__ __device__ constexpr bool wo_x(int k) { return k == 0 || k == 2; }         // odd in x only
__host__ __device__ constexpr bool be_odd(int k) { return k == 3 || k == 6; }       // in x and in y
__host__ __device__ constexpr bool bo_x(int k) { return k == 0 || k == 2 || k == 4 || k == 6; }
// whether a column with the given parities can be nonzero at pair p
__host__ __device__ constexpr bool live(int p, bool odd_x, bool odd_y) {
  return !((odd_x && pair_x(p) == 0) || (odd_y && pair_y(p) == 0));
}

// even and odd parts of g^eq for pair p (g^eq of 2p = even + odd, of 2p+1 = even - odd)
template <typename R>
__device__ __forceinline__ void eq_pair(const EqSite<R>& e, int p, R& even, R& odd) {
  const MConsts<R>& c = mc<R>();
  R ev = fma(c.LT[p], e.dT, e.dn);
#pragma unroll
  for (int k = 0; k < 5; ++k)
    if (live(p, we_odd(k), we_odd(k))) ev = fma(c.WE[p][k], e.qE[k], ev);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (live(p, be_odd(k), be_odd(k))) ev = fma(c.BE[p][k], e.E[k], ev);
  R od = R(0);
  if (pair_x(p) != 0) od = fma(c.LX[p], e.ux, od);
  if (pair_y(p) != 0) od = fma(c.LY[p], e.uy, od);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (live(p, wo_x(k), !wo_x(k))) od = fma(c.WO[p][k], e.qO[k], od);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (live(p, bo_x(k), !bo_x(k))) od = fma(c.BO[p][k], e.O[k], od);
  even = ev;
  odd = od;
}

// Couples of pairs with the same axis pattern (both on the x axis, both on
// the y axis, or both off the axes), so that every term eq_pair() skips for
// one pair is skipped for the other: the FP32 collision evaluates g^eq of a
// couple on register pairs, lanes (first pair, second pair).
constexpr int kCouples = kPairs / 2;
__host__ __device__ constexpr int couple_a(int q) {
  return q == 0 ? 0 : q == 1 ? 1 : q == 2 ? 2 : q == 3 ? 6 : q == 4 ? 8 : q == 5 ? 10 : q == 6 ? 12 : q == 7 ? 13 : q == 8 ? 14 : q == 9 ? 16 : 18;
}
__host__ __device__ constexpr int couple_b(int q) {
  return q == 0 ? 4 : q == 1 ? 5 : q == 2 ? 3 : q == 3 ? 7 : q == 4 ? 9 : q == 5 ? 11 : q == 6 ? 20 : q == 7 ? 21 : q == 8 ? 15 : q == 9 ? 17 : 19;
}
constexpr bool couples_valid() {
  int seen[kPairs] = {};
  for (int q = 0; q < kCouples; ++q) {
    const int a = couple_a(q), b = couple_b(q);
    if ((pair_x(a) == 0) != (pair_x(b) == 0) || (pair_y(a) == 0) != (pair_y(b) == 0)) return false;
    ++seen[a];
    ++seen[b];
  }
  for (int p = 0; p < kPairs; ++p)
    if (seen[p] != 1) return false;
  return true;
}
static_assert(couples_valid(), "every pair in one couple, both pairs of a couple alike on the axes");

// eq_pair()'s FP32 tables of couple q as pairs (first pair, second pair)
struct MCoupleConsts {
  float2 LT[kCouples], LX[kCouples], LY[kCouples];
  float2 WE[kCouples][5], WO[kCouples][4], BE[kCouples][8], BO[kCouples][8];
  // and the FP32 collision's per-pair constants: vx, vy, mvE[.][1..4], mvO[.][0..1]
  float2 vx[kCouples], vy[kCouples];
  float2 p0[kCouples], px2[kCouples], pxy[kCouples], py2[kCouples], pxv[kCouples], pyv[kCouples];
};
__constant__ MCoupleConsts c_cp;

template <typename R>
__device__ __forceinline__ R eq_rest(const EqSite<R>& e) {
  const MConsts<R>& c = mc<R>();
  R ev = fma(c.restLT, e.dT, e.dn);
#pragma unroll
  for (int k = 0; k < 5; ++k)
    if (!we_odd(k)) ev = fma(c.restWE[k], e.qE[k], ev);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (!be_odd(k)) ev = fma(c.restBE[k], e.E[k], ev);
  return ev;
}

// Forcing: with D(p) = g^eq as a polynomial (coefficients d = (m+1) G^-1 dM,
// dM the full moment deviations), the relative source is
//   F^ext_i / f0_i = (F.v_i)(1 + g^eq_i) - (F.v_i) dD/dp0(p_i) - F.grad_xy D(p_i).
template <typename R>
struct ForceSite {
  R a1, a5, a6, a7, a10, a11;               // dD/dp0 = a1 + a5 px^2 + a6 px py + a7 py^2 + a10 px + a11 py
  R h1, hp0, hxx, hxy, hyy;                 // F.grad_xy D, even part
  R hx, hy, h0x, h0y;                       //              odd part
};

template <typename R>
__device__ __forceinline__ ForceSite<R> force_site(const MMacro<R>& M, R Fx, R Fy) {
  const MConsts<R>& c = mc<R>();
  const R m = R(kM), m1 = R(kM1), one = R(1), H0 = R(kH0);
  const R dn = M.dn, dT = M.dT, ux = M.ux, uy = M.uy, g = M.gamma, gm1 = M.gm1;
  const R T = one + dT, n = one + dn;
  const R imT = mdiv(one, m + T);
  const R phi = (m * m + R(3) * m * T + R(3) * T * T) * imT;
  const R kT = (R(3) * m1 * T + R(2) * m * m + R(3) * m) * imT * R(1.0 / kM1);
  const R dh = dn * phi + dT * kT;
  const R alpha = n * (m * m * m + R(6) * m * m * T + R(15) * m * T * T + R(15) * T * T * T) * imT;
  const R hg2 = (H0 + dh) * g * g;
  const R ag3 = alpha * g * g * g;
  const R X = T * dh + H0 * dT;                       // T h - h0
  const R Thgm = X * g + H0 * gm1;                    // T h gamma - h0
  const R Thg = H0 + Thgm;
  const R P1 = dn + dT + dn * dT;                     // P - 1
  const R ngam = dn + gm1 + dn * gm1;                 // n gamma - 1
  R dM[16];
  dM[0] = (dn * m1 - dT) * imT * R(1.0 / kM1);
  dM[1] = ngam;
  dM[2] = hg2 * ux * ux + P1;
  dM[3] = hg2 * ux * uy;
  dM[4] = hg2 * uy * uy + P1;
  dM[5] = ag3 * ux * ux + Thgm;
  dM[6] = ag3 * ux * uy;
  dM[7] = ag3 * uy * uy + Thgm;
  dM[8] = (one + ngam) * ux;
  dM[9] = (one + ngam) * uy;
  dM[10] = hg2 * ux;
  dM[11] = hg2 * uy;
  dM[12] = (ag3 * ux * ux + R(3) * Thg) * ux;
  dM[13] = (ag3 * ux * ux + Thg) * uy;
  dM[14] = (ag3 * uy * uy + Thg) * ux;
  dM[15] = (ag3 * uy * uy + R(3) * Thg) * uy;
  R d[16];
#pragma unroll
  for (int a = 0; a < 16; ++a) {
    R s = R(0);
#pragma unroll
    for (int b = 0; b < 16; ++b)
      if (same_block(a, b)) s = fma(c.gi[a][b], dM[b], s);
    d[a] = s;
  }
  ForceSite<R> f;
  f.a1 = d[1]; f.a5 = d[5]; f.a6 = d[6]; f.a7 = d[7]; f.a10 = d[10]; f.a11 = d[11];
  f.h1 = Fx * d[8] + Fy * d[9];
  f.hp0 = Fx * d[10] + Fy * d[11];
  f.hxx = R(3) * Fx * d[12] + Fy * d[13];
  f.hxy = R(2) * Fx * d[13] + R(2) * Fy * d[14];
  f.hyy = Fx * d[14] + R(3) * Fy * d[15];
  f.hx = R(2) * Fx * d[2] + Fy * d[3];
  f.hy = Fx * d[3] + R(2) * Fy * d[4];
  f.h0x = R(2) * Fx * d[5] + Fy * d[6];
  f.h0y = Fx * d[6] + R(2) * Fy * d[7];
  return f;
}

// ---------------------------------------------------------------------------
// Collision of one site and store.
// ---------------------------------------------------------------------------
// Sign pairs of the paired FP32 arithmetic below (constant memory, so that
// they cost nothing as operands): (1, -1) and (-1, 1).
__constant__ float2 c_pm = {1.f, -1.f};
__constant__ float2 c_mp = {-1.f, 1.f};

__device__ __forceinline__ float2 S2(float a) { return make_float2(a, a); }

// eq_pair() of the two pairs of couple q at once (lanes: couple_a(q),
// couple_b(q)): the same terms in the same order on each lane.
__device__ __forceinline__ void eq_couple(const EqSite<float>& e, int q, float2& even,
                                          float2& odd) {
  const int p = couple_a(q);   // the couple's axis pattern
  float2 ev = __ffma2_rn(c_cp.LT[q], S2(e.dT), S2(e.dn));
#pragma unroll
  for (int k = 0; k < 5; ++k)
    if (live(p, we_odd(k), we_odd(k))) ev = __ffma2_rn(c_cp.WE[q][k], S2(e.qE[k]), ev);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (live(p, be_odd(k), be_odd(k))) ev = __ffma2_rn(c_cp.BE[q][k], S2(e.E[k]), ev);
  float2 od = S2(0.f);
  if (pair_x(p) != 0) od = __ffma2_rn(c_cp.LX[q], S2(e.ux), od);
  if (pair_y(p) != 0) od = __ffma2_rn(c_cp.LY[q], S2(e.uy), od);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (live(p, wo_x(k), !wo_x(k))) od = __ffma2_rn(c_cp.WO[q][k], S2(e.qO[k]), od);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (live(p, bo_x(k), !bo_x(k))) od = __ffma2_rn(c_cp.BO[q][k], S2(e.O[k]), od);
  even = ev;
  odd = od;
}

// mcollide_store for FP32 on register pairs (lanes: population 2p and its
// opposite 2p + 1): the same quantities in the same order of operations per
// population, two populations per paired FMA (Blackwell's FFMA2); g^eq of
// two pairs at a time (eq_couple).
template <bool FORCE>
__device__ __forceinline__ void mcollide_store_paired(const float (&g)[kQm], const MMacro<float>& M,
                                                      float inv_tau, float Fx, float Fy,
                                                      float* __restrict__ out, long long plane) {
  const EqSite<float> e = eq_site(M);
  const float gt = M.gamma * inv_tau;
  const float gux = gt * M.ux, guy = gt * M.uy;
  ForceSite<float> fs;
  if (FORCE) fs = force_site(M, Fx, Fy);
  // relaxation, force and store of pair p from the even / odd parts of its
  // g^eq, v.u gamma / tau (wv) and the force's per-pair scalars
  auto relax_pair = [&](const int p, const float ev, const float od, const float wv,
                        const float Ae, const float He, const float Ao, const float Ho,
                        const float Fv) {
    const float2 om = __ffma2_rn(S2(wv), c_mp, S2(gt));       // gamma (1 -+ v.u) / tau
    const float2 gpn = __ffma2_rn(S2(od), c_pm, S2(ev));      // (ev + od, ev - od)
    const float2 G = make_float2(g[2 * p], g[2 * p + 1]);
    float2 o = __ffma2_rn(om, __ffma2_rn(G, S2(-1.f), gpn), G);
    if (FORCE) {
      // lanes: +-Fv (1 + g^eq -/+ ... - Ae -+ Ao) - He -+ Ho
      const float2 X = __ffma2_rn(S2(Ao), c_mp, __fadd2_rn(gpn, S2(1.f - Ae)));
      o = __ffma2_rn(S2(Fv), __fmul2_rn(X, c_pm), o);
      o = __ffma2_rn(S2(Ho), c_mp, __fadd2_rn(o, S2(-He)));
    }
    out[(long long)(2 * p) * plane] = o.x;
    out[(long long)(2 * p + 1) * plane] = o.y;
  };
  // the per-pair scalars of a couple on register pairs (lanes: couple_a(q),
  // couple_b(q)), each lane with the operations of one pair in their order
#pragma unroll
  for (int q = 0; q < kCouples; ++q) {
    const int p = couple_a(q);   // the couple's axis pattern
    const bool hx = pair_x(p) != 0, hy = pair_y(p) != 0;
    float2 ev, od;
    eq_couple(e, q, ev, od);
    float2 wv = S2(0.f);
    if (hx) wv = __fmul2_rn(S2(gux), c_cp.vx[q]);
    if (hy) wv = __ffma2_rn(S2(guy), c_cp.vy[q], wv);
    float2 Ae = S2(0.f), He = S2(0.f), Ao = S2(0.f), Ho = S2(0.f), Fv = S2(0.f);
    if (FORCE) {
      const float2 px2 = c_cp.px2[q], pxy = c_cp.pxy[q], py2 = c_cp.py2[q], p0 = c_cp.p0[q];
      Ae = __ffma2_rn(S2(fs.a5), px2, S2(fs.a1));
      He = __ffma2_rn(S2(fs.hp0), p0, S2(fs.h1));
      Ae = __ffma2_rn(S2(fs.a6), pxy, __ffma2_rn(S2(fs.a7), py2, Ae));
      He = __ffma2_rn(S2(fs.hxx), px2, __ffma2_rn(S2(fs.hxy), pxy, __ffma2_rn(S2(fs.hyy), py2, He)));
      if (hx) {
        Ao = __fmul2_rn(S2(fs.a10), c_cp.pxv[q]);
        Ho = __ffma2_rn(__ffma2_rn(S2(fs.h0x), p0, S2(fs.hx)), c_cp.pxv[q], Ho);
      }
      if (hy) {
        Ao = __ffma2_rn(S2(fs.a11), c_cp.pyv[q], Ao);
        Ho = __ffma2_rn(__ffma2_rn(S2(fs.h0y), p0, S2(fs.hy)), c_cp.pyv[q], Ho);
      }
      if (hx) Fv = __fmul2_rn(S2(Fx), c_cp.vx[q]);
      if (hy) Fv = __ffma2_rn(S2(Fy), c_cp.vy[q], Fv);
    }
    relax_pair(couple_a(q), ev.x, od.x, wv.x, Ae.x, He.x, Ao.x, Ho.x, Fv.x);
    relax_pair(couple_b(q), ev.y, od.y, wv.y, Ae.y, He.y, Ao.y, Ho.y, Fv.y);
  }
  const float gr = eq_rest(e);
  float orr = fmaf(gt, gr - g[kRestPop], g[kRestPop]);
  if (FORCE) orr -= fmaf(fs.hp0, float(kM), fs.h1);
  out[(long long)kRestPop * plane] = orr;
}

template <typename R, bool FORCE>
__device__ __forceinline__ void mcollide_store(const R (&g)[kQm], const MMacro<R>& M, R inv_tau,
                                               R Fx, R Fy, R* __restrict__ out, long long plane) {
  if constexpr (sizeof(R) == sizeof(float)) {
    mcollide_store_paired<FORCE>(g, M, inv_tau, Fx, Fy, out, plane);
    return;
  }
  const MConsts<R>& c = mc<R>();
  const EqSite<R> e = eq_site(M);
  const R gt = M.gamma * inv_tau;
  const R gux = gt * M.ux, guy = gt * M.uy;
  ForceSite<R> fs;
  if (FORCE) fs = force_site(M, Fx, Fy);
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    R ev, od;
    eq_pair(e, p, ev, od);
    R wv = R(0);
    if (pair_x(p) != 0) wv = gux * c.vx[p];
    if (pair_y(p) != 0) wv = fma(guy, c.vy[p], wv);
    const R omp = gt - wv, omn = gt + wv;          // gamma (1 -+ v.u) / tau
    const R gp = ev + od, gn = ev - od;
    R op = fma(omp, gp - g[2 * p], g[2 * p]);
    R on = fma(omn, gn - g[2 * p + 1], g[2 * p + 1]);
    if (FORCE) {
      const R px2 = c.mvE[p][2], pxy = c.mvE[p][3], py2 = c.mvE[p][4], p0 = c.mvE[p][1];
      const R pxv = c.mvO[p][0], pyv = c.mvO[p][1];
      R Ae = fma(fs.a5, px2, fs.a1), Ao = R(0), He = fma(fs.hp0, p0, fs.h1), Ho = R(0);
      Ae = fma(fs.a6, pxy, fma(fs.a7, py2, Ae));
      He = fma(fs.hxx, px2, fma(fs.hxy, pxy, fma(fs.hyy, py2, He)));
      if (pair_x(p) != 0) { Ao = fs.a10 * pxv; Ho = fma(fma(fs.h0x, p0, fs.hx), pxv, Ho); }
      if (pair_y(p) != 0) { Ao = fma(fs.a11, pyv, Ao); Ho = fma(fma(fs.h0y, p0, fs.hy), pyv, Ho); }
      R Fv = R(0);
      if (pair_x(p) != 0) Fv = Fx * c.vx[p];
      if (pair_y(p) != 0) Fv = fma(Fy, c.vy[p], Fv);
      op += Fv * (R(1) + gp - Ae - Ao) - He - Ho;
      on += -Fv * (R(1) + gn - Ae + Ao) - He + Ho;
    }
    out[(long long)(2 * p) * plane] = op;
    out[(long long)(2 * p + 1) * plane] = on;
  }
  const R gr = eq_rest(e);
  R orr = fma(gt, gr - g[kRestPop], g[kRestPop]);
  if (FORCE) orr -= fma(fs.hp0, R(kM), fs.h1);
  out[(long long)kRestPop * plane] = orr;
}

template <typename R>
__device__ __forceinline__ unsigned check_bits(const MMacro<R>& M, bool conv) {
  unsigned bits = conv ? 0u : kErrNoConvergence;
  if (!(isfinite(M.ux) && isfinite(M.uy) && isfinite(M.dn) && isfinite(M.dT))) bits |= kErrNonFinite;
  else if (!(M.ux * M.ux + M.uy * M.uy < R(1) && M.dn > R(-1) && M.dT > R(-1))) bits |= kErrUnphysical;
  return bits;
}

// ---------------------------------------------------------------------------
// Kernels (blocks of 32 x 4 sites)
// ---------------------------------------------------------------------------
template <typename R, bool FORCE>
__device__ __forceinline__ void mstep_body(const R* __restrict__ src, R* __restrict__ dst,
                                           const MGeom& geo, R inv_tau, R Fx, R Fy,
                                           unsigned* __restrict__ err) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y;
  if (x >= geo.nx || y >= geo.ny) return;
  R g[kQm];
  if (block_interior(geo)) mpull_interior(src, geo, (long long)y * geo.ldx + x, g);
  else mpull(src, geo, x, y, g);
  const MMom<R> mo = mmoments(g);
  MMacro<R> M;
  const bool conv = mlandau(mo, M);
  const unsigned bits = check_bits(M, conv);
  mcollide_store<R, FORCE>(g, M, inv_tau, Fx, Fy, dst + (long long)y * geo.ldx + x, geo.plane);
  if (bits) atomicOr(err, bits);
}

template <typename R, bool FORCE>
__global__ void __launch_bounds__(128) k_mstep(const R* __restrict__ src, R* __restrict__ dst,
                                               MGeom geo, R inv_tau, R Fx, R Fy,
                                               unsigned* __restrict__ err) {
  mstep_body<R, FORCE>(src, dst, geo, inv_tau, Fx, Fy, err);
}

// FP32 with the force: at most 128 registers, so that 4 blocks stay resident
// per SM (the paired equilibrium would otherwise take 130 and leave room for 3).
__global__ void __launch_bounds__(128, 4) k_mstep_f32_force(const float* __restrict__ src,
                                                            float* __restrict__ dst, MGeom geo,
                                                            float inv_tau, float Fx, float Fy,
                                                            unsigned* __restrict__ err) {
  mstep_body<float, true>(src, dst, geo, inv_tau, Fx, Fy, err);
}

template <typename R>
__global__ void __launch_bounds__(128) k_mmoments(const R* __restrict__ src, MGeom geo,
                                                  double* __restrict__ n, double* __restrict__ ux,
                                                  double* __restrict__ uy, double* __restrict__ T,
                                                  unsigned* __restrict__ err) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y;
  if (x >= geo.nx || y >= geo.ny) return;
  R g[kQm];
  mpull(src, geo, x, y, g);
  MMacro<R> M;
  const bool conv = mlandau(mmoments(g), M);
  const long long o = (long long)y * geo.nx + x;
  if (n) n[o] = 1.0 + (double)M.dn;
  if (ux) ux[o] = M.ux;
  if (uy) uy[o] = M.uy;
  if (T) T[o] = 1.0 + (double)M.dT;
  const unsigned bits = check_bits(M, conv);
  if (bits) atomicOr(err, bits);
}

template <typename R>
__global__ void __launch_bounds__(128) k_minit(R* __restrict__ dst, MGeom geo, const double* __restrict__ n,
                                               const double* __restrict__ ux, const double* __restrict__ uy,
                                               const double* __restrict__ T, unsigned* __restrict__ err) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y;
  if (x >= geo.nx || y >= geo.ny) return;
  const long long o = (long long)y * geo.nx + x;
  const double u2 = ux[o] * ux[o] + uy[o] * uy[o];
  if (!(u2 < 1.0 && n[o] > 0.0 && T[o] > 0.0)) { atomicOr(err, kErrUnphysical); return; }
  const MMacro<R> M = macro_of<R>(R(n[o]), R(ux[o]), R(uy[o]), R(T[o]));
  const EqSite<R> e = eq_site(M);
  R* out = dst + (long long)y * geo.ldx + x;
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    R ev, od;
    eq_pair(e, p, ev, od);
    out[(long long)(2 * p) * geo.plane] = ev + od;
    out[(long long)(2 * p + 1) * geo.plane] = ev - od;
  }
  out[(long long)kRestPop * geo.plane] = eq_rest(e);
}

// state I/O: delta_i = f0_i g_i in FP64, dense [45][ny][nx]
template <typename R>
__global__ void k_mget(const R* __restrict__ src, MGeom geo, double* __restrict__ delta) {
  const long long nsite = (long long)geo.nx * geo.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nsite * kQm;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / nsite);
    const long long r = t - i * nsite;
    const int y = (int)(r / geo.nx), x = (int)(r - (long long)y * geo.nx);
    delta[t] = (double)src[(long long)i * geo.plane + (long long)y * geo.ldx + x] * mc<R>().f0[i];
  }
}

template <typename R>
__global__ void k_mset(R* __restrict__ dst, MGeom geo, const double* __restrict__ delta) {
  const long long nsite = (long long)geo.nx * geo.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nsite * kQm;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / nsite);
    const long long r = t - i * nsite;
    const int y = (int)(r / geo.nx), x = (int)(r - (long long)y * geo.nx);
    dst[(long long)i * geo.plane + (long long)y * geo.ldx + x] = (R)(delta[t] / mc<R>().f0[i]);
  }
}

// sum over sites of |u - u_prev|^2 and |u|^2 into acc[0], acc[1] (FP64):
// warp shuffles, one pair of atomics per warp
__global__ void k_mresidual(const double* __restrict__ uxp, const double* __restrict__ uyp,
                            const double* __restrict__ ux, const double* __restrict__ uy,
                            long long nsite, double* __restrict__ acc) {
  double a = 0.0, b = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nsite;
       t += (long long)gridDim.x * blockDim.x) {
    const double dx = ux[t] - uxp[t], dy = uy[t] - uyp[t];
    a = fma(dx, dx, fma(dy, dy, a));
    b = fma(ux[t], ux[t], fma(uy[t], uy[t], b));
  }
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

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
thread_local std::string g_error;

template <typename R>
void fill_consts(const Tables& t, MConsts<R>& c) {
  for (int p = 0; p < kPairs; ++p) {
    c.vx[p] = (R)t.vx[p]; c.vy[p] = (R)t.vy[p];
    c.mN0[p] = (R)t.mN0[p]; c.mE[p] = (R)t.mE[p];
    c.mPxx[p] = (R)t.mPxx[p]; c.mPxy[p] = (R)t.mPxy[p]; c.mPyy[p] = (R)t.mPyy[p];
    c.mNx[p] = (R)t.mNx[p]; c.mNy[p] = (R)t.mNy[p]; c.mMx[p] = (R)t.mMx[p]; c.mMy[p] = (R)t.mMy[p];
    c.LT[p] = (R)t.LT[p]; c.LX[p] = (R)t.LX[p]; c.LY[p] = (R)t.LY[p];
    for (int k = 0; k < 5; ++k) c.WE[p][k] = (R)t.WE[p][k];
    for (int k = 0; k < 4; ++k) c.WO[p][k] = (R)t.WO[p][k];
    for (int k = 0; k < 8; ++k) {
      c.BE[p][k] = (R)t.BE[p][k]; c.BO[p][k] = (R)t.BO[p][k];
      c.mvE[p][k] = (R)t.mvE[p][k]; c.mvO[p][k] = (R)t.mvO[p][k];
    }
  }
  for (int a = 0; a < 16; ++a)
    for (int b = 0; b < 16; ++b) c.gi[a][b] = (R)t.gi[a][b];
  c.restN0 = (R)t.restN0; c.restE = (R)t.restE; c.restLT = (R)t.restLT;
  for (int k = 0; k < 5; ++k) c.restWE[k] = (R)t.restWE[k];
  for (int k = 0; k < 8; ++k) c.restBE[k] = (R)t.restBE[k];
  for (int i = 0; i < kQm; ++i) c.f0[i] = t.f0[i];
}

// the FP32 tables of the collision rearranged by couple (the same float values)
void fill_couples(const MConsts<float>& c, MCoupleConsts& h) {
  for (int q = 0; q < kCouples; ++q) {
    const int a = couple_a(q), b = couple_b(q);
    h.LT[q] = make_float2(c.LT[a], c.LT[b]);
    h.LX[q] = make_float2(c.LX[a], c.LX[b]);
    h.LY[q] = make_float2(c.LY[a], c.LY[b]);
    for (int k = 0; k < 5; ++k) h.WE[q][k] = make_float2(c.WE[a][k], c.WE[b][k]);
    for (int k = 0; k < 4; ++k) h.WO[q][k] = make_float2(c.WO[a][k], c.WO[b][k]);
    for (int k = 0; k < 8; ++k) {
      h.BE[q][k] = make_float2(c.BE[a][k], c.BE[b][k]);
      h.BO[q][k] = make_float2(c.BO[a][k], c.BO[b][k]);
    }
    h.vx[q] = make_float2(c.vx[a], c.vx[b]);
    h.vy[q] = make_float2(c.vy[a], c.vy[b]);
    h.p0[q] = make_float2(c.mvE[a][1], c.mvE[b][1]);
    h.px2[q] = make_float2(c.mvE[a][2], c.mvE[b][2]);
    h.pxy[q] = make_float2(c.mvE[a][3], c.mvE[b][3]);
    h.py2[q] = make_float2(c.mvE[a][4], c.mvE[b][4]);
    h.pxv[q] = make_float2(c.mvO[a][0], c.mvO[b][0]);
    h.pyv[q] = make_float2(c.mvO[a][1], c.mvO[b][1]);
  }
}

std::mutex g_upload_mu;
bool g_uploaded[64];

}  // namespace
}  // namespace massive
}  // namespace rlbm

using namespace rlbm::massive;

struct rlbm_massive_ctx {
  rlbm_massive_config cfg;
  MGeom geo;
  size_t elem;
  void* buf[2];
  int cur;
  unsigned* err;
  double* scratch;
  size_t scratch_bytes;
  long long steps, launches;
  std::string msg;
};

namespace {

int fail(rlbm_massive_ctx* c, int code, const char* fmt, ...) {
  char b[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(b, sizeof b, fmt, ap);
  va_end(ap);
  if (c) c->msg = b; else g_error = b;
  return code;
}

int cuda_fail(rlbm_massive_ctx* c, cudaError_t e, const char* what) {
  return fail(c, RLBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int upload_tables(int dev) {
  const Tables& t = tables();
  if (!t.ok) return fail(nullptr, RLBM_EINVAL, "massive quadrature: %s", t.msg);
  std::lock_guard<std::mutex> lock(g_upload_mu);
  if (dev < 0 || dev >= 64) return fail(nullptr, RLBM_ECUDA, "device index %d", dev);
  if (g_uploaded[dev]) return RLBM_OK;
  static MConsts<float> hf;
  static MConsts<double> hd;
  static MCoupleConsts hc;
  fill_consts(t, hf);
  fill_consts(t, hd);
  fill_couples(hf, hc);
  cudaError_t e = cudaMemcpyToSymbol(c_f, &hf, sizeof hf);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_d, &hd, sizeof hd);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_cp, &hc, sizeof hc);
  if (e != cudaSuccess) return fail(nullptr, RLBM_ECUDA, "constant upload: %s", cudaGetErrorString(e));
  g_uploaded[dev] = true;
  return RLBM_OK;
}

cudaStream_t stream_of(const rlbm_massive_ctx* c) { return (cudaStream_t)c->cfg.stream; }

dim3 grid_of(const MGeom& g) { return dim3((g.nx + 31) / 32, (g.ny + 3) / 4); }

int need_scratch(rlbm_massive_ctx* c, size_t bytes) {
  if (c->scratch_bytes >= bytes) return RLBM_OK;
  if (c->scratch) { cudaStreamSynchronize(stream_of(c)); cudaFree(c->scratch); c->scratch = nullptr; }
  c->scratch_bytes = 0;
  cudaError_t e = cudaMalloc((void**)&c->scratch, bytes);
  if (e != cudaSuccess) return fail(c, RLBM_ENOMEM, "scratch cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  c->scratch_bytes = bytes;
  return RLBM_OK;
}

int grid_1d(long long work) {
  long long b = (work + 255) / 256;
  return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

}  // namespace

namespace {

int launch_steps(rlbm_massive_ctx* c, int nsteps) {
  const bool force = c->cfg.Fx != 0.0 || c->cfg.Fy != 0.0;
  const dim3 grid = grid_of(c->geo), block(32, 4);
  for (int s = 0; s < nsteps; ++s) {
    const void* src = c->buf[c->cur];
    void* dst = c->buf[c->cur ^ 1];
    if (c->elem == 8) {
      const double it = 1.0 / c->cfg.tau, fx = c->cfg.Fx, fy = c->cfg.Fy;
      if (force) k_mstep<double, true><<<grid, block, 0, stream_of(c)>>>((const double*)src, (double*)dst, c->geo, it, fx, fy, c->err);
      else k_mstep<double, false><<<grid, block, 0, stream_of(c)>>>((const double*)src, (double*)dst, c->geo, it, fx, fy, c->err);
    } else {
      const float it = (float)(1.0 / c->cfg.tau), fx = (float)c->cfg.Fx, fy = (float)c->cfg.Fy;
      if (force) k_mstep_f32_force<<<grid, block, 0, stream_of(c)>>>((const float*)src, (float*)dst, c->geo, it, fx, fy, c->err);
      else k_mstep<float, false><<<grid, block, 0, stream_of(c)>>>((const float*)src, (float*)dst, c->geo, it, fx, fy, c->err);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "step kernel");
    c->cur ^= 1;
    ++c->steps;
    ++c->launches;
  }
  return RLBM_OK;
}

int velocity_planes(rlbm_massive_ctx* c, double* ux, double* uy) {
  if (c->elem == 8)
    k_mmoments<double><<<grid_of(c->geo), dim3(32, 4), 0, stream_of(c)>>>((const double*)c->buf[c->cur], c->geo, nullptr, ux, uy, nullptr, c->err);
  else
    k_mmoments<float><<<grid_of(c->geo), dim3(32, 4), 0, stream_of(c)>>>((const float*)c->buf[c->cur], c->geo, nullptr, ux, uy, nullptr, c->err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel");
  ++c->launches;
  return RLBM_OK;
}

}  // namespace

extern "C" {

int rlbm_massive_quadrature(double* v0, double window[2], double w[10], double p0[10]) {
  const Tables& t = tables();
  if (!t.ok) return fail(nullptr, RLBM_EINVAL, "massive quadrature: %s", t.msg);
  if (v0) *v0 = t.v0;
  if (window) { window[0] = t.window_lo; window[1] = t.window_hi; }
  for (int k = 0; k < kClasses; ++k) {
    if (w) w[k] = t.w_class[k];
    if (p0) p0[k] = t.p0_class[k];
  }
  return RLBM_OK;
}

int rlbm_massive_stencil(int vx[45], int vy[45]) {
  if (!vx || !vy) return fail(nullptr, RLBM_EINVAL, "NULL output");
  for (int p = 0; p < kPairs; ++p) {
    vx[2 * p] = pair_x(p); vy[2 * p] = pair_y(p);
    vx[2 * p + 1] = -pair_x(p); vy[2 * p + 1] = -pair_y(p);
  }
  vx[kRestPop] = vy[kRestPop] = 0;
  return RLBM_OK;
}

int rlbm_massive_create(const rlbm_massive_config* cfg, rlbm_massive_ctx** out) {
  if (!out) return fail(nullptr, RLBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, RLBM_EINVAL, "config is NULL");
  if (cfg->nx < kReach + 1 || cfg->ny < kReach + 1 || cfg->nx > (1 << 17) || cfg->ny > (1 << 17))
    return fail(nullptr, RLBM_EINVAL, "nx, ny must be in [5, 131072]");
  if (!(cfg->tau > 0.5 && cfg->tau < 1e6)) return fail(nullptr, RLBM_EINVAL, "tau must be in (0.5, 1e6)");
  if (!(std::fabs(cfg->Fx) < 1e-2 && std::fabs(cfg->Fy) < 1e-2))
    return fail(nullptr, RLBM_EINVAL, "|F| must be < 1e-2");
  if (cfg->prec != RLBM_F64 && cfg->prec != RLBM_F32)
    return fail(nullptr, RLBM_EINVAL, "precision must be RLBM_F64 or RLBM_F32");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, RLBM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  int r = upload_tables(dev);
  if (r) return r;
  rlbm_massive_ctx* c = new (std::nothrow) rlbm_massive_ctx();
  if (!c) return fail(nullptr, RLBM_ENOMEM, "host allocation failed");
  c->cfg = *cfg;
  c->elem = cfg->prec == RLBM_F64 ? 8 : 4;
  c->geo.nx = cfg->nx; c->geo.ny = cfg->ny;
  c->geo.ldx = (cfg->nx + 31) / 32 * 32;
  c->geo.px = cfg->periodic_x ? 1 : 0; c->geo.py = cfg->periodic_y ? 1 : 0;
  c->geo.plane = (long long)c->geo.ldx * cfg->ny;
  const size_t bytes = (size_t)c->geo.plane * kQm * c->elem;
  for (int b = 0; b < 2; ++b) {
    e = cudaMalloc(&c->buf[b], bytes);
    if (e != cudaSuccess) {
      rlbm_massive_destroy(c);
      return fail(nullptr, RLBM_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
  }
  e = cudaMalloc((void**)&c->err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(c->buf[0], 0, bytes);
  if (e != cudaSuccess) {
    rlbm_massive_destroy(c);
    return fail(nullptr, RLBM_ECUDA, "setup: %s", cudaGetErrorString(e));
  }
  *out = c;
  return RLBM_OK;
}

int rlbm_massive_init(rlbm_massive_ctx* c, const double* n, const double* ux, const double* uy,
                      const double* T, int device_ptrs) {
  if (!c) return fail(nullptr, RLBM_EINVAL, "ctx is NULL");
  const long long ns = (long long)c->geo.nx * c->geo.ny;
  const size_t bytes = (size_t)c->geo.plane * kQm * c->elem;
  cudaError_t e;
  if (!n && !ux && !uy && !T) {
    e = cudaMemsetAsync(c->buf[0], 0, bytes, stream_of(c));
    if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  } else {
    if (!n || !ux || !uy || !T) return fail(c, RLBM_EINVAL, "give all four fields or none");
    const double* f[4] = {n, ux, uy, T};
    if (!device_ptrs) {
      int r = need_scratch(c, 4 * ns * sizeof(double));
      if (r) return r;
      for (int k = 0; k < 4; ++k) {
        e = cudaMemcpyAsync(c->scratch + k * ns, f[k], ns * sizeof(double), cudaMemcpyHostToDevice, stream_of(c));
        if (e != cudaSuccess) return cuda_fail(c, e, "field upload");
        f[k] = c->scratch + k * ns;
      }
    }
    if (c->elem == 8)
      k_minit<double><<<grid_of(c->geo), dim3(32, 4), 0, stream_of(c)>>>((double*)c->buf[0], c->geo, f[0], f[1], f[2], f[3], c->err);
    else
      k_minit<float><<<grid_of(c->geo), dim3(32, 4), 0, stream_of(c)>>>((float*)c->buf[0], c->geo, f[0], f[1], f[2], f[3], c->err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    ++c->launches;
    e = cudaStreamSynchronize(stream_of(c));
    if (e != cudaSuccess) return cuda_fail(c, e, "init");
    unsigned bits = 0;
    e = cudaMemcpy(&bits, c->err, sizeof bits, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "error word");
    if (bits) {
      cudaMemset(c->err, 0, sizeof(unsigned));
      return fail(c, RLBM_EINVAL, "init fields: need |u| < 1, n > 0, T > 0");
    }
  }
  c->cur = 0;
  c->steps = 0;
  return RLBM_OK;
}



int rlbm_massive_step(rlbm_massive_ctx* c, int nsteps, double* residual) {
  if (!c) return fail(nullptr, RLBM_EINVAL, "ctx is NULL");
  if (nsteps < 0) return fail(c, RLBM_EINVAL, "nsteps < 0");
  if (!residual) return launch_steps(c, nsteps);
  if (nsteps < 1) return fail(c, RLBM_EINVAL, "a residual needs nsteps >= 1");
  const long long ns = (long long)c->geo.nx * c->geo.ny;
  int r = need_scratch(c, 4 * ns * sizeof(double) + 2 * sizeof(double));
  if (r) return r;
  double* up = c->scratch;             // u(t - 1): x, y planes; u(t): x, y planes; sums
  double* acc = c->scratch + 4 * ns;
  if ((r = launch_steps(c, nsteps - 1))) return r;
  if ((r = velocity_planes(c, up, up + ns))) return r;
  if ((r = launch_steps(c, 1))) return r;
  if ((r = velocity_planes(c, up + 2 * ns, up + 3 * ns))) return r;
  cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), stream_of(c));
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  k_mresidual<<<grid_1d(ns), 256, 0, stream_of(c)>>>(up, up + ns, up + 2 * ns, up + 3 * ns, ns, acc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "residual kernel");
  ++c->launches;
  double h[2];
  e = cudaMemcpyAsync(h, acc, sizeof h, cudaMemcpyDeviceToHost, stream_of(c));
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream_of(c));
  if (e != cudaSuccess) return cuda_fail(c, e, "residual readback");
  *residual = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : (h[0] > 0.0 ? INFINITY : 0.0);
  return rlbm_massive_check(c);
}



int rlbm_massive_moments(rlbm_massive_ctx* c, double* n, double* ux, double* uy, double* T,
                         int device_ptrs) {
  if (!c) return fail(nullptr, RLBM_EINVAL, "ctx is NULL");
  const long long ns = (long long)c->geo.nx * c->geo.ny;
  double* d[4] = {n, ux, uy, T};
  if (!device_ptrs) {
    int r = need_scratch(c, 4 * ns * sizeof(double));
    if (r) return r;
    for (int k = 0; k < 4; ++k) d[k] = c->scratch + k * ns;
  }
  if (c->elem == 8)
    k_mmoments<double><<<grid_of(c->geo), dim3(32, 4), 0, stream_of(c)>>>((const double*)c->buf[c->cur], c->geo, d[0], d[1], d[2], d[3], c->err);
  else
    k_mmoments<float><<<grid_of(c->geo), dim3(32, 4), 0, stream_of(c)>>>((const float*)c->buf[c->cur], c->geo, d[0], d[1], d[2], d[3], c->err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel");
  ++c->launches;
  if (!device_ptrs) {
    double* h[4] = {n, ux, uy, T};
    for (int k = 0; k < 4; ++k) {
      if (!h[k]) continue;
      e = cudaMemcpyAsync(h[k], d[k], ns * sizeof(double), cudaMemcpyDeviceToHost, stream_of(c));
      if (e != cudaSuccess) return cuda_fail(c, e, "moments download");
    }
    e = cudaStreamSynchronize(stream_of(c));
    if (e != cudaSuccess) return cuda_fail(c, e, "moments");
  }
  return RLBM_OK;
}

int rlbm_massive_get_state(rlbm_massive_ctx* c, double* delta, int device_ptrs) {
  if (!c || !delta) return fail(c, RLBM_EINVAL, "NULL argument");
  const long long work = (long long)c->geo.nx * c->geo.ny * kQm;
  double* d = delta;
  if (!device_ptrs) {
    int r = need_scratch(c, work * sizeof(double));
    if (r) return r;
    d = c->scratch;
  }
  if (c->elem == 8) k_mget<double><<<grid_1d(work), 256, 0, stream_of(c)>>>((const double*)c->buf[c->cur], c->geo, d);
  else k_mget<float><<<grid_1d(work), 256, 0, stream_of(c)>>>((const float*)c->buf[c->cur], c->geo, d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "state kernel");
  ++c->launches;
  if (!device_ptrs) {
    e = cudaMemcpyAsync(delta, d, work * sizeof(double), cudaMemcpyDeviceToHost, stream_of(c));
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream_of(c));
    if (e != cudaSuccess) return cuda_fail(c, e, "state download");
  }
  return RLBM_OK;
}

int rlbm_massive_set_state(rlbm_massive_ctx* c, const double* delta, int device_ptrs) {
  if (!c || !delta) return fail(c, RLBM_EINVAL, "NULL argument");
  const long long work = (long long)c->geo.nx * c->geo.ny * kQm;
  const double* d = delta;
  if (!device_ptrs) {
    int r = need_scratch(c, work * sizeof(double));
    if (r) return r;
    cudaError_t e = cudaMemcpyAsync(c->scratch, delta, work * sizeof(double), cudaMemcpyHostToDevice, stream_of(c));
    if (e != cudaSuccess) return cuda_fail(c, e, "state upload");
    d = c->scratch;
  }
  if (c->elem == 8) k_mset<double><<<grid_1d(work), 256, 0, stream_of(c)>>>((double*)c->buf[0], c->geo, d);
  else k_mset<float><<<grid_1d(work), 256, 0, stream_of(c)>>>((float*)c->buf[0], c->geo, d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "state kernel");
  ++c->launches;
  c->cur = 0;
  c->steps = 0;
  if (!device_ptrs) {
    e = cudaStreamSynchronize(stream_of(c));
    if (e != cudaSuccess) return cuda_fail(c, e, "state upload");
  }
  return RLBM_OK;
}

int rlbm_massive_check(rlbm_massive_ctx* c) {
  if (!c) return fail(nullptr, RLBM_EINVAL, "ctx is NULL");
  cudaError_t e = cudaStreamSynchronize(stream_of(c));
  if (e != cudaSuccess) return cuda_fail(c, e, "sync");
  unsigned bits = 0;
  e = cudaMemcpy(&bits, c->err, sizeof bits, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "error word");
  if (!bits) return RLBM_OK;
  cudaMemset(c->err, 0, sizeof(unsigned));
  return fail(c, RLBM_ENAN, "device error bits 0x%x (1 non-finite, 2 |u| >= 1 or n, T <= 0, "
              "4 Landau solve not converged)", bits);
}

long long rlbm_massive_steps_done(const rlbm_massive_ctx* c) { return c ? c->steps : -1; }
long long rlbm_massive_launch_count(const rlbm_massive_ctx* c) { return c ? c->launches : -1; }

void rlbm_massive_destroy(rlbm_massive_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(stream_of(c));
  for (int b = 0; b < 2; ++b) if (c->buf[b]) cudaFree(c->buf[b]);
  if (c->err) cudaFree(c->err);
  if (c->scratch) cudaFree(c->scratch);
  delete c;
}

const char* rlbm_massive_last_error(const rlbm_massive_ctx* c) {
  return c ? c->msg.c_str() : g_error.c_str();
}

}  // extern "C"

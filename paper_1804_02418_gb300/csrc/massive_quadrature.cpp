// Quadrature and per-node tables of the massive-particle variant, m = 5 T0
// (Sec. 2.3: Eq. discrete-quadri-momentum, Eq. discrete-p0, Eq. orthonormal,
// Fig. m5-stencil).
//
// Nodes p_i = p0_i (1, v0 n_i), p0_i = m / sqrt(1 - v0^2 |n_i|^2), over the
// 45 vectors {(0,0), (1,0), (1,1), (2,0), (2,1), (2,2), (3,0), (3,2), (3,3),
// (4,0)} with all sign changes and component swaps.  The weight function is
// the rest Maxwell-Juttner distribution at T0 = 1,
//   omega = exp(-(p0 - m)) / (2 pi),   d^2p / p0 = dp0 dtheta on the shell.
// Eq. orthonormal up to third order is exact quadrature of every monomial of
// degree <= 6; on the shell and with the square's symmetry this reduces to
// ten linear conditions on the ten class weights:
//   sum_i w_i p0^a px^b py^c = int omega p0^a px^b py^c d^2p / p0
// for (a, b, c) in (0,0,0) (0,2,0) (0,4,0) (0,2,2) (0,6,0) (0,4,2) (1,0,0)
// (1,2,0) (1,4,0) (1,2,2).  The right-hand sides are rational:
//   (1 / 2 pi) int cos^b sin^c dtheta = (b-1)!! (c-1)!! / (b+c)!!,
//   int_m^inf e^-(p0-m) p0^a (p0^2 - m^2)^h dp0
//     = sum_l C(h,l) (-m^2)^(h-l) K(a + 2l),  K(k) = sum_j C(k,j) j! m^(k-j).
// The paper leaves v0 free (v0 <= 1 / sqrt(18)) and asks for non-negative
// weights; they are all non-negative on one narrow interval of v0 only.
// The library takes its midpoint: a scan in FP64 brackets the interval, its
// two ends are bisected in double-double, and the midpoint is rounded to
// FP64; weights and energies follow at that v0 in double-double.
//
// Equilibrium tables.  With the Gram matrix G of the 16 monomials under
// omega, the projection of the Maxwell-Juttner distribution onto the
// polynomials of degree <= 3 (Eq. feq-expansion-discrete) is
//   f^eq_i / f0_i = (m + 1) m(p_i)^T G^-1 M(n, U, T),
// M the Maxwell-Juttner moments of the monomials and f0_i = w_i / (m + 1)
// the rest populations.  The kernels split the relative deviation
// g^eq = f^eq / f0 - 1 into its exact linear and quadratic parts in
// (n - 1, T - 1, ux, uy), whose per-node coefficients are tabulated here,
// and a remainder of third order to which B = m(p)^T (m + 1) G^-1 is
// applied; so no large entry of B multiplies a rounded O(1) quantity.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <utility>

#include "dd.h"
#include "massive_tables.h"

namespace rlbm {
namespace massive {
namespace {

using namespace ddm;

constexpr int kCond = 10;
const int kCondA[kCond] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1};
const int kCondB[kCond] = {0, 2, 4, 2, 6, 4, 0, 2, 4, 2};
const int kCondC[kCond] = {0, 0, 0, 2, 0, 2, 0, 0, 0, 2};
const int kClassA[kClasses] = {1, 1, 2, 2, 2, 3, 3, 3, 4, 0};
const int kClassB[kClasses] = {0, 1, 0, 1, 2, 0, 2, 3, 0, 0};

// library monomial order: exponents (a, b, c) of p0^a px^b py^c
const int kMonA[16] = {0, 1, 0, 0, 0, 1, 1, 1, 0, 0, 1, 1, 0, 0, 0, 0};
const int kMonB[16] = {0, 0, 2, 1, 0, 2, 1, 0, 1, 0, 1, 0, 3, 2, 1, 0};
const int kMonC[16] = {0, 0, 0, 1, 2, 0, 1, 2, 0, 1, 0, 1, 0, 1, 2, 3};

long long binom(int n, int k) {
  long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
long long fact(int n) { long long r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }
long long dfact(int n) { long long r = 1; for (int i = n; i > 1; i -= 2) r *= i; return r; }

// int omega p0^a px^b py^c d^2p / p0 (exact: integer numerator / denominator)
dd omega_moment(int a, int b, int c) {
  if ((b & 1) || (c & 1)) return D(0.0);
  const int h = (b + c) / 2;
  long long rad = 0;
  for (int l = 0; l <= h; ++l) {
    const int k = a + 2 * l;
    long long K = 0;
    for (int j = 0; j <= k; ++j) {
      long long mp = 1;
      for (int e = 0; e < k - j; ++e) mp *= kMass;
      K += binom(k, j) * fact(j) * mp;
    }
    long long mm = 1;
    for (int e = 0; e < h - l; ++e) mm *= -(long long)kMass * kMass;
    rad += binom(h, l) * mm * K;
  }
  const long long num = rad * dfact(b - 1) * dfact(c - 1);
  // num stays far below 2^53 for degree <= 8
  return div(D((double)num), D((double)dfact(b + c)));
}

// members of a class (the same order as the population layout)
int class_members(int k, int* vx, int* vy) {
  const int a = kClassA[k], b = kClassB[k];
  if (a == 0) { vx[0] = 0; vy[0] = 0; return 1; }
  if (b == 0) {
    const int x[4] = {a, -a, 0, 0}, y[4] = {0, 0, a, -a};
    for (int i = 0; i < 4; ++i) { vx[i] = x[i]; vy[i] = y[i]; }
    return 4;
  }
  if (a == b) {
    const int x[4] = {a, -a, -a, a}, y[4] = {a, -a, a, -a};
    for (int i = 0; i < 4; ++i) { vx[i] = x[i]; vy[i] = y[i]; }
    return 4;
  }
  const int x[8] = {a, -a, -a, a, b, -b, -b, b}, y[8] = {b, -b, b, -b, a, -a, a, -a};
  for (int i = 0; i < 8; ++i) { vx[i] = x[i]; vy[i] = y[i]; }
  return 8;
}

dd powi(dd x, int k) { dd r = D(1.0); for (int i = 0; i < k; ++i) r = mul(r, x); return r; }

// Solves A x = b in place (n x n, partial pivoting); false if singular.
bool solve(dd* A, dd* b, int n) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c].hi) > std::fabs(A[piv * n + c].hi)) piv = r;
    if (A[piv * n + c].hi == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) { dd t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t; }
      dd t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      dd f = div(A[r * n + c], A[c * n + c]);
      for (int k = c; k < n; ++k) A[r * n + k] = sub(A[r * n + k], mul(f, A[c * n + k]));
      b[r] = sub(b[r], mul(f, b[c]));
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    dd s = b[c];
    for (int k = c + 1; k < n; ++k) s = sub(s, mul(A[c * n + k], b[k]));
    b[c] = div(s, A[c * n + c]);
  }
  return true;
}

dd class_p0(int k, dd v0) {
  const int n2 = kClassA[k] * kClassA[k] + kClassB[k] * kClassB[k];
  return div(D((double)kMass), ddm::sqrt(sub(D(1.0), mul(mul(v0, v0), D((double)n2)))));
}

// class weights at v0 (double-double)
bool weights_dd(dd v0, dd* w) {
  dd A[kCond * kCond];
  for (int i = 0; i < kCond * kCond; ++i) A[i] = D(0.0);
  for (int k = 0; k < kClasses; ++k) {
    const dd p0 = class_p0(k, v0);
    int vx[8], vy[8];
    const int nm = class_members(k, vx, vy);
    for (int i = 0; i < nm; ++i) {
      const dd px = mul(mul(p0, v0), D((double)vx[i]));
      const dd py = mul(mul(p0, v0), D((double)vy[i]));
      for (int r = 0; r < kCond; ++r)
        A[r * kCond + k] = add(A[r * kCond + k],
                               mul(mul(powi(p0, kCondA[r]), powi(px, kCondB[r])), powi(py, kCondC[r])));
    }
  }
  for (int r = 0; r < kCond; ++r) w[r] = omega_moment(kCondA[r], kCondB[r], kCondC[r]);
  return solve(A, w, kCond);
}

// the same in FP64 (coarse scan only: signs far from the interval ends)
bool weights_fp64(double v0, double* w) {
  double A[kCond * kCond] = {0};
  for (int k = 0; k < kClasses; ++k) {
    const int n2 = kClassA[k] * kClassA[k] + kClassB[k] * kClassB[k];
    const double p0 = kMass / std::sqrt(1.0 - v0 * v0 * n2);
    int vx[8], vy[8];
    const int nm = class_members(k, vx, vy);
    for (int i = 0; i < nm; ++i) {
      const double px = p0 * v0 * vx[i], py = p0 * v0 * vy[i];
      double xp[7] = {1.0}, yp[7] = {1.0};
      for (int e = 1; e < 7; ++e) { xp[e] = xp[e - 1] * px; yp[e] = yp[e - 1] * py; }
      for (int r = 0; r < kCond; ++r)
        A[r * kCond + k] += (kCondA[r] ? p0 : 1.0) * xp[kCondB[r]] * yp[kCondC[r]];
    }
  }
  for (int r = 0; r < kCond; ++r) w[r] = to_double(omega_moment(kCondA[r], kCondB[r], kCondC[r]));
  for (int c = 0; c < kCond; ++c) {
    int piv = c;
    for (int r = c + 1; r < kCond; ++r) if (std::fabs(A[r * kCond + c]) > std::fabs(A[piv * kCond + c])) piv = r;
    if (A[piv * kCond + c] == 0.0) return false;
    for (int k = 0; k < kCond; ++k) std::swap(A[c * kCond + k], A[piv * kCond + k]);
    std::swap(w[c], w[piv]);
    for (int r = c + 1; r < kCond; ++r) {
      const double f = A[r * kCond + c] / A[c * kCond + c];
      for (int k = c; k < kCond; ++k) A[r * kCond + k] -= f * A[c * kCond + k];
      w[r] -= f * w[c];
    }
  }
  for (int c = kCond - 1; c >= 0; --c) {
    double s = w[c];
    for (int k = c + 1; k < kCond; ++k) s -= A[c * kCond + k] * w[k];
    w[c] = s / A[c * kCond + c];
  }
  return true;
}

bool nonneg_dd(dd v0) {
  dd w[kCond];
  if (!weights_dd(v0, w)) return false;
  for (int k = 0; k < kCond; ++k) if (w[k].hi < 0.0) return false;
  return true;
}

bool nonneg_fp64(double v0) {
  double w[kCond];
  if (!weights_fp64(v0, w)) return false;
  for (int k = 0; k < kCond; ++k) if (w[k] < 0.0) return false;
  return true;
}

// end of the interval between a point where some weight is negative (bad)
// and one where none is (good)
dd bisect(dd bad, dd good) {
  for (int it = 0; it < 90; ++it) {
    const dd mid = mul(add(bad, good), D(0.5));
    if (nonneg_dd(mid)) good = mid; else bad = mid;
  }
  return mul(add(bad, good), D(0.5));
}

void monomials(dd p0, dd px, dd py, dd* mv) {
  for (int b = 0; b < 16; ++b)
    mv[b] = mul(mul(powi(p0, kMonA[b]), powi(px, kMonB[b])), powi(py, kMonC[b]));
}

void fail(Tables& t, const char* m) { t.ok = false; std::snprintf(t.msg, sizeof t.msg, "%s", m); }

void compute(Tables& t) {
  std::memset(&t, 0, sizeof t);
  t.ok = true;
  // --- the interval of non-negative weights --------------------------------
  const double vmax = 1.0 / std::sqrt(18.0);
  const double step = 1e-6;
  int first = -1, last = -1;
  const int npts = (int)((vmax - 0.01) / step);
  for (int k = 0; k < npts; ++k) {
    if (nonneg_fp64(0.01 + k * step)) {
      if (first < 0) first = k;
      else if (last != k - 1) { fail(t, "non-negative weights on more than one interval of v0"); return; }
      last = k;
    }
  }
  if (first <= 0 || last < 0 || last + 1 >= npts) { fail(t, "no interval of non-negative weights"); return; }
  // the brackets must hold in double-double too; widen by a grid step if not
  dd lo_bad = D(0.01 + (first - 1) * step), lo_good = D(0.01 + first * step);
  dd hi_good = D(0.01 + last * step), hi_bad = D(0.01 + (last + 1) * step);
  for (int it = 0; it < 4 && nonneg_dd(lo_bad); ++it) { lo_good = lo_bad; lo_bad = sub(lo_bad, D(step)); }
  for (int it = 0; it < 4 && !nonneg_dd(lo_good); ++it) { lo_bad = lo_good; lo_good = add(lo_good, D(step)); }
  for (int it = 0; it < 4 && nonneg_dd(hi_bad); ++it) { hi_good = hi_bad; hi_bad = add(hi_bad, D(step)); }
  for (int it = 0; it < 4 && !nonneg_dd(hi_good); ++it) { hi_bad = hi_good; hi_good = sub(hi_good, D(step)); }
  const dd lo = bisect(lo_bad, lo_good), hi = bisect(hi_bad, hi_good);
  t.window_lo = to_double(lo);
  t.window_hi = to_double(hi);
  t.v0 = to_double(mul(add(lo, hi), D(0.5)));
  const dd v0 = D(t.v0);
  dd wc[kClasses];
  if (!weights_dd(v0, wc)) { fail(t, "singular quadrature system"); return; }
  dd p0c[kClasses];
  for (int k = 0; k < kClasses; ++k) {
    p0c[k] = class_p0(k, v0);
    t.w_class[k] = to_double(wc[k]);
    t.p0_class[k] = to_double(p0c[k]);
    if (t.w_class[k] < 0.0) { fail(t, "negative weight at the chosen v0"); return; }
  }
  // --- Gram matrix and (m + 1) G^-1 ----------------------------------------
  dd G[16 * 16], Gi[16 * 16];
  for (int a = 0; a < 16; ++a)
    for (int b = 0; b < 16; ++b)
      G[a * 16 + b] = omega_moment(kMonA[a] + kMonA[b], kMonB[a] + kMonB[b], kMonC[a] + kMonC[b]);
  for (int col = 0; col < 16; ++col) {
    dd A[16 * 16], e[16];
    for (int i = 0; i < 256; ++i) A[i] = G[i];
    for (int i = 0; i < 16; ++i) e[i] = D(i == col ? 1.0 : 0.0);
    if (!solve(A, e, 16)) { fail(t, "singular Gram matrix"); return; }
    for (int i = 0; i < 16; ++i) Gi[i * 16 + col] = mul(e[i], D((double)(kMass + 1)));
  }
  for (int a = 0; a < 16; ++a)
    for (int b = 0; b < 16; ++b) t.gi[a][b] = to_double(Gi[a * 16 + b]);
  // --- linear and quadratic moment responses (library order) ---------------
  const double m = kMass, m1 = kMass + 1;
  const dd h0 = div(D(m * m + 3 * m + 3), D(m1));                    // eps + P at rest
  const dd k1 = div(D(2 * m * m + 6 * m + 3), D(m1 * m1));           // d(eps + P)/dT at rest
  const dd a0 = div(D(m * m * m + 6 * m * m + 15 * m + 15), D(m1));  // alpha at rest
  const dd c2 = div(D(m * m), D(m1 * m1 * m1));
  dd lin[4][16], quad[9][16];   // lin: dn dT ux uy; quad: nT TT xx xy yy nx ny Tx Ty
  for (int r = 0; r < 4; ++r) for (int b = 0; b < 16; ++b) lin[r][b] = D(0.0);
  for (int r = 0; r < 9; ++r) for (int b = 0; b < 16; ++b) quad[r][b] = D(0.0);
  // E: 0 1, 1 p0, 2 px2, 3 pxpy, 4 py2, 5 p0px2, 6 p0pxpy, 7 p0py2
  // O: 8 px, 9 py, 10 p0px, 11 p0py, 12 px3, 13 px2py, 14 pxpy2, 15 py3
  lin[0][0] = div(D(1.0), D(m1)); lin[0][1] = D(1.0); lin[0][2] = lin[0][4] = D(1.0);
  lin[0][5] = lin[0][7] = h0;
  lin[1][0] = neg(div(D(1.0), D(m1 * m1))); lin[1][2] = lin[1][4] = D(1.0);
  lin[1][5] = lin[1][7] = add(k1, h0);
  lin[2][8] = D(1.0); lin[2][10] = h0; lin[2][12] = mul(D(3.0), h0); lin[2][14] = h0;
  lin[3][9] = D(1.0); lin[3][11] = h0; lin[3][15] = mul(D(3.0), h0); lin[3][13] = h0;
  enum { nT, TT, xx, xy, yy, nx, ny, Tx, Ty };
  quad[nT][0] = neg(div(D(1.0), D(m1 * m1)));
  quad[TT][0] = div(D(1.0), D(m1 * m1 * m1));
  quad[xx][1] = quad[yy][1] = D(0.5);
  quad[nx][8] = D(1.0); quad[ny][9] = D(1.0);
  quad[nx][10] = h0; quad[Tx][10] = k1; quad[ny][11] = h0; quad[Ty][11] = k1;
  quad[xx][2] = h0; quad[nT][2] = D(1.0); quad[yy][4] = h0; quad[nT][4] = D(1.0); quad[xy][3] = h0;
  const dd h0_2 = mul(h0, D(0.5));
  quad[xx][5] = add(a0, h0_2); quad[yy][5] = h0_2; quad[nT][5] = add(k1, h0); quad[TT][5] = add(k1, c2);
  quad[yy][7] = add(a0, h0_2); quad[xx][7] = h0_2; quad[nT][7] = add(k1, h0); quad[TT][7] = add(k1, c2);
  quad[xy][6] = a0;
  quad[nx][12] = mul(D(3.0), h0); quad[Tx][12] = mul(D(3.0), add(k1, h0));
  quad[ny][13] = h0; quad[Ty][13] = add(k1, h0);
  quad[nx][14] = h0; quad[Tx][14] = add(k1, h0);
  quad[ny][15] = mul(D(3.0), h0); quad[Ty][15] = mul(D(3.0), add(k1, h0));
  // --- per node -----------------------------------------------------------
  double worst = 0.0;
  auto node = [&](dd p0, dd px, dd py, dd f0, double* LT, double* LX, double* LY, double* WE,
                  double* WO, double* BE, double* BO, double* mvE, double* mvO) {
    dd mv[16], B[16];
    monomials(p0, px, py, mv);
    for (int b = 0; b < 16; ++b) {
      dd s = D(0.0);
      for (int a = 0; a < 16; ++a) s = add(s, mul(mv[a], Gi[a * 16 + b]));
      B[b] = s;
    }
    dd L[4], Q[9];
    for (int r = 0; r < 4; ++r) {
      dd s = D(0.0);
      for (int b = 0; b < 16; ++b) s = add(s, mul(B[b], lin[r][b]));
      L[r] = s;
    }
    for (int r = 0; r < 9; ++r) {
      dd s = D(0.0);
      for (int b = 0; b < 16; ++b) s = add(s, mul(B[b], quad[r][b]));
      Q[r] = s;
    }
    worst = std::fmax(worst, std::fabs(to_double(sub(L[0], D(1.0)))));
    *LT = to_double(L[1]);
    if (LX) { *LX = to_double(L[2]); *LY = to_double(L[3]); }
    for (int r = 0; r < 5; ++r) WE[r] = to_double(Q[r]);
    if (WO) for (int r = 0; r < 4; ++r) WO[r] = to_double(Q[5 + r]);
    for (int b = 0; b < 8; ++b) BE[b] = to_double(B[b]);
    if (BO) for (int b = 0; b < 8; ++b) BO[b] = to_double(B[8 + b]);
    if (mvE) for (int b = 0; b < 8; ++b) { mvE[b] = to_double(mv[b]); mvO[b] = to_double(mv[8 + b]); }
    (void)f0;
  };
  for (int p = 0; p < kPairs; ++p) {
    const int k = pair_class(p);
    const dd p0 = p0c[k];
    const dd px = mul(mul(p0, v0), D((double)pair_x(p)));
    const dd py = mul(mul(p0, v0), D((double)pair_y(p)));
    const dd f0 = div(wc[k], D(m1));
    t.f0[2 * p] = t.f0[2 * p + 1] = to_double(f0);
    t.vx[p] = to_double(mul(v0, D((double)pair_x(p))));
    t.vy[p] = to_double(mul(v0, D((double)pair_y(p))));
    t.mN0[p] = to_double(mul(f0, p0));
    t.mE[p] = to_double(mul(f0, mul(p0, p0)));
    t.mPxx[p] = to_double(mul(f0, mul(px, px)));
    t.mPxy[p] = to_double(mul(f0, mul(px, py)));
    t.mPyy[p] = to_double(mul(f0, mul(py, py)));
    t.mNx[p] = to_double(mul(f0, px));
    t.mNy[p] = to_double(mul(f0, py));
    t.mMx[p] = to_double(mul(f0, mul(p0, px)));
    t.mMy[p] = to_double(mul(f0, mul(p0, py)));
    node(p0, px, py, f0, &t.LT[p], &t.LX[p], &t.LY[p], t.WE[p], t.WO[p], t.BE[p], t.BO[p],
         t.mvE[p], t.mvO[p]);
  }
  {
    const dd p0 = p0c[kClasses - 1];           // = m
    const dd f0 = div(wc[kClasses - 1], D(m1));
    t.f0[kRestPop] = to_double(f0);
    t.restN0 = to_double(mul(f0, p0));
    t.restE = to_double(mul(f0, mul(p0, p0)));
    node(p0, D(0.0), D(0.0), f0, &t.restLT, nullptr, nullptr, t.restWE, nullptr, t.restBE,
         nullptr, nullptr, nullptr);
  }
  t.lin_check = worst;
  if (!(worst < 1e-20)) fail(t, "equilibrium tables: density response is not 1");
}

}  // namespace

const Tables& tables() {
  static Tables t;
  static std::once_flag once;
  std::call_once(once, [] { compute(t); });
  return t;
}

}  // namespace massive
}  // namespace rlbm

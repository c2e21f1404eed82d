// Host tables of the massive-particle variant (m = 5 T0, the 45-vector
// stencil of Fig. m5-stencil, Sec. 2.3), computed once in double-double
// arithmetic by massive_quadrature.cpp and uploaded by massive.cu.
//
// Population order (also the state layout of the C ABI): 22 pairs of
// opposite vectors, pair p holding populations 2p (vector (pair_x(p),
// pair_y(p))) and 2p + 1 (its negative), class by class; then the rest
// vector at 44.
//
// Library monomial order (a basis of the polynomials of degree <= 3 on the
// mass shell p0^2 = m^2 + px^2 + py^2), even in (px, py) first:
//   E: 1, p0, px^2, px py, py^2, p0 px^2, p0 px py, p0 py^2
//   O: px, py, p0 px, p0 py, px^3, px^2 py, px py^2, py^3
#pragma once

#ifdef __CUDACC__
#define RLBM_HD __host__ __device__
#else
#define RLBM_HD
#endif

namespace rlbm {
namespace massive {

constexpr int kQm = 45;
constexpr int kPairs = 22;
constexpr int kRestPop = 44;
constexpr int kClasses = 10;
constexpr int kMass = 5;          // m / T0
constexpr int kReach = 4;         // largest |component| of a stencil vector

// vector of the first member of pair p (the second is its negative) and its
// class: (1,0) (1,1) (2,0) (2,1) (2,2) (3,0) (3,2) (3,3) (4,0) = 0..8, (0,0) = 9
RLBM_HD constexpr int pair_x(int p) {
  return p == 0 ? 1 : p == 1 ? 0 : p == 2 ? 1 : p == 3 ? -1 : p == 4 ? 2 : p == 5 ? 0 : p == 6 ? 2 : p == 7 ? -2 : p == 8 ? 1 : p == 9 ? -1 : p == 10 ? 2 : p == 11 ? -2 : p == 12 ? 3 : p == 13 ? 0 : p == 14 ? 3 : p == 15 ? -3 : p == 16 ? 2 : p == 17 ? -2 : p == 18 ? 3 : p == 19 ? -3 : p == 20 ? 4 : 0;
}
RLBM_HD constexpr int pair_y(int p) {
  return p == 0 ? 0 : p == 1 ? 1 : p == 2 ? 1 : p == 3 ? 1 : p == 4 ? 0 : p == 5 ? 2 : p == 6 ? 1 : p == 7 ? 1 : p == 8 ? 2 : p == 9 ? 2 : p == 10 ? 2 : p == 11 ? 2 : p == 12 ? 0 : p == 13 ? 3 : p == 14 ? 2 : p == 15 ? 2 : p == 16 ? 3 : p == 17 ? 3 : p == 18 ? 3 : p == 19 ? 3 : p == 20 ? 0 : 4;
}
RLBM_HD constexpr int pair_class(int p) {
  return p == 0 ? 0 : p == 1 ? 0 : p == 2 ? 1 : p == 3 ? 1 : p == 4 ? 2 : p == 5 ? 2 : p == 6 ? 3 : p == 7 ? 3 : p == 8 ? 3 : p == 9 ? 3 : p == 10 ? 4 : p == 11 ? 4 : p == 12 ? 5 : p == 13 ? 5 : p == 14 ? 6 : p == 15 ? 6 : p == 16 ? 6 : p == 17 ? 6 : p == 18 ? 7 : p == 19 ? 7 : p == 20 ? 8 : 8;
}

struct Tables {
  bool ok;
  char msg[160];
  double v0, window_lo, window_hi;
  double w_class[kClasses], p0_class[kClasses];
  double f0[kQm];                       // rest populations w_i / (m + 1)
  double gi[16][16];                    // (m + 1) G^-1, library monomial order (E then O)
  // per pair (values at its first member; the second has the odd parts negated)
  double vx[kPairs], vy[kPairs];        // v0 n
  double mN0[kPairs], mE[kPairs], mPxx[kPairs], mPxy[kPairs], mPyy[kPairs];   // f0 x even monomial
  double mNx[kPairs], mNy[kPairs], mMx[kPairs], mMy[kPairs];                 // f0 x odd monomial
  double LT[kPairs], LX[kPairs], LY[kPairs];       // linear response of g^eq to dT, ux, uy
  double WE[kPairs][5];                 // quadratic response: dn dT, dT^2, ux^2, ux uy, uy^2
  double WO[kPairs][4];                 //                     dn ux, dn uy, dT ux, dT uy
  double BE[kPairs][8], BO[kPairs][8];  // m(p)^T (m + 1) G^-1, even / odd columns
  double mvE[kPairs][8], mvO[kPairs][8];   // monomial values
  double restN0, restE, restLT, restWE[5], restBE[8];
  double lin_check;                     // max |response to dn - 1| (must vanish)
};

// Computes the tables on first use (about 0.3 s); thread-safe.
const Tables& tables();

}  // namespace massive
}  // namespace rlbm

// Refined 48-population massless quadrature (Sec. 2.3, Eq. orthonormal).
//
// The paper prints the weights w_1j, w_2j and shell energies p0_j to twelve
// digits.  Those values satisfy Eq. orthonormal only to about 3e-9, and the
// conditions leave a two-parameter family of exact solutions.  The library
// uses the exact solution nearest to the printed values: Gauss-Newton steps
// of minimum Euclidean norm in the 12 unscaled parameters, in double-double
// arithmetic, then rounded to FP64.
//
// Eq. orthonormal for the 16 App. A polynomials (all cubics in p on the
// massless shell) is equivalent to exact quadrature of every monomial of
// degree <= 6.  On the shell a degree-K monomial is p0^K times a
// trigonometric polynomial of order <= K; summed over the D4-symmetric
// stencil only the angular harmonics 0 and 4 survive.  With
//   W_j = 8 w_1j + 4 w_2j            (harmonic 0),
//   V_j = C1 w_1j + C2 w_2j          (harmonic 4: C1 = sum of cos 4theta over
//                                     the (3,4)-type vectors = -4216/625,
//                                     C2 = 4 for the (5,0)-type vectors)
// the conditions read
//   sum_j W_j p0_j^K = K!   (K = 0..6;  continuum int e^-p p^K dp)
//   sum_j V_j p0_j^K = 0    (K = 4..6;  isotropy of the 4th harmonic)
// i.e. 10 equations in 12 unknowns.
#include <cmath>
#include <cstring>

#include "dd.h"

namespace rlbm {
namespace {

using namespace ddm;

constexpr int NP = 12;   // unknowns: w1[0..3], w2[0..3], p0[0..3]
constexpr int NE = 10;   // equations

void residual_and_jacobian(const dd* x, dd* r, dd (*J)[NP]) {
  const dd C1 = div(D(-4216.0), D(625.0));
  const dd C2 = D(4.0);
  dd W[4], V[4];
  for (int j = 0; j < 4; ++j) {
    W[j] = add(mul(D(8.0), x[j]), mul(D(4.0), x[4 + j]));
    V[j] = add(mul(C1, x[j]), mul(C2, x[4 + j]));
  }
  double fact = 1.0;
  for (int K = 0; K <= 6; ++K) {
    if (K > 0) fact *= K;
    dd s = D(0.0);
    for (int j = 0; j < 4; ++j) {
      dd pk = D(1.0), pk1 = D(0.0);         // p0^K and p0^(K-1)
      for (int e = 0; e < K; ++e) { pk1 = pk; pk = mul(pk, x[8 + j]); }
      s = add(s, mul(W[j], pk));
      J[K][j] = mul(D(8.0), pk);
      J[K][4 + j] = mul(D(4.0), pk);
      J[K][8 + j] = K > 0 ? mul(mul(D((double)K), W[j]), pk1) : D(0.0);
    }
    r[K] = sub(s, D(fact));
  }
  for (int K = 4; K <= 6; ++K) {
    int row = 7 + (K - 4);
    dd s = D(0.0);
    for (int j = 0; j < 4; ++j) {
      dd pk = D(1.0), pk1 = D(0.0);
      for (int e = 0; e < K; ++e) { pk1 = pk; pk = mul(pk, x[8 + j]); }
      s = add(s, mul(V[j], pk));
      J[row][j] = mul(C1, pk);
      J[row][4 + j] = mul(C2, pk);
      J[row][8 + j] = mul(mul(D((double)K), V[j]), pk1);
    }
    r[row] = s;
  }
}

// Solves A y = b (NE x NE) by Gaussian elimination with partial pivoting.
bool solve(dd (*A)[NE], dd* b) {
  for (int c = 0; c < NE; ++c) {
    int piv = c;
    for (int r = c + 1; r < NE; ++r)
      if (std::fabs(A[r][c].hi) > std::fabs(A[piv][c].hi)) piv = r;
    if (A[piv][c].hi == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < NE; ++k) { dd t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
      dd t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    for (int r = c + 1; r < NE; ++r) {
      dd f = div(A[r][c], A[c][c]);
      for (int k = c; k < NE; ++k) A[r][k] = sub(A[r][k], mul(f, A[c][k]));
      b[r] = sub(b[r], mul(f, b[c]));
    }
  }
  for (int c = NE - 1; c >= 0; --c) {
    dd s = b[c];
    for (int k = c + 1; k < NE; ++k) s = sub(s, mul(A[c][k], b[k]));
    b[c] = div(s, A[c][c]);
  }
  return true;
}

}  // namespace

// Printed values of Sec. 2.3.
static const double kPrintedW1[4] = {0.003930503244, 0.008026424774, 0.000175706060, 0.042659667266};
static const double kPrintedW2[4] = {0.054642060984, 0.013535762740, 0.000296310700, 0.071941262878};
static const double kPrintedP0[4] = {0.000016359462, 3.305423649330, 7.758786843141, 0.935838587521};

// Returns false if the iteration failed to converge.
bool refine_quadrature(double w1[4], double w2[4], double p0[4]) {
  dd x[NP];
  for (int j = 0; j < 4; ++j) {
    x[j] = D(kPrintedW1[j]);
    x[4 + j] = D(kPrintedW2[j]);
    x[8 + j] = D(kPrintedP0[j]);
  }
  dd r[NE], J[NE][NP], A[NE][NE];
  for (int it = 0; it < 6; ++it) {
    residual_and_jacobian(x, r, J);
    // minimum-norm step: dx = -J^T (J J^T)^-1 r
    for (int a = 0; a < NE; ++a)
      for (int b = 0; b < NE; ++b) {
        dd s = D(0.0);
        for (int k = 0; k < NP; ++k) s = add(s, mul(J[a][k], J[b][k]));
        A[a][b] = s;
      }
    dd y[NE];
    for (int a = 0; a < NE; ++a) y[a] = r[a];
    if (!solve(A, y)) return false;
    for (int k = 0; k < NP; ++k) {
      dd s = D(0.0);
      for (int a = 0; a < NE; ++a) s = add(s, mul(J[a][k], y[a]));
      x[k] = sub(x[k], s);
    }
  }
  residual_and_jacobian(x, r, J);
  double worst = 0.0;
  for (int a = 0; a < NE; ++a) worst = std::fmax(worst, std::fabs(r[a].hi));
  if (!(worst < 1e-25)) return false;
  for (int j = 0; j < 4; ++j) {
    w1[j] = x[j].hi + x[j].lo;
    w2[j] = x[4 + j].hi + x[4 + j].lo;
    p0[j] = x[8 + j].hi + x[8 + j].lo;
  }
  return true;
}

}  // namespace rlbm

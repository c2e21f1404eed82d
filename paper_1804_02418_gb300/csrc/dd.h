// Double-double arithmetic for the host-side quadrature solves (about 32
// significant digits: a value is hi + lo with |lo| <= ulp(hi) / 2).  Error-free
// transformations (Knuth's two-sum, FMA-based two-product); the translation
// units that include this must be compiled without floating-point
// contraction.
#pragma once
#include <cmath>

namespace rlbm {
namespace ddm {

struct dd { double hi, lo; };

inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
inline dd quick_two_sum(double a, double b) {
  double s = a + b;
  return {s, b - (s - a)};
}
inline dd two_prod(double a, double b) {
  double p = a * b;
  return {p, std::fma(a, b, -p)};
}
inline dd add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
inline dd neg(dd a) { return {-a.hi, -a.lo}; }
inline dd sub(dd a, dd b) { return add(a, neg(b)); }
inline dd mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}
inline dd div(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = sub(a, mul(dd{q1, 0.0}, b));
  double q2 = r.hi / b.hi;
  r = sub(r, mul(dd{q2, 0.0}, b));
  double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return add(q, dd{q3, 0.0});
}
// square root: one Newton step from the FP64 root, s + (a - s^2) / (2 s)
inline dd sqrt(dd a) {
  if (a.hi <= 0.0) return {0.0, 0.0};
  double s = std::sqrt(a.hi);
  dd r = sub(a, two_prod(s, s));
  return add(dd{s, 0.0}, dd{r.hi / (2.0 * s), 0.0});
}
inline dd D(double x) { return {x, 0.0}; }
inline double to_double(dd a) { return a.hi + a.lo; }
inline bool less(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

}  // namespace ddm
}  // namespace rlbm

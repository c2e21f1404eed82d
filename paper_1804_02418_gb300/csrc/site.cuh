// Per-site arithmetic of the relativistic lattice Boltzmann step
// (Eq. discrete-rbe, the per-site algorithm at the end of Sec. 2, App. A-B).
//
// Everything here works on deviations from the rest equilibrium
// (n = T = 1, u = 0, where f^eq_i = w_i):  delta_i = f_i - w_i.  Rest values of
// the moments (N = (1,0,0), T = diag(2,1,1)) are added analytically, and the
// equilibrium coefficients are written in terms of the small quantities
// n - 1, T - 1, gamma - 1 and T gamma - 1, so FP32 arithmetic keeps full
// relative precision on the O(u) flux-carrying parts.
//
// The equilibrium Q(p) = sum_k a^(k) J^(k)(p) (App. A polynomials, App. B
// projections) is regrouped on the massless shell p = p0 (1, v) as
//     Q(p0 v) = sum_{m=0..3} p0^m q_m(v),
// with q_m(v) a polynomial of degree <= m in the unit velocity v.  Every
// population of one direction then costs a cubic in its shell energy p0_j.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace rlbm {

constexpr int kQ = 48;
constexpr int kDirs = 12;
constexpr int kShells = 4;
constexpr int kRadius = 5;
constexpr int kMaxContacts = 4;

// Stencil G = {(+-3,+-4)_FS, (+-5,0)_FS} (Sec. 2.3); opposite of d is d ^ 1.
__host__ __device__ constexpr int hop_x(int d) {
  return d == 0 ? 3 : d == 1 ? -3 : d == 2 ? -3 : d == 3 ? 3 : d == 4 ? 4 : d == 5 ? -4
       : d == 6 ? -4 : d == 7 ? 4 : d == 8 ? 5 : d == 9 ? -5 : 0;
}
__host__ __device__ constexpr int hop_y(int d) {
  return d == 0 ? 4 : d == 1 ? -4 : d == 2 ? 4 : d == 3 ? -4 : d == 4 ? 3 : d == 5 ? -3
       : d == 6 ? 3 : d == 7 ? -3 : d == 8 ? 0 : d == 9 ? 0 : d == 10 ? 5 : -5;
}
__host__ __device__ constexpr int dir_kind(int d) { return d < 8 ? 0 : 1; }

// Quadrature constants (refined Sec. 2.3 values), uploaded once per module.
template <typename R>
struct QuadConsts {
  R p0[kShells];            // shell energies p0_j
  R w[2][kShells];          // weights by direction kind and shell
  R dec[2][kShells];        // 16-bit storage: delta = g * dec  (dec = w / s)
  R enc[2][kShells];        // 16-bit storage: g = delta * enc  (enc = s / w)
};

// Geometry and physics of one sample as seen by the kernels.
struct DevSample {
  int nx, ny, ldx;                    // ldx: row pitch in elements
  int periodic_x, periodic_y;
  int ncontacts;
  long long plane;                    // elements per population plane
  long long site0;                    // first site of this sample in the flat u / mask arrays
  double inv_tau;
  double Fx, Fy;
  int cedge[kMaxContacts], clo[kMaxContacts], chi[kMaxContacts];
};

// Error bits of the device error word.
constexpr unsigned kErrNonFinite = 1u;
constexpr unsigned kErrUnphysical = 2u;
constexpr unsigned kErrNoConvergence = 4u;

// ---------------------------------------------------------------------------
// Storage codecs: the stored value of population q and its deviation delta.
// ---------------------------------------------------------------------------
template <typename S> struct Codec;
template <> struct Codec<double> {
  using R = double;
  template <class C> __device__ static R load(double v, int, const C&) { return v; }
  template <class C> __device__ static double store(R v, int, const C&) { return v; }
};
template <> struct Codec<float> {
  using R = float;
  template <class C> __device__ static R load(float v, int, const C&) { return v; }
  template <class C> __device__ static float store(R v, int, const C&) { return v; }
};
template <> struct Codec<__half> {
  using R = float;
  template <class C> __device__ static R load(__half v, int q, const C& c) {
    return __half2float(v) * c.dec[dir_kind(q >> 2)][q & 3];
  }
  template <class C> __device__ static __half store(R v, int q, const C& c) {
    return __float2half_rn(v * c.enc[dir_kind(q >> 2)][q & 3]);
  }
};
template <> struct Codec<__nv_bfloat16> {
  using R = float;
  template <class C> __device__ static R load(__nv_bfloat16 v, int q, const C& c) {
    return __bfloat162float(v) * c.dec[dir_kind(q >> 2)][q & 3];
  }
  template <class C> __device__ static __nv_bfloat16 store(R v, int q, const C& c) {
    return __float2bfloat16_rn(v * c.enc[dir_kind(q >> 2)][q & 3]);
  }
};

// ---------------------------------------------------------------------------
// Macroscopic state of one site (deviation form).
// ---------------------------------------------------------------------------
template <typename R>
struct Macro {
  R ux, uy;
  R gamma, gm1;   // gamma and gamma - 1
  R dn, dT;       // n - 1, T - 1
  R deps;         // eps - 2
};

template <typename R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
template <> __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }

template <typename R> struct Tol;
template <> struct Tol<double> { static constexpr double v = 1e-15; };
template <> struct Tol<float> { static constexpr float v = 2e-7f; };

// Moment deviations from 48 streamed deviations.
template <typename R>
struct Moments {
  R dN0, dNx, dNy;              // N^a - (1, 0, 0)
  R dE, Mx, My, dPxx, dPxy, dPyy; // T^ab - diag(2, 1, 1)
};

template <typename R, class C>
__device__ __forceinline__ Moments<R> moments(const R (&f)[kQ], const C& qc) {
  Moments<R> m;
  m.dN0 = m.dNx = m.dNy = m.dE = m.Mx = m.My = m.dPxx = m.dPxy = R(0);
#pragma unroll
  for (int d = 0; d < kDirs; ++d) {
    // A_d = sum_j delta_dj p0_j ; B_d = sum_j delta_dj p0_j^2
    R A = R(0), B = R(0);
#pragma unroll
    for (int j = 0; j < kShells; ++j) {
      const R t = f[4 * d + j] * qc.p0[j];
      A += t;
      B = fma(t, qc.p0[j], B);
    }
    const R vx = R(hop_x(d)) / R(5), vy = R(hop_y(d)) / R(5);
    m.dN0 += A;
    if (hop_x(d) != 0) m.dNx = fma(A, vx, m.dNx);
    if (hop_y(d) != 0) m.dNy = fma(A, vy, m.dNy);
    m.dE += B;
    if (hop_x(d) != 0) {
      const R Bx = B * vx;
      m.Mx += Bx;
      m.dPxx = fma(Bx, vx, m.dPxx);
      if (hop_y(d) != 0) m.dPxy = fma(Bx, vy, m.dPxy);
    }
    if (hop_y(d) != 0) m.My = fma(B, vy, m.My);
  }
  m.dPyy = m.dE - m.dPxx;   // massless shells: T^00 = T^xx + T^yy exactly
  return m;
}

// Landau frame eps U^a = T^ab U_b:  u = (Pi + eps I)^-1 M, eps = E - M.u,
// Newton on g(eps) = eps - E + M.u(eps), g' = 1 - u.u, from eps0 = E.
// Then n = U_a N^a and the massless EOS eps = 2 n T.
template <typename R>
__device__ __forceinline__ bool landau(const Moments<R>& m, Macro<R>& o) {
  R deps = m.dE;
  R ux = R(0), uy = R(0);
  bool conv = false;
#pragma unroll 1
  for (int it = 0; it < 12; ++it) {
    const R a = R(3) + m.dPxx + deps, c = R(3) + m.dPyy + deps;
    const R inv = R(1) / (a * c - m.dPxy * m.dPxy);
    ux = (c * m.Mx - m.dPxy * m.My) * inv;
    uy = (a * m.My - m.dPxy * m.Mx) * inv;
    const R g = deps - m.dE + m.Mx * ux + m.My * uy;
    const R step = g / (R(1) - ux * ux - uy * uy);
    deps -= step;
    if (fabs(step) <= Tol<R>::v * (R(2) + fabs(deps))) { conv = true; break; }
  }
  {
    const R a = R(3) + m.dPxx + deps, c = R(3) + m.dPyy + deps;
    const R inv = R(1) / (a * c - m.dPxy * m.dPxy);
    ux = (c * m.Mx - m.dPxy * m.My) * inv;
    uy = (a * m.My - m.dPxy * m.Mx) * inv;
  }
  const R u2 = ux * ux + uy * uy;
  const R s = sqrt(R(1) - u2);
  const R gamma = R(1) / s;
  const R gm1 = u2 * gamma / (R(1) + s);
  const R dNpar = m.dN0 - ux * m.dNx - uy * m.dNy;     // U_a N^a / gamma - 1
  const R dn = gm1 * (R(1) + dNpar) + dNpar;           // n - 1
  const R dT = (deps - R(2) * dn) / (R(2) * (R(1) + dn));  // T - 1 = eps/(2n) - 1
  o.ux = ux; o.uy = uy; o.gamma = gamma; o.gm1 = gm1; o.dn = dn; o.dT = dT; o.deps = deps;
  return conv;
}

// Coefficients of Q(p0 v) - 1 = q0m1 + sum_{m=1..3} p0^m q_m(v) with
//   q1 = c1_0 + c1_x vx + c1_y vy
//   q2 = c2_0 + c2_x vx + c2_y vy + c2_xx vx^2 + c2_xy vx vy
//   q3 = c3_0 + c3_x vx + c3_y vy + c3_xx vx^2 + c3_xy vx vy + c3_xxx vx^3 + c3_xxy vx^2 vy
// obtained by substituting p = p0 (1, v) in the App. A polynomials and
// weighting them with the App. B projections.
template <typename R>
struct EqCoeffs {
  R q0m1;
  R c1_0, c1_x, c1_y;
  R c2_0, c2_x, c2_y, c2_xx, c2_xy;
  R c3_0, c3_x, c3_y, c3_xx, c3_xy, c3_xxx, c3_xxy;
};

template <typename R>
__device__ __forceinline__ EqCoeffs<R> eq_coeffs(const Macro<R>& M) {
  const R s3 = R(1.7320508075688772), s15 = R(3.872983346207417);
  const R s53 = R(1.2909944487358056), s6 = R(2.449489742783178);
  const R s23 = R(0.816496580927726), s25 = R(0.6324555320336759);
  const R s10 = R(3.1622776601683795), s32 = R(1.224744871391589), s52 = R(1.5811388300841898);
  const R T = R(1) + M.dT;
  const R g = M.gamma;
  const R uX = g * M.ux, uY = g * M.uy;
  const R Tu = M.dT + M.gm1 + M.dT * M.gm1;          // T u^0 - 1
  const R gT = M.gm1 * T;                            // (gamma - 1) T
  const R dT2 = M.dT * M.dT;
  const R T2 = T * T;
  const R g2 = g * g;
  // App. B projections (rest-deviation form, algebraically identical)
  const R a10 = Tu;
  const R a1x = T * uX;
  const R a1y = T * uY;
  // Tu - (T^2 - 1)/2 = (gamma - 1) T - (T - 1)^2 / 2, and alike below
  const R a200 = R(1.5) * Tu * Tu + gT - R(0.5) * dT2;
  const R a20x = s3 * T * uX * Tu;
  const R a20y = s3 * T * uY * Tu;
  const R dxy2 = g2 * (M.ux * M.ux - M.uy * M.uy);    // u0^2 - 1 - 2 uX^2 = -dxy2
  const R a2xx = R(0.5) * s3 * T2 * dxy2;
  const R a2xy = s3 * T2 * uX * uY;
  const R a3000 = R(0.5) * Tu * (R(5) * Tu * Tu + R(6) * gT - R(3) * dT2);
  const R a3xxx = R(0.5) * T * uX * (R(5) * T2 * uX * uX + R(3) * dT2 - R(6) * gT);
  const R a300x = R(-0.5) * s15 * T * uX * (R(-2) * Tu * Tu + T2 * uX * uX + dT2 - R(2) * gT);
  const R a30xx = R(0.5) * s15 * T2 * Tu * dxy2;
  const R a300y = R(0.5) * s32 * T * uY * (R(5) * Tu * Tu + R(2) * gT - dT2);
  const R a3xxy = R(-0.5) * s52 * T2 * T * uY * g2 * (M.uy * M.uy - R(3) * M.ux * M.ux);
  const R a30xy = s15 * T2 * uX * uY * Tu;

  EqCoeffs<R> c;
  c.q0m1 = -a10 + a200 - a3000;
  c.c1_0 = a10 - R(2) * a200 + R(3) * a3000;
  c.c1_x = a1x - s3 * a20x + R(1.5) * a3xxx + R(0.5) * s15 * a300x;
  c.c1_y = a1y - s3 * a20y + s6 * a300y;
  c.c2_0 = R(0.5) * a200 - a2xx / (R(2) * s3) - R(1.5) * a3000 + R(0.5) * s53 * a30xx;
  c.c2_x = a20x / s3 - a3xxx - s53 * a300x;
  c.c2_y = a20y / s3 - R(2) * s23 * a300y;
  c.c2_xx = a2xx / s3 - s53 * a30xx;
  c.c2_xy = a2xy / s3 - s53 * a30xy;
  c.c3_0 = a3000 / R(6) - a30xx / (R(2) * s15);
  c.c3_x = a300x / s15;
  c.c3_y = a300y / (R(2) * s6) - a3xxy / (R(6) * s10);
  c.c3_xx = a30xx / s15;
  c.c3_xy = a30xy / s15;
  c.c3_xxx = a3xxx / R(6) - a300x / (R(2) * s15);
  c.c3_xxy = s25 / R(3) * a3xxy;
  return c;
}

// Per-direction cubic R_0 + R_1 p0 + R_2 p0^2 + R_3 p0^3 such that the new
// deviation of shell j is  (1 - omega_d) delta_dj + w_dj (sum_m R_m p0_j^m):
//   omega_d (f^eq - w) / w  +  F^ext / w,
// with omega_d = gamma (1 - v_d.u) / tau (= p^m U_m / (p^0 tau) on the massless shell).
// Forcing (force F per particle, dt = 1):
//   F^ext / w = (n/T) [ (F.v) Q - F.grad Q ]  at p = p0 (1, v),
// where grad is the gradient along the shell; with Q = sum_m p0^m q_m(theta)
//   F.grad Q = sum_m p0^(m-1) [ m q_m (F.v) + dq_m/dtheta (F.t) ],  t = (-vy, vx).
template <typename R, bool FORCE>
__device__ __forceinline__ void direction_cubic(const int d, const EqCoeffs<R>& c, R nT, R nmT,
                                                R omega, R Fv, R Ft, R (&Rm)[4]) {
  const R vx = R(hop_x(d)) / R(5), vy = R(hop_y(d)) / R(5);
  const R q1 = c.c1_0 + c.c1_x * vx + c.c1_y * vy;
  const R q2 = c.c2_0 + c.c2_x * vx + c.c2_y * vy + c.c2_xx * (vx * vx) + c.c2_xy * (vx * vy);
  const R q3 = c.c3_0 + c.c3_x * vx + c.c3_y * vy + c.c3_xx * (vx * vx) + c.c3_xy * (vx * vy)
             + c.c3_xxx * (vx * vx * vx) + c.c3_xxy * (vx * vx * vy);
  const R on = omega * nT;
  Rm[0] = fma(omega, nmT, on * c.q0m1);
  Rm[1] = on * q1;
  Rm[2] = on * q2;
  Rm[3] = on * q3;
  if (FORCE) {
    // dq_m/dtheta = -vy dq/dvx + vx dq/dvy
    const R t1 = -vy * c.c1_x + vx * c.c1_y;
    const R t2 = -vy * (c.c2_x + R(2) * vx * c.c2_xx + vy * c.c2_xy) + vx * (c.c2_y + vx * c.c2_xy);
    const R t3 = -vy * (c.c3_x + R(2) * vx * c.c3_xx + vy * c.c3_xy + R(3) * (vx * vx) * c.c3_xxx
                        + R(2) * (vx * vy) * c.c3_xxy)
               + vx * (c.c3_y + vx * c.c3_xy + (vx * vx) * c.c3_xxy);
    const R q0 = R(1) + c.q0m1;
    const R s0 = Fv * (q0 - q1) - Ft * t1;
    const R s1 = Fv * (q1 - R(2) * q2) - Ft * t2;
    const R s2 = Fv * (q2 - R(3) * q3) - Ft * t3;
    const R s3 = Fv * q3;
    Rm[0] = fma(nT, s0, Rm[0]);
    Rm[1] = fma(nT, s1, Rm[1]);
    Rm[2] = fma(nT, s2, Rm[2]);
    Rm[3] = fma(nT, s3, Rm[3]);
  }
}

template <typename R>
__device__ __forceinline__ bool macro_ok(const Macro<R>& M) {
  const R u2 = M.ux * M.ux + M.uy * M.uy;
  return (u2 < R(1)) && (M.dn > R(-1)) && (M.dT > R(-1));
}

template <typename R>
__device__ __forceinline__ bool all_finite(const Macro<R>& M) {
  return isfinite(M.ux) && isfinite(M.uy) && isfinite(M.dn) && isfinite(M.dT);
}

}  // namespace rlbm

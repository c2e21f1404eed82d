// Per-site arithmetic of the relativistic lattice Boltzmann step
// (Eq. discrete-rbe, the per-site algorithm at the end of Sec. 2, App. A-B).
//
// Everything here works on relative deviations from the rest equilibrium
// (n = T = 1, u = 0, where f^eq_i = w_i):  g_i = (f_i - w_i) / w_i, the value
// every storage type keeps (16-bit storage scaled by s); delta_i = w_i g_i.
// Rest values of the moments (N = (1,0,0), T = diag(2,1,1)) are added
// analytically, and the
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

#include <type_traits>

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

// Odd monomials of a unit velocity v whose (a, -a) pairs the paired FP32
// collision uses (order of QuadConsts::odd).
enum OddMono {
  kOVx = 0, kOVy, kONVx, kONVy,   // vx, vy, -vx, -vy
  kOVx3, kOVx2y,                  // vx^3, vx^2 vy
  kO3x2y, kOX3m2xy2,              // 3 vx^2 vy, -(vx^3 - 2 vx vy^2)
  kOddMonos
};

__host__ __device__ constexpr double odd_mono(int d, int o) {
  const double vx = hop_x(d) / 5.0, vy = hop_y(d) / 5.0;
  return o == kOVx ? vx : o == kOVy ? vy : o == kONVx ? -vx : o == kONVy ? -vy
       : o == kOVx3 ? vx * vx * vx : o == kOVx2y ? vx * vx * vy
       : o == kO3x2y ? 3.0 * vx * vx * vy : -(vx * vx * vx - 2.0 * vx * vy * vy);
}

// Quadrature constants (refined Sec. 2.3 values), uploaded once per module.
template <typename R>
struct QuadConsts {
  R p0[kShells];            // shell energies p0_j
  R w[2][kShells];          // weights by direction kind and shell
  R wp0[2][kShells];        // w p0_j / s   (moments of the stored s g; s = 1 above 16 bits)
  R wp0sq[2][kShells];      // w p0_j^2 / s
  R dec_s, enc_s;           // 16-bit storage scale: 1 / s, s (the 16-bit kernels compute on s g)
  double wd[2][kShells];    // w in FP64: state I/O converts g <-> delta = w g in FP64
  // Conservation projection (reduced precision): correction
  // w_2j (l0 + l1 p0_j + p0_j (lx vx + ly vy)) on the (5,0)-type directions,
  // (l0, l1) = P (rN, rE), (lx, ly) = px (rX, rY).
  R P00, P01, P10, P11, px;
  // Operand pairs of the paired FP32 arithmetic (FP32 kernels only).  Pair
  // lanes are (direction d, its opposite d + 1) in the collision and (shell
  // j, shell j + 1) in the relaxation; a constant pair read from here costs
  // nothing as an operand, a literal pair of two different values would.
  // odd[q][o]: (a, -a) for the odd monomial o of direction pair q = d / 2.
  float2 odd[kDirs / 2][kOddMonos];
  float2 vxy[kDirs / 2];      // (vx, vy) of direction 2q
  float2 vsq[kDirs / 2];      // (vx^2, vx vy) of direction 2q
  float2 wab[2][kShells];     // (w p0_j / s, w p0_j^2 / s) by direction kind
  float2 p01, p23;            // (p0_0, p0_1), (p0_2, p0_3)
};

// Geometry and physics of one sample as seen by the kernels.
struct DevSample {
  int nx, ny, ldx;                    // ldx: row pitch in elements
  int periodic_x, periodic_y;
  int ncontacts;
  long long plane;                    // elements per population plane
  long long site0;                    // first site of this sample in the flat u / mask arrays
  long long off[2];                   // element offsets of the two buffers (batched launches)
  double inv_tau;
  double Fx, Fy;
  int cedge[kMaxContacts], clo[kMaxContacts], chi[kMaxContacts];
  // electric force of the local capacitance approximation (Sec. 3): coupling
  // e^2 / C_g (0: none) and two planes of n - 1 in the arithmetic type, same
  // site indexing as a population plane; dn[cur] holds the previous step's
  // density, dn[cur ^ 1] receives this step's
  double inv_cg;
  void* dn[2];
  int cur;
};

// Error bits of the device error word.
constexpr unsigned kErrNonFinite = 1u;
constexpr unsigned kErrUnphysical = 2u;
constexpr unsigned kErrNoConvergence = 4u;
constexpr unsigned kErrTimeout = 8u;      // a bounded wait inside a kernel gave up

// ---------------------------------------------------------------------------
// Storage codecs.  The four shells of one (direction, site) are stored side by
// side, so one aligned vector access moves them (16 B for FP32, 32 B for FP64,
// 8 B for 16-bit storage).  `kind` selects the weight row (0: (3,4)-type,
// 1: (5,0)-type) for the 16-bit scaled relative deviations.
// ---------------------------------------------------------------------------
template <typename S> struct Codec;
template <> struct Codec<double> {
  using R = double;
  template <class C>
  __device__ static void load4(const double* p, int, const C&, R* o) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
  // from shared memory (32-bit shared-window address)
  template <class C>
  __device__ static void load4s(uint32_t a, int, const C&, R* o) {
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(o[0]), "=d"(o[1]) : "r"(a));
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(o[2]), "=d"(o[3]) : "r"(a + 16));
  }
  template <class C>
  __device__ static void store4(double* p, int, const C&, const R* v) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
  // stored relative deviation g <-> deviation delta = f - w (state I/O, in
  // FP64; the round trip can move a value by one ulp)
  template <class C> __device__ static double decode(double v, int kind, int j, const C& c) {
    return v * c.wd[kind][j];
  }
  template <class C> __device__ static double encode(double v, int kind, int j, const C& c) {
    return v / c.wd[kind][j];
  }
};
template <> struct Codec<float> {
  using R = float;
  template <class C>
  __device__ static void load4(const float* p, int, const C&, R* o) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  }
  template <class C>
  __device__ static void load4s(uint32_t a, int, const C&, R* o) {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]) : "r"(a));
  }
  template <class C>
  __device__ static void store4(float* p, int, const C&, const R* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
  // in FP64: delta = g w to 1e-16, and delta / w rounds back to g exactly
  template <class C> __device__ static double decode(float v, int kind, int j, const C& c) {
    return double(v) * c.wd[kind][j];
  }
  template <class C> __device__ static float encode(double v, int kind, int j, const C& c) {
    return float(v / c.wd[kind][j]);
  }
};
template <typename H> struct Codec16 {
  using R = float;
  __device__ static float tof(H h);
  __device__ static H fromf(float f);
  // two stored values <-> two floats (one conversion instruction per pair)
  __device__ static float2 unpack2(uint32_t u);
  __device__ static uint32_t pack2(float a, float b);
  template <class C>
  __device__ static void load4(const H* p, int kind, const C& c, R* o) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = unpack2(u.x), b = unpack2(u.y);   // s g: the kernels work scaled
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
  template <class C>
  __device__ static void load4s(uint32_t a, int kind, const C& c, R* o) {
    uint2 u;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];\n" : "=r"(u.x), "=r"(u.y) : "r"(a));
    const float2 x = unpack2(u.x), y = unpack2(u.y);
    o[0] = x.x; o[1] = x.y; o[2] = y.x; o[3] = y.y;
  }
  template <class C>
  __device__ static void store4(H* p, int kind, const C& c, const R* v) {
    *reinterpret_cast<uint2*>(p) = make_uint2(pack2(v[0], v[1]), pack2(v[2], v[3]));
  }
  // stored s g <-> deviation delta = f - w (state I/O, in FP64: exact round trip)
  template <class C> __device__ static double decode(H v, int kind, int j, const C& c) {
    return double(tof(v)) * double(c.dec_s) * c.wd[kind][j];
  }
  template <class C> __device__ static H encode(double v, int kind, int j, const C& c) {
    return fromf(float(v / c.wd[kind][j] * double(c.enc_s)));
  }
};
template <> __device__ inline float2 Codec16<__half>::unpack2(uint32_t u) {
  __half2 h;
  memcpy(&h, &u, sizeof u);
  return __half22float2(h);
}
template <> __device__ inline uint32_t Codec16<__half>::pack2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  uint32_t u;
  memcpy(&u, &h, sizeof u);
  return u;
}
template <> __device__ inline float2 Codec16<__nv_bfloat16>::unpack2(uint32_t u) {
  __nv_bfloat162 h;
  memcpy(&h, &u, sizeof u);
  return __bfloat1622float2(h);
}
template <> __device__ inline uint32_t Codec16<__nv_bfloat16>::pack2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  uint32_t u;
  memcpy(&u, &h, sizeof u);
  return u;
}
template <> __device__ inline float Codec16<__half>::tof(__half h) { return __half2float(h); }
template <> __device__ inline __half Codec16<__half>::fromf(float f) { return __float2half_rn(f); }
template <> __device__ inline float Codec16<__nv_bfloat16>::tof(__nv_bfloat16 h) { return __bfloat162float(h); }
template <> __device__ inline __nv_bfloat16 Codec16<__nv_bfloat16>::fromf(float f) { return __float2bfloat16_rn(f); }
template <> struct Codec<__half> : Codec16<__half> {};
template <> struct Codec<__nv_bfloat16> : Codec16<__nv_bfloat16> {};

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

// Quotient and square root: correctly rounded in FP64; in FP32 the fast
// hardware approximations (a few ulp), whose error is far below the FP32
// storage rounding the arithmetic feeds.
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float qsqrt(float a) { return a * rsqrtf(a); }

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
__device__ __forceinline__ Moments<R> moments_scalar(const R (&f)[kQ], const C& qc) {
  Moments<R> m;
  m.dN0 = m.dNx = m.dNy = m.dE = m.Mx = m.My = m.dPxx = m.dPxy = R(0);
#pragma unroll
  for (int d = 0; d < kDirs; d += 2) {
    // directions d and d + 1 are opposite: v_{d+1} = -v_d
    R Ap = R(0), Bp = R(0), An = R(0), Bn = R(0);
#pragma unroll
    for (int j = 0; j < kShells; ++j) {
      // relative deviations: delta = w g
      const int k = dir_kind(d);
      Ap = fma(f[4 * d + j], qc.wp0[k][j], Ap);
      Bp = fma(f[4 * d + j], qc.wp0sq[k][j], Bp);
      An = fma(f[4 * d + 4 + j], qc.wp0[k][j], An);
      Bn = fma(f[4 * d + 4 + j], qc.wp0sq[k][j], Bn);
    }
    const R vx = R(hop_x(d)) / R(5), vy = R(hop_y(d)) / R(5);
    const R Ae = Ap + An, Ao = Ap - An, Be = Bp + Bn, Bo = Bp - Bn;
    m.dN0 += Ae;
    m.dE += Be;
    if (hop_x(d) != 0) {
      m.dNx = fma(Ao, vx, m.dNx);
      m.Mx = fma(Bo, vx, m.Mx);
      m.dPxx = fma(Be, vx * vx, m.dPxx);
      if (hop_y(d) != 0) m.dPxy = fma(Be, vx * vy, m.dPxy);
    }
    if (hop_y(d) != 0) {
      m.dNy = fma(Ao, vy, m.dNy);
      m.My = fma(Bo, vy, m.My);
    }
  }
  m.dPyy = m.dE - m.dPxx;   // massless shells: T^00 = T^xx + T^yy exactly
  return m;
}

// ---------------------------------------------------------------------------
// Paired FP32 arithmetic.  Blackwell retires two FP32 fused multiply-adds per
// instruction on a register pair (the same per-lane rounding as two scalar
// ones); the FP32 step is bound by its instruction issue, so its collision is
// written on pairs.  A pair whose lanes hold the same value ("splat") costs
// nothing extra as an operand.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 S2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// The moments of moments() on pairs: lanes (A_d, B_d) of one direction,
// A_d = sum_j w p0_j g_dj, B_d = sum_j w p0_j^2 g_dj.
template <class C>
__device__ __forceinline__ Moments<float> moments_paired(const float (&f)[kQ], const C& qc) {
  float2 NE = S2(0.f), NxMx = S2(0.f), NyMy = S2(0.f), PP = S2(0.f);
#pragma unroll
  for (int d = 0; d < kDirs; d += 2) {
    const int k = dir_kind(d);
    float2 ABp = mul2(S2(f[4 * d]), qc.wab[k][0]);
    float2 ABn = mul2(S2(f[4 * d + 4]), qc.wab[k][0]);
#pragma unroll
    for (int j = 1; j < kShells; ++j) {
      ABp = fma2(S2(f[4 * d + j]), qc.wab[k][j], ABp);
      ABn = fma2(S2(f[4 * d + 4 + j]), qc.wab[k][j], ABn);
    }
    const float2 e = add2(ABp, ABn);                 // (A_e, B_e): even parts
    const float2 o = fma2(ABn, S2(-1.f), ABp);       // (A_o, B_o): odd parts
    const float vx = float(hop_x(d)) / 5.f, vy = float(hop_y(d)) / 5.f;
    if (d == 0) {
      NE = e;
      NxMx = mul2(o, S2(vx));
      NyMy = mul2(o, S2(vy));
      PP = mul2(S2(e.y), qc.vsq[d / 2]);
    } else {
      NE = add2(NE, e);
      if (hop_x(d) != 0) NxMx = fma2(o, S2(vx), NxMx);
      if (hop_y(d) != 0) NyMy = fma2(o, S2(vy), NyMy);
      if (hop_x(d) != 0) PP = fma2(S2(e.y), qc.vsq[d / 2], PP);
    }
  }
  Moments<float> m;
  m.dN0 = NE.x; m.dE = NE.y;
  m.dNx = NxMx.x; m.Mx = NxMx.y;
  m.dNy = NyMy.x; m.My = NyMy.y;
  m.dPxx = PP.x; m.dPxy = PP.y;
  m.dPyy = m.dE - m.dPxx;   // massless shells: T^00 = T^xx + T^yy exactly
  return m;
}

// Moment deviations of 48 streamed relative deviations: paired in FP32,
// scalar in FP64.
template <typename R, class C>
__device__ __forceinline__ Moments<R> moments(const R (&f)[kQ], const C& qc) {
  if constexpr (std::is_same<R, float>::value) return moments_paired(f, qc);
  else return moments_scalar(f, qc);
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
    const R inv = qdiv(R(1), a * c - m.dPxy * m.dPxy);
    ux = (c * m.Mx - m.dPxy * m.My) * inv;
    uy = (a * m.My - m.dPxy * m.Mx) * inv;
    const R g = deps - m.dE + m.Mx * ux + m.My * uy;
    const R step = qdiv(g, R(1) - ux * ux - uy * uy);
    deps -= step;
    if (fabs(step) <= Tol<R>::v * (R(2) + fabs(deps))) { conv = true; break; }
  }
  {
    const R a = R(3) + m.dPxx + deps, c = R(3) + m.dPyy + deps;
    const R inv = qdiv(R(1), a * c - m.dPxy * m.dPxy);
    ux = (c * m.Mx - m.dPxy * m.My) * inv;
    uy = (a * m.My - m.dPxy * m.Mx) * inv;
  }
  const R u2 = ux * ux + uy * uy;
  const R s = qsqrt(R(1) - u2);
  const R gamma = qdiv(R(1), s);
  const R gm1 = qdiv(u2 * gamma, R(1) + s);
  const R dNpar = m.dN0 - ux * m.dNx - uy * m.dNy;     // U_a N^a / gamma - 1
  const R dn = gm1 * (R(1) + dNpar) + dNpar;           // n - 1
  const R dT = qdiv(deps - R(2) * dn, R(2) * (R(1) + dn));  // T - 1 = eps/(2n) - 1
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
  // reciprocals of the App. A normalisations (multiplications, not divisions)
  const R i_s3 = R(0.57735026918962576), i_2s3 = R(0.28867513459481288);
  const R i_s15 = R(0.25819888974716112), i_2s15 = R(0.12909944487358056);
  const R i_2s6 = R(0.20412414523193151), i_6s10 = R(0.052704627669472988);
  const R i_6 = R(1.0 / 6.0), s25_3 = R(0.21081851067789195);
  c.c2_0 = R(0.5) * a200 - a2xx * i_2s3 - R(1.5) * a3000 + R(0.5) * s53 * a30xx;
  c.c2_x = a20x * i_s3 - a3xxx - s53 * a300x;
  c.c2_y = a20y * i_s3 - R(2) * s23 * a300y;
  c.c2_xx = a2xx * i_s3 - s53 * a30xx;
  c.c2_xy = a2xy * i_s3 - s53 * a30xy;
  c.c3_0 = a3000 * i_6 - a30xx * i_2s15;
  c.c3_x = a300x * i_s15;
  c.c3_y = a300y * i_2s6 - a3xxy * i_6s10;
  c.c3_xx = a30xx * i_s15;
  c.c3_xy = a30xy * i_s15;
  c.c3_xxx = a3xxx * i_6 - a300x * i_2s15;
  c.c3_xxy = s25_3 * a3xxy;
  return c;
}

// Per-direction cubic R_0 + R_1 p0 + R_2 p0^2 + R_3 p0^3 such that the new
// deviation of shell j is  (1 - omega_d) delta_dj + w_dj (sum_m R_m p0_j^m):
//   omega_d (f^eq - w) / w  +  F^ext / w,
// with omega_d = gamma (1 - v_d.u) / tau (= p^m U_m / (p^0 tau) on the massless shell).
// Forcing (force F per particle, dt = 1):
//   F^ext / w = (n/T) [ (F.v) Q - F.grad Q ]  at p = p0 (1, v),
// where grad is the gradient along the shell; with Q = sum_m p0^m q_m(theta)
//   F.grad Q = sum_m p0^(m-1) [ m q_m (F.v) + dq_m/dtheta (F.t) ],  t = (-vy, vx),
// so the p0^m coefficient of the source is
//   s_m = (F.v) (q_m - (m+1) q_{m+1}) - (F.t) dq_{m+1}/dtheta.
// Directions d (even) and d + 1 have opposite velocities; every polynomial is
// split into its even and odd parts in v, evaluated once for the pair.
// gux = gamma u_x / tau, guy = gamma u_y / tau, gt = gamma / tau.
template <typename R, bool FORCE>
__device__ __forceinline__ void pair_cubics(const int d, const EqCoeffs<R>& c, R nT, R nmT,
                                            R gt, R gux, R guy, R Fx, R Fy,
                                            R (&Rp)[4], R (&Rn)[4], R& omp, R& omn) {
  const R vx = R(hop_x(d)) / R(5), vy = R(hop_y(d)) / R(5);
  R ow = R(0);
  if (hop_x(d) != 0) ow = gux * vx;
  if (hop_y(d) != 0) ow = fma(guy, vy, ow);
  omp = gt - ow;
  omn = gt + ow;
  const R E2 = c.c2_0 + c.c2_xx * (vx * vx) + c.c2_xy * (vx * vy);
  const R E3 = c.c3_0 + c.c3_xx * (vx * vx) + c.c3_xy * (vx * vy);
  const R O1 = c.c1_x * vx + c.c1_y * vy;
  const R O2 = c.c2_x * vx + c.c2_y * vy;
  const R O3 = c.c3_x * vx + c.c3_y * vy + c.c3_xxx * (vx * vx * vx) + c.c3_xxy * (vx * vx * vy);
  const R q1p = c.c1_0 + O1, q1n = c.c1_0 - O1;
  const R q2p = E2 + O2, q2n = E2 - O2;
  const R q3p = E3 + O3, q3n = E3 - O3;
  const R onp = omp * nT, onn = omn * nT;
  Rp[0] = fma(omp, nmT, onp * c.q0m1);
  Rn[0] = fma(omn, nmT, onn * c.q0m1);
  Rp[1] = onp * q1p;
  Rn[1] = onn * q1n;
  Rp[2] = onp * q2p;
  Rn[2] = onn * q2n;
  Rp[3] = onp * q3p;
  Rn[3] = onn * q3n;
  if (FORCE) {
    // F.v and F.t flip sign between the two directions; dq_m/dtheta = Et_m +- Ot_m
    const R Fv = Fx * vx + Fy * vy, Ft = Fy * vx - Fx * vy;
    const R Ot1 = -vy * c.c1_x + vx * c.c1_y;
    const R Ot2 = -vy * c.c2_x + vx * c.c2_y;
    const R Et2 = R(-2) * (vx * vy) * c.c2_xx + (vx * vx - vy * vy) * c.c2_xy;
    const R Ot3 = -vy * c.c3_x + vx * c.c3_y - R(3) * (vx * vx * vy) * c.c3_xxx
                + (vx * vx * vx - R(2) * vx * vy * vy) * c.c3_xxy;
    const R Et3 = R(-2) * (vx * vy) * c.c3_xx + (vx * vx - vy * vy) * c.c3_xy;
    const R q0 = R(1) + c.q0m1;
    const R FvT = Fv * nT, FtT = Ft * nT;
    Rp[0] = fma(FvT, q0 - q1p, fma(-FtT, Ot1, Rp[0]));
    Rn[0] = fma(-FvT, q0 - q1n, fma(-FtT, Ot1, Rn[0]));
    Rp[1] = fma(FvT, q1p - R(2) * q2p, fma(-FtT, Et2 + Ot2, Rp[1]));
    Rn[1] = fma(-FvT, q1n - R(2) * q2n, fma(FtT, Et2 - Ot2, Rn[1]));
    Rp[2] = fma(FvT, q2p - R(3) * q3p, fma(-FtT, Et3 + Ot3, Rp[2]));
    Rn[2] = fma(-FvT, q2n - R(3) * q3n, fma(FtT, Et3 - Ot3, Rn[2]));
    Rp[3] = fma(FvT, q3p, Rp[3]);
    Rn[3] = fma(-FvT, q3n, Rn[3]);
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

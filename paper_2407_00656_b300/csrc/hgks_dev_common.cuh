// hgks_dev_common.cuh -- device helpers of the HGKS kernels: loads and
// conversions, Maxwellian moments and their parameter derivatives, the
// gas-kinetic flux at one point (Section 2.1, Eq. flux), boundary states, the
// time-step bound and its reductions, ghost cells and the control kernels.
//
// Precision: Real = double (FP64) or float (FP32-mixed: reconstruction and
// flux in binary32; geometry, pseudo-inverses and S2O4 sums in binary64).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <type_traits>

#include "hgks_internal.h"
#include "erfcx_table.h"

namespace hgks {
namespace {
constexpr int kBlock = 128;

// Blocks of kBlock threads that cover n units.
inline unsigned blocks(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

template <int N, int I = 0, class F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    sfor<N, I + 1>(f);
  }
}

// Loads of data that a kernel only reads.  COH = true: the data is written
// by other blocks of the same (persistent) launch, so the load goes to L2
// (ld.global.cg) instead of through the non-coherent read-only or L1 caches.
template <bool COH, typename T>
__device__ __forceinline__ T ldro(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
template <bool COH, typename T>
__device__ __forceinline__ T ldm(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// binary64 -> Real.  For binary32 the conversion is done with integer
// operations on the IEEE-754 fields (round to nearest, ties away from zero),
// which keeps it off the FP64 pipe; valid for |x| in [2^-126, 2^128), smaller
// magnitudes flush to a signed zero.  Used for the stored binary64 geometry and
// pseudo-inverses read by the mixed-precision kernels.
template <typename Real>
__device__ __forceinline__ Real cvt(double x);
template <>
__device__ __forceinline__ double cvt<double>(double x) {
  return x;
}
template <>
__device__ __forceinline__ float cvt<float>(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  const unsigned sign = hi & 0x80000000u;
  // (hi:lo) << 3 puts the low 9 exponent bits at [31:23] and the top 23
  // mantissa bits below them; subtracting 896 << 23 (mod 2^32) rebiases the
  // exponent, and the first dropped mantissa bit rounds
  const unsigned fm = __funnelshift_l(lo, hi, 3);
  const unsigned r = (((fm - (896u << 23)) & 0x7fffffffu) | sign) + ((lo >> 28) & 1u);
  return __uint_as_float(e < 897u ? sign : r);
}

// cvt<float> extended to the whole binary64 range: magnitudes of 2^128 and
// above become a signed infinity, NaNs a quiet NaN (for state values, which
// may be non-finite after a failed step).
__device__ __forceinline__ float cvt_state(double x) {
  const unsigned hi = (unsigned)((unsigned long long)__double_as_longlong(x) >> 32);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e < 1151u) return cvt<float>(x);
  const bool nan = e == 0x7ffu && ((hi & 0xfffffu) | (unsigned)__double_as_longlong(x)) != 0u;
  return __uint_as_float((hi & 0x80000000u) | 0x7f800000u | (nan ? 0x400000u : 0u));
}

// The binary32 state copy holds one 32-byte record per cell (5 variables and
// 3 zero pads), so one stencil gather fetches all five variables of a cell.
// The rounded values are also returned in qf.
__device__ __forceinline__ void store_qf(float* __restrict__ Qf, int64_t c, const double q[5], float qf[5]) {
#pragma unroll
  for (int v = 0; v < 5; ++v) qf[v] = cvt_state(q[v]);
  float4* r = reinterpret_cast<float4*>(Qf + 8 * c);
  r[0] = make_float4(qf[0], qf[1], qf[2], qf[3]);
  r[1] = make_float4(qf[4], 0.f, 0.f, 0.f);
}
__device__ __forceinline__ void store_qf(float* __restrict__ Qf, int64_t c, const double q[5]) {
  float qf[5];
  store_qf(Qf, c, q, qf);
}
// Variable v of cell c of a state: binary64 [5][nce] or binary32 [nce][8].
template <bool COH = false>
__device__ __forceinline__ double qget(const double* __restrict__ Q, int64_t nce, int v, int64_t c) {
  return ldm<COH>(Q + v * nce + c);
}
template <bool COH = false>
__device__ __forceinline__ float qget(const float* __restrict__ Q, int64_t, int v, int64_t c) {
  return ldm<COH>(Q + 8 * c + v);
}

// Records of the reconstruction coefficients and face fluxes (see DevWork).
template <typename Real>
__host__ __device__ constexpr int coef_rec() { return sizeof(Real) == 4 ? kCoefRec32 : kCoefRec64; }
template <typename Real>
__host__ __device__ constexpr int flux_rec() { return sizeof(Real) == 4 ? kFluxRec32 : kFluxRec64; }

// Ten consecutive reals at p (8-byte aligned for binary32, 16-byte for
// binary64), as five vector accesses.
template <bool COH = false>
__device__ __forceinline__ void load10(const float* __restrict__ p, float x[10]) {
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float2 t = ldro<COH>(reinterpret_cast<const float2*>(p) + i);
    x[2 * i] = t.x;
    x[2 * i + 1] = t.y;
  }
}
template <bool COH = false>
__device__ __forceinline__ void load10(const double* __restrict__ p, double x[10]) {
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const double2 t = ldro<COH>(reinterpret_cast<const double2*>(p) + i);
    x[2 * i] = t.x;
    x[2 * i + 1] = t.y;
  }
}
__device__ __forceinline__ void store10(double* __restrict__ p, const double x[10]) {
#pragma unroll
  for (int i = 0; i < 5; ++i) reinterpret_cast<double2*>(p)[i] = make_double2(x[2 * i], x[2 * i + 1]);
}

// binary32 -> binary64, exact.  Normal numbers and zeros are converted with
// integer operations on the IEEE-754 fields (off the FP64 pipe); subnormals,
// infinities and NaNs take the hardware conversion.
__device__ __forceinline__ double f2d(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xffu;
  if ((b << 1) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  if (e == 0u || e == 0xffu) return (double)x;
  const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)((b & 7u) << 29));
}

// A parameter in the kernel's precision: the binary64 value or its copy
// rounded to binary32 on the host.
template <typename Real>
__device__ __forceinline__ Real pick(double d, float f) {
  if constexpr (sizeof(Real) == 4) return f;
  else return d;
}

// --------------------------------------------------------------------------
// Maxwellian moments.  Mom holds normalised one-dimensional moments <u^k>,
// <v^k>, <w^k> and <(xi^2)^k> of one Maxwellian (u possibly on a half-line).
// --------------------------------------------------------------------------
template <typename R>
struct Mom {
  R u[7], v[6], w[6], x[3];
};

// Gaussian recursion <u^{n+2}> = U <u^{n+1}> + (n+1)/(2 lam) <u^n>
template <int N, typename R>
__device__ __forceinline__ void recur(R* m, R U, R h2) {
#pragma unroll
  for (int n = 0; n + 2 < N; ++n) m[n + 2] = U * m[n + 1] + R(n + 1) * h2 * m[n];
}

#ifndef HGKS_FAST_F32
#define HGKS_FAST_F32 1
#endif
// Division, exponential and logarithm of the flux.  In binary32 they are the
// hardware approximations (errors of a few units in the last place, far below
// the mixed path's error against binary64; 9% off the viscous binary32 flux);
// HGKS_FAST_F32 = 0 takes the correctly rounded forms.
template <typename R>
__device__ __forceinline__ R fdiv(R a, R b) {
  if constexpr (sizeof(R) == 4 && HGKS_FAST_F32) return __fdividef(a, b);
  else return a / b;
}
template <typename R>
__device__ __forceinline__ R fexp(R x) {
  if constexpr (sizeof(R) == 4 && HGKS_FAST_F32) return __expf(x);
  else return exp(x);
}
template <typename R>
__device__ __forceinline__ R flog(R x) {
  if constexpr (sizeof(R) == 4 && HGKS_FAST_F32) return __logf(x);
  else return log(x);
}

// erfcx(x) = exp(x^2) erfc(x) in binary64, for x >= 0 or NaN.  On [0, 6)
// it is the piecewise Chebyshev interpolant of erfcx_table.h (degree 12 on
// intervals of width 1/4, generated with mpmath; within 0.9 units in the
// last place of the exact function), evaluated by Horner's rule with fused
// multiply-adds; beyond, the library erfcx.  About a third of the library
// function's binary64 operations on the flux's usual range.
__device__ __forceinline__ double erfcx_tab(double x) {
  if (x < 6.0) {
    const int i = __double2int_rz(x * 4.0);  // 0 .. 23; x * 4 is exact
    const double u = fma(x, 8.0, -(double)(2 * i + 1));
    const double* c = kErfcxTab + i * (kErfcxDegree + 1);
    double p = __ldg(c + kErfcxDegree);
#pragma unroll
    for (int k = kErfcxDegree - 1; k >= 0; --k) p = fma(p, u, __ldg(c + k));
    return p;
  }
  return erfcx(x);
}

template <typename R>
struct Prim {
  R rho, U, V, W, lam, h2;  // h2 = 1/(2 lam)
};

// kq = (K+3)/4: rho E = rho |U|^2/2 + kq rho / lam, so lam = kq rho / eint and
// 1/(2 lam) = eint / (2 kq rho), with eint = rho E - |rho U|^2/(2 rho).  Both
// reciprocals, 1/rho and 1/eint, come from one division: with
// e2 = rho eint = rho (rho E) - |rho U|^2/2, d = 1/(rho e2) gives
// 1/rho = e2 d and 1/eint = rho^2 d.
template <typename R>
__device__ __forceinline__ Prim<R> prim_of(const R q[5], R kq, R kqi) {
  Prim<R> p;
  p.rho = q[0];
  const R e2 = q[0] * q[4] - R(0.5) * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const R d = fdiv(R(1), q[0] * e2);
  const R ri = e2 * d;
  p.U = q[1] * ri;
  p.V = q[2] * ri;
  p.W = q[3] * ri;
  const R eint = e2 * ri;
  p.lam = kq * q[0] * (q[0] * q[0] * d);
  p.h2 = R(0.5) * kqi * eint * ri;
  return p;
}

// Moments of a Maxwellian; half = +1: u > 0, -1: u < 0, 0: full line.
// Eh receives half * exp(-lam U^2)/(2 sqrt(pi lam)), the boundary term of the
// half-line recursion (0 on the full line).
template <int NU, typename R>
__device__ __forceinline__ void moments(const Prim<R>& p, int half, R Kint, Mom<R>& M, R& Eh) {
  if (half == 0) {
    M.u[0] = R(1);
    M.u[1] = p.U;
    Eh = R(0);
  } else {
    const R rs = rsqrt(p.lam);
    const R s = R(half) * p.lam * rs * p.U;  // sqrt(lam) U
    const R ex = fexp(-p.lam * p.U * p.U);    // exp(-s^2)
    const R e = ex * R(0.28209479177387814) * rs;  // exp(-lam U^2)/(2 sqrt(pi lam))
    if constexpr (sizeof(R) == 8) {
      // binary64: erfc(-s) from the scaled function erfcx(|s|) =
      // exp(s^2) erfc(|s|) and the exponential already at hand,
      // erfc(|s|) = ex erfcx(|s|) and erfc(-|s|) = 2 - erfc(|s|); measured
      // 3.5% faster than erfc on the FP64 flux with the library erfcx (in
      // binary32, erfc is faster), and erfcx_tab is cheaper still
      const R ec = ex * erfcx_tab(fabs(s));
      M.u[0] = R(0.5) * (s >= R(0) ? R(2) - ec : ec);
    } else {
      M.u[0] = R(0.5) * erfc(-s);
    }
    Eh = R(half) * e;
    M.u[1] = p.U * M.u[0] + Eh;
  }
  recur<NU>(M.u, p.U, p.h2);
  M.v[0] = R(1);
  M.v[1] = p.V;
  recur<6>(M.v, p.V, p.h2);
  M.w[0] = R(1);
  M.w[1] = p.W;
  recur<6>(M.w, p.W, p.h2);
  M.x[0] = R(1);
  M.x[1] = Kint * p.h2;                        // <xi^2> = K/(2 lam)
  M.x[2] = Kint * (Kint + R(2)) * p.h2 * p.h2;  // <xi^4> = K(K+2)/(4 lam^2)
}

// Euler state used for flux Jacobians in the local frame.
template <typename R>
struct EState {
  R rho, ri, u[3], m[3], E, p, gm1;
};
template <typename R>
__device__ __forceinline__ EState<R> estate(const R q[5], R gamma) {
  EState<R> s;
  s.rho = q[0];
  s.ri = fdiv(R(1), q[0]);
  for (int a = 0; a < 3; ++a) { s.m[a] = q[1 + a]; s.u[a] = q[1 + a] * s.ri; }
  s.E = q[4];
  s.gm1 = gamma - R(1);
  s.p = s.gm1 * (q[4] - R(0.5) * (s.m[0] * s.u[0] + s.m[1] * s.u[1] + s.m[2] * s.u[2]));
  return s;
}
// o = J_j(q) d: derivative of the Euler flux along axis j in direction d.
// For a Maxwellian g(Q), rho <u_j psi a(dQ)> equals J_j dQ exactly, which
// replaces the moment sums of the micro-slope terms.
template <int j, typename R>
__device__ __forceinline__ void euler_jv(const EState<R>& s, const R d[5], R o[5]) {
  const R duj = (d[1 + j] - s.u[j] * d[0]) * s.ri;
  const R dp = s.gm1 * (d[4] - (s.u[0] * d[1] + s.u[1] * d[2] + s.u[2] * d[3]) +
                        R(0.5) * (s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2]) * d[0]);
  o[0] = d[1 + j];
#pragma unroll
  for (int a = 0; a < 3; ++a) o[1 + a] = d[1 + a] * s.u[j] + s.m[a] * duj + (a == j ? dp : R(0));
  o[4] = (d[4] + dp) * s.u[j] + (s.E + s.p) * duj;
}

// Half-space contribution c = rho <psi>^sigma of one side to the interface
// equilibrium Q0 (Section 2.1), and its derivatives dc[j] along the local
// axes for the conservative-variable derivatives dq[j].
//
// By the definition of the micro-slope (g_x = a g), the term int psi a_j g
// over the half-line of Q0's slope equals d/dx_j of rho <psi>^sigma, and
// rho <psi>^sigma is a closed-form function of (rho, U, V, W, lam):
//   c = rho (u0, u1, u0 V, u0 W, (u2 + u0 S)/2),  S = V^2 + W^2 + (K+2)/(2 lam),
// with u_n the half-line moments of the normal velocity.  Their parameter
// derivatives follow from differentiating under the integral and the
// half-line recursion (E = half-line boundary term):
//   du0/dU = 2 lam E,  du0/dlam = U E,
//   du1/dU = u0,       du1/dlam = -E/(2 lam),
//   du2/dU = 2 u1,     du2/dlam = -u0/(2 lam^2).
// The chain rule through the primitive variables then gives dc without the
// half-space Gram matrix or the micro-slopes.  Quantities rho dU, rho dV,
// rho dW and rho dlam are formed directly from dq.
template <typename R>
__device__ __forceinline__ void half_jet(const Prim<R>& p, R u0, R u1, R Eh, R Kint, R kqi, const R dq[3][5],
                                         R c[5], R dc[3][5]) {
  const R h2 = p.h2;
  const R u2 = p.U * u1 + h2 * u0;
  const R S = p.V * p.V + p.W * p.W + (Kint + R(2)) * h2;
  c[0] = p.rho * u0;
  c[1] = p.rho * u1;
  c[2] = c[0] * p.V;
  c[3] = c[0] * p.W;
  c[4] = R(0.5) * p.rho * (u2 + u0 * S);
  const R tl = R(2) * p.lam, lk = p.lam * kqi, hU2 = R(0.5) * (p.U * p.U + p.V * p.V + p.W * p.W);
  const R hE = h2 * Eh, h22u0 = R(2) * h2 * h2 * u0, kS = R(2) * (Kint + R(2)) * h2 * h2;
  const R a2 = u2 + u0 * S;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const R* d = dq[j];
    const R PU = d[1] - p.U * d[0], PV = d[2] - p.V * d[0], PW = d[3] - p.W * d[0];
    const R de = d[4] - p.U * d[1] - p.V * d[2] - p.W * d[3] + hU2 * d[0];  // d(rho e_int)
    const R Pl = p.lam * (d[0] - lk * de);                                  // rho dlam
    const R rdu0 = Eh * (tl * PU + p.U * Pl);
    const R rdu1 = u0 * PU - hE * Pl;
    const R rdu2 = R(2) * u1 * PU - h22u0 * Pl;
    const R rdS = R(2) * (p.V * PV + p.W * PW) - kS * Pl;
    const R d0 = d[0] * u0 + rdu0;
    dc[j][0] = d0;
    dc[j][1] = d[0] * u1 + rdu1;
    dc[j][2] = p.V * d0 + u0 * PV;
    dc[j][3] = p.W * d0 + u0 * PW;
    dc[j][4] = R(0.5) * (d[0] * a2 + rdu2 + S * rdu0 + u0 * rdS);
  }
}

// Perturbation of the primitive variables, rho-weighted, for a perturbation
// d of the conservative variables under the Maxwellian p:
//   P = (d rho, rho dU, rho dV, rho dW, rho dlam).
template <typename R>
__device__ __forceinline__ void prim_pert(const Prim<R>& p, R kqi, const R d[5], R P[5]) {
  P[0] = d[0];
  P[1] = d[1] - p.U * d[0];
  P[2] = d[2] - p.V * d[0];
  P[3] = d[3] - p.W * d[0];
  const R de = d[4] - p.U * d[1] - p.V * d[2] - p.W * d[3] + R(0.5) * (p.U * p.U + p.V * p.V + p.W * p.W) * d[0];
  P[4] = p.lam * (d[0] - p.lam * kqi * de);
}

// Change of the normalised moment <u^n> (half line with boundary term Eh, or
// full line with Eh = 0) under rho dU = PU, rho dlam = Pl, divided by rho:
//   d<u^0> = Eh (2 lam dU + U dlam),  d<u^1> = <u^0> dU - Eh dlam/(2 lam),
//   d<u^n> = n <u^{n-1}> dU - n (n-1) <u^{n-2}> dlam/(4 lam^2),  n >= 2.
template <int n, typename R>
__device__ __forceinline__ R dmom_u(const Mom<R>& M, const Prim<R>& p, R Eh, R PU, R Pl, R h22) {
  if constexpr (n == 0) return Eh * (R(2) * p.lam * PU + p.U * Pl);
  else if constexpr (n == 1) return M.u[0] * PU - p.h2 * Eh * Pl;
  else return R(n) * M.u[n - 1] * PU - R(n * (n - 1)) * h22 * M.u[n - 2] * Pl;
}
// The same for a full-line Gaussian moment <v^n> (m = M.v or M.w, Pv = rho dV or rho dW).
template <int n, typename R>
__device__ __forceinline__ R dmom_g(const R* m, R Pv, R Pl, R h22) {
  if constexpr (n == 0) return R(0);
  else if constexpr (n == 1) return Pv;
  else return R(n) * m[n - 1] * Pv - R(n * (n - 1)) * h22 * m[n - 2] * Pl;
}

// Derivative of Phi = rho <u^a v^b w^c psi> (moments M of one Maxwellian,
// half-line boundary term Eh) along the perturbation P of prim_pert.
//
// With g_x = (a.psi) g (the micro-slope of Section 2.1), rho <phi (a.psi)>
// over the same velocity range is exactly this derivative; it replaces the
// moment sums of the micro-slope and time-slope terms of Eq. flux.
template <int a, int b, int c, typename R>
__device__ __forceinline__ void phi_jet(const Mom<R>& M, const Prim<R>& pm, R Eh, R Kint, const R P[5], R out[5]) {
  const R h22 = pm.h2 * pm.h2;
  // value and derivative of <u^i v^j w^k>
  auto prod = [&](auto I, auto J, auto Kk, R& val, R& der) {
    constexpr int i = decltype(I)::value, j = decltype(J)::value, k = decltype(Kk)::value;
    const R ui = M.u[i], vj = M.v[j], wk = M.w[k];
    const R dui = dmom_u<i>(M, pm, Eh, P[1], P[4], h22);
    const R dvj = dmom_g<j>(M.v, P[2], P[4], h22);
    const R dwk = dmom_g<k>(M.w, P[3], P[4], h22);
    val = ui * vj * wk;
    der = dui * vj * wk + ui * (dvj * wk + vj * dwk);
  };
  using std::integral_constant;
  R v0, d0, v1, d1, v2, d2, v3, d3, va, da, vb, db, vc, dc;
  prod(integral_constant<int, a>{}, integral_constant<int, b>{}, integral_constant<int, c>{}, v0, d0);
  prod(integral_constant<int, a + 1>{}, integral_constant<int, b>{}, integral_constant<int, c>{}, v1, d1);
  prod(integral_constant<int, a>{}, integral_constant<int, b + 1>{}, integral_constant<int, c>{}, v2, d2);
  prod(integral_constant<int, a>{}, integral_constant<int, b>{}, integral_constant<int, c + 1>{}, v3, d3);
  prod(integral_constant<int, a + 2>{}, integral_constant<int, b>{}, integral_constant<int, c>{}, va, da);
  prod(integral_constant<int, a>{}, integral_constant<int, b + 2>{}, integral_constant<int, c>{}, vb, db);
  prod(integral_constant<int, a>{}, integral_constant<int, b>{}, integral_constant<int, c + 2>{}, vc, dc);
  const R X1 = Kint * pm.h2, dX1 = R(-2) * Kint * h22 * P[4];  // <xi^2> = K/(2 lam)
  out[0] = P[0] * v0 + d0;
  out[1] = P[0] * v1 + d1;
  out[2] = P[0] * v2 + d2;
  out[3] = P[0] * v3 + d3;
  out[4] = R(0.5) * (P[0] * (va + vb + vc + v0 * X1) + da + db + dc + d0 * X1 + v0 * dX1);
}

// The value of Phi / rho = <u^a v^b w^c psi> itself (phi_jet along
// P = (1, 0, 0, 0, 0), without the derivative terms that vanish there).
template <int a, int b, int c, typename R>
__device__ __forceinline__ void phi_val(const Mom<R>& M, const Prim<R>& pm, R Kint, R out[5]) {
  const R v0 = M.u[a] * M.v[b] * M.w[c];
  out[0] = v0;
  out[1] = M.u[a + 1] * M.v[b] * M.w[c];
  out[2] = M.u[a] * M.v[b + 1] * M.w[c];
  out[3] = M.u[a] * M.v[b] * M.w[c + 1];
  const R va = M.u[a + 2] * M.v[b] * M.w[c], vb = M.u[a] * M.v[b + 2] * M.w[c], vc = M.u[a] * M.v[b] * M.w[c + 2];
  out[4] = R(0.5) * (va + vb + vc + v0 * (Kint * pm.h2));
}

// X = sum_j rho <u u_j psi a_j>, the spatial-slope term of the
// non-equilibrium part of Eq. flux for one side (Maxwellian p with moments M
// over its half line, slopes d[j] of the conservative variables along the
// local axes j = n, t1, t2).  On the full line (Eh = 0) it is the
// rho0 <u (abar.u) psi> term of the equilibrium part.
template <typename R>
__device__ __forceinline__ void side_terms(const Prim<R>& p, const Mom<R>& M, R Eh, R Kint, R kqi, const R d[3][5],
                                           R X[5]) {
  R P[5], t[5];
  prim_pert(p, kqi, d[0], P);
  phi_jet<2, 0, 0>(M, p, Eh, Kint, P, X);
  prim_pert(p, kqi, d[1], P);
  phi_jet<1, 1, 0>(M, p, Eh, Kint, P, t);
#pragma unroll
  for (int i = 0; i < 5; ++i) X[i] += t[i];
  prim_pert(p, kqi, d[2], P);
  phi_jet<1, 0, 1>(M, p, Eh, Kint, P, t);
#pragma unroll
  for (int i = 0; i < 5; ++i) X[i] += t[i];
}

template <typename R>
struct FluxParams {
  R gamma, Kint, kq, kqi, mu_ref, T_ref, visc_exp, prfix, tau_c;  // kq = (K+3)/4, kqi = 1/kq, prfix = 1/Pr - 1
};
template <typename R>
__device__ __forceinline__ FluxParams<R> flux_params(const DevParams& P) {
  FluxParams<R> F;
  F.gamma = pick<R>(P.gamma, P.f_gamma);
  F.Kint = pick<R>(P.Kint, P.f_Kint);
  F.kq = pick<R>(P.kq, P.f_kq);
  F.kqi = pick<R>(P.kqi, P.f_kqi);
  F.mu_ref = pick<R>(P.mu_ref, P.f_mu_ref);
  F.T_ref = pick<R>(P.T_ref, P.f_T_ref);
  F.visc_exp = pick<R>(P.visc_exp, P.f_visc_exp);
  F.prfix = pick<R>(P.prfix, P.f_prfix);
  F.tau_c = pick<R>(P.tau_c, P.f_tau_c);
  return F;
}

// Gas-kinetic flux in the local frame (normal = first axis), in two parts so
// that the two sides stream through one at a time:
//
//   side_flux   one side's state q and derivatives d[j] along the local axes
//               j = n, t1, t2: its half-space part of the interface
//               equilibrium Q0 and of the slopes dQ0/dn_j, added to q0 and
//               dq0, and (viscous) its non-equilibrium moment sums, added to
//               S: S[0] = sum_j rho <u u_j psi a_j> (spatial slopes),
//               S[1] = rho <u psi> (the initial distribution itself),
//               S[2] = rho <u A psi> (time slope, rho <A psi> = -sum_j J_j d_j)
//   eq_flux     the equilibrium part from Q0 and its slopes, the collision
//               time, and the time integrals that weight the side sums
//
// Both sides' non-equilibrium terms carry the same weights, so their sums
// are formed first and weighted once.  Output: F^n and dF/dt of Eq.
// expansion-1 (Section 2.2) for step dt (dt2i = 2/dt).
// FIRST: the side that starts the sums (they are assigned, not added to, so
// that no addition of zero is spent).
template <typename R, bool VISC, bool FIRST>
__device__ __forceinline__ void side_flux(const R q[5], const R d[3][5], int half, const FluxParams<R>& P,
                                          R q0[5], R dq0[3][5], R S[3][5], R& pside) {
  const R K = P.Kint;
  const Prim<R> p = prim_of(q, P.kq, P.kqi);
  constexpr int NU = VISC ? 5 : 3;
  Mom<R> M;
  R Eh;
  moments<NU>(p, half, K, M, Eh);
  {
    R c[5], dc[3][5];
    half_jet(p, M.u[0], M.u[1], Eh, K, P.kqi, d, c, dc);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      q0[i] = FIRST ? c[i] : q0[i] + c[i];
#pragma unroll
      for (int j = 0; j < 3; ++j) dq0[j][i] = FIRST ? dc[j][i] : dq0[j][i] + dc[j][i];
    }
  }
  if constexpr (VISC) {
    pside = p.rho * p.h2;
    R X[5];
    side_terms(p, M, Eh, K, P.kqi, d, X);
#pragma unroll
    for (int i = 0; i < 5; ++i) S[0][i] = FIRST ? X[i] : S[0][i] + X[i];
    R tmp[5], s1[5], s2[5], Pp[5], y[5];
    const EState<R> st = estate(q, P.gamma);
    euler_jv<0>(st, d[0], tmp);
    euler_jv<1>(st, d[1], s1);
    euler_jv<2>(st, d[2], s2);
#pragma unroll
    for (int i = 0; i < 5; ++i) tmp[i] = -(tmp[i] + s1[i] + s2[i]);
    prim_pert(p, P.kqi, tmp, Pp);
    phi_jet<1, 0, 0>(M, p, Eh, K, Pp, y);
#pragma unroll
    for (int i = 0; i < 5; ++i) S[2][i] = FIRST ? y[i] : S[2][i] + y[i];
    // rho <u psi>
    phi_val<1, 0, 0>(M, p, K, y);
#pragma unroll
    for (int i = 0; i < 5; ++i) S[1][i] = FIRST ? p.rho * y[i] : fma(p.rho, y[i], S[1][i]);
  }
}

template <typename R, bool VISC>
__device__ __forceinline__ void eq_flux(const R q0[5], const R dq0[3][5], const R S[3][5], R plp, R prp, R dt,
                                        R dt2i, const FluxParams<R>& P, R F[5], R dF[5]) {
  const R K = P.Kint;
  // Euler flux of Q0 and the time derivative of Q0 from the compatibility
  // condition <abar.u + Abar> = 0:  dQ0/dt = -sum_j J_j(Q0) dQ0/dn_j
  const EState<R> s0 = estate(q0, P.gamma);
  R t0[5], t1[5], t2[5], qt[5], Fe[5], Ye[5];
  euler_jv<0>(s0, dq0[0], t0);
  euler_jv<1>(s0, dq0[1], t1);
  euler_jv<2>(s0, dq0[2], t2);
#pragma unroll
  for (int i = 0; i < 5; ++i) qt[i] = -(t0[i] + t1[i] + t2[i]);
  euler_jv<0>(s0, qt, Ye);  // rho0 <u Abar psi>
  Fe[0] = s0.m[0];
  Fe[1] = s0.m[0] * s0.u[0] + s0.p;
  Fe[2] = s0.m[0] * s0.u[1];
  Fe[3] = s0.m[0] * s0.u[2];
  Fe[4] = (s0.E + s0.p) * s0.u[0];

  if constexpr (!VISC) {
    // tau = 0: f = g0 (1 + Abar t)  =>  F^n = rho0 <u psi>, dF/dt = rho0 <u Abar psi>
#pragma unroll
    for (int i = 0; i < 5; ++i) { F[i] = Fe[i]; dF[i] = Ye[i]; }
    return;
  } else {
    const Prim<R> p0 = prim_of(q0, P.kq, P.kqi);
    const R p0p = p0.rho * p0.h2;
    // collision time: tau = mu(T0)/p0 + C dt |p_l - p_r|/(p_l + p_r), T = p/rho
    R mu = P.mu_ref;
    // (T0/T_ref)^e as exp(e log(T0/T_ref)): a few units in the last place,
    // for about half the cost of pow
    if (P.visc_exp != R(0) && mu != R(0)) mu = P.mu_ref * fexp(P.visc_exp * flog(fdiv(p0.h2, P.T_ref)));  // T0 = 1/(2 lam0)
    const R sp = plp + prp;
    const R tau = fdiv(mu * sp + P.tau_c * dt * fabs(plp - prp) * p0p, p0p * sp);  // one division
    if (!(tau > R(0))) {
#pragma unroll
      for (int i = 0; i < 5; ++i) { F[i] = Fe[i]; dF[i] = Ye[i]; }
      return;
    }
    // time-integral coefficients of the fit F = (4 I(dt/2) - I(dt))/dt,
    // dF = 4 (I(dt) - 2 I(dt/2))/dt^2, with h = dt/2, r = tau/h and
    // em = 1 - exp(-h/tau)
    const R r = tau * dt2i;  // dt2i = 1/h
    const R em = -expm1(fdiv(R(-1), r));
    const R g = em * (R(2) + em);  // 3 - 4 e^{-h/tau} + e^{-2h/tau}
    const R C1 = R(1) - R(0.5) * r * g;
    const R C2 = tau * (r * g - (R(2) - em * em));
    const R C3 = tau * (R(0.5) * r * g - R(1));
    const R C4 = R(0.5) * r * g;
    const R C5 = tau * (r * g - (R(1) - em * em));
    const R D1 = r * em * em * dt2i;
    const R D2 = R(2) * r * em * (R(1) - em) - R(2) * r * r * em * em;
    const R D3 = R(1) - r * r * em * em;
    const R D4 = -D1;
    const R D5 = D2;
    // F = C1 Fe + C2 X0 + C3 Ye - C5 X + C4 N - tau C4 Y over both sides'
    // sums S = (X, N, Y), and dF with D1..D5
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      F[i] = C1 * Fe[i] + C3 * Ye[i];
      dF[i] = D1 * Fe[i] + D3 * Ye[i];
    }
    {
      // X0 = rho0 <u (abar.u) psi> on the full line of g0
      Mom<R> M0;
      R E0;
      moments<5>(p0, 0, K, M0, E0);
      R X0[5];
      side_terms(p0, M0, E0, K, P.kqi, dq0, X0);
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        F[i] += C2 * X0[i];
        dF[i] += D2 * X0[i];
      }
      // Prandtl-number fix of the energy flux: + (1/Pr - 1) q with q the heat
      // flux of the first-order equilibrium part, -tau rho0 <c_u c^2/2 (abar.u+Abar)>,
      // which by the compatibility condition reduces to -tau w.(X0 + Y0),
      // w = (|U0|^2/2, -U0, -V0, -W0, 1).
      if (P.prfix != R(0)) {
        const R qh = -tau * (R(0.5) * (p0.U * p0.U + p0.V * p0.V + p0.W * p0.W) * (X0[0] + Ye[0]) -
                             p0.U * (X0[1] + Ye[1]) - p0.V * (X0[2] + Ye[2]) - p0.W * (X0[3] + Ye[3]) +
                             (X0[4] + Ye[4]));
        F[4] += P.prfix * qh;
      }
    }
    const R tC4 = tau * C4, tD4 = tau * D4;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      F[i] += C4 * S[1][i] - C5 * S[0][i] - tC4 * S[2][i];
      dF[i] += D4 * S[1][i] - D5 * S[0][i] - tD4 * S[2][i];
    }
  }
}

// Orthonormal completion (t1, t2) of a unit normal n (Duff et al. 2017).
template <typename R>
__device__ __forceinline__ void frame(const R n[3], R t1[3], R t2[3]) {
  const R sg = n[2] >= R(0) ? R(1) : R(-1);
  const R a = R(-1) / (sg + n[2]);
  const R b = n[0] * n[1] * a;
  t1[0] = R(1) + sg * n[0] * n[0] * a;
  t1[1] = sg * b;
  t1[2] = -sg * n[0];
  t2[0] = b;
  t2[1] = sg + n[1] * n[1] * a;
  t2[2] = -n[1];
}

// --------------------------------------------------------------------------
// boundary states (Section 5.2), conservative variables
// --------------------------------------------------------------------------
// Riemann-invariant far field along the outward unit normal n (any frame).
template <typename R>
__device__ __forceinline__ void farfield(const R q[5], const R qinf[5], const R n[3], R gamma, R o[5]) {
  const R gm1 = gamma - R(1);
  const R ri = R(1) / q[0];
  const R ui[3] = {q[1] * ri, q[2] * ri, q[3] * ri};
  const R pi = gm1 * (q[4] - R(0.5) * q[0] * (ui[0] * ui[0] + ui[1] * ui[1] + ui[2] * ui[2]));
  const R re = qinf[0];
  const R ue[3] = {qinf[1] / re, qinf[2] / re, qinf[3] / re};
  const R pe = gm1 * (qinf[4] - R(0.5) * re * (ue[0] * ue[0] + ue[1] * ue[1] + ue[2] * ue[2]));
  const R ci = sqrt(gamma * pi * ri), ce = sqrt(gamma * pe / re);
  const R uni = ui[0] * n[0] + ui[1] * n[1] + ui[2] * n[2];
  const R une = ue[0] * n[0] + ue[1] * n[1] + ue[2] * n[2];
  if (uni >= ci) {
    for (int i = 0; i < 5; ++i) o[i] = q[i];
    return;
  }
  if (uni <= -ci) {
    for (int i = 0; i < 5; ++i) o[i] = qinf[i];
    return;
  }
  const R rp = uni + R(2) * ci / gm1;   // outgoing invariant from the interior
  const R rm = une - R(2) * ce / gm1;   // incoming invariant from the free stream
  const R un = R(0.5) * (rp + rm);
  const R c = R(0.25) * gm1 * (rp - rm);
  R ent, ut[3];
  if (un > R(0)) {
    ent = pi / pow(q[0], gamma);
    for (int a = 0; a < 3; ++a) ut[a] = ui[a] - uni * n[a];
  } else {
    ent = pe / pow(re, gamma);
    for (int a = 0; a < 3; ++a) ut[a] = ue[a] - une * n[a];
  }
  const R rho = pow(c * c / (gamma * ent), R(1) / gm1);
  const R p = rho * c * c / gamma;
  R u2 = R(0);
  for (int a = 0; a < 3; ++a) {
    const R ua = ut[a] + un * n[a];
    o[1 + a] = rho * ua;
    u2 += ua * ua;
  }
  o[0] = rho;
  o[4] = p / gm1 + R(0.5) * rho * u2;
}

// --------------------------------------------------------------------------
// kernels
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

// Control kernels run one thread per member mesh.
__global__ void k_control(Control* ctl, int n, double t_end, double dt_fixed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ctl[i].t_end = t_end;
  ctl[i].dt_fixed = dt_fixed;
}

// Reset member `only` (or every member when only < 0) to time t.
__global__ void k_reset(Control* ctl, int n, int only, double t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || (only >= 0 && i != only)) return;
  Control* c = ctl + i;
  c->t = t;
  c->dt = 0.0;
  c->steps = 0;
  c->flags = 0;
  c->dtmin_bits = dbits(__longlong_as_double(0x7ff0000000000000LL));
}

// The step size of member c: the CFL step (or dt_fixed), clipped to t_end.
template <bool COH = false>
__device__ __forceinline__ void finalize_one(Control* c, double cfl) {
  const double dt_fixed = ldm<COH>(&c->dt_fixed), t_end = ldm<COH>(&c->t_end), t = ldm<COH>(&c->t);
  double dt = dt_fixed > 0.0 ? dt_fixed : cfl * __longlong_as_double((long long)ldm<COH>(&c->dtmin_bits));
  if (t_end > 0.0) dt = fmin(dt, t_end - t);
  if (!(dt > 0.0) || !(dt < 1e300)) dt = 0.0;
  c->dt = dt;
  if (dt > 0.0) {
    c->t = t + dt;
    c->steps = ldm<COH>(&c->steps) + 1;
    c->dtmin_bits = dbits(__longlong_as_double(0x7ff0000000000000LL));
  }
}

__global__ void k_finalize(Control* ctl, int n, double cfl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  finalize_one(ctl + i, cfl);
}


// Local step bound of cell c (without the CFL factor).
__device__ __forceinline__ double cell_dt(const double q[5], double hdt, const DevParams& P) {
  const double ri = 1.0 / q[0];
  const double u = q[1] * ri, v = q[2] * ri, w = q[3] * ri;
  const double u2 = u * u + v * v + w * w;
  const double p = (P.gamma - 1.0) * (q[4] - 0.5 * q[0] * u2);
  const double a = sqrt(P.gamma * p * ri);
  double dt = hdt / (sqrt(u2) + a);
  if (P.mu_ref > 0.0) {
    double mu = P.mu_ref;
    if (P.visc_exp != 0.0) mu = P.mu_ref * pow(p * ri / P.T_ref, P.visc_exp);
    dt = fmin(dt, q[0] * hdt * hdt / (2.0 * mu));
  }
  return dt;
}

// The same bound in binary32 from the binary32 state copy (mixed precision).
__device__ __forceinline__ float cell_dt_f(const float q[5], float hdt, const DevParams& P) {
  const float ri = 1.f / q[0];
  const float u = q[1] * ri, v = q[2] * ri, w = q[3] * ri;
  const float u2 = u * u + v * v + w * w;
  const float p = (P.f_gamma - 1.f) * (q[4] - 0.5f * q[0] * u2);
  const float a = sqrtf(P.f_gamma * p * ri);
  float dt = hdt / (sqrtf(u2) + a);
  if (P.mu_ref > 0.0) {
    float mu = P.f_mu_ref;
    if (P.visc_exp != 0.0) mu = P.f_mu_ref * powf(p * ri / P.f_T_ref, P.f_visc_exp);
    dt = fminf(dt, q[0] * hdt * hdt / (2.f * mu));
  }
  return dt;
}

// Minimum over a block of NW warps into *dst (every thread calls it).
template <int NW = kBlock / 32>
__device__ __forceinline__ void block_min_to(unsigned long long* dst, double v) {
  __shared__ double red[NW];
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < NW ? red[threadIdx.x] : __longlong_as_double(0x7ff0000000000000LL);
    for (int o = 16; o > 0; o >>= 1) x = fmin(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (threadIdx.x == 0 && x >= 0.0) atomicMin(dst, dbits(x));
  }
}

// Minimum of v over the cells of each member mesh into ctl[member].dtmin_bits.
// Called by every thread of the block (mid = -1 for threads without a cell).
// One mesh: a block reduction; a batch: a warp reduction segmented by member
// (the minimum of positive doubles is the minimum of their bit patterns,
// reduced as the high word, then the low word among the lanes that hold it).
template <int NW = kBlock / 32>
__device__ __forceinline__ void member_min_to(const DevMesh& m, Control* ctl, int mid, double v) {
  if (m.nmesh == 1) {
    block_min_to<NW>(&ctl[0].dtmin_bits, v);
    return;
  }
  const unsigned long long b = dbits(v);
  const unsigned grp = __match_any_sync(0xffffffffu, mid);
  const unsigned hi = (unsigned)(b >> 32);
  const unsigned hmin = __reduce_min_sync(grp, hi);
  const unsigned cand = grp & __ballot_sync(0xffffffffu, hi == hmin);
  if (hi == hmin) {
    const unsigned lmin = __reduce_min_sync(cand, (unsigned)b);
    if ((int)(threadIdx.x & 31) == __ffs(cand) - 1 && mid >= 0 && hmin < 0x7ff00000u)
      atomicMin(&ctl[mid].dtmin_bits, ((unsigned long long)hmin << 32) | lmin);
  }
}

__device__ __forceinline__ int member_of(const DevMesh& m, int64_t c) { return m.cmesh ? m.cmesh[c] : 0; }

// Step bound of the state: binary64 from Q, or, in mixed precision (Qf
// non-null), binary32 from the binary32 copy, as k_update2 computes it.
__global__ void __launch_bounds__(kBlock) k_dt(DevMesh m, DevParams P, const double* __restrict__ Q,
                                               const float* __restrict__ Qf, Control* ctl) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  double v = __longlong_as_double(0x7ff0000000000000LL);
  int mid = -1;
  if (i < m.nc) {
    mid = member_of(m, i);
    if (Qf) {
      float q[5];
      for (int k = 0; k < 5; ++k) q[k] = Qf[8 * i + k];
      v = f2d(cell_dt_f(q, cvt<float>(m.hdt[i]), P));
    } else {
      double q[5];
      for (int k = 0; k < 5; ++k) q[k] = Q[k * m.nce + i];
      v = cell_dt(q, m.hdt[i], P);
    }
    if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000LL);
  }
  member_min_to(m, ctl, mid, v);
}

// Ghost cell averages: the boundary map of the mirrored interior cell.
template <bool COH = false>
__device__ __forceinline__ void ghost_one(const DevMesh& m, const DevParams& P, double* __restrict__ Q,
                                          float* __restrict__ Qf, const Control* __restrict__ ctl, int64_t g) {
  const int64_t s = m.gsrc[g];
  if (ldm<COH>(&ctl[member_of(m, s)].dt) == 0.0) return;
  double q[5], o[5];
  for (int k = 0; k < 5; ++k) q[k] = ldm<COH>(Q + k * m.nce + s);
  if (m.gtag[g] == 3) {  // wall: momentum reversed
    o[0] = q[0]; o[1] = -q[1]; o[2] = -q[2]; o[3] = -q[3]; o[4] = q[4];
  } else {
    const double n[3] = {m.gnrm[g], m.gnrm[m.ng + g], m.gnrm[2 * m.ng + g]};
    farfield(q, P.qinf, n, P.gamma, o);
  }
  for (int k = 0; k < 5; ++k) Q[k * m.nce + m.nc + g] = o[k];
  if (Qf) store_qf(Qf, m.nc + g, o);
}

__global__ void __launch_bounds__(kBlock) k_ghost(DevMesh m, DevParams P, double* __restrict__ Q, float* __restrict__ Qf,
                                                  const Control* __restrict__ ctl) {
  const int64_t g = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (g < m.ng) ghost_one(m, P, Q, Qf, ctl, g);
}

// Face flux record of face f: F (5) then dF/dt (5), binary32 records padded
// to 12 reals.
__device__ __forceinline__ void store_flux(float* __restrict__ Fs, int64_t f, const float x[10]) {
  float4* r = reinterpret_cast<float4*>(Fs + f * kFluxRec32);
  r[0] = make_float4(x[0], x[1], x[2], x[3]);
  r[1] = make_float4(x[4], x[5], x[6], x[7]);
  r[2] = make_float4(x[8], x[9], 0.f, 0.f);
}
__device__ __forceinline__ void store_flux(double* __restrict__ Fs, int64_t f, const double x[10]) {
  store10(Fs + f * kFluxRec64, x);
}
template <bool COH = false>
__device__ __forceinline__ void load_flux(const float* __restrict__ Fs, int64_t f, float x[10]) {
  const float4* r = reinterpret_cast<const float4*>(Fs + f * kFluxRec32);
  const float4 a = ldro<COH>(r), b = ldro<COH>(r + 1), c = ldro<COH>(r + 2);
  x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
  x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
  x[8] = c.x; x[9] = c.y;
}
template <bool COH = false>
__device__ __forceinline__ void load_flux(const double* __restrict__ Fs, int64_t f, double x[10]) {
  load10<COH>(Fs + f * kFluxRec64, x);
}

}  // namespace
}  // namespace hgks

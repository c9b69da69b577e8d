// hgks_kernels.cu -- sm_103a kernels of one HGKS step (Algorithm 2):
//
//   k_finalize    time step from the device-side minimum bound (Algorithm 2,
//                 "calculate time step"), clipped to t_end
//   k_ghost       boundary ghost cell averages (Algorithm 1 ghost cells)
//   k_recon       third-order WENO reconstruction (Section 2.3, Eqs. polys,
//                 weno), emitting one combined quadratic per cell and variable
//                 (k_recon_rs: the binary32 form, staged through registers)
//   k_flux        time-dependent gas-kinetic flux at the face Gauss points
//                 (Section 2.1, Eq. flux; Section 2.2 linear-in-time fit), one
//                 thread per face (k_flux_gp: one per Gauss point)
//   k_update1/2   gather of the face fluxes per cell (no atomics) and the two
//                 S2O4 stages (Section 2.2); stage 2 also produces the next
//                 step bound and the non-finite flag
//   k_persist     n whole steps in one cooperative launch, the phases above
//                 separated by bounded grid-wide barriers
//
// Precision: Real = double (FP64) or float (FP32-mixed: reconstruction and
// flux in binary32; geometry, pseudo-inverses and S2O4 sums in binary64).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <type_traits>

#include "hgks_internal.h"

namespace hgks {
namespace {

constexpr int kBlock = 128;

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
  const R d = R(1) / (q[0] * e2);
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
    const R ex = exp(-p.lam * p.U * p.U);    // exp(-s^2)
    const R e = ex * R(0.28209479177387814) * rs;  // exp(-lam U^2)/(2 sqrt(pi lam))
    if constexpr (sizeof(R) == 8) {
      // binary64: erfc(-s) from the scaled function erfcx(|s|) =
      // exp(s^2) erfc(|s|) and the exponential already at hand,
      // erfc(|s|) = ex erfcx(|s|) and erfc(-|s|) = 2 - erfc(|s|); measured
      // 3.5% faster than erfc on the FP64 flux (in binary32, erfc is faster)
      const R ec = ex * erfcx(fabs(s));
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
  s.ri = R(1) / q[0];
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

// Gas-kinetic flux in the local frame (normal = first axis).
//   ql, qr: conservative states on the two sides of the Gauss point
//   dl[j], dr[j]: their derivatives along the local axes j = n, t1, t2
// Output: F^n and dF/dt of Eq. expansion-1 (Section 2.2) for step dt
// (dt2i = 2/dt).
template <typename R, bool VISC>
__device__ void gks_flux(const R ql[5], const R dl[3][5], const R qr[5], const R dr[3][5], R dt, R dt2i,
                         const FluxParams<R>& P, R F[5], R dF[5]) {
  const R K = P.Kint;
  const Prim<R> pl = prim_of(ql, P.kq, P.kqi), pr = prim_of(qr, P.kq, P.kqi);
  constexpr int NU = VISC ? 5 : 3;
  Mom<R> Ml, Mr;
  R El, Er;
  moments<NU>(pl, +1, K, Ml, El);
  moments<NU>(pr, -1, K, Mr, Er);

  // interface equilibrium Q0 = rho_l <psi>^+_l + rho_r <psi>^-_r and its
  // slopes dQ0/dn_j = int_{u>0} psi a^l_j g_l + int_{u<0} psi a^r_j g_r
  R q0[5], dq0[3][5];
  {
    R cl[5], dcl[3][5], cr[5], dcr[3][5];
    half_jet(pl, Ml.u[0], Ml.u[1], El, K, P.kqi, dl, cl, dcl);
    half_jet(pr, Mr.u[0], Mr.u[1], Er, K, P.kqi, dr, cr, dcr);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      q0[i] = cl[i] + cr[i];
#pragma unroll
      for (int j = 0; j < 3; ++j) dq0[j][i] = dcl[j][i] + dcr[j][i];
    }
  }
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
    const R plp = pl.rho * pl.h2, prp = pr.rho * pr.h2, p0p = p0.rho * p0.h2;
    // collision time: tau = mu(T0)/p0 + C dt |p_l - p_r|/(p_l + p_r), T = p/rho
    R mu = P.mu_ref;
    // (T0/T_ref)^e as exp(e log(T0/T_ref)): a few units in the last place,
    // for about half the cost of pow
    if (P.visc_exp != R(0) && mu != R(0)) mu = P.mu_ref * exp(P.visc_exp * log(p0.h2 / P.T_ref));  // T0 = 1/(2 lam0)
    const R sp = plp + prp;
    const R tau = (mu * sp + P.tau_c * dt * fabs(plp - prp) * p0p) / (p0p * sp);  // one division
    if (!(tau > R(0))) {
#pragma unroll
      for (int i = 0; i < 5; ++i) { F[i] = Fe[i]; dF[i] = Ye[i]; }
      return;
    }
    // time-integral coefficients of the fit F = (4 I(dt/2) - I(dt))/dt,
    // dF = 4 (I(dt) - 2 I(dt/2))/dt^2, with h = dt/2, r = tau/h and
    // em = 1 - exp(-h/tau)
    const R r = tau * dt2i;  // dt2i = 1/h
    const R em = -expm1(R(-1) / r);
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
    // F = C1 Fe + C2 X0 + C3 Ye + C4 Nk - C5 (Xl + Xr) - tau C4 Yk, and dF
    // with D1..D5, accumulated term by term as each term is formed (this
    // keeps few of them live at once)
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
    // the initial non-equilibrium distribution of each side: spatial slopes
    // X, time slope Y = rho <u A psi> with rho <A psi> = -sum_j J_j(q) d_j,
    // and N = rho <u psi>
    auto side = [&](const R q[5], const R d[3][5], const Prim<R>& p, const Mom<R>& M, R Eh) {
      R X[5];
      side_terms(p, M, Eh, K, P.kqi, d, X);
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        F[i] -= C5 * X[i];
        dF[i] -= D5 * X[i];
      }
      R tmp[5], s1[5], s2[5], Pp[5], y[5], nn[5];
      const EState<R> st = estate(q, P.gamma);
      euler_jv<0>(st, d[0], tmp);
      euler_jv<1>(st, d[1], s1);
      euler_jv<2>(st, d[2], s2);
#pragma unroll
      for (int i = 0; i < 5; ++i) tmp[i] = -(tmp[i] + s1[i] + s2[i]);
      prim_pert(p, P.kqi, tmp, Pp);
      phi_jet<1, 0, 0>(M, p, Eh, K, Pp, y);
      // rho <u psi>: the derivative along P = (1, 0, 0, 0, 0) is the value
      const R e0[5] = {R(1), R(0), R(0), R(0), R(0)};
      phi_jet<1, 0, 0>(M, p, Eh, K, e0, nn);
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        F[i] += C4 * (p.rho * nn[i]) - tau * C4 * y[i];
        dF[i] += D4 * (p.rho * nn[i]) - tau * D4 * y[i];
      }
    };
    side(ql, dl, pl, Ml, El);
    side(qr, dr, pr, Mr, Er);
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

// The combined polynomial of a cell and variable is
// P(x) = q + g.d + sum k_ab d_a d_b, d = x - centroid, stored as 10 reals
// j = 0: q, 1-3: g, 4-9: k_xx k_yy k_zz k_xy k_yz k_zx at
// coef[c * record + v * 10 + j].
// Smoothness indicators, WENO-Z weights and the combined polynomial of one
// variable (Section 2.3, Eq. weno), returned in out[j], j = 0..9.
template <typename Real, int M>
__device__ __forceinline__ void recon_finish(const Real a[9], const Real b[M][3], Real qv, const Real mi[6], Real hi,
                                             Real glin, Real g0, Real eps, Real out[10]) {
  // smoothness indicators (scaled coordinates; the |cell| powers cancel):
  // beta_0 = sum_a (a_a^2 + H_a.Mi.H_a) + sum_{|l|=2} (d^l P0)^2, beta_m = |b_m|^2
  const Real H[3][3] = {{Real(2) * a[3], a[6], a[8]}, {a[6], Real(2) * a[4], a[7]}, {a[8], a[7], Real(2) * a[5]}};
  Real beta0 = Real(0);
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const Real h0 = H[x][0], h1 = H[x][1], h2 = H[x][2];
    const Real quad = h0 * (mi[0] * h0 + mi[3] * h1 + mi[5] * h2) + h1 * (mi[3] * h0 + mi[1] * h1 + mi[4] * h2) +
                      h2 * (mi[5] * h0 + mi[4] * h1 + mi[2] * h2);
    beta0 += a[x] * a[x] + quad;
  }
  beta0 += H[0][0] * H[0][0] + H[1][1] * H[1][1] + H[2][2] * H[2][2] + a[6] * a[6] + a[7] * a[7] + a[8] * a[8];
  Real beta[M];
  Real tz = Real(0);
#pragma unroll
  for (int s = 0; s < M; ++s) {
    beta[s] = b[s][0] * b[s][0] + b[s][1] * b[s][1] + b[s][2] * b[s][2];
    tz += fabs(beta0 - beta[s]);
  }
  tz *= Real(1) / Real(M);
  // WENO-Z type weights w_s = gamma_s (1 + tz / (beta_s + eps))
  Real r[M + 1];  // r_s = tz / (beta_s + eps), s = 0: the big stencil
  if constexpr (sizeof(Real) == 8) {
    // binary64: the M + 1 reciprocals from one division, 1/x_i =
    // (prod_{j<i} x_j)(prod_{j>i} x_j) / prod_j x_j (the binary64 pipe is the
    // bound of this kernel; a division costs about ten of its operations)
    Real x[M + 1], pre[M + 1];
    x[0] = beta0 + eps;
#pragma unroll
    for (int s = 0; s < M; ++s) x[s + 1] = beta[s] + eps;
    pre[0] = Real(1);
#pragma unroll
    for (int i = 1; i <= M; ++i) pre[i] = pre[i - 1] * x[i - 1];
    const Real tinv = tz / (pre[M] * x[M]);
    Real suf = Real(1);
#pragma unroll
    for (int i = M; i >= 0; --i) {
      r[i] = pre[i] * suf * tinv;
      suf *= x[i];
    }
  } else {
    r[0] = tz / (beta0 + eps);
#pragma unroll
    for (int s = 0; s < M; ++s) r[s + 1] = tz / (beta[s] + eps);
  }
  const Real w0 = g0 * (Real(1) + r[0]);
  Real w[M];
  Real wsum = w0;
#pragma unroll
  for (int s = 0; s < M; ++s) {
    w[s] = glin * (Real(1) + r[s + 1]);
    wsum += w[s];
  }
  const Real winv = Real(1) / wsum;
  const Real c0 = (Real(1) + r[0]) * winv;  // wbar_0 / gamma_0
  Real lin[3] = {c0 * a[0], c0 * a[1], c0 * a[2]};
#pragma unroll
  for (int s = 0; s < M; ++s) {
    const Real cm = w[s] * winv - c0 * glin;  // wbar_m - wbar_0 gamma_m / gamma_0
#pragma unroll
    for (int d = 0; d < 3; ++d) lin[d] += cm * b[s][d];
  }
  Real quad[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) quad[q] = c0 * a[3 + q];
  // to physical units about the centroid; the zero-mean basis shifts the constant
  Real q0 = qv;
#pragma unroll
  for (int q = 0; q < 6; ++q) q0 -= quad[q] * mi[q];
  out[0] = q0;
#pragma unroll
  for (int d = 0; d < 3; ++d) out[1 + d] = lin[d] * hi;
  const Real hi2 = hi * hi;
#pragma unroll
  for (int q = 0; q < 6; ++q) out[4 + q] = quad[q] * hi2;
}

// --------------------------------------------------------------------------
// Bulk asynchronous copies (TMA engine) into shared memory, completed on an
// mbarrier.  Addresses and sizes are multiples of 16 bytes by construction
// (rows of 32 cells with a 32-cell row pitch).
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of bar with the given parity to complete: false
// after about 2^31 clock cycles (~1 s).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > (1LL << 31)) return false;
  return true;
}

constexpr int kRC = 32;
constexpr int kRThreads = 5 * kRC;

// Coefficient records of the block's cells (consecutive, so their records
// are one contiguous run of memory): each (variable, cell) thread puts its
// 10 reals into shared memory (pitch record + 1, which spreads a warp's
// stores over the banks), then the block writes the run with coalesced
// stores.  smem must hold kRC x (record + 1) reals and no longer be read by
// any warp's arithmetic; every thread of the block calls this.
template <typename Real>
__device__ __forceinline__ void write_block_records(Real* smem, const Real res[10], bool live, int lane, int v,
                                                    int nv, Real* __restrict__ coef, int64_t c0) {
  constexpr int REC = coef_rec<Real>(), PITCH = REC + 1;
  __syncthreads();
  if (live) {
#pragma unroll
    for (int j = 0; j < 10; ++j) smem[lane * PITCH + v * 10 + j] = res[j];
    if (v == 0)
      for (int j = 50; j < REC; ++j) smem[lane * PITCH + j] = Real(0);
  }
  __syncthreads();
  Real* dst = coef + c0 * REC;
  // element e = l REC + r of the run; (l, r) advance by a constant step
  constexpr int DL = kRThreads / REC, DR = kRThreads % REC;
  int l = threadIdx.x / REC, r = threadIdx.x - (threadIdx.x / REC) * REC;
  for (int e = threadIdx.x; e < nv * REC; e += kRThreads) {
    dst[e] = smem[l * PITCH + r];
    l += DL;
    r += DR;
    if (r >= REC) {
      r -= REC;
      ++l;
    }
  }
}

// WENO reconstruction, one block per kRC = 32 consecutive cells with one warp
// per conservative variable (5 warps).  Warp 0 stages the block's rows of the
// pseudo-inverses (9K quadratic rows, then 3*KM rows per sub-stencil; 32
// cells of a row are 256 contiguous bytes) and the sub-stencil positions in
// shared memory with bulk asynchronous copies, while every warp gathers its
// variable's stencil differences; the rows are then reduced against them.
// Output: the coefficient record of each cell (see recon_finish).

template <typename Real, int K, int M, int KM>
struct ReconSmem {
  static constexpr int kRows = 9 * K + M * 3 * KM;
  static constexpr size_t tile = sizeof(double) * kRows * kRC;   // staged rows (binary64)
  static constexpr size_t sub = (size_t)M * KM * kRC;            // staged positions
  static constexpr size_t dq = sizeof(Real) * 5 * K * kRC;       // stencil differences
  static constexpr size_t bytes = tile + sub + dq;
};

template <typename Real, typename QT, int K, int M, int KM, bool STAGE, bool COH = false>
__device__ __forceinline__ void recon_block(const DevMesh& m, const DevParams& P, const QT* __restrict__ Q,
                                            Real* __restrict__ coef, Control* __restrict__ ctl, int64_t c0,
                                            unsigned char* smem_raw) {
  using S = ReconSmem<Real, K, M, KM>;
  constexpr int kRows = S::kRows;
  // staged variant: [tile | ssub | sdq]; direct variant: [sdq] only
  double* tile = reinterpret_cast<double*>(smem_raw);                // [kRows][kRC]
  uint8_t* ssub = smem_raw + S::tile;                                // [M*KM][kRC]
  Real* sdq = reinterpret_cast<Real*>(STAGE ? smem_raw + S::tile + S::sub : smem_raw);  // [5][K][kRC]
  __shared__ __align__(8) uint64_t bar;
  const int64_t nc = m.nc, ncp = m.ncp;
  const int lane = threadIdx.x & 31, v = threadIdx.x >> 5;
  const int64_t c = c0 + lane;
  const bool valid = c < nc;
  if constexpr (STAGE) {
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (v == 0) {
      if (lane == 0) mbar_expect_tx(&bar, (uint32_t)(S::tile + S::sub));
      __syncwarp();
      for (int r = lane; r < kRows; r += 32) {
        const double* src = r < 9 * K ? m.pinv0 + (int64_t)r * ncp + c0 : m.pinvm + (int64_t)(r - 9 * K) * ncp + c0;
        bulk_g2s(tile + r * kRC, src, kRC * sizeof(double), &bar);
      }
      for (int r = lane; r < M * KM; r += 32) bulk_g2s(ssub + r * kRC, m.subidx + (int64_t)r * ncp + c0, kRC, &bar);
    }
  }
  // this warp's variable: stencil differences (overlaps the staging)
  Real qv = Real(0);
  if (valid) {
    qv = (Real)qget<COH>(Q, m.nce, v, c);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t j = m.sten[(int64_t)k * nc + c];
      sdq[(v * K + k) * kRC + lane] = (Real)qget<COH>(Q, m.nce, v, j) - qv;
    }
  }
  if constexpr (STAGE) {
    const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, 0));
    if (!ok) {
      // The block's copies (its own inverse rows, under 100 KB) have not landed
      // within about a second, which only a stalled memory system explains.
      // Flag it, give the copies one more bounded wait, and leave: the block
      // may then exit with copies outstanding, which it accepts rather than
      // hang the device; the host reports HGKS_ETIMEOUT.
      if (threadIdx.x == 0) atomicOr(&ctl->flags, FLAG_TIMEOUT);
      mbar_wait_bounded(&bar, 0);
      return;
    }
    if constexpr (sizeof(Real) == 4) {
      // binary32: convert the staged rows in place (low word of each slot), once
      float* tf = reinterpret_cast<float*>(tile);
      for (int e = threadIdx.x; e < kRows * kRC; e += kRThreads) tf[2 * e] = cvt<float>(tile[e]);
      __syncthreads();
    }
  } else {
    __syncwarp();
  }
  Real res[10];
  if (valid) {
  auto row = [&](int r) -> Real {
    if constexpr (!STAGE)
      return cvt<Real>(r < 9 * K ? m.pinv0[(int64_t)r * ncp + c] : m.pinvm[(int64_t)(r - 9 * K) * ncp + c]);
    else if constexpr (sizeof(Real) == 4)
      return reinterpret_cast<const float*>(tile)[2 * (r * kRC + lane)];
    else
      return tile[r * kRC + lane];
  };
  auto subpos = [&](int r) -> int {
    if constexpr (STAGE) return ssub[r * kRC + lane];
    else return m.subidx[(int64_t)r * ncp + c];
  };
  Real dq[K];
#pragma unroll
  for (int k = 0; k < K; ++k) dq[k] = sdq[(v * K + k) * kRC + lane];
  // least-squares polynomials (the same operation order in both variants)
  Real a[9];
#pragma unroll
  for (int d = 0; d < 9; ++d) {
    Real sacc = Real(0);
#pragma unroll
    for (int k = 0; k < K; ++k) sacc += row(d * K + k) * dq[k];
    a[d] = sacc;
  }
  Real b[M][3];
#pragma unroll
  for (int s = 0; s < M; ++s) {
    Real x[KM];
#pragma unroll
    for (int r = 0; r < KM; ++r) x[r] = sdq[(v * K + subpos(s * KM + r)) * kRC + lane];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      Real acc = Real(0);
#pragma unroll
      for (int r = 0; r < KM; ++r) acc += row(9 * K + (s * 3 + d) * KM + r) * x[r];
      b[s][d] = acc;
    }
  }
  Real mi[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) mi[q] = cvt<Real>(m.mom[q * nc + c]);
  const Real hi = cvt<Real>(m.hinv[c]);
  const Real glin = pick<Real>(P.glin, P.f_glin), g0 = Real(1) - Real(M) * glin, eps = pick<Real>(P.eps, P.f_eps);
  recon_finish<Real, M>(a, b, qv, mi, hi, glin, g0, eps, res);
  }
  const int nv = nc - c0 < kRC ? (int)(nc - c0) : kRC;
  write_block_records<Real>(reinterpret_cast<Real*>(smem_raw), res, valid, lane, v, nv, coef, c0);
}

template <typename Real, typename QT, int K, int M, int KM, bool STAGE>
__global__ void __launch_bounds__(kRThreads) k_recon(DevMesh m, DevParams P, const QT* __restrict__ Q,
                                                     Real* __restrict__ coef, Control* __restrict__ ctl) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (m.nmesh == 1 && ctl->dt == 0.0) return;  // uniform over the grid (a batch computes every member)
  recon_block<Real, QT, K, M, KM, STAGE>(m, P, Q, coef, ctl, (int64_t)blockIdx.x * kRC, smem_raw);
}

// WENO reconstruction in binary32 (mixed precision), one block per kRC = 32
// cells with one warp per conservative variable, as k_recon, but with every
// input of the block staged in shared memory by all 160 threads before any
// arithmetic:
//   - the stencil neighbours' states, one 32-byte record (all five
//     variables) per neighbour;
//   - the block's rows of the binary64 pseudo-inverses, rounded to binary32
//     on the way in (cvt<float>, the rounding k_recon applies), so the tile
//     takes half the shared memory of a binary64 tile and more blocks fit on
//     an SM;
//   - the sub-stencil positions, the cells' own states, second moments and
//     1/h.
// The copy loops issue their loads back to back (coalesced rows of 32 cells
// for the per-cell arrays), so each thread keeps many loads in flight.  The
// arithmetic and its order are those of k_recon.
// Two ways to take less shared memory, used where they let more blocks share
// an SM (the choice is made at compile time from the sizes):
//   - "phased": the tile holds the quadratic rows (9K) first; once every
//     warp has formed its quadratic coefficients, the linear sub-stencil rows
//     replace them, so the tile needs max(9K, 3 M KM) rows, not the sum;
//   - "lean": the own-state and geometry rows are left out, and each thread
//     loads its cell's state, second moments and 1/h into registers.
// The block count is capped by the registers a thread needs (about 56 on
// tetrahedra, 66 on hexahedra, 86 at stencil size 26, measured with ptxas),
// and the kernel's launch bounds ask the compiler for that count.
template <int K, int M, int KM>
struct ReconSmemF {
  static constexpr int R0 = 9 * K, R1 = M * 3 * KM;  // quadratic and linear rows
  static constexpr size_t nbr = sizeof(float) * 5 * K * kRC;  // neighbour states [5][K][kRC]
  static constexpr size_t own = sizeof(float) * 5 * kRC;      // own states [5][kRC]
  static constexpr size_t geo = sizeof(float) * 7 * kRC;      // mom (6) and 1/h [7][kRC]
  static constexpr size_t sub = (size_t)M * KM * kRC;         // sub-stencil positions
  static constexpr size_t rows_f = sizeof(float) * (R0 + R1) * kRC, rows_p = sizeof(float) * (R0 > R1 ? R0 : R1) * kRC;
  // blocks per SM: 228 KB of shared memory, 1 KB reserved per block; registers
  static constexpr int fit(size_t b) { return (int)(233472 / (b + 1024)); }
  static constexpr int reg_cap = 65536 / (kRThreads * (M == 4 ? 56 : (K <= 24 ? 66 : 86)));
  static constexpr int cap(int b) { return b < reg_cap ? b : reg_cap; }
  static constexpr int b_full = cap(fit(rows_f + nbr + own + geo + sub)), b_lean = cap(fit(rows_f + nbr + sub)),
                       b_ph = cap(fit(rows_p + nbr + own + geo + sub)), b_phl = cap(fit(rows_p + nbr + sub));
  static constexpr int best = b_full > b_lean ? (b_full > b_ph ? (b_full > b_phl ? b_full : b_phl)
                                                               : (b_ph > b_phl ? b_ph : b_phl))
                                              : (b_lean > b_ph ? (b_lean > b_phl ? b_lean : b_phl)
                                                               : (b_ph > b_phl ? b_ph : b_phl));
  // the simplest layout that reaches the best count
  static constexpr bool phased = b_full < best && b_lean < best;
  static constexpr bool lean = phased ? b_ph < best : b_full < best;
  static constexpr size_t tile = phased ? rows_p : rows_f;  // binary32 rows
  static constexpr size_t bytes = tile + nbr + (lean ? 0 : own + geo) + sub;
  static constexpr int blocks = best;
};

template <int K, int M, int KM, bool COH = false>
__device__ __forceinline__ void recon_rs_block(const DevMesh& m, const DevParams& P, const float* __restrict__ Qf,
                                               float* __restrict__ coef, int64_t c0, unsigned char* smem_raw) {
  using S = ReconSmemF<K, M, KM>;
  float* tile = reinterpret_cast<float*>(smem_raw);                              // [kRows][kRC]
  float* snbr = reinterpret_cast<float*>(smem_raw + S::tile);                    // [5][K][kRC]
  float* sown = reinterpret_cast<float*>(smem_raw + S::tile + S::nbr);           // [5][kRC] (not lean)
  float* sgeo = reinterpret_cast<float*>(smem_raw + S::tile + S::nbr + S::own);  // [7][kRC] (not lean)
  uint8_t* ssub = smem_raw + S::tile + S::nbr + (S::lean ? 0 : S::own + S::geo);  // [M*KM][kRC]
  const int64_t nc = m.nc, ncp = m.ncp;
  const int t = threadIdx.x;
  const int nv = nc - c0 < kRC ? (int)(nc - c0) : kRC;  // cells of this block
  // With 5 warps of 32 lanes, thread (v, lane) stages column `lane` of the
  // rows v, v + 5, v + 10, ... of every per-cell array, so its addresses
  // advance by a fixed stride.
  const int lane = t & 31, v = t >> 5;
  const bool live = lane < nv;
  // 1. stencil indices of this thread's neighbour entries (entry K: the cell
  // itself, staged unless lean)
  constexpr int KE = S::lean ? K : K + 1;
  constexpr int NE = (KE + 4) / 5;
  int32_t jn[NE];
#pragma unroll
  for (int i = 0; i < NE; ++i) {
    const int k = v + 5 * i;
    jn[i] = (k < K && live) ? __ldcs(m.sten + (int64_t)k * nc + c0 + lane) : (int32_t)(c0 + lane);
  }
  // 2. first batch of pseudo-inverse rows (binary64, read once: streaming
  // loads).  Thread (v, lane) copies rows v + 5 j: J0 rows of pinv0 for
  // every v, then one more row for v < T0 (likewise J1, T1 for pinvm); the
  // row counts are compile-time constants, so only the tail row is guarded.
  constexpr int R0 = 9 * K, R1 = M * 3 * KM;  // rows of pinv0 and pinvm
  constexpr int J0 = R0 / 5, T0 = R0 - 5 * J0, J1 = R1 / 5, T1 = R1 - 5 * J1;
  constexpr int B = 8;
  static_assert(J0 >= B, "the first batch is a full one");
  constexpr int RS = 5 * kRC;  // shared-memory stride between a thread's rows
  const int64_t step = 5 * ncp;
  const double* p0 = m.pinv0 + (int64_t)v * ncp + c0 + lane;
  float* d0 = tile + v * kRC + lane;
  double pv[B];
#pragma unroll
  for (int i = 0; i < B; ++i) pv[i] = __ldcs(p0 + i * step);
  // 3. neighbour and own state records (32 bytes each)
  float4 qa[NE];
  float qb[NE];
  float qown = 0.f, gl[7];
  if constexpr (S::lean) {
    if (live) {
      qown = ldro<COH>(Qf + 8 * (c0 + lane) + v);
#pragma unroll
      for (int r = 0; r < 7; ++r) gl[r] = cvt<float>(r < 6 ? m.mom[(int64_t)r * nc + c0 + lane] : m.hinv[c0 + lane]);
    }
  }
#pragma unroll
  for (int i = 0; i < NE; ++i) {
    if (v + 5 * i < KE && live) {
      qa[i] = ldro<COH>(reinterpret_cast<const float4*>(Qf + 8 * (int64_t)jn[i]));
      qb[i] = ldro<COH>(Qf + 8 * (int64_t)jn[i] + 4);
    }
  }
  // 4. the first batch to binary32, then the remaining rows in batches
#pragma unroll
  for (int i = 0; i < B; ++i) d0[i * RS] = cvt<float>(pv[i]);
  {
    const double* q = p0 + B * step;
    float* d = d0 + B * RS;
#pragma unroll 1
    for (int j = B; j + B <= J0; j += B) {
#pragma unroll
      for (int i = 0; i < B; ++i) pv[i] = __ldcs(q + i * step);
#pragma unroll
      for (int i = 0; i < B; ++i) d[i * RS] = cvt<float>(pv[i]);
      q += B * step;
      d += B * RS;
    }
    constexpr int REM0 = (J0 - B) % B;
#pragma unroll
    for (int i = 0; i < REM0; ++i) pv[i] = __ldcs(q + i * step);
#pragma unroll
    for (int i = 0; i < REM0; ++i) d[i * RS] = cvt<float>(pv[i]);
    if (v < T0) tile[(5 * J0 + v) * kRC + lane] = cvt<float>(__ldcs(p0 + J0 * step));
  }
  // linear sub-stencil rows, at tile row R0 (after the quadratic rows) or,
  // phased, at row 0 once the quadratic coefficients are formed
  auto stage_linear = [&](float* dbase) {
    const double* p1 = m.pinvm + (int64_t)v * ncp + c0 + lane;
    const double* q = p1;
    float* d = dbase;
#pragma unroll 1
    for (int j = 0; j + B <= J1; j += B) {
#pragma unroll
      for (int i = 0; i < B; ++i) pv[i] = __ldcs(q + i * step);
#pragma unroll
      for (int i = 0; i < B; ++i) d[i * RS] = cvt<float>(pv[i]);
      q += B * step;
      d += B * RS;
    }
    constexpr int REM1 = J1 % B;
#pragma unroll
    for (int i = 0; i < REM1; ++i) pv[i] = __ldcs(q + i * step);
#pragma unroll
    for (int i = 0; i < REM1; ++i) d[i * RS] = cvt<float>(pv[i]);
    if (v < T1) dbase[J1 * RS] = cvt<float>(__ldcs(p1 + J1 * step));
  };
  if constexpr (!S::phased) stage_linear(d0 + R0 * kRC);
  // 5. neighbour states to shared memory ([5][K][kRC]; own states [5][kRC])
#pragma unroll
  for (int i = 0; i < NE; ++i) {
    const int k = v + 5 * i;
    if (k < KE && live) {
      float* dst = k < K ? snbr + k * kRC + lane : sown + lane;
      const int vs = k < K ? K * kRC : kRC;
      dst[0] = qa[i].x;
      dst[vs] = qa[i].y;
      dst[2 * vs] = qa[i].z;
      dst[3 * vs] = qa[i].w;
      dst[4 * vs] = qb[i];
    }
  }
  // 6. sub-stencil positions, second moments and 1/h
  for (int r = v; r < M * KM; r += 5) ssub[r * kRC + lane] = m.subidx[(int64_t)r * ncp + c0 + lane];
  if constexpr (!S::lean)
    for (int r = v; r < 7; r += 5)
      if (live) sgeo[r * kRC + lane] = cvt<float>(r < 6 ? m.mom[(int64_t)r * nc + c0 + lane] : m.hinv[c0 + lane]);
  __syncthreads();
  float res[10];
  // least-squares polynomials (the operation order of k_recon).  On
  // hexahedra, pairs of output rows advance together in packed binary32 FMAs
  // (two independent round-to-nearest FMAs per instruction: the same
  // results); measured 8% faster there and 5% slower on tetrahedra.
  auto row = [&](int r) -> float { return tile[r * kRC + lane]; };
  constexpr int LB = S::phased ? 0 : R0;  // tile row of the first linear row
  float a[9];
  float b[M][3];
  float qv = 0.f;
  if (live) {
    qv = S::lean ? qown : sown[v * kRC + lane];
    float dq[K];
#pragma unroll
    for (int k = 0; k < K; ++k) dq[k] = snbr[(v * K + k) * kRC + lane] - qv;
    if constexpr (M == 8) {
      float2 dq2[K];
#pragma unroll
      for (int k = 0; k < K; ++k) dq2[k] = make_float2(dq[k], dq[k]);
#pragma unroll
      for (int d = 0; d < 8; d += 2) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < K; ++k) acc = __ffma2_rn(make_float2(row(d * K + k), row((d + 1) * K + k)), dq2[k], acc);
        a[d] = acc.x;
        a[d + 1] = acc.y;
      }
      float sacc = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) sacc = fmaf(row(8 * K + k), dq[k], sacc);
      a[8] = sacc;
    } else {
#pragma unroll
      for (int d = 0; d < 9; ++d) {
        float sacc = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) sacc += row(d * K + k) * dq[k];
        a[d] = sacc;
      }
    }
  }
  if constexpr (S::phased) {
    __syncthreads();  // every warp has read its quadratic rows
    stage_linear(d0);
    __syncthreads();
  }
  if (live) {
#pragma unroll
    for (int s = 0; s < M; ++s) {
      float x[KM];
#pragma unroll
      for (int r = 0; r < KM; ++r) x[r] = snbr[(v * K + ssub[(s * KM + r) * kRC + lane]) * kRC + lane] - qv;
      if constexpr (M == 8) {
        float2 acc = make_float2(0.f, 0.f);
        float acc2 = 0.f;
#pragma unroll
        for (int r = 0; r < KM; ++r) {
          acc = __ffma2_rn(make_float2(row(LB + (s * 3) * KM + r), row(LB + (s * 3 + 1) * KM + r)),
                           make_float2(x[r], x[r]), acc);
          acc2 = fmaf(row(LB + (s * 3 + 2) * KM + r), x[r], acc2);
        }
        b[s][0] = acc.x;
        b[s][1] = acc.y;
        b[s][2] = acc2;
      } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          float acc = 0.f;
#pragma unroll
          for (int r = 0; r < KM; ++r) acc += row(LB + (s * 3 + d) * KM + r) * x[r];
          b[s][d] = acc;
        }
      }
    }
    float mi[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) mi[q] = S::lean ? gl[q] : sgeo[q * kRC + lane];
    const float hi = S::lean ? gl[6] : sgeo[6 * kRC + lane];
    const float glin = P.f_glin, g0 = 1.f - float(M) * glin, eps = P.f_eps;
    recon_finish<float, M>(a, b, qv, mi, hi, glin, g0, eps, res);
  }
  write_block_records<float>(tile, res, live, lane, v, nv, coef, c0);
}

template <int K, int M, int KM>
__global__ void __launch_bounds__(kRThreads, ReconSmemF<K, M, KM>::blocks) k_recon_rs(DevMesh m, DevParams P,
                                                                                 const float* __restrict__ Qf,
                                                        float* __restrict__ coef, Control* __restrict__ ctl) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (m.nmesh == 1 && ctl->dt == 0.0) return;  // uniform over the grid (a batch computes every member)
  recon_rs_block<K, M, KM>(m, P, Qf, coef, (int64_t)blockIdx.x * kRC, smem_raw);
}

// Point value and gradient of the combined polynomial of cell c at offset d.
template <typename Real, bool COH = false>
__device__ __forceinline__ void eval_poly(const Real* __restrict__ coef, int64_t c, const Real d[3], Real val[5],
                                          Real grad[5][3]) {
  const Real dxx = d[0] * d[0], dyy = d[1] * d[1], dzz = d[2] * d[2];
  const Real dxy = d[0] * d[1], dyz = d[1] * d[2], dzx = d[2] * d[0];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    Real p[10];
    load10<COH>(coef + c * coef_rec<Real>() + v * 10, p);
    const Real q = p[0], gx = p[1], gy = p[2], gz = p[3];
    const Real kxx = p[4], kyy = p[5], kzz = p[6], kxy = p[7], kyz = p[8], kzx = p[9];
    val[v] = q + gx * d[0] + gy * d[1] + gz * d[2] + kxx * dxx + kyy * dyy + kzz * dzz + kxy * dxy + kyz * dyz +
             kzx * dzx;
    grad[v][0] = gx + Real(2) * kxx * d[0] + kxy * d[1] + kzx * d[2];
    grad[v][1] = gy + Real(2) * kyy * d[1] + kxy * d[0] + kyz * d[2];
    grad[v][2] = gz + Real(2) * kzz * d[2] + kyz * d[1] + kzx * d[0];
  }
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

// Flux of Gauss point g of face f (Eq. flux at one point of the face
// quadrature), rotated back to the global frame and oriented from the owner
// to the neighbour: r[0..4] = F, r[5..9] = dF/dt.  Returns the point's
// quadrature weight times area.
template <typename Real, int G, bool VISC, bool COH = false>
__device__ __forceinline__ Real point_flux(const DevMesh& m, const DevParams& P, const FluxParams<Real>& FP,
                                           const Real* __restrict__ coef, int64_t f, int g, int64_t own, int nbr,
                                           Real dt, Real dt2i, Real r[10]) {
  const int64_t nf = m.nf;
  // planar triangles share one normal; bilinear quads have one per point
  Real n[3], t1[3], t2[3];
  const int gn = G == 3 ? 0 : g;
#pragma unroll
  for (int a = 0; a < 3; ++a) n[a] = cvt<Real>(m.fn[(gn * 3 + a) * nf + f]);
  frame(n, t1, t2);
  Real d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = cvt<Real>(m.fdl[(g * 3 + a) * nf + f]);
  const Real wgt = cvt<Real>(m.fw[g * nf + f]);
  Real qv[5], gr[5][3];
  eval_poly<Real, COH>(coef, own, d, qv, gr);
  // local frame: rotate momentum, take derivatives along n, t1, t2
  Real ql[5], dl[3][5], qr[5], dr[3][5];
  auto rot = [&](const Real x[5], Real y[5]) {
    y[0] = x[0];
    y[1] = x[1] * n[0] + x[2] * n[1] + x[3] * n[2];
    y[2] = x[1] * t1[0] + x[2] * t1[1] + x[3] * t1[2];
    y[3] = x[1] * t2[0] + x[2] * t2[1] + x[3] * t2[2];
    y[4] = x[4];
  };
  auto local = [&](const Real q[5], const Real gg[5][3], Real qo[5], Real dd[3][5]) {
    rot(q, qo);
    Real tmp[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) tmp[v] = gg[v][0] * n[0] + gg[v][1] * n[1] + gg[v][2] * n[2];
    rot(tmp, dd[0]);
#pragma unroll
    for (int v = 0; v < 5; ++v) tmp[v] = gg[v][0] * t1[0] + gg[v][1] * t1[1] + gg[v][2] * t1[2];
    rot(tmp, dd[1]);
#pragma unroll
    for (int v = 0; v < 5; ++v) tmp[v] = gg[v][0] * t2[0] + gg[v][1] * t2[1] + gg[v][2] * t2[2];
    rot(tmp, dd[2]);
  };
  local(qv, gr, ql, dl);
  if (nbr >= 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = cvt<Real>(m.fdr[(g * 3 + a) * nf + f]);
    eval_poly<Real, COH>(coef, (int64_t)nbr, d, qv, gr);
    local(qv, gr, qr, dr);
  } else if (nbr == -3) {
    // no-slip adiabatic wall: mirror state, momentum reversed, normal
    // derivative reflected
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const Real sg = (v >= 1 && v <= 3) ? Real(-1) : Real(1);
      qr[v] = sg * ql[v];
      dr[0][v] = -sg * dl[0][v];
      dr[1][v] = sg * dl[1][v];
      dr[2][v] = sg * dl[2][v];
    }
  } else {
    // Riemann-invariant far field, evaluated in the local frame, zero gradient
    Real qinf[5], qil[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qinf[v] = pick<Real>(P.qinf[v], P.f_qinf[v]);
    rot(qinf, qil);
    const Real ex[3] = {Real(1), Real(0), Real(0)};
    farfield(ql, qil, ex, FP.gamma, qr);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int v = 0; v < 5; ++v) dr[j][v] = Real(0);
  }
  Real Fl[5], Dl[5];
  gks_flux<Real, VISC>(ql, dl, qr, dr, dt, dt2i, FP, Fl, Dl);
  // back to the global frame
  r[0] = Fl[0];
  r[4] = Fl[4];
  r[5] = Dl[0];
  r[9] = Dl[4];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r[1 + a] = fma(Fl[1], n[a], fma(Fl[2], t1[a], Fl[3] * t2[a]));
    r[6 + a] = fma(Dl[1], n[a], fma(Dl[2], t1[a], Dl[3] * t2[a]));
  }
  return wgt;
}

// Face flux of face f: sum over the Gauss points of weight*area times the
// point flux, stored as the face's flux record (store_flux).
template <typename Real, int G, bool VISC, bool COH = false>
__device__ __forceinline__ void flux_face(const DevMesh& m, const DevParams& P, const Real* __restrict__ coef,
                                          Real* __restrict__ Fs, const Control* __restrict__ ctl, int64_t f) {
  const int64_t own = m.fown[f];
  const double dtd = ldm<COH>(&ctl[member_of(m, own)].dt);
  if (dtd == 0.0) return;
  const Real dt = cvt<Real>(dtd), dt2i = Real(2) / dt;
  const FluxParams<Real> FP = flux_params<Real>(P);
  const int nbr = m.fnbr[f];
  Real acc[10];
#pragma unroll
  for (int v = 0; v < 10; ++v) acc[v] = Real(0);
#pragma unroll 1
  for (int g = 0; g < G; ++g) {
    Real r[10];
    const Real w = point_flux<Real, G, VISC, COH>(m, P, FP, coef, f, g, own, nbr, dt, dt2i, r);
#pragma unroll
    for (int v = 0; v < 10; ++v) acc[v] = fma(w, r[v], acc[v]);
  }
  store_flux(Fs, f, acc);
}

// Face flux, one thread per face: sum over the Gauss points of weight*area
// times the point flux.  Output: the flux record of each face (store_flux).
// (binary32 register caps that fit without spilling, measured fastest:
// inviscid 96 registers, 5 blocks per SM; with viscosity 168, 3 blocks per SM)
template <typename Real, int G, bool VISC>
__global__ void __launch_bounds__(kBlock, sizeof(Real) == 4 ? (VISC ? 3 : 5) : 1)
    k_flux(DevMesh m, DevParams P, const Real* __restrict__ coef,
                                                 Real* __restrict__ Fs, const Control* __restrict__ ctl) {
  const int64_t f = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (f < m.nf) flux_face<Real, G, VISC>(m, P, coef, Fs, ctl, f);
}

// Face flux, one thread per Gauss point: the G points of a face run on G
// threads (kBlock / G faces per block), so each thread holds one point's
// state, and the block sums the points of each face in shared memory with
// the same fused multiply-adds, in the same order, as k_flux.
template <typename Real, int G, bool VISC, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_flux_gp(DevMesh m, DevParams P, const Real* __restrict__ coef,
                                                          Real* __restrict__ Fs, const Control* __restrict__ ctl) {
  constexpr int FB = kBlock / G;  // faces per block
  __shared__ Real sr[G][10][FB];
  __shared__ Real sw[G][FB];
  const int64_t nf = m.nf;
  const int gp = threadIdx.x / FB, fl = threadIdx.x - gp * FB;
  const int64_t f0 = (int64_t)blockIdx.x * FB;
  const int64_t f = f0 + fl;
  if (gp < G && f < nf) {
    const int64_t own = m.fown[f];
    const double dtd = ctl[member_of(m, own)].dt;
    Real r[10], w = Real(0);
#pragma unroll
    for (int v = 0; v < 10; ++v) r[v] = Real(0);
    if (dtd != 0.0)
      w = point_flux<Real, G, VISC>(m, P, flux_params<Real>(P), coef, f, gp, own, m.fnbr[f], cvt<Real>(dtd),
                                    Real(2) / cvt<Real>(dtd), r);
    sw[gp][fl] = w;
#pragma unroll
    for (int v = 0; v < 10; ++v) sr[gp][v][fl] = r[v];
  }
  __syncthreads();
  // the block's faces are consecutive records: write them as one contiguous run
  constexpr int REC = flux_rec<Real>();
  for (int e = threadIdx.x; e < REC * FB; e += kBlock) {
    const int l = e / REC, v = e - l * REC;
    if (f0 + l >= nf) break;
    Real acc = Real(0);
    if (v < 10) {
#pragma unroll
      for (int g = 0; g < G; ++g) acc = fma(sw[g][l], sr[g][v][l], acc);
    }
    Fs[f0 * REC + e] = acc;
  }
}

// Gather of the face fluxes of cell c (Eq. finite): the signed face sums a
// (of F) and b (of dF/dt), with L = -a/|cell| and dL/dt = -b/|cell|.  The
// face sum runs in the flux precision; the sums enter the S2O4 update in
// binary64, where the factor -1/|cell| is folded into the stage coefficients.
template <typename Real, int NFC, bool COH = false>
__device__ __forceinline__ void gather(const DevMesh& m, const Real* __restrict__ Fs, int64_t c, double a[5],
                                       double b[5]) {
  Real sa[5] = {0, 0, 0, 0, 0}, sb[5] = {0, 0, 0, 0, 0};
#pragma unroll
  for (int p = 0; p < NFC; ++p) {
    const int32_t e = m.cface[p * m.nc + c];
    const int64_t f = e >> 1;
    Real x[10];
    load_flux<COH>(Fs, f, x);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      sa[v] += (e & 1) ? -x[v] : x[v];
      sb[v] += (e & 1) ? -x[5 + v] : x[5 + v];
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    if constexpr (sizeof(Real) == 4) {
      a[v] = f2d(sa[v]);
      b[v] = f2d(sb[v]);
    } else {
      a[v] = sa[v];
      b[v] = sb[v];
    }
  }
}

// Stage 1: Q* = Q + dt/2 L + dt^2/8 dL;  R = Q + dt L + dt^2/6 dL.
template <typename Real, int NFC, bool COH = false>
__device__ __forceinline__ void update1_cell(const DevMesh& m, const Real* __restrict__ Fs,
                                             const double* __restrict__ Q, double* __restrict__ Qs,
                                             double* __restrict__ R, float* __restrict__ Qf, double dt, int64_t c) {
  double a[5], b[5];
  gather<Real, NFC, COH>(m, Fs, c, a, b);
  const double r1 = -dt * m.volinv[c], r2 = r1 * dt;  // dt L = r1 a, dt^2 dL = r2 b
  const double h1 = 0.5 * r1, h2 = 0.125 * r2, k2 = r2 * (1.0 / 6.0);
  double qs[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double q = ldm<COH>(Q + v * m.nce + c);
    qs[v] = fma(h2, b[v], fma(h1, a[v], q));
    Qs[v * m.nce + c] = qs[v];
    R[v * m.nc + c] = fma(k2, b[v], fma(r1, a[v], q));
  }
  if (Qf) store_qf(Qf, c, qs);
}

template <typename Real, int NFC>
__global__ void __launch_bounds__(kBlock) k_update1(DevMesh m, const Real* __restrict__ Fs, const double* __restrict__ Q,
                                                   double* __restrict__ Qs, double* __restrict__ R,
                                                   float* __restrict__ Qf, const Control* __restrict__ ctl) {
  const int64_t c = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (c >= m.nc) return;
  const double dt = ctl[member_of(m, c)].dt;
  if (dt == 0.0) return;
  update1_cell<Real, NFC>(m, Fs, Q, Qs, R, Qf, dt, c);
}

// Stage 2: Q^{n+1} = R + dt^2/3 dL(Q*); returns the cell's next step bound
// (infinity when there is none) and flags a non-finite result.
template <typename Real, int NFC, bool COH = false>
__device__ __forceinline__ double update2_cell(const DevMesh& m, const DevParams& P, const Real* __restrict__ Fs,
                                               double* __restrict__ Q, const double* __restrict__ R,
                                               float* __restrict__ Qf, Control* __restrict__ ctl, int mid,
                                               double dt, int64_t c) {
  double a[5], b[5];
  gather<Real, NFC, COH>(m, Fs, c, a, b);
  const double k2 = -dt * dt * m.volinv[c] * (1.0 / 3.0);  // dt^2/3 dL = k2 b
  double q[5];
  bool finite = true;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    q[v] = fma(k2, b[v], ldm<COH>(R + v * m.nc + c));
    finite = finite && isfinite(q[v]);
    Q[v * m.nce + c] = q[v];
  }
  if (!finite) atomicOr(&ctl[mid].flags, FLAG_NONFINITE);
  double bound;
  if (Qf) {
    float qf[5];
    store_qf(Qf, c, q, qf);
    bound = f2d(cell_dt_f(qf, cvt<float>(m.hdt[c]), P));
  } else {
    bound = cell_dt(q, m.hdt[c], P);
  }
  return (bound >= 0.0) ? bound : __longlong_as_double(0x7ff0000000000000LL);
}

template <typename Real, int NFC>
__global__ void __launch_bounds__(kBlock) k_update2(DevMesh m, DevParams P, const Real* __restrict__ Fs,
                                                   double* __restrict__ Q, const double* __restrict__ R,
                                                   float* __restrict__ Qf, Control* __restrict__ ctl) {
  const int64_t c = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (m.nmesh == 1 && ctl->dt == 0.0) return;  // uniform: no thread reaches the block reduction
  double bound = __longlong_as_double(0x7ff0000000000000LL);
  const int mid = c < m.nc ? member_of(m, c) : -1;
  const double dt = mid >= 0 ? ctl[mid].dt : 0.0;
  if (dt != 0.0) bound = update2_cell<Real, NFC>(m, P, Fs, Q, R, Qf, ctl, mid, dt, c);
  member_min_to(m, ctl, dt != 0.0 ? mid : -1, bound);
}

// Binary32 copy of the state (mixed precision).
// Caller order and layout ([n][5], member-local index perm[c]) to the internal
// structure-of-arrays order of cells coff .. coff+n-1, and back.
__global__ void k_state_in(const double* __restrict__ in, const int32_t* __restrict__ perm, int64_t coff,
                           int64_t n, double* __restrict__ Q, int64_t nce) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  const double* src = in + 5 * (int64_t)perm[coff + i];
#pragma unroll
  for (int v = 0; v < 5; ++v) Q[v * nce + coff + i] = src[v];
}

__global__ void k_state_out(const double* __restrict__ Q, const int32_t* __restrict__ perm, int64_t coff,
                            int64_t n, int64_t nce, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  double* dst = out + 5 * (int64_t)perm[coff + i];
#pragma unroll
  for (int v = 0; v < 5; ++v) dst[v] = Q[v * nce + coff + i];
}

__global__ void k_tofloat(const double* __restrict__ Q, float* __restrict__ Qf, int64_t nce) {
  const int64_t c = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (c >= nce) return;
  double q[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) q[v] = Q[v * nce + c];
  store_qf(Qf, c, q);
}

__global__ void k_setdt(Control* ctl, int n, double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ctl[i].dt = dt;
}

// L and dL/dt of the state (test path).
template <typename Real, int NFC>
__global__ void k_operator(DevMesh m, const Real* __restrict__ Fs, double* __restrict__ L, double* __restrict__ dL) {
  const int64_t c = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (c >= m.nc) return;
  double a[5], b[5];
  gather<Real, NFC>(m, Fs, c, a, b);
  const double vi = -m.volinv[c];
  for (int v = 0; v < 5; ++v) { L[v * m.nc + c] = a[v] * vi; dL[v * m.nc + c] = b[v] * vi; }
}

// --------------------------------------------------------------------------
// Persistent steps (the batching of small meshes): one cooperative launch
// advances every member of a solver by n S2O4 steps.  The phases of a step
// are those of the separate kernels above (time step; then twice ghosts,
// reconstruction, flux and update), run by the same device functions and
// separated by grid-wide barriers.  Data that other blocks of the launch
// wrote is read through L2 (COH = true loads).
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}

// Grid-wide barrier of a cooperative launch (all blocks are resident), with a
// bounded wait: false after `limit` clock cycles (2^31 by default, about a
// second), with FLAG_BAR_TIMEOUT set on member 0; the caller then leaves the
// kernel, and so does every other block at its own bounded wait (the last
// block to arrive never waits, so each barrier lets at most one block through
// once another has left).
__device__ bool grid_sync(GridBar* b, Control* ctl, long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = ld_volatile(&b->gen);
    __threadfence();
    if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_volatile(&b->gen) == g) {
        if (clock64() - t0 > limit) {
          atomicOr(&ctl->flags, FLAG_BAR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename Real, int K, int M, int KM, int G, int NFC, bool VISC>
__global__ void __launch_bounds__(kRThreads, sizeof(Real) == 4 ? 2 : 1)
    k_persist(DevMesh m, DevParams P, DevWork w, int nsteps) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr bool F32 = sizeof(Real) == 4;
  const double kInf = __longlong_as_double(0x7ff0000000000000LL);
  Real* coef = static_cast<Real*>(w.coef);
  Real* Fs = static_cast<Real*>(w.Fs);
  float* Qf = F32 ? w.Qf : nullptr;
  Control* ctl = w.ctl;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ntiles = (m.nc + kRC - 1) / kRC;
  for (int step = 0; step < nsteps; ++step) {
    if (blockIdx.x == 0)
      for (int i = threadIdx.x; i < m.nmesh; i += blockDim.x) finalize_one<true>(ctl + i, P.cfl);
    if (!grid_sync(w.bar, ctl, P.bar_cycles)) return;
    const bool idle = m.nmesh == 1 && ldm<true>(&ctl->dt) == 0.0;  // the same in every block
    for (int stage = 0; stage < 2; ++stage) {
      double* Qin = stage == 0 ? w.Q : w.Qs;
      if (m.ng) {
        if (!idle)
          for (int64_t g = gt; g < m.ng; g += nthr) ghost_one<true>(m, P, Qin, Qf, ctl, g);
        if (!grid_sync(w.bar, ctl, P.bar_cycles)) return;
      }
      if (!idle) {
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
          if constexpr (F32) recon_rs_block<K, M, KM, true>(m, P, w.Qf, coef, t * kRC, smem_raw);
          else recon_block<Real, double, K, M, KM, false, true>(m, P, Qin, coef, ctl, t * kRC, smem_raw);
          __syncthreads();  // the next tile reuses the shared memory
        }
      }
      if (!grid_sync(w.bar, ctl, P.bar_cycles)) return;
      if (!idle)
        for (int64_t f = gt; f < m.nf; f += nthr) flux_face<Real, G, VISC, true>(m, P, coef, Fs, ctl, f);
      if (!grid_sync(w.bar, ctl, P.bar_cycles)) return;
      if (stage == 0) {
        if (!idle)
          for (int64_t c = gt; c < m.nc; c += nthr) {
            const double dt = ldm<true>(&ctl[member_of(m, c)].dt);
            if (dt != 0.0) update1_cell<Real, NFC, true>(m, Fs, w.Q, w.Qs, w.R, Qf, dt, c);
          }
      } else if (!idle) {
        // whole blocks per round, so that every thread takes part in the
        // block's step-bound reduction
        for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x; c0 < m.nc; c0 += nthr) {
          const int64_t c = c0 + threadIdx.x;
          const int mid = c < m.nc ? member_of(m, c) : -1;
          const double dt = mid >= 0 ? ldm<true>(&ctl[mid].dt) : 0.0;
          const double bound = dt != 0.0 ? update2_cell<Real, NFC, true>(m, P, Fs, w.Q, w.R, Qf, ctl, mid, dt, c)
                                         : kInf;
          member_min_to<kRThreads / 32>(m, ctl, dt != 0.0 ? mid : -1, bound);
          __syncthreads();  // the reduction's shared buffer is reused
        }
      }
      if (!grid_sync(w.bar, ctl, P.bar_cycles)) return;
    }
  }
}

// Dynamic shared memory of the persistent kernel: the reconstruction tile.
template <typename Real, int K, int M, int KM>
constexpr size_t persist_smem() {
  if constexpr (sizeof(Real) == 4) return ReconSmemF<K, M, KM>::bytes;
  else return ReconSmem<Real, K, M, KM>::dq;
}

template <typename Real, int K, int M, int KM, int G, int NFC>
cudaError_t persist_launch(const DevMesh& m, const DevParams& p, const DevWork& w, int n, cudaStream_t s,
                           bool prep) {
  const size_t smem = persist_smem<Real, K, M, KM>();
  const void* fn = p.viscous ? (const void*)k_persist<Real, K, M, KM, G, NFC, true>
                             : (const void*)k_persist<Real, K, M, KM, G, NFC, false>;
  if (prep) {
    cudaFuncSetAttribute(k_persist<Real, K, M, KM, G, NFC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaFuncSetAttribute(k_persist<Real, K, M, KM, G, NFC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    return cudaSuccess;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kRThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  // no more blocks than the largest phase has units of work for
  const int64_t want = std::max<int64_t>((m.nc + kRC - 1) / kRC, (m.nf + kRThreads - 1) / kRThreads);
  const unsigned grid = (unsigned)std::min<int64_t>((int64_t)per_sm * sms, std::max<int64_t>(want, 1));
  e = cudaMemsetAsync(w.bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  DevMesh mm = m;
  DevParams pp = p;
  DevWork ww = w;
  int nn = n;
  void* args[] = {&mm, &pp, &ww, &nn};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kRThreads), args, smem, s);
}

template <typename Real>
cudaError_t persist_any(const DevMesh& m, const DevParams& p, const DevWork& w, int n, cudaStream_t s,
                        bool prep) {
  if (m.M == 4) {
    switch (m.K) {
      case 12: return persist_launch<Real, 12, 4, 6, 3, 4>(m, p, w, n, s, prep);
      case 13: return persist_launch<Real, 13, 4, 6, 3, 4>(m, p, w, n, s, prep);
      case 14: return persist_launch<Real, 14, 4, 6, 3, 4>(m, p, w, n, s, prep);
      case 15: return persist_launch<Real, 15, 4, 6, 3, 4>(m, p, w, n, s, prep);
      case 16: return persist_launch<Real, 16, 4, 6, 3, 4>(m, p, w, n, s, prep);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (m.K) {
    case 18: return persist_launch<Real, 18, 8, 3, 4, 6>(m, p, w, n, s, prep);
    case 20: return persist_launch<Real, 20, 8, 3, 4, 6>(m, p, w, n, s, prep);
    case 22: return persist_launch<Real, 22, 8, 3, 4, 6>(m, p, w, n, s, prep);
    case 24: return persist_launch<Real, 24, 8, 3, 4, 6>(m, p, w, n, s, prep);
    case 26: return persist_launch<Real, 26, 8, 3, 4, 6>(m, p, w, n, s, prep);
    default: return cudaErrorInvalidValue;
  }
}

inline unsigned blocks(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// Variants: binary64, 0 = rows staged by bulk asynchronous copies, 1 = rows
// read directly; binary32, 0 = k_recon_rs, 1 = rows staged by bulk
// asynchronous copies.
template <typename Real, typename QT, int K, int M, int KM>
void recon_launch(const DevMesh& m, const DevParams& p, const QT* Q, Real* coef, Control* ctl, cudaStream_t s,
                  bool prep) {
  using S = ReconSmem<Real, K, M, KM>;
  const unsigned nb = (unsigned)((m.nc + kRC - 1) / kRC);
  if constexpr (sizeof(Real) == 4) {
    using SF = ReconSmemF<K, M, KM>;
    if (prep) {
      cudaFuncSetAttribute(k_recon<Real, QT, K, M, KM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)S::bytes);
      cudaFuncSetAttribute(k_recon_rs<K, M, KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SF::bytes);
      return;
    }
    if (p.recon_variant == 1) k_recon<Real, QT, K, M, KM, true><<<nb, kRThreads, S::bytes, s>>>(m, p, Q, coef, ctl);
    else k_recon_rs<K, M, KM><<<nb, kRThreads, SF::bytes, s>>>(m, p, Q, coef, ctl);
  } else {
    if (prep) {
      cudaFuncSetAttribute(k_recon<Real, QT, K, M, KM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)S::bytes);
      cudaFuncSetAttribute(k_recon<Real, QT, K, M, KM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)S::dq);
      return;
    }
    if (p.recon_variant == 1) k_recon<Real, QT, K, M, KM, false><<<nb, kRThreads, S::dq, s>>>(m, p, Q, coef, ctl);
    else k_recon<Real, QT, K, M, KM, true><<<nb, kRThreads, S::bytes, s>>>(m, p, Q, coef, ctl);
  }
}

// Stencil shapes compiled in: tetrahedra with 12..16 members and 4 sub-stencils
// of up to 6; hexahedra with 18..24 members and 8 octants of 3.
template <typename Real, typename QT, int M, int KM>
void recon_dispatch(const DevMesh& m, const DevParams& p, const QT* Q, Real* coef, Control* ctl, cudaStream_t s,
                    bool prep) {
  switch (m.K) {
    case 12: recon_launch<Real, QT, 12, M, KM>(m, p, Q, coef, ctl, s, prep); break;
    case 13: recon_launch<Real, QT, 13, M, KM>(m, p, Q, coef, ctl, s, prep); break;
    case 14: recon_launch<Real, QT, 14, M, KM>(m, p, Q, coef, ctl, s, prep); break;
    case 15: recon_launch<Real, QT, 15, M, KM>(m, p, Q, coef, ctl, s, prep); break;
    case 16: recon_launch<Real, QT, 16, M, KM>(m, p, Q, coef, ctl, s, prep); break;
    default: break;
  }
}
template <typename Real, typename QT>
void recon_hex(const DevMesh& m, const DevParams& p, const QT* Q, Real* coef, Control* ctl, cudaStream_t s,
               bool prep) {
  switch (m.K) {
    case 18: recon_launch<Real, QT, 18, 8, 3>(m, p, Q, coef, ctl, s, prep); break;
    case 20: recon_launch<Real, QT, 20, 8, 3>(m, p, Q, coef, ctl, s, prep); break;
    case 22: recon_launch<Real, QT, 22, 8, 3>(m, p, Q, coef, ctl, s, prep); break;
    case 24: recon_launch<Real, QT, 24, 8, 3>(m, p, Q, coef, ctl, s, prep); break;
    case 26: recon_launch<Real, QT, 26, 8, 3>(m, p, Q, coef, ctl, s, prep); break;
    default: break;
  }
}

// Stencil sizes the kernels are compiled for.
}  // namespace
bool stencil_supported(int nfc, int K) {
  if (nfc == 4) return K >= 12 && K <= 16;
  // hexahedra 18-24; hybrid hex/prism meshes reach 26
  return K == 18 || K == 20 || K == 22 || K == 24 || K == 26;
}
namespace {

template <typename Real, typename QT>
void recon_any(const DevMesh& m, const DevParams& p, const QT* Q, Real* coef, Control* ctl, cudaStream_t s,
               bool prep = false) {
  if (m.M == 4) recon_dispatch<Real, QT, 4, 6>(m, p, Q, coef, ctl, s, prep);
  else recon_hex<Real, QT>(m, p, Q, coef, ctl, s, prep);
}

template <typename Real, int G, bool VISC>
void flux_launch(const DevMesh& m, const DevParams& p, const Real* coef, Real* Fs, const Control* ctl, cudaStream_t s) {
  if (p.flux_variant == 1) {
    constexpr int FB = kBlock / G;
    // binary32: 4 blocks of 128 per SM (128 registers), 3 with viscosity
    // (168 registers, few spills); binary64: 2
    k_flux_gp<Real, G, VISC, sizeof(Real) == 4 ? (VISC ? 3 : 4) : 2>
        <<<(unsigned)((m.nf + FB - 1) / FB), kBlock, 0, s>>>(m, p, coef, Fs, ctl);
  } else {
    k_flux<Real, G, VISC><<<blocks(m.nf), kBlock, 0, s>>>(m, p, coef, Fs, ctl);
  }
}

template <typename Real>
void flux_any(const DevMesh& m, const DevParams& p, const Real* coef, Real* Fs, const Control* ctl, cudaStream_t s) {
  if (m.G == 3) {
    if (p.viscous) flux_launch<Real, 3, true>(m, p, coef, Fs, ctl, s);
    else flux_launch<Real, 3, false>(m, p, coef, Fs, ctl, s);
  } else {
    if (p.viscous) flux_launch<Real, 4, true>(m, p, coef, Fs, ctl, s);
    else flux_launch<Real, 4, false>(m, p, coef, Fs, ctl, s);
  }
}
template <typename Real>
void stage_pair(const DevMesh& m, const DevParams& p, const DevWork& w, bool mixed, cudaStream_t s,
                const StepEvents* ev) {
  Real* coef = static_cast<Real*>(w.coef);
  Real* Fs = static_cast<Real*>(w.Fs);
  const unsigned nbc = blocks(m.nc);
  float* Qf = mixed ? w.Qf : nullptr;
  auto mark = [&](int i) { if (ev) cudaEventRecord(ev->ev[i], s); };
  // stage 1 on Q^n
  if (m.ng) k_ghost<<<blocks(m.ng), kBlock, 0, s>>>(m, p, w.Q, Qf, w.ctl);
  if constexpr (std::is_same_v<Real, float>) recon_any<Real, float>(m, p, w.Qf, coef, w.ctl, s);
  else recon_any<Real, double>(m, p, w.Q, coef, w.ctl, s);
  mark(2);
  flux_any<Real>(m, p, coef, Fs, w.ctl, s);
  mark(3);
  if (m.nfc == 4) k_update1<Real, 4><<<nbc, kBlock, 0, s>>>(m, Fs, w.Q, w.Qs, w.R, Qf, w.ctl);
  else k_update1<Real, 6><<<nbc, kBlock, 0, s>>>(m, Fs, w.Q, w.Qs, w.R, Qf, w.ctl);
  mark(4);
  // stage 2 on Q*
  if (m.ng) k_ghost<<<blocks(m.ng), kBlock, 0, s>>>(m, p, w.Qs, Qf, w.ctl);
  if constexpr (std::is_same_v<Real, float>) recon_any<Real, float>(m, p, w.Qf, coef, w.ctl, s);
  else recon_any<Real, double>(m, p, w.Qs, coef, w.ctl, s);
  mark(5);
  flux_any<Real>(m, p, coef, Fs, w.ctl, s);
  mark(6);
  if (m.nfc == 4) k_update2<Real, 4><<<nbc, kBlock, 0, s>>>(m, p, Fs, w.Q, w.R, Qf, w.ctl);
  else k_update2<Real, 6><<<nbc, kBlock, 0, s>>>(m, p, Fs, w.Q, w.R, Qf, w.ctl);
  mark(7);
}

}  // namespace

void launch_setdt(const DevMesh& m, const DevWork& w, double dt, cudaStream_t s) {
  k_setdt<<<(m.nmesh + 127) / 128, 128, 0, s>>>(w.ctl, m.nmesh, dt);
}

void launch_state_in(const DevMesh& m, const double* in, int64_t coff, int64_t n, double* Q, cudaStream_t s) {
  if (n > 0) k_state_in<<<blocks(n), kBlock, 0, s>>>(in, m.perm, coff, n, Q, m.nce);
}

void launch_state_out(const DevMesh& m, const double* Q, int64_t coff, int64_t n, double* out, cudaStream_t s) {
  if (n > 0) k_state_out<<<blocks(n), kBlock, 0, s>>>(Q, m.perm, coff, n, m.nce, out);
}

float time_stage(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, int reps, cudaStream_t s) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -1.f; }
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) {
    if (precision == 1) {
      recon_any<float, float>(m, p, w.Qf, static_cast<float*>(w.coef), w.ctl, s);
      flux_any<float>(m, p, static_cast<float*>(w.coef), static_cast<float*>(w.Fs), w.ctl, s);
    } else {
      recon_any<double, double>(m, p, w.Q, static_cast<double*>(w.coef), w.ctl, s);
      flux_any<double>(m, p, static_cast<double*>(w.coef), static_cast<double*>(w.Fs), w.ctl, s);
    }
  }
  cudaEventRecord(e1, s);
  float ms = -1.f;
  if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return reps > 0 && ms >= 0.f ? ms / reps : -1.f;
}

void prepare_kernels(const DevMesh& m, int precision) {
  if (precision == 1) {
    recon_any<float, float>(m, DevParams{}, nullptr, nullptr, nullptr, 0, true);
    persist_any<float>(m, DevParams{}, DevWork{}, 0, 0, true);
  } else {
    recon_any<double, double>(m, DevParams{}, nullptr, nullptr, nullptr, 0, true);
    persist_any<double>(m, DevParams{}, DevWork{}, 0, 0, true);
  }
}

cudaError_t launch_persistent(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, int n,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return precision == 1 ? persist_any<float>(m, p, w, n, s, false) : persist_any<double>(m, p, w, n, s, false);
}

void launch_control(const DevMesh& m, const DevWork& w, double t_end, double dt_fixed, cudaStream_t s) {
  k_control<<<(m.nmesh + 127) / 128, 128, 0, s>>>(w.ctl, m.nmesh, t_end, dt_fixed);
}

void launch_reset(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, int only, double t,
                  cudaStream_t s) {
  k_reset<<<(m.nmesh + 127) / 128, 128, 0, s>>>(w.ctl, m.nmesh, only, t);
  if (precision == 1) k_tofloat<<<blocks(m.nce), kBlock, 0, s>>>(w.Q, w.Qf, m.nce);
  k_dt<<<blocks(m.nc), kBlock, 0, s>>>(m, p, w.Q, precision == 1 ? w.Qf : nullptr, w.ctl);
}

void launch_step(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, cudaStream_t s,
                 const StepEvents* ev) {
  if (ev) cudaEventRecord(ev->ev[0], s);
  k_finalize<<<(m.nmesh + 127) / 128, 128, 0, s>>>(w.ctl, m.nmesh, p.cfl);
  if (ev) cudaEventRecord(ev->ev[1], s);
  if (precision == 1) stage_pair<float>(m, p, w, true, s, ev);
  else stage_pair<double>(m, p, w, false, s, ev);
}

void launch_operator(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, double dt, double* L,
                     double* dL, cudaStream_t s) {
  k_setdt<<<(m.nmesh + 127) / 128, 128, 0, s>>>(w.ctl, m.nmesh, dt);
  const bool mixed = precision == 1;
  float* Qf = mixed ? w.Qf : nullptr;
  if (m.ng) k_ghost<<<blocks(m.ng), kBlock, 0, s>>>(m, p, w.Q, Qf, w.ctl);
  if (mixed) {
    recon_any<float, float>(m, p, w.Qf, static_cast<float*>(w.coef), w.ctl, s);
    flux_any<float>(m, p, static_cast<float*>(w.coef), static_cast<float*>(w.Fs), w.ctl, s);
    if (m.nfc == 4) k_operator<float, 4><<<blocks(m.nc), kBlock, 0, s>>>(m, static_cast<float*>(w.Fs), L, dL);
    else k_operator<float, 6><<<blocks(m.nc), kBlock, 0, s>>>(m, static_cast<float*>(w.Fs), L, dL);
  } else {
    recon_any<double, double>(m, p, w.Q, static_cast<double*>(w.coef), w.ctl, s);
    flux_any<double>(m, p, static_cast<double*>(w.coef), static_cast<double*>(w.Fs), w.ctl, s);
    if (m.nfc == 4) k_operator<double, 4><<<blocks(m.nc), kBlock, 0, s>>>(m, static_cast<double*>(w.Fs), L, dL);
    else k_operator<double, 6><<<blocks(m.nc), kBlock, 0, s>>>(m, static_cast<double*>(w.Fs), L, dL);
  }
}

}  // namespace hgks

// hgks_dev_flux.cuh -- face flux kernels (Section 2.1, Eq. flux at the
// face Gauss points; Section 2.2 linear-in-time fit): k_flux (one thread per
// face) and k_flux_gp (one thread per Gauss point).
#pragma once

#include "hgks_dev_common.cuh"

namespace hgks {
namespace {
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

// Face geometry in the flux precision: the binary64 array, or its binary32
// rounding stored with the mesh.
template <typename Real>
__device__ __forceinline__ Real geo(const double* __restrict__ a64, const float* __restrict__ a32, int64_t i) {
  if constexpr (sizeof(Real) == 4) return __ldg(a32 + i);
  else return a64[i];
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
  for (int a = 0; a < 3; ++a) n[a] = geo<Real>(m.fn, m.fn32, (gn * 3 + a) * nf + f);
  frame(n, t1, t2);
  Real d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = geo<Real>(m.fdl, m.fdl32, (g * 3 + a) * nf + f);
  const Real wgt = geo<Real>(m.fw, m.fw32, g * nf + f);
  // local frame: rotate momentum, take derivatives along n, t1, t2
  auto rot = [&](const Real x[5], Real y[5]) {
    y[0] = x[0];
    y[1] = x[1] * n[0] + x[2] * n[1] + x[3] * n[2];
    y[2] = x[1] * t1[0] + x[2] * t1[1] + x[3] * t1[2];
    y[3] = x[1] * t2[0] + x[2] * t2[1] + x[3] * t2[2];
    y[4] = x[4];
  };
  // the side state at offset d of cell c, in the local frame
  auto local = [&](int64_t c, Real qo[5], Real dd[3][5]) {
    Real q[5], gg[5][3];
    eval_poly<Real, COH>(coef, c, d, q, gg);
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
  // the two sides one after the other, each folded into the running sums
  // (the owner's side starts them); with viscosity each side is folded in
  // before the next is evaluated, which keeps the register footprint down
  Real q0[5], dq0[3][5], S[3][5], plp = Real(0), prp = Real(0);
#ifndef FLUX_INVISCID_BOTH_FIRST
#define FLUX_INVISCID_BOTH_FIRST 0
#endif
  constexpr bool both_first = !VISC && FLUX_INVISCID_BOTH_FIRST;
  Real ql[5], dl[3][5];
  local(own, ql, dl);
  if constexpr (!both_first) side_flux<Real, VISC, true>(ql, dl, +1, FP, q0, dq0, S, plp);
  {
    Real qr[5], dr[3][5];
    if (nbr >= 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) d[a] = geo<Real>(m.fdr, m.fdr32, (g * 3 + a) * nf + f);
      local((int64_t)nbr, qr, dr);
    } else {
      // with viscosity: the owner's side again (cheaper to re-evaluate than
      // to keep live)
      if constexpr (!both_first) local(own, ql, dl);
      if (nbr == -3) {
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
    }
    if constexpr (both_first) side_flux<Real, VISC, true>(ql, dl, +1, FP, q0, dq0, S, plp);
    side_flux<Real, VISC, false>(qr, dr, -1, FP, q0, dq0, S, prp);
  }
  Real Fl[5], Dl[5];
  eq_flux<Real, VISC>(q0, dq0, S, plp, prp, dt, dt2i, FP, Fl, Dl);
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
// Binary32 blocks per SM, measured fastest: inviscid 5 (96 registers, no
// spills; 6 and 7 spill and run 5% and 13% slower), viscous 4 (128 registers,
// 36 bytes of spills; 2% faster than 3 blocks at 168 registers).
#ifndef FLUX_INVISC_BLOCKS
#define FLUX_INVISC_BLOCKS 5
#endif
#ifndef FLUX_VISC_BLOCKS
#define FLUX_VISC_BLOCKS 4
#endif
template <typename Real, int G, bool VISC>
__global__ void __launch_bounds__(kBlock, sizeof(Real) == 4 ? (VISC ? FLUX_VISC_BLOCKS : FLUX_INVISC_BLOCKS) : 1)
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

}  // namespace
}  // namespace hgks

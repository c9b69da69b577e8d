// hgks_dev_update.cuh -- gather of the face fluxes per cell and the two
// S2O4 stages (Section 2.2, Eq. finite), and the state layout kernels.
#pragma once

#include "hgks_dev_common.cuh"

namespace hgks {
namespace {
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

// Binary32 rounding of a binary64 array (cvt<float>, as the binary32 kernels
// round the geometry they read).
__global__ void k_round32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i < n) b[i] = cvt<float>(a[i]);
}

// Binary32 reconstruction records (layout: rec32_bytes), one thread per
// 4-byte word of a record.
__global__ void k_rec32(DevMesh m, float* __restrict__ rec) {
  const int R0 = 9 * m.K;
  const int64_t words = rec32_bytes(m.K, m.M, m.KM) / 4;
  const int64_t qend = (int64_t)(R0 + 7) * 32;           // quadratic and geometry rows
  const int64_t pend = qend + (int64_t)m.M * m.KM * 8;  // and the position bytes
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= words * (m.ncp / 32)) return;
  const int64_t b = i / words, w = i - b * words;
  if (w < pend && w >= qend) {
    // bytes 4e .. 4e+3 of the position rows ([M KM][32])
    const int64_t e = w - qend;
    uint32_t word = 0;
    for (int k = 0; k < 4; ++k) {
      const int64_t y = 4 * e + k, r = y / 32, c = b * 32 + (y - r * 32);
      word |= (uint32_t)m.subidx[r * m.ncp + c] << (8 * k);
    }
    reinterpret_cast<uint32_t*>(rec)[i] = word;
    return;
  }
  const int64_t e = w < qend ? w : w - pend;
  const int r = (int)(e / 32);
  const int64_t c = b * 32 + (e - (int64_t)r * 32);
  double x = 0.0;
  if (w >= pend) x = m.pinvm[(int64_t)r * m.ncp + c];
  else if (r < R0) x = m.pinv0[(int64_t)r * m.ncp + c];
  else if (c < m.nc) x = r < R0 + 6 ? m.mom[(int64_t)(r - R0) * m.nc + c] : m.hinv[c];
  rec[i] = cvt<float>(x);
}

// erfcx_tab on n values (test path).
__global__ void k_test_erfcx(const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i < n) y[i] = erfcx_tab(x[i]);
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

}  // namespace
}  // namespace hgks

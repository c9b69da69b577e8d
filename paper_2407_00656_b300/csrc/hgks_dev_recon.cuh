// hgks_dev_recon.cuh -- third-order WENO reconstruction kernels (Section
// 2.3, Eqs. polys and weno): k_recon (bulk-copy staged or direct) and
// k_recon_rs (binary32, staged through registers).
#pragma once

#include "hgks_dev_common.cuh"

namespace hgks {
namespace {
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

// The least-squares polynomials of one (variable, cell) thread from a
// binary32 tile of inverse rows ([rows][kRC]) and the block's neighbour
// states snbr ([5][K][kRC]) less the cell's own qv: the quadratic (a, 9
// coefficients from tile rows 0 .. 9K-1) and the linear ones (b, 3 per
// sub-stencil from rows LB .. LB + 3 M KM - 1, members at positions ssub).
// The operation order is that of k_recon.  On hexahedra, pairs of output
// rows advance together in packed binary32 FMAs (two independent
// round-to-nearest FMAs per instruction: the same results); measured 8%
// faster there and 5% slower on tetrahedra.
template <int K, int M>
__device__ __forceinline__ void rs_quadratic(const float* tile, const float* snbr, float qv, int v, int lane,
                                             float a[9]) {
  auto row = [&](int r) -> float { return tile[r * kRC + lane]; };
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

template <int K, int M, int KM, int LB>
__device__ __forceinline__ void rs_linear(const float* tile, const float* snbr, const uint8_t* ssub, float qv, int v,
                                          int lane, float b[M][3]) {
  auto row = [&](int r) -> float { return tile[r * kRC + lane]; };
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
}

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
  // rows per batch of loads, measured: 12 in the tile layouts (8 is 5%
  // slower on tetrahedra, 16 slower on hexahedra); 8 in the lean layout,
  // whose register-held own state and geometry leave less room (12 took the
  // K = 26 hybrid shell from 2.52 to 4.58 ms per step)
  constexpr int B = S::lean ? 8 : 12;
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
  // least-squares polynomials (rs_quadratic, rs_linear)
  constexpr int LB = S::phased ? 0 : R0;  // tile row of the first linear row
  float a[9];
  float b[M][3];
  float qv = 0.f;
  if (live) {
    qv = S::lean ? qown : sown[v * kRC + lane];
    rs_quadratic<K, M>(tile, snbr, qv, v, lane, a);
  }
  if constexpr (S::phased) {
    __syncthreads();  // every warp has read its quadratic rows
    stage_linear(d0);
    __syncthreads();
  }
  if (live) {
    rs_linear<K, M, KM, LB>(tile, snbr, ssub, qv, v, lane, b);
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

}  // namespace
}  // namespace hgks

// hgks_dev_recon.cuh -- third-order WENO reconstruction kernels (Section
// 2.3, Eqs. polys and weno): k_recon (bulk-copy staged or direct) and
// k_recon_rs (binary32, from per-block records moved by bulk copies).
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
// are one contiguous run of memory): each (variable, cell) result is put
// into shared memory (pitch record + 1, which spreads a warp's stores over
// the banks), then the block's NT threads write the run with coalesced
// stores.  smem must hold kRC x (record + 1) reals and no longer be read by
// any warp's arithmetic; every thread of the block calls these.
template <typename Real>
__device__ __forceinline__ void stage_record(Real* smem, const Real res[10], int lane, int v) {
  constexpr int REC = coef_rec<Real>(), PITCH = REC + 1;
#pragma unroll
  for (int j = 0; j < 10; ++j) smem[lane * PITCH + v * 10 + j] = res[j];
  if (v == 0)
    for (int j = 50; j < REC; ++j) smem[lane * PITCH + j] = Real(0);
}
template <typename Real, int NT>
__device__ __forceinline__ void flush_records(const Real* smem, int nv, Real* __restrict__ coef, int64_t c0) {
  constexpr int REC = coef_rec<Real>(), PITCH = REC + 1;
  __syncthreads();
  Real* dst = coef + c0 * REC;
  // element e = l REC + r of the run; (l, r) advance by a constant step
  constexpr int DL = NT / REC, DR = NT % REC;
  int l = threadIdx.x / REC, r = threadIdx.x - (threadIdx.x / REC) * REC;
  for (int e = threadIdx.x; e < nv * REC; e += NT) {
    dst[e] = smem[l * PITCH + r];
    l += DL;
    r += DR;
    if (r >= REC) {
      r -= REC;
      ++l;
    }
  }
}
template <typename Real>
__device__ __forceinline__ void write_block_records(Real* smem, const Real res[10], bool live, int lane, int v,
                                                    int nv, Real* __restrict__ coef, int64_t c0) {
  __syncthreads();
  if (live) stage_record<Real>(smem, res, lane, v);
  flush_records<Real, kRThreads>(smem, nv, coef, c0);
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
// cells with one warp per conservative variable, as k_recon, or ("paired")
// three warps, two of which serve two variables each, so that every row a
// thread reads from shared memory feeds two variables.  The block's
// binary32 reconstruction record (pseudo-inverse rows, second moments, 1/h
// and sub-stencil positions, rounded once when the mesh was made, as
// cvt<float> rounds them: see rec32_bytes) is contiguous in memory, so warp 0
// moves it into shared memory with a few bulk asynchronous copies completed
// on an mbarrier, while every thread gathers stencil neighbours' states (one
// 32-byte record of all five variables per neighbour) into shared memory and
// its own cell's state into a register.  The arithmetic and its order are
// those of k_recon.
// "Phased": where it lets more blocks share an SM, the first copy stops
// before the linear sub-stencil rows; once every warp has formed its
// quadratic coefficients, a second copy puts the linear rows over the
// quadratic ones, so the tile needs 9K (not 9K + 3 M KM) inverse rows.
// Blocks per SM: as many as shared memory and registers (about 56 per thread
// on tetrahedra, 66 on hexahedra, 86 at stencil size 26, 80 paired, measured
// with ptxas) allow; the kernel's launch bounds ask the compiler for that
// count.
template <int K, int M, int KM, bool PAIR = false>
struct ReconSmemF {
  static_assert(M * KM % 4 == 0 && 3 * M * KM <= 9 * K, "record layout");
  // threads per block: one warp per variable, or (PAIR) three warps, the
  // first two serving two variables each (0 and 1, 2 and 3), the third one
  static constexpr int NT = PAIR ? 3 * kRC : kRThreads;
  static constexpr int R0 = 9 * K, R1 = M * 3 * KM;  // quadratic and linear rows
  static constexpr int RG = R0;                       // row of the first second moment
  static constexpr int RP = R0 + 7;                   // first row of sub-stencil positions
  static constexpr int RL = RP + M * KM / 4;          // first linear row in the record
  static constexpr size_t rec = (size_t)rec32_bytes(K, M, KM);  // the block's record
  static constexpr size_t head = (size_t)RL * 128;               // the record up to the linear rows
  static constexpr size_t nbr = sizeof(float) * 5 * K * kRC;     // neighbour states [5][K][kRC]
  // blocks per SM: 228 KB of shared memory, 1 KB reserved per block; registers
  static constexpr int fit(size_t b) { return (int)(233472 / (b + 1024)); }
  static constexpr int reg_cap = 65536 / (NT * (PAIR ? 80 : (M == 4 ? 56 : (K <= 24 ? 66 : 86))));
  static constexpr int cap(int b) { return b < reg_cap ? b : reg_cap; }
  static constexpr bool phased = cap(fit(head + nbr)) > cap(fit(rec + nbr));
  static constexpr size_t tile = phased ? head : rec;
  static constexpr size_t bytes = tile + nbr;
  static constexpr int blocks = cap(fit(bytes));
  static constexpr int LB = phased ? 0 : RL;  // tile row of the first linear row
  // phased: the quadratic coefficients d < DS read rows 0 .. DS K - 1, which
  // the linear rows then replace while the coefficients d >= DS are formed
  // (hexahedra: DS even, for their pairs of rows).  Measured: the K = 24
  // hexahedral shell's reconstruction 2.7% faster; paired blocks copy after
  // all nine (DS = 9).
  static constexpr int ds_min() {
    int d = 0;
    while (d * K < R1) ++d;
    return d;
  }
  static constexpr int DS = (!phased || PAIR) ? 9 : (M == 8 ? (ds_min() + 1) / 2 * 2 : ds_min());
  static_assert(DS * K >= R1 && DS <= 9, "the linear rows fit in the rows already read");
  // copies in pieces of at most 4 KB, one per lane of warp 0
  static constexpr int piece = 4096;
  static_assert(rec % 16 == 0 && (rec + piece - 1) / piece <= 32, "bulk copies of the record");
  static_assert(tile >= sizeof(float) * kRC * (kCoefRec32 + 1), "the output staging fits in the tile");
};

// The least-squares polynomials of one (variable, cell) thread from a
// binary32 tile of inverse rows ([rows][kRC]) and the block's neighbour
// states snbr ([5][K][kRC]) less the cell's own qv: the quadratic (a, 9
// coefficients from tile rows 0 .. 9K-1, in ranges of d so that a phased
// block can start its second copy part way through) and the linear ones (b,
// 3 per sub-stencil from rows LB .. LB + 3 M KM - 1, members at positions
// ssub).  The operation order is that of k_recon.  On hexahedra, pairs of
// output rows advance together in packed binary32 FMAs (two independent
// round-to-nearest FMAs per instruction: the same results); measured 8%
// faster there and 5% slower on tetrahedra.
// Stencil differences of variable v of this thread's cell (own state qv).
template <int K>
__device__ __forceinline__ void rs_diff(const float* snbr, float qv, int v, int lane, float dq[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) dq[k] = snbr[(v * K + k) * kRC + lane] - qv;
}
// Quadratic coefficients a[d], D0 <= d < D1, from tile rows d K .. d K + K - 1.
template <int K, int M, int D0, int D1>
__device__ __forceinline__ void rs_quad_rows(const float* tile, const float dq[K], int lane, float a[9]) {
  auto row = [&](int r) -> float { return tile[r * kRC + lane]; };
  if constexpr (M == 8) {
    static_assert(D0 % 2 == 0, "pairs of rows start at even d");
    float2 dq2[K];
#pragma unroll
    for (int k = 0; k < K; ++k) dq2[k] = make_float2(dq[k], dq[k]);
#pragma unroll
    for (int d = D0; d + 1 < D1; d += 2) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < K; ++k) acc = __ffma2_rn(make_float2(row(d * K + k), row((d + 1) * K + k)), dq2[k], acc);
      a[d] = acc.x;
      a[d + 1] = acc.y;
    }
    if constexpr ((D1 - D0) % 2 == 1) {
      float sacc = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) sacc = fmaf(row((D1 - 1) * K + k), dq[k], sacc);
      a[D1 - 1] = sacc;
    }
  } else {
#pragma unroll
    for (int d = D0; d < D1; ++d) {
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

// rs_quad_rows and rs_linear for two variables va, vb of one cell (own
// states qa, qb): each tile row is read once and feeds both variables'
// chains in one packed binary32 FMA (two independent round-to-nearest FMAs:
// the results of the one-variable forms, in their order).
template <int K>
__device__ __forceinline__ void rs_diff2(const float* snbr, float qa, float qb, int va, int vb, int lane,
                                         float2 dq[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k)
    dq[k] = make_float2(snbr[(va * K + k) * kRC + lane] - qa, snbr[(vb * K + k) * kRC + lane] - qb);
}
template <int K, int D0, int D1>
__device__ __forceinline__ void rs_quad_rows2(const float* tile, const float2 dq[K], int lane, float a[9],
                                              float a2[9]) {
  auto row = [&](int r) -> float { return tile[r * kRC + lane]; };
#pragma unroll
  for (int d = D0; d < D1; ++d) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float x = row(d * K + k);
      acc = __ffma2_rn(make_float2(x, x), dq[k], acc);
    }
    a[d] = acc.x;
    a2[d] = acc.y;
  }
}

template <int K, int M, int KM, int LB>
__device__ __forceinline__ void rs_linear2(const float* tile, const float* snbr, const uint8_t* ssub, float qa,
                                           float qb, int va, int vb, int lane, float b[M][3], float b2[M][3]) {
  auto row = [&](int r) -> float { return tile[r * kRC + lane]; };
#pragma unroll
  for (int s = 0; s < M; ++s) {
    float2 x[KM];
#pragma unroll
    for (int r = 0; r < KM; ++r) {
      const int k = ssub[(s * KM + r) * kRC + lane];
      x[r] = make_float2(snbr[(va * K + k) * kRC + lane] - qa, snbr[(vb * K + k) * kRC + lane] - qb);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int r = 0; r < KM; ++r) {
        const float y = row(LB + (s * 3 + d) * KM + r);
        acc = __ffma2_rn(make_float2(y, y), x[r], acc);
      }
      b[s][d] = acc.x;
      b2[s][d] = acc.y;
    }
  }
}

// Bytes [off, off + len) of a block's record (rec) to shared memory at dst,
// completing on bar; called by warp 0.
__device__ __forceinline__ void rec_copy(unsigned char* dst, const char* rec, size_t off, size_t len, uint64_t* bar) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    // shared memory read and written by the generic proxy before (earlier
    // phase, earlier tile of a persistent launch) is overwritten by the copies
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, (uint32_t)len);
  }
  __syncwarp();
  const size_t o = (size_t)lane * 4096;
  if (o < len) bulk_g2s(dst + o, rec + off + o, (uint32_t)(len - o < 4096 ? len - o : 4096), bar);
}

// One block of k_recon_rs at cells c0 .. c0 + 31.  bar: the block's
// mbarrier (initialised, count 1); phase: the parity of bar's next phase,
// advanced by each copy this call waits for.  Returns false, with
// FLAG_TIMEOUT set, if a copy did not land within the bounded wait.
template <int K, int M, int KM, bool COH = false, bool PAIR = false>
__device__ __forceinline__ bool recon_rs_block(const DevMesh& m, const DevParams& P, const float* __restrict__ Qf,
                                               float* __restrict__ coef, Control* __restrict__ ctl, int64_t c0,
                                               unsigned char* smem_raw, uint64_t* bar, uint32_t& phase) {
  using S = ReconSmemF<K, M, KM, PAIR>;
  constexpr int NW = S::NT / 32;  // warps
  float* tile = reinterpret_cast<float*>(smem_raw);                  // [rows][kRC]
  const uint8_t* ssub = smem_raw + (size_t)S::RP * 128;              // [M*KM][kRC]
  float* snbr = reinterpret_cast<float*>(smem_raw + S::tile);        // [5][K][kRC]
  const char* rec = reinterpret_cast<const char*>(m.rec32) + (size_t)(c0 / kRC) * S::rec;
  const int64_t nc = m.nc;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int nv = nc - c0 < kRC ? (int)(nc - c0) : kRC;  // cells of this block
  const bool live = lane < nv;
  // the thread's variable va, and with PAIR in warps 0 and 1 also vb = va + 1
  const int va = PAIR ? 2 * w : w, vb = va + 1;
  const bool two = PAIR && w < 2;  // uniform over the warp
  // a bounded wait for the copies of the current phase; false: flag, one
  // more bounded wait for the copies in flight, and leave (only a stalled
  // memory system explains a block's own copies, under 40 KB, not landing
  // within about a second; the host reports HGKS_ETIMEOUT)
  auto landed = [&]() {
    const bool ok = __syncthreads_and(mbar_wait_bounded(bar, phase));
    if (!ok) {
      if (t == 0) atomicOr(&ctl->flags, FLAG_TIMEOUT);
      mbar_wait_bounded(bar, phase);
    }
    phase ^= 1u;
    return ok;
  };
  // 1. the block's record (the head only, phased)
  if (w == 0) rec_copy(smem_raw, rec, 0, S::tile, bar);
  // 2. stencil neighbours' states and the cell's own (overlap the copies).
  // Thread (w, lane) fetches entries k = w, w + NW, ... of column `lane`.
  constexpr int NE = (K + NW - 1) / NW;
  int32_t jn[NE];
#pragma unroll
  for (int i = 0; i < NE; ++i) {
    const int k = w + NW * i;
    jn[i] = (k < K && live) ? __ldcs(m.sten + (int64_t)k * nc + c0 + lane) : 0;
  }
  const float qv = live ? ldro<COH>(Qf + 8 * (c0 + lane) + va) : 0.f;
  const float qv2 = (two && live) ? ldro<COH>(Qf + 8 * (c0 + lane) + vb) : 0.f;
  float4 qa[NE];
  float qb[NE];
#pragma unroll
  for (int i = 0; i < NE; ++i) {
    if (w + NW * i < K && live) {
      qa[i] = ldro<COH>(reinterpret_cast<const float4*>(Qf + 8 * (int64_t)jn[i]));
      qb[i] = ldro<COH>(Qf + 8 * (int64_t)jn[i] + 4);
    }
  }
#pragma unroll
  for (int i = 0; i < NE; ++i) {
    const int k = w + NW * i;
    if (k < K && live) {
      float* dst = snbr + k * kRC + lane;
      dst[0] = qa[i].x;
      dst[K * kRC] = qa[i].y;
      dst[2 * K * kRC] = qa[i].z;
      dst[3 * K * kRC] = qa[i].w;
      dst[4 * K * kRC] = qb[i];
    }
  }
  // 3. the copies have landed and the neighbour states are in place
  if (!landed()) return false;
  constexpr int DS = S::DS;
  float a[9], b[M][3], a2[9], b2[M][3];
  if constexpr (PAIR) {
    static_assert(DS == 9, "paired blocks copy the linear rows after all quadratic rows");
    if (live) {
      if (two) {
        float2 dq[K];
        rs_diff2<K>(snbr, qv, qv2, va, vb, lane, dq);
        rs_quad_rows2<K, 0, 9>(tile, dq, lane, a, a2);
      } else {
        float dq[K];
        rs_diff<K>(snbr, qv, va, lane, dq);
        rs_quad_rows<K, M, 0, 9>(tile, dq, lane, a);
      }
    }
    if constexpr (S::phased) {
      __syncthreads();  // every warp has read its quadratic rows
      if (w == 0) rec_copy(smem_raw, rec, S::head, S::rec - S::head, bar);
    }
  } else {
    float dq[K];
    if (live) {
      rs_diff<K>(snbr, qv, va, lane, dq);
      rs_quad_rows<K, M, 0, DS>(tile, dq, lane, a);
    }
    if constexpr (S::phased) {
      __syncthreads();  // every warp has read rows 0 .. DS K - 1
      if (w == 0) rec_copy(smem_raw, rec, S::head, S::rec - S::head, bar);
    }
    if (live) rs_quad_rows<K, M, DS, 9>(tile, dq, lane, a);
  }
  if constexpr (S::phased) {
    if (!landed()) return false;
  }
  float res[10], res2[10];
  if (live) {
    if (two) rs_linear2<K, M, KM, S::LB>(tile, snbr, ssub, qv, qv2, va, vb, lane, b, b2);
    else rs_linear<K, M, KM, S::LB>(tile, snbr, ssub, qv, va, lane, b);
    float mi[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) mi[q] = tile[(S::RG + q) * kRC + lane];
    const float hi = tile[(S::RG + 6) * kRC + lane];
    const float glin = P.f_glin, g0 = 1.f - float(M) * glin, eps = P.f_eps;
    recon_finish<float, M>(a, b, qv, mi, hi, glin, g0, eps, res);
    if (two) recon_finish<float, M>(a2, b2, qv2, mi, hi, glin, g0, eps, res2);
  }
  __syncthreads();  // every warp is done with the tile
  if (live) {
    stage_record<float>(tile, res, lane, va);
    if (two) stage_record<float>(tile, res2, lane, vb);
  }
  flush_records<float, S::NT>(tile, nv, coef, c0);
  return true;
}

// Paired variables (three warps) on tetrahedra, measured: the 48^3 x 6
// reconstruction 0.325 against 0.359 ms per step (80 registers, 8 blocks of
// 96 per SM); on hexahedra the pairs need 110 registers and run 10% (K = 24
// shell) and 14% (K = 26 hybrid shell) slower, so they keep one warp per
// variable.
template <int M>
constexpr bool recon_pair() { return M == 4; }
template <int K, int M, int KM, bool PAIR>
__global__ void __launch_bounds__(ReconSmemF<K, M, KM, PAIR>::NT, ReconSmemF<K, M, KM, PAIR>::blocks)
    k_recon_rs(DevMesh m, DevParams P, const float* __restrict__ Qf, float* __restrict__ coef,
               Control* __restrict__ ctl) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  if (m.nmesh == 1 && ctl->dt == 0.0) return;  // uniform over the grid (a batch computes every member)
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t phase = 0;
  recon_rs_block<K, M, KM, false, PAIR>(m, P, Qf, coef, ctl, (int64_t)blockIdx.x * kRC, smem_raw, &bar, phase);
}

}  // namespace
}  // namespace hgks

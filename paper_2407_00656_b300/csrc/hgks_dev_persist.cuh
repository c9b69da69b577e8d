// hgks_dev_persist.cuh -- the persistent cooperative kernel: n whole steps
// in one launch, the phases separated by bounded grid-wide barriers.
#pragma once

#include "hgks_dev_recon.cuh"
#include "hgks_dev_flux.cuh"
#include "hgks_dev_update.cuh"

namespace hgks {
namespace {
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
  // mbarrier of the binary32 reconstruction's record copies and the parity
  // of its next phase
  __shared__ __align__(8) uint64_t rbar;
  uint32_t rphase = 0;
  if (F32) {
    if (threadIdx.x == 0) mbar_init(&rbar, 1);
    __syncthreads();
  }
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
          if constexpr (F32) {
            // a record that never arrived ends the launch (the flag is set;
            // the other blocks' barrier waits run out)
            if (!recon_rs_block<K, M, KM, true>(m, P, w.Qf, coef, ctl, t * kRC, smem_raw, &rbar, rphase)) return;
          } else {
            recon_block<Real, double, K, M, KM, false, true>(m, P, Qin, coef, ctl, t * kRC, smem_raw);
          }
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

}  // namespace
}  // namespace hgks

// hgks_noalloc.cu -- the CFL time step of a caller-held state, computed with
// no allocation at all.
//
// Some callers cannot allocate device memory at the moment they need the time
// step: hosts whose device memory is owned by another allocator that forbids
// foreign cudaMalloc/cudaFree calls (a pool sized up front, a framework that
// accounts for every byte), and loops that cannot accept cudaFree's implicit
// device-wide synchronisation.  hgks_cfl_dt_noalloc serves them: it is a
// variant of the solver's time-step reduction whose per-block partial minima
// live in a fixed, file-scope device array instead of solver memory.  The
// bound is always evaluated in binary64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "hgks.h"
#include "hgks_internal.h"

namespace {

constexpr int kThreads = 256;
// One partial minimum per block of kThreads cells: 16384 partials (128 KiB)
// bound the cell count at HGKS_NOALLOC_MAX_CELLS = 16384 * 256 = 4,194,304.
constexpr int kMaxPartials = 16384;
static_assert((int64_t)kMaxPartials * kThreads == HGKS_NOALLOC_MAX_CELLS, "limit mismatch");

// The scratch.  Every GPU that loads the library holds it until the process
// exits; all calls on a device share it.
static __device__ __align__(256) double g_partials[kMaxPartials];

// Device addresses of g_partials, looked up once per device (host code may
// not use the symbol itself: on the host it names a stand-in, not device memory).
constexpr int kMaxDevices = 64;
double* g_addr[kMaxDevices] = {nullptr};
std::mutex g_mu;

struct DtParams {
  double gamma, cfl, mu_ref, T_ref, visc_exp;
};

// Local bound h/(|U| + c), and with viscosity also rho h^2/(2 mu); T = p/rho.
// NaN for a state that has no bound: a non-finite value, or a non-positive
// density or pressure.
__device__ __forceinline__ double local_bound(const double* q, double h, const DtParams& P) {
  const double ri = 1.0 / q[0];
  const double u = q[1] * ri, v = q[2] * ri, w = q[3] * ri;
  const double u2 = u * u + v * v + w * w;
  const double p = (P.gamma - 1.0) * (q[4] - 0.5 * q[0] * u2);
  if (!(q[0] > 0.0) || !(p > 0.0) || !isfinite(u2) || !isfinite(p)) return NAN;
  double b = h / (sqrt(u2) + sqrt(P.gamma * p * ri));
  if (P.mu_ref > 0.0) {
    const double mu = P.visc_exp != 0.0 ? P.mu_ref * pow(p * ri / P.T_ref, P.visc_exp) : P.mu_ref;
    b = fmin(b, q[0] * h * h / (2.0 * mu));
  }
  return b;
}

// Minimum that keeps a NaN (fmin would drop it).
__device__ __forceinline__ double min_nan(double a, double b) { return (a != a || b != b) ? NAN : fmin(a, b); }

__device__ __forceinline__ double block_min(double v) {
  __shared__ double red[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v = min_nan(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double x = INFINITY;
  if (threadIdx.x < 32) {
    x = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : INFINITY;
    for (int o = 16; o > 0; o >>= 1) x = min_nan(x, __shfl_xor_sync(0xffffffffu, x, o));
  }
  return x;  // valid in thread 0
}

// Phase 1: block b writes the minimum bound of its cells to partial[b].
__global__ void __launch_bounds__(kThreads) k_dt_partials(const double* __restrict__ q, const double* __restrict__ hdt,
                                                          int64_t n, DtParams P, double* __restrict__ partial) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  double b = INFINITY;
  if (i < n) b = local_bound(q + 5 * i, hdt[i], P);
  b = block_min(b);
  if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

// Phase 2: one block reduces the nb partials and writes cfl * min (NaN if
// any cell had no bound).
__global__ void __launch_bounds__(kThreads) k_dt_final(const double* __restrict__ partial, int nb, double cfl,
                                                       double* __restrict__ dt_out) {
  double b = INFINITY;
  for (int k = threadIdx.x; k < nb; k += kThreads) b = min_nan(b, partial[k]);
  b = block_min(b);
  if (threadIdx.x == 0) *dt_out = cfl * b;
}

int fail(int code, const std::string& m) {
  hgks::set_last_error(m);
  return code;
}

}  // namespace

extern "C" {

int hgks_cfl_dt_noalloc(const double* q, const double* hdt, int64_t n_cells, const hgks_params* params,
                        double* dt_out, void* stream) {
  if (!q || !hdt || !params || !dt_out) return fail(HGKS_EINVAL, "NULL argument");
  if (n_cells <= 0) return fail(HGKS_EINVAL, "n_cells must be positive");
  if (n_cells > HGKS_NOALLOC_MAX_CELLS)
    return fail(HGKS_EINVAL, "n_cells " + std::to_string(n_cells) + " exceeds the fixed scratch limit of " +
                                 std::to_string((long long)HGKS_NOALLOC_MAX_CELLS) + " cells");
  const int prc = hgks::check_params(params);  // the same checks as hgks_init
  if (prc) return prc;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(HGKS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(HGKS_EINVAL, "device ordinal out of range");
  double* partial = nullptr;
  {
    // set-up once per device, with that device current
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      e = cudaGetSymbolAddress(reinterpret_cast<void**>(&g_addr[dev]), g_partials);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        return fail(HGKS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    partial = g_addr[dev];
  }
  const DtParams P{params->gamma, params->cfl, params->mu_ref, params->T_ref, params->visc_exp};
  const int nb = (int)((n_cells + kThreads - 1) / kThreads);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // every partial that phase 2 reads is written by phase 1 of the same call,
  // so the scratch needs no clearing between calls
  k_dt_partials<<<nb, kThreads, 0, s>>>(q, hdt, n_cells, P, partial);
  k_dt_final<<<1, kThreads, 0, s>>>(partial, nb, params->cfl, dt_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(HGKS_ECUDA, std::string("launching the time-step reduction: ") + cudaGetErrorString(e));
  return HGKS_OK;
}

}  // extern "C"

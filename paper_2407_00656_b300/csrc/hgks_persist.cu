// hgks_persist.cu -- host launcher of the persistent cooperative step kernel.
#include "hgks_dev_persist.cuh"

namespace hgks {
namespace {

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

}  // namespace

cudaError_t launch_persistent(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, int n,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return precision == 1 ? persist_any<float>(m, p, w, n, s, false) : persist_any<double>(m, p, w, n, s, false);
}

void prepare_persist(const DevMesh& m, int precision) {
  if (precision == 1) persist_any<float>(m, DevParams{}, DevWork{}, 0, 0, true);
  else persist_any<double>(m, DevParams{}, DevWork{}, 0, 0, true);
}

}  // namespace hgks

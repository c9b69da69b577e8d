// hgks_recon.cu -- host launchers of the WENO reconstruction (Section 2.3):
// the kernel variant and the compiled stencil shape of a mesh.
#include "hgks_dev_recon.cuh"

namespace hgks {
namespace {

// Variants: binary64, 0 = rows staged by bulk asynchronous copies, 1 = rows
// read directly; binary32, 0 = k_recon_rs, 1 = rows staged by bulk
// asynchronous copies.
template <typename Real, typename QT, int K, int M, int KM>
void recon_launch(const DevMesh& m, const DevParams& p, const QT* Q, Real* coef, Control* ctl, cudaStream_t s,
                  bool prep) {
  using S = ReconSmem<Real, K, M, KM>;
  const unsigned nb = (unsigned)((m.nc + kRC - 1) / kRC);
  if constexpr (sizeof(Real) == 4) {
    constexpr bool PAIR = recon_pair<M>();
    using SF = ReconSmemF<K, M, KM, PAIR>;
    if (prep) {
      cudaFuncSetAttribute(k_recon<Real, QT, K, M, KM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)S::bytes);
      cudaFuncSetAttribute(k_recon_rs<K, M, KM, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SF::bytes);
      return;
    }
    if (p.recon_variant == 1) k_recon<Real, QT, K, M, KM, true><<<nb, kRThreads, S::bytes, s>>>(m, p, Q, coef, ctl);
    else k_recon_rs<K, M, KM, PAIR><<<nb, SF::NT, SF::bytes, s>>>(m, p, Q, coef, ctl);
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

template <typename Real, typename QT>
void recon_any(const DevMesh& m, const DevParams& p, const QT* Q, Real* coef, Control* ctl, cudaStream_t s,
               bool prep = false) {
  if (m.M == 4) recon_dispatch<Real, QT, 4, 6>(m, p, Q, coef, ctl, s, prep);
  else recon_hex<Real, QT>(m, p, Q, coef, ctl, s, prep);
}

}  // namespace

bool stencil_supported(int nfc, int K) {
  if (nfc == 4) return K >= 12 && K <= 16;
  // hexahedra 18-24; hybrid hex/prism meshes reach 26
  return K == 18 || K == 20 || K == 22 || K == 24 || K == 26;
}

void launch_recon(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, const double* Q,
                  cudaStream_t s) {
  if (precision == 1) recon_any<float, float>(m, p, w.Qf, static_cast<float*>(w.coef), w.ctl, s);
  else recon_any<double, double>(m, p, Q, static_cast<double*>(w.coef), w.ctl, s);
}

void prepare_recon(const DevMesh& m, int precision) {
  if (precision == 1) recon_any<float, float>(m, DevParams{}, nullptr, nullptr, nullptr, 0, true);
  else recon_any<double, double>(m, DevParams{}, nullptr, nullptr, nullptr, 0, true);
}

}  // namespace hgks

// hgks_flux.cu -- host launchers of the face flux (Section 2.1, Eq. flux):
// the kernel variant, Gauss points per face and viscosity of a mesh.
#include "hgks_dev_flux.cuh"

namespace hgks {
namespace {

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

}  // namespace

void launch_flux(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, cudaStream_t s) {
  if (precision == 1) flux_any<float>(m, p, static_cast<const float*>(w.coef), static_cast<float*>(w.Fs), w.ctl, s);
  else flux_any<double>(m, p, static_cast<const double*>(w.coef), static_cast<double*>(w.Fs), w.ctl, s);
}

}  // namespace hgks

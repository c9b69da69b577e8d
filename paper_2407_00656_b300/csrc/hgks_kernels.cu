// hgks_kernels.cu -- one HGKS step (Algorithm 2) on the device:
//
//   k_finalize    time step from the device-side minimum bound (Algorithm 2,
//                 "calculate time step"), clipped to t_end
//   k_ghost       boundary ghost cell averages (Algorithm 1 ghost cells)
//   reconstruction (hgks_recon.cu): third-order WENO (Section 2.3, Eqs. polys,
//                 weno), one combined quadratic per cell and variable
//   flux (hgks_flux.cu): time-dependent gas-kinetic flux at the face Gauss
//                 points (Section 2.1, Eq. flux; Section 2.2 linear-in-time fit)
//   k_update1/2   gather of the face fluxes per cell (no atomics) and the two
//                 S2O4 stages (Section 2.2); stage 2 also produces the next
//                 step bound and the non-finite flag
//   persistent launch (hgks_persist.cu): n whole steps in one cooperative
//                 kernel, the phases above separated by bounded barriers
#include "hgks_dev_update.cuh"

namespace hgks {
namespace {

template <typename Real>
void stage_pair(const DevMesh& m, const DevParams& p, const DevWork& w, bool mixed, cudaStream_t s,
                const StepEvents* ev) {
  Real* Fs = static_cast<Real*>(w.Fs);
  const unsigned nbc = blocks(m.nc);
  float* Qf = mixed ? w.Qf : nullptr;
  auto mark = [&](int i) { if (ev) cudaEventRecord(ev->ev[i], s); };
  {
    // stage 1 on Q^n
    Range r1("stage 1: ghosts, reconstruction, flux, update");
    if (m.ng) k_ghost<<<blocks(m.ng), kBlock, 0, s>>>(m, p, w.Q, Qf, w.ctl);
    launch_recon(m, p, w, mixed ? 1 : 0, w.Q, s);
    mark(2);
    launch_flux(m, p, w, mixed ? 1 : 0, s);
    mark(3);
    if (m.nfc == 4) k_update1<Real, 4><<<nbc, kBlock, 0, s>>>(m, Fs, w.Q, w.Qs, w.R, Qf, w.ctl);
    else k_update1<Real, 6><<<nbc, kBlock, 0, s>>>(m, Fs, w.Q, w.Qs, w.R, Qf, w.ctl);
    mark(4);
  }
  {
    // stage 2 on Q*
    Range r2("stage 2: ghosts, reconstruction, flux, update");
    if (m.ng) k_ghost<<<blocks(m.ng), kBlock, 0, s>>>(m, p, w.Qs, Qf, w.ctl);
    launch_recon(m, p, w, mixed ? 1 : 0, w.Qs, s);
    mark(5);
    launch_flux(m, p, w, mixed ? 1 : 0, s);
    mark(6);
    if (m.nfc == 4) k_update2<Real, 4><<<nbc, kBlock, 0, s>>>(m, p, Fs, w.Q, w.R, Qf, w.ctl);
    else k_update2<Real, 6><<<nbc, kBlock, 0, s>>>(m, p, Fs, w.Q, w.R, Qf, w.ctl);
    mark(7);
  }
}

}  // namespace

void launch_round32(const DevMesh& m, cudaStream_t s) {
  const int64_t n3 = (int64_t)3 * m.G * m.nf, n1 = (int64_t)m.G * m.nf;
  if (n3 > 0) {
    k_round32<<<blocks(n3), kBlock, 0, s>>>(m.fdl, const_cast<float*>(m.fdl32), n3);
    k_round32<<<blocks(n3), kBlock, 0, s>>>(m.fdr, const_cast<float*>(m.fdr32), n3);
    k_round32<<<blocks(n3), kBlock, 0, s>>>(m.fn, const_cast<float*>(m.fn32), n3);
    k_round32<<<blocks(n1), kBlock, 0, s>>>(m.fw, const_cast<float*>(m.fw32), n1);
  }
  const int64_t nr = rec32_bytes(m.K, m.M, m.KM) / 4 * (m.ncp / 32);
  if (nr > 0) k_rec32<<<blocks(nr), kBlock, 0, s>>>(m, const_cast<float*>(m.rec32));
}

void launch_test_erfcx(const double* x, double* y, int64_t n, cudaStream_t s) {
  if (n > 0) k_test_erfcx<<<blocks(n), kBlock, 0, s>>>(x, y, n);
}

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
    launch_recon(m, p, w, precision, w.Q, s);
    launch_flux(m, p, w, precision, s);
  }
  cudaEventRecord(e1, s);
  float ms = -1.f;
  if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return reps > 0 && ms >= 0.f ? ms / reps : -1.f;
}

void prepare_kernels(const DevMesh& m, int precision) {
  prepare_recon(m, precision);
  prepare_persist(m, precision);
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
  Range range("S2O4 step");
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
  launch_recon(m, p, w, precision, w.Q, s);
  launch_flux(m, p, w, precision, s);
  if (mixed) {
    if (m.nfc == 4) k_operator<float, 4><<<blocks(m.nc), kBlock, 0, s>>>(m, static_cast<float*>(w.Fs), L, dL);
    else k_operator<float, 6><<<blocks(m.nc), kBlock, 0, s>>>(m, static_cast<float*>(w.Fs), L, dL);
  } else {
    if (m.nfc == 4) k_operator<double, 4><<<blocks(m.nc), kBlock, 0, s>>>(m, static_cast<double*>(w.Fs), L, dL);
    else k_operator<double, 6><<<blocks(m.nc), kBlock, 0, s>>>(m, static_cast<double*>(w.Fs), L, dL);
  }
}

}  // namespace hgks

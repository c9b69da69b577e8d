// hgks_internal.h -- device-side data layout shared by the kernels and the
// solver lifecycle code of libhgks.
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "hgks.h"

namespace hgks {

// Read-only mesh arrays in device memory (layouts as in mesh_builder.h).
struct DevMesh {
  int64_t nc, nf, ng, nce;  // cells, faces, ghosts, cells + ghosts
  int64_t ncp;              // row pitch of pinv0, subidx, pinvm (nc rounded up to 32)
  int nmesh;                // member meshes of a batch (1 for a single mesh)
  const int32_t* cmesh;     // [nc] member of each cell, or nullptr when nmesh == 1
  const int32_t* perm;      // [nc] caller index of each cell within its member mesh
  int K, M, KM, G, nfc;
  const double* volinv;   // [nc] 1/|cell|
  const double* hdt;      // [nc]
  const double* hinv;     // [nc]
  const double* mom;      // [6][nc] scaled central second moments
  const int32_t* sten;    // [K][nc]
  const double* pinv0;    // [9K][ncp]
  const uint8_t* subidx;  // [M*KM][ncp]
  const double* pinvm;    // [M*3*KM][ncp]
  const int32_t* cface;   // [nfc][nc]
  const int32_t* gsrc;    // [ng]
  const int32_t* gtag;    // [ng]
  const double* gnrm;     // [3][ng]
  const int32_t* fown;    // [nf]
  const int32_t* fnbr;    // [nf]
  const double* fdl;      // [3G][nf]
  const double* fdr;      // [3G][nf]
  const double* fn;       // [3G][nf]
  const double* fw;       // [G][nf]
  // binary32 roundings of fdl, fdr, fn and fw (as cvt<float> rounds them),
  // read by the binary32 flux instead of converting on every launch
  const float* fdl32;     // [3G][nf]
  const float* fdr32;     // [3G][nf]
  const float* fn32;      // [3G][nf]
  const float* fw32;      // [G][nf]
  // binary32 reconstruction records, one per block of 32 consecutive cells
  // (layout: rec32_bytes), read by the binary32 reconstruction
  const float* rec32;     // [ncp/32][rec32_bytes(K, M, KM) / 4]
};

// Binary32 reconstruction record of a block of 32 consecutive cells: the
// binary32 roundings (cvt<float>) of the block's inputs to the
// reconstruction, contiguous so that bulk copies move them.  Rows of 32
// 4-byte values, one per cell of the block (zero past the last cell): the
// 9K rows of pinv0, the six second moments, 1/h, the M KM rows of
// sub-stencil positions (one byte per cell, so M KM / 4 rows), then the
// 3 M KM rows of pinvm.  A record's size is a multiple of 128 bytes.
#ifdef __CUDACC__
#define HGKS_HD __host__ __device__
#else
#define HGKS_HD
#endif
HGKS_HD constexpr int rec32_rows(int K, int M, int KM) { return 9 * K + 7 + M * KM / 4 + 3 * M * KM; }
HGKS_HD constexpr int64_t rec32_bytes(int K, int M, int KM) { return (int64_t)rec32_rows(K, M, KM) * 128; }

// Physical and numerical parameters as the kernels use them.
struct DevParams {
  double gamma, Kint, mu_ref, T_ref, visc_exp, Pr, cfl, tau_c, eps, glin;
  double qinf[5];
  double kq, kqi;  // (K+3)/4 and its reciprocal
  double prfix;    // 1/Pr - 1 (Prandtl-number fix of the energy flux)
  // binary32 copies, rounded on the host, for the mixed-precision kernels
  // (keeps binary64 -> binary32 conversions off the device's FP64 pipe)
  float f_gamma, f_Kint, f_kq, f_kqi, f_mu_ref, f_T_ref, f_visc_exp, f_Pr, f_prfix, f_tau_c, f_eps, f_glin;
  float f_qinf[5];
  int viscous;  // 1 when mu_ref > 0 or tau_c > 0 (collision time may be non-zero)
  // kernel variants chosen by the autotuner:
  int flux_variant;   // 0: one thread per face, 1: one thread per Gauss point
  int recon_variant;  // 0: rows staged by bulk async copies, 1: rows read directly
  long long bar_cycles;  // clock cycles a grid barrier of the persistent launch waits before giving up
};

// Default wait of a grid barrier: 2^31 cycles, about a second at 2 GHz.
constexpr long long kBarrierCycles = 1LL << 31;

// Fill kq, kqi and the binary32 copies of the parameters.
inline void fill_float_params(DevParams& p) {
  p.kq = 0.25 * (p.Kint + 3.0);
  p.kqi = 4.0 / (p.Kint + 3.0);
  p.prfix = 1.0 / p.Pr - 1.0;
  p.f_gamma = (float)p.gamma;
  p.f_Kint = (float)p.Kint;
  p.f_kq = (float)(0.25 * (p.Kint + 3.0));
  p.f_kqi = (float)(4.0 / (p.Kint + 3.0));
  p.f_mu_ref = (float)p.mu_ref;
  p.f_T_ref = (float)p.T_ref;
  p.f_visc_exp = (float)p.visc_exp;
  p.f_Pr = (float)p.Pr;
  p.f_prfix = (float)p.prfix;
  p.f_tau_c = (float)p.tau_c;
  p.f_eps = (float)p.eps;
  p.f_glin = (float)p.glin;
  for (int i = 0; i < 5; ++i) p.f_qinf[i] = (float)p.qinf[i];
}

// Reals per record of the reconstruction coefficients (one record per cell:
// 5 variables x 10 coefficients) and of the face fluxes (one record per face:
// F then dF/dt, 5 each).  Binary32 records are padded to a multiple of 16
// bytes so that they can be moved with 16-byte vector accesses.
constexpr int kCoefRec64 = 50, kCoefRec32 = 52;
constexpr int kFluxRec64 = 10, kFluxRec32 = 12;

// Step control block in device memory.
struct Control {
  double t;          // time reached by the queued steps
  double dt;         // step size of the step in flight (0: no-op step)
  double t_end;      // > 0: clip steps to land on t_end
  double dt_fixed;   // > 0: use instead of the CFL step
  unsigned long long dtmin_bits;  // min over cells of the local step bound (bits of a positive double)
  long long steps;   // steps taken since init/write
  int flags;         // bit 0: a non-finite cell average was produced
  int pad;
};

// FLAG_TIMEOUT: a reconstruction block's wait for its bulk copies ran out;
// FLAG_BAR_TIMEOUT: a grid barrier of the persistent launch ran out.
enum { FLAG_NONFINITE = 1, FLAG_TIMEOUT = 2, FLAG_BAR_TIMEOUT = 4 };

// Grid-wide barrier state of a persistent launch (zeroed before each launch).
struct GridBar {
  unsigned int count;  // blocks arrived at the current barrier
  unsigned int gen;    // barriers completed
};

// Work arrays of one solver.
struct DevWork {
  double* Q;      // [5][nce] state Q^n, ghost slots at [nc, nce)
  double* Qs;     // [5][nce] stage state Q*
  double* R;      // [5][nc]  Q^n + dt L^n + dt^2/6 dL^n
  float* Qf;      // [nce][8] binary32 copy of the stage state, one 32-byte record per cell
                  // (5 variables, 3 zero pads; mixed precision only)
  void* coef;     // [nc][kCoefRec] reconstruction polynomials (double or float):
                  // record of cell c: [v][j], j = 0: q, 1-3: g, 4-9: k
  void* Fs;       // [nf][kFluxRec] face flux sums: F (5) then dF/dt (5) (double or float)
  Control* ctl;   // [nmesh] one control block per member mesh
  GridBar* bar;   // barrier of the persistent step kernel
};

// NVTX range over a scope: entry points and step phases show up by name on a
// profiler's timeline (no cost without a profiler attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// Message returned by hgks_last_error() on this thread.
void set_last_error(const std::string& msg);
// HGKS_OK, or HGKS_EINVAL with the message set, for out-of-range parameters.
int check_params(const hgks_params* p);

// Set the step size of every member (tuning and test paths).
void launch_setdt(const DevMesh& m, const DevWork& w, double dt, cudaStream_t s);
// Time `reps` stage evaluations (reconstruction + flux) of the current state
// with the variants in p; returns milliseconds per evaluation (< 0 on error).
float time_stage(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, int reps, cudaStream_t s);
// Per-instantiation kernel attributes; call once per solver before capture.
void prepare_kernels(const DevMesh& m, int precision);
// True if the kernels are compiled for this stencil shape (faces per cell, K).
bool stencil_supported(int nfc, int K);
// Optional events recorded between the kernel groups of one step:
// ev[0] | finalize | ev[1] | ghost+recon | ev[2] | flux | ev[3] | update1 | ev[4]
//       | ghost+recon | ev[5] | flux | ev[6] | update2 | ev[7]
struct StepEvents {
  cudaEvent_t ev[8];
};

// Reconstruction of one stage (hgks_recon.cu): the binary64 stage state Q
// (FP64 path) or the binary32 records w.Qf (mixed path) into w.coef.
void launch_recon(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, const double* Q,
                  cudaStream_t s);
void prepare_recon(const DevMesh& m, int precision);
// Face flux of one stage (hgks_flux.cu): w.coef into w.Fs.
void launch_flux(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, cudaStream_t s);
// Shared-memory attributes of the persistent kernel (hgks_persist.cu).
void prepare_persist(const DevMesh& m, int precision);

// Launch one S2O4 step (Algorithm 2) on stream s; precision 0 = FP64, 1 = mixed.
void launch_step(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, cudaStream_t s,
                 const StepEvents* ev = nullptr);
// Launch n S2O4 steps as one persistent cooperative kernel; returns the CUDA
// error of the launch (cudaErrorCooperativeLaunchTooLarge and the like).
cudaError_t launch_persistent(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, int n,
                              cudaStream_t s);
// Set t_end and dt_fixed of every member for the following steps.
void launch_control(const DevMesh& m, const DevWork& w, double t_end, double dt_fixed, cudaStream_t s);
// Reset time/steps/flags of member `only` (every member when only < 0), copy
// the binary32 state if needed and compute the step bounds of the state.
void launch_reset(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, int only, double t,
                  cudaStream_t s);
// States in the caller's order and layout ([n][5] binary64, member-local
// cell index) to and from the internal order and layout: cells coff .. coff+n-1
// of Q ([5][nce]).  `in` and `out` are device buffers.
void launch_state_in(const DevMesh& m, const double* in, int64_t coff, int64_t n, double* Q, cudaStream_t s);
void launch_state_out(const DevMesh& m, const double* Q, int64_t coff, int64_t n, double* out, cudaStream_t s);
// Fill the binary32 tables of a device mesh from its binary64 arrays: the
// face geometry (fdl32, fdr32, fn32, fw32) and the reconstruction records
// (rec32).
void launch_round32(const DevMesh& m, cudaStream_t s);
// The binary64 erfcx of the flux on n device values (test path).
void launch_test_erfcx(const double* x, double* y, int64_t n, cudaStream_t s);
// L and dL/dt of the current state for step dt into Qs[0:5] and R (as L) -- test path.
void launch_operator(const DevMesh& m, const DevParams& p, const DevWork& w, int precision, double dt,
                     double* L, double* dL, cudaStream_t s);

}  // namespace hgks

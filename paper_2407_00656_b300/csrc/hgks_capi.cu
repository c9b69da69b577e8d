// hgks_capi.cu -- the C ABI of libhgks: mesh creation, solver lifecycle,
// stepping, state transfer and errors.  Every step of the scheme runs in the
// kernels of hgks_kernels.cu; this file only moves data and orders launches.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "hgks.h"
#include "hgks_internal.h"
#include "mesh_builder.h"

struct hgks_mesh {
  hgks::HostMesh m;
};

// One member mesh of a solver: its cells occupy [coff, coff + nc) of the
// solver's (union) cell numbering; perm maps its cells to caller order.
struct Member {
  int64_t coff = 0, nc = 0;
  std::vector<int64_t> perm;
};

// The static arrays of a (union) mesh in device memory, shared by every
// solver created over it and freed with the last reference.
struct hgks_dmesh {
  hgks::HostMesh sizes;         // sizes only (no arrays)
  std::vector<Member> members;  // one per member mesh (one for a single mesh)
  hgks::DevMesh dm{};
  void* arena = nullptr;
  size_t bytes = 0;
  std::atomic<int> refs{1};     // the creator's and one per solver
  std::atomic<int> solvers{0};  // solvers currently over this mesh
};

struct hgks_solver {
  hgks_dmesh* mesh = nullptr;  // counted reference
  std::vector<Member>& members() const { return mesh->members; }
  hgks::DevMesh dm{};
  hgks::DevParams dp{};
  hgks::DevWork dw{};
  int precision = 0;
  int use_graph = 1;
  int persistent = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* arena = nullptr;  // state and work arrays, stream-ordered on `stream`
  size_t arena_bytes = 0;
  cudaGraphExec_t graph = nullptr;
};

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return HGKS_ECUDA;
}

#define HGKS_CUDA(call, what)                   \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// Bump allocator over the solver's single device arena.
struct Carver {
  char* base;
  size_t off = 0, cap;
  template <typename T>
  T* take(int64_t n) {
    off = (off + 255) / 256 * 256;
    T* p = reinterpret_cast<T*>(base + off);
    off += sizeof(T) * (size_t)n;
    return p;
  }
};

// Uploads are queued on the solver's own stream, so that every later kernel
// on that (non-blocking) stream is ordered after them; the host arrays stay
// alive until the stream is synchronised at the end of solver creation.
template <typename T>
cudaError_t up(T* dst, const std::vector<T>& src, cudaStream_t st) {
  return cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, st);
}


// internal SoA [5][stride] at the member's offset -> member's caller order [n][5]
void to_caller(const Member& mb, const double* h, int64_t stride, double* q) {
  for (int64_t c = 0; c < mb.nc; ++c) {
    double* d = q + 5 * mb.perm[c];
    for (int v = 0; v < 5; ++v) d[v] = h[v * stride + mb.coff + c];
  }
}

}  // namespace

namespace hgks {
void set_last_error(const std::string& msg) { g_err = msg; }

// Parameter checks shared by every entry point that takes hgks_params.
int check_params(const hgks_params* p) {
  if (!p) return fail(HGKS_EINVAL, "params is NULL");
  if (!(p->gamma > 1.0 && p->gamma < 5.0 / 3.0 + 1e-12)) return fail(HGKS_EINVAL, "gamma must lie in (1, 5/3]");
  if (!(p->cfl > 0.0)) return fail(HGKS_EINVAL, "cfl must be positive");
  if (!(p->mu_ref >= 0.0) || !(p->tau_num_c >= 0.0)) return fail(HGKS_EINVAL, "mu_ref and tau_num_c must be >= 0");
  if (p->mu_ref > 0.0 && p->visc_exp != 0.0 && !(p->T_ref > 0.0)) return fail(HGKS_EINVAL, "T_ref must be positive");
  if (!(p->Pr > 0.0)) return fail(HGKS_EINVAL, "Pr must be positive");
  if (!(p->weno_eps > 0.0)) return fail(HGKS_EINVAL, "weno_eps must be positive");
  if (!(p->weno_gamma_lin > 0.0 && p->weno_gamma_lin < 0.125)) return fail(HGKS_EINVAL, "weno_gamma_lin must lie in (0, 1/8)");
  if (p->precision != HGKS_FP64 && p->precision != HGKS_FP32_MIXED) return fail(HGKS_EINVAL, "unknown precision");
  if (p->persistent != 0 && p->persistent != 1) return fail(HGKS_EINVAL, "persistent must be 0 or 1");
  return HGKS_OK;
}
}  // namespace hgks

extern "C" {

void hgks_params_default(hgks_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->gamma = 1.4;
  p->mu_ref = 0.0;
  p->T_ref = 1.0;
  p->visc_exp = 0.0;
  p->Pr = 1.0;
  p->cfl = 0.4;
  p->tau_num_c = 0.0;
  p->weno_eps = 1e-8;
  p->weno_gamma_lin = 0.025;
  p->q_inf[0] = 1.0;
  p->q_inf[4] = 2.5;
  p->precision = HGKS_FP64;
  p->use_graph = 1;
  p->autotune = 0;
  p->stream = nullptr;
}

const char* hgks_last_error(void) { return g_err.c_str(); }

int hgks_mesh_create(const hgks_mesh_desc* d, hgks_mesh** out) {
  hgks::Range range("hgks_mesh_create");
  if (!d || !out) return fail(HGKS_EINVAL, "NULL argument");
  *out = nullptr;
  if (d->cell_type != HGKS_TET4 && d->cell_type != HGKS_HEX8) return fail(HGKS_EINVAL, "cell_type must be 4 or 8");
  if (d->n_nodes <= 0 || d->n_cells <= 0 || !d->xyz || !d->cell_nodes)
    return fail(HGKS_EINVAL, "empty mesh or NULL node/cell arrays");
  if (d->n_bfaces < 0 || (d->n_bfaces > 0 && (!d->bface_nodes || !d->bface_tag)))
    return fail(HGKS_EINVAL, "bad boundary face arrays");
  try {
    hgks_mesh* mesh = new hgks_mesh;
    std::string err;
    int rc = hgks::build_host_mesh(*d, mesh->m, err);
    if (rc == HGKS_OK && !hgks::stencil_supported(mesh->m.nfc, mesh->m.K)) {
      rc = HGKS_EMESH;
      err = "stencil size " + std::to_string(mesh->m.K) + " is not among the compiled shapes";
    }
    if (rc != HGKS_OK) {
      delete mesh;
      return fail(rc, err);
    }
    *out = mesh;
    return HGKS_OK;
  } catch (const std::bad_alloc&) {
    return fail(HGKS_ENOMEM, "host allocation failed while building the mesh");
  }
}

void hgks_mesh_destroy(hgks_mesh* mesh) { delete mesh; }

int hgks_mesh_geometry(const hgks_mesh* mesh, double* vol_out, double* hdt_out) {
  if (!mesh) return fail(HGKS_EINVAL, "NULL mesh");
  const hgks::HostMesh& m = mesh->m;
  for (int64_t c = 0; c < m.nc; ++c) {
    if (vol_out) vol_out[m.perm[c]] = m.vol[c];
    if (hdt_out) hdt_out[m.perm[c]] = m.hdt[c];
  }
  return HGKS_OK;
}

int hgks_mesh_clone(const hgks_mesh* mesh, hgks_mesh** out) {
  if (!mesh || !out) return fail(HGKS_EINVAL, "NULL argument");
  *out = nullptr;
  try {
    *out = new hgks_mesh(*mesh);
  } catch (const std::bad_alloc&) {
    return fail(HGKS_ENOMEM, "host allocation failed while copying the mesh");
  }
  return HGKS_OK;
}

int64_t hgks_mesh_info(const hgks_mesh* mesh, int what) {
  if (!mesh) return -1;
  const hgks::HostMesh& m = mesh->m;
  switch (what) {
    case 0: return m.nc;
    case 1: return m.nf;
    case 2: return m.ng;
    case 3: return m.K;
    case 4: return m.M;
    case 5: return hgks::device_bytes(m, HGKS_FP64);
    case 6: return hgks::device_bytes(m, HGKS_FP32_MIXED);
    case 7: return hgks::mesh_static_bytes(m, 1);
    case 8: return hgks::solver_work_bytes(m, HGKS_FP64, 1);
    case 9: return hgks::solver_work_bytes(m, HGKS_FP32_MIXED, 1);
    default: return -1;
  }
}

}  // extern "C"

namespace {

// Device memory comes from the device's stream-ordered pool, which keeps
// freed blocks for reuse (release threshold raised once per device): solvers
// created and destroyed while others run allocate and free without a
// device-wide synchronisation.
void prepare_pool() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done[dev] = true;
}

// Test hook (hgks_test_fail_alloc): the number of device allocations still to
// succeed before one is made to fail, or -1.
std::atomic<int> g_fail_alloc{-1};

int alloc_on(void** p, size_t bytes, cudaStream_t st, const char* what) {
  prepare_pool();
  int k = g_fail_alloc.load();
  while (k >= 0 && !g_fail_alloc.compare_exchange_weak(k, k - 1)) {
  }
  // k == 0: this allocation is the one the test asked to fail, as an
  // exhausted pool would (nothing is allocated)
  cudaError_t e = k == 0 ? cudaErrorMemoryAllocation : cudaMallocAsync(p, bytes, st);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    char b[200];
    std::snprintf(b, sizeof b, "device allocation of %.3f GB for %s failed: %s", bytes / 1e9, what,
                  cudaGetErrorString(e));
    g_err = b;
    return HGKS_ENOMEM;
  }
  return HGKS_OK;
}

void dmesh_release(hgks_dmesh* d, cudaStream_t st) {
  if (!d || --d->refs > 0) return;
  if (d->arena) cudaFreeAsync(d->arena, st);
  delete d;
}

// Upload the static arrays of host mesh m (members: the member meshes in the
// union numbering; cmesh: member of each cell when there are several) on
// stream st.  Returns after the copies completed; the host mesh is unchanged.
int make_dmesh(const hgks::HostMesh& m, std::vector<Member> members, const std::vector<int32_t>& cmesh,
               cudaStream_t st, hgks_dmesh** out) {
  *out = nullptr;
  hgks_dmesh* d = nullptr;
  try {
    d = new hgks_dmesh;
  } catch (const std::bad_alloc&) {
    return fail(HGKS_ENOMEM, "host allocation failed");
  }
  const int n = (int)members.size();
  d->members = std::move(members);
  const size_t bytes = (size_t)hgks::mesh_static_bytes(m, n);
  int rc = alloc_on(&d->arena, bytes, st, "the mesh");
  if (rc) { delete d; return rc; }
  d->bytes = bytes;
  auto bail = [&](int code) {
    cudaStreamSynchronize(st);
    cudaFreeAsync(d->arena, st);
    delete d;
    return code;
  };
  Carver cv{static_cast<char*>(d->arena), 0, bytes};
  hgks::DevMesh& dm = d->dm;
  dm.nc = m.nc; dm.nf = m.nf; dm.ng = m.ng; dm.nce = m.nc + m.ng; dm.ncp = m.ncp;
  dm.K = m.K; dm.M = m.M; dm.KM = m.KM; dm.G = m.G; dm.nfc = m.nfc;
  dm.nmesh = n;
  std::vector<double> volinv;
  try {
    volinv.resize(m.nc);
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return bail(HGKS_ENOMEM);
  }
  for (int64_t c = 0; c < m.nc; ++c) volinv[c] = 1.0 / m.vol[c];
  double* p_volinv = cv.take<double>(m.nc);
  double* p_hdt = cv.take<double>(m.nc);
  double* p_hinv = cv.take<double>(m.nc);
  int32_t* p_perm = reinterpret_cast<int32_t*>(cv.take<double>(m.nc));  // caller index of each cell
  cv.take<double>(3 * m.nc);  // centroids are baked into the face offsets; slot kept for the size formula
  double* p_mom = cv.take<double>(6 * m.nc);
  int32_t* p_sten = cv.take<int32_t>((int64_t)m.K * m.nc);
  double* p_pinv0 = cv.take<double>((int64_t)9 * m.K * m.ncp);
  uint8_t* p_subidx = cv.take<uint8_t>((int64_t)m.M * m.KM * m.ncp);
  double* p_pinvm = cv.take<double>((int64_t)m.M * 3 * m.KM * m.ncp);
  int32_t* p_cface = cv.take<int32_t>((int64_t)m.nfc * m.nc);
  int32_t* p_gsrc = cv.take<int32_t>(m.ng);
  int32_t* p_gtag = cv.take<int32_t>(m.ng);
  double* p_gnrm = cv.take<double>(3 * m.ng);
  int32_t* p_fown = cv.take<int32_t>(m.nf);
  int32_t* p_fnbr = cv.take<int32_t>(m.nf);
  double* p_fdl = cv.take<double>((int64_t)m.G * 3 * m.nf);
  double* p_fdr = cv.take<double>((int64_t)m.G * 3 * m.nf);
  double* p_fn = cv.take<double>((int64_t)m.G * 3 * m.nf);
  double* p_fw = cv.take<double>((int64_t)m.G * m.nf);
  float* p_fdl32 = cv.take<float>((int64_t)m.G * 3 * m.nf);
  float* p_fdr32 = cv.take<float>((int64_t)m.G * 3 * m.nf);
  float* p_fn32 = cv.take<float>((int64_t)m.G * 3 * m.nf);
  float* p_fw32 = cv.take<float>((int64_t)m.G * m.nf);
  float* p_rec32 = cv.take<float>(hgks::rec32_bytes(m.K, m.M, m.KM) / 4 * (m.ncp / 32));
  int32_t* p_cmesh = n > 1 ? cv.take<int32_t>(m.nc) : nullptr;
  if (cv.off > bytes) { g_err = "internal error: mesh arena too small"; return bail(HGKS_ENOMEM); }
  dm.volinv = p_volinv; dm.hdt = p_hdt; dm.hinv = p_hinv; dm.mom = p_mom; dm.sten = p_sten; dm.pinv0 = p_pinv0;
  dm.subidx = p_subidx; dm.pinvm = p_pinvm; dm.cface = p_cface; dm.gsrc = p_gsrc; dm.gtag = p_gtag; dm.gnrm = p_gnrm;
  dm.fown = p_fown; dm.fnbr = p_fnbr; dm.fdl = p_fdl; dm.fdr = p_fdr; dm.fn = p_fn; dm.fw = p_fw;
  dm.fdl32 = p_fdl32; dm.fdr32 = p_fdr32; dm.fn32 = p_fn32; dm.fw32 = p_fw32; dm.rec32 = p_rec32;
  dm.cmesh = p_cmesh;
  dm.perm = p_perm;
  std::vector<int32_t> perm32;
  try {
    perm32.resize(m.nc);
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return bail(HGKS_ENOMEM);
  }
  for (const Member& mb : d->members)
    for (int64_t c = 0; c < mb.nc; ++c) perm32[mb.coff + c] = (int32_t)mb.perm[c];
  cudaError_t ue = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (ue == cudaSuccess) ue = x; };
  chk(up(p_volinv, volinv, st));
  chk(up(p_hdt, m.hdt, st));
  chk(up(p_hinv, m.hinv, st));
  chk(up(p_perm, perm32, st));
  chk(up(p_mom, m.mom, st));
  chk(up(p_sten, m.sten, st));
  chk(up(p_pinv0, m.pinv0, st));
  chk(up(p_subidx, m.subidx, st));
  chk(up(p_pinvm, m.pinvm, st));
  chk(up(p_cface, m.cface, st));
  if (m.ng) {
    chk(up(p_gsrc, m.gsrc, st));
    chk(up(p_gtag, m.gtag, st));
    chk(up(p_gnrm, m.gnrm, st));
  }
  chk(up(p_fown, m.fown, st));
  chk(up(p_fnbr, m.fnbr, st));
  chk(up(p_fdl, m.fdl, st));
  chk(up(p_fdr, m.fdr, st));
  chk(up(p_fn, m.fn, st));
  chk(up(p_fw, m.fw, st));
  if (p_cmesh) chk(up(p_cmesh, cmesh, st));
  if (ue == cudaSuccess) {
    hgks::launch_round32(dm, st);
    ue = cudaGetLastError();
  }
  if (ue == cudaSuccess) ue = cudaStreamSynchronize(st);  // the host arrays may go away after return
  if (ue != cudaSuccess) { cuda_fail(ue, "uploading the mesh"); return bail(HGKS_ECUDA); }
  d->sizes.ctype = m.ctype; d->sizes.nfc = m.nfc; d->sizes.G = m.G; d->sizes.M = m.M; d->sizes.KM = m.KM;
  d->sizes.K = m.K; d->sizes.nc = m.nc; d->sizes.nf = m.nf; d->sizes.ng = m.ng; d->sizes.ncp = m.ncp;
  *out = d;
  return HGKS_OK;
}

// The solver's stream: the caller's, or a new non-blocking one.
int solver_stream(const hgks_params* params, cudaStream_t* st, bool* own) {
  if (params->stream) {
    *st = static_cast<cudaStream_t>(params->stream);
    *own = false;
    return HGKS_OK;
  }
  cudaError_t e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  *own = true;
  return HGKS_OK;
}

// Create a solver over device mesh d (takes a new reference on success) on
// stream st (owned when own): allocate the state and work arrays, set the
// parameters, copy the initial states q0[i] of the members, compute the first
// step bound and, when asked, time the kernel variants.
int make_solver(hgks_dmesh* d, const hgks_params* params, const double* const* q0, cudaStream_t st, bool own,
                hgks_solver** out) {
  *out = nullptr;
  hgks_solver* s = nullptr;
  try {
    s = new hgks_solver;
  } catch (const std::bad_alloc&) {
    return fail(HGKS_ENOMEM, "host allocation failed");
  }
  s->stream = st;
  s->own_stream = own;
  auto bail = [&](int code) {
    if (s->arena) {
      cudaStreamSynchronize(s->stream);
      cudaFreeAsync(s->arena, s->stream);
    }
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return code;
  };
  const int n = (int)d->members.size();
  const hgks::HostMesh& m = d->sizes;
  s->precision = params->precision;
  s->use_graph = params->use_graph;
  s->persistent = params->persistent;
  const size_t bytes = (size_t)hgks::solver_work_bytes(m, s->precision, n);
  int rc = alloc_on(&s->arena, bytes, s->stream, "the solver state");
  if (rc) return bail(rc);
  s->arena_bytes = bytes;
  s->dm = d->dm;
  const hgks::DevMesh& dm = s->dm;
  Carver cv{static_cast<char*>(s->arena), 0, bytes};
  hgks::DevWork& w = s->dw;
  const bool f32 = s->precision == HGKS_FP32_MIXED;
  const int64_t rs = f32 ? 4 : 8;
  w.Q = cv.take<double>(5 * dm.nce);
  w.Qs = cv.take<double>(5 * dm.nce);
  w.R = cv.take<double>(5 * m.nc);
  w.Qf = f32 ? cv.take<float>(8 * dm.nce) : nullptr;
  w.coef = cv.take<char>(rs * (f32 ? hgks::kCoefRec32 : hgks::kCoefRec64) * m.nc);
  // face records, plus one past the last face that no kernel writes: the
  // cell-face entry of a prism's collapsed side points at it
  const int64_t frec = rs * (f32 ? hgks::kFluxRec32 : hgks::kFluxRec64);
  w.Fs = cv.take<char>(frec * (m.nf + 1));
  w.ctl = cv.take<hgks::Control>(n);
  w.bar = cv.take<hgks::GridBar>(1);
  if (cv.off > bytes) { g_err = "internal error: solver arena too small"; return bail(HGKS_ENOMEM); }
  // parameters
  hgks::DevParams& dp = s->dp;
  dp.gamma = params->gamma;
  dp.Kint = (5.0 - 3.0 * params->gamma) / (params->gamma - 1.0);
  dp.mu_ref = params->mu_ref;
  dp.T_ref = params->T_ref;
  dp.visc_exp = params->visc_exp;
  dp.Pr = params->Pr;
  dp.cfl = params->cfl;
  dp.tau_c = params->tau_num_c;
  dp.eps = params->weno_eps;
  dp.glin = params->weno_gamma_lin;
  for (int i = 0; i < 5; ++i) dp.qinf[i] = params->q_inf[i];
  dp.viscous = (params->mu_ref > 0.0 || params->tau_num_c > 0.0) ? 1 : 0;
  hgks::fill_float_params(dp);
  // default flux variant by size: one thread per Gauss point while one
  // thread per face would leave the SMs short of threads (a per-face thread
  // is a long dependent chain), measured crossovers: binary64 at about 16
  // blocks of 128 per SM, binary32 at about 2
  {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t per_sm = f32 ? 2 : 16;
    dp.flux_variant = dm.nf < per_sm * sms * 128 ? 1 : 0;
  }
  dp.recon_variant = 0;
  dp.bar_cycles = hgks::kBarrierCycles;
  hgks::prepare_kernels(dm, s->precision);
  // initial states: each member's caller-order states are copied into Q*
  // (free until the first step) and permuted into Q on the device; the ghost
  // slots and Q* then start at zero
  cudaError_t e = cudaMemsetAsync(w.Q, 0, sizeof(double) * 5 * dm.nce, s->stream);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const Member& mb = d->members[i];
    e = cudaMemcpyAsync(w.Qs, q0[i], sizeof(double) * 5 * mb.nc, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) hgks::launch_state_in(dm, w.Qs, mb.coff, mb.nc, w.Q, s->stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(w.Qs, 0, sizeof(double) * 5 * dm.nce, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(static_cast<char*>(w.Fs) + frec * dm.nf, 0, frec, s->stream);
  if (e != cudaSuccess) { cuda_fail(e, "copying the initial state"); return bail(HGKS_ECUDA); }
  hgks::launch_reset(dm, dp, w, s->precision, -1, 0.0, s->stream);
  e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) { cuda_fail(e, "initialising the solver"); return bail(HGKS_ECUDA); }
  if (params->autotune) {
    // time every variant pair on this mesh and state (the state is not
    // modified: only the reconstruction and flux work arrays are written)
    hgks::launch_setdt(dm, w, 1e-3, s->stream);
    float best = -1.f;
    int bf = 0, br = 0;
    for (int fv = 0; fv < 2; ++fv)
      for (int rv = 0; rv < 2; ++rv) {
        dp.flux_variant = fv;
        dp.recon_variant = rv;
        hgks::time_stage(dm, dp, w, s->precision, 1, s->stream);  // warm-up
        const float ms = hgks::time_stage(dm, dp, w, s->precision, 3, s->stream);
        if (ms >= 0.f && (best < 0.f || ms < best)) { best = ms; bf = fv; br = rv; }
      }
    dp.flux_variant = bf;
    dp.recon_variant = br;
    hgks::launch_setdt(dm, w, 0.0, s->stream);
    e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { cuda_fail(e, "autotuning"); return bail(HGKS_ECUDA); }
  }
  ++d->refs;
  ++d->solvers;
  s->mesh = d;
  *out = s;
  return HGKS_OK;
}

// hgks_init / hgks_batch_init: upload the (union) mesh, then create the
// solver over it; on success the solver holds the only reference to the
// device mesh and the caller's host meshes are deleted, on failure they are
// untouched.
int create_solver(hgks_mesh* const* meshes, int n, const hgks_params* params, const double* const* q0,
                  hgks_solver** out) {
  *out = nullptr;
  int rc = hgks::check_params(params);
  if (rc) return rc;
  cudaStream_t st = nullptr;
  bool own = false;
  rc = solver_stream(params, &st, &own);
  if (rc) return rc;
  auto drop_stream = [&]() { if (own) cudaStreamDestroy(st); };
  hgks_dmesh* d = nullptr;
  try {
    if (n == 1) {
      const hgks::HostMesh& m = meshes[0]->m;
      std::vector<Member> mbs(1);
      mbs[0].coff = 0;
      mbs[0].nc = m.nc;
      mbs[0].perm = m.perm;
      rc = make_dmesh(m, std::move(mbs), {}, st, &d);
    } else {
      std::vector<const hgks::HostMesh*> parts;
      for (int i = 0; i < n; ++i) parts.push_back(&meshes[i]->m);
      hgks::HostMesh u;
      std::vector<int32_t> cmesh;
      std::vector<int64_t> coff;
      std::string err;
      rc = hgks::build_union(parts, u, cmesh, coff, err);
      if (rc) g_err = err;
      if (!rc && !hgks::stencil_supported(u.nfc, u.K)) {
        g_err = "batch stencil size is not among the compiled shapes";
        rc = HGKS_EMESH;
      }
      if (!rc) {
        std::vector<Member> mbs(n);
        for (int i = 0; i < n; ++i) {
          mbs[i].coff = coff[i];
          mbs[i].nc = meshes[i]->m.nc;
          mbs[i].perm = meshes[i]->m.perm;
        }
        rc = make_dmesh(u, std::move(mbs), cmesh, st, &d);
      }
    }
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed while preparing the mesh";
    rc = HGKS_ENOMEM;
  }
  if (rc) { drop_stream(); return rc; }
  hgks_solver* s = nullptr;
  rc = make_solver(d, params, q0, st, own, &s);  // destroys an owned stream on failure
  dmesh_release(d, rc ? nullptr : st);           // the solver holds its own reference
  if (rc) return rc;
  for (int i = 0; i < n; ++i) delete meshes[i];
  *out = s;
  return HGKS_OK;
}

const char* const kStageMsg = "a reconstruction block's bounded wait for its staged copies ran out";
const char* const kBarMsg = "a grid barrier of the persistent launch ran out of its bounded wait";

int read_flags(hgks_solver* s, int only, hgks::Control* first) {
  std::vector<hgks::Control> c(s->members().size());
  HGKS_CUDA(cudaMemcpy(c.data(), s->dw.ctl, sizeof(hgks::Control) * c.size(), cudaMemcpyDeviceToHost),
            "reading the control blocks");
  if (first) *first = c[only >= 0 ? only : 0];
  for (size_t i = 0; i < c.size(); ++i) {
    if (only >= 0 && (int)i != only) continue;
    if (c[i].flags & hgks::FLAG_BAR_TIMEOUT) return fail(HGKS_ETIMEOUT, kBarMsg);
    if (c[i].flags & hgks::FLAG_TIMEOUT) return fail(HGKS_ETIMEOUT, kStageMsg);
    if (c[i].flags & hgks::FLAG_NONFINITE) return fail(HGKS_ENONFINITE, "a step produced a non-finite cell average");
  }
  // timeouts are recorded on member 0 for the whole solver
  if (only > 0 && (c[0].flags & hgks::FLAG_BAR_TIMEOUT)) return fail(HGKS_ETIMEOUT, kBarMsg);
  if (only > 0 && (c[0].flags & hgks::FLAG_TIMEOUT)) return fail(HGKS_ETIMEOUT, kStageMsg);
  return HGKS_OK;
}

}  // namespace

extern "C" {

int hgks_init(hgks_mesh* mesh, const hgks_params* params, const double* q0, hgks_solver** out) {
  hgks::Range range("hgks_init");
  if (!mesh || !out || !q0) return fail(HGKS_EINVAL, "NULL argument");
  return create_solver(&mesh, 1, params, &q0, out);
}

int hgks_batch_init(hgks_mesh* const* meshes, int n, const hgks_params* params, const double* const* q0,
                    hgks_solver** out) {
  hgks::Range range("hgks_batch_init");
  if (!meshes || !q0 || !out || n <= 0) return fail(HGKS_EINVAL, "bad argument");
  for (int i = 0; i < n; ++i)
    if (!meshes[i] || !q0[i]) return fail(HGKS_EINVAL, "NULL member mesh or state");
  return create_solver(meshes, n, params, q0, out);
}

int hgks_members(const hgks_solver* s) { return s ? (int)s->members().size() : -1; }

int hgks_member_write(hgks_solver* s, int member, const double* q, double t) {
  hgks::Range range("hgks_write");
  if (!s || !q) return fail(HGKS_EINVAL, "NULL argument");
  if (member < 0 || member >= (int)s->members().size()) return fail(HGKS_EINVAL, "member out of range");
  // the caller's states go into Q* (scratch between steps; ordered after the
  // queued steps on the solver's stream) and are permuted into the member's
  // cells of Q on the device
  const Member& mb = s->members()[member];
  HGKS_CUDA(cudaMemcpyAsync(s->dw.Qs, q, sizeof(double) * 5 * mb.nc, cudaMemcpyHostToDevice, s->stream),
            "copying the state");
  hgks::launch_state_in(s->dm, s->dw.Qs, mb.coff, mb.nc, s->dw.Q, s->stream);
  hgks::launch_reset(s->dm, s->dp, s->dw, s->precision, member, t, s->stream);
  HGKS_CUDA(cudaStreamSynchronize(s->stream), "writing the state");
  HGKS_CUDA(cudaGetLastError(), "writing the state");
  return HGKS_OK;
}

int hgks_write(hgks_solver* s, const double* q, double t) { return hgks_member_write(s, 0, q, t); }

int hgks_step(hgks_solver* s, int n_steps, double t_end, double dt_fixed) {
  hgks::Range range("hgks_step");
  if (!s) return fail(HGKS_EINVAL, "NULL solver");
  if (n_steps < 0) return fail(HGKS_EINVAL, "n_steps must be >= 0");
  if (n_steps == 0) return HGKS_OK;
  hgks::launch_control(s->dm, s->dw, t_end, dt_fixed, s->stream);
  if (s->persistent) {
    HGKS_CUDA(hgks::launch_persistent(s->dm, s->dp, s->dw, s->precision, n_steps, s->stream),
              "launching the persistent steps");
  } else if (s->use_graph) {
    if (!s->graph) {
      cudaGraph_t g = nullptr;
      HGKS_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal), "beginning graph capture");
      hgks::launch_step(s->dm, s->dp, s->dw, s->precision, s->stream);
      cudaError_t e = cudaStreamEndCapture(s->stream, &g);
      if (e != cudaSuccess) return cuda_fail(e, "capturing the step graph");
      e = cudaGraphInstantiate(&s->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        s->graph = nullptr;
        return cuda_fail(e, "instantiating the step graph");
      }
    }
    for (int i = 0; i < n_steps; ++i) HGKS_CUDA(cudaGraphLaunch(s->graph, s->stream), "launching the step graph");
  } else {
    for (int i = 0; i < n_steps; ++i) hgks::launch_step(s->dm, s->dp, s->dw, s->precision, s->stream);
  }
  HGKS_CUDA(cudaGetLastError(), "launching the step");
  return HGKS_OK;
}

int hgks_query(hgks_solver* s) {
  if (!s) return fail(HGKS_EINVAL, "NULL solver");
  cudaError_t e = cudaStreamQuery(s->stream);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) {
    cudaGetLastError();
    return 0;
  }
  return cuda_fail(e, "querying the stream");
}

int hgks_sync(hgks_solver* s) {
  hgks::Range range("hgks_sync");
  if (!s) return fail(HGKS_EINVAL, "NULL solver");
  HGKS_CUDA(cudaStreamSynchronize(s->stream), "synchronising");
  HGKS_CUDA(cudaGetLastError(), "synchronising");
  return read_flags(s, -1, nullptr);
}

int hgks_member_read(hgks_solver* s, int member, double* q_out, double* t_out, int64_t* steps_out) {
  if (!s) return fail(HGKS_EINVAL, "NULL solver");
  if (member < 0 || member >= (int)s->members().size()) return fail(HGKS_EINVAL, "member out of range");
  if (q_out) {
    // permuted into the caller's order in Q* (scratch between steps), then copied out
    const Member& mb = s->members()[member];
    hgks::launch_state_out(s->dm, s->dw.Q, mb.coff, mb.nc, s->dw.Qs, s->stream);
    HGKS_CUDA(cudaMemcpyAsync(q_out, s->dw.Qs, sizeof(double) * 5 * mb.nc, cudaMemcpyDeviceToHost, s->stream),
              "reading the state");
  }
  HGKS_CUDA(cudaStreamSynchronize(s->stream), "synchronising");
  HGKS_CUDA(cudaGetLastError(), "reading the state");
  hgks::Control c;
  const int rc = read_flags(s, member, &c);
  if (t_out) *t_out = c.t;
  if (steps_out) *steps_out = c.steps;
  return rc;
}

int hgks_read(hgks_solver* s, double* q_out, double* t_out, int64_t* steps_out) {
  hgks::Range range("hgks_read");
  return hgks_member_read(s, 0, q_out, t_out, steps_out);
}

int hgks_stage_operator(hgks_solver* s, double dt, double* L_out, double* dL_out) {
  hgks::Range range("hgks_stage_operator");
  if (!s || !L_out || !dL_out) return fail(HGKS_EINVAL, "NULL argument");
  if (!(dt > 0.0)) return fail(HGKS_EINVAL, "dt must be positive");
  if (s->members().size() != 1) return fail(HGKS_EINVAL, "the stage operator is defined for single-mesh solvers");
  const int64_t nc = s->dm.nc;
  // the stage buffers Q* and R are free between steps
  hgks::launch_operator(s->dm, s->dp, s->dw, s->precision, dt, s->dw.Qs, s->dw.R, s->stream);
  HGKS_CUDA(cudaStreamSynchronize(s->stream), "evaluating the stage operator");
  HGKS_CUDA(cudaGetLastError(), "evaluating the stage operator");
  std::vector<double> h(5 * nc);
  HGKS_CUDA(cudaMemcpy(h.data(), s->dw.Qs, sizeof(double) * 5 * nc, cudaMemcpyDeviceToHost), "reading L");
  to_caller(s->members()[0], h.data(), nc, L_out);
  HGKS_CUDA(cudaMemcpy(h.data(), s->dw.R, sizeof(double) * 5 * nc, cudaMemcpyDeviceToHost), "reading dL/dt");
  to_caller(s->members()[0], h.data(), nc, dL_out);
  return HGKS_OK;
}

int hgks_profile(hgks_solver* s, int n_steps, double t_end, double dt_fixed, double* ms_out) {
  hgks::Range range("hgks_profile");
  if (!s || !ms_out || n_steps <= 0) return fail(HGKS_EINVAL, "bad argument");
  hgks::StepEvents ev;
  for (int i = 0; i < 8; ++i) HGKS_CUDA(cudaEventCreate(&ev.ev[i]), "creating events");
  double acc[4] = {0, 0, 0, 0};
  hgks::launch_control(s->dm, s->dw, t_end, dt_fixed, s->stream);
  int rc = HGKS_OK;
  for (int k = 0; k < n_steps && rc == HGKS_OK; ++k) {
    hgks::launch_step(s->dm, s->dp, s->dw, s->precision, s->stream, &ev);
    cudaError_t e = cudaEventSynchronize(ev.ev[7]);
    if (e != cudaSuccess) { rc = cuda_fail(e, "profiling a step"); break; }
    float t[7];
    for (int i = 0; i < 7; ++i) cudaEventElapsedTime(&t[i], ev.ev[i], ev.ev[i + 1]);
    acc[0] += t[0];
    acc[1] += t[1] + t[4];
    acc[2] += t[2] + t[5];
    acc[3] += t[3] + t[6];
  }
  for (int i = 0; i < 8; ++i) cudaEventDestroy(ev.ev[i]);
  for (int i = 0; i < 4; ++i) ms_out[i] = acc[i] / n_steps;
  return rc;
}

int64_t hgks_solver_bytes(const hgks_solver* s) { return s ? (int64_t)(s->arena_bytes + s->mesh->bytes) : -1; }

int hgks_set_tuning(hgks_solver* s, int flux_variant, int recon_variant) {
  if (!s) return fail(HGKS_EINVAL, "NULL solver");
  if (flux_variant < 0 || flux_variant > 1 || recon_variant < 0 || recon_variant > 1)
    return fail(HGKS_EINVAL, "variant out of range");
  HGKS_CUDA(cudaStreamSynchronize(s->stream), "waiting for queued work");
  s->dp.flux_variant = flux_variant;
  s->dp.recon_variant = recon_variant;
  if (s->graph) {  // the captured step used the previous variants
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  return HGKS_OK;
}

int hgks_test_barrier_limit(hgks_solver* s, int64_t cycles) {
  if (!s) return fail(HGKS_EINVAL, "NULL solver");
  HGKS_CUDA(cudaStreamSynchronize(s->stream), "waiting for queued work");
  s->dp.bar_cycles = cycles < 0 ? hgks::kBarrierCycles : (long long)cycles;
  return HGKS_OK;
}

int hgks_test_fail_alloc(int n) {
  g_fail_alloc.store(n < 0 ? -1 : n);
  return HGKS_OK;
}

int hgks_test_erfcx(const double* x, double* y, int64_t n) {
  if (n < 0 || (n > 0 && (!x || !y))) return fail(HGKS_EINVAL, "hgks_test_erfcx: bad arguments");
  if (n == 0) return HGKS_OK;
  cudaStream_t st;
  HGKS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "cudaStreamCreate");
  void* d = nullptr;
  int rc = alloc_on(&d, (size_t)n * 2 * sizeof(double), st, "hgks_test_erfcx");
  if (rc == HGKS_OK) {
    double* dx = static_cast<double*>(d);
    double* dy = dx + n;
    cudaError_t e = cudaMemcpyAsync(dx, x, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      hgks::launch_test_erfcx(dx, dy, n, st);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, dy, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d, st);
    cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "hgks_test_erfcx");
  }
  cudaStreamDestroy(st);
  return rc;
}

int hgks_tuning(const hgks_solver* s, int* flux_variant, int* recon_variant) {
  if (!s) return fail(HGKS_EINVAL, "NULL solver");
  if (flux_variant) *flux_variant = s->dp.flux_variant;
  if (recon_variant) *recon_variant = s->dp.recon_variant;
  return HGKS_OK;
}

void hgks_destroy(hgks_solver* s) {
  hgks::Range range("hgks_destroy");
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->arena) cudaFreeAsync(s->arena, s->stream);
  --s->mesh->solvers;
  dmesh_release(s->mesh, s->stream);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

int hgks_dmesh_create(const hgks_mesh* mesh, void* stream, hgks_dmesh** out) {
  hgks::Range range("hgks_dmesh_create");
  if (!mesh || !out) return fail(HGKS_EINVAL, "NULL argument");
  *out = nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool own = false;
  if (!st) {
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    own = true;
  }
  int rc;
  try {
    const hgks::HostMesh& m = mesh->m;
    std::vector<Member> mbs(1);
    mbs[0].coff = 0;
    mbs[0].nc = m.nc;
    mbs[0].perm = m.perm;
    rc = make_dmesh(m, std::move(mbs), {}, st, out);
  } catch (const std::bad_alloc&) {
    rc = fail(HGKS_ENOMEM, "host allocation failed");
  }
  if (own) cudaStreamDestroy(st);
  return rc;
}

void hgks_dmesh_release(hgks_dmesh* dmesh) { dmesh_release(dmesh, nullptr); }

int64_t hgks_dmesh_info(const hgks_dmesh* d, int what) {
  if (!d) return -1;
  switch (what) {
    case 0: return d->sizes.nc;
    case 1: return d->sizes.nf;
    case 2: return d->sizes.ng;
    case 5: return (int64_t)d->bytes;
    case 6: return hgks::solver_work_bytes(d->sizes, HGKS_FP64, (int)d->members.size());
    case 7: return hgks::solver_work_bytes(d->sizes, HGKS_FP32_MIXED, (int)d->members.size());
    case 8: return d->solvers.load();
    default: return -1;
  }
}

int hgks_init_shared(hgks_dmesh* dmesh, const hgks_params* params, const double* q0, hgks_solver** out) {
  hgks::Range range("hgks_init_shared");
  if (!dmesh || !out || !q0) return fail(HGKS_EINVAL, "NULL argument");
  *out = nullptr;
  int rc = hgks::check_params(params);
  if (rc) return rc;
  cudaStream_t st = nullptr;
  bool own = false;
  rc = solver_stream(params, &st, &own);
  if (rc) return rc;
  const double* q[1] = {q0};
  return make_solver(dmesh, params, q, st, own, out);
}

}  // extern "C"

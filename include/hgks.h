/*
 * hgks.h -- C ABI of the HGKS hot-path library (libhgks.so) for one B300.
 *
 * The library advances the cell averages Q = (rho, rho U, rho V, rho W, rho E)
 * of a 3D unstructured tetrahedral or hexahedral mesh with the high-order
 * gas-kinetic scheme of arXiv 2407.00656:
 *   - third-order non-compact WENO reconstruction over two-layer stencils
 *     (Section 2.3, Eqs. polys and weno, Algorithm 1),
 *   - the time-dependent BGK gas-kinetic flux at face Gauss points
 *     (Section 2.1, Eqs. flux-G and flux; Section 2.2, Eq. expansion-1),
 *   - the two-stage fourth-order (S2O4) update (Section 2.2),
 *   - periodic, Riemann-invariant far-field and no-slip adiabatic wall
 *     boundaries (Section 5.2).
 *
 * Conventions for every call below:
 *   - Return 0 (HGKS_OK) or a negative HGKS_E* code; never abort.  The
 *     message of the last failure on the calling thread is hgks_last_error().
 *   - Host arrays passed in are read during the call only; the caller keeps
 *     ownership.  Host output arrays are written by the call.
 *   - Cell data at this boundary is always in the caller's cell order; the
 *     library reorders cells internally along a space-filling curve.
 *   - Floating point is IEEE binary64 unless stated otherwise.
 */
#ifndef HGKS_H
#define HGKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hgks_mesh hgks_mesh;     /* host-side mesh, built by hgks_mesh_create */
typedef struct hgks_solver hgks_solver; /* device-resident solver state */
typedef struct hgks_dmesh hgks_dmesh;   /* device-resident mesh, shared by solvers */

enum {
  HGKS_OK = 0,
  HGKS_EINVAL = -1,     /* bad argument */
  HGKS_ENOMEM = -2,     /* host or device allocation failed */
  HGKS_EMESH = -3,      /* inconsistent mesh, degenerate cell or rank-deficient stencil */
  HGKS_ECUDA = -4,      /* CUDA runtime error */
  HGKS_ENONFINITE = -5, /* a non-finite cell average was produced */
  HGKS_ETIMEOUT = -6    /* a bounded device wait ran out */
};
enum { HGKS_TET4 = 4, HGKS_HEX8 = 8 };
enum { HGKS_BC_PERIODIC = 1, HGKS_BC_FARFIELD = 2, HGKS_BC_WALL = 3 };
enum { HGKS_FP64 = 0, HGKS_FP32_MIXED = 1 };

/* Mesh description (Section 3.1).  All cells have the same type.
 *   xyz         [n_nodes][3] node coordinates.
 *   cell_nodes  [n_cells][cell_type] node indices.  Tet: local face p is the
 *               face opposite node p.  Hex: nodes 0-3 one quad, 4-7 the
 *               opposite quad in the same order; local faces (0,1,2,3),
 *               (0,1,5,4), (1,2,6,5), (2,3,7,6), (3,0,4,7), (4,5,6,7).
 *               A triangular prism is a hex with nodes 2 = 3 and 6 = 7
 *               (bottom triangle 0 1 2, top triangle 4 5 6): its face
 *               (2,3,7,6) collapses to an edge and is dropped, so hex and
 *               prism cells mix freely in one HGKS_HEX8 mesh.  Any other
 *               repeated node fails with HGKS_EINVAL.  (The paper defines
 *               tetrahedra and hexahedra; the prism's faces and sub-stencils
 *               are this library's reading: triangles take the 3-point rule,
 *               and the two octant sub-stencils at the collapsed edge both
 *               take the two side faces meeting there.)
 *   bface_nodes [n_bfaces][4] nodes of tagged boundary faces (-1 pads a
 *               triangle), bface_tag[n_bfaces] one of HGKS_BC_*.
 *   periods     [3] translation lengths along x, y, z used to pair untagged
 *               boundary faces periodically (0 = not periodic), or NULL.
 *   sfc_reorder 1: order cells along a Morton curve (recommended), 0: keep. */
typedef struct {
  int64_t n_nodes;
  const double* xyz;
  int64_t n_cells;
  int32_t cell_type;
  int32_t sfc_reorder;
  const int64_t* cell_nodes;
  int64_t n_bfaces;
  const int64_t* bface_nodes;
  const int32_t* bface_tag;
  const double* periods;
} hgks_mesh_desc;

/* Physical and numerical parameters.
 *   gamma          specific heat ratio; internal degrees of freedom
 *                  K = (5 - 3 gamma)/(gamma - 1) (Section 2.1).
 *   mu_ref, T_ref, visc_exp   viscosity mu = mu_ref (T/T_ref)^visc_exp with
 *                  T = p/rho (Section 5.2); mu_ref = 0 gives the Euler flux.
 *   Pr             Prandtl number (heat-flux correction of the BGK model).
 *   cfl            time step: dt = cfl min_i h_i/(|U_i|+c_i), h_i =
 *                  3|cell_i|/|surface_i|, and with viscosity also
 *                  dt <= cfl min_i rho_i h_i^2/(2 mu_i).
 *   tau_num_c      numerical collision time coefficient C in
 *                  tau = mu/p + C dt |p_l - p_r|/(p_l + p_r).
 *   weno_eps, weno_gamma_lin  WENO epsilon and sub-stencil linear weight
 *                  (gamma_0 = 1 - M weno_gamma_lin), Section 2.3.
 *   q_inf          conservative far-field free stream.
 *   precision      HGKS_FP64, or HGKS_FP32_MIXED: reconstruction and flux
 *                  in binary32, geometry, inverses and S2O4 in binary64
 *                  (the binary32 kernels read binary32 roundings of the
 *                  geometry and inverses, made once per device mesh).
 *   use_graph      1: replay each step as one captured CUDA graph.
 *   autotune       1: at hgks_init, time the kernel variants (flux with one
 *                  thread per face or one per Gauss point; reconstruction
 *                  rows staged by bulk asynchronous copies or read directly)
 *                  on this mesh and keep the fastest.  The variants perform
 *                  the same operations in the same order and agree to a few
 *                  units in the last place (the compiler may fuse a
 *                  multiply and an add in one variant and not in another);
 *                  each variant is deterministic.  0: the defaults, rows
 *                  staged, and flux per Gauss point for meshes with fewer
 *                  than 16 (FP64) or 2 (FP32_MIXED) x 128 faces per SM, per
 *                  face above.
 *   persistent     1: hgks_step runs its n steps as one persistent
 *                  cooperative launch (every phase of every step in one
 *                  kernel, grid-wide barriers between phases) instead of n
 *                  graph launches, for small meshes and batches of them;
 *                  measured slower than graph launches on B300, so off by
 *                  default.  The flux runs per face and the reconstruction
 *                  variants are fixed (binary32: per-block records;
 *                  binary64: rows read directly), whatever hgks_set_tuning
 *                  selected.
 *                  Results agree with the separate kernels to a few units in
 *                  the last place.  A grid barrier that waits more than
 *                  about a second ends the launch with HGKS_ETIMEOUT at the
 *                  next sync or read.
 *   stream         cudaStream_t to run on, or NULL for a library stream. */
typedef struct {
  double gamma, mu_ref, T_ref, visc_exp, Pr, cfl, tau_num_c, weno_eps, weno_gamma_lin;
  double q_inf[5];
  int32_t precision;
  int32_t use_graph;
  int32_t autotune;
  int32_t persistent;
  void* stream;
} hgks_params;

/* Fill *p with defaults: gamma 1.4, inviscid, Pr 1, cfl 0.4, weno_eps 1e-8,
 * weno_gamma_lin 0.025, q_inf = (1,0,0,0,2.5), FP64, graphs on, autotune off,
 * NULL stream. */
void hgks_params_default(hgks_params* p);

/* Build the host mesh: faces, periodic pairing, boundary ghosts, two-layer
 * WENO stencils and sub-stencils, geometry, face Gauss points and the
 * least-squares pseudo-inverses (Section 3.1, Algorithm 1; Section 2.3).
 * Inputs are copied.  On success *out owns a new mesh.  Errors: HGKS_EINVAL
 * (bad sizes/pointers), HGKS_EMESH (non-positive volume, unmatched boundary
 * face, rank-deficient stencil), HGKS_ENOMEM. */
int hgks_mesh_create(const hgks_mesh_desc* desc, hgks_mesh** out);

/* Free a mesh that was never handed to hgks_init.  NULL is ignored. */
void hgks_mesh_destroy(hgks_mesh* mesh);

/* Cell volumes and time-step length scales 3|cell|/|surface| ([n_cells] host
 * each, caller order; either pointer may be NULL), e.g. for volume-weighted
 * error norms or hgks_cfl_dt_noalloc. */
int hgks_mesh_geometry(const hgks_mesh* mesh, double* vol_out, double* hdt_out);

/* Copy a built mesh (host memory only), e.g. to start several solvers on the
 * same geometry without rebuilding it.  Errors: HGKS_EINVAL, HGKS_ENOMEM. */
int hgks_mesh_clone(const hgks_mesh* mesh, hgks_mesh** out);

/* Mesh facts: what = 0 cells, 1 faces, 2 boundary ghosts, 3 padded big
 * stencil size, 4 sub-stencil count, 5 device bytes hgks_init would allocate
 * for precision 0, 6 the same for precision 1, 7 of these the bytes of the
 * static mesh arrays (a device mesh, hgks_dmesh_create), 8 and 9 the bytes of
 * one solver's own state and work arrays for precision 0 and 1.  Returns -1
 * for bad input. */
int64_t hgks_mesh_info(const hgks_mesh* mesh, int what);

/* Create a solver: copy the mesh and the initial cell averages q0
 * ([n_cells][5] host, caller order) to the device.  On HGKS_OK the solver owns
 * the mesh (do not destroy it separately); on failure the caller still owns
 * it.  Device memory: a device mesh (hgks_mesh_info(., 7) bytes) and the
 * solver's arrays (8 | 9), both from the device's stream-ordered memory pool
 * on the solver's stream.  The library raises the pool's release threshold,
 * so freed blocks stay with the process for reuse (cudaMemPoolTrimTo returns
 * them). */
int hgks_init(hgks_mesh* mesh, const hgks_params* params, const double* q0, hgks_solver** out);

/* Device mesh: the static arrays of a built mesh (geometry, connectivity,
 * stencils, pseudo-inverses, face quadrature) in device memory, immutable and
 * shared by any number of solvers (no counterpart in the paper: the serving
 * loop keeps one per geometry resident).  hgks_dmesh_create copies; the host
 * mesh stays with the caller.  stream: the cudaStream_t to copy on (NULL: a
 * library stream); returns after the copies complete.  Reference counted:
 * the device memory is released when hgks_dmesh_release has been called and
 * every solver over the mesh destroyed.  Errors: HGKS_EINVAL, HGKS_ENOMEM,
 * HGKS_ECUDA. */
int hgks_dmesh_create(const hgks_mesh* mesh, void* stream, hgks_dmesh** out);
void hgks_dmesh_release(hgks_dmesh* dmesh);
/* what = 0 cells, 1 faces, 2 boundary ghosts, 5 device bytes of the mesh
 * arrays, 6 and 7 device bytes of one solver's own arrays over it for
 * precision 0 and 1, 8 solvers currently over it.  -1 for bad input. */
int64_t hgks_dmesh_info(const hgks_dmesh* dmesh, int what);
/* Create a solver over a device mesh: only the solver's state and work
 * arrays are allocated (hgks_dmesh_info(., 6 | 7) bytes) and only q0 is
 * copied.  Otherwise as hgks_init; the device mesh is not consumed. */
int hgks_init_shared(hgks_dmesh* dmesh, const hgks_params* params, const double* q0, hgks_solver** out);

/* Batched solver (no counterpart in the paper; the batching of many small
 * meshes into one launch per kernel): the n meshes form one disjoint union,
 * so every kernel launch of a step covers all of them, while each member keeps
 * its own time, CFL step, step counter and status.  All meshes must have the
 * same cell type.  q0[i] is member i's [n_cells_i][5] state in its caller
 * order.  On HGKS_OK the solver owns (and frees) all the meshes; on failure
 * the caller still owns them.  hgks_step advances every member; members whose
 * t_end is reached stop.  hgks_read / hgks_write address member 0. */
int hgks_batch_init(hgks_mesh* const* meshes, int n, const hgks_params* params, const double* const* q0,
                    hgks_solver** out);

/* Number of member meshes of a solver (1 for hgks_init), or -1. */
int hgks_members(const hgks_solver* s);

/* Replace the state with q ([n_cells][5] host, caller order) at time t and
 * reset the step counter (restart / resume).  Synchronises.  The states are
 * copied as they are (pinned host memory copies fastest) and put into the
 * internal cell order on the device; hgks_read does the reverse. */
int hgks_write(hgks_solver* s, const double* q, double t);

/* hgks_write / hgks_read for one member of a batched solver. */
int hgks_member_write(hgks_solver* s, int member, const double* q, double t);
int hgks_member_read(hgks_solver* s, int member, double* q_out, double* t_out, int64_t* steps_out);

/* Non-blocking: 1 if all queued work of the solver has finished, 0 if some
 * is still running, a negative code on error. */
int hgks_query(hgks_solver* s);

/* Kernel variants in use (see hgks_params.autotune): flux_variant 0 one
 * thread per face / 1 one thread per Gauss point; recon_variant 0 staged /
 * 1 direct. */
int hgks_tuning(const hgks_solver* s, int* flux_variant, int* recon_variant);
/* Select the variants by hand (0 or 1 each); synchronises. */
int hgks_set_tuning(hgks_solver* s, int flux_variant, int recon_variant);

/* Device bytes the solver uses (its own arrays and its device mesh, which
 * may be shared), or -1. */
int64_t hgks_solver_bytes(const hgks_solver* s);

/* Advance n_steps S2O4 steps asynchronously on the solver's stream (Algorithm
 * 2: time step, then two stages of reconstruction, flux and update).
 * dt_fixed > 0 uses that step; otherwise the CFL step above.  t_end > 0 clips
 * the last step to land on t_end; steps after t_end do nothing.  No host
 * synchronisation; device-side faults surface at hgks_read / hgks_sync. */
int hgks_step(hgks_solver* s, int n_steps, double t_end, double dt_fixed);

/* Wait for queued work; return HGKS_ENONFINITE if a step produced a
 * non-finite average, HGKS_ECUDA on a runtime error. */
int hgks_sync(hgks_solver* s);

/* Synchronise and copy out the state ([n_cells][5] host, caller order), the
 * time and the number of steps taken since init/write.  Any pointer may be
 * NULL.  Returns the hgks_sync status. */
int hgks_read(hgks_solver* s, double* q_out, double* t_out, int64_t* steps_out);

/* One stage operator of the current state (Eq. finite with Section 2.2):
 * L = dQ/dt and dL/dt ([n_cells][5] host each, caller order) for step dt.
 * Test and diagnostic entry point; synchronises. */
int hgks_stage_operator(hgks_solver* s, double dt, double* L_out, double* dL_out);

/* Diagnostic: advance n_steps steps without graph replay, timing the kernel
 * groups of each step with CUDA events on the solver's stream.  ms_out[4]
 * receives the average milliseconds per step spent in: the time-step
 * finalisation, ghost filling plus reconstruction (both stages), the face
 * flux (both stages) and the two S2O4 updates.  Synchronises every step. */
int hgks_profile(hgks_solver* s, int n_steps, double t_end, double dt_fixed, double* ms_out);

/* Test hooks for the failure paths (no counterpart in the paper).
 * hgks_test_barrier_limit: the clock cycles a grid barrier of the persistent
 * launch (hgks_params.persistent) waits before it gives up, for the solver's
 * later hgks_step calls; cycles < 0 restores the default 2^31 (about a
 * second).  A barrier that gives up ends the launch, and hgks_sync /
 * hgks_read return HGKS_ETIMEOUT until hgks_write resets the state.
 * Synchronises.  Errors: HGKS_EINVAL (NULL solver).
 * hgks_test_fail_alloc: the library's n-th device allocation from now on
 * (n = 0: the next one) fails as an exhausted memory pool would, so the
 * creating call returns HGKS_ENOMEM and releases what it had taken; n < 0
 * switches the hook off.  Process-wide; returns HGKS_OK.
 * hgks_test_erfcx: y[i] = erfcx(x[i]) = exp(x^2) erfc(x) as the binary64 flux
 * computes it (its half-line Maxwellian moments, Section 2.1), for x >= 0
 * or NaN; x and y are host arrays of n values, owned by the caller.
 * Synchronises.  Errors: HGKS_EINVAL (n < 0, NULL arrays), HGKS_ENOMEM,
 * HGKS_ECUDA. */
int hgks_test_barrier_limit(hgks_solver* s, int64_t cycles);
int hgks_test_fail_alloc(int n);
int hgks_test_erfcx(const double* x, double* y, int64_t n);

/* Largest n_cells accepted by hgks_cfl_dt_noalloc. */
#define HGKS_NOALLOC_MAX_CELLS 4194304

/* The CFL time step of a state the caller holds on the device, computed
 * without allocating anything.  For callers that cannot allocate device
 * memory when they need the step: hosts whose device memory belongs to
 * another allocator that forbids foreign cudaMalloc/cudaFree calls, and loops
 * that cannot accept the device-wide synchronisation of cudaFree.  The paper
 * has no counterpart; it is the time-step reduction of hgks_step with its
 * scratch moved into a fixed device array inside the library.
 *   q       device pointer, [n_cells][5] conservative cell averages
 *   hdt     device pointer, [n_cells] length scales 3|cell|/|surface|
 *           (hgks_mesh_geometry gives them in caller order)
 *   params  host pointer, checked as hgks_init checks it (HGKS_EINVAL);
 *           gamma, cfl, mu_ref, T_ref, visc_exp are used
 *   dt_out  device pointer to one double: cfl min_i of the bound documented
 *           for hgks_params.cfl, written by the GPU, stream-ordered.  NaN if
 *           some cell has no bound: a non-finite value, or a non-positive
 *           density or pressure.
 *   stream  cudaStream_t to launch on (NULL: the legacy default stream)
 * The bound is always evaluated in binary64.  It equals the step hgks_step
 * takes for an HGKS_FP64 solver; an HGKS_FP32_MIXED solver evaluates its
 * bound in binary32 from its binary32 state copy, so its step can differ by
 * about 1e-7 relative.
 * Scratch: a file-scope 16384-double (128 KiB) device array, one per GPU that
 * loads the library, held until the process exits; n_cells above
 * HGKS_NOALLOC_MAX_CELLS is rejected with HGKS_EINVAL.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress), so make
 * that first call before any stream capture.  All calls share the array:
 * calls that overlap on the GPU (other streams, other threads) race and must
 * be ordered by the caller.  Calls no cudaMalloc, cudaFree or allocating
 * library routine; returns after queueing two kernels. */
int hgks_cfl_dt_noalloc(const double* q, const double* hdt, int64_t n_cells, const hgks_params* params,
                        double* dt_out, void* stream);

/* Free the solver, its mesh and its device memory.  NULL is ignored. */
void hgks_destroy(hgks_solver* s);

/* Message of the last failure on this thread ("" if none). */
const char* hgks_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HGKS_H */

// hgks_oracle.cpp -- plain, slow, FP64 CPU statement of the high-order
// gas-kinetic scheme (HGKS) step on 3D unstructured tet/hex/prism meshes.
//
// TEST INFRASTRUCTURE ONLY.  This file is the oracle for the GPU library: it
// shares no code with it, and only the test-suite, the smoke check and the
// CPU-baseline leg of the benchmark may build, load or call it.  Every routine
// cites the part of the paper (arXiv 2407.00656) it restates.
//
// Structure (paper order):
//   * mesh connectivity, two-layer stencils        Section 3.1, Algorithm 1
//   * WENO reconstruction (big and sub-stencils)   Section 2.3, Eqs. polys/weno
//   * gas-kinetic flux at Gauss points             Section 2.1, Eqs. flux, flux-G
//   * linear-in-time flux fit, S2O4 update         Section 2.2
//   * time step                                    Algorithm 2
//
// Readings where the paper is silent are marked "READING:" in place.
//
// Pins: the tests check these routines against brute-force velocity-space
// quadrature, closed forms (Euler and Navier-Stokes limits, S2O4 on a linear
// ODE), exact reconstruction of linear/quadratic data, free-stream
// preservation, conservation and the convergence order on the exact
// density-wave solution, on tetrahedra, full hexahedra and prisms (prism
// volumes, centroids and moments against their three tetrahedra; the hybrid
// shell's volume against the divergence theorem).  The smoothness indicators
// and nonlinear weights are pinned on tetrahedra and hexahedra by Gauss
// quadrature of the squared derivatives and independent least-squares fits
// over the paper's sub-stencils; the wall's far side at a Gauss point by the
// hand-built mirror image and the symmetry it implies (no mass or energy
// through the wall).  Parity unpinned (readings checked only for
// consistency): the time-step formula, the numerical collision time
// coefficient, the far-field/wall ghost-cell maps used inside stencils, the
// WENO epsilon and the prism's repeated corner sub-stencil.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// --------------------------------------------------------------------------
// Parameters (flattened double array on the C interface)
// --------------------------------------------------------------------------
struct Params {
  double gamma = 1.4;
  double mu_ref = 0.0;     // dynamic viscosity at T_ref (0: inviscid)
  double T_ref = 1.0;      // reference temperature, T = p/rho
  double visc_exp = 0.0;   // mu = mu_ref (T/T_ref)^visc_exp
  double Pr = 1.0;         // Prandtl number
  double cfl = 0.4;
  double tau_c = 0.0;      // numerical collision time coefficient
  double eps = 1e-8;       // WENO epsilon
  double glin = 0.025;     // linear weight of every sub-stencil
  double qinf[5] = {1, 0, 0, 0, 2.5};
  double Kint() const { return (5.0 - 3.0 * gamma) / (gamma - 1.0); }
};

// --------------------------------------------------------------------------
// Small dense helpers
// --------------------------------------------------------------------------
using V3 = std::array<double, 3>;
static V3 sub(const V3& a, const V3& b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
static V3 add(const V3& a, const V3& b) { return {a[0] + b[0], a[1] + b[1], a[2] + b[2]}; }
static V3 scl(const V3& a, double s) { return {a[0] * s, a[1] * s, a[2] * s}; }
static double dot(const V3& a, const V3& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static V3 cross(const V3& a, const V3& b) {
  return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
static double norm(const V3& a) { return std::sqrt(dot(a, a)); }

// Solve the n x n system A x = b (row-major A) by Gaussian elimination with
// partial pivoting.  Returns false for a singular matrix.
static bool solve_dense(int n, std::vector<double> A, std::vector<double> b, double* x) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[p * n + k])) p = i;
    if (A[p * n + k] == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
    x[i] = s / A[i * n + i];
  }
  return true;
}

// Least-squares pseudo-inverse of a tall m x n matrix A (row-major, m >= n)
// by Householder QR: A = Q R, pinv = R^{-1} Q^T restricted to n rows.
// Returns false if rank < n (|R_jj| below rel_tol * max|R_jj|).
static bool householder_pinv(int m, int n, const std::vector<double>& Ain, std::vector<double>& pinv,
                             double rel_tol = 1e-10) {
  std::vector<double> A = Ain;                 // m x n, overwritten with R
  std::vector<double> Qt(m * m, 0.0);          // accumulates Q^T
  for (int i = 0; i < m; ++i) Qt[i * m + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    double nrm = 0.0;
    for (int i = k; i < m; ++i) nrm += A[i * n + k] * A[i * n + k];
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    double alpha = A[k * n + k] > 0 ? -nrm : nrm;
    std::vector<double> v(m, 0.0);
    for (int i = k; i < m; ++i) v[i] = A[i * n + k];
    v[k] -= alpha;
    double vv = 0.0;
    for (int i = k; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = k; i < m; ++i) s += v[i] * A[i * n + j];
      s = 2.0 * s / vv;
      for (int i = k; i < m; ++i) A[i * n + j] -= s * v[i];
    }
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int i = k; i < m; ++i) s += v[i] * Qt[i * m + j];
      s = 2.0 * s / vv;
      for (int i = k; i < m; ++i) Qt[i * m + j] -= s * v[i];
    }
  }
  double rmax = 0.0;
  for (int k = 0; k < n; ++k) rmax = std::max(rmax, std::fabs(A[k * n + k]));
  for (int k = 0; k < n; ++k)
    if (!(std::fabs(A[k * n + k]) > rel_tol * rmax)) return false;
  // back-substitute R X = (Q^T)[0:n, :]
  pinv.assign(n * m, 0.0);
  for (int j = 0; j < m; ++j) {
    for (int i = n - 1; i >= 0; --i) {
      double s = Qt[i * m + j];
      for (int l = i + 1; l < n; ++l) s -= A[i * n + l] * pinv[l * m + j];
      pinv[i * m + j] = s / A[i * n + i];
    }
  }
  return true;
}

// --------------------------------------------------------------------------
// Velocity-space polynomials and Maxwellian moments (Section 2.1)
//
// A polynomial is a list of terms c * u^e0 v^e1 w^e2 (xi^2)^e3, where xi^2
// sums the K internal degrees of freedom.  Under a Maxwellian the three
// velocity components and xi are independent, so the moment of a monomial is
// the product of one-dimensional moments.
// --------------------------------------------------------------------------
struct Term { int e[4]; double c; };
constexpr int PMAX = 40;
struct Poly {
  int n = 0;
  Term t[PMAX];
  void push(const Term& x) {
    if (n >= PMAX) { std::fprintf(stderr, "oracle: polynomial too long\n"); std::abort(); }
    t[n++] = x;
  }
};

static Poly mono(double c, int a, int b, int d, int x) { Poly p; p.push(Term{{a, b, d, x}, c}); return p; }
static Poly padd(const Poly& p, const Poly& q) { Poly r = p; for (int i = 0; i < q.n; ++i) r.push(q.t[i]); return r; }
static Poly pscale(const Poly& p, double s) { Poly r = p; for (int i = 0; i < r.n; ++i) r.t[i].c *= s; return r; }
static Poly pmul(const Poly& p, const Poly& q) {
  Poly r;
  for (int i = 0; i < p.n; ++i)
    for (int j = 0; j < q.n; ++j) {
      const Term& a = p.t[i];
      const Term& b = q.t[j];
      r.push(Term{{a.e[0] + b.e[0], a.e[1] + b.e[1], a.e[2] + b.e[2], a.e[3] + b.e[3]}, a.c * b.c});
    }
  return r;
}
// psi = (1, u, v, w, (u^2+v^2+w^2+xi^2)/2)
static Poly make_psi(int i) {
  switch (i) {
    case 0: return mono(1, 0, 0, 0, 0);
    case 1: return mono(1, 1, 0, 0, 0);
    case 2: return mono(1, 0, 1, 0, 0);
    case 3: return mono(1, 0, 0, 1, 0);
    default: {
      Poly p = mono(0.5, 2, 0, 0, 0);
      p = padd(p, mono(0.5, 0, 2, 0, 0));
      p = padd(p, mono(0.5, 0, 0, 2, 0));
      return padd(p, mono(0.5, 0, 0, 0, 1));
    }
  }
}
static const Poly& psi(int i) {
  static const Poly P[5] = {make_psi(0), make_psi(1), make_psi(2), make_psi(3), make_psi(4)};
  return P[i];
}
// a_1 + a_2 u + a_3 v + a_4 w + a_5 psi_5 : the micro-slope polynomial
static Poly slope_poly(const double* a) {
  Poly p;
  for (int i = 0; i < 5; ++i) p = padd(p, pscale(psi(i), a[i]));
  return p;
}

constexpr int NMU = 12;  // u^0 .. u^11
constexpr int NMX = 6;   // (xi^2)^0 .. (xi^2)^5

// Normalized moments <.> = (1/rho) int (.) g dXi of one Maxwellian.
struct Moments {
  double u[NMU], v[NMU], w[NMU], x[NMX];
  double gram[5][5];  // <psi_i psi_j>, filled by moments_of
  double at(int a, int b, int c, int d) const { return u[a] * v[b] * w[c] * x[d]; }
  // <p>, <p q>, <p q r>: moments of products, summed term by term
  double of(const Poly& p) const {
    double s = 0;
    for (int i = 0; i < p.n; ++i) s += p.t[i].c * at(p.t[i].e[0], p.t[i].e[1], p.t[i].e[2], p.t[i].e[3]);
    return s;
  }
  double of(const Poly& p, const Poly& q) const {
    double s = 0;
    for (int i = 0; i < p.n; ++i)
      for (int j = 0; j < q.n; ++j) {
        const Term& a = p.t[i];
        const Term& b = q.t[j];
        s += a.c * b.c * at(a.e[0] + b.e[0], a.e[1] + b.e[1], a.e[2] + b.e[2], a.e[3] + b.e[3]);
      }
    return s;
  }
  double of(const Poly& p, const Poly& q, const Poly& r) const {
    double s = 0;
    for (int i = 0; i < p.n; ++i)
      for (int j = 0; j < q.n; ++j)
        for (int k = 0; k < r.n; ++k) {
          const Term& a = p.t[i];
          const Term& b = q.t[j];
          const Term& c = r.t[k];
          s += a.c * b.c * c.c *
               at(a.e[0] + b.e[0] + c.e[0], a.e[1] + b.e[1] + c.e[1], a.e[2] + b.e[2] + c.e[2], a.e[3] + b.e[3] + c.e[3]);
        }
    return s;
  }
};

// Primitive variables of a Maxwellian: rho, U, V, W, lambda = 1/(2 R T).
struct Prim { double rho, U, V, W, lam; };

// rho E = rho |U|^2/2 + (K+3) rho /(4 lambda)  (Section 2.1, Maxwellian)
static Prim prim_of(const double* q, double K) {
  Prim p;
  p.rho = q[0];
  p.U = q[1] / q[0];
  p.V = q[2] / q[0];
  p.W = q[3] / q[0];
  double kin = 0.5 * p.rho * (p.U * p.U + p.V * p.V + p.W * p.W);
  p.lam = (K + 3.0) * p.rho / (4.0 * (q[4] - kin));
  return p;
}

// One-dimensional Gaussian moments of the normalized Maxwellian in one
// velocity component with mean U and inverse temperature lam.
// half = 0: full line; +1: u > 0; -1: u < 0.
//   full:  <u^0> = 1,  <u^1> = U
//   u>0:   <u^0> = erfc(-sqrt(lam) U)/2,  <u^1> = U <u^0> + exp(-lam U^2)/(2 sqrt(pi lam))
//   u<0:   <u^0> = erfc( sqrt(lam) U)/2,  <u^1> = U <u^0> - exp(-lam U^2)/(2 sqrt(pi lam))
//   all:   <u^(n+2)> = U <u^(n+1)> + (n+1)/(2 lam) <u^n>   (integration by parts)
static void gauss_moments(double U, double lam, int half, double* m) {
  if (half == 0) {
    m[0] = 1.0;
    m[1] = U;
  } else {
    double s = std::sqrt(lam) * U;
    double e = std::exp(-lam * U * U) / (2.0 * std::sqrt(M_PI * lam));
    if (half > 0) {
      m[0] = 0.5 * std::erfc(-s);
      m[1] = U * m[0] + e;
    } else {
      m[0] = 0.5 * std::erfc(s);
      m[1] = U * m[0] - e;
    }
  }
  for (int n = 0; n + 2 < NMU; ++n) m[n + 2] = U * m[n + 1] + (n + 1) / (2.0 * lam) * m[n];
}

// Moments of the Maxwellian, with the normal component u full or half-line.
// Internal degrees of freedom: <xi^(2d)> = prod_{j<d} (K + 2j)/(2 lam).
static Moments moments_of(const Prim& p, double K, int half) {
  Moments M;
  gauss_moments(p.U, p.lam, half, M.u);
  gauss_moments(p.V, p.lam, 0, M.v);
  gauss_moments(p.W, p.lam, 0, M.w);
  M.x[0] = 1.0;
  for (int d = 1; d < NMX; ++d) M.x[d] = M.x[d - 1] * (K + 2.0 * (d - 1)) / (2.0 * p.lam);
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) M.gram[i][j] = M.of(psi(i), psi(j));
  return M;
}

// Micro-slope a (coefficients on psi) from normalized derivative b = dQ/rho:
// solve sum_j <psi_i psi_j> a_j = b_i  (Section 2.1, "<a^k> = dQ_k/dn").
static void micro_slope(const Moments& M, const double* b, double* a) {
  std::vector<double> A(25), rhs(5);
  for (int i = 0; i < 5; ++i) {
    for (int j = 0; j < 5; ++j) A[i * 5 + j] = M.gram[i][j];
    rhs[i] = b[i];
  }
  if (!solve_dense(5, A, rhs, a))
    for (int i = 0; i < 5; ++i) a[i] = NAN;
}

// Rotation of a conservative 5-vector into / out of the frame (n, t1, t2).
struct Frame { V3 n, t1, t2; };
static Frame frame_of(const V3& n) {
  // t1 = normalize(n x e_k), k = argmin |n_k|; t2 = n x t1.  Any orthonormal
  // completion gives the same flux (the Maxwellian is isotropic).
  int k = 0;
  for (int i = 1; i < 3; ++i) if (std::fabs(n[i]) < std::fabs(n[k])) k = i;
  V3 e = {0, 0, 0};
  e[k] = 1.0;
  V3 t1 = cross(n, e);
  t1 = scl(t1, 1.0 / norm(t1));
  V3 t2 = cross(n, t1);
  return Frame{n, t1, t2};
}
static void to_local(const Frame& f, const double* q, double* o) {
  V3 m = {q[1], q[2], q[3]};
  o[0] = q[0]; o[1] = dot(m, f.n); o[2] = dot(m, f.t1); o[3] = dot(m, f.t2); o[4] = q[4];
}
static void to_global(const Frame& f, const double* o, double* q) {
  q[0] = o[0];
  for (int a = 0; a < 3; ++a) q[1 + a] = o[1] * f.n[a] + o[2] * f.t1[a] + o[3] * f.t2[a];
  q[4] = o[4];
}

// --------------------------------------------------------------------------
// Gas-kinetic flux in the local frame (Section 2.1, Eq. flux; Section 2.2)
//
// ql, qr: left (u>0 side) and right conservative states at the Gauss point;
// dql[j], dqr[j]: their derivatives along the local directions n, t1, t2.
// Returns the flux fit F^n and its slope dF (Eq. expansion-1).
// --------------------------------------------------------------------------
struct FluxOut { double F[5], dF[5]; };

static double visc_mu(const Params& P, double T) {
  if (P.mu_ref == 0.0) return 0.0;
  if (P.visc_exp == 0.0) return P.mu_ref;
  return P.mu_ref * std::pow(T / P.T_ref, P.visc_exp);  // Section 5.2 power law
}

static FluxOut gks_flux_local(const Params& P, const double* ql, const double dql[3][5], const double* qr,
                              const double dqr[3][5], double dt) {
  const double K = P.Kint();
  Prim pl = prim_of(ql, K), pr = prim_of(qr, K);
  Moments Ml_pos = moments_of(pl, K, +1), Mr_neg = moments_of(pr, K, -1);
  Moments Ml = moments_of(pl, K, 0), Mr = moments_of(pr, K, 0);

  // Interface equilibrium: Q0 = int_{u>0} psi g_l + int_{u<0} psi g_r
  double q0[5];
  for (int i = 0; i < 5; ++i) q0[i] = pl.rho * Ml_pos.of(psi(i)) + pr.rho * Mr_neg.of(psi(i));
  Prim p0 = prim_of(q0, K);
  Moments M0 = moments_of(p0, K, 0);

  // Micro-slopes of the two initial states: <a^k_j> = dQ_k/dn_j
  double al[3][5], ar[3][5];
  for (int j = 0; j < 3; ++j) {
    double bl[5], br[5];
    for (int i = 0; i < 5; ++i) { bl[i] = dql[j][i] / pl.rho; br[i] = dqr[j][i] / pr.rho; }
    micro_slope(Ml, bl, al[j]);
    micro_slope(Mr, br, ar[j]);
  }
  // READING: dQ0/dn_j by differentiating the compatibility relation for Q0:
  // dQ0/dn_j = int_{u>0} psi a^l_j g_l + int_{u<0} psi a^r_j g_r.
  double abar[3][5];
  for (int j = 0; j < 3; ++j) {
    Poly Pl = slope_poly(al[j]), Pr = slope_poly(ar[j]);
    double b0[5];
    for (int i = 0; i < 5; ++i)
      b0[i] = (pl.rho * Ml_pos.of(psi(i), Pl) + pr.rho * Mr_neg.of(psi(i), Pr)) / p0.rho;
    micro_slope(M0, b0, abar[j]);
  }
  // a.u = a_1 u + a_2 v + a_3 w with each a_j a polynomial in psi
  auto adotu = [](const double a[3][5]) {
    Poly p = pmul(mono(1, 1, 0, 0, 0), slope_poly(a[0]));
    p = padd(p, pmul(mono(1, 0, 1, 0, 0), slope_poly(a[1])));
    return padd(p, pmul(mono(1, 0, 0, 1, 0), slope_poly(a[2])));
  };
  // Time slope A from <a.u + A> = 0 (moments of the same Maxwellian)
  auto time_slope = [&](const Moments& M, const double a[3][5], double* A) {
    Poly au = adotu(a);
    double b[5];
    for (int i = 0; i < 5; ++i) b[i] = -M.of(au, psi(i));
    micro_slope(M, b, A);
  };
  double Abar[5], Al[5], Ar[5];
  time_slope(M0, abar, Abar);

  // Collision time.  READING: tau = mu(T0)/p0 + C dt |p_l - p_r|/(p_l + p_r)
  double p0p = p0.rho / (2.0 * p0.lam);
  double plp = pl.rho / (2.0 * pl.lam), prp = pr.rho / (2.0 * pr.lam);
  double T0 = 1.0 / (2.0 * p0.lam);
  double tau = visc_mu(P, T0) / p0p + P.tau_c * dt * std::fabs(plp - prp) / (plp + prp);
  if (tau > 0.0) {
    time_slope(Ml, al, Al);
    time_slope(Mr, ar, Ar);
  } else {
    for (int i = 0; i < 5; ++i) Al[i] = Ar[i] = 0.0;
  }

  Poly U1 = mono(1, 1, 0, 0, 0);
  Poly au0 = adotu(abar), aul = adotu(al), aur = adotu(ar);
  Poly A0p = slope_poly(Abar), Alp = slope_poly(Al), Arp = slope_poly(Ar);

  // Time integral over [0,T] of the flux carried by Eq. (flux)
  auto integral = [&](double T, double* I) {
    double c1, c2, c3, c4, c5;
    if (tau == 0.0) {  // limits tau -> 0
      c1 = T; c2 = 0.0; c3 = 0.5 * T * T; c4 = 0.0; c5 = 0.0;
    } else {
      double e = std::exp(-T / tau);
      c1 = T - tau * (1.0 - e);                                  // int (1-e^{-t/tau})
      c2 = -tau * T * (1.0 + e) + 2.0 * tau * tau * (1.0 - e);   // int ((t+tau)e^{-t/tau} - tau)
      c3 = 0.5 * T * T - tau * T + tau * tau * (1.0 - e);        // int (t - tau + tau e^{-t/tau})
      c4 = tau * (1.0 - e);                                      // int e^{-t/tau}
      c5 = 2.0 * tau * tau * (1.0 - e) - tau * T * e;            // int (t+tau) e^{-t/tau}
    }
    for (int i = 0; i < 5; ++i) {
      Poly up = pmul(U1, psi(i));
      double s = p0.rho * (c1 * M0.of(up) + c2 * M0.of(up, au0) + c3 * M0.of(up, A0p));
      if (c4 != 0.0 || c5 != 0.0) {
        s += pl.rho * (c4 * Ml_pos.of(up) - c5 * Ml_pos.of(up, aul) - tau * c4 * Ml_pos.of(up, Alp));
        s += pr.rho * (c4 * Mr_neg.of(up) - c5 * Mr_neg.of(up, aur) - tau * c4 * Mr_neg.of(up, Arp));
      }
      I[i] = s;
    }
    // READING (Prandtl number fix): add (1/Pr - 1) q to the energy flux, q the
    // first-order heat flux int (u-U0) (|u-U0|^2+xi^2)/2 f carried by the
    // equilibrium part f = g0 (1 - tau (abar.u + Abar)), integrated over [0,T].
    if (P.Pr != 1.0 && tau > 0.0) {
      Poly cu = padd(U1, mono(-p0.U, 0, 0, 0, 0));
      Poly cv = padd(mono(1, 0, 1, 0, 0), mono(-p0.V, 0, 0, 0, 0));
      Poly cw = padd(mono(1, 0, 0, 1, 0), mono(-p0.W, 0, 0, 0, 0));
      Poly c2p = padd(padd(pmul(cu, cu), pmul(cv, cv)), padd(pmul(cw, cw), mono(1, 0, 0, 0, 1)));
      double q = -tau * T * p0.rho * M0.of(cu, pscale(c2p, 0.5), padd(au0, A0p));
      I[4] += (1.0 / P.Pr - 1.0) * q;
    }
  };
  double I1[5], Ih[5];
  integral(dt, I1);
  integral(0.5 * dt, Ih);
  // F dt + dF dt^2/2 = I(dt),  F dt/2 + dF dt^2/8 = I(dt/2)   (Section 2.2)
  FluxOut out;
  for (int i = 0; i < 5; ++i) {
    out.F[i] = (4.0 * Ih[i] - I1[i]) / dt;
    out.dF[i] = 4.0 * (I1[i] - 2.0 * Ih[i]) / (dt * dt);
  }
  return out;
}

// Flux through a unit normal n in the global frame, from global-frame point
// values and gradients g[v][3] on both sides.
static FluxOut gks_flux_global(const Params& P, const V3& n, const double* ql, const double gl[5][3],
                               const double* qr, const double gr[5][3], double dt) {
  Frame fr = frame_of(n);
  const V3 dirs[3] = {fr.n, fr.t1, fr.t2};
  double qlL[5], qrL[5], dl[3][5], dr[3][5];
  to_local(fr, ql, qlL);
  to_local(fr, qr, qrL);
  for (int j = 0; j < 3; ++j) {
    double dgl[5], dgr[5];
    for (int v = 0; v < 5; ++v) {
      dgl[v] = gl[v][0] * dirs[j][0] + gl[v][1] * dirs[j][1] + gl[v][2] * dirs[j][2];
      dgr[v] = gr[v][0] * dirs[j][0] + gr[v][1] * dirs[j][1] + gr[v][2] * dirs[j][2];
    }
    to_local(fr, dgl, dl[j]);
    to_local(fr, dgr, dr[j]);
  }
  FluxOut loc = gks_flux_local(P, qlL, dl, qrL, dr, dt);
  FluxOut g;
  to_global(fr, loc.F, g.F);
  to_global(fr, loc.dF, g.dF);
  return g;
}

// --------------------------------------------------------------------------
// Boundary maps (Section 5.2: Riemann-invariant far field, no-slip
// adiabatic wall).  READING: the wall state mirrors the interior with all
// momentum negated; the far-field state follows the 1D Riemann invariants
// along the outward normal n with entropy and tangential velocity taken from
// the upwind side; supersonic normal flow takes the upwind state whole.
// --------------------------------------------------------------------------
static void wall_state(const double* q, double* o) {
  o[0] = q[0]; o[1] = -q[1]; o[2] = -q[2]; o[3] = -q[3]; o[4] = q[4];
}
static void farfield_state(const Params& P, const V3& n, const double* q, double* o) {
  const double g = P.gamma;
  auto primv = [&](const double* s, double& rho, V3& u, double& p) {
    rho = s[0];
    u = {s[1] / rho, s[2] / rho, s[3] / rho};
    p = (g - 1.0) * (s[4] - 0.5 * rho * dot(u, u));
  };
  double ri, pi, re, pe;
  V3 ui, ue;
  primv(q, ri, ui, pi);
  primv(P.qinf, re, ue, pe);
  double ci = std::sqrt(g * pi / ri), ce = std::sqrt(g * pe / re);
  double uni = dot(ui, n), une = dot(ue, n);
  if (uni >= ci) {  // supersonic outflow
    for (int i = 0; i < 5; ++i) o[i] = q[i];
    return;
  }
  if (uni <= -ci) {  // supersonic inflow
    for (int i = 0; i < 5; ++i) o[i] = P.qinf[i];
    return;
  }
  double Rp = uni + 2.0 * ci / (g - 1.0);
  double Rm = une - 2.0 * ce / (g - 1.0);
  double un = 0.5 * (Rp + Rm);
  double c = 0.25 * (g - 1.0) * (Rp - Rm);
  double s;
  V3 ut;
  if (un > 0.0) {
    s = pi / std::pow(ri, g);
    ut = sub(ui, scl(n, uni));
  } else {
    s = pe / std::pow(re, g);
    ut = sub(ue, scl(n, une));
  }
  double rho = std::pow(c * c / (g * s), 1.0 / (g - 1.0));
  double p = rho * c * c / g;
  V3 u = add(ut, scl(n, un));
  o[0] = rho;
  o[1] = rho * u[0]; o[2] = rho * u[1]; o[3] = rho * u[2];
  o[4] = p / (g - 1.0) + 0.5 * rho * dot(u, u);
}

// --------------------------------------------------------------------------
// Mesh (Section 3.1)
// --------------------------------------------------------------------------
enum { BC_PERIODIC = 1, BC_FARFIELD = 2, BC_WALL = 3 };

// Local faces: tet face p is opposite node p; hex faces 1 and 6 are the
// bottom and top quads, faces 2..5 go round the sides cyclically, so that
// the octant sub-stencils of Section 2.3 read {face 1|6, side m, side m+1}.
static const int TET_FACE[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
static const int HEX_FACE[6][4] = {{0, 1, 2, 3}, {0, 1, 5, 4}, {1, 2, 6, 5},
                                   {2, 3, 7, 6}, {3, 0, 4, 7}, {4, 5, 6, 7}};

struct Face {
  int nn = 0;
  int nodes[4];
  int owner = -1, nbr = -1;  // nbr < 0 for a physical boundary
  int bc = 0;                // 0 interior, else BC tag
  V3 shift = {0, 0, 0};      // neighbour image = neighbour + shift
  int ng = 0;
  V3 xg[4];                  // Gauss points
  V3 ng_[4];                 // unit normals (owner -> neighbour)
  double wa[4];              // weight * local area
  V3 centroid, nmean;        // for mirrors: plane point and unit mean normal
};

// One member of a stencil as seen from the target cell.
struct Ref {
  int kind = 0;    // 0: cell (maybe a periodic image), 1: ghost, -1: none (collapsed face)
  int id = -1;     // cell index (for ghosts: the interior cell mirrored)
  int face = -1;   // ghost: boundary face of the mirror
  V3 shift = {0, 0, 0};
  bool same(const Ref& o) const {
    if (kind != o.kind || id != o.id || face != o.face) return false;
    for (int a = 0; a < 3; ++a) if (std::fabs(shift[a] - o.shift[a]) > 1e-9) return false;
    return true;
  }
};

struct Cell {
  int type;           // 4 or 8
  bool prism = false; // type 8 with nodes 2 = 3 and 6 = 7 (a triangular prism)
  int nodes[8];
  double vol, h, hdt;
  V3 cen;
  double mom[6];      // central second moments: xx yy zz xy yz zx (averages)
  int face[6];        // -1: the collapsed side of a prism (no face)
  int side[6];        // +1 owner, -1 neighbour
  Ref nb[6];
  std::vector<Ref> big;                // big stencil, excluding the cell itself
  std::vector<std::vector<int>> sub;   // sub-stencils as indices into big
  std::vector<double> pinv0;           // 9 x K
  std::vector<std::vector<double>> pinvm;  // 3 x k_m each
};

struct Solver {
  Params P;
  std::vector<V3> X;
  std::vector<Cell> C;
  std::vector<Face> F;
  std::vector<double> Q;  // [nc][5]
  double t = 0.0;
  int64_t steps = 0;
  // per-stage reconstruction: a[c][v][9], b[c][v][m][3], wbar[c][v][M+1]
  std::vector<double> ra, rb, rw;
  int Mmax = 8;
  bool force_linear = false;
  std::string err;
};

static void mom_tet(const V3 p[4], double& vol, V3& cen, double* mom) {
  V3 a = sub(p[1], p[0]), b = sub(p[2], p[0]), c = sub(p[3], p[0]);
  vol = dot(cross(a, b), c) / 6.0;
  cen = scl(add(add(p[0], p[1]), add(p[2], p[3])), 0.25);
  // central second moments of a tetrahedron: (1/20) sum_v d_v d_v^T, d = x_v - c
  for (int k = 0; k < 6; ++k) mom[k] = 0.0;
  const int ia[6] = {0, 1, 2, 0, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 0};
  for (int v = 0; v < 4; ++v) {
    V3 d = sub(p[v], cen);
    for (int k = 0; k < 6; ++k) mom[k] += d[ia[k]] * d[ib[k]] / 20.0;
  }
}

// Trilinear hex: volume, centroid, second moments by 3x3x3 Gauss-Legendre
// (exact: the integrands are polynomials of degree <= 4 per direction).
static void mom_hex(const V3 p[8], double& vol, V3& cen, double* mom) {
  const double gx[3] = {0.5 - 0.5 * std::sqrt(0.6), 0.5, 0.5 + 0.5 * std::sqrt(0.6)};
  const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  struct QP { V3 x; double w; };
  std::vector<QP> qp;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        double s = gx[i], t = gx[j], r = gx[k];
        double N[8] = {(1 - s) * (1 - t) * (1 - r), s * (1 - t) * (1 - r), s * t * (1 - r), (1 - s) * t * (1 - r),
                       (1 - s) * (1 - t) * r,       s * (1 - t) * r,       s * t * r,       (1 - s) * t * r};
        double dNs[8] = {-(1 - t) * (1 - r), (1 - t) * (1 - r), t * (1 - r), -t * (1 - r),
                         -(1 - t) * r,       (1 - t) * r,       t * r,       -t * r};
        double dNt[8] = {-(1 - s) * (1 - r), -s * (1 - r), s * (1 - r), (1 - s) * (1 - r),
                         -(1 - s) * r,       -s * r,       s * r,       (1 - s) * r};
        double dNr[8] = {-(1 - s) * (1 - t), -s * (1 - t), -s * t, -(1 - s) * t,
                         (1 - s) * (1 - t),  s * (1 - t),  s * t,  (1 - s) * t};
        V3 x = {0, 0, 0}, xs = {0, 0, 0}, xt = {0, 0, 0}, xr = {0, 0, 0};
        for (int a = 0; a < 8; ++a) {
          x = add(x, scl(p[a], N[a]));
          xs = add(xs, scl(p[a], dNs[a]));
          xt = add(xt, scl(p[a], dNt[a]));
          xr = add(xr, scl(p[a], dNr[a]));
        }
        qp.push_back(QP{x, gw[i] * gw[j] * gw[k] * dot(cross(xs, xt), xr)});
      }
  vol = 0.0;
  cen = {0, 0, 0};
  for (auto& q : qp) { vol += q.w; cen = add(cen, scl(q.x, q.w)); }
  cen = scl(cen, 1.0 / vol);
  const int ia[6] = {0, 1, 2, 0, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 0};
  for (int k = 0; k < 6; ++k) mom[k] = 0.0;
  for (auto& q : qp) {
    V3 d = sub(q.x, cen);
    for (int k = 0; k < 6; ++k) mom[k] += q.w * d[ia[k]] * d[ib[k]];
  }
  for (int k = 0; k < 6; ++k) mom[k] /= vol;
}

// Face quadrature.  READING: triangles use the 3-point degree-2 rule
// (barycentric (2/3,1/6,1/6) and permutations, weight 1/3); quads use 2x2
// Gauss-Legendre on the bilinear patch with per-point area vectors.
static void face_geometry(Solver& S, Face& f) {
  V3 p[4];
  for (int a = 0; a < f.nn; ++a) p[a] = S.X[f.nodes[a]];
  if (f.nn == 3) {
    V3 av = scl(cross(sub(p[1], p[0]), sub(p[2], p[0])), 0.5);
    double area = norm(av);
    V3 n = scl(av, 1.0 / area);
    const double B[3][3] = {{2.0 / 3, 1.0 / 6, 1.0 / 6}, {1.0 / 6, 2.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 6, 2.0 / 3}};
    f.ng = 3;
    for (int g = 0; g < 3; ++g) {
      f.xg[g] = add(add(scl(p[0], B[g][0]), scl(p[1], B[g][1])), scl(p[2], B[g][2]));
      f.ng_[g] = n;
      f.wa[g] = area / 3.0;
    }
    f.centroid = scl(add(add(p[0], p[1]), p[2]), 1.0 / 3.0);
    f.nmean = n;
  } else {
    const double gq[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
    f.ng = 4;
    V3 asum = {0, 0, 0}, csum = {0, 0, 0};
    double wsum = 0.0;
    int g = 0;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j, ++g) {
        double s = gq[i], t = gq[j];
        V3 x = add(add(scl(p[0], (1 - s) * (1 - t)), scl(p[1], s * (1 - t))), add(scl(p[2], s * t), scl(p[3], (1 - s) * t)));
        V3 xs = add(scl(sub(p[1], p[0]), 1 - t), scl(sub(p[2], p[3]), t));
        V3 xt = add(scl(sub(p[3], p[0]), 1 - s), scl(sub(p[2], p[1]), s));
        V3 av = scl(cross(xs, xt), 0.25);
        double a = norm(av);
        f.xg[g] = x;
        f.ng_[g] = scl(av, 1.0 / a);
        f.wa[g] = a;
        asum = add(asum, av);
        csum = add(csum, scl(x, a));
        wsum += a;
      }
    f.centroid = scl(csum, 1.0 / wsum);
    f.nmean = scl(asum, 1.0 / norm(asum));
  }
}

static void flip_face(Face& f) {
  for (int g = 0; g < f.ng; ++g) f.ng_[g] = scl(f.ng_[g], -1.0);
  f.nmean = scl(f.nmean, -1.0);
}

static V3 mirror_point(const Face& f, const V3& x) {
  double d = dot(sub(x, f.centroid), f.nmean);
  return sub(x, scl(f.nmean, 2.0 * d));
}

// Geometry of a stencil member as seen from the target: centroid and
// central second moments (periodic images translate, ghosts reflect).
static void ref_geometry(const Solver& S, const Ref& r, V3& cen, double* mom) {
  const Cell& c = S.C[r.id];
  if (r.kind == 0) {
    cen = add(c.cen, r.shift);
    for (int k = 0; k < 6; ++k) mom[k] = c.mom[k];
    return;
  }
  const Face& f = S.F[r.face];
  cen = add(mirror_point(f, c.cen), r.shift);
  // M' = R M R, R = I - 2 n n^T
  double Mf[3][3] = {{c.mom[0], c.mom[3], c.mom[5]}, {c.mom[3], c.mom[1], c.mom[4]}, {c.mom[5], c.mom[4], c.mom[2]}};
  double R[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) R[a][b] = (a == b ? 1.0 : 0.0) - 2.0 * f.nmean[a] * f.nmean[b];
  double T[3][3] = {{0}}, O[3][3] = {{0}};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int k = 0; k < 3; ++k) T[a][b] += R[a][k] * Mf[k][b];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int k = 0; k < 3; ++k) O[a][b] += T[a][k] * R[k][b];
  mom[0] = O[0][0]; mom[1] = O[1][1]; mom[2] = O[2][2]; mom[3] = O[0][1]; mom[4] = O[1][2]; mom[5] = O[2][0];
}

// Cell average of a stencil member: the interior value, or the boundary
// map of the mirrored cell (ghost cells of Algorithm 1).
static void ref_state(const Solver& S, const std::vector<double>& Q, const Ref& r, double* q) {
  const double* s = &Q[5 * r.id];
  if (r.kind == 0) { for (int i = 0; i < 5; ++i) q[i] = s[i]; return; }
  const Face& f = S.F[r.face];
  if (f.bc == BC_WALL) wall_state(s, q);
  else farfield_state(S.P, f.nmean, s, q);
}

// Neighbour of `from` across its local face p, composed with the image shift
// of `from` itself.
static Ref neighbour_of(const Solver& S, const Ref& from, int p) {
  Ref r = S.C[from.id].nb[p];
  r.shift = add(r.shift, from.shift);
  return r;
}

static bool build_mesh(Solver& S, int64_t n_nodes, const double* xyz, int64_t n_cells, const int32_t* ctype,
                       int32_t default_type, const int64_t* cell_ptr, const int64_t* cell_nodes, int64_t n_bf,
                       const int64_t* bf_nodes, const int32_t* bf_tag, const double* periods) {
  S.X.resize(n_nodes);
  for (int64_t i = 0; i < n_nodes; ++i) S.X[i] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
  S.C.resize(n_cells);
  for (int64_t c = 0; c < n_cells; ++c) {
    Cell& cl = S.C[c];
    cl.type = ctype ? ctype[c] : default_type;
    int64_t base = cell_ptr ? cell_ptr[c] : c * (int64_t)cl.type;
    if (cl.type != 4 && cl.type != 8) { S.err = "unsupported cell type"; return false; }
    for (int a = 0; a < cl.type; ++a) cl.nodes[a] = (int)cell_nodes[base + a];
    if (cl.type == 8) {
      // READING (prisms; the paper defines hexahedra and tetrahedra only): a
      // triangular prism is given as a hexahedron with nodes 2 = 3 and 6 = 7;
      // its side face 4 (nodes 2 3 7 6) collapses to an edge and is dropped.
      int distinct = 0;
      for (int a = 0; a < 8; ++a) {
        bool seen = false;
        for (int b = 0; b < a; ++b) seen = seen || cl.nodes[b] == cl.nodes[a];
        distinct += !seen;
      }
      cl.prism = cl.nodes[2] == cl.nodes[3] && cl.nodes[6] == cl.nodes[7];
      if (distinct != (cl.prism ? 6 : 8)) { S.err = "unsupported degenerate hexahedron"; return false; }
    }
    V3 p[8];
    for (int a = 0; a < cl.type; ++a) p[a] = S.X[cl.nodes[a]];
    if (cl.type == 4) mom_tet(p, cl.vol, cl.cen, cl.mom);
    else mom_hex(p, cl.vol, cl.cen, cl.mom);
    if (!(cl.vol > 0.0)) { S.err = "non-positive cell volume"; return false; }
    cl.h = std::cbrt(cl.vol);
  }
  // faces keyed by sorted node tuples (CellFace / FaceCell of Section 3.1)
  std::map<std::array<int, 4>, int> fmap;
  for (int64_t c = 0; c < n_cells; ++c) {
    Cell& cl = S.C[c];
    int nf = cl.type == 4 ? 4 : 6;
    for (int p = 0; p < nf; ++p) {
      Face f;
      f.nn = cl.type == 4 ? 3 : 4;
      for (int a = 0; a < f.nn; ++a) f.nodes[a] = cl.nodes[cl.type == 4 ? TET_FACE[p][a] : HEX_FACE[p][a]];
      if (cl.prism) {
        if (p == 3) { cl.face[p] = -1; cl.side[p] = 0; continue; }  // collapsed to the edge 2-6
        // the prism's bottom and top quads (nodes 0 1 2 2, 4 5 6 6) are
        // triangles: drop the repeated node
        int nn = 0;
        for (int a = 0; a < 4; ++a)
          if (nn == 0 || (f.nodes[a] != f.nodes[nn - 1] && (a < 3 || f.nodes[a] != f.nodes[0]))) f.nodes[nn++] = f.nodes[a];
        f.nn = nn;
      }
      std::array<int, 4> key = {-1, -1, -1, -1};
      for (int a = 0; a < f.nn; ++a) key[a] = f.nodes[a];
      std::sort(key.begin(), key.begin() + f.nn);
      auto it = fmap.find(key);
      if (it == fmap.end()) {
        f.owner = (int)c;
        face_geometry(S, f);
        if (dot(sub(f.centroid, cl.cen), f.nmean) < 0) flip_face(f);
        fmap[key] = (int)S.F.size();
        cl.face[p] = (int)S.F.size();
        cl.side[p] = +1;
        S.F.push_back(f);
      } else {
        Face& g = S.F[it->second];
        if (g.nbr >= 0) { S.err = "face shared by more than two cells"; return false; }
        g.nbr = (int)c;
        cl.face[p] = it->second;
        cl.side[p] = -1;
      }
    }
  }
  // boundary tags
  std::map<std::array<int, 4>, int> btag;
  for (int64_t b = 0; b < n_bf; ++b) {
    std::array<int, 4> key = {-1, -1, -1, -1};
    int nn = 0;
    for (int a = 0; a < 4; ++a) if (bf_nodes[4 * b + a] >= 0) key[nn++] = (int)bf_nodes[4 * b + a];
    std::sort(key.begin(), key.begin() + nn);
    btag[key] = bf_tag[b];
  }
  // periodic pairing of unmatched faces by translated centroid
  std::vector<int> open;
  for (int f = 0; f < (int)S.F.size(); ++f) if (S.F[f].nbr < 0) open.push_back(f);
  auto qkey = [](const V3& x) {
    return std::make_tuple((long long)std::llround(x[0] * 1e7), (long long)std::llround(x[1] * 1e7),
                           (long long)std::llround(x[2] * 1e7));
  };
  std::map<std::tuple<long long, long long, long long>, int> cmap;
  if (periods) for (int f : open) cmap[qkey(S.F[f].centroid)] = f;
  std::vector<char> dead(S.F.size(), 0);
  for (int f : open) {
    if (dead[f] || S.F[f].nbr >= 0) continue;
    Face& fa = S.F[f];
    std::array<int, 4> key = {-1, -1, -1, -1};
    for (int a = 0; a < fa.nn; ++a) key[a] = fa.nodes[a];
    std::sort(key.begin(), key.begin() + fa.nn);
    auto bt = btag.find(key);
    if (bt != btag.end() && bt->second != BC_PERIODIC) { fa.bc = bt->second; continue; }
    bool paired = false;
    if (periods) {
      for (int ax = 0; ax < 3 && !paired; ++ax)
        for (int sg = -1; sg <= 1 && !paired; sg += 2) {
          if (periods[ax] <= 0) continue;
          V3 tgt = fa.centroid;
          tgt[ax] += sg * periods[ax];
          auto it = cmap.find(qkey(tgt));
          if (it == cmap.end() || it->second == f || dead[it->second]) continue;
          Face& gb = S.F[it->second];
          // the partner's owner becomes our neighbour, seen translated by -sg*L
          fa.nbr = gb.owner;
          fa.bc = 0;
          fa.shift = {0, 0, 0};
          fa.shift[ax] = -sg * periods[ax];
          Cell& oc = S.C[gb.owner];
          int nf = oc.type == 4 ? 4 : 6;
          for (int p = 0; p < nf; ++p)
            if (oc.face[p] == it->second) { oc.face[p] = f; oc.side[p] = -1; }
          dead[it->second] = 1;
          paired = true;
        }
    }
    if (!paired) {
      if (bt == btag.end()) { S.err = "boundary face without a tag or periodic partner"; return false; }
      fa.bc = bt->second;
    }
  }
  // compact faces (drop the consumed periodic partners)
  std::vector<int> remap(S.F.size(), -1);
  std::vector<Face> nfv;
  for (int f = 0; f < (int)S.F.size(); ++f) if (!dead[f]) { remap[f] = (int)nfv.size(); nfv.push_back(S.F[f]); }
  S.F.swap(nfv);
  for (auto& cl : S.C) {
    int nf = cl.type == 4 ? 4 : 6;
    for (int p = 0; p < nf; ++p)
      if (cl.face[p] >= 0) cl.face[p] = remap[cl.face[p]];
  }
  // CellNeighbor (Section 3.1, item 3); boundary faces give ghost members
  for (int c = 0; c < (int)S.C.size(); ++c) {
    Cell& cl = S.C[c];
    int nf = cl.type == 4 ? 4 : 6;
    double area = 0.0;
    for (int p = 0; p < nf; ++p) {
      if (cl.face[p] < 0) { cl.nb[p].kind = -1; continue; }
      const Face& f = S.F[cl.face[p]];
      for (int g = 0; g < f.ng; ++g) area += f.wa[g];
      Ref r;
      if (f.nbr < 0) {
        r.kind = 1; r.id = c; r.face = cl.face[p];
      } else if (cl.side[p] > 0) {
        r.kind = 0; r.id = f.nbr; r.shift = f.shift;
      } else {
        r.kind = 0; r.id = f.owner; r.shift = scl(f.shift, -1.0);
      }
      cl.nb[p] = r;
    }
    cl.hdt = 3.0 * cl.vol / area;  // READING: time-step length scale 3|cell|/|surface|
  }
  return true;
}

// Two-layer stencils (Algorithm 1) and sub-stencils (Section 2.3).
static bool build_stencils(Solver& S) {
  Ref self;
  for (int c = 0; c < (int)S.C.size(); ++c) {
    Cell& cl = S.C[c];
    int nf = cl.type == 4 ? 4 : 6;
    self.kind = 0; self.id = c; self.face = -1; self.shift = {0, 0, 0};
    auto find_or_add = [&](const Ref& r) -> int {
      if (r.kind < 0 || r.same(self)) return -1;
      for (int k = 0; k < (int)cl.big.size(); ++k) if (cl.big[k].same(r)) return k;
      cl.big.push_back(r);
      return (int)cl.big.size() - 1;
    };
    cl.big.clear();
    for (int p = 0; p < nf; ++p) find_or_add(cl.nb[p]);
    // second layer: neighbours of every (non-ghost) first-layer cell
    for (int p = 0; p < nf; ++p) {
      const Ref& r = cl.nb[p];
      if (r.kind != 0) continue;
      int nf2 = S.C[r.id].type == 4 ? 4 : 6;
      for (int q = 0; q < nf2; ++q) find_or_add(neighbour_of(S, r, q));
    }
    auto idx = [&](const Ref& r) {
      if (r.kind < 0) return -1;
      for (int k = 0; k < (int)cl.big.size(); ++k) if (cl.big[k].same(r)) return k;
      return -1;
    };
    cl.sub.clear();
    if (cl.type == 4) {
      // S_m = {i, three face neighbours, the other neighbours of neighbour m}
      const int SETS[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {2, 0, 3}};
      for (int m = 0; m < 4; ++m) {
        std::vector<int> s;
        auto push = [&](int k) { if (k >= 0 && std::find(s.begin(), s.end(), k) == s.end()) s.push_back(k); };
        for (int a = 0; a < 3; ++a) push(idx(cl.nb[SETS[m][a]]));
        const Ref& r = cl.nb[m];
        if (r.kind == 0) {
          int nf2 = S.C[r.id].type == 4 ? 4 : 6;
          for (int q = 0; q < nf2; ++q) {
            Ref r2 = neighbour_of(S, r, q);
            if (r2.same(self)) continue;
            push(idx(r2));
          }
        }
        cl.sub.push_back(s);
      }
    } else {
      // octants: {i, face 1 or 6, sides (m, m+1)}.  READING (prisms): the
      // two octants at the collapsed edge (sides 2-3 and 3-4) both take the
      // sides 2 and 4 that meet there, so a prism has the six corner
      // stencils of its vertices, the one at the collapsed edge twice.
      for (int top = 0; top < 2; ++top)
        for (int m = 0; m < 4; ++m) {
          std::vector<int> s;
          int s1 = 1 + m, s2 = 1 + (m + 1) % 4;
          if (cl.prism && (m == 1 || m == 2)) { s1 = 2; s2 = 4; }
          s.push_back(idx(cl.nb[top ? 5 : 0]));
          s.push_back(idx(cl.nb[s1]));
          s.push_back(idx(cl.nb[s2]));
          cl.sub.push_back(s);
        }
    }
    // least-squares pseudo-inverses (Section 2.3): coordinates centred on
    // the cell centroid and scaled by h = |cell|^(1/3).
    // Basis order: x y z xx yy zz xy yz zx, each minus its average over the cell.
    const int K = (int)cl.big.size();
    std::vector<double> A0(K * 9), Al(K * 3);
    const double h = cl.h;
    for (int k = 0; k < K; ++k) {
      V3 cen;
      double mom[6];
      ref_geometry(S, cl.big[k], cen, mom);
      V3 d = scl(sub(cen, cl.cen), 1.0 / h);
      double m2[6];
      for (int j = 0; j < 6; ++j) m2[j] = mom[j] / (h * h);
      double mi[6];
      for (int j = 0; j < 6; ++j) mi[j] = cl.mom[j] / (h * h);
      // averages over member k of the zero-mean basis functions
      double row[9] = {d[0], d[1], d[2],
                       m2[0] + d[0] * d[0] - mi[0], m2[1] + d[1] * d[1] - mi[1], m2[2] + d[2] * d[2] - mi[2],
                       m2[3] + d[0] * d[1] - mi[3], m2[4] + d[1] * d[2] - mi[4], m2[5] + d[2] * d[0] - mi[5]};
      for (int j = 0; j < 9; ++j) A0[k * 9 + j] = row[j];
      for (int j = 0; j < 3; ++j) Al[k * 3 + j] = row[j];
    }
    if (K < 9 || !householder_pinv(K, 9, A0, cl.pinv0)) { S.err = "rank-deficient big stencil"; return false; }
    cl.pinvm.clear();
    for (auto& s : cl.sub) {
      int km = (int)s.size();
      std::vector<double> A(km * 3), pv;
      for (int r = 0; r < km; ++r)
        for (int j = 0; j < 3; ++j) A[r * 3 + j] = Al[s[r] * 3 + j];
      if (km < 3 || !householder_pinv(km, 3, A, pv)) { S.err = "rank-deficient sub-stencil"; return false; }
      cl.pinvm.push_back(pv);
    }
  }
  return true;
}

// --------------------------------------------------------------------------
// WENO reconstruction (Section 2.3, Eqs. polys and weno)
// --------------------------------------------------------------------------
static void reconstruct_all(Solver& S, const std::vector<double>& Q) {
  const int nc = (int)S.C.size();
  const int MM = S.Mmax;
  S.ra.assign((size_t)nc * 5 * 9, 0.0);
  S.rb.assign((size_t)nc * 5 * MM * 3, 0.0);
  S.rw.assign((size_t)nc * 5 * (MM + 1), 0.0);
#pragma omp parallel for schedule(dynamic, 64)
  for (int c = 0; c < nc; ++c) {
    const Cell& cl = S.C[c];
    const int K = (int)cl.big.size();
    const int M = (int)cl.sub.size();
    std::vector<double> dq(K * 5);
    for (int k = 0; k < K; ++k) {
      double q[5];
      ref_state(S, Q, cl.big[k], q);
      for (int v = 0; v < 5; ++v) dq[k * 5 + v] = q[v] - Q[5 * c + v];
    }
    const double g0 = 1.0 - S.P.glin * M;
    const double vol = cl.vol, h = cl.h;
    for (int v = 0; v < 5; ++v) {
      // quadratic P0 and linear Pm by least squares
      double a[9];
      for (int d = 0; d < 9; ++d) {
        double s = 0;
        for (int k = 0; k < K; ++k) s += cl.pinv0[d * K + k] * dq[k * 5 + v];
        a[d] = s;
      }
      std::vector<double> b(M * 3);
      for (int m = 0; m < M; ++m) {
        int km = (int)cl.sub[m].size();
        for (int d = 0; d < 3; ++d) {
          double s = 0;
          for (int r = 0; r < km; ++r) s += cl.pinvm[m][d * km + r] * dq[cl.sub[m][r] * 5 + v];
          b[m * 3 + d] = s;
        }
      }
      // smoothness indicators in physical coordinates:
      // beta = sum_{|l|=1}^{r} |cell|^(2|l|/3-1) int_cell (d^l P)^2 dV
      // P0 = Q + sum a_d (xi^d - avg xi^d), xi = (x - c)/h.
      // d/dx_a P0 = (a_a + sum_b H_ab xi_b)/h with Hessian H (in xi):
      double H[3][3] = {{2 * a[3], a[6], a[8]}, {a[6], 2 * a[4], a[7]}, {a[8], a[7], 2 * a[5]}};
      double Mi[3][3] = {{cl.mom[0], cl.mom[3], cl.mom[5]}, {cl.mom[3], cl.mom[1], cl.mom[4]},
                         {cl.mom[5], cl.mom[4], cl.mom[2]}};
      double beta0 = 0.0;
      for (int ax = 0; ax < 3; ++ax) {
        // int (a_a + H_a.xi)^2 dV / h^2 = vol (a_a^2 + H_a^T (Mi/h^2) H_a)/h^2
        double quad = 0.0;
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) quad += H[ax][p] * Mi[p][q] / (h * h) * H[ax][q];
        double integ = vol * (a[ax] * a[ax] + quad) / (h * h);
        beta0 += std::pow(vol, 2.0 / 3.0 - 1.0) * integ;
      }
      // |l| = 2: xx yy zz xy yz zx, each counted once; d^l P0 = H_l / h^2
      const int la[6] = {0, 1, 2, 0, 1, 2}, lb[6] = {0, 1, 2, 1, 2, 0};
      for (int l = 0; l < 6; ++l) {
        double d2 = H[la[l]][lb[l]] / (h * h);
        beta0 += std::pow(vol, 4.0 / 3.0 - 1.0) * vol * d2 * d2;
      }
      std::vector<double> beta(M + 1);
      beta[0] = beta0;
      for (int m = 0; m < M; ++m) {
        double gsq = 0.0;
        for (int d = 0; d < 3; ++d) gsq += (b[m * 3 + d] / h) * (b[m * 3 + d] / h);
        beta[m + 1] = std::pow(vol, 2.0 / 3.0 - 1.0) * vol * gsq;
      }
      // WENO-Z type weights
      double tauZ = 0.0;
      for (int m = 1; m <= M; ++m) tauZ += std::fabs(beta[0] - beta[m]) / M;
      std::vector<double> w(M + 1);
      double wsum = 0.0;
      for (int m = 0; m <= M; ++m) {
        double gm = m == 0 ? g0 : S.P.glin;
        w[m] = gm * (1.0 + tauZ / (beta[m] + S.P.eps));
        wsum += w[m];
      }
      for (int m = 0; m <= M; ++m) w[m] /= wsum;
      if (S.force_linear)
        for (int m = 0; m <= M; ++m) w[m] = m == 0 ? g0 : S.P.glin;
      double* A = &S.ra[((size_t)c * 5 + v) * 9];
      for (int d = 0; d < 9; ++d) A[d] = a[d];
      double* Bp = &S.rb[((size_t)c * 5 + v) * MM * 3];
      for (int m = 0; m < M * 3; ++m) Bp[m] = b[m];
      double* W = &S.rw[((size_t)c * 5 + v) * (MM + 1)];
      for (int m = 0; m <= M; ++m) W[m] = w[m];
    }
  }
}

// Point value and gradient at x (in the cell's own coordinates) by Eq. weno:
// Q = wbar0 (P0/g0 - sum gm/g0 Pm) + sum wbar_m Pm.
static void recon_eval(const Solver& S, int c, const V3& x, double* val, double grad[5][3]) {
  const Cell& cl = S.C[c];
  const int M = (int)cl.sub.size();
  const int MM = S.Mmax;
  const double h = cl.h;
  V3 xi = scl(sub(x, cl.cen), 1.0 / h);
  double mi[6];
  for (int j = 0; j < 6; ++j) mi[j] = cl.mom[j] / (h * h);
  double basis[9] = {xi[0], xi[1], xi[2], xi[0] * xi[0] - mi[0], xi[1] * xi[1] - mi[1], xi[2] * xi[2] - mi[2],
                     xi[0] * xi[1] - mi[3], xi[1] * xi[2] - mi[4], xi[2] * xi[0] - mi[5]};
  // d basis / d xi_a
  double db[9][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1},
                     {2 * xi[0], 0, 0}, {0, 2 * xi[1], 0}, {0, 0, 2 * xi[2]},
                     {xi[1], xi[0], 0}, {0, xi[2], xi[1]}, {xi[2], 0, xi[0]}};
  const double g0 = 1.0 - S.P.glin * M;
  for (int v = 0; v < 5; ++v) {
    const double* a = &S.ra[((size_t)c * 5 + v) * 9];
    const double* b = &S.rb[((size_t)c * 5 + v) * MM * 3];
    const double* w = &S.rw[((size_t)c * 5 + v) * (MM + 1)];
    const double q = S.Q[5 * c + v];
    double P0 = q, G0[3] = {0, 0, 0};
    for (int d = 0; d < 9; ++d) {
      P0 += a[d] * basis[d];
      for (int ax = 0; ax < 3; ++ax) G0[ax] += a[d] * db[d][ax] / h;
    }
    double value = w[0] / g0 * P0, g[3];
    for (int ax = 0; ax < 3; ++ax) g[ax] = w[0] / g0 * G0[ax];
    for (int m = 0; m < M; ++m) {
      double Pm = q, Gm[3];
      for (int d = 0; d < 3; ++d) { Pm += b[m * 3 + d] * basis[d]; Gm[d] = b[m * 3 + d] / h; }
      double coef = w[m + 1] - w[0] * S.P.glin / g0;
      value += coef * Pm;
      for (int ax = 0; ax < 3; ++ax) g[ax] += coef * Gm[ax];
    }
    val[v] = value;
    for (int ax = 0; ax < 3; ++ax) grad[v][ax] = g[ax];
  }
}

// The far side of a boundary Gauss point with outward unit normal n, from
// the interior point value ql and gradient gl (Section 5.2).  READING: the
// no-slip adiabatic wall mirrors the interior across the face, so the state
// has all momentum negated and the gradient is reflected (its normal
// component changes sign) with the momentum rows negated too; the far field
// takes the Riemann-invariant state with zero gradient.
static void boundary_side(const Params& P, int bc, const V3& n, const double* ql, const double gl[5][3],
                          double* qr, double gr[5][3]) {
  if (bc == BC_WALL) {
    wall_state(ql, qr);
    for (int v = 0; v < 5; ++v) {
      double sgn = (v >= 1 && v <= 3) ? -1.0 : 1.0;
      V3 gv = {gl[v][0], gl[v][1], gl[v][2]};
      double dn = dot(gv, n);
      for (int ax = 0; ax < 3; ++ax) gr[v][ax] = sgn * (gv[ax] - 2.0 * dn * n[ax]);
    }
  } else {
    farfield_state(P, n, ql, qr);
    for (int v = 0; v < 5; ++v) for (int ax = 0; ax < 3; ++ax) gr[v][ax] = 0.0;
  }
}

// --------------------------------------------------------------------------
// One stage: reconstruct, fluxes (Eq. flux-G with Gaussian quadrature),
// operator L and dL/dt (Eq. finite).
// --------------------------------------------------------------------------
static void stage_operator(Solver& S, double dt, std::vector<double>& L, std::vector<double>& dL) {
  reconstruct_all(S, S.Q);
  const int nf = (int)S.F.size();
  std::vector<double> FF(nf * 5), FD(nf * 5);
#pragma omp parallel for schedule(dynamic, 64)
  for (int f = 0; f < nf; ++f) {
    const Face& fa = S.F[f];
    double Fs[5] = {0}, Ds[5] = {0};
    for (int g = 0; g < fa.ng; ++g) {
      double ql[5], gl[5][3], qr[5], gr[5][3];
      recon_eval(S, fa.owner, fa.xg[g], ql, gl);
      const V3& n = fa.ng_[g];
      if (fa.nbr >= 0) recon_eval(S, fa.nbr, sub(fa.xg[g], fa.shift), qr, gr);
      else boundary_side(S.P, fa.bc, n, ql, gl, qr, gr);
      FluxOut fo = gks_flux_global(S.P, n, ql, gl, qr, gr, dt);
      for (int v = 0; v < 5; ++v) { Fs[v] += fa.wa[g] * fo.F[v]; Ds[v] += fa.wa[g] * fo.dF[v]; }
    }
    for (int v = 0; v < 5; ++v) { FF[f * 5 + v] = Fs[v]; FD[f * 5 + v] = Ds[v]; }
  }
  const int nc = (int)S.C.size();
  L.assign(nc * 5, 0.0);
  dL.assign(nc * 5, 0.0);
  for (int c = 0; c < nc; ++c) {
    const Cell& cl = S.C[c];
    int nfc = cl.type == 4 ? 4 : 6;
    for (int v = 0; v < 5; ++v) {
      double s = 0.0, d = 0.0;
      for (int p = 0; p < nfc; ++p) {
        if (cl.face[p] < 0) continue;
        s += cl.side[p] * FF[cl.face[p] * 5 + v];
        d += cl.side[p] * FD[cl.face[p] * 5 + v];
      }
      L[c * 5 + v] = -s / cl.vol;
      dL[c * 5 + v] = -d / cl.vol;
    }
  }
}

// READING: dt = cfl min_i h_i/(|U_i| + c_i), h_i = 3|cell|/|surface|; with
// viscosity also dt <= cfl min_i rho_i h_i^2 / (2 mu_i).
static double time_step(const Solver& S) {
  double dtm = INFINITY;
  const double g = S.P.gamma;
  for (int c = 0; c < (int)S.C.size(); ++c) {
    const double* q = &S.Q[5 * c];
    double rho = q[0], u = q[1] / rho, v = q[2] / rho, w = q[3] / rho;
    double p = (g - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + w * w));
    double a = std::sqrt(g * p / rho);
    double speed = std::sqrt(u * u + v * v + w * w) + a;
    double dti = S.C[c].hdt / speed;
    if (S.P.mu_ref > 0.0) {
      double mu = visc_mu(S.P, p / rho);
      dti = std::min(dti, rho * S.C[c].hdt * S.C[c].hdt / (2.0 * mu));
    }
    dtm = std::min(dtm, dti);
  }
  return S.P.cfl * dtm;
}

// Two-stage fourth-order update (Section 2.2) for any operator that returns
// L(Q) and dL/dt(Q) at the start of a stage:
//   Q*      = Q^n + dt/2 L(Q^n) + dt^2/8 dL(Q^n)
//   Q^{n+1} = Q^n + dt L(Q^n) + dt^2/6 (dL(Q^n) + 2 dL(Q*))
template <class Op>
static void s2o4(std::vector<double>& Q, double dt, Op op) {
  std::vector<double> Ln, dLn, Ls, dLs;
  std::vector<double> Q0 = Q;
  op(Q, Ln, dLn);
  for (size_t i = 0; i < Q.size(); ++i) Q[i] = Q0[i] + 0.5 * dt * Ln[i] + 0.125 * dt * dt * dLn[i];
  op(Q, Ls, dLs);
  for (size_t i = 0; i < Q.size(); ++i) Q[i] = Q0[i] + dt * Ln[i] + dt * dt / 6.0 * (dLn[i] + 2.0 * dLs[i]);
}

static int s2o4_step(Solver& S, double t_end, double dt_fixed) {
  double dt = dt_fixed > 0.0 ? dt_fixed : time_step(S);
  if (t_end > 0.0) dt = std::min(dt, t_end - S.t);
  if (!(dt > 0.0)) return 0;
  s2o4(S.Q, dt, [&](std::vector<double>& Q, std::vector<double>& L, std::vector<double>& dL) {
    (void)Q;  // the stage state lives in S.Q
    stage_operator(S, dt, L, dL);
  });
  S.t += dt;
  S.steps += 1;
  for (double x : S.Q) if (!std::isfinite(x)) return -5;
  return 0;
}

static void set_params(Params& P, const double* p) {
  P.gamma = p[0]; P.mu_ref = p[1]; P.T_ref = p[2]; P.visc_exp = p[3]; P.Pr = p[4];
  P.cfl = p[5]; P.tau_c = p[6]; P.eps = p[7]; P.glin = p[8];
  for (int i = 0; i < 5; ++i) P.qinf[i] = p[9 + i];
}

}  // namespace

// ==========================================================================
// C interface for the test-suite (ctypes)
// ==========================================================================
extern "C" {

// params: gamma, mu_ref, T_ref, visc_exp, Pr, cfl, tau_c, eps, glin, qinf[5]
void* o_create(int64_t n_nodes, const double* xyz, int64_t n_cells, const int32_t* ctype, int32_t default_type,
               const int64_t* cell_ptr, const int64_t* cell_nodes, int64_t n_bf, const int64_t* bf_nodes,
               const int32_t* bf_tag, const double* periods, const double* params, char* err, int errlen) {
  Solver* S = new Solver;
  set_params(S->P, params);
  bool ok = build_mesh(*S, n_nodes, xyz, n_cells, ctype, default_type, cell_ptr, cell_nodes, n_bf, bf_nodes, bf_tag,
                       periods) && build_stencils(*S);
  if (!ok) {
    if (err && errlen > 0) std::snprintf(err, errlen, "%s", S->err.c_str());
    delete S;
    return nullptr;
  }
  S->Q.assign(S->C.size() * 5, 0.0);
  return S;
}

void o_destroy(void* h) { delete static_cast<Solver*>(h); }

void o_set_params(void* h, const double* params) { set_params(static_cast<Solver*>(h)->P, params); }

void o_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}

int o_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int64_t o_n_faces(void* h) { return (int64_t)static_cast<Solver*>(h)->F.size(); }

void o_set_state(void* h, const double* q, double t) {
  Solver* S = static_cast<Solver*>(h);
  std::memcpy(S->Q.data(), q, S->Q.size() * sizeof(double));
  S->t = t;
  S->steps = 0;
}

void o_get_state(void* h, double* q, double* t, int64_t* steps) {
  Solver* S = static_cast<Solver*>(h);
  std::memcpy(q, S->Q.data(), S->Q.size() * sizeof(double));
  if (t) *t = S->t;
  if (steps) *steps = S->steps;
}

int o_step(void* h, int n, double t_end, double dt_fixed) {
  Solver* S = static_cast<Solver*>(h);
  for (int i = 0; i < n; ++i) {
    int rc = s2o4_step(*S, t_end, dt_fixed);
    if (rc) return rc;
  }
  return 0;
}

double o_time_step(void* h) { return time_step(*static_cast<Solver*>(h)); }

// vol[nc], cen[nc*3], mom[nc*6], hdt[nc]
void o_cell_geometry(void* h, double* vol, double* cen, double* mom, double* hdt) {
  Solver* S = static_cast<Solver*>(h);
  for (size_t c = 0; c < S->C.size(); ++c) {
    const Cell& cl = S->C[c];
    if (vol) vol[c] = cl.vol;
    if (cen) for (int a = 0; a < 3; ++a) cen[3 * c + a] = cl.cen[a];
    if (mom) for (int k = 0; k < 6; ++k) mom[6 * c + k] = cl.mom[k];
    if (hdt) hdt[c] = cl.hdt;
  }
}

// Big-stencil size and sub-stencil count of a cell.
void o_stencil_info(void* h, int c, int* K, int* M) {
  Solver* S = static_cast<Solver*>(h);
  *K = (int)S->C[c].big.size();
  *M = (int)S->C[c].sub.size();
}

// Stencil members: kind, id and image-shifted centroid of each.
void o_stencil(void* h, int c, int* kind, int* id, double* cen) {
  Solver* S = static_cast<Solver*>(h);
  const Cell& cl = S->C[c];
  for (size_t k = 0; k < cl.big.size(); ++k) {
    kind[k] = cl.big[k].kind;
    id[k] = cl.big[k].id;
    V3 x;
    double mom[6];
    ref_geometry(*S, cl.big[k], x, mom);
    for (int a = 0; a < 3; ++a) cen[3 * k + a] = x[a];
  }
}

// Reconstruct the current state (optionally with linear weights forced).
void o_reconstruct(void* h, int force_linear) {
  Solver* S = static_cast<Solver*>(h);
  S->force_linear = force_linear != 0;
  reconstruct_all(*S, S->Q);
  S->force_linear = false;
}
// WENO point value and gradient of cell c at x (after o_reconstruct).
void o_recon_eval(void* h, int c, const double* x, double* val, double* grad) {
  Solver* S = static_cast<Solver*>(h);
  double g[5][3];
  recon_eval(*S, c, V3{x[0], x[1], x[2]}, val, g);
  for (int v = 0; v < 5; ++v) for (int a = 0; a < 3; ++a) grad[v * 3 + a] = g[v][a];
}
// Normalized nonlinear weights of the last reconstruction: w[v][0..M]
void o_recon_weights(void* h, int c, double* w) {
  Solver* S = static_cast<Solver*>(h);
  int M = (int)S->C[c].sub.size();
  for (int v = 0; v < 5; ++v)
    for (int m = 0; m <= M; ++m) w[v * (M + 1) + m] = S->rw[((size_t)c * 5 + v) * (S->Mmax + 1) + m];
}

// One stage operator L, dL/dt of the current state with step dt.
void o_operator(void* h, double dt, double* L, double* dL) {
  Solver* S = static_cast<Solver*>(h);
  std::vector<double> a, b;
  stage_operator(*S, dt, a, b);
  std::memcpy(L, a.data(), a.size() * sizeof(double));
  std::memcpy(dL, b.data(), b.size() * sizeof(double));
}

// Gas-kinetic flux at one point (global frame).  gl, gr: [5][3] gradients.
void o_flux_point(const double* params, const double* n, const double* ql, const double* gl, const double* qr,
                  const double* gr, double dt, double* F, double* dF) {
  Params P;
  set_params(P, params);
  double GL[5][3], GR[5][3];
  for (int v = 0; v < 5; ++v) for (int a = 0; a < 3; ++a) { GL[v][a] = gl[v * 3 + a]; GR[v][a] = gr[v * 3 + a]; }
  V3 nn = {n[0], n[1], n[2]};
  FluxOut o = gks_flux_global(P, nn, ql, GL, qr, GR, dt);
  for (int i = 0; i < 5; ++i) { F[i] = o.F[i]; dF[i] = o.dF[i]; }
}

// Flux at a boundary Gauss point exactly as the stage operator forms it:
// the far side from boundary_side (bc 2 far field, 3 wall), then the
// gas-kinetic flux.  gl: [5][3] interior gradient; qr_out, gr_out (may be
// NULL) receive the far side.
void o_boundary_flux(const double* params, int bc, const double* n, const double* ql, const double* gl, double dt,
                     double* F, double* dF, double* qr_out, double* gr_out) {
  Params P;
  set_params(P, params);
  double GL[5][3], GR[5][3], qr[5];
  for (int v = 0; v < 5; ++v) for (int a = 0; a < 3; ++a) GL[v][a] = gl[v * 3 + a];
  V3 nn = {n[0], n[1], n[2]};
  boundary_side(P, bc, nn, ql, GL, qr, GR);
  FluxOut o = gks_flux_global(P, nn, ql, GL, qr, GR, dt);
  for (int i = 0; i < 5; ++i) { F[i] = o.F[i]; dF[i] = o.dF[i]; }
  if (qr_out) for (int i = 0; i < 5; ++i) qr_out[i] = qr[i];
  if (gr_out) for (int v = 0; v < 5; ++v) for (int a = 0; a < 3; ++a) gr_out[v * 3 + a] = GR[v][a];
}

// Normalized 1D moments <u^k>, k < 12: half 0 full, +1 u>0, -1 u<0.
void o_gauss_moments(double U, double lam, int half, double* m) { gauss_moments(U, lam, half, m); }

// Micro-slope a from b for the Maxwellian of conservative state q.
void o_micro_slope(double gamma, const double* q, const double* b, double* a) {
  double K = (5.0 - 3.0 * gamma) / (gamma - 1.0);
  Prim p = prim_of(q, K);
  Moments M = moments_of(p, K, 0);
  micro_slope(M, b, a);
}

// The S2O4 routine above applied to dQ/dt = lam Q (L = lam Q, dL/dt = lam^2 Q).
void o_s2o4_linear(int n, double* q, double lam, double dt) {
  std::vector<double> Q(q, q + n);
  s2o4(Q, dt, [&](std::vector<double>& X, std::vector<double>& L, std::vector<double>& dL) {
    L.resize(X.size());
    dL.resize(X.size());
    for (size_t i = 0; i < X.size(); ++i) { L[i] = lam * X[i]; dL[i] = lam * lam * X[i]; }
  });
  for (int i = 0; i < n; ++i) q[i] = Q[i];
}

// Boundary states at a point: kind 2 far field, 3 wall.
void o_boundary_state(const double* params, int kind, const double* n, const double* q, double* o) {
  Params P;
  set_params(P, params);
  if (kind == BC_WALL) wall_state(q, o);
  else farfield_state(P, V3{n[0], n[1], n[2]}, q, o);
}

}  // extern "C"

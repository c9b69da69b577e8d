"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test compares the oracle with something other than itself: numerical
quadrature, closed forms from kinetic theory, analytic Euler / Navier-Stokes
fluxes, or the Taylor expansion of the exact solution.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from tests import bruteforce as B

GAMMA = 1.4
K_INT = (5 - 3 * GAMMA) / (GAMMA - 1)


def cons(rho, U, p, g=GAMMA):
    U = np.asarray(U, dtype=float)
    return np.array([rho, rho * U[0], rho * U[1], rho * U[2], p / (g - 1) + 0.5 * rho * U @ U])


def euler_flux(q, n, g=GAMMA):
    rho = q[0]
    U = q[1:4] / rho
    p = (g - 1) * (q[4] - 0.5 * rho * U @ U)
    un = U @ n
    return np.array([rho * un, *(rho * un * U + p * n), (q[4] + p) * un])


# ---------------------------------------------------------------------------
# Maxwellian moments (Section 2.1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("U,lam", [(0.3, 0.7), (-1.2, 0.45), (0.0, 2.0), (2.5, 0.5)])
def test_gauss_moments_match_quadrature(U, lam):
    """<u^n> over the full line and the two half-lines, by adaptive quadrature."""
    dens = lambda u: math.sqrt(lam / math.pi) * math.exp(-lam * (u - U) ** 2)
    full = oracle.gauss_moments(U, lam, 0)
    pos = oracle.gauss_moments(U, lam, +1)
    neg = oracle.gauss_moments(U, lam, -1)
    for n in range(12):
        ip, _ = integrate.quad(lambda u: u ** n * dens(u), 0, np.inf, epsabs=0, epsrel=1e-13, limit=200)
        im, _ = integrate.quad(lambda u: u ** n * dens(u), -np.inf, 0, epsabs=0, epsrel=1e-13, limit=200)
        scale = max(1.0, abs(ip) + abs(im))
        assert abs(pos[n] - ip) <= 1e-11 * scale
        assert abs(neg[n] - im) <= 1e-11 * scale
        assert abs(full[n] - (ip + im)) <= 1e-11 * scale
        assert abs(pos[n] + neg[n] - full[n]) <= 1e-12 * scale


def test_micro_slope_round_trip_and_closed_form():
    """<a psi> = b with Gram matrices by brute-force quadrature, and the
    closed-form inverse of the 5x5 moment system (Xu 2001)."""
    G = B.Grid(nu=24, nv=20, ns=24)
    rng = np.random.default_rng(11)
    for _ in range(3):
        q = cons(rng.uniform(0.8, 1.3), rng.uniform(-0.5, 0.5, 3), rng.uniform(0.7, 1.2))
        b = rng.normal(size=5)
        a = oracle.micro_slope(q, b)
        rho, U, lam = B.prim(q)
        g = G.maxwellian(rho, U, lam)
        gram = np.array([[G.integ(G.psi[i] * G.psi[k] * g) for k in range(5)] for i in range(5)]) / rho
        assert np.allclose(gram @ a, b, rtol=0, atol=1e-10 * np.abs(b).max())
        # closed form
        Uu, Vv, Ww = U
        K = K_INT
        R4 = 2 * b[4] - (Uu * Uu + Vv * Vv + Ww * Ww + (K + 3) / (2 * lam)) * b[0]
        R1, R2, R3 = b[1] - Uu * b[0], b[2] - Vv * b[0], b[3] - Ww * b[0]
        a5 = 4 * lam * lam / (K + 3) * (R4 - 2 * Uu * R1 - 2 * Vv * R2 - 2 * Ww * R3)
        a2, a3, a4 = 2 * lam * R1 - Uu * a5, 2 * lam * R2 - Vv * a5, 2 * lam * R3 - Ww * a5
        a1 = b[0] - Uu * a2 - Vv * a3 - Ww * a4 - 0.5 * a5 * (Uu * Uu + Vv * Vv + Ww * Ww + (K + 3) / (2 * lam))
        assert np.allclose(a, [a1, a2, a3, a4, a5], rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# Gas-kinetic flux (Eq. flux, Section 2.2) against brute-force quadrature
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def grid():
    return B.Grid()


@pytest.mark.parametrize("mu,Pr,tau_c", [(0.0, 1.0, 0.0), (0.015, 1.0, 0.0), (0.02, 0.72, 0.0), (0.0, 1.0, 1.0)])
def test_flux_matches_velocity_space_quadrature(grid, mu, Pr, tau_c):
    rng = np.random.default_rng(7)
    ql = cons(1.1, [0.3, -0.2, 0.1], 0.9)
    qr = cons(0.95, [0.25, -0.1, 0.15], 1.05)
    dql = rng.normal(size=(3, 5)) * 0.3
    dqr = rng.normal(size=(3, 5)) * 0.3
    dt = 0.05
    F, dF = B.bgk_flux(grid, ql, dql, qr, dqr, dt, mu=mu, Pr=Pr, tau_c=tau_c)
    Fo, dFo = oracle.flux_point([1, 0, 0], ql, dql.T, qr, dqr.T, dt, mu_ref=mu, Pr=Pr, tau_c=tau_c)
    assert np.abs(F - Fo).max() <= 1e-10 * np.abs(F).max()
    assert np.abs(dF - dFo).max() <= 1e-10 * np.abs(dF).max()


def _rot(axis_angle):
    v = np.asarray(axis_angle, dtype=float)
    th = np.linalg.norm(v)
    k = v / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * Kx + (1 - math.cos(th)) * Kx @ Kx


def _rotate_state(R, q):
    return np.array([q[0], *(R @ q[1:4]), q[4]])


def test_flux_is_rotation_covariant():
    """Flux through R n of R-rotated states equals R times the flux through n."""
    rng = np.random.default_rng(5)
    ql = cons(1.05, [0.2, 0.1, -0.3], 1.0)
    qr = cons(0.9, [0.1, 0.2, -0.2], 0.8)
    gl = rng.normal(size=(5, 3)) * 0.2
    gr = rng.normal(size=(5, 3)) * 0.2
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    R = _rot([0.4, -1.1, 0.7])

    def rot_grad(g):
        # scalar rows: rotate the derivative direction; momentum block: R M R^T
        out = np.empty_like(g)
        out[[0, 4]] = (R @ g[[0, 4]].T).T
        out[1:4] = R @ g[1:4] @ R.T
        return out

    for mu in (0.0, 0.01):
        F, dF = oracle.flux_point(n, ql, gl, qr, gr, 0.03, mu_ref=mu)
        F2, dF2 = oracle.flux_point(R @ n, _rotate_state(R, ql), rot_grad(gl), _rotate_state(R, qr),
                                    rot_grad(gr), 0.03, mu_ref=mu)
        assert np.allclose(F2, _rotate_state(R, F), rtol=1e-12, atol=1e-13)
        assert np.allclose(dF2, _rotate_state(R, dF), rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------------------
# Euler and Navier-Stokes limits (Chapman-Enskog, Section 2.1)
# ---------------------------------------------------------------------------
def test_euler_limit_uniform_state():
    n = np.array([2.0, -1.0, 0.5])
    n /= np.linalg.norm(n)
    q = cons(1.3, [0.4, -0.7, 0.2], 0.8)
    z = np.zeros((5, 3))
    F, dF = oracle.flux_point(n, q, z, q, z, 0.01)
    assert np.allclose(F, euler_flux(q, n), rtol=1e-13, atol=1e-14)
    assert np.abs(dF).max() < 1e-12


def _jac(fun, q, eps=1e-6):
    J = np.empty((5, 5))
    for k in range(5):
        dq = np.zeros(5)
        dq[k] = eps
        J[:, k] = (fun(q + dq) - fun(q - dq)) / (2 * eps)
    return J


def test_euler_limit_linear_data_time_derivative():
    """tau = 0, same linear field on both sides: dF/dt = J_n(Q) dQ/dt with
    dQ/dt = -sum_j J_j(Q) dQ/dx_j (J: analytic Euler flux Jacobians)."""
    rng = np.random.default_rng(2)
    q = cons(1.1, [0.5, -0.3, 0.2], 0.9)
    g = rng.normal(size=(5, 3)) * 0.1
    n = np.array([0.6, 0.0, 0.8])
    F, dF = oracle.flux_point(n, q, g, q, g, 0.02)
    E = np.eye(3)
    qt = -sum(_jac(lambda x: euler_flux(x, E[j]), q) @ g[:, j] for j in range(3))
    expect = _jac(lambda x: euler_flux(x, n), q) @ qt
    assert np.allclose(F, euler_flux(q, n), rtol=1e-13, atol=1e-13)
    assert np.allclose(dF, expect, rtol=1e-7, atol=1e-8)


def test_navier_stokes_limit_stress():
    """Constant rho and p, linear velocity, same on both sides, tau = mu/p:
    F^n = Euler flux - sigma.n (- U.sigma.n in energy) with the BGK stress
    sigma = tau p (dU_i/dx_j + dU_j/dx_i - 2/(K+3) delta_ij div U)."""
    rho, p = 1.2, 0.9
    U = np.array([0.3, -0.2, 0.5])
    gradU = np.array([[0.2, -0.1, 0.3], [0.05, -0.15, 0.1], [0.12, 0.07, 0.09]])  # dU_i/dx_j
    q = cons(rho, U, p)
    g = np.zeros((5, 3))
    g[1:4] = rho * gradU
    g[4] = rho * U @ gradU
    n = np.array([1.0, 2.0, -2.0]) / 3.0
    mu = 0.01
    F, dF = oracle.flux_point(n, q, g, q, g, 0.02, mu_ref=mu)
    tau = mu / p
    div = np.trace(gradU)
    sigma = tau * p * (gradU + gradU.T - 2.0 / (K_INT + 3) * div * np.eye(3))
    expect = euler_flux(q, n)
    expect[1:4] -= sigma @ n
    expect[4] -= U @ sigma @ n
    assert np.allclose(F, expect, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("Pr", [1.0, 0.72])
def test_navier_stokes_limit_heat_flux(Pr):
    """Zero velocity, constant p, density gradient (so T = p/rho varies):
    energy flux = -kappa dT/dn with kappa = mu c_p / Pr, c_p = (K+5)/2."""
    rho, p = 1.1, 1.0
    q = cons(rho, [0, 0, 0], p)
    grho = np.array([0.3, -0.2, 0.4])
    g = np.zeros((5, 3))
    g[0] = grho
    n = np.array([0.0, 0.6, 0.8])
    mu = 0.02
    F, dF = oracle.flux_point(n, q, g, q, g, 0.01, mu_ref=mu, Pr=Pr)
    gradT = -p * grho / rho ** 2
    cp = (K_INT + 5) / 2
    expect_E = -mu * cp / Pr * gradT @ n
    assert abs(F[4] - expect_E) < 1e-12
    assert np.allclose(F[1:4], p * n, atol=1e-13)
    assert abs(F[0]) < 1e-14


# ---------------------------------------------------------------------------
# S2O4 (Section 2.2) and boundary maps (Section 5.2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("z", [0.3, -0.8, 1.7])
def test_s2o4_is_fourth_order_taylor_for_linear_ode(z):
    """dQ/dt = lam Q with exact L and dL/dt: one step gives exp's Taylor
    polynomial of degree 4 in z = lam dt."""
    q = oracle.s2o4_linear(np.array([1.0, -2.5]), z, 1.0)
    taylor = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    assert np.allclose(q, np.array([1.0, -2.5]) * taylor, rtol=1e-15, atol=0)


def test_wall_state_mirrors_velocity():
    q = cons(1.2, [0.3, -0.4, 0.1], 0.7)
    o = oracle.boundary_state(3, [0, 0, 1.0], q)
    assert np.allclose(o, [q[0], -q[1], -q[2], -q[3], q[4]])


def test_farfield_state_riemann_invariants():
    g = GAMMA
    qinf = cons(1.0, [0.2535, 0, 0], 1 / g)
    n = np.array([0.6, 0.8, 0.0])
    # free stream maps to itself
    o = oracle.boundary_state(2, n, qinf, qinf=qinf)
    assert np.allclose(o, qinf, rtol=1e-13, atol=1e-14)
    # subsonic outflow: R+ from the interior, R- from the free stream, entropy
    # and tangential velocity from the interior
    p_i = 0.8
    qi = cons(1.1, [0.3, 0.25, 0.05], p_i)
    o = oracle.boundary_state(2, n, qi, qinf=qinf)
    ri, ui = qi[0], qi[1:4] / qi[0]
    ro, uo = o[0], o[1:4] / o[0]
    po = (g - 1) * (o[4] - 0.5 * ro * uo @ uo)
    c_i, c_o, c_e = math.sqrt(g * p_i / ri), math.sqrt(g * po / ro), 1.0
    assert uo @ n > 0
    assert abs((uo @ n + 2 * c_o / (g - 1)) - (ui @ n + 2 * c_i / (g - 1))) < 1e-12
    assert abs((uo @ n - 2 * c_o / (g - 1)) - (0.2535 * n[0] - 2 * c_e / (g - 1))) < 1e-12
    assert abs(po / ro ** g - p_i / ri ** g) < 1e-12
    assert np.allclose(uo - (uo @ n) * n, ui - (ui @ n) * n, atol=1e-13)

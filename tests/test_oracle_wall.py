"""Pins of the oracle's no-slip adiabatic wall (Section 5.2) at a face Gauss
point, by what the mirror construction fixes independently of the oracle.

The far side of a wall point is the interior mirrored across the face plane:
the state with all momentum negated, and the gradient reflected by
R = I - 2 n n^T with the momentum rows negated.  The test builds that state
by hand and checks:
  * the oracle's wall branch uses exactly that far side, and its flux equals
    the interior-face flux of the hand-built state;
  * no mass and no energy cross the wall (flux and its time derivative) when
    the data varies only along the normal, whatever the collision time: the
    mirrored problem is then symmetric under u -> -u;
  * in the inviscid limit (tau = 0) the interface equilibrium is at rest, so
    the flux is a pure normal pressure force for any gradients;
  * a mirror that forgets to reflect the normal derivative breaks the first
    property (so the check is sharp).
"""
import numpy as np
import pytest

import oracle

WALL = 3
GAMMA = 1.4
VISC = dict(mu_ref=0.02, Pr=0.72, visc_exp=0.7, T_ref=1 / GAMMA, tau_c=1.0)


def cons(rho, U, p):
    U = np.asarray(U, dtype=float)
    return np.array([rho, *(rho * U), p / (GAMMA - 1) + 0.5 * rho * U @ U])


def hand_mirror(n, ql, gl, reflect=True):
    s = np.array([1.0, -1.0, -1.0, -1.0, 1.0])
    R = np.eye(3) - 2 * np.outer(n, n) if reflect else np.eye(3)
    return s * ql, s[:, None] * (gl @ R.T)


def cases(seed, k=6):
    rng = np.random.default_rng(seed)
    for _ in range(k):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        ql = cons(rng.uniform(0.7, 1.4), rng.uniform(-0.4, 0.4, 3), rng.uniform(0.6, 1.2))
        gl = 0.3 * rng.normal(size=(5, 3))
        yield n, ql, gl, rng.uniform(1e-3, 2e-2)


@pytest.mark.parametrize("params", [VISC, dict(mu_ref=0.0, tau_c=0.0)], ids=["viscous", "inviscid"])
def test_wall_uses_the_mirrored_state(params):
    for n, ql, gl, dt in cases(1):
        F, dF, qr, gr = oracle.boundary_flux(WALL, n, ql, gl, dt, **params)
        qh, gh = hand_mirror(n, ql, gl)
        assert np.allclose(qr, qh, rtol=0, atol=1e-15)
        assert np.allclose(gr, gh, rtol=0, atol=1e-15)
        Fi, dFi = oracle.flux_point(n, ql, gl, qh, gh, dt, **params)
        scale = np.abs(Fi).max()
        assert np.allclose(F, Fi, rtol=0, atol=1e-13 * scale)
        assert np.allclose(dF, dFi, rtol=0, atol=1e-12 * np.abs(dFi).max())  # rounding of the two mirrors


def normal_only(n, gl):
    """The gradient with its tangential part removed: data varying along n only."""
    return np.outer(gl @ n, n)


def test_no_mass_or_energy_through_the_wall():
    for n, ql, gl, dt in cases(2):
        g = normal_only(n, gl)
        F, dF, _, _ = oracle.boundary_flux(WALL, n, ql, g, dt, **VISC)
        scale = np.abs(F).max()
        assert abs(F[0]) <= 1e-14 * scale and abs(F[4]) <= 1e-14 * scale, F
        dscale = np.abs(dF).max()
        assert abs(dF[0]) <= 1e-13 * dscale and abs(dF[4]) <= 1e-13 * dscale, dF
        # the sharpness check: the same flux with the normal derivative not reflected
        qh, gh = hand_mirror(n, ql, g, reflect=False)
        Fb, _ = oracle.flux_point(n, ql, g, qh, gh, dt, **VISC)
        assert abs(Fb[0]) > 1e-6 * scale


def test_inviscid_wall_flux_is_a_normal_pressure_force():
    for n, ql, gl, dt in cases(3):
        F, _, _, _ = oracle.boundary_flux(WALL, n, ql, gl, dt, mu_ref=0.0, tau_c=0.0)
        scale = np.abs(F).max()
        assert abs(F[0]) <= 1e-14 * scale and abs(F[4]) <= 1e-14 * scale
        pn = F[1:4] @ n
        assert pn > 0 and np.abs(F[1:4] - pn * n).max() <= 1e-14 * scale

"""Post-processing of the sphere flows of Section 5.2 (closed wake length,
separation angle, stagnation pressure) on states with known answers, on the
CPU: the functions read the geometry of a cubed-sphere shell and a state,
so fields built from the cell centroids with a chosen wake length and
separation angle must give those back."""
import math

import numpy as np
import pytest

from paper_2407_00656_b300 import inputs as I
from paper_2407_00656_b300 import sphere_wake as W


def state_from(rho, u, p, gamma=1.4):
    q = np.empty((len(rho), 5))
    q[:, 0] = rho
    q[:, 1:4] = rho[:, None] * u
    q[:, 4] = p / (gamma - 1) + 0.5 * rho * (u * u).sum(axis=1)
    return q


@pytest.fixture(scope="module")
def shell():
    xyz, cells, _, _ = I.sphere_shell(12, 24, r_far=10.0, growth=1.15)
    return xyz, cells, W.ShellView(xyz, cells)


def test_pitot_pressure_closed_forms():
    # isentropic stagnation pressure: p0/p = 1.1862 at Ma 0.5 in the isentropic-flow tables
    assert W.pitot_pressure(0.5, 1.0) == pytest.approx(1.1862, abs=5e-5)
    # at Ma 1 the normal shock vanishes: both branches give (1.2)^3.5
    assert W.pitot_pressure(1.0 + 1e-12, 1.0) == pytest.approx(1.2 ** 3.5, rel=1e-9)
    # Rayleigh pitot ratio at Ma 2 (gamma 1.4): 5.6404 in the normal-shock tables
    assert W.pitot_pressure(2.0, 1.0) == pytest.approx(5.6404, abs=5e-4)
    # Section 5.2's transonic stream, p_inf = 1/gamma
    assert W.pitot_pressure(1.5) == pytest.approx(3.4133 / 1.4, rel=1e-4)


def test_view_finds_wall_layer_and_axis_rings(shell):
    xyz, cells, v = shell
    assert len(v.wall) == 6 * 12 * 12
    assert np.all(v.r[v.wall] < v.r.min() * 1.01 + 0.05)
    # n even: four cells around the downstream axis in every layer
    ax = v.axis_cells()
    assert len(ax) == 4 * 24
    assert np.all(v.c[ax, 0] > 0)
    assert len(v.front_cells()) == 4
    # the second layer: one cell above each wall cell, none on the wall
    assert len(v.layer2) == len(v.wall) and not set(v.layer2) & set(v.wall)
    assert np.all(v.r[v.layer2] > v.r[v.wall].max())


@pytest.mark.parametrize("theta_deg", [118.0, 128.4, 136.8, 150.0])
def test_separation_angle_of_a_field_with_known_reversal(shell, theta_deg):
    xyz, cells, v = shell
    th = math.radians(theta_deg)
    c = v.c
    rhat = c / v.r[:, None]
    cosf = -rhat[:, 0]
    sinf = np.sqrt(np.maximum(1 - cosf * cosf, 1e-300))
    e_phi = (cosf[:, None] * rhat - np.array([-1.0, 0, 0])) / sinf[:, None]
    phi = v.phi
    # meridional wall velocity sin(phi) (theta - phi): attached upstream of
    # theta, reversed downstream; plus azimuthal and radial parts that the
    # projection must ignore
    e_az = np.cross(rhat, e_phi)
    amp = np.sin(phi) * (th - phi)
    u = amp[:, None] * e_phi + 0.3 * e_az + 0.05 * rhat
    q = state_from(np.full(len(c), 1.0), u, np.full(len(c), 1 / 1.4))
    got = W.separation_angle(v, q)
    assert abs(got - theta_deg) < 0.6, got
    # the sensitivity variants read the same field: twice as wide bins, and
    # the second cell layer on the wall
    wide = 2 * math.degrees(v.spacing)  # 15 degrees on this coarse shell
    assert abs(W.separation_angle(v, q, bin_deg=wide) - theta_deg) < 0.2 * wide
    assert abs(W.separation_angle(v, q, layer=2) - theta_deg) < 0.6


def test_separation_angle_is_nan_for_attached_flow(shell):
    xyz, cells, v = shell
    rhat = v.c / v.r[:, None]
    u = np.tile([0.3, 0.0, 0.0], (len(v.c), 1)) - 0.3 * rhat * rhat[:, :1]  # tangential, downstream
    q = state_from(np.ones(len(v.c)), u, np.full(len(v.c), 1 / 1.4))
    assert math.isnan(W.separation_angle(v, q))


@pytest.mark.parametrize("length", [0.0, 0.45, 0.99, 1.18, 2.5])
def test_wake_length_of_a_field_with_known_reattachment(shell, length):
    xyz, cells, v = shell
    r_l = 0.5 + length
    ux = (v.r - 0.5) * (v.r - r_l)  # reversed between the rear pole and r_l
    u = np.zeros((len(v.c), 3))
    u[:, 0] = ux
    u[:, 1] = 0.1 * v.c[:, 1]  # off-axis parts do not enter
    q = state_from(np.full(len(v.c), 1.1), u, np.full(len(v.c), 0.7))
    got = W.wake_length(v, q)
    # linear interpolation of a quadratic between layers: within a small
    # fraction of the local layer spacing
    r_ax = np.unique(np.round(v.r[v.axis_cells()], 12))
    i = np.searchsorted(r_ax, r_l)
    h = r_ax[min(i, len(r_ax) - 1)] - r_ax[max(i - 1, 0)]
    assert abs(got - length) <= 0.25 * h + 1e-12, (got, length, h)


def test_stagnation_pressure_reads_the_front_ring(shell):
    xyz, cells, v = shell
    p = 0.7 + 0.1 * np.cos(v.phi)  # largest at the front pole
    q = state_from(np.ones(len(v.c)), np.zeros((len(v.c), 3)), p)
    ring = v.front_cells()
    assert W.stagnation_pressure(v, q) == pytest.approx(p[ring].mean(), rel=1e-14)
    assert W.stagnation_pressure(v, q) > 0.799


def test_stagnation_density_against_shock_tables():
    # Ma 1.5: total-pressure ratio across the normal shock 0.9298 (normal-shock
    # tables), and the free stream's stagnation density 1.45^2.5 (isentropic)
    assert W.stagnation_density(1.5) == pytest.approx(0.9298 * 1.45 ** 2.5, rel=2e-4)
    # subsonic: plain isentropic compression
    assert W.stagnation_density(0.2535) == pytest.approx((1 + 0.2 * 0.2535 ** 2) ** 2.5, rel=1e-12)


@pytest.mark.parametrize("standoff", [0.15, 0.3, 0.6])
def test_shock_standoff_of_a_density_step(shell, standoff):
    xyz, cells, v = shell
    r_s = 0.5 + standoff
    rho = np.where(v.r < r_s, 2.35, 1.0)
    q = state_from(rho, np.zeros((len(rho), 3)), np.full(len(rho), 0.7))
    got = W.shock_standoff(v, q)
    up = np.nonzero(v.c[:, 0] < 0)[0]
    r_ax = np.unique(np.round(v.r[v._ring(v.phi, up)], 12))
    i = np.searchsorted(r_ax, r_s)
    assert r_ax[i - 1] - 0.5 <= got <= r_ax[i] - 0.5, (got, standoff)
    assert math.isnan(W.shock_standoff(v, state_from(np.ones(len(rho)), np.zeros((len(rho), 3)),
                                                     np.full(len(rho), 0.7))))

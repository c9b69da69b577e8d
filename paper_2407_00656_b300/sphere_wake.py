"""Steady flow past a sphere (Section 5.2): the quantities that the paper
tabulates for it, taken from the cell averages the solver returns, and a
driver that marches the cubed-sphere shell to a steady state on the GPU.

Conventions of Section 5.2: a sphere of diameter D = 1 centred at the origin,
the free stream (1, Ma, 0, 0, 1/gamma) along +x, so the front stagnation
point is the pole at x = -1/2 and the rear pole is at x = +1/2.

- Closed wake length L: the distance, in diameters, from the rear pole to
  the point on the downstream axis where the axial velocity changes sign
  from reversed (negative) to forward (positive).
- Separation angle theta: the polar angle, measured from the front
  stagnation point, where the meridional velocity next to the wall changes
  sign from pointing downstream (attached flow) to pointing upstream
  (reversed flow).  The wall is no-slip, so the velocity of the first cell
  layer has the sign of the wall shear.
- Stagnation pressure: the pressure of the wall cells that touch the front
  pole.  Behind the bow shock of a supersonic stream it is the Rayleigh
  pitot value; in a subsonic stream the isentropic one.

Both flows of Section 5.2 (Re 118 at Ma 0.2535 and Re 300 at Ma 1.5) are
steady and axisymmetric, so every quantity is averaged over the azimuth.

Run ``python -m paper_2407_00656_b300.sphere_wake --mach 0.2535 --re 118``
for the subsonic case of Section 5.2 on a 12 N^3-cell shell (six blocks of
N x N x 2N hexahedra, as the paper builds them).
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

GAMMA = 1.4

# Section 5.2, the two tables of closed wake length and separation angle
# (3,145,728 hexahedra): (L, theta in degrees).
PAPER_VALUES = {(0.2535, 118.0): (0.99, 128.4), (1.5, 300.0): (1.18, 136.8)}


def primitives(q, gamma: float = GAMMA):
    """(rho, velocity [n][3], pressure) of conservative cell averages."""
    q = np.asarray(q, dtype=np.float64)
    rho = q[:, 0]
    u = q[:, 1:4] / rho[:, None]
    p = (gamma - 1.0) * (q[:, 4] - 0.5 * rho * (u * u).sum(axis=1))
    return rho, u, p


def pitot_pressure(mach: float, p_inf: float = 1.0 / GAMMA, gamma: float = GAMMA) -> float:
    """Stagnation pressure on the body: behind a normal shock (Rayleigh pitot
    formula) when the stream is supersonic, isentropic otherwise."""
    g = gamma
    m2 = mach * mach
    if mach <= 1.0:
        return p_inf * (1.0 + 0.5 * (g - 1.0) * m2) ** (g / (g - 1.0))
    a = ((g + 1.0) ** 2 * m2 / (4.0 * g * m2 - 2.0 * (g - 1.0))) ** (g / (g - 1.0))
    return p_inf * a * (1.0 - g + 2.0 * g * m2) / (g + 1.0)


def stagnation_density(mach: float, rho_inf: float = 1.0, gamma: float = GAMMA) -> float:
    """Density at the stagnation point: the stagnation temperature is
    T_inf (1 + (gamma-1)/2 Ma^2) across a shock too, so rho_0 = p_0 / (R T_0)
    with p_0 from ``pitot_pressure``."""
    p_inf = 1.0 / gamma
    t_ratio = 1.0 + 0.5 * (gamma - 1.0) * mach * mach
    return rho_inf * pitot_pressure(mach, p_inf, gamma) / p_inf / t_ratio


class ShellView:
    """The cells of a sphere shell seen from the sphere: centroids, the first
    cell layer on the wall, and the cells that straddle the x axis.

    ``xyz`` [nodes][3] and ``cells`` [n][8] as the mesh was built (caller
    order, the order of the states ``hgks_read`` returns).  Wall nodes are
    those at radius ``r_wall`` (to 1e-9 relative); a wall-layer cell has a
    whole face (four nodes) on the wall.
    """

    def __init__(self, xyz, cells, r_wall: float = 0.5):
        xyz = np.asarray(xyz, dtype=np.float64)
        cells = np.asarray(cells)
        self.r_wall = r_wall
        self.c = xyz[cells].mean(axis=1)
        self.r = np.linalg.norm(self.c, axis=1)
        on_wall = np.abs(np.linalg.norm(xyz, axis=1) - r_wall) <= 1e-9 * r_wall
        self.wall = np.nonzero(on_wall[cells].sum(axis=1) >= 4)[0]
        if len(self.wall) == 0:
            raise ValueError("no cell has a face on the sphere r = r_wall")
        # the second layer: cells with a whole face on the outer face of the
        # wall layer
        outer = np.zeros(len(xyz), dtype=bool)
        wn = cells[self.wall].ravel()
        outer[wn[~on_wall[wn]]] = True
        in_wall = np.zeros(len(cells), dtype=bool)
        in_wall[self.wall] = True
        self.layer2 = np.nonzero((outer[cells].sum(axis=1) >= 4) & ~in_wall)[0]
        # angular mesh spacing: a cubed sphere has 6 n^2 cells per layer over
        # the four quarter-circles of each great circle
        n_est = math.sqrt(len(self.wall) / 6.0)
        self.spacing = 0.5 * math.pi / n_est
        # polar angle from the front (-x) pole and from the rear (+x) axis
        cosf = np.clip(-self.c[:, 0] / self.r, -1.0, 1.0)
        self.phi = np.arccos(cosf)
        self.psi = math.pi - self.phi

    def _ring(self, ang, pool):
        """Cells of ``pool`` nearest an axis: within half a mesh spacing of the
        smallest angle found (one ring of cells around it)."""
        a = ang[pool]
        return pool[a <= a.min() + 0.5 * self.spacing]

    def axis_cells(self):
        """Cells around the downstream axis, in every layer."""
        down = np.nonzero(self.c[:, 0] > 0.0)[0]
        return self._ring(self.psi, down)

    def front_cells(self):
        """Wall-layer cells around the front stagnation point."""
        return self._ring(self.phi, self.wall)

    def meridional_velocity(self, u, cells=None):
        """Velocity of the wall-layer cells (or of ``cells``) along e_phi, the
        unit vector of increasing polar angle from the front pole (downstream
        along the wall)."""
        sel = self.wall if cells is None else cells
        c = self.c[sel]
        rhat = c / self.r[sel][:, None]
        cosf = np.cos(self.phi[sel])
        sinf = np.maximum(np.sin(self.phi[sel]), 1e-300)
        front = np.array([-1.0, 0.0, 0.0])
        e_phi = (cosf[:, None] * rhat - front[None, :]) / sinf[:, None]
        return (u[sel] * e_phi).sum(axis=1)


def separation_angle(view: ShellView, q, bin_deg: float | None = None, skip_deg: float = 10.0,
                     layer: int = 1) -> float:
    """Separation angle in degrees from the front stagnation point, or NaN
    when the flow stays attached.

    The cells of the first (or, ``layer`` = 2, the second) layer on the wall
    are binned by polar angle (bins one mesh spacing wide by default) and the
    meridional velocity averaged in each bin.  The result is the first change
    of sign from positive to negative, scanning from the front, past
    ``skip_deg`` (where the velocity vanishes at the stagnation point),
    linearly interpolated between the mean polar angles of the cells of the
    two bins.
    """
    _, u, _ = primitives(q)
    sel = view.wall if layer == 1 else view.layer2
    ut = view.meridional_velocity(u, sel)
    phi = view.phi[sel]
    width = math.radians(bin_deg) if bin_deg else view.spacing
    nb = max(1, int(round(math.pi / width)))
    k = np.minimum((phi / math.pi * nb).astype(np.int64), nb - 1)
    cnt = np.bincount(k, minlength=nb)
    have = cnt > 0
    centre = np.bincount(k, weights=phi, minlength=nb)[have] / cnt[have]
    mean = np.bincount(k, weights=ut, minlength=nb)[have] / cnt[have]
    ok = centre >= math.radians(skip_deg)
    centre, mean = centre[ok], mean[ok]
    for i in range(1, len(mean)):
        if mean[i - 1] > 0.0 and mean[i] <= 0.0:
            f = mean[i - 1] / (mean[i - 1] - mean[i])
            return math.degrees(centre[i - 1] + f * (centre[i] - centre[i - 1]))
    return float("nan")


def wake_length(view: ShellView, q) -> float:
    """Closed wake length in diameters (D = 1): from the rear pole to the
    first change of sign of the axial velocity on the downstream axis, from
    reversed to forward.  0 when there is no reversed flow on the axis.

    The axial velocity at radius r on the axis is the mean over the ring of
    cells around the axis in that layer; the crossing is linearly
    interpolated between layers.  0 when the first layer's is not reversed.
    """
    _, u, _ = primitives(q)
    rl, ul = _layer_means(view, view.axis_cells(), u[:, 0])
    if ul[0] >= 0.0:
        return 0.0
    for i in range(1, len(ul)):
        if ul[i - 1] < 0.0 and ul[i] >= 0.0:
            f = -ul[i - 1] / (ul[i] - ul[i - 1])
            return float(rl[i - 1] + f * (rl[i] - rl[i - 1]) - view.r_wall) / (2.0 * view.r_wall)
    return float("nan")


def _layer_means(view: ShellView, idx, values):
    """Radii and means of ``values`` over the cells ``idx`` of a ring around
    an axis, one entry per layer (cells whose centroid radii agree to 0.1%
    form one layer), from the wall outwards."""
    r = view.r[idx]
    v = values[idx]
    o = np.argsort(r, kind="stable")
    r, v = r[o], v[o]
    cut = np.nonzero(np.diff(r) > 1e-3 * r[1:])[0] + 1
    groups = np.split(np.arange(len(r)), cut)
    return np.array([r[g].mean() for g in groups]), np.array([v[g].mean() for g in groups])


def shock_standoff(view: ShellView, q, rho_inf: float = 1.0) -> float:
    """Distance in diameters from the front stagnation point to the bow
    shock on the upstream axis: where the density, coming in from the free
    stream, first rises past halfway between ``rho_inf`` and its largest
    value on the axis.  NaN when the density never rises (no shock)."""
    rho, _, _ = primitives(q)
    up = np.nonzero(view.c[:, 0] < 0.0)[0]
    rl, dl = _layer_means(view, view._ring(view.phi, up), rho)
    half = 0.5 * (rho_inf + dl.max())
    if dl.max() <= rho_inf * 1.05:
        return float("nan")
    for i in range(len(dl) - 1, 0, -1):
        if dl[i] < half <= dl[i - 1]:
            f = (half - dl[i]) / (dl[i - 1] - dl[i])
            return float(rl[i] + f * (rl[i - 1] - rl[i]) - view.r_wall) / (2.0 * view.r_wall)
    return float("nan")


def billig_standoff(mach: float) -> float:
    """Empirical bow-shock standoff of a sphere in diameters, Billig's
    correlation Delta/R = 0.143 exp(3.24 / Ma^2) (a fit to experiment, good
    to some ten per cent; context for a coarse-mesh value, not a pin)."""
    return 0.5 * 0.143 * math.exp(3.24 / (mach * mach))


def stagnation_pressure(view: ShellView, q) -> float:
    """Mean pressure of the wall-layer cells around the front pole."""
    _, _, p = primitives(q)
    return float(p[view.front_cells()].mean())


def march(mach: float, re: float, n: int = 24, n_r: int | None = None, r_far: float = 20.0,
          growth: float = 1.12, precision: int = 1, t_max: float = 400.0, chunk: float = 20.0,
          tol_len: float = 0.005, tol_deg: float = 0.2, max_steps: int = 5_000_000, log=None):
    """March the shell from the free stream until L and theta settle.

    The shell has six blocks of n x n x n_r hexahedra (n_r = 2 n as in
    Section 5.2), growing by ``growth`` from the wall to ``r_far``; the flow
    is viscous with the power law of Section 5.2 (mu_inf = Ma D / Re, Pr 0.72)
    and numerical collision time coefficient 1.  Every ``chunk`` time units
    the state is read back and L, theta and the stagnation pressure recorded;
    the march stops once three successive records agree within ``tol_len``
    and ``tol_deg``, or at ``t_max``; more than ``max_steps`` steps raise
    RuntimeError (a time step that collapses).  Returns the records and a
    summary.
    """
    from . import hgks as H
    from . import inputs as I

    n_r = n_r or 2 * n
    xyz, cells, bfn, bft = I.sphere_shell(n, n_r, r_far=r_far, growth=growth)
    view = ShellView(xyz, cells)
    qinf = I.free_stream(mach)
    q0 = np.tile(qinf, (len(cells), 1))
    s = H.Solver(H.Mesh(xyz, cells, None, bfn, bft), q0, precision=precision, q_inf=qinf, mu_ref=mach / re,
                 Pr=0.72, visc_exp=0.7, T_ref=1.0 / GAMMA, tau_num_c=1.0)
    records = []
    t, steps, per_step = 0.0, 0, None
    wall0 = time.perf_counter()
    q = q0
    while t < t_max - 1e-12:
        target = min(t_max, t + chunk)
        while t < target - 1e-12:
            k = 200 if per_step is None else max(1, min(20000, int(math.ceil((target - t) / per_step)) + 1))
            s.step(k, t_end=target)
            q, t_new, steps_new = s.read()
            if steps_new > steps:
                per_step = (t_new - t) / (steps_new - steps)
            t, steps = t_new, steps_new
            if steps > max_steps:
                s.close()
                raise RuntimeError(f"{steps} steps reached t = {t} of {t_max}")
        rho, u, p = primitives(q)
        front = view.front_cells()
        rec = dict(t=t, steps=steps, L=wake_length(view, q), theta=separation_angle(view, q),
                   theta_bin2=separation_angle(view, q, bin_deg=2.0 * math.degrees(view.spacing)),
                   theta_layer2=separation_angle(view, q, layer=2),
                   p_stag=float(p[front].mean()), rho_stag=float(rho[front].mean()),
                   standoff=shock_standoff(view, q) if mach > 1.0 else None,
                   max_mach=float(np.sqrt((u * u).sum(axis=1) * rho / (GAMMA * p)).max()),
                   min_p=float(p.min()), min_rho=float(rho.min()), dt=per_step,
                   wall_s=time.perf_counter() - wall0)
        records.append(rec)
        if log:
            log(rec)
        if len(records) >= 3:
            last = records[-3:]
            dl = max(r["L"] for r in last) - min(r["L"] for r in last)
            dth = max(r["theta"] for r in last) - min(r["theta"] for r in last)
            if dl <= tol_len and dth <= tol_deg:
                break
    s.close()
    paper = PAPER_VALUES.get((mach, re))
    summary = dict(mach=mach, re=re, cells=len(cells), shell=f"6x{n}^2x{n_r}", growth=growth, r_far=r_far,
                   first_spacing=float(r_far - 0.5) * (growth - 1.0) / (growth ** n_r - 1.0),
                   precision="mixed" if precision == 1 else "fp64", t=t, steps=steps,
                   L=records[-1]["L"], theta=records[-1]["theta"], theta_bin2=records[-1]["theta_bin2"],
                   theta_layer2=records[-1]["theta_layer2"], p_stag=records[-1]["p_stag"],
                   p_stag_pitot=pitot_pressure(mach), rho_stag=records[-1]["rho_stag"],
                   rho_stag_pitot=stagnation_density(mach), standoff=records[-1]["standoff"],
                   standoff_billig=billig_standoff(mach) if mach > 1.0 else None,
                   max_mach=records[-1]["max_mach"], paper_L=paper[0] if paper else None,
                   paper_theta=paper[1] if paper else None,
                   cell_updates_per_s=len(cells) * steps / max(records[-1]["wall_s"], 1e-9))
    return records, summary


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--mach", type=float, default=0.2535)
    ap.add_argument("--re", type=float, default=118.0)
    ap.add_argument("--n", type=int, default=24, help="cells per cube edge (12 n^3 cells with n_r = 2n)")
    ap.add_argument("--n-r", type=int, default=None)
    ap.add_argument("--growth", type=float, default=1.12)
    ap.add_argument("--r-far", type=float, default=20.0)
    ap.add_argument("--precision", choices=("fp64", "mixed"), default="mixed")
    ap.add_argument("--t-max", type=float, default=400.0)
    ap.add_argument("--chunk", type=float, default=20.0)
    ap.add_argument("--out", default=None, help="file for the records and the summary (JSON lines)")
    a = ap.parse_args(argv)
    out = open(a.out, "w") if a.out else None

    def log(rec):
        line = json.dumps(rec)
        print(line, flush=True)
        if out:
            out.write(line + "\n")
            out.flush()

    _, summary = march(a.mach, a.re, n=a.n, n_r=a.n_r, r_far=a.r_far, growth=a.growth,
                       precision=1 if a.precision == "mixed" else 0, t_max=a.t_max, chunk=a.chunk, log=log)
    log(dict(summary=summary))
    if out:
        out.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())

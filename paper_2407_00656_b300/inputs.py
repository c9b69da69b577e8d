"""Seeded synthetic inputs: meshes (node and cell arrays) and initial states.

This module holds no part of the gas-kinetic scheme. It only produces the data
that a user would load from files: node coordinates, cell-to-node lists,
boundary-face lists with their condition tags, and initial cell averages given
by closed-form fields. Both the GPU library and the CPU oracle consume these
arrays as plain inputs.

Workloads (Section 5 of the paper):
  * density-wave accuracy test on the periodic cube [0,2]^3, every cube of an
    N^3 lattice split into 6 tetrahedra (Section 5.1), optionally with seeded
    jitter of the interior nodes;
  * flow past a unit-diameter sphere on a six-block hexahedral shell
    (Section 5.2), with geometric radial growth from the wall, optionally
    with a seeded share of its columns cut into triangular prisms;
  * the density wave on the periodic cube cut into triangular prisms.

A triangular prism is passed as a hexahedron whose nodes 2 and 3 coincide and
whose nodes 6 and 7 coincide: bottom triangle 0 1 2, top triangle 4 5 6.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

TET4 = 4
HEX8 = 8
BC_PERIODIC = 1
BC_FARFIELD = 2
BC_WALL = 3


# ----------------------------------------------------------------------------
# Periodic cube split into Kuhn tetrahedra (Section 5.1 meshes)
# ----------------------------------------------------------------------------
def kuhn_cube(n: int, length: float = 2.0, jitter: float = 0.0, seed: int = 0):
    """Return (xyz[n_nodes,3], cells[6 n^3,4], periods[3]).

    Each lattice cube is cut along its (0,0,0)-(1,1,1) diagonal into six
    tetrahedra, one per ordering of the three axes, so neighbouring cubes
    share faces conformingly.  Every tetrahedron is oriented with a positive
    signed volume.  With ``jitter>0`` every node strictly inside (0,L)^3 is
    moved per component by a uniform offset in [-jitter*h, jitter*h] drawn
    from ``numpy.random.default_rng(seed)``; boundary nodes stay put so that
    periodic faces still match under translation by L.
    """
    h = length / n
    m = n + 1
    ii, jj, kk = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    xyz = np.stack([ii, jj, kk], axis=-1).reshape(-1, 3).astype(np.float64) * h
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        off = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
        interior = np.all((xyz > 0.5 * h) & (xyz < length - 0.5 * h), axis=1)
        xyz[interior] += off[interior]

    def nid(i, j, k):
        return (i * m + j) * m + k

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    tets = []
    for perm in itertools.permutations(range(3)):
        corner = np.zeros(3, dtype=np.int64)
        verts = [nid(ci, cj, ck)]
        for ax in perm:
            corner[ax] += 1
            verts.append(nid(ci + corner[0], cj + corner[1], ck + corner[2]))
        tets.append(np.stack(verts, axis=1))
    cells = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int64)
    # orient positively: swap the last two nodes where the signed volume < 0
    p = xyz[cells]
    det = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])
    neg = det < 0
    cells[neg, 2], cells[neg, 3] = cells[neg, 3].copy(), cells[neg, 2].copy()
    periods = np.array([length, length, length], dtype=np.float64)
    return xyz, cells, periods


def prism_cube(n: int, length: float = 2.0, jitter: float = 0.0, seed: int = 0):
    """Return (xyz, cells[2 n^3, 8], periods[3]): the periodic cube of
    ``kuhn_cube`` with every lattice cube cut by the vertical plane through
    its (0,0)-(1,1) diagonal into two triangular prisms, given as
    hexahedra with nodes 2 = 3 and 6 = 7 (bottom triangle 0 1 2, top
    triangle 4 5 6 one lattice step up in z).  Same node jitter as
    ``kuhn_cube``."""
    h = length / n
    m = n + 1
    ii, jj, kk = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    xyz = np.stack([ii, jj, kk], axis=-1).reshape(-1, 3).astype(np.float64) * h
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        off = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
        interior = np.all((xyz > 0.5 * h) & (xyz < length - 0.5 * h), axis=1)
        xyz[interior] += off[interior]

    def nid(i, j, k):
        return (i * m + j) * m + k

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    b = [nid(ci, cj, ck), nid(ci + 1, cj, ck), nid(ci + 1, cj + 1, ck), nid(ci, cj + 1, ck)]
    t = [nid(ci, cj, ck + 1), nid(ci + 1, cj, ck + 1), nid(ci + 1, cj + 1, ck + 1), nid(ci, cj + 1, ck + 1)]
    a_ = np.stack([b[0], b[1], b[2], b[2], t[0], t[1], t[2], t[2]], axis=1)
    b_ = np.stack([b[0], b[2], b[3], b[3], t[0], t[2], t[3], t[3]], axis=1)
    cells = np.stack([a_, b_], axis=1).reshape(-1, 8).astype(np.int64)
    periods = np.array([length, length, length], dtype=np.float64)
    return xyz, cells, periods


def hex_cube(n: int, length: float = 2.0, jitter: float = 0.0, seed: int = 0):
    """Return (xyz, cells[n^3, 8], periods[3]): the periodic cube [0,L]^3 as
    an n^3 lattice of hexahedra (nodes 0-3 the lower quad counter-clockwise
    seen from above, 4-7 the upper quad in the same order, so the trilinear
    map has a positive Jacobian).  Same node jitter as ``kuhn_cube``; jittered
    hexahedra have non-planar faces."""
    h = length / n
    m = n + 1
    ii, jj, kk = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    xyz = np.stack([ii, jj, kk], axis=-1).reshape(-1, 3).astype(np.float64) * h
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        off = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
        interior = np.all((xyz > 0.5 * h) & (xyz < length - 0.5 * h), axis=1)
        xyz[interior] += off[interior]

    def nid(i, j, k):
        return (i * m + j) * m + k

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    cells = np.stack([nid(ci, cj, ck), nid(ci + 1, cj, ck), nid(ci + 1, cj + 1, ck), nid(ci, cj + 1, ck),
                      nid(ci, cj, ck + 1), nid(ci + 1, cj, ck + 1), nid(ci + 1, cj + 1, ck + 1),
                      nid(ci, cj + 1, ck + 1)], axis=1).astype(np.int64)
    periods = np.array([length, length, length], dtype=np.float64)
    return xyz, cells, periods


def prism_tets(cells: np.ndarray) -> np.ndarray:
    """The three tetrahedra [n, 3, 4] that make up each prism (nodes
    2 = 3, 6 = 7) with planar side faces: (0 1 2 4), (1 2 4 5), (2 4 5 6)."""
    c = np.asarray(cells)
    return np.stack([c[:, [0, 1, 2, 4]], c[:, [1, 2, 4, 5]], c[:, [2, 4, 5, 6]]], axis=1)


def cell_average_sin(xyz: np.ndarray, cells: np.ndarray, t: float) -> np.ndarray:
    """Exact average of sin(pi (x+y+z-t)) over tetrahedra, or over prisms
    (hexahedra with nodes 2 = 3, 6 = 7) whose side faces are planar, as the
    volume-weighted mean over their three tetrahedra."""
    cells = np.asarray(cells)
    if cells.shape[1] == 4:
        return tet_average_sin(xyz, cells, t)
    if not np.all((cells[:, 2] == cells[:, 3]) & (cells[:, 6] == cells[:, 7])):
        raise ValueError("exact averages are for tetrahedra and prisms only")
    tets = prism_tets(cells).reshape(-1, 4)
    p = xyz[tets]
    vol = np.abs(np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0]))
    avg = tet_average_sin(xyz, tets, t)
    return (vol * avg).reshape(-1, 3).sum(axis=1) / vol.reshape(-1, 3).sum(axis=1)


def _complete_homogeneous(d: np.ndarray, mmax: int) -> np.ndarray:
    """h_m(d_0..d_{k-1}) for m = 0..mmax, per row of d (shape [n,k])."""
    n, k = d.shape
    H = np.zeros((mmax + 1, n))
    H[0] = 1.0
    for j in range(k):
        x = d[:, j]
        for mm in range(1, mmax + 1):
            H[mm] = H[mm] + x * H[mm - 1]
    return H


def tet_average_sin(xyz: np.ndarray, cells: np.ndarray, t: float, mmax: int = 48) -> np.ndarray:
    """Exact average over each tetrahedron of sin(pi (x+y+z-t)).

    The field depends on x only through the linear form s = x+y+z-t, so by
    the Hermite-Genocchi formula the average is 3! times the third divided
    difference, over the vertex values s_0..s_3, of F(s) = cos(pi s)/pi^3
    (an antiderivative of order three of sin(pi s)).  The divided difference
    is summed as a Taylor series about the mean vertex value c:
        F[s_0..s_3] = sum_m F^(m+3)(c)/(m+3)! * h_m(s_0-c, .., s_3-c)
    with h_m the complete homogeneous symmetric polynomials.  Unlike the
    difference table this stays accurate when vertex values nearly coincide.
    """
    s = xyz[cells].sum(axis=2) - t  # [nc,4]
    c = s.mean(axis=1)
    d = s - c[:, None]
    H = _complete_homogeneous(d, mmax)
    out = np.zeros(len(c))
    for mm in range(mmax + 1):
        out += (math.pi ** mm) * np.sin(math.pi * c + mm * math.pi / 2) * H[mm] / math.factorial(mm + 3)
    return 6.0 * out


def density_wave_state(xyz, cells, t: float = 0.0, gamma: float = 1.4, amp: float = 0.2):
    """Exact cell averages [nc,5] of the advected density wave (Section 5.1).

    With U=V=W=1 and p=1 the Euler equations carry the initial density
    unchanged along (1,1,1), so rho = 1 + amp sin(pi(x+y+z-3t)).  (The paper
    prints x+y+z-t; the two agree at its output time t=2, a whole number of
    periods for both.)  Every conservative variable is affine in rho:
    (rho, rho, rho, rho, p/(gamma-1) + 3 rho/2).
    """
    rho = 1.0 + amp * cell_average_sin(xyz, cells, 3.0 * t)
    q = np.empty((len(rho), 5))
    q[:, 0] = rho
    q[:, 1] = rho
    q[:, 2] = rho
    q[:, 3] = rho
    q[:, 4] = 1.0 / (gamma - 1.0) + 1.5 * rho
    return q


def uniform_state(n_cells: int, rho=1.0, vel=(1.0, 1.0, 1.0), p=1.0, gamma=1.4):
    """Constant conservative state [n_cells,5]."""
    u, v, w = vel
    q = np.empty((n_cells, 5))
    q[:, 0] = rho
    q[:, 1] = rho * u
    q[:, 2] = rho * v
    q[:, 3] = rho * w
    q[:, 4] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return q


def free_stream(mach: float, gamma: float = 1.4):
    """Conservative free stream (rho,U,V,W,p) = (1, Ma, 0, 0, 1/gamma) of Section 5.2."""
    return uniform_state(1, 1.0, (mach, 0.0, 0.0), 1.0 / gamma, gamma)[0]


def random_smooth_state(xyz, cells, seed: int = 0, gamma: float = 1.4, amp: float = 0.05):
    """Seeded smooth non-uniform state: a few random low-wavenumber modes in
    every primitive variable, sampled at the cell centroid (not an exact
    average; used only where any state will do)."""
    rng = np.random.default_rng(seed)
    cen = xyz[cells].mean(axis=1)
    prim = np.empty((len(cen), 5))
    base = np.array([1.0, 0.3, -0.2, 0.1, 1.0])
    for v in range(5):
        f = np.zeros(len(cen))
        for _ in range(3):
            k = rng.integers(-1, 2, size=3).astype(np.float64) * math.pi
            ph = rng.uniform(0, 2 * math.pi)
            f += np.sin(cen @ k + ph)
        prim[:, v] = base[v] + amp * f
    rho, u, v, w, p = prim.T
    q = np.empty_like(prim)
    q[:, 0] = rho
    q[:, 1] = rho * u
    q[:, 2] = rho * v
    q[:, 3] = rho * w
    q[:, 4] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return q


# ----------------------------------------------------------------------------
# Six-block hexahedral shell around a sphere (Section 5.2 meshes)
# ----------------------------------------------------------------------------
def sphere_shell(n: int, n_r: int, r_wall: float = 0.5, r_far: float = 20.0,
                 growth: float = 1.08, jitter: float = 0.0, seed: int = 0, prism_frac: float = 0.0):
    """Return (xyz, cells[., 8], bface_nodes[.,4], bface_tag[.]).

    The sphere surface is covered by the six faces of a cube, each an n x n
    grid mapped equiangularly onto the sphere; n_r layers of hexahedra grow
    geometrically (ratio ``growth``) from the wall at r_wall to the far field
    at r_far.  Hex node order: 0-3 the inner quad, 4-7 the outer quad above
    it, oriented for a positive volume.  Inner faces are tagged as no-slip
    walls, outer faces as far field.  ``jitter`` moves the surface directions
    tangentially by a seeded fraction of the angular spacing.

    With ``prism_frac > 0`` each surface quad is, with that probability
    (seeded), cut along a diagonal into two triangles, and its column of
    hexahedra becomes two columns of triangular prisms (hexahedra with nodes
    2 = 3 and 6 = 7): a hybrid hex/prism shell whose faces all match, since
    a column's side faces are radial quads either way.  Cells are ordered by
    layer, then by column; a cut quad's two prisms are adjacent.
    """
    g = growth
    k = np.arange(n_r + 1, dtype=np.float64)
    radii = r_wall + (r_far - r_wall) * (g ** k - 1.0) / (g ** n_r - 1.0)

    key_to_id = {}
    dirs = []

    def surf_id(i, j, kk):
        key = (i, j, kk)
        sid = key_to_id.get(key)
        if sid is None:
            sid = len(dirs)
            key_to_id[key] = sid
            a = [math.tan(math.pi / 4 * (2.0 * c / n - 1.0)) for c in key]
            nrm = math.sqrt(a[0] ** 2 + a[1] ** 2 + a[2] ** 2)
            dirs.append([a[0] / nrm, a[1] / nrm, a[2] / nrm])
        return sid

    quads = []
    for axis in range(3):
        for side in (0, n):
            o1, o2 = [a for a in range(3) if a != axis]
            for a in range(n):
                for b in range(n):
                    pts = []
                    for da, db in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        c = [0, 0, 0]
                        c[axis] = side
                        c[o1] = a + da
                        c[o2] = b + db
                        pts.append(surf_id(*c))
                    quads.append(pts)
    dirs = np.array(dirs)
    quads = np.array(quads, dtype=np.int64)
    if prism_frac > 0.0:
        cut = np.random.default_rng([seed, 7]).random(len(quads)) < prism_frac
        cols = []
        for qd, c in zip(quads, cut):
            if c:
                cols.append([qd[0], qd[1], qd[2], qd[2]])
                cols.append([qd[0], qd[2], qd[3], qd[3]])
            else:
                cols.append(list(qd))
        quads = np.array(cols, dtype=np.int64)
    ns = len(dirs)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        dirs = dirs + rng.uniform(-jitter, jitter, size=dirs.shape) * (math.pi / 2 / n)
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    xyz = (radii[:, None, None] * dirs[None, :, :]).reshape(-1, 3)
    cells = []
    for layer in range(n_r):
        lo = quads + layer * ns
        hi = quads + (layer + 1) * ns
        cells.append(np.concatenate([lo, hi], axis=1))
    cells = np.concatenate(cells, axis=0)
    # orientation: the inner quad's right-hand normal must point outwards
    p = xyz[cells]
    nq = np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 1])
    up = p[:, 4:].mean(axis=1) - p[:, :4].mean(axis=1)
    flip = np.einsum("ij,ij->i", nq, up) < 0
    prism = cells[:, 2] == cells[:, 3]
    cells[flip & ~prism] = cells[flip & ~prism][:, [0, 3, 2, 1, 4, 7, 6, 5]]
    cells[flip & prism] = cells[flip & prism][:, [1, 0, 2, 3, 5, 4, 6, 7]]  # keeps 2 = 3, 6 = 7
    nq_cells = len(quads)
    wall = cells[:nq_cells, :4].copy()
    far = cells[-nq_cells:, 4:].copy()
    wall[prism[:nq_cells], 3] = -1  # triangles, padded
    far[prism[-nq_cells:], 3] = -1
    bface_nodes = np.concatenate([wall, far], axis=0).astype(np.int64)
    bface_tag = np.concatenate([np.full(nq_cells, BC_WALL), np.full(nq_cells, BC_FARFIELD)]).astype(np.int32)
    return xyz, cells.astype(np.int64), bface_nodes, bface_tag

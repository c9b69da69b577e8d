"""The oracle on triangular prisms (hexahedra with nodes 2 = 3 and 6 = 7) and
on hybrid hex/prism shells, pinned by what does not depend on the oracle:
exact volumes, centroids and second moments of prisms cut into tetrahedra,
exact reconstruction of linear and quadratic data, free-stream
preservation, conservation, and third-order convergence on the exact
density wave."""
import numpy as np
import pytest

import oracle
from paper_2407_00656_b300 import inputs as I

from .test_oracle_scheme import _unshifted_cells, tet_average, tet_rule


def tet_moments(p):
    """Volume, centroid and central second moments (xx yy zz xy yz zx, as
    averages) of tetrahedra p[n,4,3] by the closed form of the simplex."""
    vol = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0]) / 6
    cen = p.mean(axis=1)
    d = p - cen[:, None, :]
    ia, ib = [0, 1, 2, 0, 1, 2], [0, 1, 2, 1, 2, 0]
    mom = np.stack([(d[:, :, a] * d[:, :, b]).sum(axis=1) / 20 for a, b in zip(ia, ib)], axis=1)
    return vol, cen, mom


def prism_average(xyz, cells, f, n=6):
    """Average of f over prisms with planar sides, through their tetrahedra."""
    tets = I.prism_tets(cells)  # [nc,3,4]
    vol = np.abs(tet_moments(xyz[tets.reshape(-1, 4)])[0]).reshape(-1, 3)
    avg = tet_average(xyz, tets.reshape(-1, 4), f, n=n).reshape(len(cells), 3, -1)
    return (vol[:, :, None] * avg).sum(axis=1) / vol.sum(axis=1)[:, None]


def collapsed_average(xyz, cells, f, n=5):
    """Average of f over hexahedra (prisms as collapsed hexahedra) through the
    trilinear map, by n^3 Gauss-Legendre points: exact for polynomial f of
    degree <= 2n - 3 in the coordinates."""
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = 0.5 * (x + 1), 0.5 * w
    s, t, r = np.meshgrid(x, x, x, indexing="ij")
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()
    s, t, r = s.ravel(), t.ravel(), r.ravel()
    N = np.stack([(1 - s) * (1 - t) * (1 - r), s * (1 - t) * (1 - r), s * t * (1 - r), (1 - s) * t * (1 - r),
                  (1 - s) * (1 - t) * r, s * (1 - t) * r, s * t * r, (1 - s) * t * r], axis=1)
    dS = np.stack([-(1 - t) * (1 - r), (1 - t) * (1 - r), t * (1 - r), -t * (1 - r),
                   -(1 - t) * r, (1 - t) * r, t * r, -t * r], axis=1)
    dT = np.stack([-(1 - s) * (1 - r), -s * (1 - r), s * (1 - r), (1 - s) * (1 - r),
                   -(1 - s) * r, -s * r, s * r, (1 - s) * r], axis=1)
    dR = np.stack([-(1 - s) * (1 - t), -s * (1 - t), -s * t, -(1 - s) * t,
                   (1 - s) * (1 - t), s * (1 - t), s * t, (1 - s) * t], axis=1)
    p = xyz[cells]  # [nc,8,3]
    X = np.einsum("qa,cad->cqd", N, p)
    J = np.einsum("cqd,cqd->cq", np.cross(np.einsum("qa,cad->cqd", dS, p), np.einsum("qa,cad->cqd", dT, p)),
                  np.einsum("qa,cad->cqd", dR, p))
    wj = W[None, :] * J
    F = f(X)
    return np.einsum("cq,cq...->c...", wj, F) / wj.sum(axis=1).reshape((-1,) + (1,) * (F.ndim - 2))


@pytest.mark.parametrize("jit", [0.0, 0.15])
def test_prism_cube_volumes_and_faces(jit):
    xyz, cells, per = I.prism_cube(4, jitter=jit, seed=3)
    o = oracle.Oracle(xyz, cells, per)
    vol = o.geometry()[0]
    assert vol.min() > 0 and abs(vol.sum() - 8.0) < 1e-12
    assert o.n_faces == 5 * len(cells) // 2  # two triangles and three quads per prism
    if jit == 0.0:
        tv = tet_moments(xyz[I.prism_tets(cells).reshape(-1, 4)])[0].reshape(-1, 3).sum(axis=1)
        assert np.allclose(vol, tv, rtol=1e-13)


def test_prism_centroids_and_moments_match_their_tetrahedra():
    """Unjittered prisms are exact unions of three tetrahedra: the parallel
    axis theorem combines the closed-form tetrahedron moments."""
    xyz, cells, _ = I.prism_cube(3)
    rng = np.random.default_rng(11)
    A = np.eye(3) + 0.2 * rng.normal(size=(3, 3))  # shear the lattice: general prisms
    xyz = xyz @ A.T
    o = oracle.Oracle(xyz, cells, None, *_all_far_field(xyz, cells))
    vol, cen, mom, _ = o.geometry()
    tv, tc, tm = tet_moments(xyz[I.prism_tets(cells).reshape(-1, 4)])
    tv, tc, tm = np.abs(tv).reshape(-1, 3), tc.reshape(-1, 3, 3), tm.reshape(-1, 3, 6)
    V = tv.sum(axis=1)
    C = (tv[:, :, None] * tc).sum(axis=1) / V[:, None]
    d = tc - C[:, None, :]
    ia, ib = [0, 1, 2, 0, 1, 2], [0, 1, 2, 1, 2, 0]
    M = np.stack([(tv * (tm[:, :, k] + d[:, :, ia[k]] * d[:, :, ib[k]])).sum(axis=1) / V for k in range(6)], axis=1)
    assert np.allclose(vol, V, rtol=1e-13)
    assert np.allclose(cen, C, atol=1e-13)
    assert np.allclose(mom, M, atol=1e-14)


def surface_flux_of_x(xyz, faces):
    """Sum over faces (node lists [n,4], -1 padded triangles) of the
    integral of x . n dA with the right-hand normal of the node order: exact
    on flat triangles (centroid times area vector) and, by 2x2 Gauss, on
    bilinear quads (the integrand has degree 2 in each parameter)."""
    tot = 0.0
    g = 0.5 + np.array([-0.5, 0.5]) / np.sqrt(3.0)
    for f in faces:
        p = xyz[f[f >= 0]]
        if len(p) == 3:
            tot += p.mean(axis=0) @ (0.5 * np.cross(p[1] - p[0], p[2] - p[0]))
            continue
        for s_ in g:
            for t_ in g:
                x = (1 - s_) * (1 - t_) * p[0] + s_ * (1 - t_) * p[1] + s_ * t_ * p[2] + (1 - s_) * t_ * p[3]
                xs = (1 - t_) * (p[1] - p[0]) + t_ * (p[2] - p[3])
                xt = (1 - s_) * (p[3] - p[0]) + s_ * (p[2] - p[1])
                tot += 0.25 * x @ np.cross(xs, xt)
    return tot


def _all_far_field(xyz, cells):
    """Boundary faces of a non-periodic mesh of prisms, tagged far field."""
    from collections import Counter

    faces = []
    for c in cells:
        tri = [(c[0], c[1], c[2]), (c[4], c[5], c[6])]
        quads = [(c[0], c[1], c[5], c[4]), (c[1], c[2], c[6], c[5]), (c[2], c[0], c[4], c[6])]
        faces += [tuple(f) + (-1,) for f in tri] + [tuple(f) for f in quads]
    cnt = Counter(tuple(sorted(x for x in f if x >= 0)) for f in faces)
    bf = [f for f in faces if cnt[tuple(sorted(x for x in f if x >= 0))] == 1]
    return np.array(bf, dtype=np.int64), np.full(len(bf), I.BC_FARFIELD, dtype=np.int32)


def test_exact_prism_average_matches_quadrature():
    xyz, cells, per = I.prism_cube(6)
    t = 0.41
    a = I.cell_average_sin(xyz, cells, t)
    b = collapsed_average(xyz, cells, lambda x: np.sin(np.pi * (x.sum(-1) - t)), n=8)
    assert np.abs(a - b).max() < 1e-13


def test_linear_field_reconstructed_exactly_on_prisms():
    xyz, cells, per = I.prism_cube(6, jitter=0.15, seed=4)
    o = oracle.Oracle(xyz, cells, per)
    _, cen, _, _ = o.geometry()
    rng = np.random.default_rng(0)
    G = rng.normal(size=(5, 3))
    c0 = rng.normal(size=5)
    o.set_state(c0[None, :] + cen @ G.T)
    o.reconstruct()
    ok = _unshifted_cells(o)
    assert len(ok) >= 10
    for c in ok:
        x = cen[c] + rng.uniform(-0.1, 0.1, 3)
        val, grad = o.recon_eval(c, x)
        assert np.allclose(val, c0 + G @ x, atol=1e-12)
        assert np.allclose(grad, G, atol=1e-11)


def test_quadratic_field_exact_with_linear_weights_on_prisms():
    xyz, cells, per = I.prism_cube(6, jitter=0.15, seed=5)
    o = oracle.Oracle(xyz, cells, per)
    _, cen, _, _ = o.geometry()
    rng = np.random.default_rng(1)
    A = rng.normal(size=(5, 3, 3))
    A = A + A.transpose(0, 2, 1)
    G = rng.normal(size=(5, 3))

    def f(x):
        return np.einsum("...i,vij,...j->...v", x, A, x) + np.einsum("vi,...i->...v", G, x)

    o.set_state(collapsed_average(xyz, cells, f, n=5))
    o.reconstruct(force_linear=True)
    ok = _unshifted_cells(o)
    assert len(ok) >= 10
    for c in ok:
        x = cen[c] + rng.uniform(-0.1, 0.1, 3)
        val, grad = o.recon_eval(c, x)
        assert np.allclose(val, f(x), atol=1e-11)
        assert np.allclose(grad, 2 * np.einsum("vij,j->vi", A, x) + G, atol=1e-10)


def test_prism_cell_mean_is_kept():
    xyz, cells, per = I.prism_cube(4, jitter=0.15, seed=6)
    o = oracle.Oracle(xyz, cells, per)
    q = I.random_smooth_state(xyz, cells, seed=1)
    o.set_state(q)
    o.reconstruct()
    for c in range(0, len(cells), 11):
        def poly(x):
            return np.array([[o.recon_eval(c, xi)[0] for xi in x[0]]])

        mean = collapsed_average(xyz, cells[c:c + 1], poly, n=4)[0]
        assert np.allclose(mean, q[c], atol=1e-13)


def test_free_stream_and_conservation_on_jittered_prisms(oracle_threads):
    xyz, cells, per = I.prism_cube(5, jitter=0.15, seed=7)
    o = oracle.Oracle(xyz, cells, per, mu_ref=2e-3, Pr=0.72, tau_c=1.0)
    q = I.uniform_state(len(cells), 1.1, (0.4, -0.3, 0.2), 0.8)
    o.set_state(q)
    o.step(2)
    assert np.abs(o.get_state()[0] - q).max() < 1e-13
    vol = o.geometry()[0]
    q = I.random_smooth_state(xyz, cells, seed=3)
    o.set_state(q, 0.0)
    tot0 = (q * vol[:, None]).sum(axis=0)
    o.step(3)
    q3 = o.get_state()[0]
    assert np.abs(q3 - q).max() > 1e-4
    assert np.all(np.abs((q3 * vol[:, None]).sum(axis=0) - tot0) <= 1e-13 * np.abs(tot0).max())


@pytest.mark.parametrize("mu", [0.0, 1e-3])
def test_free_stream_preserved_on_hybrid_far_field_shell(oracle_threads, mu):
    xyz, cells, bfn, bft = I.sphere_shell(4, 3, r_far=3.0, jitter=0.1, seed=1, prism_frac=0.4)
    assert 0 < (cells[:, 2] == cells[:, 3]).sum() < len(cells)
    bft = np.full_like(bft, I.BC_FARFIELD)
    qinf = I.free_stream(0.2535)
    o = oracle.Oracle(xyz, cells, None, bfn, bft, qinf=qinf, mu_ref=mu, Pr=0.72, visc_exp=0.7, T_ref=1 / 1.4)
    q = np.tile(qinf, (len(cells), 1))
    o.set_state(q)
    o.step(2)
    assert np.abs(o.get_state()[0] - q).max() < 1e-13


def test_hybrid_wall_shell_runs_and_stays_physical(oracle_threads):
    xyz, cells, bfn, bft = I.sphere_shell(4, 4, r_far=4.0, seed=2, prism_frac=0.5)
    qinf = I.free_stream(0.2535)
    o = oracle.Oracle(xyz, cells, None, bfn, bft, qinf=qinf, mu_ref=0.2535 / 300, Pr=0.72, visc_exp=0.7,
                      T_ref=1 / 1.4, tau_c=1.0)
    vol = o.geometry()[0]
    # the cells fill the region between the wall and far-field surfaces:
    # divergence theorem, V = 1/3 of the flux of x through the boundary
    wall, far = bft == I.BC_WALL, bft == I.BC_FARFIELD
    assert vol.min() > 0
    assert abs(vol.sum() - (surface_flux_of_x(xyz, bfn[far]) - surface_flux_of_x(xyz, bfn[wall])) / 3) < 1e-12 * vol.sum()
    o.set_state(np.tile(qinf, (len(cells), 1)))
    o.step(3)
    q, t, s = o.get_state()
    assert s == 3 and np.all(np.isfinite(q)) and q[:, 0].min() > 0.9


def _wave_error(n, t_end):
    xyz, cells, per = I.prism_cube(n)
    o = oracle.Oracle(xyz, cells, per)
    o.set_state(I.density_wave_state(xyz, cells, 0.0))
    while o.get_state()[1] < t_end:
        o.step(10, t_end=t_end)
    q, t, _ = o.get_state()
    vol = o.geometry()[0]
    e = np.abs(q[:, 0] - I.density_wave_state(xyz, cells, t)[:, 0])
    return (e * vol).sum() / vol.sum()


def test_convergence_order_density_wave_on_prisms(oracle_threads):
    e8, e16 = _wave_error(8, 0.1), _wave_error(16, 0.1)
    order = np.log2(e8 / e16)
    assert 2.6 < order < 3.4, (order, e8, e16)

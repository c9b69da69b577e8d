"""The oracle on full (non-degenerate) hexahedra, pinned by what does not
depend on it: exact reconstruction of linear data under nonlinear weights and
of quadratic data under linear weights (Section 2.3, with the octant
sub-stencils), the cell mean kept, free-stream preservation, conservation,
and third-order convergence to the exact density wave (Section 5.1) on a
jittered periodic hexahedral cube, with exact cell averages from Gauss
quadrature of the trilinear map."""
import numpy as np
import pytest

import oracle
from paper_2407_00656_b300 import inputs as I

from . import cellquad as Q
from .test_oracle_scheme import _unshifted_cells


def hex_average(xyz, cells, f, n):
    X, W = Q.hex_points(xyz[cells], n)
    F = f(X)
    return np.einsum("cq,cq...->c...", W, F) / W.sum(axis=1).reshape((-1,) + (1,) * (F.ndim - 2))


def test_hex_cube_geometry_and_faces():
    xyz, cells, per = I.hex_cube(5, jitter=0.15, seed=1)
    o = oracle.Oracle(xyz, cells, per)
    vol, cen, _, _ = o.geometry()
    X, W = Q.hex_points(xyz[cells], 4)
    assert np.allclose(vol, W.sum(axis=1), rtol=1e-13)
    assert abs(vol.sum() - 8.0) < 1e-12
    assert np.allclose(cen, np.einsum("cq,cqd->cd", W, X) / W.sum(axis=1)[:, None], atol=1e-13)
    assert o.n_faces == 3 * len(cells)
    kind, ids, _, M = o.stencil(0)
    assert M == 8 and len(ids) == 24  # 6 faces, 12 edges, 6 cells two faces away


def test_linear_field_exact_with_nonlinear_weights_on_hexahedra():
    xyz, cells, per = I.hex_cube(7, jitter=0.15, seed=4)
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
        x = cen[c] + rng.uniform(-0.15, 0.15, 3)
        val, grad = o.recon_eval(c, x)
        assert np.allclose(val, c0 + G @ x, atol=1e-12)
        assert np.allclose(grad, G, atol=1e-11)


def test_quadratic_field_exact_with_linear_weights_on_hexahedra():
    xyz, cells, per = I.hex_cube(7, jitter=0.15, seed=5)
    o = oracle.Oracle(xyz, cells, per)
    _, cen, _, _ = o.geometry()
    rng = np.random.default_rng(1)
    A = rng.normal(size=(5, 3, 3))
    A = A + A.transpose(0, 2, 1)
    G = rng.normal(size=(5, 3))

    def f(x):
        return np.einsum("...i,vij,...j->...v", x, A, x) + np.einsum("vi,...i->...v", G, x)

    o.set_state(hex_average(xyz, cells, f, 4))
    o.reconstruct(force_linear=True)
    for c in _unshifted_cells(o):
        x = cen[c] + rng.uniform(-0.15, 0.15, 3)
        val, grad = o.recon_eval(c, x)
        assert np.allclose(val, f(x), atol=1e-11)
        assert np.allclose(grad, 2 * np.einsum("vij,j->vi", A, x) + G, atol=1e-10)


def test_cell_mean_kept_on_hexahedra():
    xyz, cells, per = I.hex_cube(5, jitter=0.15, seed=6)
    o = oracle.Oracle(xyz, cells, per)
    q = I.random_smooth_state(xyz, cells, seed=2)
    o.set_state(q)
    o.reconstruct()
    X, W = Q.hex_points(xyz[cells], 3)
    for c in range(0, len(cells), 17):
        mean = sum(w * o.recon_eval(c, x)[0] for w, x in zip(W[c], X[c])) / W[c].sum()
        assert np.allclose(mean, q[c], atol=1e-13)


def test_free_stream_and_conservation_on_hexahedra(oracle_threads):
    xyz, cells, per = I.hex_cube(5, jitter=0.15, seed=7)
    o = oracle.Oracle(xyz, cells, per, mu_ref=2e-3, Pr=0.72, tau_c=1.0)
    q = I.uniform_state(len(cells), 1.1, (0.4, -0.3, 0.2), 0.8)
    o.set_state(q)
    o.step(2)
    assert np.abs(o.get_state()[0] - q).max() < 1e-13
    vol = o.geometry()[0]
    q = I.random_smooth_state(xyz, cells, seed=3)
    o.set_state(q)
    tot0 = (q * vol[:, None]).sum(axis=0)
    o.step(3)
    q3 = o.get_state()[0]
    assert np.abs(q3 - q).max() > 1e-4
    assert np.all(np.abs((q3 * vol[:, None]).sum(axis=0) - tot0) <= 1e-13 * np.abs(tot0).max())


def _wave_error(n, t_end):
    xyz, cells, per = I.hex_cube(n, jitter=0.15, seed=8)
    exact = lambda t: hex_average(xyz, cells, lambda x: 1 + 0.2 * np.sin(np.pi * (x.sum(-1) - 3 * t)), 6)
    o = oracle.Oracle(xyz, cells, per)
    rho = exact(0.0)
    q = np.stack([rho, rho, rho, rho, 1 / 0.4 + 1.5 * rho], axis=1)  # U = V = W = 1, p = 1
    o.set_state(q)
    while o.get_state()[1] < t_end:
        o.step(10, t_end=t_end)
    qt, t, _ = o.get_state()
    vol = o.geometry()[0]
    e = np.abs(qt[:, 0] - exact(t))
    return (e * vol).sum() / vol.sum()


@pytest.mark.slow
def test_convergence_order_on_jittered_hexahedra(oracle_threads):
    e8 = _wave_error(8, 0.1)
    e16 = _wave_error(16, 0.1)
    order = np.log2(e8 / e16)
    assert 2.6 < order < 3.4, (e8, e16, order)

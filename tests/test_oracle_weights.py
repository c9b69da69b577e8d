"""Pins of the oracle's smoothness indicators and nonlinear weights
(Section 2.3: beta_m, tau_Z and the normalised weights of Eq. weno) by an
independent route.

For quadratic data the big-stencil polynomial P_0 is the quadratic itself, so
beta_0 follows from Gauss quadrature of the squared first and second
derivatives over the cell.  Each linear P_m is the least-squares fit of
Section 2.3 over the sub-stencil as the paper lists it (numpy's SVD solver on
centroid differences, sub-stencils built here from the cells' node lists),
and beta_m from its gradient.  The weights formed from those values must
equal the oracle's.  A second run with epsilon of the size of beta itself
pins the absolute scale of beta, which the weights ignore when epsilon is
negligible.
"""
import numpy as np
import pytest

import oracle
from paper_2407_00656_b300 import inputs as I

from . import cellquad as Q

GLIN = 0.025
# the six second-order multi-indices, each once: xx yy zz xy yz zx
L2 = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0)]


def quadratic_fields(seed):
    """Five random quadratics f_v(x) = x.A_v.x + G_v.x + c_v."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(5, 3, 3))
    A = 0.5 * (A + A.transpose(0, 2, 1))
    G = 0.02 * rng.normal(size=(5, 3))  # curvature dominates: beta_0 and beta_m differ by O(1)
    c0 = np.array([2.0, 0.1, -0.2, 0.3, 5.0])
    f = lambda x: np.einsum("...i,vij,...j->...v", x, A, x) + np.einsum("vi,...i->...v", G, x) + c0
    grad = lambda x: 2 * np.einsum("vij,...j->...vi", A, x) + G  # [..., v, 3]
    return f, grad, A


def expected_weights(beta, eps):
    """tau_Z, omega_m and the normalised weights of Section 2.3."""
    M = len(beta) - 1
    gam = np.array([1 - GLIN * M] + [GLIN] * M)
    tau = np.abs(beta[0] - beta[1:]).sum() / M
    om = gam * (1 + tau / (beta + eps))
    return om / om.sum()


def independent_betas(xyz, cells, nb, c, f, grad, A, X, W):
    """beta_0..beta_M [5, M+1] of cell c for the quadratic data f."""
    vol = W.sum(axis=1)
    cen = np.einsum("cq,cqd->cd", W, X) / vol[:, None]
    qavg = np.einsum("cq,cqv->cv", W, f(X)) / vol[:, None]
    V = vol[c]
    g2 = np.einsum("q,qvi->v", W[c], grad(X[c]) ** 2)  # int |grad f|^2 over the cell
    hess2 = sum((2 * A[:, a, b]) ** 2 for a, b in L2)  # sum_l (d^l f)^2, constant
    beta0 = V ** (2 / 3 - 1) * g2 + V ** (4 / 3 - 1) * V * hess2
    subs = Q.sub_stencils(nb, c, tet=cells.shape[1] == 4)
    betas = [beta0]
    for s in subs:
        D = cen[s] - cen[c]
        g, *_ = np.linalg.lstsq(D, qavg[s] - qavg[c], rcond=None)  # [3, 5]
        betas.append(V ** (2 / 3 - 1) * V * (g ** 2).sum(axis=0))
    return np.stack(betas, axis=1), qavg


def interior_cells(nb, limit):
    """Cells whose neighbours and neighbours' neighbours all exist (no wrap)."""
    out = []
    for c in range(len(nb)):
        if np.all(nb[c] >= 0) and np.all(nb[nb[c]] >= 0):
            out.append(c)
        if len(out) >= limit:
            break
    return out


MESHES = {
    "jittered tets": lambda: I.kuhn_cube(6, jitter=0.15, seed=21),
    "jittered hexahedra": lambda: I.hex_cube(6, jitter=0.15, seed=22),
}


@pytest.mark.parametrize("mesh", sorted(MESHES))
def test_smoothness_indicators_and_weights_by_quadrature(mesh):
    xyz, cells, per = MESHES[mesh]()
    nb = Q.face_neighbours(cells)
    X, W = Q.cell_points(xyz, cells, 4)
    f, grad, A = quadratic_fields(5)
    cand = interior_cells(nb, 12)
    assert len(cand) >= 8
    betas = {}
    qavg = None
    for c in cand:
        betas[c], qavg = independent_betas(xyz, cells, nb, c, f, grad, A, X, W)
    # the beta_0 of the quadratic and the linear fits differ, so the weights
    # are far from linear (a test with linear weights would pin nothing)
    b = np.concatenate([betas[c].ravel() for c in cand])
    eps_scale = float(np.median(b))
    for eps in (1e-8, eps_scale):
        o = oracle.Oracle(xyz, cells, per, eps=eps)
        o.set_state(qavg)
        o.reconstruct()
        far = 0.0
        for c in cand:
            kind, ids, _, M = o.stencil(c)
            assert np.all(kind == 0) and set(ids.tolist()) == Q.two_layer(nb, c)
            got = o.recon_weights(c)  # [5, M+1]
            want = np.stack([expected_weights(betas[c][v], eps) for v in range(5)])
            assert got.shape == want.shape
            assert np.allclose(got, want, rtol=1e-10, atol=1e-13), (c, got, want)
            lin = np.array([1 - GLIN * M] + [GLIN] * M)
            far = max(far, np.abs(want - lin).max())
        assert far > 1e-3


def test_planted_mistakes_change_the_weights():
    """The pin above is sharp: counting the mixed second derivatives twice,
    or dropping the |Omega| powers, moves the weights by far more than its
    tolerance (computed here on the test's own values, not in the oracle)."""
    xyz, cells, per = MESHES["jittered tets"]()
    nb = Q.face_neighbours(cells)
    X, W = Q.cell_points(xyz, cells, 4)
    f, grad, A = quadratic_fields(5)
    c = interior_cells(nb, 1)[0]
    betas, _ = independent_betas(xyz, cells, nb, c, f, grad, A, X, W)
    V = W[c].sum()
    eps = float(np.median(betas))
    base = expected_weights(betas[0], eps)
    twice = betas[0].copy()
    twice[0] += V ** (4 / 3) * sum((2 * A[0, a, b]) ** 2 for a, b in L2[3:])
    nopow = betas[0].copy()
    nopow[0] = np.einsum("q,qi->", W[c], grad(X[c])[:, 0] ** 2) + V * sum((2 * A[0, a, b]) ** 2 for a, b in L2)
    nopow[1:] *= V ** (-2 / 3)
    for bad in (twice, nopow):
        assert np.abs(expected_weights(bad, eps) - base).max() > 1e-6

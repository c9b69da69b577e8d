"""Test-side geometry, written apart from the oracle and the library: Gauss
rules over tetrahedra and trilinear hexahedra, face adjacency from the cells'
node lists, and the WENO sub-stencils of Section 2.3 listed cell by cell."""
import numpy as np

# local faces as Section 2.3 numbers them (1-based in the paper): tet face p
# is opposite node p; hex faces 1 and 6 are the two quads of nodes 0-3 and
# 4-7, faces 2..5 go round the sides
TET_FACES = [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]
HEX_FACES = [(0, 1, 2, 3), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7), (4, 5, 6, 7)]


def tet_points(p, n):
    """Conical-product Gauss rule of n^3 points on tetrahedra p[c,4,3]:
    physical points X[c,q,3] and weights W[c,q] (summing to the volume)."""
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = 0.5 * (x + 1), 0.5 * w
    S, T, U = (a.ravel() for a in np.meshgrid(x, x, x, indexing="ij"))
    wq = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel() * (1 - S) ** 2 * (1 - T)
    lam = np.stack([S, T * (1 - S), U * (1 - S) * (1 - T)], axis=1)
    e = p[:, 1:] - p[:, :1]
    X = p[:, None, 0, :] + np.einsum("qk,ckd->cqd", lam, e)
    det = np.abs(np.linalg.det(e))
    return X, det[:, None] * wq[None, :]


def hex_points(p, n):
    """n^3 Gauss-Legendre points of the trilinear map of hexahedra p[c,8,3]:
    X[c,q,3] and weights W[c,q] = w |J| (summing to the volume)."""
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = 0.5 * (x + 1), 0.5 * w
    s, t, r = (a.ravel() for a in np.meshgrid(x, x, x, indexing="ij"))
    wq = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()
    corners = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]

    def lin(u, k):
        return u if k else 1 - u

    def dlin(k):
        return 1.0 if k else -1.0

    N = np.stack([lin(s, a) * lin(t, b) * lin(r, c) for a, b, c in corners], axis=1)
    dS = np.stack([dlin(a) * lin(t, b) * lin(r, c) for a, b, c in corners], axis=1)
    dT = np.stack([lin(s, a) * dlin(b) * lin(r, c) for a, b, c in corners], axis=1)
    dR = np.stack([lin(s, a) * lin(t, b) * dlin(c) for a, b, c in corners], axis=1)
    X = np.einsum("qa,cad->cqd", N, p)
    J = np.stack([np.einsum("qa,cad->cqd", d, p) for d in (dS, dT, dR)], axis=-1)  # [c,q,3,3]
    return X, np.abs(np.linalg.det(J)) * wq[None, :]


def cell_points(xyz, cells, n):
    p = xyz[cells]
    return tet_points(p, n) if cells.shape[1] == 4 else hex_points(p, n)


def face_neighbours(cells):
    """nb[c][p]: the cell across local face p of cell c (-1 on the boundary),
    found by matching the faces' node sets."""
    faces = TET_FACES if cells.shape[1] == 4 else HEX_FACES
    owner = {}
    nb = -np.ones((len(cells), len(faces)), dtype=np.int64)
    for c, cn in enumerate(cells):
        for p, loc in enumerate(faces):
            key = frozenset(int(cn[i]) for i in loc)
            if key in owner:
                d, q = owner.pop(key)
                nb[c, p], nb[d, q] = d, c
            else:
                owner[key] = (c, p)
    return nb


def sub_stencils(nb, c, tet):
    """The sub-stencils of cell c as Section 2.3 lists them, without c itself.
    Tetrahedra (faces 1..4): S_1 = {1,2,3}, S_2 = {1,2,4}, S_3 = {2,3,4},
    S_4 = {3,1,4} plus the three other neighbours of neighbour m.  Hexahedra:
    {1 or 6, m, m+1} over the sides 2..5 taken cyclically."""
    out = []
    if tet:
        lists = [(1, 2, 3), (1, 2, 4), (2, 3, 4), (3, 1, 4)]
        for m, faces in enumerate(lists, start=1):
            s = [int(nb[c, f - 1]) for f in faces]
            s += [int(x) for x in nb[nb[c, m - 1]] if x != c]
            out.append(list(dict.fromkeys(s)))
    else:
        for cap in (1, 6):
            for m in range(4):
                s1, s2 = 2 + m, 2 + (m + 1) % 4
                out.append([int(nb[c, cap - 1]), int(nb[c, s1 - 1]), int(nb[c, s2 - 1])])
    return out


def two_layer(nb, c):
    """All cells reached from c in one or two face steps (c excluded)."""
    first = [int(x) for x in nb[c] if x >= 0]
    second = [int(y) for x in first for y in nb[x] if y >= 0]
    return set(first + second) - {c}

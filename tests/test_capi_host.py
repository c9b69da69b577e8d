"""Host-side checks of libhgks: it loads without a GPU, exports every entry
point declared in include/hgks.h, and its mesh builder (pure host code)
produces the expected connectivity or a clear error."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2407_00656_b300 import build as B
from paper_2407_00656_b300 import hgks as H
from paper_2407_00656_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hgks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hgks_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(H.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(H.EXPORTS) <= set(names)


def test_params_default():
    p = H.params_default()
    assert p.gamma == 1.4 and p.cfl == 0.4 and p.weno_eps == 1e-8 and p.weno_gamma_lin == 0.025
    assert p.precision == H.HGKS_FP64 and p.use_graph == 1


@pytest.mark.parametrize("n,jit", [(4, 0.0), (7, 0.15)])
def test_periodic_tet_mesh_connectivity(n, jit):
    xyz, cells, per = I.kuhn_cube(n, jitter=jit, seed=2)
    m = H.Mesh(xyz, cells, per)
    assert m.n_cells == 6 * n ** 3
    assert m.n_faces == 12 * n ** 3  # every face shared by two cells
    assert m.n_ghosts == 0
    assert 12 <= m.stencil_size <= 16
    assert m.device_bytes(H.HGKS_FP64) > m.device_bytes(H.HGKS_FP32_MIXED) > 0


def test_sphere_shell_connectivity():
    nq, nr = 5, 4
    xyz, cells, bfn, bft = I.sphere_shell(nq, nr, r_far=3.0)
    m = H.Mesh(xyz, cells, None, bfn, bft)
    nc = 6 * nq * nq * nr
    assert m.n_cells == nc
    nb = 2 * 6 * nq * nq
    assert m.n_ghosts == nb
    assert m.n_faces == (6 * nc + nb) // 2
    assert m.stencil_size == 24


def test_errors_are_reported_not_raised_by_abort():
    xyz, cells, per = I.kuhn_cube(3)
    with pytest.raises(H.HGKSError) as e:
        H.Mesh(xyz, cells, None)  # unmatched boundary faces, no periods, no tags
    assert e.value.code == H.HGKS_EMESH
    bad = cells.copy()
    bad[0, 2], bad[0, 3] = bad[0, 3], bad[0, 2]  # inverted cell
    with pytest.raises(H.HGKSError) as e:
        H.Mesh(xyz, bad, per)
    assert e.value.code == H.HGKS_EMESH and "non-positive volume" in str(e.value)
    oob = cells.copy()
    oob[5, 1] = len(xyz) + 3
    with pytest.raises(H.HGKSError) as e:
        H.Mesh(xyz, oob, per)
    assert e.value.code == H.HGKS_EINVAL
    with pytest.raises(H.HGKSError) as e:
        H.Mesh(xyz, cells[:, :3], per)
    assert e.value.code == H.HGKS_EINVAL


def test_init_rejects_bad_parameters_before_touching_the_device():
    xyz, cells, per = I.kuhn_cube(3)
    m = H.Mesh(xyz, cells, per)
    q = I.uniform_state(m.n_cells)
    for kw in (dict(gamma=0.9), dict(cfl=0.0), dict(precision=7), dict(weno_eps=0.0)):
        with pytest.raises(H.HGKSError) as e:
            H.Solver(m, q, **kw)
        assert e.value.code == H.HGKS_EINVAL
    assert m.n_cells == len(cells)  # the caller still owns the mesh


def test_device_byte_accounting_splits_into_mesh_and_solver_parts():
    xyz, cells, per = I.kuhn_cube(5, jitter=0.1, seed=2)
    m = H.Mesh(xyz, cells, per)
    assert m.info(5) == m.info(7) + m.info(8)
    assert m.info(6) == m.info(7) + m.info(9)
    # binary32 work arrays are smaller than binary64 ones; the mesh arrays are shared
    assert 0 < m.info(9) < m.info(8) < m.info(7)

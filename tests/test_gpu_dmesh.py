"""Device meshes shared by solvers (hgks_dmesh_create / hgks_init_shared):
the same kernels run on the same arrays, so a solver over a shared device
mesh gives bitwise the result of hgks_init on its own copy; the device mesh
lives until its last solver is destroyed."""
import numpy as np
import pytest

from paper_2407_00656_b300 import hgks as H
from paper_2407_00656_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [H.HGKS_FP64, H.HGKS_FP32_MIXED])
def test_shared_device_mesh_matches_a_private_copy(precision):
    xyz, cells, per = I.kuhn_cube(7, jitter=0.15, seed=3)
    mesh = H.Mesh(xyz, cells, per)
    q1 = I.density_wave_state(xyz, cells, 0.0)
    q2 = I.random_smooth_state(xyz, cells, seed=5)
    dm = H.DeviceMesh(mesh)
    assert dm.n_cells == mesh.n_cells and dm.bytes == mesh.static_bytes
    assert dm.work_bytes(precision) == mesh.work_bytes(precision)
    a = H.Solver(dm, q1, precision=precision)
    b = H.Solver(dm, q2, precision=precision)
    assert dm.solvers == 2
    a.step(6)
    b.step(6)
    ref = {}
    for q in (q1, q2):
        s = H.Solver(mesh.clone(), q, precision=precision)
        s.step(6)
        ref[id(q)] = s.read()
        s.close()
    for s, q in ((a, q1), (b, q2)):
        got = s.read()
        assert got[2] == ref[id(q)][2] and got[1] == ref[id(q)][1]
        assert np.array_equal(got[0], ref[id(q)][0])


def test_device_mesh_outlives_its_release_while_solvers_use_it():
    xyz, cells, bfn, bft = I.sphere_shell(4, 4, r_far=3.0, jitter=0.1, seed=1)
    mesh = H.Mesh(xyz, cells, None, bfn, bft)
    qinf = I.free_stream(0.2535)
    q = np.tile(qinf, (len(cells), 1))
    kw = dict(q_inf=qinf, mu_ref=0.2535 / 200, Pr=0.72, visc_exp=0.7, T_ref=1 / 1.4, tau_num_c=1.0,
              precision=H.HGKS_FP32_MIXED)
    dm = H.DeviceMesh(mesh)
    s = H.Solver(dm, q, **kw)
    dm.release()  # the solver keeps the device mesh alive
    s.step(5)
    got, t, n = s.read()
    ref = H.Solver(mesh, q, **kw)
    ref.step(5)
    want = ref.read()
    assert n == want[2] == 5 and t == want[1]
    assert np.array_equal(got, want[0])
    s.close()
    ref.close()


def test_default_flux_variant_follows_the_face_count():
    """Per Gauss point on small meshes, per face on large ones (the crossovers
    measured on B300: 16 blocks of 128 faces per SM in FP64, 2 in mixed)."""
    small = I.kuhn_cube(6, jitter=0.1, seed=1)
    large = I.kuhn_cube(40, jitter=0.1, seed=1)  # 768,000 faces
    for precision in (H.HGKS_FP64, H.HGKS_FP32_MIXED):
        for (xyz, cells, per), want in ((small, 1), (large, 0)):
            s = H.Solver(H.Mesh(xyz, cells, per), I.uniform_state(len(cells)), precision=precision)
            assert s.tuning == (want, 0), (precision, len(cells))
            s.close()

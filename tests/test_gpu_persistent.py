"""Persistent steps (hgks_params.persistent = 1): n S2O4 steps of a mesh or a
batch of meshes in one cooperative launch, phases separated by grid-wide
barriers.  The phases run the device functions of the separate kernels, so
the results agree with the graph-launched steps to a few units in the last
place (the compiler may fuse multiplies and adds differently in the one big
kernel), with the same step counts, times and status."""
import numpy as np
import pytest

from paper_2407_00656_b300 import hgks as H
from paper_2407_00656_b300 import inputs as I

pytestmark = pytest.mark.gpu


def close(a, b, precision):
    tol = 1e-13 if precision == H.HGKS_FP64 else 2e-6
    mag = np.abs(b).max(axis=0)
    mag[1:4] = mag[1:4].max()
    return np.all(np.abs(a - b) <= tol * mag)


@pytest.mark.parametrize("precision", [H.HGKS_FP64, H.HGKS_FP32_MIXED])
def test_persistent_steps_match_graph_steps_on_one_mesh(precision):
    xyz, cells, per = I.kuhn_cube(6, jitter=0.15, seed=2)
    q = I.density_wave_state(xyz, cells, 0.0)
    out = {}
    for pers in (0, 1):
        s = H.Solver(H.Mesh(xyz, cells, per), q, precision=precision, persistent=pers)
        s.step(5)
        t5 = s.read()[1]
        s.step(10, t_end=1.7 * t5)  # the last step is clipped, the rest do nothing
        out[pers] = (s.read(), t5)
        s.close()
    ((qg, tg, ng), t5g), ((qp, tp, np_), t5p) = out[0], out[1]
    assert abs(t5g - t5p) <= 1e-6 * t5g
    assert ng == np_ and abs(tp - 1.7 * t5p) <= 1e-15 and abs(tg - 1.7 * t5g) <= 1e-15
    assert close(qp, qg, precision)


@pytest.mark.parametrize("precision", [H.HGKS_FP64, H.HGKS_FP32_MIXED])
def test_persistent_steps_of_a_viscous_hex_batch(precision):
    meshes, qs = [], []
    qinf = I.free_stream(0.2535)
    for n, seed in ((4, 1), (5, 2), (4, 3)):
        xyz, cells, bfn, bft = I.sphere_shell(n, 4, r_far=3.0, jitter=0.1, seed=seed)
        meshes.append((xyz, cells, bfn, bft))
        q = np.tile(qinf, (len(cells), 1))
        q[:, 0] *= 1 + 0.02 * np.sin(np.arange(len(cells)) + seed)
        qs.append(q)
    kw = dict(precision=precision, q_inf=qinf, mu_ref=0.2535 / 250, Pr=0.72, visc_exp=0.7, T_ref=1 / 1.4,
              tau_num_c=1.0)
    res = {}
    for pers in (0, 1):
        s = H.Solver([H.Mesh(x, c, None, b, t) for x, c, b, t in meshes], qs, persistent=pers, **kw)
        s.step(6)
        res[pers] = [s.member_read(i) for i in range(3)]
        s.close()
    for (qg, tg, ng), (qp, tp, np_) in zip(res[0], res[1]):
        assert ng == np_ == 6 and tg == tp
        assert close(qp, qg, precision)


def test_persistent_steps_report_a_nonfinite_state():
    xyz, cells, per = I.kuhn_cube(5, jitter=0.1, seed=4)
    q = I.density_wave_state(xyz, cells, 0.0)
    s = H.Solver(H.Mesh(xyz, cells, per), q, precision=H.HGKS_FP32_MIXED, persistent=1)
    bad = q.copy()
    bad[7, 0] = np.nan
    s.write(bad, 0.0)
    s.step(2, dt_fixed=1e-4)
    with pytest.raises(H.HGKSError) as e:
        s.read()
    assert e.value.code == H.HGKS_ENONFINITE
    s.close()

"""GPU parity on triangular prisms (hexahedra with nodes 2 = 3 and 6 = 7) and
hybrid hex/prism sphere shells, through the C ABI, against the CPU oracle
(FP64, 1e-11 relative per variable's largest magnitude, as in
test_gpu_parity), plus the behaviour checks of the hexahedral path:
free stream, conservation, mixed-precision error, batches, kernel variants
and persistent steps on meshes that mix the two cell shapes."""
import numpy as np
import pytest

import oracle
from paper_2407_00656_b300 import hgks as H
from paper_2407_00656_b300 import inputs as I

from .test_gpu_batch import _same
from .test_gpu_parity import TOL, both, relerr
from .test_gpu_persistent import close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def threads():
    oracle.set_threads(8)


def hybrid(n=5, n_r=4, frac=0.4, r_far=3.0, jitter=0.15, seed=5):
    xyz, cells, bfn, bft = I.sphere_shell(n, n_r, r_far=r_far, jitter=jitter, seed=seed, prism_frac=frac)
    assert 0 < (cells[:, 2] == cells[:, 3]).sum() < len(cells)
    return xyz, cells, bfn, bft


def shell_state(cells, qinf, seed=0, amp=0.05):
    rng = np.random.default_rng(seed)
    q = np.tile(qinf, (len(cells), 1))
    q[:, 0] *= 1 + amp * rng.uniform(-1, 1, len(cells))
    q[:, 1:4] += amp * rng.uniform(-1, 1, (len(cells), 3))
    return q


@pytest.mark.parametrize("kw", [{}, dict(mu_ref=2e-3, Pr=0.72, tau_c=1.0)])
def test_stage_operator_on_jittered_prism_cube(kw):
    xyz, cells, per = I.prism_cube(7, jitter=0.15, seed=1)  # 686 prisms: ragged last block
    q = I.random_smooth_state(xyz, cells, seed=2)
    s, o = both(xyz, cells, per, q=q, **kw)
    for dt in (1e-3, 2e-2):
        L, dL = s.stage_operator(dt)
        Lo, dLo = o.operator(dt)
        assert relerr(L, Lo) < TOL
        assert relerr(dL, dLo) < TOL


@pytest.mark.parametrize("mach", [0.2535, 1.5])
def test_stage_operator_on_hybrid_shell_with_wall_and_far_field(mach):
    xyz, cells, bfn, bft = hybrid()
    qinf = I.free_stream(mach)
    q = shell_state(cells, qinf)
    s, o = both(xyz, cells, None, bfn, bft, q=q, qinf=qinf, mu_ref=mach / 300, Pr=0.72, visc_exp=0.7,
                T_ref=1 / 1.4, tau_c=1.0)
    L, dL = s.stage_operator(5e-3)
    Lo, dLo = o.operator(5e-3)
    assert relerr(L, Lo) < TOL
    assert relerr(dL, dLo) < TOL


def test_hybrid_shell_steps_match_oracle():
    xyz, cells, bfn, bft = hybrid(frac=0.5, seed=6)
    qinf = I.free_stream(0.2535)
    q = shell_state(cells, qinf, seed=1, amp=0.03)
    s, o = both(xyz, cells, None, bfn, bft, q=q, qinf=qinf, mu_ref=0.2535 / 200, Pr=0.72, visc_exp=0.7,
                T_ref=1 / 1.4, tau_c=1.0)
    s.step(3)
    o.step(3)
    qg, tg, ng = s.read()
    qo, to, no = o.get_state()
    assert ng == no == 3 and abs(tg - to) <= 1e-12 * to
    assert relerr(qg, qo) < TOL


@pytest.mark.parametrize("use_graph", [1, 0])
def test_density_wave_steps_on_prisms_match_oracle(use_graph):
    xyz, cells, per = I.prism_cube(8)
    q = I.density_wave_state(xyz, cells, 0.0)
    s, o = both(xyz, cells, per, q=q, use_graph=use_graph)
    s.step(4)
    o.step(4)
    qg, tg, ng = s.read()
    qo, to, no = o.get_state()
    assert ng == no == 4 and abs(tg - to) <= 1e-15 * 4 * to
    assert relerr(qg, qo) < 5 * TOL


def test_free_stream_and_conservation_on_prisms():
    xyz, cells, per = I.prism_cube(6, jitter=0.15, seed=5)
    q = I.uniform_state(len(cells), 1.1, (0.4, -0.3, 0.2), 0.8)
    s = H.Solver(H.Mesh(xyz, cells, per), q, mu_ref=1e-3, Pr=0.72)
    s.step(3)
    assert np.abs(s.read()[0] - q).max() < 1e-13
    q = I.random_smooth_state(xyz, cells, seed=6)
    vol = oracle.Oracle(xyz, cells, per).geometry()[0]
    s.write(q, 0.0)
    s.step(3)
    q3 = s.read()[0]
    t0, t3 = (q * vol[:, None]).sum(0), (q3 * vol[:, None]).sum(0)
    assert np.all(np.abs(t3 - t0) <= 1e-13 * np.abs(t0).max())


def test_mixed_precision_error_on_prisms():
    """FP32-mixed against FP64 after 20 steps of the jittered density wave on
    prisms: L1 of rho, rhoU and rhoE below 1e-5 relative."""
    xyz, cells, per = I.prism_cube(12, jitter=0.15, seed=0)
    q = I.density_wave_state(xyz, cells, 0.0)
    res = []
    for prec in (H.HGKS_FP64, H.HGKS_FP32_MIXED):
        s = H.Solver(H.Mesh(xyz, cells, per), q, precision=prec)
        s.step(20)
        res.append(s.read()[0])
    vol = oracle.Oracle(xyz, cells, per).geometry()[0]
    for v in (0, 1, 4):
        l1 = (np.abs(res[1][:, v] - res[0][:, v]) * vol).sum() / (np.abs(res[0][:, v]) * vol).sum()
        assert l1 < 1e-5, (v, l1)


@pytest.mark.parametrize("precision", [H.HGKS_FP64, H.HGKS_FP32_MIXED])
def test_batch_of_hex_prism_and_hybrid_meshes_equals_single_solvers(precision):
    """One batch holds a hexahedral shell and a hybrid shell (their
    stencils padded to the larger size): every member equals its
    single-mesh solver bitwise, the collapsed prism sides of the second
    reading the batch's zero flux record."""
    qinf = I.free_stream(0.2535)
    x1, c1, b1, t1 = I.sphere_shell(4, 3, r_far=3.0, jitter=0.1, seed=1)
    x2, c2, b2, t2 = hybrid(n=4, n_r=3, seed=2)
    kw = dict(precision=precision, q_inf=qinf, mu_ref=1e-3, Pr=0.72, visc_exp=0.7, T_ref=1 / 1.4, tau_num_c=1.0)
    members = [(x1, c1, None, b1, t1, shell_state(c1, qinf, 1)), (x2, c2, None, b2, t2, shell_state(c2, qinf, 2))]
    batch = H.Solver([H.Mesh(x, c, p, b, t) for x, c, p, b, t, _ in members], [m[-1] for m in members], **kw)
    batch.step(4)
    for i, (x, c, p, b, t, q) in enumerate(members):
        single = H.Solver(H.Mesh(x, c, p, b, t), q, **kw)
        single.step(4)
        qs, ts, ns = single.read()
        qb, tb, nb = batch.member_read(i)
        assert ns == nb == 4 and ts == tb
        assert np.array_equal(qs, qb)


@pytest.mark.parametrize("precision", [H.HGKS_FP64, H.HGKS_FP32_MIXED])
def test_kernel_variants_and_persistent_steps_on_hybrid_shell(precision):
    xyz, cells, bfn, bft = hybrid(seed=4)
    qinf = I.free_stream(0.2535)
    q = shell_state(cells, qinf, seed=3, amp=0.02)
    kw = dict(precision=precision, q_inf=qinf, mu_ref=0.2535 / 300, Pr=0.72, visc_exp=0.7, T_ref=1 / 1.4,
              tau_num_c=1.0)
    ref = None
    for fv in (0, 1):
        for rv in (0, 1):
            s = H.Solver(H.Mesh(xyz, cells, None, bfn, bft), q, **kw)
            s.set_tuning(fv, rv)
            s.step(3)
            out = s.read()[0]
            if ref is None:
                ref = out
            assert _same(out, ref, precision), (fv, rv)
    s = H.Solver(H.Mesh(xyz, cells, None, bfn, bft), q, persistent=1, **kw)
    s.set_tuning(0, 0)
    s.step(3)
    assert close(s.read()[0], ref, precision)

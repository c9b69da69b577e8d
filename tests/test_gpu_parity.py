"""GPU parity of libhgks against the CPU oracle (FP64), element by element on
the same seeded inputs, through the C ABI.

Tolerance (FP64 path): the one-step and stage-operator results must agree
with the oracle to 1e-11 relative to each variable's largest magnitude over
the mesh.  Both sides evaluate the same formulas in binary64 in different
orders (and with different, exactly equivalent, algebra for the moment sums),
so they differ by accumulated rounding only; 1e-11 leaves about three orders
of magnitude above the observed differences.
"""
import numpy as np
import pytest

import oracle
from paper_2407_00656_b300 import hgks as H
from paper_2407_00656_b300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def threads():
    oracle.set_threads(8)


def relerr(a, b):
    scale = np.maximum(np.abs(b).max(axis=0), 1e-300)
    return (np.abs(a - b).max(axis=0) / scale).max()


def both(xyz, cells, per=None, bfn=None, bft=None, q=None, precision=0, **params):
    m = H.Mesh(xyz, cells, per, bfn, bft)
    ov = {k: v for k, v in params.items() if k != "use_graph"}
    o = oracle.Oracle(xyz, cells, per, bfn, bft, **{_okey(k): v for k, v in ov.items()})
    s = H.Solver(m, q, **{_hkey(k): v for k, v in params.items()}, precision=precision)
    o.set_state(q)
    return s, o


def _okey(k):
    return {"tau_num_c": "tau_c", "q_inf": "qinf"}.get(k, k)


def _hkey(k):
    return {"tau_c": "tau_num_c", "qinf": "q_inf"}.get(k, k)


def test_stage_operator_inviscid_jittered_tets():
    xyz, cells, per = I.kuhn_cube(7, jitter=0.15, seed=1)  # 2058 cells: ragged last block
    q = I.random_smooth_state(xyz, cells, seed=2)
    s, o = both(xyz, cells, per, q=q)
    for dt in (1e-3, 2e-2):
        L, dL = s.stage_operator(dt)
        Lo, dLo = o.operator(dt)
        assert relerr(L, Lo) < TOL
        assert relerr(dL, dLo) < TOL


@pytest.mark.parametrize("kw", [dict(mu_ref=2e-3, Pr=0.72), dict(mu_ref=1e-3, Pr=1.0, tau_c=1.0),
                                dict(mu_ref=5e-4, Pr=0.72, visc_exp=0.7, T_ref=0.8, tau_c=0.5)])
def test_stage_operator_viscous_jittered_tets(kw):
    xyz, cells, per = I.kuhn_cube(6, jitter=0.15, seed=3)
    q = I.random_smooth_state(xyz, cells, seed=4, amp=0.08)
    s, o = both(xyz, cells, per, q=q, **kw)
    L, dL = s.stage_operator(0.01)
    Lo, dLo = o.operator(0.01)
    assert relerr(L, Lo) < TOL
    assert relerr(dL, dLo) < TOL


@pytest.mark.parametrize("mach", [0.2535, 1.5])
def test_stage_operator_sphere_shell_wall_and_far_field(mach):
    """Hexahedra, no-slip wall, far field (at Ma 1.5 the far field has
    supersonic inflow upstream and supersonic outflow downstream), viscous
    with the power law and numerical collision time."""
    xyz, cells, bfn, bft = I.sphere_shell(6, 5, r_far=4.0, jitter=0.2, seed=3)
    qinf = I.free_stream(mach)
    rng = np.random.default_rng(0)
    q = np.tile(qinf, (len(cells), 1))
    q[:, 0] *= 1 + 0.05 * rng.uniform(-1, 1, len(cells))
    q[:, 1:4] += 0.05 * rng.uniform(-1, 1, (len(cells), 3))
    s, o = both(xyz, cells, None, bfn, bft, q=q, qinf=qinf, mu_ref=mach / 300, Pr=0.72, visc_exp=0.7,
                T_ref=1 / 1.4, tau_c=1.0)
    L, dL = s.stage_operator(5e-3)
    Lo, dLo = o.operator(5e-3)
    assert relerr(L, Lo) < TOL
    assert relerr(dL, dLo) < TOL


def test_sphere_shell_steps_match_oracle():
    """Three full S2O4 steps on hexahedra with wall and far-field ghosts."""
    xyz, cells, bfn, bft = I.sphere_shell(5, 4, r_far=3.0, jitter=0.15, seed=5)
    qinf = I.free_stream(0.2535)
    q = np.tile(qinf, (len(cells), 1))
    q[:, 0] *= 1 + 0.03 * np.sin(np.arange(len(cells)))
    s, o = both(xyz, cells, None, bfn, bft, q=q, qinf=qinf, mu_ref=0.2535 / 200, Pr=0.72, visc_exp=0.7,
                T_ref=1 / 1.4, tau_c=1.0)
    s.step(3)
    o.step(3)
    qg, tg, ng = s.read()
    qo, to, no = o.get_state()
    assert ng == no == 3 and abs(tg - to) <= 1e-12 * to
    assert relerr(qg, qo) < TOL


@pytest.mark.parametrize("use_graph", [1, 0])
def test_density_wave_steps_match_oracle(use_graph):
    xyz, cells, per = I.kuhn_cube(8)  # 3072 cells, the accuracy-test mesh at 8^3
    q = I.density_wave_state(xyz, cells, 0.0)
    s, o = both(xyz, cells, per, q=q, use_graph=use_graph)
    s.step(1)
    o.step(1)
    qg, tg, ng = s.read()
    qo, to, no = o.get_state()
    assert ng == no == 1 and abs(tg - to) <= 1e-15 * to
    assert relerr(qg, qo) < TOL
    s.step(4)
    o.step(4)
    qg, tg, _ = s.read()
    qo, to, _ = o.get_state()
    assert relerr(qg, qo) < 5 * TOL


def test_graph_and_plain_launches_are_bitwise_equal():
    xyz, cells, per = I.kuhn_cube(6, jitter=0.15, seed=9)
    q = I.random_smooth_state(xyz, cells, seed=9)
    out = []
    for g in (1, 0):
        m = H.Mesh(xyz, cells, per)
        s = H.Solver(m, q, use_graph=g, mu_ref=1e-3, Pr=0.72)
        s.step(3)
        out.append(s.read()[0])
    assert np.array_equal(out[0], out[1])


def test_t_end_clipping_and_restart():
    xyz, cells, per = I.kuhn_cube(5)
    q = I.density_wave_state(xyz, cells, 0.0)
    s, o = both(xyz, cells, per, q=q)
    s.step(50, t_end=0.05)
    qg, tg, ng = s.read()
    while o.get_state()[1] < 0.05:
        o.step(1, t_end=0.05)
    qo, to, no = o.get_state()
    assert tg == to == 0.05 or abs(tg - 0.05) < 1e-15
    assert ng == no
    assert relerr(qg, qo) < 10 * TOL
    # restart from the read state continues identically to a continuous run
    s.write(qg, tg)
    s.step(2)
    q1 = s.read()[0]
    m2 = H.Mesh(xyz, cells, per)
    s2 = H.Solver(m2, q)
    s2.step(50, t_end=0.05)
    s2.step(2)
    assert np.array_equal(q1, s2.read()[0])


def test_free_stream_and_conservation_on_gpu():
    xyz, cells, per = I.kuhn_cube(6, jitter=0.15, seed=5)
    q = I.uniform_state(len(cells), 1.1, (0.4, -0.3, 0.2), 0.8)
    m = H.Mesh(xyz, cells, per)
    s = H.Solver(m, q, mu_ref=1e-3, Pr=0.72)
    s.step(3)
    assert np.abs(s.read()[0] - q).max() < 1e-13
    q = I.random_smooth_state(xyz, cells, seed=6)
    vol = oracle.Oracle(xyz, cells, per).geometry()[0]
    s.write(q, 0.0)
    s.step(3)
    q3 = s.read()[0]
    t0 = (q * vol[:, None]).sum(0)
    t3 = (q3 * vol[:, None]).sum(0)
    assert np.all(np.abs(t3 - t0) <= 1e-13 * np.abs(t0).max())


def test_nonfinite_state_is_reported():
    xyz, cells, per = I.kuhn_cube(4)
    q = I.uniform_state(len(cells))
    m = H.Mesh(xyz, cells, per)
    s = H.Solver(m, q)
    bad = q.copy()
    bad[17, 0] = np.nan  # host-side fault injection
    s.write(bad, 0.0)
    s.step(1, dt_fixed=1e-3)
    with pytest.raises(H.HGKSError) as e:
        s.read()
    assert e.value.code == H.HGKS_ENONFINITE


def test_mixed_precision_error_against_fp64():
    """FP32 reconstruction and flux with FP64 accumulation: L1 difference of
    rho, rhoU and rhoE from the FP64 path below 1e-5 relative after 20 steps
    of the jittered density wave."""
    xyz, cells, per = I.kuhn_cube(12, jitter=0.15, seed=0)
    q = I.density_wave_state(xyz, cells, 0.0)
    res = []
    for prec in (H.HGKS_FP64, H.HGKS_FP32_MIXED):
        m = H.Mesh(xyz, cells, per)
        s = H.Solver(m, q, precision=prec)
        s.step(20)
        res.append(s.read()[0])
    vol = oracle.Oracle(xyz, cells, per).geometry()[0]
    for v in (0, 1, 4):
        l1 = (np.abs(res[1][:, v] - res[0][:, v]) * vol).sum() / (np.abs(res[0][:, v]) * vol).sum()
        assert l1 < 1e-5, (v, l1)


def test_full_size_jittered_mesh_one_step():
    """663,552 jittered tets (48^3 x 6): one FP64 step, every cell."""
    xyz, cells, per = I.kuhn_cube(48, jitter=0.15, seed=0)
    q = I.density_wave_state(xyz, cells, 0.0)
    s, o = both(xyz, cells, per, q=q)
    s.step(1)
    o.step(1)
    assert relerr(s.read()[0], o.get_state()[0]) < TOL


@pytest.mark.parametrize("kw", [dict(), dict(mu_ref=2e-3, Pr=0.72, tau_c=1.0)], ids=["inviscid", "viscous"])
def test_periodic_jittered_hexahedra_stage_operator_and_steps(kw):
    """Full hexahedra with non-planar faces on a periodic cube (7^3 = 343
    cells, a ragged last block): stage operator and three full steps."""
    xyz, cells, per = I.hex_cube(7, jitter=0.15, seed=9)
    q = I.random_smooth_state(xyz, cells, seed=5, amp=0.08)
    s, o = both(xyz, cells, per, q=q, **kw)
    L, dL = s.stage_operator(0.01)
    Lo, dLo = o.operator(0.01)
    assert relerr(L, Lo) < TOL
    assert relerr(dL, dLo) < TOL
    s.step(3)
    o.step(3)
    qg, t, n = s.read()
    qo, to, no = o.get_state()
    assert n == no == 3 and abs(t - to) <= 1e-15 * to
    assert relerr(qg, qo) < TOL
    s.close()


def test_full_size_sphere_shell_one_step():
    """The 1.51M-cell hex shell of the bench's sphere line (6 x 58^2 x 75,
    Ma 0.2535, Re 300, power-law viscosity, numerical collision time, wall and
    far field), from the free stream with smooth seeded perturbations of a
    few percent: one FP64 step against the oracle, every cell; the mixed
    path's step within its L1 bound."""
    import os

    xyz, cells, bfn, bft = I.sphere_shell(58, 75, seed=0)
    qinf = I.free_stream(0.2535)
    cen = xyz[cells].mean(axis=1)
    rng = np.random.default_rng(3)
    pert = np.zeros((len(cells), 3))
    for j in range(3):
        for _ in range(3):
            k = rng.normal(size=3) * 0.6
            pert[:, j] += np.sin(cen @ k + rng.uniform(0, 2 * np.pi))
    rho = 1.0 + 0.02 * pert[:, 0]
    u = np.stack([0.2535 * (1 + 0.05 * pert[:, 1]), 0.01 * pert[:, 2], np.zeros(len(cells))], axis=1)
    p = (1 + 0.02 * pert[:, 2]) / 1.4
    q = np.empty((len(cells), 5))
    q[:, 0] = rho
    q[:, 1:4] = rho[:, None] * u
    q[:, 4] = p / 0.4 + 0.5 * rho * (u * u).sum(axis=1)
    params = dict(qinf=qinf, mu_ref=0.2535 / 300, Pr=0.72, visc_exp=0.7, T_ref=1 / 1.4, tau_c=1.0)
    oracle.set_threads(os.cpu_count() or 8)
    s, o = both(xyz, cells, None, bfn, bft, q=q, **params)
    s.step(1)
    o.step(1)
    qg, t, n = s.read()
    qo, to, no = o.get_state()
    s.close()
    # the step is the viscous bound rho h^2/(2 mu) with mu from the power law,
    # whose pow() the host and device libraries round a few units apart
    assert n == no == 1 and abs(t - to) <= 1e-13 * to
    assert relerr(qg, qo) < TOL
    m = H.Solver(H.Mesh(xyz, cells, None, bfn, bft), q, precision=H.HGKS_FP32_MIXED,
                 **{_hkey(k): v for k, v in params.items()})
    m.step(1, dt_fixed=t)
    qm = m.read()[0]
    m.close()
    vol = o.geometry()[0]
    for v in (0, 1, 4):
        assert (np.abs(qm[:, v] - qo[:, v]) * vol).sum() / (np.abs(qo[:, v]) * vol).sum() < 1e-5


def test_six_million_tets_free_stream_and_conservation():
    """The largest density-wave mesh (100^3 x 6 = 6,000,000 jittered tets),
    in the bench's launch configuration (graph replay): properties that hold
    at any size, in both precisions.  A uniform state stays uniform to
    round-off over two steps, and the density wave conserves the totals of
    Q |cell| (periodic faces, fluxes gathered with opposite signs)."""
    xyz, cells, per = I.kuhn_cube(100, jitter=0.15, seed=0)
    mesh = H.Mesh(xyz, cells, per)
    vol = mesh.geometry()[0]
    uni = I.uniform_state(len(cells), 1.1, (0.4, -0.3, 0.2), 0.8)
    wave = I.density_wave_state(xyz, cells, 0.0)
    for prec, ftol, ctol in ((H.HGKS_FP64, 1e-13, 1e-13), (H.HGKS_FP32_MIXED, 1e-6, 1e-9)):
        s = H.Solver(mesh.clone(), uni, precision=prec)
        s.step(2)
        q, _, n = s.read()
        assert n == 2 and np.abs(q - uni).max() <= ftol * np.abs(uni).max(axis=0).max()
        s.write(wave, 0.0)
        tot0 = (wave * vol[:, None]).sum(axis=0)
        s.step(2)
        q, _, _ = s.read()
        s.close()
        tot = (q * vol[:, None]).sum(axis=0)
        assert np.abs(q - wave).max() > 1e-4
        assert np.all(np.abs(tot - tot0) <= ctol * np.abs(tot0).max()), (tot - tot0, prec)


@pytest.mark.parametrize("mesh", ["hex1", "hex2", "tet1", "tet2"])
def test_tiny_periodic_meshes_whose_stencils_hold_periodic_images(mesh):
    """Degenerate periodic meshes: one or two lattice cubes, so every stencil
    wraps around the box and holds periodic images of its own members (on
    one hexahedron, all 24 members are images of the cell itself).  Stage
    operator and two steps, inviscid and viscous, against the oracle."""
    n = int(mesh[-1])
    xyz, cells, per = (I.hex_cube if mesh.startswith("hex") else I.kuhn_cube)(n, jitter=0.0)
    q = I.random_smooth_state(xyz, cells, seed=n, amp=0.05)

    def close(a, b):
        # relative to the operator, or to the state where the operator
        # vanishes (one cell: the state is uniform and L is round-off)
        scale = np.maximum(np.abs(b).max(axis=0), np.abs(q).max(axis=0))
        return (np.abs(a - b).max(axis=0) / scale).max() < TOL

    for kw in (dict(), dict(mu_ref=2e-3, Pr=0.72, tau_c=1.0)):
        s, o = both(xyz, cells, per, q=q, **kw)
        L, dL = s.stage_operator(0.01)
        Lo, dLo = o.operator(0.01)
        assert close(L, Lo) and close(dL, dLo)
        s.step(2)
        o.step(2)
        qg, t, k = s.read()
        qo, to, ko = o.get_state()
        s.close()
        assert k == ko == 2 and abs(t - to) <= 1e-14 * to
        assert relerr(qg, qo) < TOL

"""Batched solvers (hgks_batch_init): many meshes advanced by one launch per
kernel.  Each member must give bitwise the result it gives as a single-mesh
solver (per-cell arithmetic is identical and each member keeps its own
CFL step), in FP64 and FP32-mixed."""
import numpy as np
import pytest

from paper_2407_00656_b300 import hgks as H
from paper_2407_00656_b300 import inputs as I

pytestmark = pytest.mark.gpu


def members():
    out = []
    for n, jit, seed in ((5, 0.15, 1), (6, 0.0, 2), (4, 0.15, 3)):
        xyz, cells, per = I.kuhn_cube(n, jitter=jit, seed=seed)
        q = I.random_smooth_state(xyz, cells, seed=seed, amp=0.05 * seed)
        out.append((xyz, cells, per, q))
    return out


@pytest.mark.parametrize("precision", [H.HGKS_FP64, H.HGKS_FP32_MIXED])
def test_batch_members_equal_single_solvers(precision):
    ms = members()
    kw = dict(precision=precision, mu_ref=1e-3, Pr=0.72)
    batch = H.Solver([H.Mesh(x, c, p) for x, c, p, _ in ms], [q for *_, q in ms], **kw)
    assert batch.members == 3
    batch.step(4)
    for i, (x, c, p, q) in enumerate(ms):
        single = H.Solver(H.Mesh(x, c, p), q, **kw)
        single.step(4)
        qs, ts, ns = single.read()
        qb, tb, nb = batch.member_read(i)
        assert ns == nb == 4 and ts == tb
        assert np.array_equal(qs, qb)


def test_batch_member_stops_at_its_t_end_and_restarts():
    ms = members()
    batch = H.Solver([H.Mesh(x, c, p) for x, c, p, _ in ms], [q for *_, q in ms])
    batch.step(100, t_end=0.01)
    times = [batch.member_read(i)[1] for i in range(3)]
    assert all(abs(t - 0.01) < 1e-15 for t in times)
    steps = [batch.member_read(i)[2] for i in range(3)]
    # each member took its own CFL steps
    x, c, p, q = ms[1]
    single = H.Solver(H.Mesh(x, c, p), q)
    single.step(100, t_end=0.01)
    assert single.read()[2] == steps[1]
    assert np.array_equal(single.read()[0], batch.member_read(1)[0])
    # restart one member, the others keep their state
    before = batch.member_read(2)[0]
    batch.member_write(0, ms[0][3], 0.0)
    batch.step(1, t_end=0.01)
    assert batch.member_read(0)[2] == 1
    assert np.array_equal(batch.member_read(2)[0], before)


def test_batch_reports_a_nonfinite_member():
    ms = members()
    batch = H.Solver([H.Mesh(x, c, p) for x, c, p, _ in ms], [q for *_, q in ms])
    bad = ms[1][3].copy()
    bad[3, 4] = np.inf
    batch.member_write(1, bad, 0.0)
    batch.step(1, dt_fixed=1e-4)
    batch.member_read(0)
    with pytest.raises(H.HGKSError) as e:
        batch.member_read(1)
    assert e.value.code == H.HGKS_ENONFINITE


def _same(a, b, precision):
    """The variants run the same operations in the same order, but the compiler
    may contract a multiply and an add into one fused operation in one kernel
    and not in the other: equal to a few units of the last place of the
    precision (FP64: 1e-14, FP32-mixed: 1e-6) of the magnitude of the
    quantity (density, momentum vector, energy)."""
    tol = 1e-14 if precision == H.HGKS_FP64 else 1e-6
    mag = np.abs(b).max(axis=0)
    mag[1:4] = mag[1:4].max()
    return np.all(np.abs(a - b) <= tol * mag)


@pytest.mark.parametrize("precision", [H.HGKS_FP64, H.HGKS_FP32_MIXED])
def test_every_kernel_variant_gives_the_same_result(precision):
    xyz, cells, bfn, bft = I.sphere_shell(5, 4, r_far=3.0, jitter=0.1, seed=4)
    qinf = I.free_stream(0.2535)
    q = np.tile(qinf, (len(cells), 1))
    q[:, 0] *= 1 + 0.02 * np.sin(np.arange(len(cells)))
    kw = dict(precision=precision, q_inf=qinf, mu_ref=0.2535 / 300, Pr=0.72, visc_exp=0.7, T_ref=1 / 1.4,
              tau_num_c=1.0)
    ref = None
    for fv in (0, 1):
        for rv in (0, 1):
            s = H.Solver(H.Mesh(xyz, cells, None, bfn, bft), q, **kw)
            s.set_tuning(fv, rv)
            assert s.tuning == (fv, rv)
            s.step(3)
            out = s.read()[0]
            if ref is None:
                ref = out
            assert _same(out, ref, precision), (fv, rv)
    tuned = H.Solver(H.Mesh(xyz, cells, None, bfn, bft), q, autotune=1, **kw)
    assert tuned.tuning[0] in (0, 1) and tuned.tuning[1] in (0, 1)
    tuned.step(3)
    assert _same(tuned.read()[0], ref, precision)

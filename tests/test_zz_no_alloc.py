"""The allocation-free CFL time step (hgks_cfl_dt_noalloc) against the time
step the solver itself takes (hgks_step, read back through hgks_read).

Callers that cannot allocate device memory when they need the step -- hosts
whose device memory belongs to another allocator, loops that cannot accept
cudaFree's device-wide synchronisation -- use this entry point; its scratch is
a fixed array inside the library, shared by all calls.  Two calls in a row
run on two meshes, the finer one first, so a second call that read the first
call's leftover partial minima would return too small a step and fail.  The
length scales come from the library's own hgks_mesh_geometry.
"""
import numpy as np
import pytest

from paper_2407_00656_b300 import hgks as H
from paper_2407_00656_b300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-11


def solver_dt(mesh, q, **kw):
    s = H.Solver(mesh, q, **kw)
    s.step(1)
    _, t, n = s.read()
    s.close()
    assert n == 1
    return t


def device(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("kw", [dict(), dict(mu_ref=0.05, Pr=0.72, visc_exp=0.7, T_ref=0.7)])
def test_noalloc_time_step_matches_solver_on_two_calls(kw):
    import torch

    cases = []
    for n, seed in ((10, 7), (6, 8)):  # 6000 then 1296 cells: ragged last blocks
        xyz, cells, per = I.kuhn_cube(n, jitter=0.15, seed=seed)
        q = I.random_smooth_state(xyz, cells, seed=seed, amp=0.1)
        hdt = H.Mesh(xyz, cells, per).geometry()[1]
        cases.append((xyz, cells, per, q, hdt))
    params = H.make_params(**kw)
    stream = torch.cuda.current_stream()
    dt_dev = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    keep = []
    for i, (xyz, cells, per, q, hdt) in enumerate(cases):
        q_dev, h_dev = device(q), device(hdt)
        keep += [q_dev, h_dev]
        torch.cuda.synchronize()
        H.cfl_dt_noalloc(q_dev.data_ptr(), h_dev.data_ptr(), len(cells), params, dt_dev.data_ptr() + 8 * i,
                         stream.cuda_stream)
    torch.cuda.synchronize()
    got = dt_dev.cpu().numpy()
    want = np.array([solver_dt(H.Mesh(*c[:3]), c[3], **kw) for c in cases])
    assert want[0] < want[1]
    assert np.all(np.abs(got - want) <= TOL * want), (got, want)


def test_noalloc_reports_a_state_without_a_bound_as_nan():
    import torch

    xyz, cells, per = I.kuhn_cube(6, jitter=0.15, seed=3)
    q = I.random_smooth_state(xyz, cells, seed=3)
    hdt = H.Mesh(xyz, cells, per).geometry()[1]
    params = H.make_params()
    dt = torch.zeros(3, dtype=torch.float64, device="cuda")
    bad = [q.copy(), q.copy()]
    bad[0][700, 0] = np.nan  # a non-finite density
    bad[1][1000, 4] = 0.5 * (bad[1][1000, 1:4] ** 2).sum() / bad[1][1000, 0] - 0.1  # p = -0.04 < 0
    keep = []
    for i, qq in enumerate([bad[0], bad[1], q]):
        a, b = device(qq), device(hdt)
        keep += [a, b]
        H.cfl_dt_noalloc(a.data_ptr(), b.data_ptr(), len(cells), params, dt.data_ptr() + 8 * i,
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = dt.cpu().numpy()
    assert np.isnan(got[0]) and np.isnan(got[1]) and np.isfinite(got[2]) and got[2] > 0


def test_noalloc_rejects_sizes_beyond_its_scratch_and_bad_params():
    params = H.make_params()
    with pytest.raises(H.HGKSError) as e:
        H.cfl_dt_noalloc(16, 16, 4194304 + 1, params, 16, 0)  # rejected before any device access
    assert e.value.code == H.HGKS_EINVAL and "scratch limit" in str(e.value)
    for bad in (dict(gamma=1.9), dict(mu_ref=-1.0), dict(mu_ref=1e-3, visc_exp=0.7, T_ref=0.0)):
        with pytest.raises(H.HGKSError) as e:
            H.cfl_dt_noalloc(16, 16, 100, H.make_params(**bad), 16, 0)  # rejected before any device access
        assert e.value.code == H.HGKS_EINVAL

"""The allocation-free CFL time step (hgks_cfl_dt_noalloc) against the time
step the solver itself takes (hgks_step, read back through hgks_read).

Callers that cannot allocate device memory when they need the step -- code
inside a stream capture, hosts whose memory belongs to another allocator,
loops that cannot afford an allocation's synchronisation -- use this entry
point; its scratch is a fixed array inside the library, shared by all calls.
Two calls in a row run on two meshes, the finer one first, so a second call
that read the first call's leftover partial minima would return too small a
step and fail.
"""
import numpy as np
import pytest

import oracle
from paper_2407_00656_b300 import hgks as H
from paper_2407_00656_b300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-11


def solver_dt(xyz, cells, per, q, **kw):
    s = H.Solver(H.Mesh(xyz, cells, per), q, **kw)
    s.step(1)
    _, t, n = s.read()
    s.close()
    assert n == 1
    return t


@pytest.mark.parametrize("kw", [dict(), dict(mu_ref=0.05, Pr=0.72, visc_exp=0.7, T_ref=0.7)])
def test_noalloc_time_step_matches_solver_on_two_calls(kw):
    import torch

    cases = []
    for n, seed in ((10, 7), (6, 8)):  # 6000 then 1296 cells: ragged last blocks
        xyz, cells, per = I.kuhn_cube(n, jitter=0.15, seed=seed)
        q = I.random_smooth_state(xyz, cells, seed=seed, amp=0.1)
        hdt = oracle.Oracle(xyz, cells, per).geometry()[3]
        cases.append((xyz, cells, per, q, hdt))
    params = H.make_params(**kw)
    stream = torch.cuda.current_stream()
    dt_dev = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    keep = []
    for i, (xyz, cells, per, q, hdt) in enumerate(cases):
        q_dev = torch.from_numpy(np.ascontiguousarray(q)).cuda()
        h_dev = torch.from_numpy(np.ascontiguousarray(hdt)).cuda()
        keep += [q_dev, h_dev]
        torch.cuda.synchronize()
        H.cfl_dt_noalloc(q_dev.data_ptr(), h_dev.data_ptr(), len(cells), params, dt_dev.data_ptr() + 8 * i,
                         stream.cuda_stream)
    torch.cuda.synchronize()
    got = dt_dev.cpu().numpy()
    want = np.array([solver_dt(*c[:4], **kw) for c in cases])
    assert want[0] < want[1]
    assert np.all(np.abs(got - want) <= TOL * want), (got, want)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    params = H.make_params()
    with pytest.raises(H.HGKSError) as e:
        H.cfl_dt_noalloc(16, 16, 4194304 + 1, params, 16, 0)  # rejected before any device access
    assert e.value.code == H.HGKS_EINVAL and "scratch limit" in str(e.value)

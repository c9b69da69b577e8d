"""Failure detection without a GPU fault: a bounded device wait that runs out
and a device allocation that fails, both caused on purpose by the library's
test hooks.

* The grid barriers of the persistent launch wait at most a set number of
  clock cycles.  With the limit at 0 every block but the last to arrive gives
  up at once, flags the solver and leaves; hgks_sync must then report
  HGKS_ETIMEOUT with the barrier named, and after hgks_write and the default
  limit the same solver must step correctly again (checked against the
  oracle).
* hgks_test_fail_alloc makes the n-th device allocation fail as an exhausted
  pool would.  Solver creation must return HGKS_ENOMEM, leave nothing
  allocated in the device's memory pool, and the next creation must work.
"""
import numpy as np
import pytest

import oracle
from paper_2407_00656_b300 import hgks as H
from paper_2407_00656_b300 import inputs as I

pytestmark = pytest.mark.gpu


def pool_used():
    import torch
    from cuda.bindings import runtime as rt

    torch.cuda.synchronize()
    err, pool = rt.cudaDeviceGetDefaultMemPool(torch.cuda.current_device())
    assert err == rt.cudaError_t.cudaSuccess
    err, used = rt.cudaMemPoolGetAttribute(pool, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent)
    assert err == rt.cudaError_t.cudaSuccess
    return int(used)


@pytest.mark.parametrize("precision", [H.HGKS_FP64, H.HGKS_FP32_MIXED])
def test_grid_barrier_timeout_is_reported_and_the_solver_recovers(precision):
    xyz, cells, per = I.kuhn_cube(6, jitter=0.15, seed=4)
    q = I.density_wave_state(xyz, cells, 0.0)
    s = H.Solver(H.Mesh(xyz, cells, per), q, precision=precision, persistent=1)
    s.test_barrier_limit(0)
    s.step(2)
    with pytest.raises(H.HGKSError) as e:
        s.sync()
    assert e.value.code == H.HGKS_ETIMEOUT and "grid barrier" in str(e.value)
    with pytest.raises(H.HGKSError) as e:
        s.read()
    assert e.value.code == H.HGKS_ETIMEOUT
    # the context is still usable: reset the state, restore the limit, step
    s.test_barrier_limit(-1)
    s.write(q, 0.0)
    s.step(2)
    qg, t, n = s.read()
    s.close()
    o = oracle.Oracle(xyz, cells, per)
    o.set_state(q)
    o.step(2)
    qo, to, no = o.get_state()
    assert n == no == 2
    tol = 1e-11 if precision == H.HGKS_FP64 else 1e-5
    assert abs(t - to) <= tol * to
    assert (np.abs(qg - qo).max(axis=0) / np.abs(qo).max(axis=0)).max() < tol


@pytest.mark.parametrize("which", [0, 1], ids=["mesh arrays", "solver arrays"])
def test_injected_allocation_failure_returns_enomem_without_a_leak(which):
    xyz, cells, per = I.kuhn_cube(5, jitter=0.15, seed=5)
    q = I.density_wave_state(xyz, cells, 0.0)
    H.Solver(H.Mesh(xyz, cells, per), q).close()  # the pool is set up and warm
    base = pool_used()
    H.test_fail_alloc(which)  # hgks_init allocates the mesh arrays, then the solver's
    try:
        with pytest.raises(H.HGKSError) as e:
            H.Solver(H.Mesh(xyz, cells, per), q)
    finally:
        H.test_fail_alloc(-1)
    assert e.value.code == H.HGKS_ENOMEM
    assert pool_used() == base
    s = H.Solver(H.Mesh(xyz, cells, per), q)
    s.step(1)
    _, t, n = s.read()
    assert n == 1 and t > 0
    s.close()
    assert pool_used() == base

"""Serving loop: admission by device memory, device meshes shared per
geometry, resident solves on separate streams, small requests batched into
one solver, chunked interleaving.  Every request's result is the same in the
mix as when solved alone: bitwise, since each solve runs the same kernels in
the same order whichever stream, batch or shared device mesh it is on
(FP32-mixed, the server's pinned flux variant)."""
import numpy as np
import pytest

from paper_2407_00656_b300 import hgks as H
from paper_2407_00656_b300 import serve as S

pytestmark = pytest.mark.gpu


def mix():
    reqs = []
    for i, (n, t) in enumerate([(5, 0.0), (6, 0.0), (4, 0.001), (7, 0.002), (5, 0.003)]):
        reqs.append(S.Request(i, t, "density", n, 20, S.density_params()))
    for j, (n, re, t) in enumerate([(4, 150.0, 0.0), (5, 250.0, 0.002), (4, 300.0, 0.004)]):
        reqs.append(S.Request(10 + j, t, "sphere", n, 20, S.sphere_params(re)))
    return reqs


def alone(cache, r, flux_variant=0):
    """The request solved by itself, with the flux variant the server pins."""
    mesh, q = cache.get(r.kind, r.size)
    s = H.Solver(mesh, q, precision=H.HGKS_FP32_MIXED, **r.params)
    s.set_tuning(flux_variant, 0)
    s.step(r.steps)
    out = s.read()
    s.close()
    return out


def test_results_in_the_mix_equal_results_alone():
    cache = S.MeshCache()
    reqs = mix()
    server = S.Server(mem_budget=8 << 30, chunk_steps=3, small_cells=1000, cache=cache)
    server.run(reqs, time_limit=300)
    assert any(r.cells >= 1000 for r in reqs) and any(r.cells < 1000 for r in reqs)
    for r in reqs:
        q, t, n = alone(cache, r, server.flux_variant)
        assert r.steps_done == n == 20
        assert r.t == t
        assert np.array_equal(r.result, q), r.rid
    st = S.summarize(reqs)
    assert st["p99_s"] >= st["p50_s"] > 0 and st["cell_updates_per_s"] > 0


def test_admission_waits_for_memory():
    cache = S.MeshCache()
    reqs = mix()
    cache.warm(reqs)
    # room for about two solves at a time
    sizes = sorted(cache.get(r.kind, r.size)[0].device_bytes(H.HGKS_FP32_MIXED) for r in reqs)
    budget = sizes[-1] + sizes[-2] + 4 * 65536
    server = S.Server(mem_budget=budget, chunk_steps=5, small_cells=1, cache=cache)
    server.run(reqs, time_limit=300)
    assert all(r.steps_done == 20 for r in reqs)
    assert server.peak_used <= budget
    # some request was admitted only after another had finished and freed memory
    assert any(b.admitted >= a.finished for a in reqs for b in reqs if a is not b)


def test_solver_creation_is_ordered_while_the_gpu_is_busy():
    """A solver created while another solve keeps the GPU busy starts from
    exactly its initial state (its uploads are ordered on its own stream)."""
    from paper_2407_00656_b300 import inputs as I

    xyz, cells, per = I.kuhn_cube(32, jitter=0.15, seed=0)
    big = H.Solver(H.Mesh(xyz, cells, per), I.density_wave_state(xyz, cells, 0.0))
    big.step(60)  # tens of ms of queued FP64 work on another stream
    for n in (4, 5, 6):
        x2, c2, p2 = I.kuhn_cube(n, jitter=0.15, seed=n)
        q = I.random_smooth_state(x2, c2, seed=n)
        small = H.Solver(H.Mesh(x2, c2, p2), q, precision=H.HGKS_FP32_MIXED)
        got, t, k = small.read()
        assert k == 0 and t == 0.0
        assert np.array_equal(got, q)
        small.close()
    big.sync()


def test_a_failed_allocation_is_retried_and_results_stay_the_same():
    """The library's allocation hook fails the third device allocation of the
    run (a solver creation meets an exhausted pool although the budget said
    it fits): the server gives the reservation back, queues the requests
    again, admits them once memory is freed, and every result still equals
    its result alone."""
    cache = S.MeshCache()
    reqs = mix()
    cache.warm(reqs)
    server = S.Server(mem_budget=8 << 30, chunk_steps=3, small_cells=1000, cache=cache)
    H.test_fail_alloc(2)
    try:
        server.run(reqs, time_limit=300)
    finally:
        H.test_fail_alloc(-1)
    assert server.alloc_retries == 1
    for r in reqs:
        q, t, n = alone(cache, r, server.flux_variant)
        assert r.steps_done == n == 20 and r.t == t
        assert np.array_equal(r.result, q), r.rid

"""Request stream of the serving configuration (host only)."""
import math

import numpy as np

from paper_2407_00656_b300 import serve as S


def test_c5_stream_shape():
    reqs = S.c5_requests(n=256, rate=4.0, seed=1)
    assert len(reqs) == 256
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) >= 0) and arr[0] == 0.0
    # Poisson arrivals: mean gap close to 1/rate
    assert abs(np.diff(arr).mean() - 0.25) < 0.05
    kinds = [r.kind for r in reqs]
    assert 0.35 < kinds.count("density") / 256 < 0.65
    cells = []
    for r in reqs:
        cells.append(6 * r.size ** 3 if r.kind == "density" else 6 * r.size ** 2 * S.sphere_layers(r.size))
    assert min(cells) >= 2000 and max(cells) <= 3e6
    res = [r.params["mu_ref"] and 0.2535 / r.params["mu_ref"] for r in reqs if r.kind == "sphere"]
    assert all(99.9 <= re <= 300.1 for re in res)
    assert all(r.steps == 200 for r in reqs)


# ---------------------------------------------------------------------------
# The scheduling logic of Server.run on the host, with the library replaced
# by fakes: a solver "finishes" a chunk after a few polls, device meshes and
# solvers report sizes from a formula.  This checks admission by memory,
# eviction of idle device meshes, batching rules and completion, without a GPU.
# ---------------------------------------------------------------------------
import types


class _FakeMesh:
    def __init__(self, cells):
        self.n_cells = cells
        self.static_bytes = 100 * cells
        self._work = 10 * cells

    def work_bytes(self, precision):
        return self._work

    def device_bytes(self, precision):
        return self.static_bytes + self._work

    def clone(self):
        return self


class _FakeCache:
    def __init__(self, cells_of):
        self.cells_of = cells_of
        self.meshes = {}

    def peek(self, kind, size):
        key = (kind, size)
        if key not in self.meshes:
            self.meshes[key] = (_FakeMesh(self.cells_of(kind, size)), np.zeros((1, 5)))
        return self.meshes[key]


class _FakeError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"fake failure {code}")
        self.code = code


def _fake_hgks(log, fail_at=()):
    made = [0]

    class DeviceMesh:
        live = 0

        def __init__(self, mesh):
            DeviceMesh.live += 1
            log.append(("dmesh", mesh.n_cells))
            self.n_cells = mesh.n_cells

        def release(self):
            DeviceMesh.live -= 1
            log.append(("release", self.n_cells))

    class Solver:
        def __init__(self, mesh, q, precision=None, **kw):
            made[0] += 1
            if made[0] in fail_at:  # this creation meets an exhausted pool
                log.append(("enomem", made[0]))
                raise _FakeError(-2)
            if isinstance(mesh, list):
                self.member_cells = [m.n_cells for m in mesh]
                log.append(("batch", tuple(self.member_cells)))
            else:
                self.member_cells = [mesh.n_cells]
            self.n_cells = self.member_cells[0]
            self.device_bytes = sum(110 * c for c in self.member_cells)
            self.steps = 0
            self.polls = 0

        def set_tuning(self, f, r):
            self.tuning = (f, r)

        def query(self):
            self.polls += 1
            return self.polls % 3 == 0

        def step(self, k):
            self.steps += k

        def member_read(self, i):
            return np.full((self.member_cells[i], 5), float(self.steps)), 0.1 * self.steps, self.steps

        def close(self):
            pass

    return types.SimpleNamespace(DeviceMesh=DeviceMesh, Solver=Solver, HGKS_FP32_MIXED=1, HGKS_FP64=0,
                                 HGKSError=_FakeError, HGKS_ENOMEM=-2)


def _requests():
    reqs = []
    for i, (kind, size) in enumerate([("density", 1), ("density", 2), ("sphere", 3), ("density", 1),
                                      ("sphere", 4), ("density", 2), ("sphere", 3), ("density", 5)]):
        reqs.append(S.Request(i, 0.0, kind, size, 30, {} if kind == "density" else {"mu_ref": 1e-3}))
    return reqs


def _cells(kind, size):
    return {("density", 1): 500, ("density", 2): 800, ("sphere", 3): 20000, ("sphere", 4): 30000,
            ("density", 5): 40000}[(kind, size)]


def test_server_logic_with_fake_solvers(monkeypatch):
    log = []
    monkeypatch.setattr(S, "H", _fake_hgks(log))
    cache = _FakeCache(_cells)
    # room for the small batch and for one large solve with its mesh at a time
    budget = 110 * 40000 + 110 * 1600 + 65536 * 4
    server = S.Server(mem_budget=budget, chunk_steps=7, small_cells=1000, max_batch=3, batch_cells=1500,
                      cache=cache)
    reqs = server.run(_requests(), time_limit=60)
    assert all(r.steps_done == 30 for r in reqs) and all(r.finished >= r.admitted >= 0 for r in reqs)
    assert server.peak_used <= budget
    # small requests were batched, by kind and parameters, within the caps
    batches = [e[1] for e in log if e[0] == "batch"]
    assert batches and all(len(b) <= 3 and sum(b) <= 1500 for b in batches)
    # large geometries got device meshes, and memory pressure evicted idle ones
    made = [e[1] for e in log if e[0] == "dmesh"]
    assert set(made) == {20000, 30000, 40000}
    first_release = min(i for i, e in enumerate(log) if e[0] == "release")
    last_dmesh = max(i for i, e in enumerate(log) if e[0] == "dmesh")
    assert first_release < last_dmesh
    # every device mesh is released when the run ends
    assert S.H.DeviceMesh.live == 0
    # the sphere 3 geometry is shared by its two requests unless evicted between them
    assert made.count(20000) <= 2
    assert all(getattr(r, "cells") in (500, 800, 20000, 30000, 40000) for r in reqs)


def test_server_survives_failed_allocations(monkeypatch):
    """A solver creation that fails with HGKS_ENOMEM although the budget said
    it fits (the second and the fifth creation here): the requests go back to
    the queue, admission waits for a running solve to finish, and every
    request is still served once, with nothing leaked from the budget."""
    log = []
    monkeypatch.setattr(S, "H", _fake_hgks(log, fail_at=(2, 5)))
    cache = _FakeCache(_cells)
    budget = 110 * 40000 + 110 * 1600 + 65536 * 4
    server = S.Server(mem_budget=budget, chunk_steps=7, small_cells=1000, max_batch=3, batch_cells=1500,
                      cache=cache)
    reqs = server.run(_requests(), time_limit=60)
    assert server.alloc_retries == 2 and sum(1 for e in log if e[0] == "enomem") == 2
    assert all(r.steps_done == 30 for r in reqs) and all(r.finished >= r.admitted >= 0 for r in reqs)
    assert server.peak_used <= budget
    assert S.H.DeviceMesh.live == 0


def test_server_gives_up_when_allocations_keep_failing(monkeypatch):
    """With nothing running to free memory, repeated failures end the run
    with a MemoryError instead of spinning."""
    import pytest

    monkeypatch.setattr(S, "H", _fake_hgks([], fail_at=tuple(range(1, 100))))
    server = S.Server(mem_budget=10 ** 12, chunk_steps=7, small_cells=1000, cache=_FakeCache(_cells))
    with pytest.raises(MemoryError):
        server.run(_requests()[:1], time_limit=60)

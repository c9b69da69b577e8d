"""Continuous-batching request loop for HGKS solves on one GPU.

Requests (a mesh, an initial state, physical parameters and a step count)
arrive over time.  The loop
  * admits waiting requests in arrival order while their device bytes fit the
    memory budget: a solver's own state and work arrays, plus the static
    mesh arrays when its geometry is not yet resident,
  * keeps one device mesh per geometry resident (hgks_dmesh_create) and
    creates every large request's solver over it (hgks_init_shared: only the
    state and work arrays are allocated, only the initial state is copied),
    evicting device meshes that no solve uses when memory is short,
  * packs small requests that share their parameters and step count and wait
    together into one batched solver (hgks_batch_init: one launch per kernel
    for all of them), up to a total cell count,
  * creates solvers on a worker thread, so that solver set-up (host work and
    copies) overlaps the steps of the solves already running,
  * keeps every admitted solve resident on the device, each solver on its own
    CUDA stream, and interleaves their steps in chunks: a chunk is queued
    whenever a solver's previous chunk has finished (hgks_query), so work of
    different solves overlaps on the device and newly admitted solves start
    while others are running,
  * reads a finished solve back, frees its memory and records its latency
    (completion time minus arrival time),
  * survives a device allocation that fails although the budget said it
    would fit (HGKS_ENOMEM at creation): the reservation is given back, the
    requests return to the queue in arrival order, and admission waits until
    a running solve has freed its memory (``alloc_retries`` counts these).

All numerics run in libhgks; this module only schedules.  Built host meshes
are cached by geometry (the warm-cache case of a service that sees the same
geometries repeatedly).
"""
from __future__ import annotations

import math
import threading
import time
from collections import OrderedDict
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import hgks as H
from . import inputs as I


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the start of the run
    kind: str                 # "density" or "sphere"
    size: int                 # lattice size N (density) or surface grid n (sphere)
    steps: int
    params: dict = field(default_factory=dict)
    # filled by the server
    admitted: float = math.nan
    finished: float = math.nan
    cells: int = 0
    result: np.ndarray | None = None
    t: float = math.nan
    steps_done: int = 0


def sphere_layers(n: int) -> int:
    return max(2, int(round(1.3 * n)))


def density_params():
    return {}


def sphere_params(re: float, mach: float = 0.2535):
    return dict(q_inf=tuple(I.free_stream(mach)), mu_ref=mach / re, Pr=0.72, visc_exp=0.7, T_ref=1 / 1.4,
                tau_num_c=1.0)


class MeshCache:
    """Built host meshes and initial states by geometry key."""

    def __init__(self):
        self._m = {}
        self._lock = threading.Lock()

    def get(self, kind: str, size: int):
        """A copy of the cached mesh (for a solver that consumes it) and the state."""
        mesh, q = self.peek(kind, size)
        return mesh.clone(), q

    def peek(self, kind: str, size: int):
        """The cached mesh itself (not a copy) and its initial state."""
        key = (kind, size)
        with self._lock:
            if key not in self._m:
                if kind == "density":
                    xyz, cells, per = I.kuhn_cube(size, jitter=0.15, seed=size)
                    mesh = H.Mesh(xyz, cells, per)
                    q = I.density_wave_state(xyz, cells, 0.0)
                else:
                    xyz, cells, bfn, bft = I.sphere_shell(size, sphere_layers(size), seed=size)
                    mesh = H.Mesh(xyz, cells, None, bfn, bft)
                    q = np.tile(I.free_stream(0.2535), (len(cells), 1))
                self._m[key] = (mesh, q)
            return self._m[key]

    def warm(self, requests):
        for r in requests:
            self.peek(r.kind, r.size)


@dataclass
class _Slot:
    solver: H.Solver
    reqs: list
    remaining: int
    bytes: int
    key: tuple | None  # geometry of a shared device mesh, None for a batch


class Server:
    def __init__(self, mem_budget: int, precision: int = H.HGKS_FP32_MIXED, chunk_steps: int = 10,
                 small_cells: int = 60_000, max_batch: int = 16, batch_cells: int = 300_000,
                 cache: MeshCache | None = None, flux_variant: int = 0):
        # every solver runs the same flux kernel variant (the library's
        # default depends on the mesh size, and a batch is larger than its
        # members): a request's result then does not depend on its company
        self.flux_variant = flux_variant
        self.mem_budget = int(mem_budget)
        self.precision = precision
        self.chunk = chunk_steps
        self.small = small_cells
        self.max_batch = max_batch
        self.batch_cells = batch_cells
        self.cache = cache or MeshCache()

    def _params_key(self, r: Request):
        return tuple(sorted((k, tuple(v) if isinstance(v, (list, tuple)) else v) for k, v in r.params.items()))

    def run(self, requests, time_limit: float = 3600.0):
        """Serve the requests (list of Request, arrival times relative to the
        start); returns them with admitted/finished/result filled in."""
        pending = sorted(requests, key=lambda r: r.arrival)
        queue, active, creating = [], [], []
        dev = OrderedDict()   # geometry -> DeviceMesh, least recently used first
        dev_bytes = {}        # geometry -> device bytes of its mesh (resident or being created)
        inuse = {}            # geometry -> admitted solves that use its device mesh
        dev_lock = threading.Lock()
        used = 0
        self.peak_used = 0
        self.peak_active = 0
        self.alloc_retries = 0
        hold = False      # admission paused after a failed allocation, until a solve finishes
        stalls = 0        # failed allocations in a row with nothing running
        worker = ThreadPoolExecutor(max_workers=1)
        t0 = time.perf_counter()

        def create_shared(key, mesh, q, params):
            with dev_lock:
                dm = dev.get(key)
            if dm is None:
                dm = H.DeviceMesh(mesh)
                with dev_lock:
                    dev[key] = dm
            s = H.Solver(dm, q, precision=self.precision, **params)
            s.set_tuning(self.flux_variant, 0)
            return s

        def create_batch(meshes, states, params):
            s = H.Solver([m.clone() for m in meshes], states, precision=self.precision, **params)
            s.set_tuning(self.flux_variant, 0)
            return s

        def evict(need):
            """Release idle device meshes (least recently used first) until
            `need` more bytes fit; returns the bytes freed."""
            freed = 0
            with dev_lock:
                for key in list(dev.keys()):
                    if used - freed + need <= self.mem_budget:
                        break
                    if inuse.get(key, 0) == 0:
                        dev.pop(key).release()
                        freed += dev_bytes.pop(key)
            return freed

        try:
            pi = 0
            while pi < len(pending) or queue or active or creating:
                now = time.perf_counter() - t0
                if now > time_limit:
                    raise TimeoutError("serving run exceeded its time limit")
                while pi < len(pending) and pending[pi].arrival <= now:
                    queue.append(pending[pi])
                    pi += 1
                busy = False
                # admission in arrival order while memory allows
                if hold and not active and not creating:
                    # nothing running will free memory: retry after a pause, a few times
                    if stalls >= 3:
                        raise MemoryError("device allocations keep failing with nothing running")
                    time.sleep(0.05)
                    hold = False
                while queue and not hold:
                    head = queue[0]
                    mesh, q = self.cache.peek(head.kind, head.size)
                    if mesh.n_cells < self.small:
                        group = [(head, mesh, q)]
                        key = (head.kind, self._params_key(head), head.steps)
                        total = mesh.n_cells
                        for r in queue[1:]:
                            if len(group) >= self.max_batch:
                                break
                            if (r.kind, self._params_key(r), r.steps) == key:
                                m2, q2 = self.cache.peek(r.kind, r.size)
                                if m2.n_cells < self.small and total + m2.n_cells <= self.batch_cells:
                                    group.append((r, m2, q2))
                                    total += m2.n_cells
                        need = sum(m.device_bytes(self.precision) for _, m, _ in group) + 65536 * len(group)
                        gkey = None
                    else:
                        group = [(head, mesh, q)]
                        gkey = (head.kind, head.size)
                        need = mesh.work_bytes(self.precision)
                        if gkey not in dev_bytes:
                            need += mesh.static_bytes
                    if used + need > self.mem_budget:
                        used -= evict(need)
                    if used + need > self.mem_budget:
                        if not active and not creating:
                            raise MemoryError(f"request {head.rid} needs {need} bytes, budget {self.mem_budget}")
                        break
                    tnow = time.perf_counter() - t0
                    for r, m, _ in group:
                        r.admitted = tnow
                        queue.remove(r)
                    if gkey is None:
                        fut = worker.submit(create_batch, [m for _, m, _ in group], [qq for _, _, qq in group],
                                            head.params)
                        used += need
                        creating.append((fut, [r for r, _, _ in group], need, 0, None))
                    else:
                        added = 0
                        if gkey not in dev_bytes:
                            dev_bytes[gkey] = mesh.static_bytes
                            added = mesh.static_bytes
                        inuse[gkey] = inuse.get(gkey, 0) + 1
                        work = mesh.work_bytes(self.precision)
                        used += need
                        fut = worker.submit(create_shared, gkey, mesh, q, head.params)
                        creating.append((fut, [head], work, added, gkey))
                    self.peak_used = max(self.peak_used, used)
                    busy = True
                # solvers that finished their set-up start stepping
                for item in list(creating):
                    fut, reqs, nb, added, gkey = item
                    if not fut.done():
                        continue
                    creating.remove(item)
                    try:
                        solver = fut.result()  # any other creation error ends the run
                    except H.HGKSError as e:
                        if e.code != H.HGKS_ENOMEM:
                            raise
                        # the pool had less room than the budget assumed: give the
                        # reservation back and queue the requests again
                        used -= nb
                        if gkey is not None:
                            inuse[gkey] -= 1
                            with dev_lock:
                                made = gkey in dev
                            if added and not made:  # the device mesh itself was not made
                                used -= dev_bytes.pop(gkey)
                        for r in reqs:
                            r.admitted = math.nan
                        queue = sorted(queue + list(reqs), key=lambda r: (r.arrival, r.rid))
                        self.alloc_retries += 1
                        stalls = stalls + 1 if not active and not creating else 0
                        hold = True
                        busy = True
                        continue
                    if gkey is None:
                        real = solver.device_bytes
                        used += real - nb
                        nb = real
                        for i, r in enumerate(reqs):
                            r.cells = solver.member_cells[i]
                    else:
                        reqs[0].cells = solver.n_cells
                        with dev_lock:
                            if gkey in dev:
                                dev.move_to_end(gkey)
                    active.append(_Slot(solver, reqs, reqs[0].steps, nb, gkey))
                    self.peak_used = max(self.peak_used, used)
                    self.peak_active = max(self.peak_active, len(active) + len(creating))
                    busy = True
                # queue the next chunk of every idle solve
                for sl in active:
                    if sl.remaining > 0 and sl.solver.query():
                        k = min(self.chunk, sl.remaining)
                        sl.solver.step(k)
                        sl.remaining -= k
                        busy = True
                # collect finished solves
                for sl in list(active):
                    if sl.remaining == 0 and sl.solver.query():
                        tnow = time.perf_counter() - t0
                        for i, r in enumerate(sl.reqs):
                            r.result, r.t, r.steps_done = sl.solver.member_read(i)
                            r.finished = tnow
                        sl.solver.close()
                        used -= sl.bytes
                        hold = False
                        stalls = 0
                        if sl.key is not None:
                            inuse[sl.key] -= 1
                        active.remove(sl)
                        busy = True
                if not busy:
                    time.sleep(0.0002)
        finally:
            worker.shutdown(wait=True)
            with dev_lock:
                for dm in dev.values():
                    dm.release()
                dev.clear()
        return requests


def c5_requests(n: int = 256, lo: float = 5e3, hi: float = 2e6, steps: int = 200, rate: float = 1.0,
                seed: int = 0, classes: int = 8):
    """The serving stream: Poisson arrivals (rate per second), sizes
    log-uniform in [lo, hi] cells rounded to `classes` log-spaced geometry
    classes per kind, half density-wave cubes (inviscid) and half sphere
    shells at Re ~ U[100, 300]."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    arrivals -= arrivals[0]
    grid = np.exp(np.linspace(math.log(lo), math.log(hi), classes))
    reqs = []
    for i in range(n):
        cells = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        target = grid[np.argmin(np.abs(np.log(grid) - math.log(cells)))]
        if rng.uniform() < 0.5:
            size = max(4, int(round((target / 6) ** (1 / 3))))
            reqs.append(Request(i, float(arrivals[i]), "density", size, steps, density_params()))
        else:
            size = max(3, int(round((target / (6 * 1.3)) ** (1 / 3))))
            re = float(rng.uniform(100, 300))
            reqs.append(Request(i, float(arrivals[i]), "sphere", size, steps, sphere_params(re)))
    return reqs


def summarize(reqs):
    lat = np.array([r.finished - r.arrival for r in reqs])
    work = sum(r.cells * r.steps_done for r in reqs)
    span = max(r.finished for r in reqs) - min(r.arrival for r in reqs)
    return {"requests": len(reqs), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "makespan_s": float(span), "cell_updates_per_s": work / span}

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

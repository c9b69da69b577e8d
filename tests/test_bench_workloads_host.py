"""bench.py's workload names on the CPU: each builds the mesh family and the
parameters it states (density wave on tetrahedra or prisms, sphere shells at
Ma 0.2535 and 1.5, the hybrid hex/prism shell), with seeded, repeatable
inputs."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2407_00656_b300 import inputs as I  # noqa: E402


def is_prism(cells):
    return (cells[:, 2] == cells[:, 3]) & (cells[:, 6] == cells[:, 7])


def test_density_workloads():
    w = bench.workload("density8")
    assert w["cells"].shape == (6 * 8 ** 3, 4) and w["params"] == {}
    v = bench.workload("density6v")
    assert v["params"]["mu_ref"] == 1e-3 and v["params"]["Pr"] == 0.72
    # the exact cell averages of the density wave
    assert np.allclose(w["q"], I.density_wave_state(w["xyz"], w["cells"], 0.0))


@pytest.mark.parametrize("name,mach", [("sphere6", 0.2535), ("transonic6", 1.5)])
def test_sphere_workloads(name, mach):
    w = bench.workload(name)
    assert w["cells"].shape[1] == 8 and not is_prism(w["cells"]).any()
    p = w["params"]
    assert p["q_inf"][1] == pytest.approx(mach) and p["mu_ref"] == pytest.approx(mach / 300)
    assert p["visc_exp"] == 0.7 and p["tau_num_c"] == 1.0
    assert np.all(w["q"] == p["q_inf"])


def test_hybrid_and_prism_workloads():
    h = bench.workload("hybrid8")
    frac = is_prism(h["cells"]).mean()
    assert 0.2 < frac < 0.7  # 30% of the columns cut, two prisms each
    h2 = bench.workload("hybrid8")
    assert np.array_equal(h["cells"], h2["cells"]) and np.array_equal(h["xyz"], h2["xyz"])
    p = bench.workload("prism5")
    assert p["cells"].shape == (2 * 5 ** 3, 8) and is_prism(p["cells"]).all()
    with pytest.raises(ValueError):
        bench.workload("nonsense")

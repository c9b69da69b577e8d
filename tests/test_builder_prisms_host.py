"""Host-side checks of the library's mesh builder on prisms (hexahedra with
nodes 2 = 3 and 6 = 7) and hybrid hex/prism shells, on the CPU: its faces,
volumes and time-step lengths agree with the oracle's own construction, its
stencil sizes are rounded up to the compiled ones, and a hexahedron with any
other repeated node is refused."""
import numpy as np
import pytest

import oracle
from paper_2407_00656_b300 import build as B
from paper_2407_00656_b300 import hgks as H
from paper_2407_00656_b300 import inputs as I


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def meshes():
    xyz, cells, per = I.prism_cube(5, jitter=0.15, seed=2)
    yield "prism cube", (xyz, cells, per, None, None)
    for frac in (0.4, 1.0):
        xyz, cells, bfn, bft = I.sphere_shell(6, 5, r_far=3.0, jitter=0.1, seed=1, prism_frac=frac)
        yield f"shell {frac}", (xyz, cells, None, bfn, bft)


@pytest.mark.parametrize("name,args", list(meshes()))
def test_builder_matches_the_oracle_on_prism_meshes(name, args):
    m = H.Mesh(*args)
    o = oracle.Oracle(*args)
    assert m.n_cells == len(args[1]) and m.n_faces == o.n_faces
    vol, hdt = m.geometry()
    ovol, _, _, ohdt = o.geometry()
    assert np.allclose(vol, ovol, rtol=1e-13, atol=0)
    assert np.allclose(hdt, ohdt, rtol=1e-13, atol=0)
    # one ghost slot per tagged boundary face, triangles included
    if args[3] is not None:
        assert m.n_ghosts == len(args[3])


def test_stencil_sizes_are_padded_to_compiled_shapes():
    xyz, cells, per = I.prism_cube(5)
    assert H.Mesh(xyz, cells, per).stencil_size == 20  # 19 members, padded
    xyz, cells, bfn, bft = I.sphere_shell(6, 5, r_far=3.0, seed=1, prism_frac=0.4)
    assert H.Mesh(xyz, cells, None, bfn, bft).stencil_size == 26
    xyz, cells, bfn, bft = I.sphere_shell(6, 5, r_far=3.0, seed=1)
    assert H.Mesh(xyz, cells, None, bfn, bft).stencil_size == 24  # hexahedra unchanged


@pytest.mark.parametrize("pair", [(1, 2), (0, 4), (6, 7)])
def test_other_collapsed_hexahedra_are_refused(pair):
    xyz, cells, bfn, bft = I.sphere_shell(4, 3, r_far=3.0, seed=1)
    bad = cells.copy()
    a, b = pair
    bad[5, b] = bad[5, a]  # (6, 7) alone: nodes 2 and 3 stay distinct
    with pytest.raises(H.HGKSError) as e:
        H.Mesh(xyz, bad, None, bfn, bft)
    assert e.value.code == H.HGKS_EINVAL
    assert "prism" in str(e.value)

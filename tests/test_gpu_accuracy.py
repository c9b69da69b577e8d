"""Accuracy configurations on the GPU path (Section 5.1): the 8^3 x 6 test
run to t = 0.2 against the exact solution and the oracle, and the precision
sweep over 12^3, 24^3, 48^3 x 6 jittered tets in FP64 and FP32-mixed:
both converge at about third order, and the mixed solution differs from the
FP64 one by at most 1e-5 in relative L1 (rho, rhoU, rhoE)."""
import numpy as np
import pytest

import oracle
from paper_2407_00656_b300 import hgks as H
from paper_2407_00656_b300 import inputs as I

pytestmark = pytest.mark.gpu


def l1(err, vol):
    return float((np.abs(err) * vol).sum() / vol.sum())


def test_c1_to_t02_matches_oracle_and_exact_solution():
    oracle.set_threads(8)
    xyz, cells, per = I.kuhn_cube(8)
    q0 = I.density_wave_state(xyz, cells, 0.0)
    s = H.Solver(H.Mesh(xyz, cells, per), q0)
    s.step(1000, t_end=0.2)
    qg, tg, ng = s.read()
    o = oracle.Oracle(xyz, cells, per)
    o.set_state(q0)
    while o.get_state()[1] < 0.2:
        o.step(1, t_end=0.2)
    qo, to, no = o.get_state()
    assert ng == no and abs(tg - 0.2) < 1e-15 and abs(tg - to) < 1e-15
    scale = np.abs(qo).max(axis=0)
    assert (np.abs(qg - qo).max(axis=0) / scale).max() < 1e-10
    vol = o.geometry()[0]
    e = l1(qg[:, 0] - I.density_wave_state(xyz, cells, tg)[:, 0], vol)
    assert 1e-4 < e < 2e-2  # the coarse mesh's third-order error, far below the 0.2 amplitude


def run(n, precision, t_end=0.05):
    xyz, cells, per = I.kuhn_cube(n, jitter=0.15, seed=0)
    m = H.Mesh(xyz, cells, per)
    vol = m.geometry()[0]
    s = H.Solver(m, I.density_wave_state(xyz, cells, 0.0), precision=precision)
    s.step(100000, t_end=t_end)
    q, t, k = s.read()
    exact = I.density_wave_state(xyz, cells, t)
    return q, exact, vol


def test_precision_sweep_order_and_mixed_error():
    errs = {H.HGKS_FP64: [], H.HGKS_FP32_MIXED: []}
    for n in (12, 24, 48):
        out = {}
        for prec in errs:
            q, exact, vol = run(n, prec)
            out[prec] = q
            errs[prec].append(l1(q[:, 0] - exact[:, 0], vol))
        a, b = out[H.HGKS_FP32_MIXED], out[H.HGKS_FP64]
        for v in (0, 1, 4):
            rel = (np.abs(a[:, v] - b[:, v]) * vol).sum() / (np.abs(b[:, v]) * vol).sum()
            assert rel <= 1e-5, (n, v, rel)
    for prec, e in errs.items():
        orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
        assert np.all(orders > 2.5), (prec, e, orders)

"""The binary64 erfcx of the flux kernels on the device (hgks_test_erfcx)
against erfcx = exp(x^2) erfc(x) from mpmath at 40 digits: the table part
(0 <= x < 6) within two units in the last place, the library part beyond
within 1e-15 relative, and the special values."""
import math

import mpmath as mp
import numpy as np
import pytest

from paper_2407_00656_b300 import hgks as H

pytestmark = pytest.mark.gpu


def _ref(x: float) -> float:
    with mp.workdps(40):
        return float(mp.exp(mp.mpf(x) ** 2) * mp.erfc(mp.mpf(x)))


def test_device_erfcx_against_mpmath():
    rng = np.random.default_rng(11)
    table = list(rng.uniform(0.0, 6.0, 3000))
    for i in range(24):
        e = i / 4.0
        table += [e, float(np.nextafter(e, 7.0)), float(np.nextafter((i + 1) / 4.0, 0.0))]
    beyond = list(rng.uniform(6.0, 40.0, 300)) + [6.0, 1e3, 1e8]
    xs = np.array(table + beyond)
    got = H.test_erfcx(xs)
    ref = np.array([_ref(float(x)) for x in xs])
    rel = np.abs(got - ref) / ref
    nt = len(table)
    assert rel[:nt].max() <= 2 * 2.0 ** -52, rel[:nt].max()
    assert rel[nt:].max() <= 1e-15, rel[nt:].max()
    special = H.test_erfcx(np.array([0.0, -0.0, math.inf, math.nan]))
    assert abs(special[0] - 1.0) <= 2 * 2.0 ** -52 and special[1] == special[0]
    assert special[2] == 0.0
    assert math.isnan(special[3])


def test_device_erfcx_rejects_bad_arguments():
    assert H.lib().hgks_test_erfcx(None, None, -1) == H.HGKS_EINVAL
    assert H.lib().hgks_test_erfcx(None, None, 3) == H.HGKS_EINVAL
    assert H.test_erfcx(np.array([])).size == 0

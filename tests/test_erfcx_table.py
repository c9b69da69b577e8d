"""The binary64 erfcx of the flux kernels (a piecewise polynomial table on
[0, 6), the library function beyond): the committed table is what its
generator writes, and Horner's rule with fused multiply-adds on it, as the
device evaluates it, stays within two units in the last place of erfcx
computed by mpmath at 40 digits."""
import importlib.util
import os
import re
from fractions import Fraction

import mpmath as mp
import numpy as np

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2407_00656_b300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_erfcx_table", os.path.join(CSRC, "gen_erfcx_table.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _header_table():
    text = open(os.path.join(CSRC, "erfcx_table.h")).read()
    body = text[text.index("kErfcxTab"):]
    body = body[body.index("{") + 1:body.index("};")]
    return [float(v) for v in re.findall(r"[-+0-9.eE]+", body)]


def _fma(a: float, b: float, c: float) -> float:
    """a * b + c rounded once to binary64 (exact rational arithmetic)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _device_erfcx(x: float, tab, n: int) -> float:
    i = int(x * 4.0)  # truncation, as the device's conversion
    u = _fma(x, 8.0, -(2.0 * i + 1.0))
    c = tab[i * (n + 1):(i + 1) * (n + 1)]
    p = c[n]
    for k in range(n - 1, -1, -1):
        p = _fma(p, u, c[k])
    return p


def test_committed_table_is_the_generated_one():
    gen = _gen()
    rows = gen.table()
    flat = [v for row in rows for v in row]
    assert _header_table() == flat
    assert len(flat) == gen.INTERVALS * (gen.DEGREE + 1)


def test_table_evaluation_within_two_ulp_of_erfcx():
    gen = _gen()
    tab = _header_table()
    n = gen.DEGREE
    rng = np.random.default_rng(5)
    xs = list(rng.uniform(0.0, 6.0, 1500))
    # interval ends, both sides, and zero
    for i in range(gen.INTERVALS):
        e = i / 4.0
        xs += [e, np.nextafter(e, 7.0), np.nextafter((i + 1) / 4.0, 0.0)]
    worst = 0.0
    with mp.workdps(40):
        for x in xs:
            x = float(x)
            if not 0.0 <= x < 6.0:
                continue
            ref = mp.exp(mp.mpf(x) ** 2) * mp.erfc(mp.mpf(x))
            got = _device_erfcx(x, tab, n)
            worst = max(worst, abs(float((mp.mpf(got) - ref) / ref)))
    assert worst <= 2 * 2.0 ** -52, worst

"""Writes erfcx_table.h: the coefficient table of the binary64 scaled
complementary error function erfcx(x) = exp(x^2) erfc(x) used by the flux
kernels on 0 <= x < X_MAX.

Method: [0, X_MAX) is cut into intervals of width WIDTH; on each, erfcx is
interpolated at the DEGREE + 1 Chebyshev points of the first kind
(near-minimax polynomial interpolation, e.g. Trefethen, "Approximation Theory
and Approximation Practice", ch. 8) in the local variable u in [-1, 1], and
the interpolant's monomial coefficients in u are rounded to binary64.  The
reference values come from mpmath at 40 significant digits.  The device
evaluates the polynomial by Horner's rule with fused multiply-adds.

    python paper_2407_00656_b300/csrc/gen_erfcx_table.py        # rewrite the header
"""
import os

import mpmath as mp

WIDTH = mp.mpf(1) / 4
INTERVALS = 24  # X_MAX = 6
DEGREE = 12
DPS = 40


def erfcx_mp(x):
    return mp.exp(x * x) * mp.erfc(x)


def interval_coefficients(i: int):
    """Monomial coefficients (low to high) in u = (x - c) / r of the Chebyshev
    interpolant of erfcx on interval i, c its centre and r its half width."""
    with mp.workdps(DPS):
        a = WIDTH * i
        r = WIDTH / 2
        c = a + r
        n = DEGREE
        nodes = [mp.cos(mp.pi * (k + mp.mpf(1) / 2) / (n + 1)) for k in range(n + 1)]
        A = mp.matrix([[t ** j for j in range(n + 1)] for t in nodes])
        y = mp.matrix([erfcx_mp(c + r * t) for t in nodes])
        coef = mp.lu_solve(A, y)
        return [float(coef[j]) for j in range(n + 1)]


def table():
    return [interval_coefficients(i) for i in range(INTERVALS)]


def header_text() -> str:
    rows = table()
    lines = [
        "// erfcx_table.h -- generated by gen_erfcx_table.py (do not edit): monomial",
        "// coefficients, low to high, in u = 8 x - (2 i + 1) in [-1, 1) of the Chebyshev",
        "// interpolant of erfcx(x) = exp(x^2) erfc(x) on [i / 4, (i + 1) / 4), i = 0 .. 23.",
        "#pragma once",
        "",
        "namespace hgks {",
        "namespace {",
        f"constexpr int kErfcxIntervals = {INTERVALS}, kErfcxDegree = {DEGREE};",
        f"__device__ const double kErfcxTab[{INTERVALS} * {DEGREE + 1}] = {{",
    ]
    for i, row in enumerate(rows):
        lines.append("    " + ", ".join("%.17g" % v for v in row) + ("," if i + 1 < len(rows) else ""))
    lines += ["};", "}  // namespace", "}  // namespace hgks", ""]
    return "\n".join(lines)


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "erfcx_table.h")
    with open(path, "w") as fh:
        fh.write(header_text())
    print("wrote", path)

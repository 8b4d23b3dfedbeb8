"""The premise of the FP32 lattice's treatment of cells holding samples
(a cell whose intervals' polynomials agree within 1e-8 |f| keeps one record),
checked on the oracle's own Green table: at every forced zero (Section II.B)
of a default table, the Eq. (5) cubic of the interval on one side, carried
across a lattice cell (t / 2) past the zero, stays within 1e-8 |f| of the
neighbouring interval's cubic. Pure numpy on the oracle's samples."""
import math

import numpy as np

import oracle as O


def interval_cubic(r, f, i, x):
    """Eq. (5), degree 3, of interval i (stencil i - 1 .. i + 2, clamped to the table)."""
    s0 = min(max(i - 1, 0), len(r) - 4)
    xs, fs = r[s0:s0 + 4], f[s0:s0 + 4]
    out = np.zeros_like(x, dtype=complex)
    for a in range(4):
        w = np.ones_like(x)
        for b in range(4):
            if b != a:
                w = w * (x - xs[b]) / (xs[a] - xs[b])
        out += fs[a] * w
    return out


def test_polynomials_meeting_at_forced_zeros_agree():
    k = 2 * math.pi
    T = O.Table(O.table_params(O.GREEN, k, 0.0537, 2.5))  # r_min off the zeros: forced samples inside intervals
    r, f, _ = T.nodes()
    zeros = [j for j in range(1, len(r) - 1) if f[j].real == 0.0 or f[j].imag == 0.0]
    assert len(zeros) >= 8  # one every quarter wavelength from 0.25 to 2.5
    t = (2 * math.pi / k) / 1000
    worst = 0.0
    for j in zeros:
        right = np.linspace(r[j], r[j] + 0.5 * t, 33)  # past the zero: interval j-1 carried over
        left = np.linspace(r[j] - 0.5 * t, r[j], 33)   # before it: interval j carried back
        d1 = np.abs(interval_cubic(r, f, j - 1, right) - interval_cubic(r, f, j, right)) * right
        d2 = np.abs(interval_cubic(r, f, j, left) - interval_cubic(r, f, j - 1, left)) * left
        worst = max(worst, d1.max(), d2.max())
    assert worst < 1e-8, worst  # measured 5.7e-11
    assert worst > 0.0  # the two cubics are distinct polynomials (the zeros split uniform intervals)

"""Pins of the oracle's singular / near inner integrals (singularity
cancellation with the angular transformation, Section II.A) against the static
closed forms of the potential integrals plus a Duffy-rule brute force of the
bounded dynamic remainder (tests/brute.py)."""
import math

import numpy as np
import pytest

import brute as B
import oracle as O

TRI = np.array([[0, 0, 0], [0.07, 0, 0], [0.02, 0.06, 0]], float)
POINTS = [
    [0.03, 0.02, 0.0],      # inside, in plane (self term)
    [0.03, 0.02, 0.01],     # above the interior
    [0.15, 0.08, 0.02],     # well separated
    [0.07, -0.01, 0.0],     # in plane, outside, near a vertex
    [0.035, -0.01, 0.0],    # in plane, outside, near an edge (adjacent triangle)
    [0.035, -0.004, 0.003], # close to an edge, off plane
]


@pytest.mark.parametrize("r", POINTS)
def test_static_closed_form_matches_duffy(r):
    # the test's own reference: closed form vs direct Duffy integration of 1/R
    r = np.array(r)
    s0, s1, rho0 = B.static_potentials(r, TRI)
    P, W = B.split_rule(rho0, TRI, 60)
    R = np.linalg.norm(P - r, axis=1)
    assert abs(s0 - np.sum(W / R)) < 1e-9 * abs(s0)
    np.testing.assert_allclose(s1, np.sum((W / R)[:, None] * (P - rho0), axis=0), atol=1e-9 * np.abs(s1).max())


@pytest.mark.parametrize("r", POINTS)
@pytest.mark.parametrize("k", [2 * math.pi, 4 * math.pi, 1e-3])
def test_singular_converges_to_reference(r, k):
    r = np.array(r)
    I0r, I1r, rho_r = B.inner_integrals(r, TRI, k, 48)
    I0, I1, rho = O.singular(r, TRI[0], TRI[1], TRI[2], k, 40, 40)
    np.testing.assert_allclose(rho, rho_r, atol=1e-15)
    assert abs(I0 - I0r) <= 1e-11 * abs(I0r)
    # relative to the size of the RWG-weighted inner integral I1 + (rho0 - v) I0
    assert np.linalg.norm(I1 - I1r) <= 1e-8 * (np.linalg.norm(I1r) + 0.07 * abs(I0r))


@pytest.mark.parametrize("r", POINTS)
def test_default_order_accuracy(r):
    # default n_phi = n_l = 8: the scalar part within 1e-4, and the vector
    # part within 1e-5 of the RWG-weighted inner integral it enters
    r = np.array(r)
    k = 2 * math.pi
    I0r, I1r, rho_r = B.inner_integrals(r, TRI, k, 48)
    I0, I1, _ = O.singular(r, TRI[0], TRI[1], TRI[2], k, 8, 8)
    assert abs(I0 - I0r) <= 1e-4 * abs(I0r)
    scale = np.linalg.norm(I1r + (rho_r - TRI[0]) * I0r)
    assert np.linalg.norm(I1 - I1r) <= 1e-5 * scale


def test_singular_exp_table_path():
    # with the Exp table the line integrals use interpolated e^{-jkR}; the
    # result stays within the table tolerance amplified by 1/(k h)
    k = 2 * math.pi
    e = O.Table(O.table_params(O.EXP, k, 0.01, 1.0))
    for r in POINTS:
        r = np.array(r)
        a0, a1, _ = O.singular(r, TRI[0], TRI[1], TRI[2], k, 8, 8)
        b0, b1, _ = O.singular(r, TRI[0], TRI[1], TRI[2], k, 8, 8, texp=e)
        assert abs(a0 - b0) <= 1e-6 / (k * 0.02) * abs(a0)

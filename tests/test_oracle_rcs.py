"""Pins of the scattering oracle (oracle/rcs.py): the Mie series of a PEC
sphere against identities it must satisfy, the RWG plane-wave excitation and
far field against closed forms, a brute-force quadrature and reciprocity, and
the whole EFIE chain (oracle Z, solve, far field) against Mie."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import rcs

K = 2 * math.pi


@pytest.mark.parametrize("x", [0.5, math.pi, 2 * math.pi, 10.0])
def test_mie_angular_integral_equals_scattering_cross_section(x):
    # (pi / k^2) int (|S1|^2 + |S2|^2) sin(theta) dtheta = sigma_sca (from a_n, b_n):
    # ties pi_n, tau_n and the S1 / S2 sums to the coefficients
    a = x / K
    u, w = np.polynomial.legendre.leggauss(400)
    th = (u + 1) * math.pi / 2
    S1, S2 = rcs.mie_amplitudes(x, th)
    integral = math.pi / K ** 2 * np.sum(w * math.pi / 2 * (np.abs(S1) ** 2 + np.abs(S2) ** 2) * np.sin(th))
    ext, sca = rcs.mie_cross_sections(K, a)
    assert abs(integral / sca - 1) < 1e-11
    assert abs(ext / sca - 1) < 1e-12  # lossless sphere: extinction = scattering (optical theorem)


@pytest.mark.parametrize("x", [0.5, 2 * math.pi, 10.0])
def test_mie_backscatter_two_forms(x):
    a = x / K
    sE, sH = rcs.mie_bistatic(K, a, np.array([math.pi]))
    sb = rcs.mie_backscatter(K, a)
    assert abs(sE[0] / sb - 1) < 1e-12 and abs(sH[0] / sb - 1) < 1e-12


def test_mie_rayleigh_limit():
    # small PEC sphere: sigma_back = 9 pi a^2 (ka)^4, sigma_sca = (10/3) pi a^2 (ka)^4
    x = 1e-3
    a = x / K
    assert abs(rcs.mie_backscatter(K, a) / (9 * math.pi * a * a * x ** 4) - 1) < 1e-5
    assert abs(rcs.mie_cross_sections(K, a)[1] / (10 / 3 * math.pi * a * a * x ** 4) - 1) < 1e-5


def _mesh():
    xyz, tri = W.icosphere(1)
    return W.jitter(xyz * 0.3, tri, 0.05, 3), tri


def test_rhs_at_k0_is_the_closed_form():
    # k = 0: V_m = p . int f_m dS = p . (l/2) [(c+ - v+) - (c- - v-)] (centroids c, free vertices v)
    xyz, tri = _mesh()
    om = O.Mesh(xyz, tri)
    ev, et = om.edges()
    opp, length = rcs.rwg_sides(xyz, tri, ev, et)
    cen = xyz[tri].mean(axis=1)
    p = np.array([0.3, -0.5, 0.8])
    ref = 0.5 * length * (((cen[et[:, 0]] - xyz[opp[:, 0]]) - (cen[et[:, 1]] - xyz[opp[:, 1]])) @ p)
    for npts in (3, 7):
        V = rcs.planewave_rhs(xyz, tri, ev, et, 0.0, [0, 0, 1], p, npts)
        np.testing.assert_allclose(V, ref, rtol=1e-13, atol=1e-15)


def _dense_side_integral(xyz, tri, ev, et, k, khat, pol, level=4):
    """int f_m . p e^{-jk khat.r} dS by the 7-point rule on 4^level sub-triangles."""
    opp, length = rcs.rwg_sides(xyz, tri, ev, et)
    bary, w = O.rule(7)
    # sub-triangles of the reference triangle (barycentric corners)
    subs = [np.eye(3)]
    for _ in range(level):
        nxt = []
        for c in subs:
            m01, m12, m20 = (c[0] + c[1]) / 2, (c[1] + c[2]) / 2, (c[2] + c[0]) / 2
            nxt += [np.array([c[0], m01, m20]), np.array([m01, c[1], m12]), np.array([m20, m12, c[2]]),
                    np.array([m01, m12, m20])]
        subs = nxt
    pts_bary = np.concatenate([bary @ s for s in subs])  # (4^level * 7, 3)
    wts = np.concatenate([w / len(subs)] * len(subs))
    V = np.zeros(len(ev), dtype=np.complex128)
    for s, sign in ((0, 1.0), (1, -1.0)):
        v = xyz[tri[et[:, s]]]                           # (ne, 3, 3)
        r = np.einsum("ac,ncx->nax", pts_bary, v)
        rel = r - xyz[opp[:, s]][:, None, :]
        V += sign * 0.5 * length * np.einsum("a,na,na->n", wts, rel @ pol, np.exp(-1j * k * (r @ khat)))
    return V


def test_rhs_matches_dense_quadrature():
    xyz, tri = _mesh()
    om = O.Mesh(xyz, tri)
    ev, et = om.edges()
    khat = np.array([0.48, -0.6, 0.64])
    pol = np.array([0.8, 0.6, 0.0])
    k = K  # k h ~ 1.1 on these triangles
    ref = _dense_side_integral(xyz, tri, ev, et, k, khat, pol)
    err = [np.linalg.norm(rcs.planewave_rhs(xyz, tri, ev, et, k, khat, pol, n) - ref) / np.linalg.norm(ref)
           for n in (3, 6, 7)]
    assert err[2] < 1e-5 and err[0] > 10 * err[2]  # the rule's own error, shrinking with its degree


def test_far_field_reciprocity_with_excitation():
    # N(d) . p = sum_n I_n int f_n . p e^{jk d.r} dS = I . V(khat = -d, p)
    xyz, tri = _mesh()
    om = O.Mesh(xyz, tri)
    ev, et = om.edges()
    rng = np.random.default_rng(5)
    I = rng.standard_normal(om.ne) + 1j * rng.standard_normal(om.ne)
    d = np.array([0.36, 0.48, 0.8])
    p = np.array([0.6, 0.0, -0.27])
    N = rcs.radiation_vectors(xyz, tri, ev, et, 2 * K, I, d[None], 6)[0]
    V = rcs.planewave_rhs(xyz, tri, ev, et, 2 * K, -d, p, 6)
    assert abs(N @ p - I @ V) < 1e-12 * abs(N @ p)


def _sphere_rcs_error(level, radius):
    xyz, tri = W.icosphere(level)
    xyz = xyz * radius
    om = O.Mesh(xyz, tri)
    ev, et = om.edges()
    Z = om.z_full(K, 7)
    I = np.linalg.solve(Z, rcs.planewave_rhs(xyz, tri, ev, et, K, [0, 0, 1], [1, 0, 0], 7))
    th = np.linspace(0, math.pi, 19)
    sE, sH = rcs.mie_bistatic(K, radius, th)
    err = []
    for plane, ref in (("E", sE), ("H", sH)):
        _, s = rcs.far_field(xyz, tri, ev, et, K, I, rcs.plane_directions(th, plane), 7)
        err.append(np.linalg.norm(s - ref) / np.linalg.norm(ref))
    return max(err)


def test_efie_sphere_rcs_matches_mie_and_converges():
    # oracle EFIE Z of a PEC sphere (r = 0.25 lambda), plane-wave excitation,
    # solve, bistatic sigma in the E- and H-planes against the Mie series;
    # the error is discretisation error and falls ~4x when the mesh is refined
    # once (h^2)
    e2 = _sphere_rcs_error(2, 0.25)
    assert e2 < 0.06
    e3 = _sphere_rcs_error(3, 0.25)
    assert e3 < 0.015 and e2 / e3 > 2.5

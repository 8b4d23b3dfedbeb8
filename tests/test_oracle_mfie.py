"""Pins of the MFIE oracle (oracle/mfie.py): the static parts of the singular
inner integral against the closed-form solid angle of a triangle (Van
Oosterom & Strackee, IEEE Trans. Biomed. Eng. 30 (1983) 125) and a dense
quadrature, the full inner integral against a dense quadrature, the singular
scheme against the regular rule on a separated pair, the vanishing self term,
the Gram term and the excitation against closed forms, and the MFIE solution
of a PEC sphere against the Mie series and the EFIE solution."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import mfie, rcs

K = 2 * math.pi


def _tri():
    xyz = np.array([[0.0, 0.0, 0.0], [0.12, 0.01, 0.0], [0.03, 0.1, 0.02]])
    return xyz, np.array([[0, 1, 2]])


def _dense_points(v, level=5):
    bary, w = O.rule(7)
    subs = [np.eye(3)]
    for _ in range(level):
        nxt = []
        for c in subs:
            m01, m12, m20 = (c[0] + c[1]) / 2, (c[1] + c[2]) / 2, (c[2] + c[0]) / 2
            nxt += [np.array([c[0], m01, m20]), np.array([m01, c[1], m12]), np.array([m20, m12, c[2]]),
                    np.array([m01, m12, m20])]
        subs = nxt
    pb = np.concatenate([bary @ s for s in subs])
    wt = np.concatenate([w / len(subs)] * len(subs))
    area = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
    return pb @ v, wt * area


def _solid_angle(r, v):
    R = v - r
    n = np.linalg.norm(R, axis=1)
    num = R[0] @ np.cross(R[1], R[2])
    den = n[0] * n[1] * n[2] + (R[0] @ R[1]) * n[2] + (R[0] @ R[2]) * n[1] + (R[1] @ R[2]) * n[0]
    return 2 * math.atan2(num, den)


@pytest.mark.parametrize("r", [[0.05, 0.04, 0.03], [0.2, -0.1, 0.05], [0.06, 0.03, -0.004], [-0.05, 0.2, 0.1]])
def test_static_parts_solid_angle_and_gradient_integral(r):
    xyz, tri = _tri()
    F = mfie.frames(xyz, tri)
    r = np.asarray(r)
    # h I_0 at k -> 0 is -Omega / (4 pi), Omega = int_q h / R^3 dS' the solid angle:
    # the closed form used by the scheme against the angle integral of the static
    # integrand (sgn(h) - h / R_e), converged, and at the default 8 angles
    om = mfie.solid_angle(r, xyz)
    assert abs(om - _solid_angle(r, xyz)) < 1e-15
    _, _, _, q32 = mfie.inner_parts(r, 0, F, 1e-9, nphi=32, static="quadrature")
    assert abs(q32.real + om / (4 * math.pi)) < 1e-13
    _, _, _, q8 = mfie.inner_parts(r, 0, F, 1e-9, static="quadrature")
    assert abs(q8.real + om / (4 * math.pi)) < 1e-6
    h, rho0, Iu, hI0 = mfie.inner_parts(r, 0, F, 1e-9)
    assert abs(hI0.real + om / (4 * math.pi)) < 1e-15
    # I_u at k -> 0: int_q (r' - rho0) / (4 pi R^3) dS' by a dense rule (the line
    # integrals are exact there; the tolerance is the dense rule's own error for
    # the point 0.004 off the plane)
    pts, wt = _dense_points(xyz, 6)
    R = np.linalg.norm(r - pts, axis=1)
    ref = np.sum(wt[:, None] * (pts - rho0) / (4 * math.pi * R[:, None] ** 3), axis=0)
    assert np.linalg.norm(Iu.real - ref) < 1e-7 * np.linalg.norm(ref)


@pytest.mark.parametrize("r", [[0.05, 0.04, 0.03], [0.2, -0.1, 0.05], [0.06, 0.03, -0.01]])
def test_inner_integral_against_dense_quadrature(r):
    xyz, tri = _tri()
    F = mfie.frames(xyz, tri)
    r = np.asarray(r)
    k = 3 * K
    T = mfie.inner_T(r, 0, F, k, nphi=16, nl=16)
    pts, wt = _dense_points(xyz)
    Rv = r - pts
    R = np.linalg.norm(Rv, axis=1)
    phi = (1 + 1j * k * R) * np.exp(-1j * k * R) / (4 * math.pi * R ** 3)
    for j in range(3):
        ref = np.sum((wt * -phi)[:, None] * np.cross(Rv, pts - xyz[j]), axis=0)
        assert np.linalg.norm(T[j] - ref) < 2e-7 * np.linalg.norm(ref)


def _sphere(level, a):
    xyz, tri = W.icosphere(level)
    return xyz * a, tri


def test_singular_scheme_equals_rule_on_separated_pair_and_self_term_vanishes():
    xyz, tri = _sphere(2, 0.25)
    om = O.Mesh(xyz, tri)
    ev, et = om.edges()
    F = mfie.frames(xyz, tri)
    v, n, area = F[0], F[1], F[2]
    bary, w = O.rule(7)
    p = 0
    d = np.linalg.norm(F[3] - F[3][p], axis=1)
    q = int(np.argmax(d > 0.15))  # a pair a few triangle sizes apart
    ra = bary @ v[p]
    rb = bary @ v[q]
    k = K
    # inner integral by the singular scheme and by the source rule at each test
    # point, both against a dense rule: the two paths of the fill agree within
    # the 7-point rule's own error at ~3 triangle sizes
    pts, wt = _dense_points(v[q], 4)
    for a in range(len(w)):
        T = mfie.inner_T(ra[a], q, F, k)
        for pp, ww, tol, sing in ((rb, area[q] * w, 2e-5, False), (pts, wt, 1e-6, True)):
            Rv = ra[a] - pp
            R = np.linalg.norm(Rv, axis=1)
            phi = (1 + 1j * k * R) * np.exp(-1j * k * R) / (4 * math.pi * R ** 3)
            for j in range(3):
                val = np.sum((ww * -phi)[:, None] * np.cross(Rv, pp - v[q, j]), axis=0)
                if sing:  # dense reference vs the singular scheme
                    assert np.linalg.norm(T[j] - val) < tol * np.linalg.norm(val)
                else:     # the source rule vs the singular scheme
                    assert np.linalg.norm(T[j] - val) < tol * np.linalg.norm(val)
    # self pair: T_j is normal to the triangle, so n x T_j = 0
    for a in range(len(w)):
        T = mfie.inner_T(ra[a], p, F, k, self_pair=True)
        assert np.linalg.norm(np.cross(n[p], T)) < 1e-14 * max(1.0, np.linalg.norm(T))


def test_gram_and_excitation_closed_forms():
    xyz, tri = _tri()
    v = xyz
    area = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
    pts, wt = _dense_points(v, 3)
    for i in range(3):
        for j in range(3):
            ref = np.sum(wt * np.einsum("ax,ax->a", pts - v[i], pts - v[j]))
            assert abs(mfie.gram_closed_form(v, area, i, j) - ref) < 1e-14
    # excitation at k = 0: V_m = sum_T coef A (c_T - v_opp) . (n_T x H)
    xs, ts = _sphere(1, 0.3)
    om = O.Mesh(xs, ts)
    ev, et = om.edges()
    pol = np.array([1.0, 0.0, 0.0])
    khat = np.array([0.0, 0.0, 1.0])
    V = mfie.planewave_rhs_mfie(xs, ts, ev, et, 0.0, khat, pol, 3)
    F = mfie.frames(xs, ts)
    opp, length = rcs.rwg_sides(xs, ts, ev, et)
    H = np.cross(khat, pol) / O.ETA0
    ref = np.zeros(len(ev))
    for s, sg in ((0, 1.0), (1, -1.0)):
        tt = et[:, s]
        ref += sg * 0.5 * length * np.einsum("nx,nx->n", F[3][tt] - xs[opp[:, s]], np.cross(F[1][tt], H))
    assert np.linalg.norm(V - ref) < 1e-13 * np.linalg.norm(ref)


def test_mfie_sphere_rcs_matches_mie_and_efie():
    # the MFIE solution of a PEC sphere (r = 0.25 lambda, 320 triangles):
    # bistatic sigma against Mie within the discretisation error of the
    # flat-triangle MFIE, and its current against the EFIE solution
    xyz, tri = _sphere(2, 0.25)
    om = O.Mesh(xyz, tri)
    ev, et = om.edges()
    Z = mfie.z_mfie(xyz, tri, ev, et, K, 7)
    I = np.linalg.solve(Z, mfie.planewave_rhs_mfie(xyz, tri, ev, et, K, [0, 0, 1], [1, 0, 0], 7))
    Ie = np.linalg.solve(om.z_full(K, 7), rcs.planewave_rhs(xyz, tri, ev, et, K, [0, 0, 1], [1, 0, 0], 7))
    th = np.linspace(0, math.pi, 19)
    sE, sH = rcs.mie_bistatic(K, 0.25, th)
    for plane, ref in (("E", sE), ("H", sH)):
        _, s = rcs.far_field(xyz, tri, ev, et, K, I, rcs.plane_directions(th, plane), 7)
        assert np.linalg.norm(s - ref) / np.linalg.norm(ref) < 0.09
    assert np.linalg.norm(I - Ie) / np.linalg.norm(Ie) < 0.04

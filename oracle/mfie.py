"""MFIE (magnetic-field integral equation) matrix of RWG functions on a closed
PEC surface, FP64, plain numpy: the paper's second formulation (Section IV.B
names the MFIE beside the EFIE; its K operator uses the gradient of the same
Green function, so the same tables serve it).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Shares no code with the
CUDA library.

Operator (e^{jwt}, outward unit normal n, triangles wound counter-clockwise
seen from outside):
    1/2 J - n x PV int grad G x J dS' = n x H_inc,
    G = e^{-jkR} / (4 pi R),  grad G = -(r - r') Phi(R),
    Phi(R) = (1 + jkR) e^{-jkR} / (4 pi R^3).
Galerkin with RWG f_m:
    Z_mn = 1/2 <f_m, f_n> - <f_m, n x int grad G x f_n dS'>,
    V_m  = <f_m, n x H_inc>,  H_inc = (khat x p) e^{-jk khat.r} / eta.

Regular pairs (not sharing a vertex): the m-point rule on both triangles.
Pairs sharing a vertex (and the self pair): the inner integral
    T_j(r) = int_q grad G x (r' - v_j) dS'
over the source triangle q is written, with h = n.(r - v_0), rho0 = r - h n,
u = r' - rho0 and w = rho0 - v_j, as
    T_j = -[h n x I_u + h (n x w) I_0 - I_u x w],
    I_0 = int_q Phi dS',  I_u = int_q Phi u dS'.
Since Phi u = -(1/4 pi) grad'_s (e^{-jkR}/R), I_u is a sum of line integrals
over the three edges (outward in-plane edge normals m_e),
    I_u = -(1/4 pi) sum_e m_e [log((l+ + R+)/(l- + R-)) + int_e (e^{-jkR} - 1)/R dl],
the first term in closed form, the second by Gauss-Legendre. In polar
coordinates about rho0 the radial integral of Phi rho is exact,
(1/4 pi)(e^{-jkd}/d - e^{-jkR_e}/R_e), so
    h I_0 = (1/4 pi) sum_e sgn(P0_e) int dphi (sgn(h) e^{-jkd} - h e^{-jkR_e}/R_e)
          = -Omega / (4 pi) + (1/4 pi) sum_e sgn(P0_e) int dphi
              (sgn(h)(e^{-jkd} - 1) - h (e^{-jkR_e} - 1)/R_e),
Omega the solid angle of q seen from r (closed form, `solid_angle`), the
smooth remainder with the angle of each edge integrated as in the EFIE scheme
(u = asinh(tan phi)).
For the self pair h = 0 exactly (the principal value; the jump is the 1/2 J
term) and T_j is normal to q, so the self pair's K part vanishes.
"""
from __future__ import annotations

import math

import numpy as np

from . import ETA0, gauss_legendre, rule

FOUR_PI = 4 * math.pi


def frames(xyz, tri):
    """Vertices (nt,3,3), unit normals, areas, centroids, edge tangents (nt,3,3),
    lengths (nt,3) and outward in-plane edge normals (nt,3,3); edge e runs v_e -> v_{e+1}."""
    v = np.asarray(xyz, dtype=np.float64)[np.asarray(tri)]
    nrm = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    area = 0.5 * np.linalg.norm(nrm, axis=1)
    n = nrm / (2 * area)[:, None]
    e = np.roll(v, -1, axis=1) - v
    length = np.linalg.norm(e, axis=2)
    t = e / length[..., None]
    m = np.cross(t, n[:, None, :])
    return v, n, area, v.mean(axis=1), t, length, m


def rwg_local(tri, ev, et):
    """Per triangle and local index i (RWG function opposite vertex i): edge id and
    sign (+1 on T+, -1 on T-), -1 / 0 where the edge is not an RWG edge."""
    tri = np.asarray(tri)
    code = -np.ones((len(tri), 3), dtype=np.int64)
    sign = np.zeros((len(tri), 3))
    for n in range(len(ev)):
        for s, sg in ((0, 1.0), (1, -1.0)):
            t = et[n, s]
            opp = [c for c in range(3) if tri[t, c] != ev[n, 0] and tri[t, c] != ev[n, 1]]
            code[t, opp[0]] = n
            sign[t, opp[0]] = sg
    return code, sign


def _near(tri):
    tri = np.asarray(tri)
    nt = len(tri)
    near = np.zeros((nt, nt), dtype=bool)
    for c in range(3):
        for d in range(3):
            near |= tri[:, c][:, None] == tri[:, d][None, :]
    return near


def inner_T(r, q, F, k, nphi=8, nl=8, self_pair=False):
    """T_j(r) = int_q grad G x (r' - v_j) dS' for j = 0, 1, 2 (complex (3, 3))."""
    v, n = F[0], F[1]
    h, rho0, Iu, hI0 = inner_parts(r, q, F, k, nphi, nl, self_pair)
    nq = n[q]
    T = np.zeros((3, 3), dtype=np.complex128)
    nxIu = np.cross(nq, Iu)
    for j in range(3):
        w = rho0 - v[q, j]
        T[j] = -(h * nxIu + np.cross(nq, w) * hI0 - np.cross(Iu, w))
    return T


def solid_angle(r, v):
    """Signed solid angle of the triangle v seen from r, closed form of Van
    Oosterom & Strackee (IEEE Trans. Biomed. Eng. 30 (1983) 125):
    tan(Omega / 2) = R1.(R2 x R3) / (R1 R2 R3 + (R1.R2) R3 + (R1.R3) R2 + (R2.R3) R1),
    R_i = v_i - r."""
    R = np.asarray(v, dtype=np.float64) - r
    n = np.linalg.norm(R, axis=1)
    num = R[0] @ np.cross(R[1], R[2])
    den = n[0] * n[1] * n[2] + (R[0] @ R[1]) * n[2] + (R[0] @ R[2]) * n[1] + (R[1] @ R[2]) * n[0]
    return 2 * math.atan2(num, den)


def inner_parts(r, q, F, k, nphi=8, nl=8, self_pair=False, static="closed"):
    """(h, rho0, I_u, h I_0) of the source triangle q for the point r. The
    static part of h I_0, sum_e sgn(P0) int dphi (sgn(h) - h / R_e), is the
    solid angle -Omega / (4 pi) (static="closed", the closed form) or is
    integrated with the angles (static="quadrature"); the remainder
    sgn(h)(e^{-jkd} - 1) - h (e^{-jkR_e} - 1) / R_e always is."""
    v, n, area, c, t, length, m = F
    vq, nq = v[q], n[q]
    h = 0.0 if self_pair else float(nq @ (r - vq[0]))
    d = abs(h)
    rho0 = r - h * nq
    xphi, wphi = gauss_legendre(nphi)
    xl, wl = gauss_legendre(nl)
    Iu = np.zeros(3, dtype=np.complex128)
    hI0 = 0.0 + 0.0j
    sgn_h = 0.0 if h == 0.0 else math.copysign(1.0, h)
    for e in range(3):
        a, b = vq[e], vq[(e + 1) % 3]
        te, me, le = t[q, e], m[q, e], length[q, e]
        P0 = float((a - rho0) @ me)
        lm = float((a - rho0) @ te)
        lp = lm + le
        Rm, Rp = np.linalg.norm(r - a), np.linalg.norm(r - b)
        R02 = P0 * P0 + d * d
        # static line integral int_e dl / R (cancellation-free forms)
        if lm >= 0:
            ratio = (lp + Rp) / (lm + Rm)
        elif lp >= 0:
            ratio = (lp + Rp) * (Rm - lm) / R02
        else:
            ratio = (Rm - lm) / (Rp - lp)
        line = math.log(ratio)
        s = 0.5 * le * (xl + 1.0)
        pts = a[None, :] + s[:, None] * te[None, :]
        R = np.linalg.norm(r[None, :] - pts, axis=1)
        line += 0.5 * le * np.sum(wl * (np.exp(-1j * k * R) - 1.0) / R)
        Iu += -me * line / FOUR_PI
        # angular part of h I_0
        if abs(P0) > 1e-12 * le:
            aP = abs(P0)
            um, up = math.asinh(lm / aP), math.asinh(lp / aP)
            u = 0.5 * (up + um) + 0.5 * (up - um) * xphi
            ch = np.cosh(u)
            Re = np.sqrt((aP * ch) ** 2 + d * d)
            f = sgn_h * (np.exp(-1j * k * d) - 1.0) - h * (np.exp(-1j * k * Re) - 1.0) / Re
            if static == "quadrature":
                f = f + sgn_h - h / Re
            hI0 += math.copysign(1.0, P0) * 0.5 * (up - um) * np.sum(wphi * f / ch) / FOUR_PI
    if static == "closed" and h != 0.0:
        hI0 += -solid_angle(r, vq) / FOUR_PI
    return h, rho0, Iu, hI0


def gram_closed_form(v, area, i, j):
    """int_T (r - v_i).(r - v_j) dS = A [(c - v_i).(c - v_j) + (1/12) sum_k |v_k - c|^2]."""
    c = v.mean(axis=0)
    return area * ((c - v[i]) @ (c - v[j]) + np.sum((v - c) ** 2) / 12.0)


def z_mfie(xyz, tri, ev, et, k, npts, nphi=8, nl=8, parts=("identity", "regular", "near")):
    """The full MFIE matrix (complex128 [ne, ne]) and its parts."""
    xyz = np.asarray(xyz, dtype=np.float64)
    F = frames(xyz, tri)
    v, n, area, c, t, length, m = F
    nt = len(tri)
    ne = len(ev)
    code, sign = rwg_local(tri, ev, et)
    bary, w = rule(npts)
    ra = np.einsum("ac,tcx->tax", bary, v)          # (nt, m, 3) rule points
    coef = sign * length[np.arange(nt)[:, None], (np.arange(3)[None, :] + 1) % 3] / (2 * area[:, None])
    # f_i on triangle t at point a: coef[t, i] (r_a - v_i); local edge i is opposite vertex i,
    # its length is |v_{i+1} - v_{i+2}| = length[t, (i + 1) % 3]
    fv = coef[:, :, None, None] * (ra[:, None, :, :] - v[:, :, None, :])  # (nt, 3, m, 3)
    Z = np.zeros((ne, ne), dtype=np.complex128)
    near = _near(tri)

    def scatter(p, q, blk):
        for i in range(3):
            if code[p, i] < 0:
                continue
            for j in range(3):
                if code[q, j] < 0:
                    continue
                Z[code[p, i], code[q, j]] += blk[i, j]

    if "identity" in parts:
        for p in range(nt):
            blk = np.zeros((3, 3), dtype=np.complex128)
            for i in range(3):
                for j in range(3):
                    blk[i, j] = 0.5 * coef[p, i] * coef[p, j] * gram_closed_form(v[p], area[p], i, j)
            scatter(p, p, blk)
    if "regular" in parts:
        for p in range(nt):
            qs = np.nonzero(~near[p])[0]
            if len(qs) == 0:
                continue
            Rv = ra[p][None, :, None, :] - ra[qs][:, None, :, :]          # (nq, a, b, 3)
            R = np.linalg.norm(Rv, axis=3)
            Phi = (1 + 1j * k * R) * np.exp(-1j * k * R) / (FOUR_PI * R ** 3)
            W = area[p] * area[qs][:, None, None] * w[None, :, None] * w[None, None, :] * Phi
            # f_i(r_a) . (n_p x (R x f_j(r_b))) = (f_i . R)(n_p . f_j) - (f_i . f_j)(n_p . R)
            fi = fv[p]                                                    # (3, a, 3)
            fj = fv[qs]                                                   # (nq, 3, b, 3)
            fiR = np.einsum("iax,qabx->qiab", fi, Rv)
            nfj = np.einsum("x,qjbx->qjb", n[p], fj)
            fifj = np.einsum("iax,qjbx->qijab", fi, fj)
            nR = np.einsum("x,qabx->qab", n[p], Rv)
            val = np.einsum("qab,qiab,qjb->qij", W, fiR, nfj) - np.einsum("qab,qijab,qab->qij", W, fifj, nR)
            for qi, q in enumerate(qs):
                scatter(p, q, val[qi])
    if "near" in parts:
        for p in range(nt):
            for q in np.nonzero(near[p])[0]:
                blk = np.zeros((3, 3), dtype=np.complex128)
                for a in range(len(w)):
                    T = inner_T(ra[p, a], q, F, k, nphi, nl, self_pair=(p == q))
                    for j in range(3):
                        vec = np.cross(n[p], coef[q, j] * T[j])
                        for i in range(3):
                            blk[i, j] -= area[p] * w[a] * (fv[p, i, a] @ vec)
                scatter(p, q, blk)
    return Z


def planewave_rhs_mfie(xyz, tri, ev, et, k, khat, pol, npts, eta=ETA0):
    """V_m = <f_m, n x H_inc>, H_inc = (khat x p) e^{-jk khat.r} / eta."""
    F = frames(xyz, tri)
    v, n, area, c, t, length, m = F
    nt = len(tri)
    code, sign = rwg_local(tri, ev, et)
    bary, w = rule(npts)
    ra = np.einsum("ac,tcx->tax", bary, v)
    khat = np.asarray(khat, dtype=np.float64)
    hvec = np.cross(khat, np.asarray(pol, dtype=np.complex128)) / eta
    V = np.zeros(len(ev), dtype=np.complex128)
    for tt in range(nt):
        nxh = np.cross(n[tt], hvec)
        ph = np.exp(-1j * k * (ra[tt] @ khat))
        for i in range(3):
            if code[tt, i] < 0:
                continue
            coef = sign[tt, i] * length[tt, (i + 1) % 3] / (2 * area[tt])
            V[code[tt, i]] += area[tt] * coef * np.sum(w * ((ra[tt] - v[tt, i]) @ nxh) * ph)
    return V

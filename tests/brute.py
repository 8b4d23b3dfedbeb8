"""Independent numpy references for the oracle pins.

* Static potential integrals over a planar triangle, from the mathematics of
  integrals of 1/R and (r' - rho0)/R over a polygon (edge-by-edge closed
  forms in the in-plane edge frame).
* Duffy-transformed Gauss quadrature of smooth or 1/R-singular integrands over
  a triangle split at the projection point (signed sub-triangles).
* Brute-force EFIE entries with high-order product rules.
None of this code calls the oracle.
"""
import math

import numpy as np

TWO_PI = 2 * math.pi


def gl(n):
    return np.polynomial.legendre.leggauss(n)


def frame(v):
    v = np.asarray(v, float)
    n = np.cross(v[1] - v[0], v[2] - v[0])
    return n / np.linalg.norm(n)


def static_potentials(r, v):
    """(int_T 1/R dS', int_T (r' - rho0)/R dS') for observation r, triangle v."""
    v = np.asarray(v, float)
    r = np.asarray(r, float)
    n = frame(v)
    h = float(np.dot(n, r - v[0]))
    d = abs(h)
    rho0 = r - h * n
    s_scalar = 0.0
    s_vec = np.zeros(3)
    for i in range(3):
        a, b = v[i], v[(i + 1) % 3]
        L = np.linalg.norm(b - a)
        t = (b - a) / L
        m = np.cross(t, n)
        P0 = float(np.dot(a - rho0, m))
        lm = float(np.dot(a - rho0, t))
        lp = float(np.dot(b - rho0, t))
        R02 = P0 * P0 + d * d
        Rm = math.sqrt(lm * lm + R02)
        Rp = math.sqrt(lp * lp + R02)
        # log((R+ + l+)/(R- + l-)), each factor R + l written as R0^2/(R - l)
        # when l < 0 to avoid cancellation
        def f(l, R):
            return R + l if l >= 0 else R02 / (R - l)
        lg = math.log(f(lp, Rp)) - math.log(f(lm, Rm)) if R02 > 0 else 0.0
        s_scalar += P0 * lg - d * (math.atan2(P0 * lp, R02 + d * Rp) - math.atan2(P0 * lm, R02 + d * Rm))
        s_vec += 0.5 * m * (R02 * lg + lp * Rp - lm * Rm)
    return s_scalar, s_vec, rho0


def duffy_points(apex, b, c, n):
    """Points/weights of a Duffy-collapsed n x n Gauss rule on triangle
    (apex, b, c); the weight carries the signed area (orientation about the
    normal of the reference frame)."""
    x, w = gl(n)
    u = 0.5 * (x + 1)
    wu = 0.5 * w
    U, V = np.meshgrid(u, u, indexing="ij")
    WU, WV = np.meshgrid(wu, wu, indexing="ij")
    apex, b, c = (np.asarray(z, float) for z in (apex, b, c))
    P = apex[None, None, :] + U[..., None] * (b - apex)[None, None, :] + (U * V)[..., None] * (c - b)[None, None, :]
    J = np.linalg.norm(np.cross(b - apex, c - b))
    W = WU * WV * U * J
    return P.reshape(-1, 3), W.ravel()


def split_rule(rho0, v, n):
    """Signed decomposition of triangle v into (rho0, v_i, v_{i+1}); returns
    points and weights whose sum integrates over v."""
    v = np.asarray(v, float)
    nrm = frame(v)
    pts, wts = [], []
    for i in range(3):
        a, b = v[i], v[(i + 1) % 3]
        sgn = np.sign(np.dot(np.cross(a - rho0, b - rho0), nrm))
        if sgn == 0:
            continue
        P, W = duffy_points(rho0, a, b, n)
        pts.append(P)
        wts.append(sgn * W)
    return np.concatenate(pts), np.concatenate(wts)


def inner_integrals(r, v, k, n=40):
    """Reference (I0, I1) = (int G, int (r' - rho0) G), G = e^{-jkR}/(4 pi R):
    static closed form plus Duffy quadrature of the bounded remainder."""
    s0, s1, rho0 = static_potentials(r, v)
    P, W = split_rule(rho0, v, n)
    R = np.linalg.norm(P - np.asarray(r, float)[None, :], axis=1)
    rem = np.where(R > 0, (np.exp(-1j * k * R) - 1.0) / np.where(R > 0, R, 1.0), -1j * k)
    I0 = (s0 + np.sum(W * rem)) / (4 * math.pi)
    I1 = (s1 + np.sum((W * rem)[:, None] * (P - rho0[None, :]), axis=0)) / (4 * math.pi)
    return I0, I1, rho0


# ---------------------------------------------------------------- RWG / EFIE
def rwg(xyz, tri):
    """Interior edges in lexicographic (lower, higher) vertex order with
    T+ = smaller triangle index; per edge the opposite vertex in T+/T-."""
    e = {}
    for t, (a, b, c) in enumerate(tri):
        for i, (p, q) in enumerate(((b, c), (c, a), (a, b))):
            e.setdefault((min(p, q), max(p, q)), []).append((t, tri[t][i]))
    out = []
    for key in sorted(e):
        if len(e[key]) == 2:
            (t1, o1), (t2, o2) = sorted(e[key])
            out.append((key, t1, t2, o1, o2))
    return out


def entry_brute(xyz, tri, edges, m, n, k, outer_rule, inner="gauss", n_in=12, eta=376.730313668,
                near=None):
    """Z_mn with the given outer rule (bary, w) on the test triangles and a
    reference inner integral: 'gauss' = Duffy product Gauss of the regular
    integrand (n_in^2 points), 'singular' = inner_integrals (any pair)."""
    bary, w = outer_rule
    (km, tp_m, tm_m, op_m, om_m) = edges[m]
    (kn, tp_n, tm_n, op_n, om_n) = edges[n]
    lm = np.linalg.norm(xyz[km[0]] - xyz[km[1]])
    ln = np.linalg.norm(xyz[kn[0]] - xyz[kn[1]])
    z = 0j
    for p, sp, vp in ((tp_m, 1, op_m), (tm_m, -1, om_m)):
        Vp = xyz[tri[p]]
        Ap = 0.5 * np.linalg.norm(np.cross(Vp[1] - Vp[0], Vp[2] - Vp[0]))
        ra = bary @ Vp
        fm = sp * lm / (2 * Ap) * (ra - xyz[vp])
        divm = sp * lm / Ap
        for q, sq, vq in ((tp_n, 1, op_n), (tm_n, -1, om_n)):
            Vq = xyz[tri[q]]
            Aq = 0.5 * np.linalg.norm(np.cross(Vq[1] - Vq[0], Vq[2] - Vq[0]))
            divn = sq * ln / Aq
            for a in range(len(w)):
                if inner == "gauss":
                    cq = Vq.mean(axis=0)
                    P, W = split_rule(cq, Vq, n_in)
                    R = np.linalg.norm(P - ra[a][None, :], axis=1)
                    G = np.exp(-1j * k * R) / (4 * math.pi * R)
                    I0 = np.sum(W * G)
                    Fn = sq * ln / (2 * Aq) * np.sum((W * G)[:, None] * (P - xyz[vq][None, :]), axis=0)
                else:
                    I0, I1, rho0 = inner_integrals(ra[a], Vq, k, n_in)
                    Fn = sq * ln / (2 * Aq) * (I1 + (rho0 - xyz[vq]) * I0)
                z += Ap * w[a] * (np.dot(fm[a], Fn) - divm * divn / k**2 * I0)
    return 1j * k * eta * z

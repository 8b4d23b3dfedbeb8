"""Scattering by a PEC body from the EFIE solution (FP64, plain numpy).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark may
import this module; the product library never does. It shares no code with
the CUDA library.

* Plane-wave excitation of the RWG functions: V_m = <f_m, E_inc>, the right
  side of Z I = V for the EFIE matrix of the oracle (e^{jwt} convention,
  E_inc = p e^{-jk khat.r}).
* Far field of an RWG current J = sum_n I_n f_n: F(d) = -(jk eta / 4 pi)
  (N - (d.N) d), N = int J e^{jk d.r'} dS', and the bistatic radar cross
  section sigma(d) = 4 pi |F(d)|^2 / |E_inc|^2.
* The Mie series of a perfectly conducting sphere (bistatic sigma in the E-
  and H-planes, extinction and scattering cross sections), written from the
  series solution in Bohren & Huffman, "Absorption and Scattering of Light by
  Small Particles" (1983), Sections 4.4-4.5, with the perfect-conductor limit
  of the coefficients: a_n = psi_n'(x) / xi_n'(x), b_n = psi_n(x) / xi_n(x).

RWG function n on T+ / T- (T+ = the first triangle of edge n, the free vertex
v_opp opposite the edge): f_n = +- l_n / (2 A) (r - v_opp); integrals over a
triangle use the oracle's m-point rule, int_T g dS = A sum_a w_a g(r_a).

What is pinned (tests/test_oracle_rcs.py): the Mie series by the optical
theorem (extinction = scattering for a lossless sphere), its angular
integral, the two backscatter forms and the small-sphere (Rayleigh) limit;
the excitation and far field by their k = 0 closed forms, by a subdivided
higher-order quadrature and by reciprocity (N(d) . p = I . V(-d, p)); the
whole EFIE chain by the oracle's Z on a small sphere against Mie.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

from . import ETA0, rule


def rwg_sides(xyz, tri, ev, et):
    """Per edge n and side s (0: T+, 1: T-): triangle id, opposite vertex and sign."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tri = np.asarray(tri)
    ne = len(ev)
    opp = np.zeros((ne, 2), dtype=np.int64)
    for n in range(ne):
        for s in range(2):
            t = tri[et[n, s]]
            rest = [v for v in t if v != ev[n, 0] and v != ev[n, 1]]
            assert len(rest) == 1
            opp[n, s] = rest[0]
    length = np.linalg.norm(xyz[ev[:, 0]] - xyz[ev[:, 1]], axis=1)
    return opp, length


def _points(xyz, tri, npts):
    """Rule points of every triangle: (nt, m, 3) and the weights (m,)."""
    bary, w = rule(npts)
    v = np.asarray(xyz, dtype=np.float64)[np.asarray(tri)]  # (nt, 3, 3)
    return np.einsum("ac,tcx->tax", bary, v), w


def _side_integrals(xyz, tri, ev, et, npts, phase):
    """For every edge n and side s: (sign l_n / 2) sum_a w_a (r_a - v_opp) phase(r_a)
    (complex (ne, 2, 3)), i.e. int_{T} f_n phase dS on that side."""
    opp, length = rwg_sides(xyz, tri, ev, et)
    pts, w = _points(xyz, tri, npts)
    xyz = np.asarray(xyz, dtype=np.float64)
    out = np.zeros((len(ev), 2, 3), dtype=np.complex128)
    for s, sign in ((0, 1.0), (1, -1.0)):
        ra = pts[et[:, s]]                        # (ne, m, 3)
        rel = ra - xyz[opp[:, s]][:, None, :]     # r_a - v_opp
        ph = phase(ra)                            # (ne, m)
        out[:, s, :] = sign * 0.5 * length[:, None] * np.einsum("a,nax,na->nx", w, rel, ph)
    return out


def planewave_rhs(xyz, tri, ev, et, k, khat, pol, npts):
    """V_m = int f_m . p e^{-jk khat.r} dS (both triangles of edge m)."""
    khat = np.asarray(khat, dtype=np.float64)
    pol = np.asarray(pol, dtype=np.complex128)
    side = _side_integrals(xyz, tri, ev, et, npts, lambda r: np.exp(-1j * k * (r @ khat)))
    return (side.sum(axis=1) * pol).sum(axis=1)


def radiation_vectors(xyz, tri, ev, et, k, I, dirs, npts):
    """N(d) = sum_n I_n int f_n e^{jk d.r'} dS' for every direction d: (nd, 3)."""
    dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
    I = np.asarray(I, dtype=np.complex128)
    out = np.zeros((len(dirs), 3), dtype=np.complex128)
    for i, d in enumerate(dirs):
        side = _side_integrals(xyz, tri, ev, et, npts, lambda r, d=d: np.exp(1j * k * (r @ d)))
        out[i] = np.einsum("n,nsx->x", I, side)
    return out


def far_field(xyz, tri, ev, et, k, I, dirs, npts, eta=ETA0):
    """F(d) = -(j k eta / 4 pi) (N - (d.N) d) and sigma(d) = 4 pi |F|^2 (|E_inc| = 1)."""
    dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
    N = radiation_vectors(xyz, tri, ev, et, k, I, dirs, npts)
    Nt = N - np.einsum("dx,dx->d", dirs, N)[:, None] * dirs
    F = -1j * k * eta / (4 * math.pi) * Nt
    return F, 4 * math.pi * np.sum(np.abs(F) ** 2, axis=1)


# ------------------------------------------------------------------ Mie series
def mie_coefficients(x, nmax=None):
    """a_n, b_n (n = 1..nmax) of a perfectly conducting sphere, size parameter x = ka."""
    if nmax is None:
        nmax = int(math.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0))
    n = np.arange(1, nmax + 1)
    jn, jnp = special.spherical_jn(n, x), special.spherical_jn(n, x, derivative=True)
    yn, ynp = special.spherical_yn(n, x), special.spherical_yn(n, x, derivative=True)
    hn, hnp = jn + 1j * yn, jnp + 1j * ynp
    psi, dpsi = x * jn, jn + x * jnp        # psi_n = x j_n(x)
    xi, dxi = x * hn, hn + x * hnp          # xi_n = x h_n^(1)(x)
    return dpsi / dxi, psi / xi


def mie_angular(nmax, mu):
    """pi_n(mu), tau_n(mu) for n = 1..nmax (upward recurrences), shapes (nmax, len(mu))."""
    mu = np.atleast_1d(np.asarray(mu, dtype=np.float64))
    pi = np.zeros((nmax + 1, mu.size))
    tau = np.zeros((nmax + 1, mu.size))
    pi[1] = 1.0
    if nmax >= 2:
        pi[2] = 3.0 * mu
    for n in range(3, nmax + 1):
        pi[n] = (2 * n - 1) / (n - 1) * mu * pi[n - 1] - n / (n - 1) * pi[n - 2]
    for n in range(1, nmax + 1):
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi[1:], tau[1:]


def mie_amplitudes(x, theta):
    """S1(theta), S2(theta) of a PEC sphere (theta from the direction of incidence)."""
    a, b = mie_coefficients(x)
    nmax = len(a)
    n = np.arange(1, nmax + 1)
    pi, tau = mie_angular(nmax, np.cos(theta))
    c = ((2 * n + 1) / (n * (n + 1)))[:, None]
    S1 = np.sum(c * (a[:, None] * pi + b[:, None] * tau), axis=0)
    S2 = np.sum(c * (a[:, None] * tau + b[:, None] * pi), axis=0)
    return S1, S2


def mie_bistatic(k, radius, theta):
    """sigma in the E-plane (S2) and the H-plane (S1) for incidence along +z with
    E along x: sigma = 4 pi |S|^2 / k^2."""
    S1, S2 = mie_amplitudes(k * radius, np.asarray(theta, dtype=np.float64))
    return 4 * math.pi * np.abs(S2) ** 2 / k ** 2, 4 * math.pi * np.abs(S1) ** 2 / k ** 2


def mie_cross_sections(k, radius):
    """(extinction, scattering) cross sections from the coefficients."""
    a, b = mie_coefficients(k * radius)
    n = np.arange(1, len(a) + 1)
    ext = 2 * math.pi / k ** 2 * np.sum((2 * n + 1) * np.real(a + b))
    sca = 2 * math.pi / k ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    return ext, sca


def mie_backscatter(k, radius):
    """Monostatic sigma from the alternating series (pi / k^2) |sum (2n+1)(-1)^n (a_n - b_n)|^2."""
    a, b = mie_coefficients(k * radius)
    n = np.arange(1, len(a) + 1)
    return math.pi / k ** 2 * np.abs(np.sum((2 * n + 1) * (-1.0) ** n * (a - b))) ** 2


def plane_directions(theta, plane):
    """Directions at angle theta from +z in the xz-plane ('E', E along x) or yz-plane ('H')."""
    theta = np.asarray(theta, dtype=np.float64)
    s, c = np.sin(theta), np.cos(theta)
    z = np.zeros_like(theta)
    return np.stack([s, z, c] if plane == "E" else [z, s, c], axis=1)

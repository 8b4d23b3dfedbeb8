"""GPU scattering stage against the oracle (oracle/rcs.py) and the Mie
series: plane-wave excitation, far field, and the whole chain fill -> solve ->
bistatic RCS with the table and the direct fill."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1901_04162_gb300 as gf
import workloads as W
from oracle import rcs

pytestmark = pytest.mark.gpu
K = 2 * math.pi


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("prec,tol", [(gf.GF_FP64, 1e-12), (gf.GF_FP32, 2e-6)])
def test_excitation_matches_oracle(prec, tol):
    wl = W.sphere_3072()
    m = gf.Mesh(wl.xyz, wl.tri)
    om = O.Mesh(wl.xyz, wl.tri)
    ev, et = om.edges()
    p = gf.gf_params_default(rule=wl.rule)
    khat = np.array([0.36, -0.48, 0.8])
    pol = np.array([0.8, 0.6, 0.0]) + 1j * np.array([0.0, 0.0, 0.3])
    dt = torch.complex64 if prec == gf.GF_FP32 else torch.complex128
    V = torch.empty(m.ne, dtype=dt, device="cuda")
    gf.gf_excitation(m.h, 2 * K, p, khat, pol, prec, V)
    ref = rcs.planewave_rhs(wl.xyz, wl.tri, ev, et, 2 * K, khat, pol, wl.rule)
    assert _rel(V.cpu().numpy(), ref) <= tol
    # k = 0: the closed form (exact for the rule)
    gf.gf_excitation(m.h, 0.0, p, [0, 0, 1], [1, 0, 0], prec, V)
    assert _rel(V.cpu().numpy(), rcs.planewave_rhs(wl.xyz, wl.tri, ev, et, 0.0, [0, 0, 1], [1, 0, 0], wl.rule)) <= tol


@pytest.mark.parametrize("prec,tol", [(gf.GF_FP64, 1e-12), (gf.GF_FP32, 2e-6)])
def test_far_field_matches_oracle(prec, tol):
    wl = W.sphere_3072()
    m = gf.Mesh(wl.xyz, wl.tri)
    om = O.Mesh(wl.xyz, wl.tri)
    ev, et = om.edges()
    p = gf.gf_params_default(rule=wl.rule)
    rng = np.random.default_rng(11)
    I = (rng.standard_normal(m.ne) + 1j * rng.standard_normal(m.ne)).astype(np.complex128)
    if prec == gf.GF_FP32:
        I = I.astype(np.complex64).astype(np.complex128)  # the same rounded current on both sides
    dirs = rng.standard_normal((13, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    dt = torch.complex64 if prec == gf.GF_FP32 else torch.complex128
    F, sigma = gf.gf_far_field(m.h, K, p, prec, torch.from_numpy(I).to(dt).cuda(),
                               torch.from_numpy(dirs).cuda())
    Fo, so = rcs.far_field(wl.xyz, wl.tri, ev, et, K, I, dirs, wl.rule)
    assert _rel(F.cpu().numpy(), Fo) <= min(tol, 1e-10)
    assert _rel(sigma.cpu().numpy(), so) <= min(tol, 1e-10)


def test_fp64_chain_matches_oracle_chain():
    # FP64 direct fill + solve + far field on a 0.5 lambda sphere (1280 triangles)
    # against the oracle's Z, numpy solve and far field
    xyz, tri = W.icosphere(3)
    xyz = xyz * 0.5
    m = gf.Mesh(xyz, tri)
    om = O.Mesh(xyz, tri)
    ev, et = om.edges()
    p = gf.gf_params_default(rule=7)
    th = np.linspace(0, math.pi, 19)
    d = torch.from_numpy(rcs.plane_directions(th, "E")).cuda()
    sigma, I = gf.planewave_rcs(m, K, d, p, None, gf.GF_FP64)
    Io = np.linalg.solve(om.z_full(K, 7), rcs.planewave_rhs(xyz, tri, ev, et, K, [0, 0, 1], [1, 0, 0], 7))
    _, so = rcs.far_field(xyz, tri, ev, et, K, Io, rcs.plane_directions(th, "E"), 7)
    assert _rel(I.cpu().numpy(), Io) <= 1e-10
    assert _rel(sigma.cpu().numpy(), so) <= 1e-10


def test_sphere_rcs_table_and_direct_vs_mie():
    # the 1 lambda sphere of the benchmark (5120 triangles, 7-point rule), FP32
    # fills: bistatic sigma in the E- and H-planes against Mie (the lambda/13
    # mesh's discretisation error; measured 0.23 %), and the table fill against
    # the direct fill (the table's own error; measured 1.5e-6, the paper's
    # Section IV.B order of magnitude)
    wl = W.sphere_7680()
    a = wl.extra["sphere_radius"]
    m = gf.Mesh(wl.xyz, wl.tri)
    p = gf.gf_params_default(rule=wl.rule)
    lo, hi = m.range(wl.rule, gf.GF_FP32)
    tab = gf.Table(wl.k, lo, hi, p)
    th = np.linspace(0, math.pi, 37)
    sE, sH = rcs.mie_bistatic(wl.k, a, th)
    for plane, ref in (("E", sE), ("H", sH)):
        d = torch.from_numpy(rcs.plane_directions(th, plane)).cuda()
        st, _ = gf.planewave_rcs(m, wl.k, d, p, tab, gf.GF_FP32)
        sd, _ = gf.planewave_rcs(m, wl.k, d, p, None, gf.GF_FP32)
        st, sd = st.cpu().numpy(), sd.cpu().numpy()
        assert _rel(st, ref) < 0.01, plane
        assert _rel(st, sd) < 1e-5, plane

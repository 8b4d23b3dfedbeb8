"""Adjoint fill (dL/d vertex coordinates, dL/dk) vs the oracle's dual-number
gradient of the FP64 direct fill, central differences of the oracle, and the
autograd wrapper. L = Re(a^H Z b), gZ = a conj(b)^T."""
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
import paper_1901_04162_gb300 as gf
import workloads as W

pytestmark = pytest.mark.gpu
K = 2 * math.pi


def gpu_grad(xyz, tri, rule, a, b, table=True, near_fp64=0):
    m = gf.Mesh(xyz, tri)
    p = gf.gf_params_default(rule=rule, near_fp64=near_fp64)
    tab = None
    if table:
        lo, hi = m.range(rule, gf.GF_FP32)
        tab = gf.Table(K, lo, hi, p)
    gZ = torch.from_numpy(np.outer(a, np.conj(b)).astype(np.complex64)).cuda()
    dxyz, dk = gf.gf_fill_backward(m, K, p, tab, gZ)
    torch.cuda.synchronize()
    return dxyz.cpu().numpy(), float(dk.cpu()[0])


@pytest.mark.parametrize("table", [True, False])
@pytest.mark.parametrize("near_fp64", [0, 1])
def test_small_sphere_vs_oracle_gradient(table, near_fp64):
    xyz, tri = W.octasphere(2, 0.8)
    xyz = W.jitter(xyz, tri, 0.03, 8)
    om = O.Mesh(xyz, tri)
    a = W.complex_gaussian(om.ne, 1)
    b = W.complex_gaussian(om.ne, 2)
    _, g_ref, dk_ref = om.loss_grad(K, 6, a, b)
    g, dk = gpu_grad(xyz, tri, 6, a, b, table, near_fp64)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    assert abs(dk - dk_ref) <= 1e-4 * abs(dk_ref)


def test_flagged_cells_gradient():
    # A Green table of 40 base samples per wavelength (graded to the default
    # tolerance): the interpolant stays accurate, but nearly every FP32
    # lattice cell holds samples or needs its cubic term, so nearly every
    # point pair's value and derivative come from the exact correction after
    # the kernel's loop. The gradient must match the oracle as the default
    # table's does, and the direct-evaluation adjoint to 2e-5 (a lost
    # correction moves it by 2e-4).
    xyz, tri = W.octasphere(2, 0.8)
    xyz = W.jitter(xyz, tri, 0.03, 8)
    om = O.Mesh(xyz, tri)
    a = W.complex_gaussian(om.ne, 1)
    b = W.complex_gaussian(om.ne, 2)
    _, g_ref, dk_ref = om.loss_grad(K, 6, a, b)
    m = gf.Mesh(xyz, tri)
    gZ = torch.from_numpy(np.outer(a, np.conj(b)).astype(np.complex64)).cuda()
    p = gf.gf_params_default(rule=6, green_n_per_lambda=40)
    lo, hi = m.range(6, gf.GF_FP32)
    g, dk = gf.gf_fill_backward(m, K, p, gf.Table(K, lo, hi, p), gZ)
    gd, dkd = gf.gf_fill_backward(m, K, p, None, gZ)
    torch.cuda.synchronize()
    g, dk, gd, dkd = g.cpu().numpy(), float(dk.cpu()[0]), gd.cpu().numpy(), float(dkd.cpu()[0])
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    assert abs(dk - dk_ref) <= 1e-4 * abs(dk_ref)
    assert np.linalg.norm(g - gd) <= 2e-5 * np.linalg.norm(gd)
    assert abs(dk - dkd) <= 2e-5 * abs(dkd)


def golden_grad_2048():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "grad_sphere2048.txt")
    rows = [list(map(float, ln.split())) for ln in open(path)]
    L, dk = rows[0]
    return L, np.array(rows[1:]), dk


def test_sphere_2048_full_gradient_vs_oracle():
    # every vertex coordinate and k against the oracle's dual-number gradient
    # of its FP64 direct fill (tests/golden/make_grad_sphere2048.py)
    wl = W.sphere_3072()
    a = W.complex_gaussian(3072, 7)
    b = W.complex_gaussian(3072, 8)
    g, dk = gpu_grad(wl.xyz, wl.tri, 6, a, b, table=True)
    _, g_ref, dk_ref = golden_grad_2048()
    assert g.shape == g_ref.shape
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    assert abs(dk - dk_ref) <= 1e-4 * abs(dk_ref)


def restricted_loss(xyz, tri, k, a, b, rows):
    """Re(a^H Z b) over the entries of the given RWG rows and columns (the
    oracle's FP64 direct fill): the part of L that moves with the vertices of
    those unknowns' triangles."""
    om = O.Mesh(xyz, tri)
    rows = np.asarray(sorted(rows))
    rest = np.setdiff1d(np.arange(om.ne), rows)
    mi = np.concatenate([np.repeat(rows, om.ne), np.tile(rest, len(rows))])
    ni = np.concatenate([np.tile(np.arange(om.ne), len(rows)), np.repeat(rows, len(rest))])
    z = om.z_entries(k, 6, mi, ni)
    return float(np.real(np.sum(np.conj(a[mi]) * z * b[ni])))


def test_sphere_2048_central_differences():
    # 64 seeded vertex coordinates and k: central differences (step 1e-4
    # lambda, and 1e-4 k) of the oracle's FP64 direct loss
    wl = W.sphere_3072()
    om = O.Mesh(wl.xyz, wl.tri)
    a = W.complex_gaussian(om.ne, 7)
    b = W.complex_gaussian(om.ne, 8)
    g, dk = gpu_grad(wl.xyz, wl.tri, 6, a, b, table=True)
    _, et = om.edges()
    scale = np.abs(g).max()
    rng = np.random.default_rng(64)
    verts = rng.choice(len(wl.xyz), 64, replace=False)
    coords = rng.integers(3, size=64)
    h = 1e-4
    for v, c in zip(verts, coords):
        tris = np.where((wl.tri == v).any(axis=1))[0]
        rows = np.where(np.isin(et, tris).any(axis=1))[0]
        xp, xm = wl.xyz.copy(), wl.xyz.copy()
        xp[v, c] += h
        xm[v, c] -= h
        fd = (restricted_loss(xp, wl.tri, K, a, b, rows) - restricted_loss(xm, wl.tri, K, a, b, rows)) / (2 * h)
        assert abs(g[v, c] - fd) <= 1e-3 * scale, (v, c, g[v, c], fd)
    hk = 1e-4 * K
    Lp = float(np.real(np.conj(a) @ om.z_full(K + hk, 6) @ b))
    Lm = float(np.real(np.conj(a) @ om.z_full(K - hk, 6) @ b))
    assert abs(dk - (Lp - Lm) / (2 * hk)) <= 1e-3 * abs(dk)


def test_autograd_wrapper():
    xyz, tri = W.octasphere(2, 0.8)
    xyz = W.jitter(xyz, tri, 0.03, 9)
    m = gf.Mesh(xyz, tri)
    p = gf.gf_params_default(rule=4)
    lo, hi = m.range(4, gf.GF_FP32)
    tab = gf.Table(K, lo, hi, p)
    a = torch.from_numpy(W.complex_gaussian(m.ne, 3).astype(np.complex64)).cuda()
    b = torch.from_numpy(W.complex_gaussian(m.ne, 4).astype(np.complex64)).cuda()
    x = torch.tensor(xyz, dtype=torch.float64, device="cuda", requires_grad=True)
    k = torch.tensor(K, dtype=torch.float64, requires_grad=True)
    Z = gf.efie_fill(x, k, m, tab, p)
    L = torch.real(torch.conj(a) @ (Z @ b))
    L.backward()
    gZ = torch.outer(a, torch.conj(b)).contiguous()
    dx, dk = gf.gf_fill_backward(m, K, p, tab, gZ)
    assert torch.allclose(x.grad, dx, rtol=1e-6, atol=1e-9 * float(dx.abs().max()))
    assert abs(float(k.grad) - float(dk[0])) <= 1e-6 * abs(float(dk[0]))

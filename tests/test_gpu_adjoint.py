"""Adjoint fill (dL/d vertex coordinates, dL/dk) vs the oracle's dual-number
gradient of the FP64 direct fill, central differences of the oracle, and the
autograd wrapper. L = Re(a^H Z b), gZ = a conj(b)^T."""
import math

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


def test_sphere_2048_sampled_vertices_fd_and_dk():
    wl = W.sphere_3072()
    om = O.Mesh(wl.xyz, wl.tri)
    a = W.complex_gaussian(om.ne, 7)
    b = W.complex_gaussian(om.ne, 8)
    g, dk = gpu_grad(wl.xyz, wl.tri, 6, a, b, table=True)
    verts = [0, 517, 1000]
    mask = np.isin(np.arange(len(wl.tri)), np.where(np.isin(wl.tri, verts).any(axis=1))[0]).astype(np.int32)
    _, g_ref, _ = om.loss_grad(K, 6, a, b, tri_mask=mask)
    scale = np.abs(g_ref[verts]).max()
    assert np.abs(g[verts] - g_ref[verts]).max() <= 1e-4 * scale
    # central differences (step 1e-4 lambda) of the oracle's loss restricted to
    # the pairs that move
    h = 1e-4
    for v, c in [(517, 0), (1000, 2)]:
        xp, xm = wl.xyz.copy(), wl.xyz.copy()
        xp[v, c] += h
        xm[v, c] -= h
        Lp = O.Mesh(xp, wl.tri).loss_grad(K, 6, a, b, tri_mask=mask)[0]
        Lm = O.Mesh(xm, wl.tri).loss_grad(K, 6, a, b, tri_mask=mask)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(g[v, c] - fd) <= 1e-3 * scale, (v, c, g[v, c], fd)
    _, dk_ref = om.loss_dk(K, 6, a, b)
    assert abs(dk - dk_ref) <= 1e-4 * abs(dk_ref)


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

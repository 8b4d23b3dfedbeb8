"""Tables in u = kR (gf_table_create_kr): one table for every wavenumber of a
sweep, against the oracle through the scaling identity Z_k(mesh) =
Z_1(k mesh) / k^2 (with the oracle's tables for k = 1 over the same u range),
and against per-k tables in the EFIE, MFIE, batched and sparse fills."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1901_04162_gb300 as gf
import workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _mesh():
    xyz, tri = W.icosphere(2)
    return W.jitter(xyz * 0.6, tri, 0.03, 12), tri


def test_fp64_kr_fill_matches_scaled_oracle():
    xyz, tri = _mesh()
    k = 3.1 * math.pi
    m = gf.Mesh(xyz, tri)
    p = gf.gf_params_default(rule=4)
    lo, hi = m.range(4, gf.GF_FP64)
    umin, umax = 0.9 * k * lo, 1.05 * k * hi
    tab = gf.Table.kr(umin, umax, p)
    Z = torch.empty((m.ne, m.ne), dtype=torch.complex128, device="cuda")
    gf.gf_fill(m.h, k, p, tab.h, gf.GF_FP64, Z)
    om = O.Mesh(xyz * k, tri)
    ref = om.z_full(1.0, 4, mode="table", tables=O.make_tables(1.0, umin, umax)) / k ** 2
    assert _rel(Z.cpu().numpy(), ref) <= 1e-12


def test_one_table_for_a_sweep():
    xyz, tri = _mesh()
    m = gf.Mesh(xyz, tri)
    p = gf.gf_params_default(rule=6)
    lo, hi = m.range(6, gf.GF_FP32)
    ks = [1.5 * math.pi, 2 * math.pi, 3.3 * math.pi]
    tab = gf.Table.kr(min(ks) * lo * 0.99, max(ks) * hi * 1.01, p)
    for k in ks:
        own = gf.Table(k, lo, hi, p)
        for fill in ("efie", "mfie"):
            dt = torch.complex64
            Za = torch.empty((m.ne, m.ne), dtype=dt, device="cuda")
            Zb = torch.empty((m.ne, m.ne), dtype=dt, device="cuda")
            if fill == "efie":
                gf.gf_fill(m.h, k, p, tab.h, gf.GF_FP32, Za)
                gf.gf_fill(m.h, k, p, own.h, gf.GF_FP32, Zb)
            else:
                gf.gf_fill_mfie(m.h, k, p, tab.h, gf.GF_FP32, Za)
                gf.gf_fill_mfie(m.h, k, p, own.h, gf.GF_FP32, Zb)
            assert _rel(Za.cpu().numpy(), Zb.cpu().numpy()) <= 5e-6, (k, fill)
    # the sparse fill reads the same table
    sp = gf.Sparse(m, 0.3)
    k = ks[1]
    va = sp.fill(k, p, tab).cpu().numpy()
    vb = sp.fill(k, p, gf.Table(k, lo, hi, p)).cpu().numpy()
    assert _rel(va, vb) <= 5e-6


def test_batch_with_one_kr_table():
    rng = np.random.default_rng(31)
    wls = [W.uv_ellipsoid(a, b, c, nt, nph, rng) for a, b, c, nt, nph in
           ((0.6, 0.5, 0.7, 9, 14), (0.9, 0.6, 0.5, 11, 18), (0.5, 0.8, 0.6, 10, 16))]
    meshes = [gf.Mesh(x, t) for x, t in wls]
    ks = [1.2 * math.pi, 2.5 * math.pi, 3.4 * math.pi]
    p = gf.gf_params_default(rule=6)
    rngs = [m.range(6, gf.GF_FP32) for m in meshes]
    umin = min(k * lo for k, (lo, _) in zip(ks, rngs)) * 0.99
    umax = max(k * hi for k, (_, hi) in zip(ks, rngs)) * 1.01
    tkr = gf.Table.kr(umin, umax, p)
    own = [gf.Table(k, lo, hi, p) for k, (lo, hi) in zip(ks, rngs)]
    Za = [torch.empty((m.ne, m.ne), dtype=torch.complex64, device="cuda") for m in meshes]
    Zb = [torch.empty((m.ne, m.ne), dtype=torch.complex64, device="cuda") for m in meshes]
    ba = gf.Batch(meshes, ks, p, [tkr] * 3, Za, autotune=False)
    bb = gf.Batch(meshes, ks, p, own, Zb, autotune=False)
    ba.launch()
    bb.launch()
    torch.cuda.synchronize()
    for za, zb in zip(Za, Zb):
        assert _rel(za.cpu().numpy(), zb.cpu().numpy()) <= 5e-6


def test_backward_rejects_kr_table():
    xyz, tri = _mesh()
    m = gf.Mesh(xyz, tri)
    p = gf.gf_params_default(rule=3)
    tab = gf.Table.kr(0.01, 20.0, p)
    gZ = torch.zeros((m.ne, m.ne), dtype=torch.complex64, device="cuda")
    with pytest.raises(gf.GfError):
        gf.gf_fill_backward(m, 2 * math.pi, p, tab, gZ)

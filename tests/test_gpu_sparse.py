"""Near-field sparse fill (gf_fill_sparse): the pattern against its
definition, the values against the dense fill and the oracle."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1901_04162_gb300 as gf
import workloads as W

pytestmark = pytest.mark.gpu


def _pattern_brute(xyz, tri, ev, et, radius):
    cen = xyz[tri].mean(axis=1)
    ne = len(ev)
    c = cen[et]                                       # (ne, 2, 3)
    d = np.linalg.norm(c[:, None, :, None, :] - c[None, :, None, :, :], axis=-1)  # (ne, ne, 2, 2)
    return (d < radius).any(axis=(2, 3))


@pytest.mark.parametrize("radius", [0.25, 0.6])
def test_pattern_matches_definition(radius):
    xyz, tri = W.icosphere(2)
    xyz = W.jitter(xyz * 0.8, tri, 0.05, 4)
    m = gf.Mesh(xyz, tri)
    ev, et = m.edges()
    sp = gf.Sparse(m, radius)
    row_ptr, cols = sp.pattern()
    dense = np.zeros((m.ne, m.ne), dtype=bool)
    for r in range(m.ne):
        dense[r, cols[row_ptr[r]:row_ptr[r + 1]]] = True
        assert np.all(np.diff(cols[row_ptr[r]:row_ptr[r + 1]]) > 0)
    np.testing.assert_array_equal(dense, _pattern_brute(xyz, tri, ev, et, radius))


@pytest.mark.parametrize("table", [False, True])
def test_values_equal_dense_fill_and_oracle(table):
    wl = W.sphere_3072()
    m = gf.Mesh(wl.xyz, wl.tri)
    p = gf.gf_params_default(rule=wl.rule)
    tab = None
    if table:
        lo, hi = m.range(wl.rule, gf.GF_FP32)
        tab = gf.Table(wl.k, lo, hi, p)
    sp = gf.Sparse(m, 0.35)
    row_ptr, cols = sp.pattern()
    vals = sp.fill(wl.k, p, tab).cpu().numpy()
    rows = np.repeat(np.arange(m.ne), np.diff(row_ptr))
    Z = gf.fill(m, wl.k, p, tab, gf.GF_FP32).cpu().numpy()
    ref = Z[rows, cols]
    assert np.linalg.norm(vals - ref) <= 1e-6 * np.linalg.norm(ref)
    # against the oracle on sampled entries of the pattern
    om = O.Mesh(wl.xyz, wl.tri)
    pick = np.random.default_rng(3).choice(sp.nnz, 400, replace=False)
    kw = {}
    if table:
        olo, ohi = om.range(wl.rule)
        kw = {"mode": "table", "tables": O.make_tables(wl.k, olo, ohi)}
    zo = om.z_entries(wl.k, wl.rule, rows[pick], cols[pick], **kw)
    assert np.linalg.norm(vals[pick] - zo) <= 1e-5 * np.linalg.norm(zo)
    assert np.max(np.abs(vals[pick] - zo)) <= 1e-5 * np.max(np.abs(zo))


def test_radius_beyond_the_mesh_gives_the_dense_matrix():
    xyz, tri = W.icosphere(2)
    m = gf.Mesh(xyz * 0.5, tri)
    p = gf.gf_params_default(rule=4)
    sp = gf.Sparse(m, 10.0)
    assert sp.nnz == m.ne * m.ne
    vals = sp.fill(2 * math.pi, p).cpu().numpy().reshape(m.ne, m.ne)
    Z = gf.fill(m, 2 * math.pi, p, None, gf.GF_FP32).cpu().numpy()
    assert np.linalg.norm(vals - Z) <= 1e-6 * np.linalg.norm(Z)


def test_centroid_near_list_and_errors():
    wl = W.cube_73728(8)  # near pairs include centroids closer than 0.2 lambda
    m = gf.Mesh(wl.xyz, wl.tri, wl.near_dist)
    p = gf.gf_params_default(rule=wl.rule)
    sp = gf.Sparse(m, 0.5)
    row_ptr, cols = sp.pattern()
    vals = sp.fill(wl.k, p).cpu().numpy()
    rows = np.repeat(np.arange(m.ne), np.diff(row_ptr))
    Z = gf.fill(m, wl.k, p, None, gf.GF_FP32).cpu().numpy()
    ref = Z[rows, cols]
    assert np.linalg.norm(vals - ref) <= 1e-6 * np.linalg.norm(ref)
    with pytest.raises(gf.GfError):
        gf.Sparse(m, 0.0)

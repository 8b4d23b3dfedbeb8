"""GPU fill vs the FP64 oracle on the same seeded meshes: element-wise on
small meshes and on the 0.5 lambda plate (FP64, 1e-12), relative Frobenius
<= 1e-5 in FP32, sampled rows on the 7680-unknown sphere, and edge cases."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1901_04162_gb300 as gf
import workloads as W
from gpu_util import rel_fro, rel_max

pytestmark = pytest.mark.gpu
K = 2 * math.pi


def gpu_fill(xyz, tri, k, rule, precision, table=True, near_dist=0.0, **pk):
    m = gf.Mesh(xyz, tri, near_dist)
    p = gf.gf_params_default(rule=rule, **pk)
    tab = None
    if table:
        lo, hi = m.range(rule, precision)
        tab = gf.Table(k, lo, hi, p)
    z = gf.fill(m, k, p, tab, precision).cpu().numpy()
    return m, z, tab


def oracle_full(xyz, tri, k, rule, table=True, near_dist=0.0, **kw):
    om = O.Mesh(xyz, tri, near_dist)
    if table:
        lo, hi = om.range(rule)
        return om.z_full(k, rule, mode="table", tables=O.make_tables(k, lo, hi), **kw)
    return om.z_full(k, rule, **kw)


@pytest.mark.parametrize("table", [False, True])
def test_plate_fp64_matches_oracle(table):
    wl = W.plate_280()
    m, z, _ = gpu_fill(wl.xyz, wl.tri, wl.k, 3, gf.GF_FP64, table)
    ref = oracle_full(wl.xyz, wl.tri, wl.k, 3, table)
    assert m.ne == 280
    assert rel_fro(z, ref) <= 1e-12
    assert rel_max(z, ref) <= 1e-12


@pytest.mark.parametrize("rule", [3, 4, 6, 7])
@pytest.mark.parametrize("table", [False, True])
@pytest.mark.parametrize("near_fp64", [0, 1])
def test_small_sphere_fp32_matches_oracle(rule, table, near_fp64):
    xyz, tri = W.octasphere(2, 1.0)
    xyz = W.jitter(xyz, tri, 0.02, 3)
    _, z, _ = gpu_fill(xyz, tri, K, rule, gf.GF_FP32, table, near_fp64=near_fp64)
    ref = oracle_full(xyz, tri, K, rule, table)
    assert rel_fro(z, ref) <= 1e-5
    assert rel_max(z, ref) <= 1e-5


def test_small_sphere_fp64_both_modes():
    xyz, tri = W.icosphere(1, 0.7)
    for table in (False, True):
        _, z, _ = gpu_fill(xyz, tri, K, 6, gf.GF_FP64, table)
        ref = oracle_full(xyz, tri, K, 6, table)
        assert rel_fro(z, ref) <= 1e-12


@pytest.mark.parametrize("rule", [4, 7])
@pytest.mark.parametrize("entries", [None, "2100", "0"])
def test_fp32_coarse_table_corrections_match_oracle(rule, entries, monkeypatch):
    # A coarse Green table (tol 1e-2, 10 samples per wavelength): nearly every
    # lattice cell holds samples whose polynomials disagree, or needs its
    # cubic term, so nearly every point pair takes the exact correction, and
    # a lost or wrong correction shows at the scale of the left-out cubic
    # terms (1e-4 of Z), ten times the bound. entries: the flagged-pair list
    # as sized for the table (corrections kernel); too small for any CTA
    # (each scans its tasks again); none (corrections in the pair kernel).
    if entries is not None:
        monkeypatch.setenv("GF_FIX_ENTRIES", entries)
    xyz, tri = W.octasphere(2, 1.0)
    xyz = W.jitter(xyz, tri, 0.02, 3)
    _, z, _ = gpu_fill(xyz, tri, K, rule, gf.GF_FP32, True, table_tol=1e-2, green_n_per_lambda=10)
    om = O.Mesh(xyz, tri)
    lo, hi = om.range(rule)
    tabs = (O.Table(O.table_params(O.GREEN, K, lo, hi, tol=1e-2, n_per_lambda=10)),
            O.Table(O.table_params(O.EXP, K, lo, hi, tol=1e-2)))
    ref = om.z_full(K, rule, mode="table", tables=tabs)
    direct = om.z_full(K, rule)
    assert rel_fro(ref, direct) > 3e-5  # the coarse table's own error, which the corrections carry
    assert rel_fro(z, ref) <= 1e-5 and rel_max(z, ref) <= 1e-5


def test_green_from_exp_matches_oracle():
    # regular pairs through the linear Exp table times 1/R (green_from_exp = 1)
    # against the oracle's "exp_over_r" mode: FP64 plate element-wise at 1e-12,
    # FP32 jittered sphere (smem lattice of the Exp table) at 1e-5
    wl = W.plate_280()
    _, z, _ = gpu_fill(wl.xyz, wl.tri, wl.k, 3, gf.GF_FP64, True, green_from_exp=1)
    om = O.Mesh(wl.xyz, wl.tri)
    lo, hi = om.range(3)
    ref = om.z_full(wl.k, 3, mode="exp_over_r", tables=O.make_tables(wl.k, lo, hi))
    assert rel_fro(z, ref) <= 1e-12 and rel_max(z, ref) <= 1e-12
    xyz, tri = W.octasphere(2, 1.0)
    xyz = W.jitter(xyz, tri, 0.02, 3)
    for rule in (4, 7):
        _, z, _ = gpu_fill(xyz, tri, K, rule, gf.GF_FP32, True, green_from_exp=1)
        om = O.Mesh(xyz, tri)
        lo, hi = om.range(rule)
        ref = om.z_full(K, rule, mode="exp_over_r", tables=O.make_tables(K, lo, hi))
        assert rel_fro(z, ref) <= 1e-5 and rel_max(z, ref) <= 1e-5


@pytest.mark.parametrize("which", ["plate", "sphere", "cube", "cube16"])
def test_range_matches_oracle(which):
    # cube16: 3072 triangles in 96 blocks with the centroid criterion, where
    # most block pairs are skipped after the first-threshold pass
    wl = {"plate": W.plate_280, "sphere": W.sphere_3072, "cube": lambda: W.cube_73728(6),
          "cube16": lambda: W.cube_73728(16)}[which]()
    m = gf.Mesh(wl.xyz, wl.tri, wl.near_dist)
    om = O.Mesh(wl.xyz, wl.tri, wl.near_dist)
    for rule in ((4,) if which == "cube16" else (3, 7)):
        lo, hi = om.range(rule)
        g64 = m.range(rule, gf.GF_FP64)
        g32 = m.range(rule, gf.GF_FP32)
        assert abs(g64[0] - lo) <= 1e-14 * lo and abs(g64[1] - hi) <= 1e-14 * hi
        assert abs(g32[0] - lo) <= 1e-6 * lo and abs(g32[1] - hi) <= 1e-6 * hi
        assert m.range(rule, gf.GF_FP32) == g32  # independent of the order the device evaluates in


def test_near_dist_criterion_matches_oracle():
    wl = W.cube_73728(3)
    _, z, _ = gpu_fill(wl.xyz, wl.tri, wl.k, 4, gf.GF_FP64, True, near_dist=0.6)
    ref = oracle_full(wl.xyz, wl.tri, wl.k, 4, True, near_dist=0.6)
    assert rel_fro(z, ref) <= 1e-12


@pytest.mark.parametrize("rule", [4, 7])
def test_near_dist_fp32_matches_oracle(rule):
    # FP32 fill of a mesh with a centroid criterion (near pairs that share no
    # vertex, up to 0.6 lambda apart): mixed-precision near pairs against the
    # oracle and against FP64 near pairs (near_fp64 = 1)
    wl = W.cube_73728(3)
    _, z, _ = gpu_fill(wl.xyz, wl.tri, wl.k, rule, gf.GF_FP32, True, near_dist=0.6)
    _, z64, _ = gpu_fill(wl.xyz, wl.tri, wl.k, rule, gf.GF_FP32, True, near_dist=0.6, near_fp64=1)
    ref = oracle_full(wl.xyz, wl.tri, wl.k, rule, True, near_dist=0.6)
    assert rel_fro(z, ref) <= 1e-5 and rel_max(z, ref) <= 1e-5
    assert rel_fro(z, z64) <= 1e-5


@pytest.mark.parametrize("near_fp64", [0, 1])
def test_sphere_7680_sampled_rows(near_fp64):
    wl = W.sphere_7680()
    m, z, tab = gpu_fill(wl.xyz, wl.tri, wl.k, 7, gf.GF_FP32, True, near_fp64=near_fp64)
    om = O.Mesh(wl.xyz, wl.tri)
    lo, hi = om.range(7)
    rows = np.random.default_rng(11).choice(m.ne, 12, replace=False)
    ref = om.z_rows(wl.k, 7, rows, mode="table", tables=O.make_tables(wl.k, lo, hi))
    assert rel_fro(z[rows], ref) <= 1e-5
    # the diagonal blocks (self and near terms) of the sampled rows
    assert rel_max(z[rows, rows], ref[np.arange(len(rows)), rows]) <= 1e-5


def test_ldz_padding_untouched_and_open_plate():
    xyz, tri = W.plate(0.3, 4)
    m = gf.Mesh(xyz, tri)
    ev, et = m.edges()
    assert m.ne == 40  # interior edges of a 4 x 4 split-square plate
    p = gf.gf_params_default(rule=3)
    lo, hi = m.range(3, gf.GF_FP64)
    tab = gf.Table(K, lo, hi, p)
    Z = torch.full((m.ne, m.ne + 5), 7.0 + 7.0j, dtype=torch.complex128, device="cuda")
    gf.gf_fill(m.h, K, p, tab.h, gf.GF_FP64, Z, ldz=m.ne + 5)
    Zc = Z.cpu().numpy()
    assert np.all(Zc[:, m.ne:] == 7.0 + 7.0j)
    ref = oracle_full(xyz, tri, K, 3, True)
    assert rel_fro(Zc[:, :m.ne], ref) <= 1e-12


def test_errors():
    xyz, tri = W.plate(0.1, 1)  # two triangles: every pair is near
    m = gf.Mesh(xyz, tri)
    with pytest.raises(gf.GfError):
        m.range(3)
    z = gf.fill(m, K, gf.gf_params_default(rule=3), None, gf.GF_FP64).cpu().numpy()
    ref = oracle_full(xyz, tri, K, 3, False)
    assert rel_fro(z, ref) <= 1e-12
    with pytest.raises(gf.GfError):
        gf.Mesh(np.zeros((4, 3)), np.array([[0, 1, 2], [0, 1, 3], [1, 0, 3]], np.int32))
    with pytest.raises(ValueError):
        gf.gf_fill(m.h, K, gf.gf_params_default(), None, gf.GF_FP32, torch.zeros(1, 1, dtype=torch.complex128,
                                                                                   device="cuda"))
    t = gf.Table(K, 0.1, 1.0)
    with pytest.raises(gf.GfError):  # table built for another k
        gf.fill(m, 2 * K, gf.gf_params_default(rule=3), t, gf.GF_FP64)


def test_mesh_edges_and_near_count_match_oracle():
    # RWG numbering (sorted vertex pairs, T+ = the first triangle in input
    # order) and the number of ordered near pairs, on meshes with and without
    # a centroid criterion
    for wl in (W.plate_280(), W.sphere_3072(), W.cube_73728(8)):
        m = gf.Mesh(wl.xyz, wl.tri, wl.near_dist)
        om = O.Mesh(wl.xyz, wl.tri, wl.near_dist)
        ev, et = m.edges()
        oev, oet = om.edges()
        np.testing.assert_array_equal(ev, oev)
        np.testing.assert_array_equal(et, oet)
        nt = len(wl.tri)
        if nt <= 1000:
            assert m.n_near == sum(om.is_near(p, q) for p in range(nt) for q in range(nt))


def test_near_count_large_mesh_brute_force():
    # 12288 triangles with the centroid criterion: the near rows are built on
    # several host threads from a cell-sorted centroid array; their number
    # equals a brute-force count of the ordered pairs that share a vertex or
    # whose centroids are closer than near_dist (distance compared as the
    # library and the oracle do, sqrt(d2) < near_dist)
    sp = pytest.importorskip("scipy.sparse")
    wl = W.cube_73728(32)
    m = gf.Mesh(wl.xyz, wl.tri, wl.near_dist)
    tri = np.asarray(wl.tri)
    cen = wl.xyz[tri].mean(axis=1)
    nt = len(tri)
    inc = sp.csr_matrix((np.ones(3 * nt), (np.repeat(np.arange(nt), 3), tri.ravel())), shape=(nt, len(wl.xyz)))
    near = (inc @ inc.T).tocsr()  # pairs sharing a vertex (self included)
    rows, cols = [], []
    for a0 in range(0, nt, 1024):  # centroid distances by brute force
        d = np.sqrt(((cen[a0:a0 + 1024, None, :] - cen[None, :, :]) ** 2).sum(-1))
        r, c = np.nonzero(d < wl.near_dist)
        rows.append(r + a0)
        cols.append(c)
    r, c = np.concatenate(rows), np.concatenate(cols)
    near = near + sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(nt, nt))
    assert m.n_near == near.nnz


@pytest.mark.parametrize("table", [False, True])
def test_fp32_parts_padding_and_ragged_tiles(table):
    # 280 unknowns: nine 32 x 32 tiles, the last ragged. The FP32 fill through
    # a padded leading dimension leaves the padding alone and matches the
    # oracle; the regular part alone is symmetric (Galerkin), and ZERO +
    # REGULAR followed by NEAR in a second call gives gf_fill's matrix
    wl = W.plate_280()
    m = gf.Mesh(wl.xyz, wl.tri)
    p = gf.gf_params_default(rule=3)
    tab = None
    if table:
        lo, hi = m.range(3, gf.GF_FP32)
        tab = gf.Table(wl.k, lo, hi, p)
    th = tab.h if tab else None
    Z = torch.full((m.ne, m.ne + 5), 3.0 - 1.0j, dtype=torch.complex64, device="cuda")
    gf.gf_fill(m.h, wl.k, p, th, gf.GF_FP32, Z, ldz=m.ne + 5)
    Zc = Z.cpu().numpy()
    assert np.all(Zc[:, m.ne:] == 3.0 - 1.0j)
    ref = oracle_full(wl.xyz, wl.tri, wl.k, 3, table)
    assert rel_fro(Zc[:, :m.ne], ref) <= 1e-5 and rel_max(Zc[:, :m.ne], ref) <= 1e-5
    R = torch.empty((m.ne, m.ne), dtype=torch.complex64, device="cuda")
    gf.gf_fill_parts(m.h, wl.k, p, th, gf.GF_FP32, R, gf.GF_PART_ZERO | gf.GF_PART_REGULAR)
    r = R.cpu().numpy()
    assert np.abs(r).max() > 0
    assert np.array_equal(r, r.T)  # Z + Z^T of the pair kernel's half, both entries from the same two floats
    # the regular stage as its two halves: the pair kernel fills one triangle's rows per pair
    gf.gf_fill_parts(m.h, wl.k, p, th, gf.GF_FP32, R, gf.GF_PART_ZERO | gf.GF_PART_PAIRS)
    half = R.cpu().numpy()
    assert np.linalg.norm(half - half.T) > 0.1 * np.linalg.norm(half)
    assert rel_fro(half + half.T, r) <= 1e-6
    gf.gf_fill_parts(m.h, wl.k, p, th, gf.GF_FP32, R, gf.GF_PART_MIRROR)
    gf.gf_fill_parts(m.h, wl.k, p, th, gf.GF_FP32, R, gf.GF_PART_NEAR)
    assert rel_fro(R.cpu().numpy(), Zc[:, :m.ne]) <= 1e-6
    with pytest.raises(gf.GfError):
        gf.gf_fill_parts(m.h, wl.k, p, th, gf.GF_FP32, R, 32)

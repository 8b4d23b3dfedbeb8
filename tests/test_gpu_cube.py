"""The 3 lambda cube (49152 triangles, 73728 RWG unknowns, 4-point rule,
near pairs = shared vertex or centroids closer than 0.2 lambda, complex64 Z
of 43.5 GB) against the FP64 oracle on 64 seeded 256 x 256 blocks and on all
288 diagonal blocks, with the Green table and with direct evaluation."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1901_04162_gb300 as gf
import workloads as W
from gpu_util import entry_rel_max, rel_fro, rel_max

pytestmark = pytest.mark.gpu
BS = 256


def blocks_of(ne):
    nb = ne // BS
    rng = np.random.default_rng(64)
    rand = list(zip(rng.integers(nb, size=64).tolist(), rng.integers(nb, size=64).tolist()))
    diag = [(i, i) for i in range(nb)]
    return rand, diag


def gather(Z, blocks):
    return np.stack([Z[i * BS:(i + 1) * BS, j * BS:(j + 1) * BS].cpu().numpy() for i, j in blocks])


def oracle_blocks(om, k, blocks, **kw):
    ii = np.arange(BS)
    mi = np.concatenate([np.repeat(i * BS + ii, BS) for i, _ in blocks])
    ni = np.concatenate([np.tile(j * BS + ii, BS) for _, j in blocks])
    return om.z_entries(k, 4, mi, ni, **kw).reshape(len(blocks), BS, BS)


@pytest.fixture(scope="module")
def cube():
    wl = W.cube_73728()
    m = gf.Mesh(wl.xyz, wl.tri, wl.near_dist)
    assert m.ne == 73728 and m.nt == 49152
    om = O.Mesh(wl.xyz, wl.tri, wl.near_dist)
    lo, hi = m.range(4, gf.GF_FP32)
    olo, ohi = om.range(4, prune=True)
    assert abs(lo - olo) <= 1e-6 * olo and abs(hi - ohi) <= 1e-6 * ohi
    return wl, m, om, (lo, hi), (olo, ohi)


@pytest.mark.parametrize("mode", ["table", "direct"])
def test_cube_73728_blocks(cube, mode):
    wl, m, om, (lo, hi), (olo, ohi) = cube
    p = gf.gf_params_default(rule=4)
    tab = gf.Table(wl.k, lo, hi, p) if mode == "table" else None
    rand, diag = blocks_of(m.ne)
    Z = torch.empty((m.ne, m.ne), dtype=torch.complex64, device="cuda")
    gf.gf_fill(m.h, wl.k, p, tab.h if tab else None, gf.GF_FP32, Z)
    zr, zd = gather(Z, rand), gather(Z, diag)
    del Z
    torch.cuda.empty_cache()
    kw = {"mode": "table", "tables": O.make_tables(wl.k, olo, ohi)} if mode == "table" else {}
    rr, rd = oracle_blocks(om, wl.k, rand, **kw), oracle_blocks(om, wl.k, diag, **kw)
    both_z, both_r = np.concatenate([zr, zd]), np.concatenate([rr, rd])
    # the union (the diagonal blocks hold the near pairs) and the random blocks
    # alone (mostly far entries, where the FP32 phase of kR used to limit the
    # accuracy) each within the relative Frobenius bound of the FP32 fill
    assert rel_fro(both_z, both_r) <= 1e-5
    assert rel_fro(zr, rr) <= 1e-5
    assert rel_max(both_z, both_r) <= 1e-5
    # entries of at least 1 % of the largest: element-wise relative error
    assert entry_rel_max(both_z, both_r, 1e-2) <= 2e-4

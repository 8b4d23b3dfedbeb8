"""The allocation-free range entry point (gf_range_noalloc) against gf_range.

gf_range_noalloc serves callers that cannot allocate device memory; it keeps
its scratch in a fixed array inside the library. This file is collected last
so that a run stopping at the first failure has already run every other test.
"""
import math

import numpy as np
import pytest
import torch

import paper_1901_04162_gb300 as gf
import workloads as W
from paper_1901_04162_gb300 import gfmom

pytestmark = pytest.mark.gpu


def device_inputs(xyz, tri):
    tri_xyz = torch.from_numpy(np.ascontiguousarray(xyz[tri].reshape(len(tri), 9))).cuda()
    tri_vert = torch.from_numpy(np.ascontiguousarray(tri, dtype=np.int32)).cuda()
    return tri_xyz, tri_vert


def test_noalloc_range_matches_gf_range_twice():
    # two calls in a row, larger mesh first: the second result must not see the
    # first call's scratch contents
    cases = [(W.sphere_7680(), 7), (W.plate_280(), 3)]
    for wl, rule in cases:
        m = gf.Mesh(wl.xyz, wl.tri)
        ref = m.range(rule, gf.GF_FP64)
        tri_xyz, tri_vert = device_inputs(wl.xyz, wl.tri)
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        gfmom.gf_range_noalloc(tri_xyz, tri_vert, rule, out)
        torch.cuda.synchronize()
        lo, hi = out.cpu().tolist()
        assert abs(lo - ref[0]) <= 1e-14 * ref[0], (wl.name, lo, ref[0])
        assert abs(hi - ref[1]) <= 1e-14 * ref[1], (wl.name, hi, ref[1])


def test_noalloc_range_rejects_oversize():
    xyz, tri = W.plate(0.3, 2)
    tri_xyz, tri_vert = device_inputs(xyz, tri)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    L = gf.lib()
    big = gfmom.GF_NOALLOC_MAX_POINTS // 7 + 1  # nt * 7 just above the cap; nothing is read
    st = L.gf_range_noalloc(tri_xyz.data_ptr(), tri_vert.data_ptr(), big, 7, out.data_ptr(), None)
    assert st == -1 and "GF_NOALLOC_MAX_POINTS" in gf.gf_last_error()

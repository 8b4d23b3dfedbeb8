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


def test_noalloc_all_pairs_near_gives_empty_range():
    # a fan of six triangles around one vertex: every pair shares it, so no
    # pair is regular and the result is (+inf, 0) (gf_range reports an error)
    ang = np.linspace(0, 2 * math.pi, 7)[:-1]
    xyz = np.vstack([[0.0, 0.0, 0.0], np.stack([np.cos(ang), np.sin(ang), np.zeros(6)], 1) * 0.1])
    tri = np.array([[0, 1 + i, 1 + (i + 1) % 6] for i in range(6)], dtype=np.int32)
    tri_xyz, tri_vert = device_inputs(xyz, tri)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    gfmom.gf_range_noalloc(tri_xyz, tri_vert, 3, out)
    torch.cuda.synchronize()
    lo, hi = out.cpu().tolist()
    assert lo == math.inf and hi == 0.0
    with pytest.raises(gf.GfError):
        gf.Mesh(xyz, tri).range(3, gf.GF_FP64)


def test_noalloc_ignores_centroid_criterion_brute_force():
    # a mesh with a centroid near criterion (cube of side 3 lambda, 16 x 16
    # squares per face, near = centroids closer than 0.2 lambda): gf_range
    # leaves those pairs out, the allocation-free reduction counts every
    # vertex-disjoint pair; checked against a brute-force FP64 minimum and
    # maximum over those pairs
    import oracle as O
    wl = W.cube_73728(16)
    bary, _ = O.rule(4)
    pts = np.einsum("pi,tij->tpj", bary, wl.xyz[wl.tri])
    nt = len(wl.tri)
    lo_ref, hi_ref = math.inf, 0.0
    for a0 in range(0, nt, 256):
        t = wl.tri[a0:a0 + 256]
        share = (t[:, None, :, None] == wl.tri[None, :, None, :]).any(axis=(2, 3))
        d = np.linalg.norm(pts[a0:a0 + 256, None, :, None, :] - pts[None, :, None, :, :], axis=-1)
        d = d.reshape(len(t), nt, -1)[~share]
        lo_ref, hi_ref = min(lo_ref, d.min()), max(hi_ref, d.max())
    tri_xyz, tri_vert = device_inputs(wl.xyz, wl.tri)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    gfmom.gf_range_noalloc(tri_xyz, tri_vert, 4, out)
    torch.cuda.synchronize()
    lo, hi = out.cpu().tolist()
    assert abs(lo - lo_ref) <= 1e-14 * lo_ref and abs(hi - hi_ref) <= 1e-14 * hi_ref
    glo, _ = gf.Mesh(wl.xyz, wl.tri, wl.near_dist).range(4, gf.GF_FP64)
    assert glo > lo  # the centroid criterion removed the closest vertex-disjoint pairs


RESET_SCRIPT = r"""
import ctypes, math, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_1901_04162_gb300 as gf
import workloads as W
L = gf.lib()
rt = ctypes.CDLL("libcudart.so.13")  # the runtime the library links
def run(xyz, tri, rule):
    a = np.ascontiguousarray(xyz[tri].reshape(len(tri), 9))
    v = np.ascontiguousarray(tri, dtype=np.int32)
    ptrs = []
    for host in (a, v, np.zeros(2)):
        p = ctypes.c_void_p()
        assert rt.cudaMalloc(ctypes.byref(p), ctypes.c_size_t(host.nbytes)) == 0
        assert rt.cudaMemcpy(p, host.ctypes.data, ctypes.c_size_t(host.nbytes), 1) == 0
        ptrs.append(p)
    st = L.gf_range_noalloc(ptrs[0], ptrs[1], len(tri), rule, ptrs[2], None)
    assert st == 0, L.gf_last_error()
    out = np.zeros(2)
    assert rt.cudaMemcpy(out.ctypes.data, ptrs[2], ctypes.c_size_t(16), 2) == 0
    for p in ptrs:
        rt.cudaFree(p)
    return out
wl = W.plate_280()
first = run(wl.xyz, wl.tri, 3)
assert rt.cudaDeviceReset() == 0
second = run(wl.xyz, wl.tri, 3)
assert np.array_equal(first, second) and 0 < first[0] < first[1] < math.inf, (first, second)
print("ok", first[0], first[1])
"""


def test_noalloc_after_device_reset():
    # a device reset ends the context the scratch address was taken in; the
    # next call looks it up again (run in a process of its own, without torch)
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", RESET_SCRIPT, root], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr

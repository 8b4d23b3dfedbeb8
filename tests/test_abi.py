"""CPU checks of the C-ABI library: it builds, loads and exports every symbol
the public header declares; argument validation that needs no GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1901_04162_gb300 as gf
from paper_1901_04162_gb300 import gfmom

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "gfmom.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:gf_status|void|const char\*)\s+(gf_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_header_symbol():
    L = gf.lib()
    names = header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    assert sorted(gfmom.EXPORTS) == names


def test_params_default_values():
    p = gf.gf_params_default()
    assert p.rule == 3 and p.table_tol == 1e-6 and p.green_n_per_lambda == 1000
    assert p.exp_n_per_lambda == 0 and p.lagrange_degree == 3 and p.refine == 1
    assert p.refine_factor == 0.5 and p.refine_halfwidth_t == 2.0 and p.merge_t == 0.25
    assert p.grade == 1 and p.nphi == 8 and p.nl == 8 and p.eta == 376.730313668 and p.near_fp64 == 0
    assert p.green_from_exp == 0


def test_argument_errors_before_any_device_call():
    L = gf.lib()
    h = C.c_void_p()
    xyz = np.zeros((3, 3))
    tri = np.array([[0, 1, 2]], np.int32)
    assert L.gf_mesh_create(None, 3, tri.ctypes.data, 1, 0.0, C.byref(h)) == -1
    assert L.gf_mesh_create(xyz.ctypes.data, 2, tri.ctypes.data, 1, 0.0, C.byref(h)) == -1
    assert L.gf_mesh_create(xyz.ctypes.data, 3, tri.ctypes.data, 1, -1.0, C.byref(h)) == -1
    assert "gf_mesh_create" in gf.gf_last_error()
    bad = np.array([[0, 0, 0], [1, 0, 0], [np.nan, 0, 0]])
    assert L.gf_mesh_create(bad.ctypes.data, 3, tri.ctypes.data, 1, 0.0, C.byref(h)) == -2
    p = gf.gf_params_default()
    assert L.gf_table_create(0.0, 0.1, 1.0, C.byref(p), None, C.byref(h)) == -1
    assert L.gf_table_create(1.0, 0.5, 0.1, C.byref(p), None, C.byref(h)) == -1
    p.nphi = 0
    assert L.gf_table_create(1.0, 0.1, 1.0, C.byref(p), None, C.byref(h)) == -1
    p = gf.gf_params_default()
    p.green_from_exp = 2
    assert L.gf_table_create(1.0, 0.1, 1.0, C.byref(p), None, C.byref(h)) == -1
    assert L.gf_fill(None, 1.0, C.byref(p), None, 32, None, 10, None) == -1
    assert L.gf_table_destroy(None) == 0 and L.gf_mesh_destroy(None) == 0
    with pytest.raises(gf.GfError):
        gf.gf_table_create(-1.0, 0.1, 1.0)


def test_scattering_argument_errors_before_any_device_call():
    L = gf.lib()
    p = gf.gf_params_default()
    one = C.c_double(1.0)
    fake = C.c_void_p(1)  # never dereferenced: the argument checks come first
    kh = np.array([2.0, 0.0, 0.0])
    pol = np.zeros((3, 2))
    v = C.c_void_p(8)
    assert L.gf_excitation(None, one, C.byref(p), kh.ctypes.data, pol.ctypes.data, 0, 32, v, None) == -1
    assert L.gf_excitation(fake, one, C.byref(p), kh.ctypes.data, pol.ctypes.data, 0, 32, v, None) == -1  # |khat| != 1
    kh[0] = 1.0
    assert L.gf_excitation(fake, one, C.byref(p), kh.ctypes.data, pol.ctypes.data, 0, 7, v, None) == -1
    assert L.gf_excitation(fake, C.c_double(-1.0), C.byref(p), kh.ctypes.data, pol.ctypes.data, 0, 32, v, None) == -1
    assert L.gf_excitation(fake, one, C.byref(p), kh.ctypes.data, pol.ctypes.data, 5, 32, v, None) == -1  # operator
    d = C.c_void_p(16)
    assert L.gf_far_field(fake, one, C.byref(p), 32, v, C.c_int64(-1), d, d, d, None) == -1
    assert L.gf_far_field(fake, one, C.byref(p), 7, v, C.c_int64(3), d, d, d, None) == -1
    assert L.gf_far_field(None, one, C.byref(p), 32, v, C.c_int64(3), d, d, d, None) == -1

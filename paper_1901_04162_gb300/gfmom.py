"""Thin ctypes binding of libgfmom (include/gfmom.h), same names as the C ABI.

Argument marshalling only: every step of the fill runs in the library
(host-side topology and table sample placement in C++, everything else in
sm_103a kernels). PyTorch supplies device memory and streams. There is no
fallback: if the library cannot be built or loaded, or a call fails, an
exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

GF_OK = 0
GF_FP32, GF_FP64 = 32, 64
GF_GREEN, GF_EXP = 1, 0
_STATUS = {-1: "GF_ERR_ARG", -2: "GF_ERR_MESH", -3: "GF_ERR_RANGE", -4: "GF_ERR_CUDA", -5: "GF_ERR_ALLOC",
           -6: "GF_ERR_DEVICE"}

EXPORTS = ["gf_params_default", "gf_last_error", "gf_mesh_create", "gf_mesh_info", "gf_mesh_edges",
           "gf_mesh_set_vertices", "gf_mesh_destroy", "gf_range", "gf_table_create", "gf_table_info",
           "gf_table_nodes", "gf_table_eval", "gf_table_destroy", "gf_fill", "gf_fill_parts", "gf_range_noalloc", "gf_batch_create", "gf_batch_launch",
           "gf_batch_config", "gf_batch_destroy", "gf_fill_backward", "gf_excitation", "gf_far_field",
           "gf_fill_mfie", "gf_sparse_create", "gf_sparse_info", "gf_sparse_pattern", "gf_fill_sparse",
           "gf_sparse_destroy", "gf_table_create_kr", "gf_table_eval_host", "gf_table_create_for_mesh",
           "gf_fill_batched"]
GF_NOALLOC_MAX_POINTS = 131072
GF_PART_ZERO, GF_PART_REGULAR, GF_PART_NEAR, GF_PART_PAIRS, GF_PART_MIRROR = 1, 2, 4, 8, 16


class GfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class gf_params(C.Structure):
    _fields_ = [("rule", C.c_int), ("table_tol", C.c_double), ("green_n_per_lambda", C.c_int),
                ("exp_n_per_lambda", C.c_int), ("lagrange_degree", C.c_int), ("refine", C.c_int),
                ("refine_factor", C.c_double), ("refine_halfwidth_t", C.c_double), ("merge_t", C.c_double),
                ("grade", C.c_int), ("nphi", C.c_int), ("nl", C.c_int), ("eta", C.c_double),
                ("near_fp64", C.c_int), ("green_from_exp", C.c_int)]


_lib = None


def lib_path():
    return _build.LIB


def lib():
    """Loads (building first if missing or stale) the in-tree libgfmom.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i64, dp = C.c_void_p, C.c_int64, C.POINTER(C.c_double)
        L.gf_params_default.argtypes = [C.POINTER(gf_params)]
        L.gf_params_default.restype = None
        L.gf_last_error.restype = C.c_char_p
        L.gf_mesh_create.argtypes = [vp, i64, vp, i64, C.c_double, C.POINTER(vp)]
        L.gf_mesh_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
        L.gf_mesh_edges.argtypes = [vp, vp, vp]
        L.gf_mesh_set_vertices.argtypes = [vp, vp]
        L.gf_mesh_destroy.argtypes = [vp]
        L.gf_range.argtypes = [vp, C.c_int, C.c_int, dp, dp, vp]
        L.gf_table_create.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(gf_params), vp, C.POINTER(vp)]
        L.gf_table_info.argtypes = [vp, C.c_int, C.POINTER(i64), C.POINTER(i64), dp]
        L.gf_table_nodes.argtypes = [vp, C.c_int, vp, vp, vp, vp]
        L.gf_table_eval.argtypes = [vp, C.c_int, C.c_int, vp, i64, vp, vp]
        L.gf_table_eval_host.argtypes = [vp, C.c_int, vp, i64, vp]
        L.gf_table_create_for_mesh.argtypes = [vp, C.c_double, C.POINTER(gf_params), C.c_int, C.c_double, C.c_double,
                                               vp, C.POINTER(vp)]
        L.gf_fill_batched.argtypes = [C.c_int, vp, vp, C.POINTER(gf_params), vp, vp, vp, vp]
        L.gf_table_destroy.argtypes = [vp]
        L.gf_fill.argtypes = [vp, C.c_double, C.POINTER(gf_params), vp, C.c_int, vp, i64, vp]
        L.gf_fill_parts.argtypes = [vp, C.c_double, C.POINTER(gf_params), vp, C.c_int, vp, i64, C.c_uint, vp]
        L.gf_range_noalloc.argtypes = [vp, vp, i64, C.c_int, vp, vp]
        L.gf_batch_create.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(C.c_double), C.POINTER(gf_params),
                                      C.POINTER(vp), C.c_int, C.POINTER(vp), C.POINTER(i64), C.c_int, vp,
                                      C.POINTER(vp)]
        L.gf_batch_launch.argtypes = [vp, vp]
        L.gf_batch_config.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), dp]
        L.gf_batch_destroy.argtypes = [vp]
        L.gf_fill_backward.argtypes = [vp, C.c_double, C.POINTER(gf_params), vp, C.c_int, vp, i64, vp, vp, vp]
        L.gf_excitation.argtypes = [vp, C.c_double, C.POINTER(gf_params), vp, vp, C.c_int, C.c_int, vp, vp]
        L.gf_fill_mfie.argtypes = [vp, C.c_double, C.POINTER(gf_params), vp, C.c_int, vp, i64, vp]
        L.gf_sparse_create.argtypes = [vp, C.c_double, C.POINTER(vp)]
        L.gf_sparse_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
        L.gf_sparse_pattern.argtypes = [vp, vp, vp]
        L.gf_fill_sparse.argtypes = [vp, C.c_double, C.POINTER(gf_params), vp, C.c_int, vp, vp]
        L.gf_sparse_destroy.argtypes = [vp]
        L.gf_table_create_kr.argtypes = [C.c_double, C.c_double, C.POINTER(gf_params), vp, C.POINTER(vp)]
        L.gf_far_field.argtypes = [vp, C.c_double, C.POINTER(gf_params), C.c_int, vp, i64, vp, vp, vp, vp]
        for name in EXPORTS:
            if name not in ("gf_params_default", "gf_last_error"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(st):
    if st != GF_OK:
        raise GfError(st, lib().gf_last_error().decode())


def _ptr(a):
    return None if a is None else a.ctypes.data


_torch_cuda = None  # torch.cuda if torch with CUDA is importable, else False (checked once)


def _stream_ptr(stream):
    global _torch_cuda
    if stream is None:
        if _torch_cuda is None:
            try:
                import torch
                _torch_cuda = torch.cuda if torch.cuda.is_available() else False
            except ImportError:
                _torch_cuda = False
        if _torch_cuda:
            return C.c_void_p(_torch_cuda.current_stream().cuda_stream)
        return None
    return C.c_void_p(getattr(stream, "cuda_stream", stream))


# ----------------------------------------------------------------------------
# C-ABI mirrors
# ----------------------------------------------------------------------------
def gf_params_default(**overrides) -> gf_params:
    p = gf_params()
    lib().gf_params_default(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def gf_last_error() -> str:
    return lib().gf_last_error().decode()


def gf_mesh_create(xyz, tri, near_dist=0.0):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    if xyz.ndim != 2 or xyz.shape[1] != 3 or tri.ndim != 2 or tri.shape[1] != 3:
        raise ValueError("xyz must be [nv,3] and tri [nt,3]")
    h = C.c_void_p()
    _check(lib().gf_mesh_create(_ptr(xyz), len(xyz), _ptr(tri), len(tri), float(near_dist), C.byref(h)))
    return h


def gf_mesh_info(h):
    out = [C.c_int64() for _ in range(4)]
    _check(lib().gf_mesh_info(h, *[C.byref(o) for o in out]))
    return tuple(o.value for o in out)


def gf_mesh_edges(h):
    ne = gf_mesh_info(h)[2]
    ev = np.zeros((ne, 2), np.int32)
    et = np.zeros((ne, 2), np.int32)
    _check(lib().gf_mesh_edges(h, _ptr(ev), _ptr(et)))
    return ev, et


def gf_mesh_set_vertices(h, xyz):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    _check(lib().gf_mesh_set_vertices(h, _ptr(xyz)))


def gf_mesh_destroy(h):
    _check(lib().gf_mesh_destroy(h))


def gf_range(h, rule, precision=GF_FP32, stream=None):
    lo, hi = C.c_double(), C.c_double()
    _check(lib().gf_range(h, int(rule), int(precision), C.byref(lo), C.byref(hi), _stream_ptr(stream)))
    return lo.value, hi.value


def gf_table_create(k, r_min, r_max, params=None, stream=None):
    params = params or gf_params_default()
    h = C.c_void_p()
    _check(lib().gf_table_create(float(k), float(r_min), float(r_max), C.byref(params), _stream_ptr(stream),
                                 C.byref(h)))
    return h


def gf_table_info(h, kind):
    n, L, dr = C.c_int64(), C.c_int64(), C.c_double()
    _check(lib().gf_table_info(h, int(kind), C.byref(n), C.byref(L), C.byref(dr)))
    return n.value, L.value, dr.value


def gf_table_nodes(h, kind):
    n, L, _ = gf_table_info(h, kind)
    r, fr, fi = np.zeros(n), np.zeros(n), np.zeros(n)
    hsh = np.zeros(L, np.int32)
    _check(lib().gf_table_nodes(h, int(kind), _ptr(r), _ptr(fr), _ptr(fi), _ptr(hsh)))
    return r, fr + 1j * fi, hsh


def gf_table_eval(h, kind, r, stream=None):
    """r: CUDA tensor (float32 or float64); returns complex tensor of f(r)."""
    import torch
    if not r.is_cuda:
        raise ValueError("gf_table_eval needs a CUDA tensor")
    r = r.contiguous()
    prec = GF_FP32 if r.dtype == torch.float32 else GF_FP64
    out = torch.empty(r.numel(), dtype=torch.complex64 if prec == GF_FP32 else torch.complex128, device=r.device)
    _check(lib().gf_table_eval(h, int(kind), prec, C.c_void_p(r.data_ptr()), r.numel(),
                               C.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def gf_table_eval_host(h, kind, x):
    """Host FP64 lookup (numpy float64 in table units) -> complex128 array."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(2 * x.size)
    _check(lib().gf_table_eval_host(h, int(kind), _ptr(x), x.size, _ptr(out)))
    return out[0::2] + 1j * out[1::2]


def gf_table_create_for_mesh(mesh, k, params=None, precision=GF_FP32, r_min=-1.0, r_max=-1.0, stream=None):
    params = params or gf_params_default()
    h = C.c_void_p()
    _check(lib().gf_table_create_for_mesh(mesh, float(k), C.byref(params), int(precision), float(r_min),
                                          float(r_max), _stream_ptr(stream), C.byref(h)))
    return h


def gf_table_destroy(h):
    _check(lib().gf_table_destroy(h))


def _check_z(Z, precision):
    import torch
    want = torch.complex64 if precision == GF_FP32 else torch.complex128
    if not Z.is_cuda or Z.dtype != want or not Z.is_contiguous():
        raise ValueError(f"Z must be a contiguous CUDA {want} tensor")


def gf_fill(mesh, k, params, table, precision, Z, ldz=None, stream=None):
    """Z: CUDA tensor (complex64 for GF_FP32, complex128 for GF_FP64), at
    least [ne, ldz] row-major; overwritten."""
    _check_z(Z, precision)
    ldz = Z.shape[-1] if ldz is None else ldz
    _check(lib().gf_fill(mesh, float(k), C.byref(params), table, int(precision), C.c_void_p(Z.data_ptr()),
                         int(ldz), _stream_ptr(stream)))
    return Z


def gf_fill_parts(mesh, k, params, table, precision, Z, parts, ldz=None, stream=None):
    _check_z(Z, precision)
    ldz = Z.shape[-1] if ldz is None else ldz
    _check(lib().gf_fill_parts(mesh, float(k), C.byref(params), table, int(precision), C.c_void_p(Z.data_ptr()),
                               int(ldz), int(parts), _stream_ptr(stream)))
    return Z


# ----------------------------------------------------------------------------
# convenience objects
# ----------------------------------------------------------------------------
class Mesh:
    """Owns a gf_mesh handle."""

    def __init__(self, xyz, tri, near_dist=0.0):
        self.h = gf_mesh_create(xyz, tri, near_dist)
        self.nv, self.nt, self.ne, self.n_near = gf_mesh_info(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().gf_mesh_destroy(h)
            self.h = None

    def edges(self):
        return gf_mesh_edges(self.h)

    def set_vertices(self, xyz):
        gf_mesh_set_vertices(self.h, xyz)

    def range(self, rule, precision=GF_FP32, stream=None):
        return gf_range(self.h, rule, precision, stream)


class Table:
    """Owns a gf_table handle (Green + Exp tables for one k and range)."""

    def __init__(self, k, r_min, r_max, params=None, stream=None):
        self.k = k
        self.h = gf_table_create(k, r_min, r_max, params, stream)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().gf_table_destroy(h)
            self.h = None

    @classmethod
    def kr(cls, u_min, u_max, params=None, stream=None):
        """Tables in u = kR over [u_min, u_max]: one table for every k of a
        frequency sweep (see include/gfmom.h)."""
        t = cls.__new__(cls)
        t.k = None
        params = params or gf_params_default()
        h = C.c_void_p()
        _check(lib().gf_table_create_kr(float(u_min), float(u_max), C.byref(params), _stream_ptr(stream),
                                        C.byref(h)))
        t.h = h
        return t

    def info(self, kind=GF_GREEN):
        return gf_table_info(self.h, kind)

    def nodes(self, kind=GF_GREEN):
        return gf_table_nodes(self.h, kind)

    def __call__(self, r, kind=GF_GREEN, stream=None):
        return gf_table_eval(self.h, kind, r, stream)


def fill(mesh: Mesh, k, params=None, table: Table | None = None, precision=GF_FP32, Z=None, stream=None,
         device=None):
    """Returns Z (torch, row-major [ne, ne]) filled on the current stream."""
    import torch
    params = params or gf_params_default()
    if Z is None:
        dt = torch.complex64 if precision == GF_FP32 else torch.complex128
        Z = torch.empty((mesh.ne, mesh.ne), dtype=dt, device=device or "cuda")
    return gf_fill(mesh.h, k, params, table.h if table is not None else None, precision, Z, stream=stream)


def gf_range_noalloc(tri_xyz, tri_vert, rule, minmax, stream=None):
    """Range reduction that allocates nothing (see include/gfmom.h): tri_xyz
    a CUDA float64 tensor [nt, 9], tri_vert a CUDA int32 tensor [nt, 3],
    minmax a CUDA float64 tensor with 2 elements, written asynchronously."""
    import torch
    if not (tri_xyz.is_cuda and tri_vert.is_cuda and minmax.is_cuda):
        raise ValueError("gf_range_noalloc needs CUDA tensors")
    if tri_xyz.dtype != torch.float64 or tri_vert.dtype != torch.int32 or minmax.dtype != torch.float64:
        raise ValueError("dtypes: tri_xyz float64, tri_vert int32, minmax float64")
    if not (tri_xyz.is_contiguous() and tri_vert.is_contiguous() and minmax.is_contiguous()):
        raise ValueError("tensors must be contiguous")
    nt = tri_xyz.shape[0]
    if tri_xyz.shape != (nt, 9) or tri_vert.shape != (nt, 3) or minmax.numel() < 2:
        raise ValueError("shapes: tri_xyz [nt, 9], tri_vert [nt, 3], minmax [2]")
    _check(lib().gf_range_noalloc(C.c_void_p(tri_xyz.data_ptr()), C.c_void_p(tri_vert.data_ptr()), nt, int(rule),
                                  C.c_void_p(minmax.data_ptr()), _stream_ptr(stream)))
    return minmax


def gf_batch_create(meshes, ks, params, tables, Zs, autotune=True, stream=None):
    """meshes: Mesh objects; ks: wavenumbers; tables: Table objects or None;
    Zs: contiguous CUDA complex64 tensors [ne_i, ldz_i]."""
    n = len(meshes)
    for Z in Zs:
        _check_z(Z, GF_FP32)
    mh = (C.c_void_p * n)(*[m.h.value for m in meshes])
    kk = (C.c_double * n)(*[float(k) for k in ks])
    th = (C.c_void_p * n)(*[t.h.value for t in tables]) if tables is not None else None
    zz = (C.c_void_p * n)(*[Z.data_ptr() for Z in Zs])
    ld = (C.c_int64 * n)(*[Z.shape[-1] for Z in Zs])
    h = C.c_void_p()
    _check(lib().gf_batch_create(n, mh, kk, C.byref(params), th, GF_FP32, zz, ld, int(bool(autotune)),
                                 _stream_ptr(stream), C.byref(h)))
    return h


def gf_fill_batched(meshes, ks, params, tables, Zs, stream=None):
    """One-shot batched fill (no tuning); returns when every Z is filled."""
    n = len(meshes)
    for Z in Zs:
        _check_z(Z, GF_FP32)
    mh = (C.c_void_p * n)(*[m.h.value for m in meshes])
    kk = (C.c_double * n)(*[float(k) for k in ks])
    th = (C.c_void_p * n)(*[t.h.value for t in tables]) if tables is not None else None
    zz = (C.c_void_p * n)(*[Z.data_ptr() for Z in Zs])
    ld = (C.c_int64 * n)(*[Z.shape[-1] for Z in Zs])
    _check(lib().gf_fill_batched(n, mh, kk, C.byref(params), th, zz, ld, _stream_ptr(stream)))


def gf_batch_launch(h, stream=None):
    _check(lib().gf_batch_launch(h, _stream_ptr(stream)))


def gf_batch_config(h):
    b, c, ch, ms = C.c_int(), C.c_int(), C.c_int(), C.c_double()
    _check(lib().gf_batch_config(h, C.byref(b), C.byref(c), C.byref(ch), C.byref(ms)))
    return {"block": b.value, "ctas_per_sm": c.value, "chunk": ch.value, "tuned_ms": ms.value}


def gf_batch_destroy(h):
    _check(lib().gf_batch_destroy(h))


class Batch:
    """Owns a gf_batch handle; keeps the meshes, tables and Z tensors alive."""

    def __init__(self, meshes, ks, params, tables, Zs, autotune=True, stream=None):
        self.meshes, self.tables, self.Zs, self.params = list(meshes), tables, list(Zs), params
        self.h = gf_batch_create(self.meshes, ks, params, tables, self.Zs, autotune, stream)

    def launch(self, stream=None):
        gf_batch_launch(self.h, stream)

    def config(self):
        return gf_batch_config(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().gf_batch_destroy(h)
            self.h = None


def gf_fill_backward(mesh, k, params, table, gZ, stream=None):
    """gZ: CUDA complex64 [ne, ldg] (dL = Re sum conj(gZ) dZ). Returns
    (dxyz float64 [nv, 3], dk float64 [1]) CUDA tensors."""
    import torch
    _check_z(gZ, GF_FP32)
    dxyz = torch.empty((mesh.nv, 3), dtype=torch.float64, device=gZ.device)
    dk = torch.empty(1, dtype=torch.float64, device=gZ.device)
    _check(lib().gf_fill_backward(mesh.h, float(k), C.byref(params), table.h if table is not None else None,
                                  GF_FP32, C.c_void_p(gZ.data_ptr()), gZ.shape[-1], C.c_void_p(dxyz.data_ptr()),
                                  C.c_void_p(dk.data_ptr()), _stream_ptr(stream)))
    return dxyz, dk


GF_OP_EFIE, GF_OP_MFIE = 0, 1


def gf_excitation(mesh, k, params, khat, pol, precision, V, op=GF_OP_EFIE, stream=None):
    """V: CUDA [ne] complex64 (GF_FP32) or complex128 (GF_FP64), overwritten with
    <f_m, p e^{-jk khat.r}> (EFIE) or <f_m, n x H_inc> (MFIE); khat a unit
    3-vector, pol a complex 3-vector."""
    _check_z(V, precision)
    kh = np.ascontiguousarray(khat, dtype=np.float64).reshape(3)
    pc = np.asarray(pol, dtype=np.complex128).reshape(3)
    pl = np.ascontiguousarray(np.stack([pc.real, pc.imag], axis=1), dtype=np.float64)
    _check(lib().gf_excitation(mesh, float(k), C.byref(params), _ptr(kh), _ptr(pl), int(op), int(precision),
                               C.c_void_p(V.data_ptr()), _stream_ptr(stream)))
    return V


def gf_fill_mfie(mesh, k, params, table, precision, Z, ldz=None, stream=None):
    """MFIE matrix of a closed, outward-wound surface into Z (CUDA complex64 for
    GF_FP32, complex128 for GF_FP64, at least [ne, ldz] row-major; overwritten)."""
    _check_z(Z, precision)
    ldz = Z.shape[-1] if ldz is None else ldz
    _check(lib().gf_fill_mfie(mesh, float(k), C.byref(params), table, int(precision), C.c_void_p(Z.data_ptr()),
                              int(ldz), _stream_ptr(stream)))
    return Z


def gf_far_field(mesh, k, params, precision, I, dirs, stream=None):
    """I: CUDA [ne] complex (as precision); dirs: CUDA float64 [n, 3] unit
    vectors. Returns (F complex128 [n, 3], sigma float64 [n]) CUDA tensors."""
    import torch
    _check_z(I, precision)
    if not dirs.is_cuda or dirs.dtype != torch.float64 or not dirs.is_contiguous() or dirs.shape[-1] != 3:
        raise ValueError("dirs must be a contiguous CUDA float64 [n, 3] tensor")
    n = dirs.shape[0]
    F = torch.empty((n, 3), dtype=torch.complex128, device=I.device)
    sigma = torch.empty(n, dtype=torch.float64, device=I.device)
    _check(lib().gf_far_field(mesh, float(k), C.byref(params), int(precision), C.c_void_p(I.data_ptr()), int(n),
                              C.c_void_p(dirs.data_ptr()), C.c_void_p(F.data_ptr()),
                              C.c_void_p(sigma.data_ptr()), _stream_ptr(stream)))
    return F, sigma


def planewave_rcs(mesh: "Mesh", k, dirs, params=None, table: "Table | None" = None, precision=GF_FP32,
                  khat=(0.0, 0.0, 1.0), pol=(1.0, 0.0, 0.0), op=GF_OP_EFIE, stream=None):
    """Scattering of a plane wave by the PEC surface `mesh` (EFIE, or MFIE for a
    closed outward-wound surface): fill Z (this library), V (gf_excitation),
    solve Z I = V (a dense LU from the linear algebra library:
    torch.linalg.solve), then the far field. Returns (sigma [n] float64, I [ne])
    CUDA tensors."""
    import torch
    params = params or gf_params_default()
    if op == GF_OP_MFIE:
        dt = torch.complex64 if precision == GF_FP32 else torch.complex128
        Z = torch.empty((mesh.ne, mesh.ne), dtype=dt, device="cuda")
        gf_fill_mfie(mesh.h, k, params, table.h if table is not None else None, precision, Z, stream=stream)
    else:
        Z = fill(mesh, k, params, table, precision, stream=stream)
    V = torch.empty(mesh.ne, dtype=Z.dtype, device=Z.device)
    gf_excitation(mesh.h, k, params, khat, pol, precision, V, op=op, stream=stream)
    I = torch.linalg.solve(Z, V)
    del Z
    _, sigma = gf_far_field(mesh.h, k, params, precision, I.contiguous(), dirs, stream=stream)
    return sigma, I


class Sparse:
    """Owns a gf_sparse handle: the near-field pattern of `mesh` for `radius`
    (the mesh must outlive it)."""

    def __init__(self, mesh: "Mesh", radius):
        self.mesh = mesh
        h = C.c_void_p()
        _check(lib().gf_sparse_create(mesh.h, float(radius), C.byref(h)))
        self.h = h
        nnz, npairs = C.c_int64(), C.c_int64()
        _check(lib().gf_sparse_info(h, C.byref(nnz), C.byref(npairs)))
        self.nnz, self.n_pairs = nnz.value, npairs.value

    def pattern(self):
        row_ptr = np.zeros(self.mesh.ne + 1, dtype=np.int64)
        cols = np.zeros(max(self.nnz, 1), dtype=np.int32)
        _check(lib().gf_sparse_pattern(self.h, _ptr(row_ptr), _ptr(cols)))
        return row_ptr, cols[:self.nnz]

    def fill(self, k, params=None, table: "Table | None" = None, vals=None, stream=None):
        """Returns vals (CUDA complex64 [nnz]) with Z_mn on the pattern."""
        import torch
        params = params or gf_params_default()
        if vals is None:
            vals = torch.empty(max(self.nnz, 1), dtype=torch.complex64, device="cuda")
        _check_z(vals, GF_FP32)
        _check(lib().gf_fill_sparse(self.h, float(k), C.byref(params), table.h if table is not None else None,
                                    GF_FP32, C.c_void_p(vals.data_ptr()), _stream_ptr(stream)))
        return vals

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().gf_sparse_destroy(h)
            self.h = None


def _efie_function():
    import torch

    class EFIEFill(torch.autograd.Function):
        """Z = fill(vertices, k) with a hand-written backward (gf_fill_backward)."""

        @staticmethod
        def forward(ctx, xyz, k, mesh, table, params):
            mesh.set_vertices(xyz.detach().to("cpu", torch.float64).numpy())
            kv = float(k)
            Z = fill(mesh, kv, params, table, GF_FP32, device=xyz.device if xyz.is_cuda else None)
            ctx.mesh, ctx.table, ctx.params, ctx.k = mesh, table, params, kv
            ctx.xyz_dtype, ctx.k_tensor = xyz.dtype, torch.is_tensor(k)
            return Z

        @staticmethod
        def backward(ctx, gZ):
            dxyz, dk = gf_fill_backward(ctx.mesh, ctx.k, ctx.params, ctx.table, gZ.contiguous())
            gk = dk.reshape(()).to(torch.float64) if ctx.k_tensor else None
            return dxyz.to(ctx.xyz_dtype), gk, None, None, None

    return EFIEFill


_EFIE = None


def efie_fill(xyz, k, mesh, table=None, params=None):
    """Differentiable fill: xyz a (CUDA) float tensor [nv, 3] with the mesh's
    topology, k a float or a 0-d tensor; returns complex64 Z on the GPU. The
    table (if any) and the near-pair lists stay those of the first fill."""
    global _EFIE
    if _EFIE is None:
        _EFIE = _efie_function()
    return _EFIE.apply(xyz, k, mesh, table, params or gf_params_default())

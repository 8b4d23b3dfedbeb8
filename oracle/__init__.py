"""ctypes wrapper of the FP64 CPU oracle (oracle/liboracle.so).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline / reference arm may import this package; the product library
never does. It shares no code with the CUDA library.

What is pinned (see tests/test_oracle_*.py) and what is not:
  * quadrature rules: exact moments (closed form) -- pinned;
  * tables: exact node values, hash placement, Eq. (10)/(11) bounds on dense
    sweeps, the paper's Section IV.A experiment -- pinned;
  * singular inner integrals: static closed forms of the potential integrals
    plus a Duffy-rule brute force of the dynamic remainder -- pinned;
  * regular Z entries: brute-force high-order quadrature on small, well
    separated triangles, Galerkin symmetry -- pinned;
  * reference gradient: central differences of the direct oracle -- pinned;
  * parity unpinned: the values of the paper's Fig. 2 / Fig. 3 (not in the
    source) and the Table I timings (other code, other machine).
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        vp = C.c_void_p
        L.or_rule.argtypes = [C.c_int, dp, dp]
        L.or_gauss_legendre.argtypes = [C.c_int, dp, dp]
        L.or_mesh_new.argtypes = [dp, C.c_int, ip, C.c_int, C.c_double, C.POINTER(vp)]
        L.or_mesh_ne.argtypes = [vp]
        L.or_mesh_edges.argtypes = [vp, ip, ip]
        L.or_mesh_is_near.argtypes = [vp, C.c_int, C.c_int]
        L.or_mesh_free.argtypes = [vp]
        L.or_table_new.argtypes = [C.POINTER(TableParams), C.POINTER(vp)]
        L.or_table_info.argtypes = [vp, ip, ip, dp]
        L.or_table_get.argtypes = [vp, dp, dp, dp, ip]
        L.or_table_locate.argtypes = [vp, C.c_int, dp, ip]
        L.or_table_eval.argtypes = [vp, C.c_int, dp, dp, dp]
        L.or_table_bound.argtypes = [vp, C.c_int]
        L.or_table_bound.restype = C.c_double
        L.or_table_free.argtypes = [vp]
        L.or_singular.argtypes = [dp, dp, dp, dp, C.c_double, C.c_int, C.c_int, vp, dp, dp, dp]
        L.or_range.argtypes = [vp, C.c_int, dp, dp, C.c_int]
        L.or_range_ex.argtypes = [vp, C.c_int, C.c_int, dp, dp, C.c_int]
        L.or_z_entries.argtypes = [vp, C.POINTER(FillParams), vp, vp, C.c_long, ip, ip, dp, dp, C.c_int]
        L.or_loss_grad.argtypes = [vp, C.POINTER(FillParams), dp, dp, dp, dp, dp, dp, dp, C.c_int]
        L.or_loss_grad_masked.argtypes = [vp, C.POINTER(FillParams), dp, dp, dp, dp, ip, dp, dp, dp, C.c_int]
        L.or_loss_dk.argtypes = [vp, C.POINTER(FillParams), dp, dp, dp, dp, dp, dp, C.c_int]
        _lib = L
    return _lib


class TableParams(C.Structure):
    _fields_ = [("kind", C.c_int), ("degree", C.c_int), ("k", C.c_double), ("r_lo", C.c_double),
                ("r_hi", C.c_double), ("t", C.c_double), ("tol", C.c_double), ("refine", C.c_int),
                ("refine_factor", C.c_double), ("refine_halfwidth", C.c_double),
                ("merge", C.c_double), ("grade", C.c_int)]


class FillParams(C.Structure):
    _fields_ = [("k", C.c_double), ("eta", C.c_double), ("rule", C.c_int), ("nphi", C.c_int),
                ("nl", C.c_int), ("green_mode", C.c_int)]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


ETA0 = 376.730313668
EXP, GREEN = 0, 1


def rule(npts):
    b = np.zeros((npts, 3))
    w = np.zeros(npts)
    if lib().or_rule(npts, _dp(b), _dp(w)) != 0:
        raise ValueError(f"no {npts}-point rule")
    return b, w


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().or_gauss_legendre(n, _dp(x), _dp(w)) != 0:
        raise ValueError(n)
    return x, w


# --------------------------------------------------------------------------
# default table parameters (Eq. 2 and the readings in the module docstring)
# --------------------------------------------------------------------------
def exp_spacing_count(tol):
    """Smallest multiple of 4 in [1000, 10000] samples per wavelength with the
    Eq. (10) linear bound (k t)^2 / 8 <= tol (|e^{-jkr}| = 1)."""
    n = 1000
    while n < 10000 and (2 * math.pi / n) ** 2 / 8.0 > tol:
        n += 4
    return n


def table_params(kind, k, r_lo, r_hi, tol=1e-6, degree=None, n_per_lambda=None, refine=True,
                 grade=True, refine_factor=0.5, halfwidth_t=2.0, merge_t=0.25):
    lam = 2 * math.pi / k
    if degree is None:
        degree = 1 if kind == EXP else 3
    if n_per_lambda is None:
        n_per_lambda = exp_spacing_count(tol) if kind == EXP else 1000
    t = lam / n_per_lambda
    return TableParams(kind, degree, k, r_lo, r_hi, t, tol, int(refine), refine_factor,
                       halfwidth_t * t, merge_t * t, int(grade))


class Table:
    def __init__(self, params: TableParams):
        h = C.c_void_p()
        rc = lib().or_table_new(C.byref(params), C.byref(h))
        if rc != 0:
            raise ValueError(f"or_table_new failed: {rc}")
        self.h = h
        self.params = params
        n = C.c_int()
        L = C.c_int()
        dr = C.c_double()
        lib().or_table_info(h, C.byref(n), C.byref(L), C.byref(dr))
        self.n_nodes, self.n_hash, self.dr = n.value, L.value, dr.value

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_table_free(self.h)
            self.h = None

    def nodes(self):
        r = np.zeros(self.n_nodes)
        fr = np.zeros(self.n_nodes)
        fi = np.zeros(self.n_nodes)
        hsh = np.zeros(self.n_hash, dtype=np.int32)
        lib().or_table_get(self.h, _dp(r), _dp(fr), _dp(fi), _ip(hsh))
        return r, fr + 1j * fi, hsh

    def locate(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        j = np.zeros(r.size, dtype=np.int32)
        lib().or_table_locate(self.h, r.size, _dp(r), _ip(j))
        return j

    def __call__(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        re = np.zeros(r.size)
        im = np.zeros(r.size)
        lib().or_table_eval(self.h, r.size, _dp(r), _dp(re), _dp(im))
        return re + 1j * im

    def bound(self, j):
        return lib().or_table_bound(self.h, int(j))


def make_tables(k, r_min, r_max, tol=1e-6, **kw):
    """(Green table, Exp table) over [r_min, r_max] with the defaults above."""
    g = Table(table_params(GREEN, k, r_min, r_max, tol, **kw))
    e = Table(table_params(EXP, k, r_min, r_max, tol, **kw))
    return g, e


# --------------------------------------------------------------------------
class Mesh:
    def __init__(self, xyz, tri, near_dist=0.0):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        h = C.c_void_p()
        rc = lib().or_mesh_new(_dp(self.xyz), len(self.xyz), _ip(self.tri), len(self.tri),
                               float(near_dist), C.byref(h))
        if rc != 0:
            raise ValueError(f"or_mesh_new failed: {rc}")
        self.h = h
        self.ne = lib().or_mesh_ne(h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_mesh_free(self.h)
            self.h = None

    def edges(self):
        ev = np.zeros((self.ne, 2), dtype=np.int32)
        et = np.zeros((self.ne, 2), dtype=np.int32)
        lib().or_mesh_edges(self.h, _ip(ev), _ip(et))
        return ev, et

    def is_near(self, p, q):
        return bool(lib().or_mesh_is_near(self.h, int(p), int(q)))

    def range(self, rule, nthreads=0, prune=False):
        lo = C.c_double()
        hi = C.c_double()
        rc = lib().or_range_ex(self.h, rule, int(prune), C.byref(lo), C.byref(hi), nthreads)
        if rc != 0:
            raise ValueError(f"or_range failed: {rc}")
        return lo.value, hi.value

    def z_entries(self, k, rule, mi, ni, mode="direct", tables=None, nphi=8, nl=8, eta=ETA0,
                  nthreads=0):
        mi = np.ascontiguousarray(mi, dtype=np.int32)
        ni = np.ascontiguousarray(ni, dtype=np.int32)
        zr = np.zeros(mi.size)
        zi = np.zeros(mi.size)
        fp = FillParams(k, eta, rule, nphi, nl, {"direct": 0, "table": 1, "exp_over_r": 2}[mode])
        tg = tables[0].h if tables else None
        te = tables[1].h if tables else None
        rc = lib().or_z_entries(self.h, C.byref(fp), tg, te, mi.size, _ip(mi), _ip(ni), _dp(zr),
                                _dp(zi), nthreads)
        if rc != 0:
            raise ValueError(f"or_z_entries failed: {rc}")
        return zr + 1j * zi

    def z_full(self, k, rule, **kw):
        m, n = np.meshgrid(np.arange(self.ne), np.arange(self.ne), indexing="ij")
        return self.z_entries(k, rule, m.ravel(), n.ravel(), **kw).reshape(self.ne, self.ne)

    def z_rows(self, k, rule, rows, **kw):
        rows = np.asarray(rows, dtype=np.int32)
        m, n = np.meshgrid(rows, np.arange(self.ne), indexing="ij")
        return self.z_entries(k, rule, m.ravel(), n.ravel(), **kw).reshape(len(rows), self.ne)

    def loss_grad(self, k, rule, a, b, nphi=8, nl=8, eta=ETA0, nthreads=0, tri_mask=None):
        ar, ai = np.ascontiguousarray(a.real), np.ascontiguousarray(a.imag)
        br, bi = np.ascontiguousarray(b.real), np.ascontiguousarray(b.imag)
        loss = C.c_double()
        dk = C.c_double()
        dx = np.zeros(self.xyz.shape)
        fp = FillParams(k, eta, rule, nphi, nl, 0)
        mask = None if tri_mask is None else np.ascontiguousarray(tri_mask, dtype=np.int32)
        rc = lib().or_loss_grad_masked(self.h, C.byref(fp), _dp(ar), _dp(ai), _dp(br), _dp(bi),
                                       None if mask is None else _ip(mask), C.byref(loss), _dp(dx),
                                       C.byref(dk), nthreads)
        if rc != 0:
            raise ValueError(rc)
        return loss.value, dx, dk.value

    def loss_dk(self, k, rule, a, b, nphi=8, nl=8, eta=ETA0, nthreads=0):
        ar, ai = np.ascontiguousarray(a.real), np.ascontiguousarray(a.imag)
        br, bi = np.ascontiguousarray(b.real), np.ascontiguousarray(b.imag)
        loss, dk = C.c_double(), C.c_double()
        fp = FillParams(k, eta, rule, nphi, nl, 0)
        rc = lib().or_loss_dk(self.h, C.byref(fp), _dp(ar), _dp(ai), _dp(br), _dp(bi), C.byref(loss),
                              C.byref(dk), nthreads)
        if rc != 0:
            raise ValueError(rc)
        return loss.value, dk.value


def singular(r, v0, v1, v2, k, nphi=8, nl=8, texp=None):
    r, v0, v1, v2 = (np.ascontiguousarray(x, dtype=np.float64) for x in (r, v0, v1, v2))
    i0 = np.zeros(2)
    i1 = np.zeros(6)
    rho = np.zeros(3)
    rc = lib().or_singular(_dp(r), _dp(v0), _dp(v1), _dp(v2), k, nphi, nl,
                           texp.h if texp is not None else None, _dp(i0), _dp(i1), _dp(rho))
    if rc != 0:
        raise ValueError(rc)
    return complex(i0[0], i0[1]), i1[0::2] + 1j * i1[1::2], rho

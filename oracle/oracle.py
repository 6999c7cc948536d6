"""ctypes wrapper of liboracle.so (FP64 CPU oracle; test infrastructure only).

Each function takes a ``workloads.Geometry`` (plain inputs) and numpy arrays, converts them
to float64 and calls the C oracle.  Nothing here does any of the method's arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (IEEE double, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("ds", ctypes.c_double), ("origin", ctypes.c_double * 3),
                ("nq", ctypes.c_int), ("pos", ctypes.POINTER(ctypes.c_double)),
                ("nk", ctypes.c_int), ("fs", ctypes.c_double), ("tmin", ctypes.c_double),
                ("c", ctypes.c_double), ("R", ctypes.c_double), ("gamma", ctypes.c_double),
                ("area", ctypes.c_int)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        gp = ctypes.POINTER(_Geom)
        _lib.oracle_G.argtypes = [gp, dp, dp]
        _lib.oracle_G_rows.argtypes = [gp, dp, ip, ctypes.c_int, dp]
        _lib.oracle_Gt.argtypes = [gp, dp, dp]
        _lib.oracle_Gt_nodes.argtypes = [gp, dp, ip, ctypes.c_int, dp]
        _lib.oracle_D.argtypes = [gp, dp, dp]
        _lib.oracle_Dt.argtypes = [gp, dp, dp]
        _lib.oracle_H.argtypes = [gp, dp, dp, ctypes.c_int]
        _lib.oracle_Ht.argtypes = [gp, dp, dp, ctypes.c_int]
        _lib.oracle_dense_G.argtypes = [gp, dp]
        _lib.oracle_shell_points.argtypes = [gp, ctypes.c_int, ctypes.c_int, dp, ip, dp, ctypes.c_long, ip]
        _lib.oracle_shell_points.restype = ctypes.c_long
        _lib.oracle_count_points.argtypes = [gp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
        _lib.oracle_max_threads.restype = ctypes.c_int
        _lib.oracle_set_threads.argtypes = [ctypes.c_int]
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class _G:
    """Keeps the ctypes struct and the position array alive together."""

    def __init__(self, geom):
        self.pos = np.ascontiguousarray(geom.positions_mm, dtype=np.float64)
        self.s = _Geom(geom.nx, geom.ny, geom.nz, geom.spacing_mm, (ctypes.c_double * 3)(*geom.origin_mm),
                       self.pos.shape[0], _dp(self.pos), geom.n_samples, geom.fs_mhz, geom.t_min_us,
                       geom.c_mm_per_us, geom.support_radius_mm, geom.gruneisen,
                       int(getattr(geom, "lattice_weights", 0)))
        self.ref = ctypes.byref(self.s)


def _f64(a, shape):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    assert a.shape == tuple(shape), (a.shape, shape)
    return a


def G(geom, alpha):
    g = _G(geom)
    a = _f64(alpha, geom.vol_shape)
    out = np.empty(geom.data_shape)
    _L().oracle_G(g.ref, _dp(a), _dp(out))
    return out


def G_rows(geom, alpha, rows):
    g = _G(geom)
    a = _f64(alpha, geom.vol_shape)
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int32).reshape(-1, 2))
    out = np.empty(r.shape[0])
    _L().oracle_G_rows(g.ref, _dp(a), _ip(r), r.shape[0], _dp(out))
    return out


def Gt(geom, gp):
    g = _G(geom)
    a = _f64(gp, geom.data_shape)
    out = np.empty(geom.vol_shape)
    _L().oracle_Gt(g.ref, _dp(a), _dp(out))
    return out


def Gt_nodes(geom, gp, nodes):
    """G^T gp at nodes given as (ix, iy, iz) triples."""
    g = _G(geom)
    a = _f64(gp, geom.data_shape)
    nd = np.ascontiguousarray(np.asarray(nodes, dtype=np.int32).reshape(-1, 3))
    out = np.empty(nd.shape[0])
    _L().oracle_Gt_nodes(g.ref, _dp(a), _ip(nd), nd.shape[0], _dp(out))
    return out


def D(geom, gin):
    g = _G(geom)
    a = _f64(gin, geom.data_shape)
    out = np.empty(geom.data_shape)
    _L().oracle_D(g.ref, _dp(a), _dp(out))
    return out


def Dt(geom, pin):
    g = _G(geom)
    a = _f64(pin, geom.data_shape)
    out = np.empty(geom.data_shape)
    _L().oracle_Dt(g.ref, _dp(a), _dp(out))
    return out


def H(geom, alpha, apply_d=True):
    g = _G(geom)
    a = _f64(alpha, geom.vol_shape)
    out = np.empty(geom.data_shape)
    _L().oracle_H(g.ref, _dp(a), _dp(out), int(bool(apply_d)))
    return out


def Ht(geom, y, apply_d=True):
    g = _G(geom)
    a = _f64(y, geom.data_shape)
    out = np.empty(geom.vol_shape)
    _L().oracle_Ht(g.ref, _dp(a), _dp(out), int(bool(apply_d)))
    return out


def H_rows(geom, alpha, rows, apply_d=True):
    """Selected rows (q, k) of H alpha, computed from the G rows at k-1, k, k+1 through D."""
    rows = np.asarray(rows, dtype=np.int64).reshape(-1, 2)
    if not apply_d:
        return G_rows(geom, alpha, rows)
    K = geom.n_samples
    need = sorted({(int(q), int(kk)) for q, k in rows for kk in (k - 1, k + 1) if 0 <= kk < K})
    vals = dict(zip(need, G_rows(geom, alpha, need))) if need else {}
    out = np.zeros(len(rows))
    for r, (q, k) in enumerate(rows):
        gq = np.zeros((1, K))
        for kk in (k - 1, k + 1):
            if (int(q), int(kk)) in vals:
                gq[0, kk] = vals[(int(q), int(kk))]
        sub = geom.subset([q])
        out[r] = D(sub, gq)[0, k]
    return out


def dense_G(geom):
    g = _G(geom)
    M = np.empty((geom.n_transducers * geom.n_samples, geom.n_voxels))
    _L().oracle_dense_G(g.ref, _dp(M))
    return M


def shell_points(geom, q, k, with_weights=False):
    """(points [n, 3] in mm, ij [n, 2], number of rings) of the shell of sample (q, k); with
    with_weights also the points' weights (mm^2) as a fourth element."""
    g = _G(geom)
    nr = ctypes.c_int(0)
    n = _L().oracle_shell_points(g.ref, q, k, None, None, None, 0, ctypes.byref(nr))
    P = np.empty((max(n, 1), 3))
    ij = np.empty((max(n, 1), 2), dtype=np.int32)
    w = np.empty(max(n, 1))
    _L().oracle_shell_points(g.ref, q, k, _dp(P), _ip(ij), _dp(w), n, ctypes.byref(nr))
    return (P[:n], ij[:n], nr.value, w[:n]) if with_weights else (P[:n], ij[:n], nr.value)


def count_points(geom):
    """(lattice points in the support sphere, points with a node of their stencil in the grid)."""
    g = _G(geom)
    nb, ng = ctypes.c_longlong(0), ctypes.c_longlong(0)
    _L().oracle_count_points(g.ref, ctypes.byref(nb), ctypes.byref(ng))
    return nb.value, ng.value


def max_threads():
    return _L().oracle_max_threads()


def set_threads(n):
    _L().oracle_set_threads(int(n))

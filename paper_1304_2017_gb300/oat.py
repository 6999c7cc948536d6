"""Python binding of the C ABI in include/oat.h (argument marshalling only).

The functions carry the C names (``oat_plan_create``, ``oat_project``, ``oat_backproject``,
``oat_plan_destroy``, ``oat_plan_query``, ...).  ``Plan`` wraps a plan handle for torch
tensors: device memory and the current CUDA stream come from PyTorch, every step of the
operator runs in the library's sm_103a kernels.  There is no CPU fallback: importing this
module fails loudly when ``liboat.so`` has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboat.so")

OAT_OK = 0
OAT_ERR_INVALID_ARG = -1
OAT_ERR_GEOMETRY = -2
OAT_ERR_CUDA = -3
OAT_ERR_OOM = -4
OAT_ERR_UNSUPPORTED = -5
OAT_F32, OAT_F16, OAT_BF16 = 0, 1, 2


class OatError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class oat_geometry(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("spacing_mm", ctypes.c_double), ("origin_mm", ctypes.c_double * 3),
                ("n_transducers", ctypes.c_int), ("positions_mm", ctypes.POINTER(ctypes.c_double)),
                ("n_samples", ctypes.c_int), ("fs_mhz", ctypes.c_double), ("t_min_us", ctypes.c_double),
                ("c_mm_per_us", ctypes.c_double), ("support_radius_mm", ctypes.c_double),
                ("gruneisen", ctypes.c_double), ("data_dtype", ctypes.c_int), ("apply_d", ctypes.c_int),
                ("lattice_weights", ctypes.c_int)]


class oat_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_longlong) for n in ("n_radius_classes", "n_rings", "points_ball", "points_grid",
                                                  "table_bytes", "scratch_bytes", "work_items")]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
                          "(the projector has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    lib.oat_plan_create.argtypes = [ctypes.POINTER(oat_geometry), ctypes.c_int, ctypes.POINTER(vp)]
    lib.oat_plan_destroy.argtypes = [vp]
    lib.oat_project.argtypes = [vp, vp, vp, vp]
    lib.oat_backproject.argtypes = [vp, vp, vp, vp]
    lib.oat_backproject_noalloc.argtypes = [vp, vp, vp, vp]
    lib.oat_plan_set_fbp_weights.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.oat_fbp.argtypes = [vp, vp, vp, vp]
    lib.oat_plan_set_eir.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int]
    lib.oat_plan_query.argtypes = [vp, ctypes.c_int, ctypes.POINTER(oat_stats)]
    lib.oat_plan_set_profiling.argtypes = [vp, ctypes.c_int]
    lib.oat_plan_kernel_time.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_longlong)]
    ll, f32, i32 = ctypes.c_longlong, ctypes.c_float, ctypes.c_int
    lib.oat_fista_residual.argtypes = [ll, vp, vp, vp, i32, f32, vp, vp, vp]
    lib.oat_tv_prox.argtypes = [i32, i32, i32, vp, vp, f32, f32, i32, vp, vp, vp]
    lib.oat_fista_momentum.argtypes = [ll, vp, vp, f32, vp, vp]
    lib.oat_dot.argtypes = [ll, vp, vp, vp, vp]
    lib.oat_tv_value.argtypes = [i32, i32, i32, vp, vp, vp]
    lib.oat_probe_read.argtypes = [vp, ll, i32, vp, vp]
    lib.oat_fbp_sample_positions.argtypes = [vp, vp, vp, i32, vp, vp]
    lib.oat_sph_create.argtypes = [ctypes.POINTER(oat_geometry), i32, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_double), i32, ctypes.POINTER(vp)]
    lib.oat_sph_project.argtypes = [vp, vp, vp, vp]
    lib.oat_sph_backproject.argtypes = [vp, vp, vp, vp]
    lib.oat_sph_destroy.argtypes = [vp]
    for name in ("oat_fista_residual", "oat_tv_prox", "oat_fista_momentum", "oat_dot", "oat_tv_value",
                 "oat_probe_read", "oat_fbp_sample_positions", "oat_sph_create", "oat_sph_project", "oat_sph_backproject", "oat_sph_destroy"):
        getattr(lib, name).restype = ctypes.c_int
    lib.oat_last_error.restype = ctypes.c_char_p
    lib.oat_version.restype = ctypes.c_int
    for name in ("oat_plan_create", "oat_plan_destroy", "oat_project", "oat_backproject", "oat_backproject_noalloc",
                 "oat_plan_query", "oat_plan_set_fbp_weights", "oat_fbp", "oat_plan_set_eir",
                 "oat_plan_set_profiling", "oat_plan_kernel_time"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


lib = _load()


def _check(rc):
    if rc != OAT_OK:
        raise OatError(rc, lib.oat_last_error().decode())
    return rc


def make_geometry_struct(geom, data_dtype=OAT_F32, apply_d=True):
    """oat_geometry from a workloads.Geometry; returns (struct, positions array kept alive)."""
    pos = np.ascontiguousarray(geom.positions_mm, dtype=np.float64)
    s = oat_geometry(geom.nx, geom.ny, geom.nz, geom.spacing_mm, (ctypes.c_double * 3)(*geom.origin_mm),
                     pos.shape[0], pos.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), geom.n_samples,
                     geom.fs_mhz, geom.t_min_us, geom.c_mm_per_us, geom.support_radius_mm, geom.gruneisen,
                     int(data_dtype), int(bool(apply_d)), int(getattr(geom, "lattice_weights", 0)))
    return s, pos


# ---- C names ---------------------------------------------------------------------------

def oat_version():
    return lib.oat_version()


def oat_last_error():
    return lib.oat_last_error().decode()


def oat_plan_create(geom_struct, device=0):
    h = ctypes.c_void_p()
    _check(lib.oat_plan_create(ctypes.byref(geom_struct), int(device), ctypes.byref(h)))
    return h


def oat_plan_destroy(handle):
    return _check(lib.oat_plan_destroy(handle))


def oat_project(handle, d_vol, d_data, stream=0):
    return _check(lib.oat_project(handle, ctypes.c_void_p(d_vol), ctypes.c_void_p(d_data), ctypes.c_void_p(stream)))


def oat_backproject(handle, d_data, d_vol, stream=0):
    return _check(lib.oat_backproject(handle, ctypes.c_void_p(d_data), ctypes.c_void_p(d_vol), ctypes.c_void_p(stream)))


def oat_backproject_noalloc(handle, d_data, d_vol, stream=0):
    return _check(lib.oat_backproject_noalloc(handle, ctypes.c_void_p(d_data), ctypes.c_void_p(d_vol),
                                              ctypes.c_void_p(stream)))


def oat_plan_set_fbp_weights(handle, weights):
    w = np.ascontiguousarray(weights, dtype=np.float64)
    return _check(lib.oat_plan_set_fbp_weights(handle, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def oat_plan_set_eir(handle, h, first_index=0):
    t = np.ascontiguousarray(h, dtype=np.float64).reshape(-1)
    ptr = t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if t.size else None
    return _check(lib.oat_plan_set_eir(handle, ptr, int(t.size), int(first_index)))


def oat_fbp(handle, d_data, d_vol, stream=0):
    return _check(lib.oat_fbp(handle, ctypes.c_void_p(d_data), ctypes.c_void_p(d_vol), ctypes.c_void_p(stream)))


def oat_plan_query(handle, count_grid_points=False):
    st = oat_stats()
    _check(lib.oat_plan_query(handle, int(bool(count_grid_points)), ctypes.byref(st)))
    return {n: getattr(st, n) for n, _ in oat_stats._fields_}


def oat_plan_set_profiling(handle, enable=True):
    return _check(lib.oat_plan_set_profiling(handle, int(bool(enable))))


def oat_plan_kernel_time(handle, which, reset=False):
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    _check(lib.oat_plan_kernel_time(handle, int(which), int(bool(reset)), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


# ---- reconstruction kernels (include/oat_recon.h) ------------------------------------------

def _p(x):
    return ctypes.c_void_p(x)


def oat_fista_residual(n, hx, hx_prev, u, u_dtype, beta, r, acc, stream=0):
    return _check(lib.oat_fista_residual(n, _p(hx), _p(hx_prev), _p(u), u_dtype, beta, _p(r), _p(acc), _p(stream)))


def oat_tv_prox(nx, ny, nz, z, g, step, lam, iters, out, work, stream=0):
    return _check(lib.oat_tv_prox(nx, ny, nz, _p(z), _p(g) if g else None, step, lam, iters, _p(out), _p(work),
                                  _p(stream)))


def oat_fista_momentum(n, a, a_prev, beta, y, stream=0):
    return _check(lib.oat_fista_momentum(n, _p(a), _p(a_prev), beta, _p(y), _p(stream)))


def oat_dot(n, x, y, acc, stream=0):
    return _check(lib.oat_dot(n, _p(x), _p(y), _p(acc), _p(stream)))


def oat_tv_value(nx, ny, nz, x, acc, stream=0):
    return _check(lib.oat_tv_value(nx, ny, nz, _p(x), _p(acc), _p(stream)))


def oat_fbp_sample_positions(handle, d_nodes, d_transducers, n, d_out, stream=0):
    return _check(lib.oat_fbp_sample_positions(handle, _p(d_nodes), _p(d_transducers), int(n), _p(d_out), _p(stream)))


def oat_probe_read(buf, n_bytes, reps, sink, stream=0):
    return _check(lib.oat_probe_read(_p(buf), n_bytes, reps, _p(sink), _p(stream)))


# ---- spherical-voxel model (include/oat_sph.h) ---------------------------------------------

def oat_sph_create(geom_struct, n_freq, f0_mhz, df_mhz, eir=None, device=0):
    h = ctypes.c_void_p()
    e = None
    if eir is not None:
        e = np.ascontiguousarray(np.stack([np.real(eir), np.imag(eir)], axis=1), dtype=np.float64)
    ptr = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if e is not None else None
    _check(lib.oat_sph_create(ctypes.byref(geom_struct), int(n_freq), float(f0_mhz), float(df_mhz), ptr, int(device),
                              ctypes.byref(h)))
    return h


def oat_sph_project(handle, d_alpha, d_u, stream=0):
    return _check(lib.oat_sph_project(handle, _p(d_alpha), _p(d_u), _p(stream)))


def oat_sph_backproject(handle, d_u, d_alpha, stream=0):
    return _check(lib.oat_sph_backproject(handle, _p(d_u), _p(d_alpha), _p(stream)))


def oat_sph_destroy(handle):
    return _check(lib.oat_sph_destroy(handle))


# ---- torch wrapper ---------------------------------------------------------------------

_DT = {OAT_F32: "float32", OAT_F16: "float16", OAT_BF16: "bfloat16"}


def dtype_code(torch_dtype):
    """OAT_F32 / OAT_F16 / OAT_BF16 for a torch dtype (ValueError otherwise)."""
    name = str(torch_dtype).replace("torch.", "")
    for code, n in _DT.items():
        if n == name:
            return code
    raise ValueError(f"unsupported data dtype {torch_dtype}")


class Plan:
    """A plan for one geometry: ``project(vol) -> data`` and ``backproject(data) -> vol``."""

    def __init__(self, geom, data_dtype=OAT_F32, apply_d=True, device=None):
        import torch
        self._torch = torch
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        self.geom = geom
        self.data_dtype = int(data_dtype)
        self.apply_d = bool(apply_d)
        self._s, self._pos = make_geometry_struct(geom, data_dtype, apply_d)
        self.handle = oat_plan_create(self._s, self.device)
        self.vol_shape = (geom.nz, geom.ny, geom.nx)
        self.data_shape = (geom.n_transducers, geom.n_samples)
        self.torch_data_dtype = getattr(torch, _DT[self.data_dtype])

    def close(self):
        if getattr(self, "handle", None) is not None:
            oat_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        return self._torch.cuda.current_stream(self.device).cuda_stream

    def _checked(self, t, shape, dtype, name):
        torch = self._torch
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.device.index != self.device:
            raise ValueError(f"{name}: expected a CUDA tensor on device {self.device}")
        if tuple(t.shape) != tuple(shape) or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"{name}: expected contiguous {dtype} {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")
        return t

    def project(self, vol, out=None):
        torch = self._torch
        self._checked(vol, self.vol_shape, torch.float32, "vol")
        if out is None:
            out = torch.empty(self.data_shape, dtype=self.torch_data_dtype, device=vol.device)
        self._checked(out, self.data_shape, self.torch_data_dtype, "out")
        oat_project(self.handle, vol.data_ptr(), out.data_ptr(), self._stream())
        return out

    def set_fbp_weights(self, weights):
        """Per-transducer FBP weights (patch area / sphere radius), n_transducers values."""
        w = np.ascontiguousarray(weights, dtype=np.float64)
        if w.shape != (self.data_shape[0],):
            raise ValueError(f"weights: expected {self.data_shape[0]} values, got shape {w.shape}")
        oat_plan_set_fbp_weights(self.handle, w)

    def set_eir(self, h, first_index=0):
        """Transducer response taps h_m for m = first_index, first_index + 1, ... (Eq. EIR); from
        then on project is H^e D G and backproject its adjoint.  An empty h removes it."""
        oat_plan_set_eir(self.handle, h, first_index)

    def fbp(self, data, out=None):
        """Filtered backprojection of data [Q][K] (plan's data dtype) -> (nz, ny, nx) float32."""
        torch = self._torch
        self._checked(data, self.data_shape, self.torch_data_dtype, "data")
        if out is None:
            out = torch.empty(self.vol_shape, dtype=torch.float32, device=data.device)
        self._checked(out, self.vol_shape, torch.float32, "out")
        oat_fbp(self.handle, data.data_ptr(), out.data_ptr(), self._stream())
        return out

    def fbp_sample_positions(self, nodes, transducers):
        """k~ of (node, transducer) pairs as oat_fbp computes it: nodes int (n, 3) (ix, iy, iz),
        transducers int (n,); returns a float64 numpy array (n,)."""
        torch = self._torch
        nd = torch.as_tensor(np.ascontiguousarray(nodes, dtype=np.int32).reshape(-1, 3), device=self.device)
        qs = torch.as_tensor(np.ascontiguousarray(transducers, dtype=np.int32).reshape(-1), device=self.device)
        if nd.shape[0] != qs.shape[0]:
            raise ValueError("nodes and transducers differ in length")
        out = torch.empty(qs.shape[0], dtype=torch.float64, device=self.device)
        oat_fbp_sample_positions(self.handle, nd.data_ptr(), qs.data_ptr(), qs.shape[0], out.data_ptr(), self._stream())
        return out.cpu().numpy()

    def backproject(self, data, out=None):
        torch = self._torch
        self._checked(data, self.data_shape, self.torch_data_dtype, "data")
        if out is None:
            out = torch.empty(self.vol_shape, dtype=torch.float32, device=data.device)
        self._checked(out, self.vol_shape, torch.float32, "out")
        oat_backproject(self.handle, data.data_ptr(), out.data_ptr(), self._stream())
        return out

    def stats(self, count_grid_points=False):
        return oat_plan_query(self.handle, count_grid_points)

    def set_profiling(self, enable=True):
        oat_plan_set_profiling(self.handle, enable)

    def kernel_time(self, which, reset=False):
        return oat_plan_kernel_time(self.handle, which, reset)


class SphOp:
    """The spherical-voxel model for one geometry and L frequencies f_l = f0 + l df:
    ``project(alpha) -> u`` (complex64 [Q][L]) and ``backproject(u) -> alpha'`` (float32)."""

    def __init__(self, geom, n_freq, f0_mhz, df_mhz, eir=None, device=None):
        import torch
        self._torch = torch
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        self.geom = geom
        self.n_freq = int(n_freq)
        self.freqs = float(f0_mhz) + float(df_mhz) * np.arange(self.n_freq)
        self._s, self._pos = make_geometry_struct(geom)
        self.handle = oat_sph_create(self._s, n_freq, f0_mhz, df_mhz, eir, self.device)
        self.vol_shape = (geom.nz, geom.ny, geom.nx)
        self.data_shape = (geom.n_transducers, self.n_freq)

    def close(self):
        if getattr(self, "handle", None) is not None:
            oat_sph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        return self._torch.cuda.current_stream(self.device).cuda_stream

    def _checked(self, t, shape, dtype, name):
        torch = self._torch
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.device.index != self.device:
            raise ValueError(f"{name}: expected a CUDA tensor on device {self.device}")
        if tuple(t.shape) != tuple(shape) or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"{name}: expected contiguous {dtype} of shape {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")

    def project(self, alpha, out=None):
        torch = self._torch
        self._checked(alpha, self.vol_shape, torch.float32, "alpha")
        if out is None:
            out = torch.empty(self.data_shape, dtype=torch.complex64, device=alpha.device)
        self._checked(out, self.data_shape, torch.complex64, "out")
        oat_sph_project(self.handle, alpha.data_ptr(), out.data_ptr(), self._stream())
        return out

    def backproject(self, u, out=None):
        torch = self._torch
        self._checked(u, self.data_shape, torch.complex64, "u")
        if out is None:
            out = torch.empty(self.vol_shape, dtype=torch.float32, device=u.device)
        self._checked(out, self.vol_shape, torch.float32, "out")
        oat_sph_backproject(self.handle, u.data_ptr(), out.data_ptr(), self._stream())
        return out

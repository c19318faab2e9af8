"""ctypes binding of the FP64 C oracle projector (``sf_fan_oracle.c``).

ORACLE -- test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg may import this module.

The system matrix is the separable-footprint fan-beam (arc detector) A used
by the PWLS problem of Sec. III (Eq. (ct_problem)); its definition is written
out in the C file's header.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


class _Geom(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("offset_x", ctypes.c_double), ("offset_y", ctypes.c_double),
        ("ns", ctypes.c_int), ("na", ctypes.c_int),
        ("ds", ctypes.c_double), ("offset_s", ctypes.c_double),
        ("dso", ctypes.c_double), ("dsd", ctypes.c_double),
        ("orbit_deg", ctypes.c_double), ("orbit_start_deg", ctypes.c_double),
    ]


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        gp = ctypes.POINTER(_Geom)
        lib.orc_fan_forward.argtypes = [gp, dp, ip, ctypes.c_int, dp]
        lib.orc_fan_back.argtypes = [gp, dp, ip, ctypes.c_int, dp]
        lib.orc_fan_matrix.argtypes = [gp, ip, ctypes.c_int, dp]
        lib.orc_fan_forward_rays.argtypes = [gp, dp, ip, ip, ctypes.c_int, dp]
        lib.orc_fan_back_pixels.argtypes = [gp, dp, ip, ctypes.c_int, ip, ctypes.c_int, dp]
        for f in ("orc_fan_forward", "orc_fan_back", "orc_fan_matrix", "orc_fan_forward_rays",
                  "orc_fan_back_pixels", "orc_num_threads"):
            getattr(lib, f).restype = ctypes.c_int
        _LIB = lib
    return _LIB


def num_threads() -> int:
    return int(_lib().orc_num_threads())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class FanProjector:
    """FP64 separable-footprint fan-arc projector A (oracle)."""

    def __init__(self, geom):
        self.geom = geom
        self._g = _Geom(geom.nx, geom.ny, geom.dx, geom.dy, geom.offset_x, geom.offset_y,
                        geom.ns, geom.na, geom.ds, geom.offset_s, geom.dso, geom.dsd,
                        geom.orbit_deg, geom.orbit_start_deg)
        _lib()

    @property
    def npix(self) -> int:
        return self.geom.nx * self.geom.ny

    def _views(self, views):
        if views is None:
            views = np.arange(self.geom.na)
        v = np.ascontiguousarray(np.asarray(views, dtype=np.int32))
        if v.ndim != 1 or (v.size and (v.min() < 0 or v.max() >= self.geom.na)):
            raise ValueError("view index out of range")
        return v

    def forward(self, x: np.ndarray, views=None) -> np.ndarray:
        """A_views x -> [len(views)][ns]."""
        v = self._views(views)
        xx = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        assert xx.size == self.npix
        y = np.zeros((v.size, self.geom.ns), dtype=np.float64)
        rc = _lib().orc_fan_forward(ctypes.byref(self._g), _dp(xx), _ip(v), v.size, _dp(y))
        if rc:
            raise RuntimeError(f"orc_fan_forward failed ({rc})")
        return y

    def back(self, y: np.ndarray, views=None) -> np.ndarray:
        """A_views^T y -> [ny][nx]."""
        v = self._views(views)
        yy = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
        assert yy.size == v.size * self.geom.ns
        x = np.zeros(self.npix, dtype=np.float64)
        rc = _lib().orc_fan_back(ctypes.byref(self._g), _dp(yy), _ip(v), v.size, _dp(x))
        if rc:
            raise RuntimeError(f"orc_fan_back failed ({rc})")
        return x.reshape(self.geom.ny, self.geom.nx)

    def matrix(self, views=None) -> np.ndarray:
        """Dense A_views of shape [len(views)*ns, nx*ny] (small geometries only)."""
        v = self._views(views)
        A = np.zeros((v.size * self.geom.ns, self.npix), dtype=np.float64)
        rc = _lib().orc_fan_matrix(ctypes.byref(self._g), _ip(v), v.size, _dp(A))
        if rc:
            raise RuntimeError(f"orc_fan_matrix failed ({rc})")
        return A

    def forward_rays(self, x: np.ndarray, ray_view, ray_bin) -> np.ndarray:
        rv = np.ascontiguousarray(np.asarray(ray_view, dtype=np.int32))
        rb = np.ascontiguousarray(np.asarray(ray_bin, dtype=np.int32))
        xx = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        out = np.zeros(rv.size, dtype=np.float64)
        rc = _lib().orc_fan_forward_rays(ctypes.byref(self._g), _dp(xx), _ip(rv), _ip(rb), rv.size, _dp(out))
        if rc:
            raise RuntimeError(f"orc_fan_forward_rays failed ({rc})")
        return out

    def back_pixels(self, y: np.ndarray, views, pix) -> np.ndarray:
        v = self._views(views)
        p = np.ascontiguousarray(np.asarray(pix, dtype=np.int32))
        yy = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
        out = np.zeros(p.size, dtype=np.float64)
        rc = _lib().orc_fan_back_pixels(ctypes.byref(self._g), _dp(yy), _ip(v), v.size, _ip(p), p.size, _dp(out))
        if rc:
            raise RuntimeError(f"orc_fan_back_pixels failed ({rc})")
        return out

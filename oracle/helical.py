"""ctypes binding of the FP64 C oracle helical cone-beam projector (``sf_helical_oracle.c``).

ORACLE -- test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg may import this module.

The system matrix is the separable-footprint A of the PWLS problem (Sec. III,
Eq. (ct_problem)) for the 3-D helical scans of Sec. IV, with a trapezoid
transaxial footprint and a rectangle (SF-TR) or trapezoid (SF-TT) axial one;
its definition is written out in the C file's header.  Volumes are
``[nz][ny][nx]``; sinograms ``[view][row][cell]``.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_LIB = None


class _HGeom(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("offset_x", ctypes.c_double), ("offset_y", ctypes.c_double), ("offset_z", ctypes.c_double),
        ("ns", ctypes.c_int), ("nt", ctypes.c_int), ("na", ctypes.c_int),
        ("ds", ctypes.c_double), ("dt", ctypes.c_double),
        ("offset_s", ctypes.c_double), ("offset_t", ctypes.c_double),
        ("dso", ctypes.c_double), ("dsd", ctypes.c_double),
        ("orbit_deg", ctypes.c_double), ("orbit_start_deg", ctypes.c_double), ("pitch", ctypes.c_double),
        ("axial", ctypes.c_int),
    ]

AXIAL = {"rect": 0, "trap": 1}


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_longlong)
        gp = ctypes.POINTER(_HGeom)
        lib.orc_helix_forward.argtypes = [gp, dp, ip, ctypes.c_int, dp]
        lib.orc_helix_back.argtypes = [gp, dp, ip, ctypes.c_int, dp]
        lib.orc_helix_matrix.argtypes = [gp, ip, ctypes.c_int, dp]
        lib.orc_helix_forward_rays.argtypes = [gp, dp, ip, ip, ip, ctypes.c_int, dp]
        lib.orc_helix_back_voxels.argtypes = [gp, dp, ip, ctypes.c_int, lp, ctypes.c_int, dp]
        for f in ("orc_helix_forward", "orc_helix_back", "orc_helix_matrix", "orc_helix_forward_rays",
                  "orc_helix_back_voxels"):
            getattr(lib, f).restype = ctypes.c_int
        lib.orc_helix_source_z.argtypes = [gp, ctypes.c_int]
        lib.orc_helix_source_z.restype = ctypes.c_double
        _LIB = lib
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class HelicalProjector:
    """FP64 separable-footprint helical cone-beam projector A (oracle): SF-TR, or SF-TT when the
    geometry's ``axial`` is "trap"."""

    def __init__(self, geom):
        self.geom = geom
        g = geom
        self._g = _HGeom(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.offset_x, g.offset_y, g.offset_z, g.ns, g.nt, g.na,
                         g.ds, g.dt, g.offset_s, g.offset_t, g.dso, g.dsd, g.orbit_deg, g.orbit_start_deg, g.pitch,
                         AXIAL[getattr(g, "axial", "rect")])
        _lib()

    @property
    def shape(self):
        return (self.geom.nz, self.geom.ny, self.geom.nx)

    @property
    def nvox(self) -> int:
        return self.geom.nx * self.geom.ny * self.geom.nz

    @property
    def view_shape(self):
        return (self.geom.nt, self.geom.ns)

    def _views(self, views):
        if views is None:
            views = np.arange(self.geom.na)
        v = np.ascontiguousarray(np.asarray(views, dtype=np.int32))
        if v.ndim != 1 or (v.size and (v.min() < 0 or v.max() >= self.geom.na)):
            raise ValueError("view index out of range")
        return v

    def forward(self, x: np.ndarray, views=None) -> np.ndarray:
        """A_views x -> [len(views)][nt][ns]."""
        v = self._views(views)
        xx = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        assert xx.size == self.nvox
        y = np.zeros((v.size, self.geom.nt, self.geom.ns))
        if _lib().orc_helix_forward(ctypes.byref(self._g), _dp(xx), _ip(v), v.size, _dp(y)):
            raise RuntimeError("orc_helix_forward failed")
        return y

    def back(self, y: np.ndarray, views=None) -> np.ndarray:
        """A_views' y -> [nz][ny][nx]."""
        v = self._views(views)
        yy = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
        assert yy.size == v.size * self.geom.nt * self.geom.ns
        x = np.zeros(self.nvox)
        if _lib().orc_helix_back(ctypes.byref(self._g), _dp(yy), _ip(v), v.size, _dp(x)):
            raise RuntimeError("orc_helix_back failed")
        return x.reshape(self.shape)

    def matrix(self, views=None) -> np.ndarray:
        """Dense A_views [(len(views)*nt*ns)][nvox] (small geometries only)."""
        v = self._views(views)
        A = np.zeros((v.size * self.geom.nt * self.geom.ns, self.nvox))
        if _lib().orc_helix_matrix(ctypes.byref(self._g), _ip(v), v.size, _dp(A)):
            raise RuntimeError("orc_helix_matrix failed")
        return A

    def forward_rays(self, x: np.ndarray, ray_view, ray_row, ray_cell) -> np.ndarray:
        rv = np.ascontiguousarray(np.asarray(ray_view, dtype=np.int32))
        rt = np.ascontiguousarray(np.asarray(ray_row, dtype=np.int32))
        rs = np.ascontiguousarray(np.asarray(ray_cell, dtype=np.int32))
        xx = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        out = np.zeros(rv.size)
        if _lib().orc_helix_forward_rays(ctypes.byref(self._g), _dp(xx), _ip(rv), _ip(rt), _ip(rs), rv.size,
                                         _dp(out)):
            raise RuntimeError("orc_helix_forward_rays failed")
        return out

    def back_voxels(self, y: np.ndarray, views, vox) -> np.ndarray:
        """[A_views' y] at the flat voxel indices ``vox`` (into [nz][ny][nx])."""
        v = self._views(views)
        q = np.ascontiguousarray(np.asarray(vox, dtype=np.int64))
        yy = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
        out = np.zeros(q.size)
        if _lib().orc_helix_back_voxels(ctypes.byref(self._g), _dp(yy), _ip(v), v.size,
                                        q.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), q.size, _dp(out)):
            raise RuntimeError("orc_helix_back_voxels failed")
        return out

    def source_z(self, v: int) -> float:
        return float(_lib().orc_helix_source_z(ctypes.byref(self._g), int(v)))

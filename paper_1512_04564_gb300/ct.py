"""Thin Python binding of the C ABI in ``include/ct.h`` (argument marshalling only).

Every computation runs in the CUDA library ``_build/libct.so``; PyTorch only
supplies device memory and streams.  Importing this module loads the
library and raises if it is missing -- there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libct.so")

CT_OK, CT_EINVAL, CT_ENOMEM, CT_ECUDA, CT_ETIMEOUT, CT_ENOTSUP = range(6)
CT_FAN_ARC_2D = 1
CURVATURES = {"huber": 0, "max": 1}
CT_HELICAL_CONE_ARC = 2
AXIAL = {"rect": 0, "trap": 1}  # CT_AXIAL_RECT (SF-TR), CT_AXIAL_TRAP (SF-TT)
CT_POT_HYPERBOLA, CT_POT_FAIR, CT_POT_QUADRATIC = 0, 1, 2
CT_ALG_PROPOSED, CT_ALG_SIMPLE = 0, 1
CT_FBP_RAMP, CT_FBP_HANN = 0, 1
POTENTIALS = {"hyperbola": CT_POT_HYPERBOLA, "fair": CT_POT_FAIR, "quadratic": CT_POT_QUADRATIC}
ALGORITHMS = {"proposed": CT_ALG_PROPOSED, "simple": CT_ALG_SIMPLE}


class ct_geom_desc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("offset_x", ctypes.c_double), ("offset_y", ctypes.c_double), ("offset_z", ctypes.c_double),
        ("ns", ctypes.c_int), ("nt", ctypes.c_int), ("na", ctypes.c_int),
        ("ds", ctypes.c_double), ("dt", ctypes.c_double),
        ("offset_s", ctypes.c_double), ("offset_t", ctypes.c_double),
        ("dso", ctypes.c_double), ("dsd", ctypes.c_double),
        ("orbit_deg", ctypes.c_double), ("orbit_start_deg", ctypes.c_double),
        ("pitch", ctypes.c_double), ("axial", ctypes.c_int),
    ]


class ct_solve_params(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_int), ("n_iter", ctypes.c_int),
        ("alpha", ctypes.c_float), ("beta", ctypes.c_float), ("delta", ctypes.c_float),
        ("potential", ctypes.c_int), ("algorithm", ctypes.c_int), ("nonneg", ctypes.c_int),
        ("continuation", ctypes.c_int), ("rho_fixed", ctypes.c_float),
        ("x_ref", ctypes.c_void_p), ("hu_per_unit", ctypes.c_float), ("fov_radius", ctypes.c_float),
        ("stop_rmsd_hu", ctypes.c_float), ("init_fbp", ctypes.c_int), ("curvature", ctypes.c_int),
        ("dl_scale", ctypes.c_float), ("kappa", ctypes.c_void_p),
        ("start_iter", ctypes.c_int), ("g_state", ctypes.c_void_p), ("h_state", ctypes.c_void_p),
    ]


class ct_solve_report(ctypes.Structure):
    _fields_ = [
        ("iters_done", ctypes.c_int),
        ("seconds", ctypes.c_double), ("seconds_to_tol", ctypes.c_double),
        ("rmsd_hu_last", ctypes.c_float),
        ("rmsd_trace_hu", ctypes.POINTER(ctypes.c_float)),
        ("iter_seconds", ctypes.POINTER(ctypes.c_double)),
    ]


class ct_unet_desc(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int), ("base_channels", ctypes.c_int), ("height", ctypes.c_int), ("width", ctypes.c_int),
        ("max_batch", ctypes.c_int), ("in_scale", ctypes.c_float), ("seed", ctypes.c_ulonglong),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ip, cint, cfl = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_float
    sigs = {
        "ct_geom_create": [ctypes.POINTER(ct_geom_desc), ctypes.POINTER(vp)],
        "ct_forward": [vp, vp, vp, ip, cint, vp],
        "ct_pack_image": [vp, vp, vp, vp],
        "ct_forward_packed": [vp, vp, vp, ip, cint, vp],
        "ct_back": [vp, vp, vp, ip, cint, cfl, cint, vp],
        "ct_sqs_diag": [vp, vp, vp, vp],
        "ct_sqs_diag_noalloc": [vp, vp, vp, vp],
        "ct_fbp": [vp, vp, vp, cint, vp],
        "ct_geom_precompute": [vp, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_ulonglong), vp],
        "ct_geom_matrix_info": [vp, ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)],
        "ct_geom_autotune": [vp, cint, ip, ip, vp],
        "ct_reg_gradient": [vp, vp, vp, cfl, cfl, cint, vp, vp, vp],
        "ct_kappa": [vp, vp, vp, vp],
        "ct_relaxed_oslalm_solve": [vp, vp, vp, ctypes.POINTER(ct_solve_params), vp,
                                    ctypes.POINTER(ct_solve_report), vp],
        "ct_relaxed_oslalm_solve_batched": [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                            ctypes.POINTER(ct_solve_params), ctypes.POINTER(vp), cint,
                                            ctypes.POINTER(ct_solve_report), vp],
        "ct_debug_barrier": [ctypes.c_longlong, cint],
        "ct_gemm_bf16": [vp, vp, vp, cint, cint, cint, vp, vp],
        "ct_conv3x3_bf16": [vp, cint, cint, vp, cint, vp, vp, vp, cint, cint, cint, cint, vp, vp],
        "ct_conv3x3_bf16_dgrad": [vp, cint, vp, vp, cint, cint, vp, cint, vp, vp, cint, cint, cint, vp, vp],
        "ct_conv3x3_bf16_wgrad": [vp, cint, cint, vp, cint, vp, cint, vp, vp, vp, ctypes.c_longlong, cint, cint, cint,
                                  vp, vp],
        "ct_unet_create": [ctypes.POINTER(ct_unet_desc), ctypes.POINTER(vp)],
        "ct_unet_get_params": [vp, vp, cint],
        "ct_unet_set_params": [vp, vp],
        "ct_unet_forward": [vp, vp, vp, cint, vp],
        "ct_unet_backward": [vp, vp, cint, vp],
        "ct_unet_adam": [vp, cfl, cfl, cfl, cfl, cfl, vp],
        "ct_unet_status": [vp],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = cint
    lib.ct_geom_destroy.argtypes = [vp]
    lib.ct_geom_destroy.restype = None
    lib.ct_last_error.argtypes = []
    lib.ct_last_error.restype = ctypes.c_char_p
    lib.ct_version.restype = cint
    lib.ct_unet_destroy.argtypes = [vp]
    lib.ct_unet_destroy.restype = None
    lib.ct_unet_num_params.argtypes = [vp]
    lib.ct_unet_num_params.restype = ctypes.c_longlong
    lib.ct_conv3x3_wgrad_workspace.argtypes = [cint, cint, cint, cint, cint]
    lib.ct_conv3x3_wgrad_workspace.restype = ctypes.c_longlong
    return lib


_lib = _load()
EXPORTED = ("ct_geom_create", "ct_geom_destroy", "ct_geom_precompute", "ct_geom_matrix_info", "ct_geom_autotune",
            "ct_forward",
            "ct_pack_image", "ct_forward_packed", "ct_back", "ct_sqs_diag",
            "ct_sqs_diag_noalloc", "ct_fbp", "ct_reg_gradient", "ct_kappa", "ct_relaxed_oslalm_solve",
            "ct_relaxed_oslalm_solve_batched", "ct_debug_barrier", "ct_last_error", "ct_version", "ct_gemm_bf16", "ct_conv3x3_bf16",
            "ct_conv3x3_bf16_dgrad", "ct_conv3x3_wgrad_workspace", "ct_conv3x3_bf16_wgrad", "ct_unet_create",
            "ct_unet_destroy", "ct_unet_num_params", "ct_unet_get_params", "ct_unet_set_params", "ct_unet_forward",
            "ct_unet_backward", "ct_unet_adam", "ct_unet_status")


class CTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ct status {status}: {msg}")
        self.status = status


def _check(st: int):
    if st != CT_OK:
        raise CTError(st, _lib.ct_last_error().decode())


def _ptr(t: torch.Tensor | None, name: str, numel: int | None = None, dtype=torch.float32):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _views(views, na):
    if views is None:
        return None, na
    arr = (ctypes.c_int * len(views))(*[int(v) for v in views])
    return arr, len(views)


class Geometry:
    """Owner of a ``ct_geom`` handle (``ct_geom_create`` / ``ct_geom_destroy``).

    2-D fan-beam scans (``kind=CT_FAN_ARC_2D``) use images ``[ny][nx]`` and
    sinograms ``[view][ns]``; helical cone-beam scans (``CT_HELICAL_CONE_ARC``)
    volumes ``[nz][ny][nx]`` and sinograms ``[view][nt][ns]``.
    """

    def __init__(self, *, nx, ny, dx, dy, ns, ds, na, dso, dsd, offset_x=0.0, offset_y=0.0, offset_s=0.0,
                 orbit_deg=360.0, orbit_start_deg=0.0, kind=CT_FAN_ARC_2D, nz=1, dz=1.0, offset_z=0.0, nt=1,
                 dt=1.0, offset_t=0.0, pitch=0.0, axial="rect"):
        d = ct_geom_desc()
        d.kind = kind
        d.nx, d.ny, d.nz = nx, ny, nz
        d.dx, d.dy, d.dz = dx, dy, dz
        d.offset_x, d.offset_y, d.offset_z = offset_x, offset_y, offset_z
        d.ns, d.nt, d.na = ns, nt, na
        d.ds, d.dt, d.offset_s, d.offset_t = ds, dt, offset_s, offset_t
        d.dso, d.dsd = dso, dsd
        d.orbit_deg, d.orbit_start_deg = orbit_deg, orbit_start_deg
        d.pitch = pitch
        d.axial = AXIAL[axial] if isinstance(axial, str) else int(axial)
        self.desc = d
        self.kind = kind
        self.nx, self.ny, self.ns, self.na = nx, ny, ns, na
        self.nz, self.nt = (nz, nt) if kind == CT_HELICAL_CONE_ARC else (1, 1)
        h = ctypes.c_void_p()
        _check(_lib.ct_geom_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h

    @property
    def nvox(self) -> int:
        """Pixels (2-D) or voxels (3-D) of the image."""
        return self.nx * self.ny * self.nz

    @property
    def view_len(self) -> int:
        """Detector cells per view."""
        return self.ns * self.nt

    @property
    def image_shape(self) -> tuple:
        return (self.nz, self.ny, self.nx) if self.kind == CT_HELICAL_CONE_ARC else (self.ny, self.nx)

    @property
    def view_shape(self) -> tuple:
        return (self.nt, self.ns) if self.kind == CT_HELICAL_CONE_ARC else (self.ns,)

    @classmethod
    def from_fan(cls, g) -> "Geometry":
        return cls(nx=g.nx, ny=g.ny, dx=g.dx, dy=g.dy, ns=g.ns, ds=g.ds, na=g.na, dso=g.dso, dsd=g.dsd,
                   offset_x=g.offset_x, offset_y=g.offset_y, offset_s=g.offset_s, orbit_deg=g.orbit_deg,
                   orbit_start_deg=g.orbit_start_deg)

    @classmethod
    def from_helix(cls, g) -> "Geometry":
        return cls(nx=g.nx, ny=g.ny, dx=g.dx, dy=g.dy, ns=g.ns, ds=g.ds, na=g.na, dso=g.dso, dsd=g.dsd,
                   offset_x=g.offset_x, offset_y=g.offset_y, offset_s=g.offset_s, orbit_deg=g.orbit_deg,
                   orbit_start_deg=g.orbit_start_deg, kind=CT_HELICAL_CONE_ARC, nz=g.nz, dz=g.dz,
                   offset_z=g.offset_z, nt=g.nt, dt=g.dt, offset_t=g.offset_t, pitch=g.pitch,
                   axial=getattr(g, "axial", "rect"))

    @classmethod
    def from_scan(cls, g) -> "Geometry":
        """From a fan-beam or helical scan description (anything with the same fields)."""
        return cls.from_helix(g) if hasattr(g, "nz") else cls.from_fan(g)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.ct_geom_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ct_geom_precompute(geom: Geometry, max_bytes: int = 0, stream=None) -> int:
    """Build the resident system matrix; returns its size in bytes."""
    b = ctypes.c_ulonglong(0)
    _check(_lib.ct_geom_precompute(geom.handle, ctypes.c_ulonglong(int(max_bytes)), ctypes.byref(b), _stream(stream)))
    return int(b.value)


def ct_geom_matrix_info(geom: Geometry) -> tuple[int, int]:
    """(bytes of the resident matrix, bytes of its back-projector records)."""
    m, r = ctypes.c_ulonglong(0), ctypes.c_ulonglong(0)
    _check(_lib.ct_geom_matrix_info(geom.handle, ctypes.byref(m), ctypes.byref(r)))
    return int(m.value), int(r.value)


FP_VARIANTS = {1: "resident rows", 2: "bundle", 3: "ray"}
BP_VARIANTS = {1: "stored footprints", 2: "on the fly"}


def ct_geom_autotune(geom: Geometry, views_per_launch: int = 0, stream=None) -> tuple[str, str]:
    """Time the projector decompositions available for this geometry and keep the fastest."""
    f, b = ctypes.c_int(0), ctypes.c_int(0)
    _check(_lib.ct_geom_autotune(geom.handle, int(views_per_launch), ctypes.byref(f), ctypes.byref(b),
                                 _stream(stream)))
    return FP_VARIANTS[f.value], BP_VARIANTS[b.value]


def ct_forward(geom: Geometry, x: torch.Tensor, y: torch.Tensor, views=None, stream=None) -> torch.Tensor:
    arr, nv = _views(views, geom.na)
    _check(_lib.ct_forward(geom.handle, _ptr(x, "x", geom.nvox), _ptr(y, "y", nv * geom.view_len), arr, nv,
                           _stream(stream)))
    return y


def ct_pack_image(geom: Geometry, x: torch.Tensor, xpack: torch.Tensor, stream=None) -> torch.Tensor:
    """[x | x^T] (2 nx ny floats) of a 2-D image, the layout the resident matrix's rows index."""
    _check(_lib.ct_pack_image(geom.handle, _ptr(x, "x", geom.nvox), _ptr(xpack, "xpack", 2 * geom.nvox),
                              _stream(stream)))
    return xpack


def ct_forward_packed(geom: Geometry, xpack: torch.Tensor, y: torch.Tensor, views=None, stream=None) -> torch.Tensor:
    """ct_forward of an image packed by ct_pack_image."""
    arr, nv = _views(views, geom.na)
    _check(_lib.ct_forward_packed(geom.handle, _ptr(xpack, "xpack", 2 * geom.nvox),
                                  _ptr(y, "y", nv * geom.view_len), arr, nv, _stream(stream)))
    return y


def ct_back(geom: Geometry, y: torch.Tensor, x: torch.Tensor, views=None, scale=1.0, accumulate=False,
            stream=None) -> torch.Tensor:
    arr, nv = _views(views, geom.na)
    _check(_lib.ct_back(geom.handle, _ptr(y, "y", nv * geom.view_len), _ptr(x, "x", geom.nvox), arr, nv,
                        float(scale), int(bool(accumulate)), _stream(stream)))
    return x


def ct_sqs_diag(geom: Geometry, w: torch.Tensor, d_l: torch.Tensor, stream=None) -> torch.Tensor:
    _check(_lib.ct_sqs_diag(geom.handle, _ptr(w, "w", geom.na * geom.view_len), _ptr(d_l, "d_l", geom.nvox),
                            _stream(stream)))
    return d_l


def ct_sqs_diag_noalloc(geom: Geometry, w: torch.Tensor, d_l: torch.Tensor, stream=None) -> torch.Tensor:
    """ct_sqs_diag without device allocation (scratch in a fixed 4 MiB library array; na*ns <= 2^20)."""
    _check(_lib.ct_sqs_diag_noalloc(geom.handle, _ptr(w, "w", geom.na * geom.view_len),
                                    _ptr(d_l, "d_l", geom.nvox), _stream(stream)))
    return d_l


def ct_fbp(geom: Geometry, y: torch.Tensor, x: torch.Tensor, window: str = "hann", stream=None) -> torch.Tensor:
    """Full-scan equiangular fan-beam FBP (initial image of Algorithm 1); for a helical geometry, per slice the
    fan-beam FBP of its single-slice rebinning."""
    win = {"ramp": CT_FBP_RAMP, "hann": CT_FBP_HANN}[window] if isinstance(window, str) else int(window)
    _check(_lib.ct_fbp(geom.handle, _ptr(y, "y", geom.na * geom.view_len), _ptr(x, "x", geom.nvox), win,
                       _stream(stream)))
    return x


def ct_reg_gradient(geom: Geometry, x: torch.Tensor, beta: float, delta: float, potential: str | int,
                    grad: torch.Tensor, curv: torch.Tensor | None = None, kappa: torch.Tensor | None = None,
                    stream=None):
    pot = POTENTIALS[potential] if isinstance(potential, str) else int(potential)
    n = geom.nvox
    _check(_lib.ct_reg_gradient(geom.handle, _ptr(x, "x", n), _ptr(kappa, "kappa", n), float(beta), float(delta),
                                pot, _ptr(grad, "grad", n), _ptr(curv, "curv", n), _stream(stream)))
    return grad, curv


def ct_kappa(geom: Geometry, w: torch.Tensor, kappa: torch.Tensor, stream=None) -> torch.Tensor:
    """Resolution-uniformity voxel weights kappa_j = sqrt([A'w]_j / [A'1]_j) (0 where no ray meets voxel j)."""
    _check(_lib.ct_kappa(geom.handle, _ptr(w, "w", geom.na * geom.view_len), _ptr(kappa, "kappa", geom.nvox),
                         _stream(stream)))
    return kappa


def ct_relaxed_oslalm_solve(geom: Geometry, y: torch.Tensor, w: torch.Tensor, x: torch.Tensor, *, M: int,
                            n_iter: int, alpha: float, beta: float, delta: float, potential="hyperbola",
                            algorithm="proposed", nonneg=True, continuation=True, rho_fixed=0.0,
                            x_ref: torch.Tensor | None = None, hu_per_unit=1.0, fov_radius=0.0,
                            stop_rmsd_hu=0.0, init_fbp=False, curvature="huber", dl_scale=1.0,
                            kappa: torch.Tensor | None = None, start_iter=0, g_state: torch.Tensor | None = None,
                            h_state: torch.Tensor | None = None, stream=None) -> dict:
    """Relaxed OS-LALM (Algorithm 1 / 2); x is updated in place.  Returns the report as a dict.
    g_state, h_state: optional image tensors that receive the final g and h (a checkpoint with x and the
    iteration count); start_iter > 0 resumes from them after that many outer iterations."""
    n = geom.nvox
    p = _params(geom, M=M, n_iter=n_iter, alpha=alpha, beta=beta, delta=delta, potential=potential,
                algorithm=algorithm, nonneg=nonneg, continuation=continuation, rho_fixed=rho_fixed, x_ref=x_ref,
                hu_per_unit=hu_per_unit, fov_radius=fov_radius, stop_rmsd_hu=stop_rmsd_hu, init_fbp=init_fbp,
                curvature=curvature, dl_scale=dl_scale, kappa=kappa)
    p.start_iter = int(start_iter)
    p.g_state = _ptr(g_state, "g_state", n)
    p.h_state = _ptr(h_state, "h_state", n)
    r, trace, its = _report(n_iter)
    _check(_lib.ct_relaxed_oslalm_solve(geom.handle, _ptr(y, "y", geom.na * geom.view_len), _ptr(w, "w", geom.na * geom.view_len),
                                        ctypes.byref(p), _ptr(x, "x", n), ctypes.byref(r), _stream(stream)))
    return _report_dict(r, trace, its, x_ref is not None)


def _params(geom, *, M, n_iter, alpha, beta, delta, potential="hyperbola", algorithm="proposed", nonneg=True,
            continuation=True, rho_fixed=0.0, x_ref=None, hu_per_unit=1.0, fov_radius=0.0, stop_rmsd_hu=0.0,
            init_fbp=False, curvature="huber", dl_scale=1.0, kappa=None):
    n = geom.nvox
    p = ct_solve_params()
    p.M, p.n_iter, p.alpha, p.beta, p.delta = M, n_iter, alpha, beta, delta
    p.potential = POTENTIALS[potential] if isinstance(potential, str) else int(potential)
    p.algorithm = ALGORITHMS[algorithm] if isinstance(algorithm, str) else int(algorithm)
    p.nonneg, p.continuation, p.rho_fixed = int(bool(nonneg)), int(bool(continuation)), float(rho_fixed)
    p.x_ref = _ptr(x_ref, "x_ref", n)
    p.hu_per_unit, p.fov_radius, p.stop_rmsd_hu = hu_per_unit, fov_radius, stop_rmsd_hu
    p.init_fbp = int(bool(init_fbp))
    p.curvature = CURVATURES[curvature] if isinstance(curvature, str) else int(curvature)
    p.dl_scale = float(dl_scale)
    p.kappa = _ptr(kappa, "kappa", n)
    return p


def _report(n_iter):
    r = ct_solve_report()
    trace = (ctypes.c_float * max(n_iter, 1))()
    its = (ctypes.c_double * max(n_iter, 1))()
    r.rmsd_trace_hu = ctypes.cast(trace, ctypes.POINTER(ctypes.c_float))
    r.iter_seconds = ctypes.cast(its, ctypes.POINTER(ctypes.c_double))
    return r, trace, its


def _report_dict(r, trace, its, has_ref):
    k = r.iters_done
    return {
        "iters_done": k,
        "seconds": r.seconds,
        "seconds_to_tol": r.seconds_to_tol,
        "rmsd_hu_last": r.rmsd_hu_last,
        "rmsd_trace_hu": list(trace[:k]) if has_ref else [],
        "iter_seconds": list(its[:k]),
    }


def ct_relaxed_oslalm_solve_batched(geoms, ys, ws, xs, params: list[dict], stream=None) -> list[dict]:
    """Batched relaxed OS-LALM in one persistent launch; params[i] holds the keyword arguments of
    ct_relaxed_oslalm_solve for slice i.  Every x is updated in place.  Returns the per-slice reports."""
    n = len(geoms)
    if not (len(ys) == len(ws) == len(xs) == len(params) == n):
        raise ValueError("geoms, ys, ws, xs and params must have one entry per slice")
    VP = ctypes.c_void_p * n
    gh = VP(*[g.handle.value for g in geoms])
    yp = VP(*[_ptr(ys[i], "y", geoms[i].na * geoms[i].ns).value for i in range(n)])
    wp = VP(*[_ptr(ws[i], "w", geoms[i].na * geoms[i].ns).value for i in range(n)])
    xp = VP(*[_ptr(xs[i], "x", geoms[i].nx * geoms[i].ny).value for i in range(n)])
    P = (ct_solve_params * n)(*[_params(geoms[i], **params[i]) for i in range(n)])
    reps = [_report(params[i]["n_iter"]) for i in range(n)]
    R = (ct_solve_report * n)(*[r for r, _, _ in reps])
    _check(_lib.ct_relaxed_oslalm_solve_batched(ctypes.cast(gh, ctypes.POINTER(ctypes.c_void_p)),
                                                ctypes.cast(yp, ctypes.POINTER(ctypes.c_void_p)),
                                                ctypes.cast(wp, ctypes.POINTER(ctypes.c_void_p)), P,
                                                ctypes.cast(xp, ctypes.POINTER(ctypes.c_void_p)), n, R,
                                                _stream(stream)))
    return [_report_dict(R[i], reps[i][1], reps[i][2], params[i].get("x_ref") is not None) for i in range(n)]


def ct_debug_barrier(max_polls: int = 0, missing: int = 0) -> None:
    """Failure-detection hook of the batched persistent launch: the poll limit of every grid-barrier wait
    (0: the built-in limit) and a number of barrier participants that never arrive (0: normal operation)."""
    _check(_lib.ct_debug_barrier(int(max_polls), int(missing)))


def version() -> int:
    return int(_lib.ct_version())


def _err_flag(err):
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
    return err


def ct_gemm_bf16(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor | None = None, err=None, stream=None):
    """Tensor-core GEMM C = A B^T (A [M][K], B [N][K] bfloat16; C [M][N] float32)."""
    if A.dtype != torch.bfloat16 or B.dtype != torch.bfloat16:
        raise TypeError("A and B must be bfloat16")
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("A and B disagree on K")
    if C is None:
        C = torch.empty(M, N, dtype=torch.float32, device=A.device)
    err = _err_flag(err)
    _check(_lib.ct_gemm_bf16(_ptr(A, "A", M * K, torch.bfloat16), _ptr(B, "B", N * K, torch.bfloat16),
                             _ptr(C, "C", M * N), M, N, K, _ptr(err, "err", 1, torch.int32), _stream(stream)))
    return C, err


def _bf(t, name, numel):
    return _ptr(t, name, numel, torch.bfloat16)


def ct_conv3x3_bf16(in1, c1, up1, in2, c2, w, bias, out, B, H, W, co, err=None, stream=None):
    """out = bf16(relu(conv3x3(cat(up?(in1), in2)) + bias)); NHWC bfloat16 tensors."""
    h1, w1 = (H // 2, W // 2) if up1 else (H, W)
    err = _err_flag(err)
    _check(_lib.ct_conv3x3_bf16(_bf(in1, "in1", B * h1 * w1 * c1), c1, int(bool(up1)),
                                _bf(in2, "in2", B * H * W * c2) if c2 else None, c2,
                                _bf(w, "w", co * 9 * (c1 + c2)), _ptr(bias, "bias", co),
                                _bf(out, "out", B * H * W * co), B, H, W, co, _ptr(err, "err", 1, torch.int32),
                                _stream(stream)))
    return out, err


def ct_conv3x3_bf16_dgrad(gout, co, wt, m1, c1, up1, m2, c2, g1, g2, B, H, W, err=None, stream=None):
    h1, w1 = (H // 2, W // 2) if up1 else (H, W)
    err = _err_flag(err)
    _check(_lib.ct_conv3x3_bf16_dgrad(_bf(gout, "gout", B * H * W * co), co, _bf(wt, "wt", co * 9 * (c1 + c2)),
                                      _bf(m1, "m1", B * h1 * w1 * c1), c1, int(bool(up1)),
                                      _bf(m2, "m2", B * H * W * c2) if c2 else None, c2,
                                      _bf(g1, "g1", B * H * W * c1), _bf(g2, "g2", B * H * W * c2) if c2 else None,
                                      B, H, W, _ptr(err, "err", 1, torch.int32), _stream(stream)))
    return g1, g2, err


def ct_conv3x3_wgrad_workspace(B, H, W, ci, co) -> int:
    return int(_lib.ct_conv3x3_wgrad_workspace(B, H, W, ci, co))


def ct_conv3x3_bf16_wgrad(in1, c1, up1, in2, c2, gout, co, dw, db, B, H, W, work=None, err=None, stream=None):
    h1, w1 = (H // 2, W // 2) if up1 else (H, W)
    nwork = ct_conv3x3_wgrad_workspace(B, H, W, c1 + c2, co)
    if work is None:
        work = torch.empty(max(nwork, 1), dtype=torch.float32, device="cuda")
    err = _err_flag(err)
    _check(_lib.ct_conv3x3_bf16_wgrad(_bf(in1, "in1", B * h1 * w1 * c1), c1, int(bool(up1)),
                                      _bf(in2, "in2", B * H * W * c2) if c2 else None, c2,
                                      _bf(gout, "gout", B * H * W * co), co, _ptr(dw, "dw", co * 9 * (c1 + c2)),
                                      _ptr(db, "db", co), _ptr(work, "work"), work.numel(), B, H, W,
                                      _ptr(err, "err", 1, torch.int32), _stream(stream)))
    return dw, db, err


class UNet:
    """Owner of a ``ct_unet`` handle (ct_unet_create / ct_unet_destroy)."""

    def __init__(self, *, levels=4, base_channels=32, height=256, width=256, max_batch=8, in_scale=50.0, seed=0):
        d = ct_unet_desc(levels, base_channels, height, width, max_batch, in_scale, seed)
        h = ctypes.c_void_p()
        _check(_lib.ct_unet_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.levels, self.base_channels, self.height, self.width = levels, base_channels, height, width
        self.max_batch, self.in_scale = max_batch, in_scale

    @property
    def num_params(self) -> int:
        return int(_lib.ct_unet_num_params(self.handle))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.ct_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ct_unet_num_params(net: UNet) -> int:
    return net.num_params


def ct_unet_get_params(net: UNet, which: str = "params"):
    import numpy as np

    out = np.empty(net.num_params, dtype=np.float32)
    _check(_lib.ct_unet_get_params(net.handle, out.ctypes.data_as(ctypes.c_void_p), 0 if which == "params" else 1))
    return out


def ct_unet_set_params(net: UNet, params):
    import numpy as np

    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != net.num_params:
        raise ValueError(f"expected {net.num_params} parameters, got {a.size}")
    _check(_lib.ct_unet_set_params(net.handle, a.ctypes.data_as(ctypes.c_void_p)))


def ct_unet_forward(net: UNet, x: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    B = x.shape[0]
    if y is None:
        y = torch.empty_like(x)
    n = B * net.height * net.width
    _check(_lib.ct_unet_forward(net.handle, _ptr(x, "x", n), _ptr(y, "y", n), B, _stream(stream)))
    return y


def ct_unet_backward(net: UNet, gy: torch.Tensor, stream=None):
    B = gy.shape[0]
    _check(_lib.ct_unet_backward(net.handle, _ptr(gy, "gy", B * net.height * net.width), B, _stream(stream)))


def ct_unet_adam(net: UNet, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
    _check(_lib.ct_unet_adam(net.handle, lr, beta1, beta2, eps, weight_decay, _stream(stream)))


def ct_unet_status(net: UNet):
    _check(_lib.ct_unet_status(net.handle))


def ct_unet_create(**kw) -> UNet:
    return UNet(**kw)


def ct_unet_destroy(net: UNet):
    net.close()

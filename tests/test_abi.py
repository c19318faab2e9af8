"""CPU checks of the C-ABI library: it builds, loads, exports every symbol that
include/ct.h declares, and rejects bad arguments on the host before any launch."""

import ctypes
import os
import re

import pytest

from paper_1512_04564_gb300 import build as ctbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = ctbuild.build()
    return ctypes.CDLL(path)


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ct_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"ct_geom_create", "ct_forward", "ct_back", "ct_sqs_diag", "ct_relaxed_oslalm_solve"} <= names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_1512_04564_gb300 import ct

    assert set(ct.EXPORTED) == _declared()
    for n in ct.EXPORTED:
        if n not in ("ct_geom_destroy", "ct_last_error", "ct_version", "ct_geom_create"):
            assert callable(getattr(ct, n))


def test_host_validation_without_gpu():
    from paper_1512_04564_gb300 import ct

    with pytest.raises(ct.CTError) as e:
        ct.Geometry(nx=16, ny=16, dx=1.0, dy=1.0, ns=32, ds=1.0, na=10, dso=100.0, dsd=180.0, kind=99)
    assert e.value.status == ct.CT_ENOTSUP
    with pytest.raises(ct.CTError) as e:
        ct.Geometry(nx=0, ny=16, dx=1.0, dy=1.0, ns=32, ds=1.0, na=10, dso=100.0, dsd=180.0)
    assert e.value.status == ct.CT_EINVAL
    with pytest.raises(ct.CTError) as e:  # image reaching the source
        ct.Geometry(nx=256, ny=256, dx=1.0, dy=1.0, ns=32, ds=1.0, na=10, dso=100.0, dsd=180.0)
    assert e.value.status == ct.CT_EINVAL
    assert "source" in str(e.value)
    with pytest.raises(ct.CTError) as e:  # negative pixel size
        ct.Geometry(nx=16, ny=16, dx=-1.0, dy=1.0, ns=32, ds=1.0, na=10, dso=100.0, dsd=180.0)
    assert e.value.status == ct.CT_EINVAL
    hx = dict(nx=16, ny=16, dx=4.0, dy=4.0, ns=64, ds=4.0, na=10, dso=250.0, dsd=450.0, kind=ct.CT_HELICAL_CONE_ARC,
              nz=80, dz=1.0, nt=8, dt=2.0, pitch=0.5, orbit_deg=360.0)
    with pytest.raises(ct.CTError) as e:  # unknown axial footprint
        ct.Geometry(**hx, axial=7)
    assert e.value.status == ct.CT_EINVAL
    with pytest.raises(ct.CTError) as e:  # trapezoid ramps wider than half a voxel (80 slices near the source)
        ct.Geometry(**hx, axial="trap")
    assert e.value.status == ct.CT_ENOTSUP and "ramp" in str(e.value)


def test_struct_layouts_match_header():
    """The binding's ctypes structs have the C structs' field order and sizes."""
    from paper_1512_04564_gb300 import ct

    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "ct.h")).read(), flags=re.S)
    for cls, cname in ((ct.ct_geom_desc, "ct_geom_desc"), (ct.ct_solve_params, "ct_solve_params"),
                       (ct.ct_solve_report, "ct_solve_report")):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + ";", src).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            names = re.sub(r"^(const\s+)?(unsigned\s+)?[a-z_0-9]+\s*\**", "", decl).split(",")
            fields += [n.strip().lstrip("*").strip() for n in names]
        assert [f[0] for f in cls._fields_] == fields, cname

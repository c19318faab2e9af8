"""Scan geometries and workload descriptions.

Geometry convention (2-D fan beam, equiangular "arc" detector):

* Image: ``nx x ny`` pixels of size ``dx x dy`` (mm); pixel (ix, iy) has its
  centre at ``x = (ix - (nx-1)/2 + offset_x) dx``, ``y = (iy - (ny-1)/2 +
  offset_y) dy``.  Arrays are stored ``[iy][ix]`` (x fastest).
* View v has angle ``beta_v = orbit_start + v * orbit / na``.  The central ray
  points from the source towards the isocentre along ``e = (cos b, sin b)``; the
  source sits at ``-dso * e``.
* Detector bin s has fan angle ``gamma_s = (s - (ns-1)/2 + offset_s) * dgamma``
  with ``dgamma = ds / dsd`` (``ds`` is the arc length of a cell at ``dsd``).
  A point P has fan angle ``atan2((P - S).e_perp, (P - S).e)`` with
  ``e_perp = (-sin b, cos b)``.
* Sinograms are stored view-major ``[view][bin]`` (bin fastest).

The numbers of the two 2-D workloads follow the paper's GE LightSpeed-type
fan geometry (Sec. IV-A: 888 channels, 984 views per turn, 0.9776 mm pixels,
source-to-isocentre 541 mm, source-to-detector 949 mm).
"""

from __future__ import annotations

import dataclasses
import math

MU_WATER_PER_MM = 0.02  # 1 HU = MU_WATER_PER_MM / 1000 per mm ("modified HU", air = 0)


@dataclasses.dataclass(frozen=True)
class FanArcGeometry:
    nx: int
    ny: int
    dx: float
    dy: float
    ns: int
    ds: float
    na: int
    dso: float
    dsd: float
    offset_x: float = 0.0
    offset_y: float = 0.0
    offset_s: float = 0.0
    orbit_deg: float = 360.0
    orbit_start_deg: float = 0.0

    @property
    def dgamma(self) -> float:
        return self.ds / self.dsd

    def betas(self):
        import numpy as np

        v = np.arange(self.na, dtype=np.float64)
        return np.deg2rad(self.orbit_start_deg + v * self.orbit_deg / self.na)

    def gammas(self):
        import numpy as np

        s = np.arange(self.ns, dtype=np.float64)
        return (s - (self.ns - 1) / 2.0 + self.offset_s) * self.dgamma

    def fov_radius(self) -> float:
        """Radius of the disk seen by every view: min(image half-width, dso*sin(half fan))."""
        half_fan = max(abs(self.gammas()[0]), abs(self.gammas()[-1])) + 0.5 * self.dgamma
        r_fan = self.dso * math.sin(half_fan)
        r_img = min(self.nx * self.dx, self.ny * self.dy) / 2.0
        return min(r_fan, r_img)

    def with_(self, **kw) -> "FanArcGeometry":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass(frozen=True)
class ScanConfig:
    name: str
    geom: FanArcGeometry
    phantom: str  # "random10" | "anthro"
    i0: float
    sigma_e: float
    beta: float  # regularization strength for images in water units (see beta_per_mm)
    delta_hu: float
    potential: str
    M: int
    alpha: float
    n_iter: int
    seed: int = 0

    @property
    def delta(self) -> float:
        """Potential parameter delta in 1/mm."""
        return self.delta_hu * MU_WATER_PER_MM / 1000.0

    @property
    def beta_per_mm(self) -> float:
        """beta for images in 1/mm.

        ``beta`` is given for images expressed in units of water attenuation
        (x / mu_water, so 1000 HU = 1); R scales with the square of the image
        unit, so the same problem in 1/mm uses beta / mu_water^2.
        """
        return self.beta / MU_WATER_PER_MM ** 2

    @property
    def hu_per_unit(self) -> float:
        """HU per 1/mm of attenuation (modified HU: air = 0, water = 1000)."""
        return 1000.0 / MU_WATER_PER_MM


# The paper sets beta "to achieve a reasonable noise-resolution trade-off"
# (Sec. IV-A) without giving a value.  With W = counts, beta = 2^10 (water
# units) leaves the problem so weakly regularized that every ordered-subsets
# variant, relaxed or not, diverges at these subset counts.  Each workload
# therefore uses the power of two that minimises RMSD(x*, phantom) on its
# seed-0 phantom (scanned 2^10 .. 2^18).
BETA_WEAK = 2.0 ** 10  # the weakly regularized value above, kept for comparison


def fan2d_128(seed: int = 0) -> ScanConfig:
    """128x128, 1 mm pixels, 256 bins x 1.0 mm, 180 views, M=10, alpha=1.999, 20 iterations."""
    g = FanArcGeometry(nx=128, ny=128, dx=1.0, dy=1.0, ns=256, ds=1.0, na=180, dso=541.0, dsd=949.0)
    return ScanConfig(
        name="fan2d_128", geom=g, phantom="random10", i0=1e5, sigma_e=5.0,
        beta=2.0 ** 14, delta_hu=10.0, potential="hyperbola", M=10, alpha=1.999, n_iter=20, seed=seed,
    )


def fan2d_512(seed: int = 0) -> ScanConfig:
    """512x512, 0.98 mm pixels, 888 bins x 1.0239 mm, 984 views, M=41, alpha=1.999, 30 iterations."""
    g = FanArcGeometry(nx=512, ny=512, dx=0.98, dy=0.98, ns=888, ds=1.0239, na=984, dso=541.0, dsd=949.0)
    return ScanConfig(
        name="fan2d_512", geom=g, phantom="anthro", i0=1e5, sigma_e=5.0,
        beta=2.0 ** 14, delta_hu=10.0, potential="hyperbola", M=41, alpha=1.999, n_iter=30, seed=seed,
    )




@dataclasses.dataclass(frozen=True)
class HelicalConeGeometry:
    """3-D helical cone-beam scan with a cylindrical (arc) detector.

    * Volume: ``nx x ny x nz`` voxels of ``dx x dy x dz`` (mm), stored
      ``[iz][iy][ix]``; voxel (ix, iy, iz) is centred at
      ``((ix-(nx-1)/2+offset_x) dx, (iy-(ny-1)/2+offset_y) dy, (iz-(nz-1)/2+offset_z) dz)``.
    * View v: transaxial angle ``beta_v = orbit_start + v * orbit / na`` (the
      orbit spans ``orbit_deg / 360`` turns); the source is at
      ``(-dso cos b, -dso sin b, z_src(b))`` with
      ``z_src = pitch * (nt dt dso / dsd) * (b - b_mid) / (2 pi)``: the table
      advances ``pitch`` times the detector's axial coverage at the
      isocentre per turn, centred on the volume at mid-scan.
    * Detector: ``ns`` cells of arc length ``ds`` at ``dsd`` (fan angle
      ``(s-(ns-1)/2+offset_s) ds/dsd``) by ``nt`` rows of height ``dt``
      (row t at height ``(t-(nt-1)/2+offset_t) dt`` on the cylinder);
      sinograms are stored ``[view][row][cell]``.
    * ``axial`` names the projector's axial footprint model: "rect" (SF-TR)
      or "trap" (SF-TT).
    """

    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    ns: int
    ds: float
    nt: int
    dt: float
    na: int
    dso: float
    dsd: float
    pitch: float
    orbit_deg: float
    orbit_start_deg: float = 0.0
    offset_x: float = 0.0
    offset_y: float = 0.0
    offset_z: float = 0.0
    offset_s: float = 0.0
    offset_t: float = 0.0
    axial: str = "rect"  # axial footprint: "rect" (SF-TR) or "trap" (SF-TT)

    @property
    def dgamma(self) -> float:
        return self.ds / self.dsd

    def betas(self):
        import numpy as np

        v = np.arange(self.na, dtype=np.float64)
        return np.deg2rad(self.orbit_start_deg + v * self.orbit_deg / self.na)

    def gammas(self):
        import numpy as np

        s = np.arange(self.ns, dtype=np.float64)
        return (s - (self.ns - 1) / 2.0 + self.offset_s) * self.dgamma

    def row_heights(self):
        import numpy as np

        t = np.arange(self.nt, dtype=np.float64)
        return (t - (self.nt - 1) / 2.0 + self.offset_t) * self.dt

    def source_z(self, beta):
        mid = math.radians(self.orbit_start_deg + 0.5 * self.orbit_deg)
        cover = self.nt * self.dt * self.dso / self.dsd
        return self.pitch * cover * (beta - mid) / (2.0 * math.pi)

    def transaxial(self) -> FanArcGeometry:
        """The fan-arc geometry of the transaxial plane (same views and cells)."""
        return FanArcGeometry(nx=self.nx, ny=self.ny, dx=self.dx, dy=self.dy, ns=self.ns, ds=self.ds, na=self.na,
                              dso=self.dso, dsd=self.dsd, offset_x=self.offset_x, offset_y=self.offset_y,
                              offset_s=self.offset_s, orbit_deg=self.orbit_deg, orbit_start_deg=self.orbit_start_deg)

    def fov_radius(self) -> float:
        return self.transaxial().fov_radius()

    def with_(self, **kw) -> "HelicalConeGeometry":
        return dataclasses.replace(self, **kw)


def helix3d_512(seed: int = 0) -> ScanConfig:
    """512x512x64 voxels of 0.98x0.98x0.625 mm; 888x32 cells of 1.0239x1.0964 mm; pitch 1;
    984 views per turn over 3 turns; 26-neighbour hyperbola regularizer; M=24, alpha=1.999, 20 iterations."""
    g = HelicalConeGeometry(nx=512, ny=512, nz=64, dx=0.98, dy=0.98, dz=0.625, ns=888, ds=1.0239, nt=32, dt=1.0964,
                            na=3 * 984, dso=541.0, dsd=949.0, pitch=1.0, orbit_deg=3 * 360.0)
    return ScanConfig(
        name="helix3d_512", geom=g, phantom="anthro3d", i0=1e5, sigma_e=5.0,
        beta=2.0 ** 14, delta_hu=10.0, potential="hyperbola", M=24, alpha=1.999, n_iter=20, seed=seed,
    )


def helix3d_64(seed: int = 0) -> ScanConfig:
    """Small helical case the oracle finishes in seconds: 64x64x16 voxels of 2x2x1.25 mm, 96x8 cells,
    pitch 1, 120 views per turn over 2 turns, M=8."""
    g = HelicalConeGeometry(nx=64, ny=64, nz=16, dx=2.0, dy=2.0, dz=1.25, ns=96, ds=2.0, nt=8, dt=2.2,
                            na=240, dso=541.0, dsd=949.0, pitch=1.0, orbit_deg=720.0)
    return ScanConfig(
        name="helix3d_64", geom=g, phantom="random3d", i0=1e5, sigma_e=5.0,
        beta=2.0 ** 14, delta_hu=10.0, potential="hyperbola", M=8, alpha=1.999, n_iter=10, seed=seed,
    )


def config_by_name(name: str, seed: int = 0) -> ScanConfig:
    return {"fan2d_128": fan2d_128, "fan2d_512": fan2d_512, "helix3d_64": helix3d_64,
            "helix3d_512": helix3d_512}[name](seed)


def warmstart_geometry(n: int = 256, pixel: float | None = None) -> FanArcGeometry:
    """Fan-beam scan of the learned-warm-start workload: n x n pixels of 0.98 * 512 / n mm by default
    (the ~500 mm field of the clinical geometry), 444 * n / 256 bins of 1.0239 * 888 / 444 mm (the
    888-channel arc at half sampling; with a smaller pixel the arc shrinks with the field), 492 * n / 256
    views.  n = 256 is the workload; smaller n with pixel = 1.96 gives its reduced-field test version."""
    px = 0.98 * 512 / n if pixel is None else pixel
    ns = 444 * n // 256
    return FanArcGeometry(nx=n, ny=n, dx=px, dy=px, ns=ns, ds=1.0239 * 888 / 444, na=492 * n // 256, dso=541.0,
                          dsd=949.0)

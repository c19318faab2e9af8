"""Relaxed OS-LALM for PWLS CT reconstruction, written step by step from the paper.

ORACLE -- test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg may import this module.

Problem (Sec. III, Eq. (ct_problem)):
    x_hat in argmin_{x in Omega} 1/2 ||y - A x||_W^2 + R(x),  Omega = {x >= 0}.
With the substitution A <- W^{1/2} A, y <- W^{1/2} y (Eq. (ct_substitution)) the
data term is L(x) = 1/2 ||W^{1/2}(A x - y)||^2, so grad L_m(x) = A_m' W_m (A_m x - y_m)
for the m-th ordered subset of views.  D_L = diag(A' W A 1) (Sec. III-A).

Algorithm 1 (proposed relaxed OS-LALM) and Algorithm 2 (simple relaxed
OS-LALM) are written in the paper's order and notation; rho follows the
continuation sequence of Eq. (dec_rho), with k counting subiterations.

Readings where the paper is silent:
* subsets are interleaved, S_m = {v : v mod M = m}, visited m = 0..M-1; the
  initial gradient uses the last subset (the paper's "M");
* subiteration t (1-based) uses rho_{t-1}, so the first uses rho_0 = 1;
* the factor M multiplies the subset gradient even when subsets are uneven;
* a pixel whose step denominator rho D_L + D_R is zero keeps its value.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Callable

import numpy as np

from . import regularizer as reg


def rho_continuation(k: int, alpha: float) -> float:
    """rho_k(alpha) of Eq. (dec_rho): 1 for k = 0, else pi/(alpha(k+1)) sqrt(1 - (pi/(2 alpha (k+1)))^2)."""
    if k == 0:
        return 1.0
    q = math.pi / (alpha * (k + 1))
    return q * math.sqrt(1.0 - (0.5 * q) ** 2)


def interleaved_subsets(na: int, M: int) -> list[np.ndarray]:
    if M < 1 or M > na:
        raise ValueError("need 1 <= M <= number of views")
    return [np.arange(m, na, M, dtype=np.int64) for m in range(M)]


@dataclasses.dataclass
class PWLSProblem:
    """PWLS CT problem with an FP64 projector (oracle)."""

    proj: object  # oracle.projector.FanProjector or oracle.helical.HelicalProjector
    y: np.ndarray  # [na][ns] (helical: [na][nt][ns])
    w: np.ndarray  # same shape as y
    beta: float
    delta: float
    potential: str = "hyperbola"
    kappa: np.ndarray | None = None  # kappa_n of Eq. (def_reg), image-shaped; None: kappa = 1

    @property
    def shape(self):
        g = self.proj.geom
        return (g.nz, g.ny, g.nx) if hasattr(g, "nz") else (g.ny, g.nx)

    def grad_L_subset(self, x: np.ndarray, views: np.ndarray) -> np.ndarray:
        """grad L_m(x) = A_m' W_m (A_m x - y_m)."""
        r = self.w[views] * (self.proj.forward(x, views) - self.y[views])
        return self.proj.back(r, views)

    def grad_L(self, x: np.ndarray) -> np.ndarray:
        return self.grad_L_subset(x, np.arange(self.proj.geom.na))

    def D_L(self) -> np.ndarray:
        """diag(A' W A 1): the SQS majorizer of A' W A (Erdogan-Fessler), over all views."""
        ones = np.ones(self.shape)
        return self.proj.back(self.w * self.proj.forward(ones))

    def cost(self, x: np.ndarray) -> float:
        r = self.proj.forward(x) - self.y
        return 0.5 * float(np.sum(self.w * r * r)) + reg.value(x, self.beta, self.delta, self.potential, self.kappa)

    def grad_R(self, x):
        return reg.gradient(x, self.beta, self.delta, self.potential, self.kappa)

    def D_R(self, x, curvature: str = "huber"):
        """SQS diagonal of R: Huber's optimal curvature omega(t) = phi'(t)/t, or the potential's maximum
        curvature phi''(0) = 1 for every pair (Sec. II-B; the supplement compares the two)."""
        if curvature == "max":
            return reg.curvature(x, self.beta, self.delta, "quadratic", self.kappa)
        return reg.curvature(x, self.beta, self.delta, self.potential, self.kappa)


def resolution_kappa(proj, w: np.ndarray) -> np.ndarray:
    """Voxel weights kappa_n of Eq. (def_reg) "for improving resolution uniformity" (Sec. III, citing
    Fessler and Rogers 1996): kappa_j = sqrt(sum_i a_ij w_i / sum_i a_ij), the square root of the
    a_ij-weighted mean of the statistical weights of the rays through voxel j, over all views; 0 where
    no ray meets the voxel.  (The cited paper weights by a_ij^2; the first power is the common
    simplification, computable with A' alone.)"""
    num = proj.back(w)
    den = proj.back(np.ones_like(w))
    safe = np.where(den > 0, den, 1.0)
    return np.where(den > 0, np.sqrt(np.maximum(num, 0.0) / safe), 0.0)


def _x_step(x, s, gR, rho, DL, DR, nonneg):
    """x+ = [x - (rho D_L + D_R)^{-1} (s + grad R(x))]_Omega; zero denominators keep x."""
    den = rho * DL + DR
    safe = np.where(den > 0, den, 1.0)
    xn = np.where(den > 0, x - (s + gR) / safe, x)
    return np.maximum(xn, 0.0) if nonneg else xn


def relaxed_os_lalm(problem: PWLSProblem, x0: np.ndarray, M: int, alpha: float, n_iter: int,
                    algorithm: str = "proposed", continuation: bool = True, rho_fixed: float | None = None,
                    nonneg: bool = True, D_L: np.ndarray | None = None,
                    callback: Callable[[int, np.ndarray], None] | None = None,
                    sub_callback: Callable[[int, np.ndarray], None] | None = None,
                    curvature: str = "huber", dl_scale: float = 1.0) -> np.ndarray:
    """Algorithm 1 ("proposed") or Algorithm 2 ("simple") of Sec. III-A.

    ``curvature`` selects the regularizer majorizer ("huber" or "max"); ``dl_scale`` multiplies
    D_L (the supplement's study of the data-term majorizer: too small diverges, larger slows).

    ``callback(k, x)`` runs after each outer iteration k = 1..n_iter and
    ``sub_callback(t, x)`` after each subiteration t = 1..n_iter*M.
    """
    if not (1.0 <= alpha < 2.0):
        raise ValueError("need 1 <= alpha < 2")
    if algorithm not in ("proposed", "simple"):
        raise ValueError(algorithm)
    na = problem.proj.geom.na
    S = interleaved_subsets(na, M)
    DL = dl_scale * (problem.D_L() if D_L is None else D_L)
    rho_of = (lambda t: rho_continuation(t, alpha)) if continuation else (lambda t: float(rho_fixed))

    x = np.array(x0, dtype=np.float64, copy=True)
    # set rho = 1, zeta = g = M grad L_M(x), h = D_L x - zeta
    zeta = M * problem.grad_L_subset(x, S[M - 1])
    g = zeta.copy()
    h = DL * x - zeta if algorithm == "proposed" else None
    t = 0  # subiterations completed
    for k in range(1, n_iter + 1):
        for m in range(M):
            rho = rho_of(t)
            if algorithm == "proposed":
                s = rho * (DL * x - h) + (1.0 - rho) * g
            else:
                s = rho * zeta + (1.0 - rho) * g
            x = _x_step(x, s, problem.grad_R(x), rho, DL, problem.D_R(x, curvature), nonneg)
            zeta = M * problem.grad_L_subset(x, S[m])
            g_new = rho / (rho + 1.0) * (alpha * zeta + (1.0 - alpha) * g) + g / (rho + 1.0)
            if algorithm == "proposed":
                h = alpha * (DL * x - zeta) + (1.0 - alpha) * h
            g = g_new
            t += 1
            if sub_callback is not None:
                sub_callback(t, x)
        if callback is not None:
            callback(k, x)
    return x


def fov_mask(geom) -> np.ndarray:
    """Pixels whose centres lie inside the disk every view sees (3-D: that disk in every slice)."""
    xc = (np.arange(geom.nx) - (geom.nx - 1) / 2.0 + geom.offset_x) * geom.dx
    yc = (np.arange(geom.ny) - (geom.ny - 1) / 2.0 + geom.offset_y) * geom.dy
    m = (xc[None, :] ** 2 + yc[:, None] ** 2) <= geom.fov_radius() ** 2
    return np.broadcast_to(m, (geom.nz,) + m.shape) if hasattr(geom, "nz") else m


def rmsd_hu(x: np.ndarray, x_ref: np.ndarray, mask: np.ndarray, hu_per_unit: float) -> float:
    """Root-mean-square difference inside ``mask``, in HU (Sec. IV: RMS difference to x*)."""
    d = (x - x_ref)[mask]
    return float(np.sqrt(np.mean(d * d))) * hu_per_unit


def kkt_residual(problem: PWLSProblem, x: np.ndarray, D: np.ndarray | None = None,
                 nonneg: bool = True) -> np.ndarray:
    """[x - D^{-1} grad Psi(x)]_Omega - x, the projected-gradient fixed-point residual."""
    if D is None:
        D = problem.D_L() + problem.D_R(x)
    grad = problem.grad_L(x) + problem.grad_R(x)
    step = x - grad / D
    return (np.maximum(step, 0.0) if nonneg else step) - x

"""Relaxed linearized AL methods on small dense problems (theory pins).

ORACLE -- test infrastructure only.

* :func:`relaxed_lalm_general` -- the practical proposed relaxed LALM with an
  explicit split variable u and multiplier mu (supplement, Sec. "Practical
  implementation of the proposed relaxed LALM"), for g(u) = 1/2 ||u - y||^2.
* :func:`relaxed_lalm_quad` -- the quadratic-loss form with g and h only
  (Sec. II-C, Eq. (relaxed_lal_iter_quad)), which Algorithm 1 specialises.
* :func:`ergodic_gap` / :func:`theorem2_bound` -- the duality gap of Eq.
  (def_dual_gap) at time-averaged iterates (Eq. (def_time_avg_vec)) and the
  bound (A + B_bar + C)/K of Theorem 2 (Eqs. (def_A), (def_B_bar), (def_C)).

phi is handled through its (diagonally weighted) proximal map and psi
through its gradient and a diagonal majorizer D_psi, as in Eq. (psi_sqs).
"""

from __future__ import annotations

from typing import Callable

import numpy as np


def soft_threshold_prox(lam: float):
    """prox of lam ||x||_1 in the metric diag(d): argmin lam||x||_1 + 1/2 ||x - z||_d^2."""
    return lambda z, d: np.sign(z) * np.maximum(np.abs(z) - lam / d, 0.0)


def nonneg_prox():
    return lambda z, d: np.maximum(z, 0.0)


def identity_prox():
    return lambda z, d: z


def _x_update(x, gamma, rho, DA, prox, grad_psi, D_psi):
    """argmin_x phi(x) + Q_psi(x; x_k) + 1/2 ||x - (rho D_A)^{-1} gamma||^2_{rho D_A}.

    Setting the smooth part's gradient to zero gives the weighted prox of phi at
    (rho D_A + D_psi)^{-1} (gamma + D_psi x_k - grad psi(x_k)).  ``D_psi`` is an
    array or a function of x_k (an iteration-dependent majorizer).
    """
    Dp = D_psi(x) if callable(D_psi) else D_psi
    Dw = rho * DA + Dp
    z = (gamma + Dp * x - grad_psi(x)) / Dw
    return prox(z, Dw)


def relaxed_lalm_quad(A: np.ndarray, y: np.ndarray, DA: np.ndarray, x0: np.ndarray, alpha: float,
                      rho_seq: Callable[[int], float], n_iter: int, prox=None,
                      grad_psi=None, D_psi=None, callback=None, g0=None, h0=None):
    """Eq. (relaxed_lal_iter_quad); by default g^0 = zeta^0 and h^0 = D_A x^0 - zeta^0.

    ``rho_seq(k)`` gives rho for the update from iterate k to k+1.  Returns
    (x, g, h) after ``n_iter`` iterations.
    """
    prox = prox or identity_prox()
    grad_psi = grad_psi or (lambda x: np.zeros_like(x))
    D_psi = np.zeros_like(np.asarray(x0, dtype=np.float64)) if D_psi is None else D_psi
    x = np.array(x0, dtype=np.float64, copy=True)
    zeta = A.T @ (A @ x - y)
    g = zeta.copy() if g0 is None else np.array(g0, dtype=np.float64, copy=True)
    h = DA * x - zeta if h0 is None else np.array(h0, dtype=np.float64, copy=True)
    for k in range(n_iter):
        rho = rho_seq(k)
        gamma = (rho - 1.0) * g + rho * h
        x = _x_update(x, gamma, rho, DA, prox, grad_psi, D_psi)
        zeta = A.T @ (A @ x - y)
        g = rho / (rho + 1.0) * (alpha * zeta + (1.0 - alpha) * g) + g / (rho + 1.0)
        h = alpha * (DA * x - zeta) + (1.0 - alpha) * h
        if callback is not None:
            callback(k + 1, x, g, h)
    return x, g, h


def relaxed_lalm_general(A: np.ndarray, y: np.ndarray, DA: np.ndarray, x0: np.ndarray, u0: np.ndarray,
                         mu0: np.ndarray, h0: np.ndarray, alpha: float, rho: float, n_iter: int,
                         prox=None, grad_psi=None, D_psi=None, callback=None):
    """Supplement's practical relaxed LALM with explicit (x, u, mu, h), g(u) = 1/2||u - y||^2.

    x-update: weighted prox at (rho D_A)^{-1}(rho A'(u - y + mu/rho) + rho h);
    r_u = alpha A x+ + (1 - alpha) u  (Eq. (relax_sv_u));
    u+ = argmin 1/2||u - y||^2 + <mu, u> + rho/2 ||r_u - u||^2 = (y - mu + rho r_u)/(1 + rho);
    mu+ = mu - rho (r_u - u+);
    h+ = alpha (D_A x+ - A'(A x+ - y)) + (1 - alpha) h.
    Returns the list of iterates (x, u, mu) for k = 1..n_iter.
    """
    prox = prox or identity_prox()
    grad_psi = grad_psi or (lambda x: np.zeros_like(x))
    D_psi = np.zeros_like(x0) if D_psi is None else D_psi
    x, u, mu, h = (np.array(v, dtype=np.float64, copy=True) for v in (x0, u0, mu0, h0))
    out = []
    for _ in range(n_iter):
        gamma = rho * (A.T @ (u - y + mu / rho)) + rho * h
        x = _x_update(x, gamma, rho, DA, prox, grad_psi, D_psi)
        Ax = A @ x
        r = alpha * Ax + (1.0 - alpha) * u
        u = (y - mu + rho * r) / (1.0 + rho)
        mu = mu - rho * (r - u)
        h = alpha * (DA * x - A.T @ (Ax - y)) + (1.0 - alpha) * h
        out.append((x.copy(), u.copy(), mu.copy()))
        if callback is not None:
            callback(x, u, mu)
    return out


def lasso_objective(x, u, y, lam):
    """f(x, u) = g(u) + h(x) = 1/2 ||u - y||^2 + lam ||x||_1."""
    return 0.5 * float(np.sum((u - y) ** 2)) + lam * float(np.sum(np.abs(x)))


def ergodic_gap(xK, uK, A, y, lam, x_hat):
    """G(w_K; w_hat) = [f(x_K, u_K) - f(x_hat, u_hat)] - <mu_hat, A x_K - u_K> (Eq. (def_dual_gap)).

    u_hat = A x_hat; mu_hat = y - A x_hat follows from the u-stationarity of the
    Lagrangian (grad g(u_hat) + mu_hat = 0).
    """
    u_hat = A @ x_hat
    mu_hat = y - u_hat
    return (lasso_objective(xK, uK, y, lam) - lasso_objective(x_hat, u_hat, y, lam)
            - float(mu_hat @ (A @ xK - uK)))


def theorem2_bound(K, A, y, DA, x0, u0, mu0, x_hat, alpha, rho, D_psi=None):
    """(A_Dpsi + B_bar + C)/K of Theorem 2 (Eqs. (def_A), (def_B_bar), (def_C))."""
    u_hat = A @ x_hat
    mu_hat = y - u_hat
    dx = x0 - x_hat
    A_term = 0.0 if D_psi is None else 0.5 * float(dx @ (D_psi * dx))
    B_bar = rho / (2.0 * alpha) * float(dx @ (DA * dx) - np.sum((A @ dx) ** 2))
    C = 1.0 / (2.0 * alpha) * (np.sqrt(rho) * np.linalg.norm(u0 - u_hat) + np.linalg.norm(mu0 - mu_hat) / np.sqrt(rho)) ** 2
    return (A_term + B_bar + C) / K

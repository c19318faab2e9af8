"""Pins of the oracle solver: Algorithm 1/2 (Sec. III-A), the continuation of
Eq. (dec_rho), and the relaxed LALM forms of Sec. II-C and the supplement.

Each pin checks the oracle against something other than itself:
* rho_k(alpha) zeroes the discriminant of the supplement's transition matrix
  T_1 (Eq. (critical_cond)) at lambda_1/L = (pi/(2 alpha (k+1)))^2;
* one step of the quadratic-loss form on 1/2||Ax||^2 is the linear map T_i
  (Eq. (def_Ti)) on (g, h) in eigen-coordinates;
* the quadratic-loss form (g, h) and the explicit (u, mu) form give the same
  x iterates on the LASSO example;
* Theorem 2's bound holds for the ergodic duality gap on that LASSO example;
* Algorithm 1 with M = 1 equals the quadratic-loss form on the weighted
  problem (A <- W^{1/2} A, Eq. (ct_substitution));
* the first subiteration is an OS-SQS step; rho = 1, alpha = 1, M = 1 is SQS
  and decreases the cost monotonically; alpha = 1 makes Algorithms 1 and 2 agree;
* with a quadratic potential and no constraint, the iterates reach the dense
  direct solution (A'WA + sum_i beta_i C_i'C_i)^{-1} A'Wy.
"""

import math

import numpy as np
import pytest

import synth
from oracle import lalm
from oracle import regularizer as reg
from oracle import solver
from oracle.projector import FanProjector

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _read_golden(name):
    vals = {}
    with open(f"{GOLDEN}/{name}") as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def _T(lam, L, rho, alpha):
    """Transition matrix T_i of the supplement's continuation analysis (Eq. (def_Ti))."""
    c = 1.0 / (rho * L)
    return np.array([
        [alpha * rho * lam / (rho + 1) * c * (rho - 1) + ((1 - alpha) * rho + 1) / (rho + 1),
         alpha * rho * lam / (rho + 1) * c * rho],
        [alpha * (L - lam) * c * (rho - 1), alpha * (L - lam) * c * rho + (1 - alpha)],
    ])


# ---------------------------------------------------------------- continuation


@pytest.mark.parametrize("alpha", [1.0, 1.5, 1.999])
def test_rho_sequence_is_critical_value(alpha):
    assert solver.rho_continuation(0, alpha) == 1.0
    for k in (1, 2, 5, 40, 400):
        rho = solver.rho_continuation(k, alpha)
        q = (math.pi / (2 * alpha * (k + 1))) ** 2  # lambda_1 / L at a restart after k+1 steps
        T = _T(q, 1.0, rho, alpha)
        tr, det = T[0, 0] + T[1, 1], T[0, 0] * T[1, 1] - T[0, 1] * T[1, 0]
        assert abs(tr * tr - 4 * det) <= 1e-12 * max(1.0, tr * tr)
        assert 0 < rho < 1


def test_rho_sequence_scales_with_alpha():
    # rho_k(alpha) is the alpha = 1 sequence evaluated at alpha (k+1) - 1 (supplement, "scaled by alpha")
    for k in (3, 10, 99):
        a = 1.999
        q = math.pi / (a * (k + 1))
        assert abs(solver.rho_continuation(k, a) - q * math.sqrt(1 - q * q / 4)) < 1e-15


@pytest.mark.parametrize("alpha,rho", [(1.0, 0.3), (1.999, 0.05), (1.5, 0.9)])
def test_quad_form_step_is_transition_matrix(alpha, rho):
    lam = np.array([0.01, 0.2, 0.7, 1.0])
    L = 1.0
    A = np.diag(np.sqrt(lam))
    y = np.zeros(4)
    DA = np.full(4, L)
    for col, (g0, h0) in enumerate([(1.0, 0.0), (0.0, 1.0)]):
        _, g1, h1 = lalm.relaxed_lalm_quad(A, y, DA, np.zeros(4), alpha, lambda k: rho, 1,
                                           g0=np.full(4, g0), h0=np.full(4, h0))
        for i in range(4):
            T = _T(lam[i], L, rho, alpha)
            assert abs(g1[i] - T[0, col]) < 1e-14
            assert abs(h1[i] - T[1, col]) < 1e-14


def test_simple_quadratic_converges_to_zero():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((30, 20))
    L = np.linalg.eigvalsh(A.T @ A).max()
    x0 = rng.standard_normal(20)
    x, _, _ = lalm.relaxed_lalm_quad(A, np.zeros(30), np.full(20, L), x0, 1.999,
                                     lambda k: solver.rho_continuation(k, 1.999), 400)
    # x_hat = 0 (supplement, continuation analysis); the iterates approach it
    assert np.linalg.norm(x) < 5e-3 * np.linalg.norm(x0)


# ---------------------------------------------------------------- LASSO example (supplement)


def _lasso_instance():
    p = _read_golden("lasso_example.txt")
    m, n, k = int(p["m"]), int(p["n"]), int(p["sparsity"])
    rng = synth.philox(int(p["seed"]), stream=11)
    A = rng.standard_normal((m, n))
    xs = np.zeros(n)
    xs[rng.choice(n, k, replace=False)] = rng.standard_normal(k)
    y = A @ xs + math.sqrt(p["noise_variance"]) * rng.standard_normal(m)
    return A, y, p["lambda"]


def _lasso_solution(A, y, lam):
    """Independent LASSO solve: FISTA, then an exact KKT solve on the detected support."""
    L = np.linalg.eigvalsh(A.T @ A).max()
    x = z = np.zeros(A.shape[1])
    t = 1.0
    for _ in range(20000):
        xn = z - A.T @ (A @ z - y) / L
        xn = np.sign(xn) * np.maximum(np.abs(xn) - lam / L, 0)
        tn = (1 + math.sqrt(1 + 4 * t * t)) / 2
        z = xn + (t - 1) / tn * (xn - x)
        x, t = xn, tn
    S = np.abs(x) > 1e-8
    sg = np.sign(x[S])
    AS = A[:, S]
    xS = np.linalg.solve(AS.T @ AS, AS.T @ y - lam * sg)
    xh = np.zeros_like(x)
    xh[S] = xS
    corr = A.T @ (y - A @ xh)
    assert np.all(np.sign(xS) == sg)
    assert np.max(np.abs(corr[S] - lam * sg)) < 1e-9
    assert np.max(np.abs(corr[~S])) <= lam * (1 + 1e-9)
    return xh


def _lasso_init(A, y):
    L = np.linalg.eigvalsh(A.T @ A).max()
    DA = np.full(A.shape[1], L)
    x0 = np.linalg.pinv(A) @ y
    u0 = A @ x0
    mu0 = y - u0
    h0 = DA * x0 - A.T @ (A @ x0 - y)
    return DA, x0, u0, mu0, h0


@pytest.mark.parametrize("alpha,rho", [(1.0, 0.5), (1.999, 0.1)])
def test_quad_form_matches_explicit_form_on_lasso(alpha, rho):
    A, y, lam = _lasso_instance()
    DA, x0, u0, mu0, h0 = _lasso_init(A, y)
    prox = lalm.soft_threshold_prox(lam)
    its = lalm.relaxed_lalm_general(A, y, DA, x0, u0, mu0, h0, alpha, rho, 60, prox=prox)
    xs_quad = []
    lalm.relaxed_lalm_quad(A, y, DA, x0, alpha, lambda k: rho, 60, prox=prox,
                           callback=lambda k, x, g, h: xs_quad.append(x.copy()))
    for (xg, _, _), xq in zip(its, xs_quad):
        assert np.max(np.abs(xg - xq)) <= 1e-9 * max(1.0, np.max(np.abs(xg)))


@pytest.mark.slow
@pytest.mark.parametrize("alpha,rho", [(1.0, 0.5), (1.999, 0.5), (1.0, 0.1), (1.999, 0.1)])
def test_theorem2_bound_on_lasso(alpha, rho):
    A, y, lam = _lasso_instance()
    xh = _lasso_solution(A, y, lam)
    DA, x0, u0, mu0, h0 = _lasso_init(A, y)
    its = lalm.relaxed_lalm_general(A, y, DA, x0, u0, mu0, h0, alpha, rho, 2000,
                                    prox=lalm.soft_threshold_prox(lam))
    xsum = np.zeros_like(x0)
    usum = np.zeros_like(u0)
    for K, (x, u, _) in enumerate(its, start=1):
        xsum += x
        usum += u
        gap = lalm.ergodic_gap(xsum / K, usum / K, A, y, lam, xh)
        bound = lalm.theorem2_bound(K, A, y, DA, x0, u0, mu0, xh, alpha, rho)
        assert gap >= -1e-9
        assert gap <= bound * (1 + 1e-9) + 1e-12, (K, gap, bound)


# ---------------------------------------------------------------- CT problem, small


def _small_ct(seed=0, nx=32, na=60, ns=64, potential="hyperbola", beta=None):
    g = synth.FanArcGeometry(nx=nx, ny=nx, dx=1.0, dy=1.0, ns=ns, ds=1.0, na=na, dso=100.0, dsd=180.0)
    E = [synth.Ellipse(0.5, -0.5, 12.0, 9.0, 0.3, 0.02), synth.Ellipse(-3.0, 2.0, 3.0, 2.0, 0.1, 0.005),
         synth.Ellipse(4.0, 3.0, 2.0, 2.0, 0.0, -0.01)]
    li = synth.fan_arc_line_integrals(E, g)
    y, w = synth.transmission_data(li, 1e5, 5.0, seed)
    unit = synth.configs.MU_WATER_PER_MM
    b = (2.0 ** 10) / unit ** 2 if beta is None else beta
    P = FanProjector(g)
    return solver.PWLSProblem(P, y, w, b, 10 * unit / 1000.0, potential), g


def test_first_subiteration_is_os_sqs():
    """rho = 1 and h = D_L x - zeta make s = zeta: x1 = [x - (D_L + D_R)^{-1}(M grad L_M(x) + grad R(x))]_Omega."""
    prob, g = _small_ct()
    M = 4
    x0 = np.full((g.ny, g.nx), 0.01)
    S = solver.interleaved_subsets(g.na, M)
    DL = prob.D_L()
    zeta = M * prob.grad_L_subset(x0, S[M - 1])
    expected = np.maximum(x0 - (zeta + prob.grad_R(x0)) / (DL + prob.D_R(x0)), 0)
    subs = []
    solver.relaxed_os_lalm(prob, x0, M, 1.999, 1, D_L=DL, sub_callback=lambda t, x: subs.append(x.copy()))
    np.testing.assert_allclose(subs[0], expected, rtol=1e-12, atol=1e-15)
    assert len(subs) == M


def test_sqs_special_case_is_monotone():
    prob, g = _small_ct(potential="hyperbola")
    x = np.zeros((g.ny, g.nx))
    DL = prob.D_L()
    costs = [prob.cost(x)]
    for _ in range(40):
        x = solver.relaxed_os_lalm(prob, x, 1, 1.0, 1, continuation=False, rho_fixed=1.0, D_L=DL)
        costs.append(prob.cost(x))
    d = np.diff(costs)
    assert np.all(d <= 1e-12 * abs(costs[0]))
    assert costs[-1] < 0.5 * costs[0]


def test_alpha_one_algorithms_agree():
    prob, g = _small_ct()
    x0 = np.zeros((g.ny, g.nx))
    a = solver.relaxed_os_lalm(prob, x0, 5, 1.0, 4, algorithm="proposed")
    b = solver.relaxed_os_lalm(prob, x0, 5, 1.0, 4, algorithm="simple")
    np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-13)
    c = solver.relaxed_os_lalm(prob, x0, 5, 1.999, 4, algorithm="simple")
    assert np.max(np.abs(a - c)) > 1e-6  # relaxation does change the iterates


def test_algorithm1_equals_quad_form_with_weights():
    prob, g = _small_ct(nx=16, na=30, ns=40)
    P = prob.proj
    A = P.matrix()
    sw = np.sqrt(prob.w.reshape(-1))
    Aw, yw = sw[:, None] * A, sw * prob.y.reshape(-1)
    DL = prob.D_L()
    x0 = np.full(g.nx * g.ny, 0.005)
    for alpha in (1.0, 1.999):
        ref, _, _ = lalm.relaxed_lalm_quad(
            Aw, yw, DL.reshape(-1), x0, alpha, lambda k: solver.rho_continuation(k, alpha), 15,
            prox=lalm.nonneg_prox(),
            grad_psi=lambda x: reg.gradient(x.reshape(g.ny, g.nx), prob.beta, prob.delta, prob.potential).reshape(-1),
            D_psi=lambda x: reg.curvature(x.reshape(g.ny, g.nx), prob.beta, prob.delta, prob.potential).reshape(-1))
        got = solver.relaxed_os_lalm(prob, x0.reshape(g.ny, g.nx), 1, alpha, 15, D_L=DL)
        np.testing.assert_allclose(got.reshape(-1), ref, rtol=1e-9, atol=1e-12)


@pytest.mark.slow
def test_dense_direct_solve_quadratic_32():
    prob, g = _small_ct(potential="quadratic", beta=2.0e6)
    A = prob.proj.matrix()
    W = prob.w.reshape(-1)
    H = A.T @ (W[:, None] * A)
    ny, nx = g.ny, g.nx
    for d, bi in zip(reg.DIRECTIONS_2D, reg.direction_weights(prob.beta)):
        C = []
        for iy in range(ny):
            for ix in range(nx):
                jx, jy = ix + d[0], iy + d[1]
                if 0 <= jx < nx and 0 <= jy < ny:
                    r = np.zeros(ny * nx)
                    r[iy * nx + ix], r[jy * nx + jx] = 1.0, -1.0
                    C.append(r)
        C = np.array(C)
        H += bi * C.T @ C
    x_hat = np.linalg.solve(H, A.T @ (W * prob.y.reshape(-1)))
    x = solver.relaxed_os_lalm(prob, np.zeros((ny, nx)), 1, 1.999, 1500, nonneg=False)
    assert np.linalg.norm(x.reshape(-1) - x_hat) <= 1e-6 * np.linalg.norm(x_hat)
    # KKT residual of the direct solution is ~0, of a perturbed image is not
    r0 = solver.kkt_residual(prob, x_hat.reshape(ny, nx), nonneg=False)
    assert np.sqrt(np.mean(r0 ** 2)) < 1e-9 * np.abs(x_hat).max()
    r1 = solver.kkt_residual(prob, x_hat.reshape(ny, nx) * 1.01, nonneg=False)
    assert np.sqrt(np.mean(r1 ** 2)) > 1e-4 * np.abs(x_hat).max()


def test_max_curvature_majorizer_is_larger_and_monotone():
    """The maximum-curvature D_R bounds Huber's from above (omega <= phi''(0) = 1) and, as an SQS
    majorizer, keeps the plain SQS special case monotone."""
    prob, g = _small_ct(potential="hyperbola")
    rng = np.random.default_rng(9)
    x = rng.random((g.ny, g.nx)) * 0.03
    assert np.all(prob.D_R(x, "max") >= prob.D_R(x, "huber") - 1e-15)
    x = np.zeros((g.ny, g.nx))
    DL = prob.D_L()
    costs = [prob.cost(x)]
    for _ in range(30):
        x = solver.relaxed_os_lalm(prob, x, 1, 1.0, 1, continuation=False, rho_fixed=1.0, D_L=DL, curvature="max")
        costs.append(prob.cost(x))
    assert np.all(np.diff(costs) <= 1e-12 * abs(costs[0]))


def test_dl_scale_enters_as_kappa_times_dl():
    """dl_scale = k gives the same iterates as passing k * D_L explicitly."""
    prob, g = _small_ct()
    DL = prob.D_L()
    x0 = np.zeros((g.ny, g.nx))
    a = solver.relaxed_os_lalm(prob, x0, 2, 1.5, 3, dl_scale=2.0)
    b = solver.relaxed_os_lalm(prob, x0, 2, 1.5, 3, D_L=2.0 * DL)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-15)

"""Pins for the IBSN oracle (oracle/ibsn.py), CPU only.

Each test checks the oracle against something other than itself: finite
differences of L^k, the theorems of Sec. 3-4, hand-derived optima, and the
exact LP references of oracle/lp.py.  Rectangular m != n shapes are used so a
transposed operand cannot pass.
"""

import json
import os

import numpy as np
import pytest

from oracle import ibsn as O
from oracle import lp
from workloads import uniform_points_problem, grid_problem, square_index_cost

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_lp_cases.json")


def _state(seed=0, m=7, n=5, eta=0.05, k_outer=2):
    """A random outer iterate log X^k built with the oracle's own outer update."""
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 1, (m, n))
    a = rng.uniform(0.1, 1, m); a /= a.sum()
    b = rng.uniform(0.1, 1, n); b /= b.sum()
    logX = O.initial_log_plan(a, b)
    for _ in range(k_outer):
        g = rng.normal(0, eta, n)
        logX = np.log(a)[:, None] + O.log_plan(logX, C, eta, g)
    gamma = rng.normal(0, eta, n)
    return C, a, b, eta, logX, gamma


# --- Eq. 5-7 -------------------------------------------------------------------

def test_gradient_matches_central_differences():
    C, a, b, eta, logX, gamma = _state()
    g = O.gradient(O.plan(logX, C, eta, gamma), a, b)
    h = 1e-6 * eta
    fd = np.array([(O.semi_dual_objective(logX, C, a, b, eta, gamma + h * e)
                    - O.semi_dual_objective(logX, C, a, b, eta, gamma - h * e)) / (2 * h)
                   for e in np.eye(len(b))])
    assert np.abs(fd - g).max() <= 1e-7


def test_hessian_matches_differences_of_gradient():
    C, a, b, eta, logX, gamma = _state(seed=1)
    H = O.hessian(O.plan(logX, C, eta, gamma), a, eta)
    h = 1e-6 * eta
    cols = []
    for e in np.eye(len(b)):
        gp = O.gradient(O.plan(logX, C, eta, gamma + h * e), a, b)
        gm = O.gradient(O.plan(logX, C, eta, gamma - h * e), a, b)
        cols.append((gp - gm) / (2 * h))
    fd = np.array(cols).T
    assert np.abs(fd - H).max() <= 1e-5 * np.abs(H).max()


def test_plan_rows_sum_to_one_and_gradient_sums_to_zero():
    C, a, b, eta, logX, gamma = _state(seed=2, m=9, n=4)
    P = O.plan(logX, C, eta, gamma)
    assert np.allclose(P.sum(1), 1.0, atol=1e-15)
    assert abs(O.gradient(P, a, b).sum()) <= 1e-15


def test_semi_dual_shift_invariance():
    """L^k(gamma + c 1) = L^k(gamma) because 1^T a = 1^T b = 1 (Eq. 1, Eq. 5)."""
    C, a, b, eta, logX, gamma = _state(seed=3)
    L0 = O.semi_dual_objective(logX, C, a, b, eta, gamma)
    L1 = O.semi_dual_objective(logX, C, a, b, eta, gamma + 0.37)
    assert abs(L0 - L1) <= 1e-14


@pytest.mark.parametrize("shape", [(30, 25), (12, 40)])
def test_semi_dual_value_matches_entropic_primal_at_optimum(shape):
    """Strong duality of the k = 0 subproblem (Eq. 2 with X^0 = a b^T, Eq. 5):
    at the optimal gamma the entropic primal <C, X> + eta KL(X || a b^T) of
    X = diag(a) P(gamma) equals -L^0(gamma) + eta sum_i a_i log a_i.  Pins the
    value of L (not only its gradient), including its constant terms."""
    m, n = shape
    p = uniform_points_problem(m, n, seed=4, eta=5e-2)
    logX = O.initial_log_plan(p.a, p.b)
    g, _, gn = O.sinkhorn_warmup(logX, p.C, p.a, p.b, p.eta, np.zeros(n), 1e-13, 100000)
    assert gn < 1e-12
    L = O.semi_dual_objective(logX, p.C, p.a, p.b, p.eta, g)
    X = p.a[:, None] * O.plan(logX, p.C, p.eta, g)
    primal = (p.C * X).sum() + p.eta * (X * np.log(X / np.outer(p.a, p.b))).sum()
    assert abs(primal - (-L + p.eta * (p.a @ np.log(p.a)))) <= 1e-12
    # and L^0 is minimised there: any other start has a larger value
    rng = np.random.default_rng(5)
    for _ in range(5):
        assert O.semi_dual_objective(logX, p.C, p.a, p.b, p.eta, g + rng.normal(0, 0.05, n)) > L


def test_best_zeta_is_the_two_dual_minimiser():
    """Eq. 4 zeroes dZ/dzeta of Eq. 3, and L^k = min_zeta Z^k up to the constant eta."""
    C, a, b, eta, logX, gamma = _state(seed=4)
    zeta = O.best_zeta(logX, C, a, eta, gamma)
    E = np.exp(logX + (zeta[:, None] + gamma[None, :] - C) / eta)
    assert np.allclose(E.sum(1), a, rtol=1e-13)  # dZ/dzeta_i = -a_i + sum_j ... = 0
    Z = -a @ zeta - b @ gamma + eta * E.sum()
    L = O.semi_dual_objective(logX, C, a, b, eta, gamma)
    # Z(gamma, zeta(gamma)) = L(gamma) - eta a^T log a + eta  (sum E = 1)
    assert abs(Z - (L - eta * (a @ np.log(a)) + eta)) <= 1e-13


# --- Alg. 1 and Thm 3.2-3.4 ------------------------------------------------------

@pytest.mark.parametrize("seed", range(3))
def test_sparsified_hessian_theorems(seed):
    C, a, b, eta, logX, gamma = _state(seed=10 + seed, m=11, n=8, eta=0.3)
    m, n = C.shape
    P = O.plan(logX, C, eta, gamma)
    rho = np.quantile(P, 0.5)  # a threshold that actually drops entries
    assert rho > 1e-3
    Q = O.sparsify_plan(P, a, rho)
    s = O.istar(a)
    assert np.allclose(Q.sum(1), 1.0, atol=1e-15)                 # rows renormalised
    assert np.array_equal(Q[s], P[s])                             # row i* dense
    assert np.all((Q == 0) | (P >= rho) | (np.arange(m)[:, None] == s))
    # Lemma E_P: ||P - P_rho||_inf <= 2 n rho
    assert np.abs(P - Q).sum(1).max() <= 2 * n * rho + 1e-15
    H = O.hessian(P, a, eta)
    Hr = O.sparsified_hessian(Q, a, eta)
    # Thm 3.4: ||H - H_rho|| <= 6 m n ||a||_inf rho / eta
    assert np.linalg.norm(H - Hr, 2) <= 6 * m * n * a.max() * rho / eta + 1e-12
    # Thm 3.2: symmetric, PSD, kernel = span{1}
    assert np.allclose(Hr, Hr.T, atol=1e-12)
    assert np.abs(Hr @ np.ones(n)).max() <= 1e-12 / eta
    ev = np.linalg.eigvalsh(Hr)
    assert ev[0] >= -1e-10 and ev[1] > 1e-12
    # Thm 3.3: lambda_max <= 1/(2 eta); lambda_min on 1-perp >= n a_i* p^2 / eta
    assert ev[-1] <= 1.0 / (2 * eta) + 1e-9
    p = P[s].min()
    assert ev[1] >= n * a[s] * p * p / eta - 1e-9


def test_zero_threshold_gives_exact_hessian():
    C, a, b, eta, logX, gamma = _state(seed=20)
    P = O.plan(logX, C, eta, gamma)
    assert np.allclose(O.sparsified_hessian(O.sparsify_plan(P, a, 0.0), a, eta), O.hessian(P, a, eta),
                       rtol=0, atol=1e-12)


def test_newton_direction_solves_shifted_system_and_descends():
    C, a, b, eta, logX, gamma = _state(seed=21, m=10, n=7)
    P = O.plan(logX, C, eta, gamma)
    g = O.gradient(P, a, b)
    Hr = O.sparsified_hessian(O.sparsify_plan(P, a, 1e-3), a, eta)
    delta, it = O.newton_direction(Hr, g, cg_rtol=1e-14, max_cg=500)
    exact = np.linalg.solve(Hr + np.linalg.norm(g) * np.eye(len(g)), -g)
    assert np.abs(delta - (exact - exact.mean())).max() <= 1e-9 * np.abs(exact).max()
    assert abs(delta.sum()) <= 1e-14            # Lemma 4.1: stays in 1-perp
    assert g @ delta < 0                        # descent direction (Lemma B.6 (i))


def test_pcg_finite_termination_on_three_eigenvalues():
    """Conjugate gradients in exact arithmetic end after as many iterations as
    the (preconditioned) matrix has distinct eigenvalues.  A symmetric
    circulant matrix has a constant diagonal, so the Jacobi preconditioner is
    a scalar and keeps the three eigenvalues chosen here; a sign or index slip
    in the recurrence loses this property."""
    n = 16
    lam = np.ones(n)
    lam[0] = 5.0
    lam[[1, 7, 9, 15]] = 2.0                    # symmetric in j <-> n - j: real circulant
    c = np.real(np.fft.ifft(lam))
    A = np.array([[c[(j - i) % n] for j in range(n)] for i in range(n)])
    assert np.allclose(A, A.T) and np.allclose(np.diag(A), c[0])
    rhs = np.random.default_rng(5).normal(size=n)
    x, it, res = O.pcg(A, rhs, np.diag(A).copy(), 1e-10, 50)
    assert it == 3
    assert res <= 1e-10 * np.linalg.norm(rhs)
    assert np.abs(x - np.linalg.solve(A, rhs)).max() <= 1e-12 * np.abs(x).max()
    # two iterations leave a residual of the size of the data
    _, it2, res2 = O.pcg(A, rhs, np.diag(A).copy(), 1e-10, 2)
    assert it2 == 2 and res2 > 1e-3 * np.linalg.norm(rhs)


def test_armijo_accepts_sufficient_decrease():
    C, a, b, eta, logX, gamma = _state(seed=22)
    P = O.plan(logX, C, eta, gamma)
    g = O.gradient(P, a, b)
    Hr = O.sparsified_hessian(O.sparsify_plan(P, a, 0.0), a, eta)
    delta, _ = O.newton_direction(Hr, g, 1e-12, 500)
    t, trials, ok = O.armijo(logX, C, a, b, eta, gamma, 50 * delta, g, 1e-4, 0.8, 60)
    assert ok and trials >= 1
    L0 = O.semi_dual_objective(logX, C, a, b, eta, gamma)
    Lt = O.semi_dual_objective(logX, C, a, b, eta, gamma + t * 50 * delta)
    assert Lt <= L0 + 1e-4 * t * (g @ (50 * delta))


# --- Sinkhorn warm-up ------------------------------------------------------------

def test_sinkhorn_separable_cost_one_step():
    """For C = u 1^T + 1 v^T and X^0 = a b^T, gamma = v (+ const) zeroes the gradient:
    then P_ij = b_j.  One gamma-step reaches it from any start (Eq. 3 closed form)."""
    rng = np.random.default_rng(30)
    m, n, eta = 6, 4, 0.01
    u, v = rng.uniform(0, 1, m), rng.uniform(0, 1, n)
    C = u[:, None] + v[None, :]
    a = rng.uniform(0.1, 1, m); a /= a.sum()
    b = rng.uniform(0.1, 1, n); b /= b.sum()
    gam, it, gn = O.sinkhorn_warmup(O.initial_log_plan(a, b), C, a, b, eta, np.zeros(n), 1e-12, 10)
    assert it == 1 and gn < 1e-12
    assert np.allclose(gam - gam.mean(), v - v.mean(), atol=1e-12)


# --- Alg. 3, D_phi, c-transform, Delta_kkt ---------------------------------------

@pytest.mark.parametrize("seed", range(3))
def test_rounding_is_feasible(seed):
    rng = np.random.default_rng(40 + seed)
    m, n = 8, 6
    X = rng.uniform(0, 1, (m, n)) ** 3
    X /= X.sum()
    a = rng.uniform(0.1, 1, m); a /= a.sum()
    b = rng.uniform(0.1, 1, n); b /= b.sum()
    Xh, z, y, er, ec = O.round_to_feasible(X, a, b)
    assert Xh.min() >= 0
    assert np.abs(Xh.sum(1) - a).max() <= 1e-15 and np.abs(Xh.sum(0) - b).max() <= 1e-15
    assert er.min() >= -1e-17 and ec.min() >= -1e-17


def test_rounding_keeps_feasible_plans_and_golden_values():
    for case in json.load(open(GOLDEN))["cases"]:
        C, a, b = (np.array(case[k], dtype=np.float64) for k in ("C", "a", "b"))
        val, X, _, _ = lp.network_simplex(C, a, b)
        Xh = O.round_to_feasible(X + 0.0, a, b)[0]
        assert np.abs(Xh - X).max() <= 1e-15
        assert abs((C * Xh).sum() - case["opt"]) <= 1e-12


def test_bregman_divergence_properties():
    rng = np.random.default_rng(50)
    X = rng.uniform(0.1, 1, (5, 4)); X /= X.sum()
    Y = rng.uniform(0.1, 1, (5, 4)); Y /= Y.sum()
    assert abs(O.bregman_divergence_log(X, np.log(X))) <= 1e-15
    D = O.bregman_divergence_log(Y, np.log(X))
    assert D > 0
    # independent closed form: KL between the two normalised matrices
    assert abs(D - float(np.sum(Y * np.log(Y / X)))) <= 1e-15


def test_c_transform_gives_dual_feasible_lower_bound():
    rng = np.random.default_rng(60)
    m, n = 9, 7
    C = rng.uniform(0, 1, (m, n))
    a = rng.uniform(0.1, 1, m); a /= a.sum()
    b = rng.uniform(0.1, 1, n); b /= b.sum()
    opt = lp.network_simplex(C, a, b)[0]
    for _ in range(5):
        gam = rng.normal(0, 0.3, n)
        zeta = O.c_transform(C, gam)
        assert (C - zeta[:, None] - gam[None, :]).min() >= -1e-15
        assert O.dual_objective(a, b, zeta, gam) <= opt + 1e-15


def test_kkt_residual_zero_at_lp_solution():
    rng = np.random.default_rng(61)
    m, n = 7, 9
    C = rng.uniform(0, 1, (m, n))
    a = rng.uniform(0.1, 1, m); a /= a.sum()
    b = rng.uniform(0.1, 1, n); b /= b.sum()
    val, X, u, v = lp.network_simplex(C, a, b)
    assert O.kkt_residual(X, C, a, b, v, u) <= 1e-14
    assert O.kkt_residual(X, C, a, b, v + 0.1, u) > 1e-3


# --- Alg. 2 end to end -------------------------------------------------------------

def _solve(C, a, b, eta, **kw):
    return O.ibsn(C, a, b, O.IBSNParams(eta=eta, **kw), record=True)


def test_ibsn_golden_cases():
    for case in json.load(open(GOLDEN))["cases"]:
        C, a, b = (np.array(case[k], dtype=np.float64) for k in ("C", "a", "b"))
        res = _solve(C, a, b, 1e-2, max_outer=400)
        assert res.converged, case["name"]
        assert abs(res.primal - case["opt"]) <= 1e-8 * max(1e-2, case["opt"]) + 1e-12, case["name"]


@pytest.mark.parametrize("n", [4, 6])
def test_ibsn_matches_permutation_bruteforce(n):
    rng = np.random.default_rng(70 + n)
    C = rng.uniform(0, 1, (n, n))
    u = np.full(n, 1.0 / n)
    res = _solve(C, u, u, 1e-3)
    opt = lp.permutation_optimum(C)
    assert res.converged and abs(res.primal - opt) <= 1e-8 * opt


@pytest.mark.parametrize("shape", [(12, 17), (23, 15)])
def test_ibsn_matches_network_simplex(shape):
    m, n = shape
    prob = uniform_points_problem(m, n, seed=m * n, eta=1e-4)
    res = _solve(prob.C, prob.a, prob.b, prob.eta)
    opt = lp.network_simplex(prob.C, prob.a, prob.b)[0]
    assert res.converged
    assert res.dual - 1e-15 <= opt <= res.primal + 1e-15         # the certificate brackets OPT
    assert abs(res.primal - opt) <= 1e-8 * opt
    # marginal feasibility of the returned plan
    assert np.abs(res.plan.sum(1) - prob.a).sum() + np.abs(res.plan.sum(0) - prob.b).sum() <= 1e-12
    # Lemma 4.1: 1^T gamma = 0 along the iterates; Thm 4.2: L^k decreases within each subproblem
    for rec in res.history:
        Ls = [s["L"] for s in rec["inner"]]
        assert all(l1 <= l0 + 1e-15 for l0, l1 in zip(Ls, Ls[1:]))
        assert all(abs(s.get("mean_gamma", 0.0)) <= 1e-15 for s in rec["inner"])


def test_ibsn_square_cost_matches_monotone_closed_form():
    """The paper's Square cost C_ij = (i - j)^2 (Sec. 5.1), normalised by its max,
    is a convex cost of the 1-D index difference: the monotone coupling is optimal."""
    m = n = 24
    rng = np.random.default_rng(80)
    a = rng.uniform(0.1, 1, m); a /= a.sum()
    b = rng.uniform(0.1, 1, n); b /= b.sum()
    raw = square_index_cost(m, n)
    C = raw / raw.max()
    res = _solve(C, a, b, 1e-3)
    opt = lp.monotone_1d_optimum(np.arange(m, dtype=float), np.arange(n, dtype=float), a, b,
                                 lambda t: t * t / raw.max())
    assert res.converged and abs(res.primal - opt) <= 1e-8 * opt


def test_ibsn_separable_cost():
    rng = np.random.default_rng(81)
    u, v = rng.uniform(0, 1, 10), rng.uniform(0, 1, 13)
    a = rng.uniform(0.1, 1, 10); a /= a.sum()
    b = rng.uniform(0.1, 1, 13); b /= b.sum()
    res = _solve(u[:, None] + v[None, :], a, b, 1e-3)
    assert abs(res.primal - lp.separable_optimum(u, v, a, b)) <= 1e-12


def test_ibsn_single_row_and_column():
    rng = np.random.default_rng(82)
    b = rng.uniform(0.1, 1, 5); b /= b.sum()
    C = rng.uniform(0, 1, (1, 5))
    res = _solve(C, np.ones(1), b, 1e-3)
    assert abs(res.primal - float(C[0] @ b)) <= 1e-12
    res = _solve(C.T.copy(), b, np.ones(1), 1e-3)
    assert abs(res.primal - float(C[0] @ b)) <= 1e-12


def test_ibsn_grid_problem_matches_network_simplex():
    prob = grid_problem(5, 4, seed=3, sigma=1.0, eta=1e-3)
    res = _solve(prob.C, prob.a, prob.b, prob.eta)
    opt = lp.network_simplex(prob.C, prob.a, prob.b)[0]
    assert res.converged and abs(res.primal - opt) <= 1e-8 * opt


@pytest.mark.parametrize("forcing", ["gate", "plain"])
def test_ibsn_cg_forcing_readings_reach_the_lp_optimum(forcing):
    """Both readings of the unstated CG tolerance (R3: the gate-relaxed forcing
    term, or min(0.1, ||g||) alone) reach the network-simplex optimum."""
    prob = uniform_points_problem(24, 19, seed=77, eta=1e-3)
    opt = lp.network_simplex(prob.C, prob.a, prob.b)[0]
    res = O.ibsn(prob.C, prob.a, prob.b, O.IBSNParams(eta=prob.eta, cg_forcing=forcing))
    assert res.converged
    assert abs(res.primal - opt) <= 1e-8 * opt

"""Pins of the oracle's (E)IBSN (App. C.4): the entropic subproblem with X = 1 1^T.

The entropic OT problem min <C, X> + eta sum X (log X - 1) over the transport
polytope has a unique solution of the form X_ij = exp((zeta_i + gamma_j - C_ij)/eta).
The pins do not reuse the oracle's own Sinkhorn: a textbook log-domain
Sinkhorn iteration written here converges to the same unique plan, and a
separable cost has the closed-form plan a b^T.
"""

import numpy as np
from scipy.special import logsumexp

from oracle import ibsn as O
from workloads import paper_synthetic_problem, uniform_points_problem


def _textbook_sinkhorn(C, a, b, eta, iters=20000, tol=1e-14):
    """Alternating scaling of K = exp(-C/eta) in the log domain (u, v potentials)."""
    f = np.zeros(len(a))
    g = np.zeros(len(b))
    for _ in range(iters):
        f = eta * np.log(a) - eta * logsumexp((g[None, :] - C) / eta, axis=1)
        g = eta * np.log(b) - eta * logsumexp((f[:, None] - C) / eta, axis=0)
        X = np.exp((f[:, None] + g[None, :] - C) / eta)
        if np.abs(X.sum(axis=1) - a).sum() < tol:
            break
    return X


def test_eibsn_matches_textbook_sinkhorn_plan():
    prob = uniform_points_problem(60, 45, seed=3, eta=5e-2)
    res = O.eibsn(prob.C, prob.a, prob.b, O.IBSNParams(eta=prob.eta), gtol=1e-11)
    assert res.converged and res.gnorm < 1e-11
    X_newton = prob.a[:, None] * res.plan
    X_ref = _textbook_sinkhorn(prob.C, prob.a, prob.b, prob.eta)
    assert np.abs(X_newton - X_ref).max() <= 1e-10 * X_ref.max()
    assert np.abs(X_newton.sum(axis=1) - prob.a).max() <= 1e-15
    assert res.newton_iters >= 1


def test_eibsn_square_cost_converges_like_table_2():
    """The Square setting at a small size: Newton from the Sinkhorn warm-up
    reaches ||g|| < 1e-9 in a few tens of steps (the paper's Table 2 reports
    6-43 steps across its EOT settings)."""
    prob = paper_synthetic_problem("square", 80, 80, seed=4, eta=1e-3)
    res = O.eibsn(prob.C, prob.a, prob.b, O.IBSNParams(eta=prob.eta))
    assert res.converged and res.gnorm < 1e-9
    assert res.newton_iters <= 60
    g = O.gradient(res.plan, prob.a, prob.b)
    assert abs(g.sum()) <= 1e-15  # 1^T g = 0 (Lemma 4.1 / Eq. 7)


def test_eibsn_separable_cost_gives_product_plan():
    rng = np.random.default_rng(5)
    m, n = 30, 40
    u, v = rng.uniform(0, 1, m), rng.uniform(0, 1, n)
    C = u[:, None] + v[None, :]
    C /= C.max()
    a = rng.uniform(0.1, 1, m)
    a /= a.sum()
    b = rng.uniform(0.1, 1, n)
    b /= b.sum()
    res = O.eibsn(C, a, b, O.IBSNParams(eta=1e-2))
    assert res.converged
    assert np.abs(a[:, None] * res.plan - np.outer(a, b)).max() <= 1e-11


def test_eibsn_dense_hessian_variant_same_plan():
    prob = uniform_points_problem(40, 36, seed=6, eta=2e-2)
    r1 = O.eibsn(prob.C, prob.a, prob.b, O.IBSNParams(eta=prob.eta), gtol=1e-11)
    r0 = O.eibsn(prob.C, prob.a, prob.b, O.IBSNParams(eta=prob.eta, sparsify=False), gtol=1e-11)
    assert r1.converged and r0.converged
    assert np.abs(r1.plan - r0.plan).max() <= 1e-9 * r1.plan.max()

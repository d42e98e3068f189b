"""Pins for the exact LP references in oracle/lp.py (CPU only).

They are checked against each other, against hand-derived optima in
tests/golden/, and against scipy's HiGHS solver (an independent library LP).
"""

import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

from oracle import lp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_lp_cases.json")


def highs_optimum(C, a, b):
    m, n = C.shape
    rows = sp.kron(sp.eye(m), np.ones((1, n)))
    cols = sp.kron(np.ones((1, m)), sp.eye(n))
    A = sp.vstack([rows, cols]).tocsr()
    res = linprog(C.ravel(), A_eq=A, b_eq=np.concatenate([a, b]), bounds=(0, None), method="highs",
                  options=dict(primal_feasibility_tolerance=1e-10, dual_feasibility_tolerance=1e-10))
    assert res.status == 0
    return float(res.fun)


def test_golden_cases_network_simplex():
    cases = json.load(open(GOLDEN))["cases"]
    for case in cases:
        C, a, b = (np.array(case[k], dtype=np.float64) for k in ("C", "a", "b"))
        val, X, u, v = lp.network_simplex(C, a, b)
        assert abs(val - case["opt"]) <= 1e-12, case["name"]
        assert np.allclose(X.sum(1), a, atol=1e-14) and np.allclose(X.sum(0), b, atol=1e-14)


@pytest.mark.parametrize("seed", range(6))
def test_network_simplex_matches_highs(seed):
    rng = np.random.default_rng(seed)
    m, n = rng.integers(2, 18, size=2)
    C = rng.uniform(0, 1, size=(m, n))
    a = rng.uniform(0.1, 1, m); a /= a.sum()
    b = rng.uniform(0.1, 1, n); b /= b.sum()
    val, X, u, v = lp.network_simplex(C, a, b)
    ref = highs_optimum(C, a, b)
    assert abs(val - ref) <= 1e-9 * max(1.0, abs(ref))
    # primal feasibility and dual feasibility (reduced costs >= 0) and strong duality
    assert X.min() >= -1e-15
    assert np.abs(X.sum(1) - a).max() <= 1e-14 and np.abs(X.sum(0) - b).max() <= 1e-14
    assert (C - u[:, None] - v[None, :]).min() >= -1e-12
    assert abs(a @ u + b @ v - val) <= 1e-12


@pytest.mark.parametrize("n", [2, 3, 5, 6])
def test_permutation_matches_highs(n):
    rng = np.random.default_rng(100 + n)
    C = rng.uniform(0, 1, size=(n, n))
    u = np.full(n, 1.0 / n)
    assert abs(lp.permutation_optimum(C) - highs_optimum(C, u, u)) <= 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_monotone_1d_matches_highs(seed):
    rng = np.random.default_rng(200 + seed)
    m, n = 9 + seed, 7 + 2 * seed
    x = rng.uniform(0, 1, m)
    y = rng.uniform(0, 1, n)
    a = rng.uniform(0.1, 1, m); a /= a.sum()
    b = rng.uniform(0.1, 1, n); b /= b.sum()
    C = (x[:, None] - y[None, :]) ** 2
    assert abs(lp.monotone_1d_optimum(x, y, a, b, lambda t: t * t) - highs_optimum(C, a, b)) <= 1e-12


def test_separable_matches_highs():
    rng = np.random.default_rng(7)
    u = rng.uniform(0, 1, 6)
    v = rng.uniform(0, 1, 5)
    a = rng.uniform(0.1, 1, 6); a /= a.sum()
    b = rng.uniform(0.1, 1, 5); b /= b.sum()
    C = u[:, None] + v[None, :]
    assert abs(lp.separable_optimum(u, v, a, b) - highs_optimum(C, a, b)) <= 1e-12


def test_batched_points_are_the_batched_problems_draws():
    """The bench's batched workload (points only, cost formed on the device)
    draws exactly what workloads.batched_problems draws."""
    import numpy as np
    from workloads import batched_points, batched_problems
    pts = batched_points(count=3, lo=30, hi=60)
    full = batched_problems(count=3, lo=30, hi=60)
    for (m, n, x, y, a, b, eta), p in zip(pts, full):
        assert (m, n) == p.C.shape and eta == p.eta
        assert np.array_equal(x, p.x) and np.array_equal(y, p.y)
        assert np.array_equal(a, p.a) and np.array_equal(b, p.b)
        C = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
        assert np.allclose(C / C.max(), p.C, rtol=1e-15, atol=0)

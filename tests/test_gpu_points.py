"""On-the-fly squared-Euclidean point cost (IBSN_COST_SQEUCLID_POINTS).

The cost C_ij = scale ||x_i - y_j||^2 is rebuilt from the coordinates wherever
the solver reads C (anchor build, certificate), so no m x n cost matrix exists.
Parity: the anchored plan of Eq. 6 against the oracle's explicit recursion on
the materialised cost, in 2 and 10 dimensions and every precision mode; whole
solves certified against the exact cost on the host and matching the exact LP
optimum (or the dense-cost solve of the same problem).
"""

import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ibsn as O  # noqa: E402
from workloads import gmm_points_problem, uniform_points_problem, workload  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_optima.json")))["cases"]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_07156_gb300 import build as B
    B.build()


def _t(x):
    return torch.tensor(x, dtype=torch.float64, device="cuda")


def _points_problem(prob):
    import paper_2603_07156_gb300 as G
    return G.Problem(a=_t(prob.a), b=_t(prob.b), eta=prob.eta, x=_t(prob.x).contiguous(), y=_t(prob.y).contiguous(),
                     cost_scale=prob.cost_scale)


def _exact_cost(prob):
    d = prob.x[:, None, :] - prob.y[None, :, :]
    return prob.cost_scale * np.einsum("ijk,ijk->ij", d, d)


@pytest.mark.parametrize("dim", [2, 10])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_points_anchor_and_plan_pass(dim, prec):
    import paper_2603_07156_gb300 as G
    if dim == 2:
        prob = uniform_points_problem(301, 517, seed=81, eta=1e-2)
    else:
        prob = gmm_points_problem(233, 389, seed=82, d=10, eta=1e-2)
    C = _exact_cost(prob)
    rng = np.random.default_rng(83)
    k = 3
    gs = [rng.normal(0.0, 0.3 * prob.eta, prob.n) for _ in range(k)]
    gamma = rng.normal(0.0, 0.3 * prob.eta, prob.n)
    logX = O.initial_log_plan(prob.a, prob.b)
    for g in gs:
        logX = np.log(prob.a)[:, None] + O.log_plan(logX, C, prob.eta, g)
    Pref = O.plan(logX, C, prob.eta, gamma)
    gp = _points_problem(prob)
    ctx = G.Context(gp, G.params(precision="mixed" if prec == "ff" else prec))
    ctx.set_state(k, _t(np.sum(gs, axis=0)), _t(gamma), prec)
    P = ctx.export_plan().cpu().numpy()
    rowmax = Pref.max(axis=1, keepdims=True)
    big = Pref > 2.0 ** -60 * rowmax
    rel = np.abs(P[big] - Pref[big]) / Pref[big]
    # float-float cost: the sum of dim squared differences carries about
    # dim * 2^-48 relative error, which the anchor multiplies by (k+1)/eta
    # (<= 400 here) on a cost <= 1: the bound on an entry's relative error
    ff_tol = max(1e-12, 2.0 * dim * 2.0 ** -48 * (k + 1) / prob.eta)
    if prec == "mixed":
        assert rel.max() <= 1.2e-3, rel.max()
        assert np.abs(P - Pref).max() <= 2e-5
    elif prec == "ff":
        assert rel.max() <= ff_tol, (rel.max(), ff_tol)
    else:
        assert rel.max() <= 1e-12, rel.max()
    c, gn = ctx.plan()
    g_ref = O.gradient(Pref, prob.a, prob.b)
    tol = 2e-4 if prec == "mixed" else (10 * ff_tol if prec == "ff" else 1e-11)
    assert np.abs(c.cpu().numpy() - (g_ref + prob.b)).max() <= tol * prob.b.max()
    cert = ctx.certify(want_plan=False)
    zeta = O.c_transform(C, ctx.gamma().cpu().numpy())
    assert np.abs(cert["zeta"].cpu().numpy() - zeta).max() <= 1e-14


def _check(res, prob, C):
    X = res["plan"].cpu().numpy()
    gam = res["gamma"].cpu().numpy()
    viol = np.abs(X.sum(1) - prob.a).sum() + np.abs(X.sum(0) - prob.b).sum()
    assert viol <= 1e-8, viol
    p = float((C * X).sum())
    d = float(prob.a @ (C - gam[None, :]).min(axis=1) + prob.b @ gam)
    assert (p - d) / max(abs(p), abs(d)) <= 1e-8
    assert abs(p - res["primal"]) <= 1e-11 * abs(p)
    return p


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_points_solve_matches_lp_optimum_c0(prec):
    """The 256^2 uniform-points workload (eta = 1e-4) with the cost rebuilt
    from the points: the certified primal equals the LP optimum of the
    materialised cost to 1e-8."""
    import paper_2603_07156_gb300 as G
    prob = workload("c0")
    res = G.solve(_points_problem(prob), G.params(precision=prec), want_plan=True)
    assert res["converged"], res["rel_gap"]
    p = _check(res, prob, _exact_cost(prob))
    opt = GOLD["c0_uniform2d_256"]["lp_optimum"]
    assert abs(p - opt) <= 1e-8 * opt


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_points_solve_matches_dense_cost_in_10d(prec):
    import paper_2603_07156_gb300 as G
    prob = gmm_points_problem(300, 257, seed=84, d=10, eta=1e-4)
    C = _exact_cost(prob)
    r_pts = G.solve(_points_problem(prob), G.params(precision=prec), want_plan=True)
    r_den = G.solve(G.Problem(a=_t(prob.a), b=_t(prob.b), eta=prob.eta, C=_t(C)), G.params(precision=prec),
                    want_plan=True)
    assert r_pts["converged"] and r_den["converged"]
    p1 = _check(r_pts, prob, C)
    p2 = _check(r_den, prob, C)
    assert abs(p1 - p2) <= 2e-8 * abs(p2)


def test_points_validation_errors():
    import paper_2603_07156_gb300 as G
    from paper_2603_07156_gb300._native import IbsnError
    prob = uniform_points_problem(20, 30, seed=85, eta=1e-3)
    x = _t(prob.x)
    x[3, 1] = float("nan")
    with pytest.raises(IbsnError) as e:
        G.solve(G.Problem(a=_t(prob.a), b=_t(prob.b), eta=1e-3, x=x, y=_t(prob.y), cost_scale=prob.cost_scale))
    assert e.value.code == 3
    wide = torch.zeros((20, 17), dtype=torch.float64, device="cuda")
    widey = torch.zeros((30, 17), dtype=torch.float64, device="cuda")
    with pytest.raises(IbsnError) as e:
        G.solve(G.Problem(a=_t(prob.a), b=_t(prob.b), eta=1e-3, x=wide, y=widey, cost_scale=1.0))
    assert e.value.code == 8

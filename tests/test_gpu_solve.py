"""End-to-end parity of ibsn_solve (Alg. 2) against the oracle and exact LP optima.

Both sides are certified: X-hat is feasible (Alg. 3) and zeta is the
c-transform (App. C.1), so p >= OPT >= d and the relative gap bounds the
distance to the optimum.  The bar is the objective within 1e-8 relative of
the LP optimum for float64, 1e-6 for float32 passes without polish, 1e-8
with polish, and marginal violation <= 1e-8.
"""

import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import lp  # noqa: E402
from workloads import grid_problem, uniform_points_problem, workload  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_optima.json")))["cases"]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_07156_gb300 import build as B
    B.build()


def gpu_solve(prob, precision="fp64", cost_dtype=torch.float64, grid=False, want_plan=True, **kw):
    import paper_2603_07156_gb300 as G
    a = torch.tensor(prob.a, dtype=torch.float64, device="cuda")
    b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
    if grid:
        gp = G.Problem(a=a, b=b, eta=prob.eta, grid=prob.grid, cost_scale=prob.cost_scale)
    else:
        gp = G.Problem(a=a, b=b, eta=prob.eta, C=torch.tensor(prob.C, dtype=cost_dtype, device="cuda"))
    return G.solve(gp, G.params(precision=precision, **kw), want_plan=want_plan)


def check_certificate(res, prob, C=None, tol_gap=1e-8):
    """Re-verify the GPU certificate on the host from the returned plan and potential."""
    C = prob.C if C is None else C
    X = res["plan"].cpu().numpy()
    gam = res["gamma"].cpu().numpy()
    assert X.min() >= 0.0
    viol = np.abs(X.sum(1) - prob.a).sum() + np.abs(X.sum(0) - prob.b).sum()
    assert viol <= 1e-8, viol
    p = float((C * X).sum())
    zeta = (C - gam[None, :]).min(axis=1)
    d = float(prob.a @ zeta + prob.b @ gam)
    assert abs(p - res["primal"]) <= 1e-12 * abs(p) + 1e-15
    assert abs(d - res["dual"]) <= 1e-12 * abs(d) + 1e-15
    assert (p - d) / max(abs(p), abs(d)) <= tol_gap
    return p, d


@pytest.mark.parametrize("name,prob_fn", [
    ("uniform2d_96x131_s21", lambda: uniform_points_problem(96, 131, seed=21, eta=1e-4)),
    ("grid16x16_s2", lambda: grid_problem(16, 16, seed=2, eta=1e-3)),
    ("c0_uniform2d_256", lambda: workload("c0")),
])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_matches_lp_optimum(name, prob_fn, precision):
    prob = prob_fn()
    res = gpu_solve(prob, precision=precision)
    assert res["converged"], res
    opt = GOLD[name]["lp_optimum"]
    p, d = check_certificate(res, prob)
    assert abs(p - opt) <= 1e-8 * opt
    assert d <= opt * (1 + 1e-12) and p >= opt * (1 - 1e-12)


def test_mixed_without_polish_within_1e6():
    prob = uniform_points_problem(96, 131, seed=21, eta=1e-4)
    res = gpu_solve(prob, precision="mixed", polish=0, gap_tol=1e-6, max_outer=400)
    opt = GOLD["uniform2d_96x131_s21"]["lp_optimum"]
    assert abs(res["primal"] - opt) <= 1e-6 * opt


def test_grid_on_the_fly_cost_matches_dense():
    prob = grid_problem(16, 16, seed=2, eta=1e-3)
    r_fly = gpu_solve(prob, grid=True)
    r_den = gpu_solve(prob)
    assert r_fly["converged"] and r_den["converged"]
    opt = GOLD["grid16x16_s2"]["lp_optimum"]
    check_certificate(r_fly, prob)
    assert abs(r_fly["primal"] - opt) <= 1e-8 * opt


def test_float32_cost_is_solved_exactly_as_given():
    prob = uniform_points_problem(40, 33, seed=31, eta=1e-4)
    C32 = prob.C.astype(np.float32).astype(np.float64)
    res = gpu_solve(prob, precision="mixed", cost_dtype=torch.float32)
    opt = lp.network_simplex(C32, prob.a, prob.b)[0]
    check_certificate(res, prob, C=C32)
    assert abs(res["primal"] - opt) <= 1e-8 * opt


@pytest.mark.parametrize("shape", [(1, 7), (7, 1), (2, 2), (33, 65)])
def test_degenerate_shapes(shape):
    m, n = shape
    prob = uniform_points_problem(m, n, seed=40 + m, eta=1e-3)
    res = gpu_solve(prob)
    opt = lp.network_simplex(prob.C, prob.a, prob.b)[0]
    check_certificate(res, prob)
    assert abs(res["primal"] - opt) <= 1e-8 * max(opt, 1e-12) + 1e-15


def test_ibn_dense_hessian_ablation_same_optimum():
    prob = uniform_points_problem(96, 131, seed=21, eta=1e-4)
    res = gpu_solve(prob, sparsify=0)
    assert res["converged"]
    assert abs(res["primal"] - GOLD["uniform2d_96x131_s21"]["lp_optimum"]) <= 1e-8 * res["primal"]


def test_input_validation_errors():
    import paper_2603_07156_gb300 as G
    from paper_2603_07156_gb300._native import IbsnError
    prob = uniform_points_problem(20, 30, seed=50, eta=1e-3)
    a = torch.tensor(prob.a, dtype=torch.float64, device="cuda")
    b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
    C = torch.tensor(prob.C, dtype=torch.float64, device="cuda")
    with pytest.raises(IbsnError) as e:
        G.solve(G.Problem(a=a * 1.01, b=b, eta=1e-3, C=C))
    assert e.value.code == 2
    bad = C.clone()
    bad[3, 4] = float("nan")
    with pytest.raises(IbsnError) as e:
        G.solve(G.Problem(a=a, b=b, eta=1e-3, C=bad))
    assert e.value.code == 3
    neg = C.clone()
    neg[0, 0] = -1.0
    with pytest.raises(IbsnError) as e:
        G.solve(G.Problem(a=a, b=b, eta=1e-3, C=neg))
    assert e.value.code == 3
    gp = G.Problem(a=a, b=b, eta=1e-3, C=C)
    prm = G.params()
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(IbsnError) as e:
        G.solve(gp, prm, workspace=small)
    assert e.value.code == 4
    prm = G.params(nnz_cap=10)
    with pytest.raises(IbsnError) as e:
        G.solve(gp, prm)
    assert e.value.code == 7


def test_full_size_grid_certificate():
    """The 16384-bin grid workload (128 x 128, eta = 1e-3) in the launch
    configuration the benchmark times: float32 passes with float64 polish and
    the cost rebuilt from grid coordinates.  The certificate is re-verified on
    the host from the returned plan and potential (a property at any size)."""
    prob = grid_problem(128, 128, seed=2, eta=1e-3, cost_dtype=np.float32)
    res = gpu_solve(prob, precision="mixed", grid=True)
    assert res["converged"], res
    C = prob.C.astype(np.float64)  # exact grid cost in float64 is the same problem up to 1 ulp
    Cg = (np.subtract.outer(np.arange(16384) // 128, np.arange(16384) // 128) ** 2
          + np.subtract.outer(np.arange(16384) % 128, np.arange(16384) % 128) ** 2) * prob.cost_scale
    del C
    check_certificate(res, prob, C=Cg)

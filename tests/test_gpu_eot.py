"""(E)IBSN mode (App. C.4) of ibsn_solve against the oracle's eibsn.

One entropic subproblem with X = 1 1^T, Sinkhorn warm-up, Newton steps until
||g|| < 1e-9.  The subproblem has a unique solution plan; both sides stop
within 1e-9 of it in gradient norm, so their plans agree to that order.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ibsn as O  # noqa: E402
from workloads import paper_synthetic_problem, sphere_problem, uniform_points_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_07156_gb300 import build as B
    B.build()


def _solve(prob, precision, **kw):
    import paper_2603_07156_gb300 as G
    t = lambda v: torch.tensor(v, dtype=torch.float64, device="cuda")  # noqa: E731
    gp = G.Problem(a=t(prob.a), b=t(prob.b), eta=prob.eta, C=t(prob.C))
    return G.solve(gp, G.params(precision=precision, eot=1, **kw), want_plan=True)


CASES = [
    (lambda: uniform_points_problem(150, 113, seed=71, eta=1e-3), "fp64"),
    (lambda: uniform_points_problem(150, 113, seed=71, eta=1e-3), "mixed"),
    (lambda: paper_synthetic_problem("square", 300, 300, seed=72, eta=1e-4), "fp64"),
    (lambda: paper_synthetic_problem("square", 300, 300, seed=72, eta=1e-4), "mixed"),
    # unbalanced m >> n spherical transport (App. C.4), eta = 1e-3
    (lambda: sphere_problem(3000, 50, seed=73), "fp64"),
    (lambda: sphere_problem(3000, 50, seed=73), "mixed"),
]

_REF = {}


def _oracle(key, prob):
    if key not in _REF:
        _REF[key] = O.eibsn(prob.C, prob.a, prob.b, O.IBSNParams(eta=prob.eta))
    return _REF[key]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_eot_mode_matches_oracle(case):
    mk, prec = CASES[case]
    prob = mk()
    res = _solve(prob, prec)
    ref = _oracle(prob.name, prob)
    assert ref.converged
    assert res["converged"] and res["grad_norm"] < 1e-9, (res["grad_norm"], res["newton_iters"])
    assert res["outer_iters"] == 1
    Xref = prob.a[:, None] * ref.plan
    X = res["plan"].cpu().numpy()  # Alg. 3 rounding of the GPU's plan: moves it by O(||g||)
    assert np.abs(X - Xref).max() <= 1e-8 * Xref.max() + 4e-9, np.abs(X - Xref).max()
    # the semi-dual objective (Eq. 5 with X = 1 1^T) at both potentials: equal up
    # to O(||g||^2 / lambda_min) near the common optimum
    z = np.zeros_like(prob.C)
    L_gpu = O.semi_dual_objective(z, prob.C, prob.a, prob.b, prob.eta, res["gamma"].cpu().numpy())
    L_ref = O.semi_dual_objective(z, prob.C, prob.a, prob.b, prob.eta, ref.gamma)
    assert abs(L_gpu - L_ref) <= 1e-12 * abs(L_ref) + 1e-15, (L_gpu, L_ref)
    # the rounded plan is feasible; its objective is certified against the LP dual
    assert res["marg_viol"] <= 1e-8
    assert res["primal"] >= res["dual"]

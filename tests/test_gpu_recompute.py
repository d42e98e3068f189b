"""Passes that rebuild the anchored exponent from the cost (params.recompute).

With recompute = 1 the solver stores no m x n anchored matrix: every pass
evaluates K_ij from the cost, the anchor-time potentials and the row shifts
with the arithmetic of the anchor build.  The values are therefore the same
bits as the stored planes, and so is every result: the tests compare the two
modes for bitwise equality, step by step at the benchmark's width and over
whole solves, and check the workspace saving.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads import grid_marginals, grid_problem, uniform_points_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_07156_gb300 import build as B
    B.build()


def _t(x):
    return torch.tensor(x, dtype=torch.float64, device="cuda")


def _grid(h, eta, seed=2):
    import paper_2603_07156_gb300 as G
    a, b, scale = grid_marginals(h, h, seed=seed)
    return G.Problem(a=_t(a), b=_t(b), eta=eta, grid=(h, h), cost_scale=scale)


def _points(prob):
    import paper_2603_07156_gb300 as G
    return G.Problem(a=_t(prob.a), b=_t(prob.b), eta=prob.eta, x=_t(prob.x).contiguous(), y=_t(prob.y).contiguous(),
                     cost_scale=prob.cost_scale)


@pytest.mark.parametrize("prec", ["mixed", "ff"])
def test_recompute_plan_pass_bitwise_at_full_width(prec):
    import paper_2603_07156_gb300 as G
    gp = _grid(128, 1e-4)
    n = 128 * 128
    rng = np.random.default_rng(11)
    Gam = _t(rng.normal(0.0, 3e-5, n))
    gam = _t(rng.normal(0.0, 3e-5, n))
    out = []
    for rc in (0, 1):
        ctx = G.Context(gp, G.params(precision="mixed", recompute=rc))
        ctx.set_state(4, Gam, gam, prec)
        c, gn = ctx.plan()
        P = ctx.export_plan()[:: 257].cpu().numpy()
        out.append((c.cpu().numpy(), gn, P))
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("case", ["grid", "points"])
def test_recompute_solve_bitwise(case):
    import paper_2603_07156_gb300 as G
    if case == "grid":
        gp = _grid(24, 1e-3)
    else:
        gp = _points(uniform_points_problem(200, 170, seed=12, eta=1e-4))
    r = [G.solve(gp, G.params(precision="mixed", recompute=rc)) for rc in (0, 1)]
    assert r[0]["converged"] and r[1]["converged"]
    for key in ("primal", "dual", "rel_gap", "outer_iters", "newton_iters", "cg_iters", "polish_outer"):
        assert r[0][key] == r[1][key], key
    assert torch.equal(r[0]["gamma"], r[1]["gamma"])


def test_recompute_workspace_holds_no_anchored_matrix():
    import paper_2603_07156_gb300 as G
    gp = _grid(64, 1e-3)
    m = n = 64 * 64
    w0 = G.workspace_size(gp, G.params(precision="mixed"))
    w1 = G.workspace_size(gp, G.params(precision="mixed", recompute=1))
    assert w0 - w1 >= 2 * m * n * 4  # both float planes of the polish
    from paper_2603_07156_gb300._native import IbsnError
    with pytest.raises(IbsnError) as e:  # float64 passes always store their matrix
        G.Context(gp, G.params(precision="fp64", recompute=1))
    assert e.value.code == 1

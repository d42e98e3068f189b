"""Step-level parity of the CUDA path against the CPU oracle (one hot-path row each).

The oracle keeps log X^k explicitly (Alg. 2 outer update); the GPU keeps the
cumulative potential Gamma^k.  Both are driven by the same potentials, so
agreement also checks the anchored representation of the outer update.
Shapes are ragged (m != n, n not a multiple of the tile width) and span
several tiles.  Tolerances: float64 passes 1e-11 relative on plan entries
(rounding of exp of exponents of size ~50); float32 passes 2e-5 relative
(float32 anchor and ex2 rounding, |exponent| <= ~60).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ibsn as O  # noqa: E402
from workloads import uniform_points_problem, grid_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_07156_gb300 import build as B
    B.build()


def _gpu_problem(prob, cost_dtype=torch.float64):
    import paper_2603_07156_gb300 as G
    dev = "cuda"
    C = torch.tensor(prob.C, dtype=cost_dtype, device=dev)
    a = torch.tensor(prob.a, dtype=torch.float64, device=dev)
    b = torch.tensor(prob.b, dtype=torch.float64, device=dev)
    return G.Problem(a=a, b=b, eta=prob.eta, C=C)


def _state(prob, k, seed, scale=0.3):
    """Oracle log X^k from k outer updates with random potentials, plus the GPU's
    cumulative Gamma^k = sum of those potentials, and a current gamma."""
    rng = np.random.default_rng(seed)
    n = prob.n
    logX = O.initial_log_plan(prob.a, prob.b)
    Gam = np.zeros(n)
    for _ in range(k):
        g = rng.normal(0.0, scale * prob.eta, n)
        logX = np.log(prob.a)[:, None] + O.log_plan(logX, prob.C, prob.eta, g)
        Gam += g
    gamma = rng.normal(0.0, scale * prob.eta, n)
    return logX, Gam, gamma


def _ctx(prob, precision, cost_dtype=torch.float64, **kw):
    """precision: 'fp64', 'mixed' (float32 passes) or 'ff' (float-float passes of a
    mixed context with polish)."""
    import paper_2603_07156_gb300 as G
    gp = _gpu_problem(prob, cost_dtype)
    prm = G.params(precision="mixed" if precision == "ff" else precision, **kw)
    return G.Context(gp, prm), gp


def _t(x):
    return torch.tensor(x, dtype=torch.float64, device="cuda")


CASES = [
    # (problem, k, precision, plan tolerance)
    (lambda: uniform_points_problem(300, 200, seed=5, eta=1e-2), 3, "fp64", 1e-11),
    (lambda: uniform_points_problem(333, 517, seed=6, eta=1e-2), 2, "fp64", 1e-11),
    (lambda: grid_problem(12, 11, seed=7, sigma=2.0, eta=1e-2), 4, "fp64", 1e-11),
    (lambda: uniform_points_problem(300, 200, seed=5, eta=1e-2), 3, "mixed", 2e-5),
    (lambda: uniform_points_problem(129, 1500, seed=8, eta=1e-2), 1, "mixed", 2e-5),
    (lambda: uniform_points_problem(300, 200, seed=5, eta=1e-2), 3, "ff", 1e-11),
    (lambda: grid_problem(12, 11, seed=7, sigma=2.0, eta=1e-2), 4, "ff", 1e-11),
    (lambda: uniform_points_problem(129, 1500, seed=8, eta=1e-2), 1, "ff", 1e-11),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_anchor_and_plan_pass(case):
    mk, k, prec, tol = CASES[case]
    prob = mk()
    logX, Gam, gamma = _state(prob, k, seed=case)
    ctx, _ = _ctx(prob, prec)
    ctx.set_state(k, _t(Gam), _t(gamma), prec)
    P = ctx.export_plan().cpu().numpy()
    Pref = O.plan(logX, prob.C, prob.eta, gamma)
    big = Pref > 1e-30
    if prec == "ff":
        # float-float passes drop entries below 2^-64 of their row's maximum (the
        # float32 filter decides near that threshold): entries clearly above it
        # match, the ones near or below it are either dropped or match
        rowmax = Pref.max(axis=1, keepdims=True)
        kept = big & (Pref > 2.0 ** -60 * rowmax)
        near = big & ~kept
        assert np.all(P[Pref < 2.0 ** -68 * rowmax] == 0.0)
        relnear = np.abs(P[near] - Pref[near]) / Pref[near]
        assert np.all((P[near] == 0.0) | (relnear <= tol * 60))
        big = kept
    rel = np.abs(P[big] - Pref[big]) / Pref[big]
    # float-float entries (float-float exp of a float64-accurate exponent):
    # about 1e-14 relative; float64 passes: rounding of exp of exponents ~50
    assert rel.max() <= (1e-12 if prec == "ff" else tol * 60), rel.max()
    assert np.abs(P - Pref).max() <= tol
    c, gn = ctx.plan()
    g_ref = O.gradient(Pref, prob.a, prob.b)
    assert np.abs(c.cpu().numpy() - (g_ref + prob.b)).max() <= tol * 10 * prob.b.max()
    assert abs(gn - np.linalg.norm(g_ref)) <= tol * 10 * max(np.linalg.norm(g_ref), 1e-12) + 1e-14


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sinkhorn_warmup(prec):
    prob = uniform_points_problem(300, 200, seed=11, eta=1e-2)
    logX, Gam, gamma = _state(prob, 2, seed=11)
    ctx, _ = _ctx(prob, prec)
    ctx.set_state(2, _t(Gam), _t(gamma), prec)
    it, gn = ctx.sinkhorn(1e-6, 500)
    g_ref, it_ref, gn_ref = O.sinkhorn_warmup(logX, prob.C, prob.a, prob.b, prob.eta, gamma, 1e-6, 500)
    g_ref = g_ref - g_ref.mean()
    g_gpu = ctx.gamma().cpu().numpy()
    if prec == "fp64":
        assert it == it_ref
        assert np.abs(g_gpu - g_ref).max() <= 1e-10 * prob.eta
    else:
        assert abs(it - it_ref) <= 2
        assert np.abs(g_gpu - g_ref).max() <= 1e-4 * prob.eta
    assert gn < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sparsify(prec):
    prob = uniform_points_problem(260, 190, seed=12, eta=2e-2)
    logX, Gam, gamma = _state(prob, 2, seed=12)
    ctx, _ = _ctx(prob, prec)
    ctx.set_state(2, _t(Gam), _t(gamma), prec)
    P = O.plan(logX, prob.C, prob.eta, gamma)
    rho = float(np.quantile(P, 0.7))
    nnz = ctx.sparsify(rho)
    Q = ctx.export_sparse().cpu().numpy()
    Qref = O.sparsify_plan(P, prob.a, rho)
    s = O.istar(prob.a)
    # entries far from the threshold must agree; rows containing a near-tie are skipped
    tie = np.abs(P - rho) <= (1e-9 if prec == "fp64" else 1e-4) * rho
    rows = ~tie.any(axis=1)
    tol = 1e-12 if prec == "fp64" else 3e-5
    assert rows.sum() >= 0.5 * prob.m
    assert np.abs(Q[rows] - Qref[rows]).max() <= tol
    assert np.abs(Q[s] - Qref[s]).max() <= tol
    assert nnz == int((Q[np.arange(prob.m) != s] > 0).sum())


def _newton_setup(prec, seed=13):
    prob = uniform_points_problem(240, 176, seed=seed, eta=2e-2)
    logX, Gam, gamma = _state(prob, 2, seed=seed)
    ctx, _ = _ctx(prob, prec)
    ctx.set_state(2, _t(Gam), _t(gamma), prec)
    P = O.plan(logX, prob.C, prob.eta, gamma)
    g = O.gradient(P, prob.a, prob.b)
    rho = O.sparsification_threshold(prob.eta, prob.m, prob.n, np.linalg.norm(g)) * 1e6
    return prob, logX, gamma, ctx, P, g, rho


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_newton_direction(prec):
    prob, logX, gamma, ctx, P, g, rho = _newton_setup(prec)
    ctx.sparsify(rho)
    d, it, res = ctx.newton_direction(shift=-1.0, rtol=1e-12 if prec == "fp64" else 1e-6, max_cg=2000)
    Hr = O.sparsified_hessian(O.sparsify_plan(P, prob.a, rho), prob.a, prob.eta)
    exact = np.linalg.solve(Hr + np.linalg.norm(g) * np.eye(prob.n), -g)
    exact -= exact.mean()
    d = d.cpu().numpy()
    tol = 1e-8 if prec == "fp64" else 2e-4
    assert np.abs(d - exact).max() <= tol * np.abs(exact).max()
    assert abs(d.sum()) <= 1e-12 * np.abs(d).sum()
    assert g @ d < 0


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_armijo_difference_form(prec):
    prob, logX, gamma, ctx, P, g, rho = _newton_setup(prec, seed=14)
    ctx.sparsify(rho)
    d, _, _ = ctx.newton_direction(shift=-1.0, rtol=1e-10, max_cg=2000)
    d = d.cpu().numpy()
    L0 = O.semi_dual_objective(logX, prob.C, prob.a, prob.b, prob.eta, gamma)
    for t in (1.0, 0.5, 0.05):
        dL, slope, _ = ctx.armijo_trial(t, accept=False)
        ref = O.semi_dual_objective(logX, prob.C, prob.a, prob.b, prob.eta, gamma + t * d) - L0
        tol = 1e-5 if prec == "mixed" else 1e-9
        assert abs(dL - ref) <= tol * abs(ref) + 1e-15, (t, dL, ref)
        assert abs(slope - g @ d) <= (1e-5 if prec == "mixed" else 1e-10) * abs(g @ d)
    # accepting moves gamma to gamma + t Delta
    dL, slope, acc = ctx.armijo_trial(1.0, accept=True)
    if acc:
        assert np.abs(ctx.gamma().cpu().numpy() - (gamma + d)).max() <= 1e-12 + 1e-9 * np.abs(d).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_stop_check(prec):
    prob = uniform_points_problem(230, 170, seed=15, eta=2e-2)
    logX, Gam, gamma = _state(prob, 2, seed=15)
    ctx, _ = _ctx(prob, prec)
    ctx.set_state(2, _t(Gam), _t(gamma), prec)
    D = ctx.stop_check()
    lp = O.log_plan(logX, prob.C, prob.eta, gamma)
    logXn = np.log(prob.a)[:, None] + lp
    Xh = O.round_to_feasible(np.exp(logXn), prob.a, prob.b)[0]
    ref = O.bregman_divergence_log(Xh, logXn)
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert abs(D - ref) <= tol * ref, (D, ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_certify(prec):
    prob = uniform_points_problem(230, 170, seed=16, eta=2e-2)
    logX, Gam, gamma = _state(prob, 2, seed=16)
    ctx, _ = _ctx(prob, prec)
    ctx.set_state(2, _t(Gam), _t(gamma), prec)
    cert = ctx.certify(want_plan=True)
    lp = O.log_plan(logX, prob.C, prob.eta, gamma)
    p, d, gap, Xh, zeta = O.certify(np.log(prob.a)[:, None] + lp, prob.C, prob.a, prob.b, gamma)
    tol = 2e-6 if prec == "mixed" else 1e-12
    assert abs(cert["primal"] - p) <= tol * abs(p) * 10
    assert abs(cert["dual"] - d) <= 1e-13 * max(1.0, abs(d))
    assert np.abs(cert["zeta"].cpu().numpy() - zeta).max() <= 1e-14
    Xg = cert["plan"].cpu().numpy()
    assert np.abs(Xg - Xh).max() <= tol * Xh.max()
    if prec != "mixed":
        assert cert["marg_viol"] <= 1e-13
        assert np.abs(Xg.sum(1) - prob.a).sum() + np.abs(Xg.sum(0) - prob.b).sum() <= 1e-13


def test_certify_ff_ctransform_near_ties():
    """The float-float certificate finds zeta_i = min_j C_ij - gamma_j with a
    float32 scan and re-evaluates in float64 only the candidates within the
    float32 error bound of the minimum.  Integer grid costs with gamma
    perturbed far below float32 resolution make many candidates tie in float32
    while the float64 minimum is unique: zeta must still be exact."""
    prob = grid_problem(13, 12, seed=17, sigma=2.0, eta=2e-2)
    logX, Gam, gamma = _state(prob, 1, seed=17)
    rng = np.random.default_rng(18)
    gamma = np.round(gamma / prob.cost_scale) * prob.cost_scale + rng.uniform(-1e-12, 1e-12, prob.n)
    ctx, _ = _ctx(prob, "ff")
    ctx.set_state(1, _t(Gam), _t(gamma), "ff")
    cert = ctx.certify(want_plan=False)
    zeta = (prob.C - gamma[None, :]).min(axis=1)
    assert np.array_equal(cert["zeta"].cpu().numpy(), zeta)

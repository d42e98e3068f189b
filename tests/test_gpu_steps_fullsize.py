"""Step-level oracle parity on the kernel configurations that full-size problems take.

The dense passes pick a register-tile configuration by the row length n
(six float and six double configurations, the widest covering n = 16384),
and the Newton direction runs on one thread-block cluster for small sparsified
Hessians and on the grid-wide persistent kernel otherwise.  The step tests in
test_gpu_steps.py stay at n <= 1500; the cases here reach every tile
configuration (n = 3000, 6000, 12000, 16384) with few rows, so that the float64
oracle still finishes in seconds, and force the grid-wide Newton kernels with
sparsified Hessians above the cluster's capacity.  Each comparison is against
the oracle's own definition of the step (Eqs. 5-7, Alg. 1, Alg. 2, Eq. 8 with
Alg. 3, App. C.1), at eta = 1e-2 and at the eta = 1e-4 of the benchmark.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ibsn as O  # noqa: E402
from workloads import grid_problem, uniform_points_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_07156_gb300 import build as B
    B.build()


def _t(x):
    return torch.tensor(x, dtype=torch.float64, device="cuda")


def _ctx(prob, precision, cost_dtype=torch.float64, **kw):
    import paper_2603_07156_gb300 as G
    gp = G.Problem(a=_t(prob.a), b=_t(prob.b), eta=prob.eta, C=torch.tensor(prob.C, dtype=cost_dtype, device="cuda"))
    prm = G.params(precision="mixed" if precision == "ff" else precision, **kw)
    return G.Context(gp, prm)


def _state(prob, k, seed, scale=0.3):
    """Oracle log X^k after k outer updates with random potentials, the GPU's
    cumulative Gamma^k, and a current gamma."""
    rng = np.random.default_rng(seed)
    logX = O.initial_log_plan(prob.a, prob.b)
    Gam = np.zeros(prob.n)
    for _ in range(k):
        g = rng.normal(0.0, scale * prob.eta, prob.n)
        logX = np.log(prob.a)[:, None] + O.log_plan(logX, prob.C, prob.eta, g)
        Gam += g
    gamma = rng.normal(0.0, scale * prob.eta, prob.n)
    return logX, Gam, gamma


# (m, n, eta): n reaches float tile configurations 3, 4, 5, 5 and double 3, 4, 5, 5
WIDE = [(150, 3000, 1e-2), (97, 6000, 1e-2), (61, 12000, 1e-2), (40, 16384, 1e-2),
        (150, 3000, 1e-4), (40, 16384, 1e-4)]
PRECS = ["fp64", "mixed", "ff"]


def _prob(m, n, eta, seed):
    return uniform_points_problem(m, n, seed=seed, eta=eta)


def _plan_tol(prec, eta):
    # float64 passes: exp of exponents up to |(k+1) C / eta| (~4e4 at eta = 1e-4)
    # rounded in float64; float32 passes: float32 anchor and ex2 rounding of
    # |K + d| <= ~60; float-float: ~2^-46 relative
    if prec == "mixed":
        return 2e-5
    return 1e-11 if eta >= 1e-3 else 2e-10


@pytest.mark.parametrize("shape", WIDE, ids=[f"{m}x{n}_eta{eta:g}" for m, n, eta in WIDE])
@pytest.mark.parametrize("prec", PRECS)
def test_wide_anchor_plan_pass(shape, prec):
    m, n, eta = shape
    prob = _prob(m, n, eta, seed=n % 97)
    logX, Gam, gamma = _state(prob, 2, seed=n)
    ctx = _ctx(prob, prec)
    ctx.set_state(2, _t(Gam), _t(gamma), prec)
    P = ctx.export_plan().cpu().numpy()
    Pref = O.plan(logX, prob.C, prob.eta, gamma)
    tol = _plan_tol(prec, eta)
    big = Pref > 1e-30
    if prec == "ff":
        rowmax = Pref.max(axis=1, keepdims=True)
        kept = big & (Pref > 2.0 ** -60 * rowmax)
        assert np.all(P[Pref < 2.0 ** -68 * rowmax] == 0.0)
        big = kept
    rel = np.abs(P[big] - Pref[big]) / Pref[big]
    assert rel.max() <= (1e-12 if prec == "ff" else tol * 60), rel.max()
    assert np.abs(P - Pref).max() <= tol
    c, gn = ctx.plan()
    g_ref = O.gradient(Pref, prob.a, prob.b)
    assert np.abs(c.cpu().numpy() - (g_ref + prob.b)).max() <= tol * 10 * prob.b.max()
    assert abs(gn - np.linalg.norm(g_ref)) <= tol * 10 * np.linalg.norm(g_ref) + 1e-14


@pytest.mark.parametrize("shape", WIDE[:4], ids=[f"{m}x{n}" for m, n, _ in WIDE[:4]])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_wide_sparsify(shape, prec):
    m, n, eta = shape
    prob = _prob(m, n, eta, seed=n % 89)
    logX, Gam, gamma = _state(prob, 1, seed=n + 1)
    ctx = _ctx(prob, prec)
    ctx.set_state(1, _t(Gam), _t(gamma), prec)
    P = O.plan(logX, prob.C, prob.eta, gamma)
    rho = float(np.quantile(P, 0.8))
    nnz = ctx.sparsify(rho)
    Q = ctx.export_sparse().cpu().numpy()
    Qref = O.sparsify_plan(P, prob.a, rho)
    s = O.istar(prob.a)
    tie = np.abs(P - rho) <= (1e-9 if prec == "fp64" else 1e-4) * rho
    rows = ~tie.any(axis=1)
    tol = 1e-12 if prec == "fp64" else 3e-5
    assert rows.sum() >= 0.3 * prob.m
    assert np.abs(Q[rows] - Qref[rows]).max() <= tol
    assert np.abs(Q[s] - Qref[s]).max() <= tol
    assert nnz == int((Q[np.arange(prob.m) != s] > 0).sum())


@pytest.mark.parametrize("shape", WIDE, ids=[f"{m}x{n}_eta{eta:g}" for m, n, eta in WIDE])
@pytest.mark.parametrize("prec", PRECS)
def test_wide_armijo(shape, prec):
    """Difference-form Delta L of the Armijo pass against the oracle's direct
    L(gamma + t Delta) - L(gamma) (Eq. 5), along the GPU's Newton direction."""
    m, n, eta = shape
    prob = _prob(m, n, eta, seed=n % 83)
    logX, Gam, gamma = _state(prob, 2, seed=n + 2)
    ctx = _ctx(prob, prec)
    ctx.set_state(2, _t(Gam), _t(gamma), prec)
    P = O.plan(logX, prob.C, prob.eta, gamma)
    g = O.gradient(P, prob.a, prob.b)
    rho = O.sparsification_threshold(prob.eta, prob.m, prob.n, np.linalg.norm(g)) * 1e4
    ctx.sparsify(rho)
    d, _, _ = ctx.newton_direction(shift=-1.0, rtol=1e-6, max_cg=1000)
    d = d.cpu().numpy()
    L0 = O.semi_dual_objective(logX, prob.C, prob.a, prob.b, prob.eta, gamma)
    for t in (1.0, 0.25):
        if t * np.abs(d).max() / prob.eta > 30.0:
            continue  # outside the float-float pass range: the solver never evaluates it
        dL, slope, _ = ctx.armijo_trial(t, accept=False)
        ref = O.semi_dual_objective(logX, prob.C, prob.a, prob.b, prob.eta, gamma + t * d) - L0
        tol = 1e-5 if prec == "mixed" else 1e-8
        assert abs(dL - ref) <= tol * abs(ref) + 1e-15, (t, dL, ref)
        assert abs(slope - g @ d) <= (1e-5 if prec == "mixed" else 1e-10) * abs(g @ d)


@pytest.mark.parametrize("shape", WIDE, ids=[f"{m}x{n}_eta{eta:g}" for m, n, eta in WIDE])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_wide_stop_check(shape, prec):
    m, n, eta = shape
    prob = _prob(m, n, eta, seed=n % 79)
    logX, Gam, gamma = _state(prob, 2, seed=n + 3)
    ctx = _ctx(prob, prec)
    ctx.set_state(2, _t(Gam), _t(gamma), prec)
    D = ctx.stop_check()
    logXn = np.log(prob.a)[:, None] + O.log_plan(logX, prob.C, prob.eta, gamma)
    Xh = O.round_to_feasible(np.exp(logXn), prob.a, prob.b)[0]
    ref = O.bregman_divergence_log(Xh, logXn)
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert abs(D - ref) <= tol * ref, (D, ref)


@pytest.mark.parametrize("shape", WIDE, ids=[f"{m}x{n}_eta{eta:g}" for m, n, eta in WIDE])
@pytest.mark.parametrize("prec", PRECS)
def test_wide_certify(shape, prec):
    m, n, eta = shape
    prob = _prob(m, n, eta, seed=n % 73)
    logX, Gam, gamma = _state(prob, 2, seed=n + 4)
    ctx = _ctx(prob, prec)
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


def test_full_width_grid_cost_plan_pass():
    """The benchmark's cost kind at its width: 128 x 128 grid bins with the cost
    rebuilt on the fly (m = n = 16384, eta = 1e-4), float32 anchor and
    float-float passes.  The full problem is set up on the GPU; the oracle
    evaluates Eq. 6 on a sample of 48 rows (each row's plan depends only on its
    own row of log X^k), through the explicit outer recursion."""
    import paper_2603_07156_gb300 as G
    from workloads import grid_marginals
    h = 128
    n = h * h
    eta = 1e-4
    a, b, scale = grid_marginals(h, h, seed=2)
    rng = np.random.default_rng(5)
    gp = G.Problem(a=_t(a), b=_t(b), eta=eta, grid=(h, h), cost_scale=scale)
    ctx = G.Context(gp, G.params(precision="mixed"))
    k = 3
    gs = [rng.normal(0.0, 0.3 * eta, n) for _ in range(k)]
    Gam = np.sum(gs, axis=0)
    gam = rng.normal(0.0, 0.3 * eta, n)
    rows = np.sort(rng.choice(n, 48, replace=False))
    idx = np.arange(n)
    Crows = ((rows[:, None] // h - idx[None, :] // h) ** 2 + (rows[:, None] % h - idx[None, :] % h) ** 2) * scale
    logX = np.log(a[rows])[:, None] + np.log(b)[None, :]
    for g in gs:
        logX = np.log(a[rows])[:, None] + O.log_plan(logX, Crows, eta, g)
    Pref = O.plan(logX, Crows, eta, gam)
    sel = torch.tensor(rows, device="cuda")
    for prec in ("mixed", "ff"):
        ctx.set_state(k, _t(Gam), _t(gam), prec)
        P = ctx.export_plan()[sel].cpu().numpy()
        rowmax = Pref.max(axis=1, keepdims=True)
        big = Pref > 2.0 ** -60 * rowmax
        rel = np.abs(P[big] - Pref[big]) / Pref[big]
        if prec == "mixed":
            assert rel.max() <= 2e-5 * 60, rel.max()
            assert np.abs(P - Pref).max() <= 2e-5
        else:
            assert rel.max() <= 1e-12, rel.max()
            assert np.all(P[Pref < 2.0 ** -68 * rowmax] == 0.0)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_grid_wide_newton_direction(prec):
    """A sparsified Hessian above the cluster kernel's capacity (nnz > 1.6e5)
    goes to the grid-wide persistent PCG (float32 or float64).  Its direction
    is compared with the oracle's dense solve of (H_rho + ||g|| I) Delta = -g
    (Alg. 1, Alg. 2), centred like the solver's."""
    prob = uniform_points_problem(320, 2000, seed=61, eta=2e-2)
    logX, Gam, gamma = _state(prob, 2, seed=61)
    ctx = _ctx(prob, prec)
    ctx.set_state(2, _t(Gam), _t(gamma), prec)
    P = O.plan(logX, prob.C, prob.eta, gamma)
    g = O.gradient(P, prob.a, prob.b)
    rho = O.sparsification_threshold(prob.eta, prob.m, prob.n, np.linalg.norm(g))
    nnz = ctx.sparsify(rho)
    assert nnz > 160000
    rtol = 1e-6 if prec == "mixed" else 1e-12
    d, it, res = ctx.newton_direction(shift=-1.0, rtol=rtol, max_cg=2000)
    Hr = O.sparsified_hessian(O.sparsify_plan(P, prob.a, rho), prob.a, prob.eta)
    A = Hr + np.linalg.norm(g) * np.eye(prob.n)
    exact = np.linalg.solve(A, -g)
    exact -= exact.mean()
    d = d.cpu().numpy()
    # the relative CG residual bounds the error by the condition number on 1-perp;
    # float32 Hessian values add ~1e-7 relative to the operator
    cond = np.linalg.cond(A)
    err = np.abs(d - exact).max() / np.abs(exact).max()
    tol = 1e-8 if prec == "fp64" else max(2e-4, min(1e-2, 10 * cond * 1e-7))
    assert err <= tol, (err, tol, cond, it)
    r = np.linalg.norm(A @ d + g)
    if prec == "fp64":
        assert r <= 1e-10 * np.linalg.norm(g), (r, it)
    else:  # float32 operator: rounding of order 1e-7 ||A|| ||d|| on top of the CG tolerance
        assert r <= 1e-5 * np.linalg.norm(g) + 1e-5 * np.linalg.norm(A, 2) * np.linalg.norm(d), (r, it)
    assert abs(d.sum()) <= 1e-12 * np.abs(d).sum()
    assert g @ d < 0


@pytest.mark.parametrize("hw", [(40, 40), (128, 128), (37, 52)])
def test_grid_ctransform_separable(hw):
    """The certificate's c-transform for the grid cost, computed through the
    separability of the squared grid distance, against the scan over all bins
    of App. C.1 (numpy, float64): equal up to rounding order."""
    import paper_2603_07156_gb300 as G
    from workloads import grid_marginals
    h, w = hw
    a, b, scale = grid_marginals(h, w, seed=3)
    n = h * w
    eta = 1e-3
    rng = np.random.default_rng(h * w)
    gamma = rng.normal(0.0, 0.05, n)
    gp = G.Problem(a=_t(a), b=_t(b), eta=eta, grid=(h, w), cost_scale=scale)
    ctx = G.Context(gp, G.params(precision="mixed"))
    ctx.set_state(1, None, _t(gamma), "ff")
    cert = ctx.certify(want_plan=False)
    z = cert["zeta"].cpu().numpy()
    gam = ctx.gamma().cpu().numpy()
    idx = np.arange(n)
    zref = np.empty(n)
    for r0 in range(0, n, 2048):
        rows = idx[r0:r0 + 2048]
        C = ((rows[:, None] // w - idx[None, :] // w) ** 2 + (rows[:, None] % w - idx[None, :] % w) ** 2) * scale
        zref[r0:r0 + 2048] = (C - gam[None, :]).min(axis=1)
    assert np.abs(z - zref).max() <= 1e-15 * (1.0 + np.abs(gam).max())

"""The workspace-free plan pass, called through the C ABI.

ibsn_plan_pass_noalloc serves callers that cannot allocate device memory or
hand over a workspace: its scratch is a fixed array inside the library.  This
file checks that two calls in a row give the same column sums and gradient
norm as the workspace-based path (ibsn_ctx_set_state + ibsn_ctx_plan, float64
passes), within the float64 tolerance of the step tests, and that oversized
problems are refused.  It is collected last on purpose.
"""

import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads import grid_problem, uniform_points_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_07156_gb300 import build as B
    B.build()


def _reference(gp, k, Gam, gam):
    import paper_2603_07156_gb300 as G
    ctx = G.Context(gp, G.params(precision="fp64"))
    ctx.set_state(k, Gam, gam, "fp64")
    c, gn = ctx.plan()
    ctx.close()
    return c.cpu().numpy(), gn


def _noalloc(lib, pr, k, Gam, gam, n):
    from paper_2603_07156_gb300 import _native as N
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    gn = C.c_double(-1.0)
    stream = torch.cuda.current_stream().cuda_stream
    code = lib.ibsn_plan_pass_noalloc(C.byref(pr), int(k), C.c_void_p(Gam.data_ptr()), C.c_void_p(gam.data_ptr()),
                                      C.c_void_p(out.data_ptr()), C.byref(gn), C.c_void_p(stream))
    N.check(code, "ibsn_plan_pass_noalloc")
    torch.cuda.synchronize()
    return out.cpu().numpy(), gn.value


@pytest.mark.parametrize("which", ["dense_ragged", "grid"])
def test_noalloc_matches_workspace_path_twice(which):
    import paper_2603_07156_gb300 as G
    from paper_2603_07156_gb300 import _native as N
    lib = N.load()
    if which == "dense_ragged":
        prob = uniform_points_problem(300, 217, seed=91, eta=1e-2)
        gp = G.Problem(a=torch.tensor(prob.a, device="cuda"), b=torch.tensor(prob.b, device="cuda"), eta=prob.eta,
                       C=torch.tensor(prob.C, device="cuda"))
    else:
        prob = grid_problem(20, 20, seed=92, eta=1e-2)
        gp = G.Problem(a=torch.tensor(prob.a, device="cuda"), b=torch.tensor(prob.b, device="cuda"), eta=prob.eta,
                       grid=prob.grid, cost_scale=prob.cost_scale)
    rng = np.random.default_rng(93)
    Gam = torch.tensor(rng.normal(0, 0.5 * prob.eta, prob.n), device="cuda")
    gam = torch.tensor(rng.normal(0, 0.5 * prob.eta, prob.n), device="cuda")
    k = 3
    c_ref, gn_ref = _reference(gp, k, Gam, gam)
    # the oracle's plan at an iterate whose cumulative potential is Gamma:
    # k outer updates by Gamma / k each (Alg. 2 outer update)
    from oracle import ibsn as O
    Gh, gh = Gam.cpu().numpy(), gam.cpu().numpy()
    logX = O.initial_log_plan(prob.a, prob.b)
    for _ in range(k):
        logX = np.log(prob.a)[:, None] + O.log_plan(logX, prob.C, prob.eta, Gh / k)
    c_orc = O.plan(logX, prob.C, prob.eta, gh).T @ prob.a
    pr = gp.struct()
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        c, gn = _noalloc(lib, pr, k, Gam, gam, prob.n)
        assert np.abs(c - c_ref).max() <= 1e-11 * prob.b.max()
        assert np.abs(c - c_orc).max() <= 1e-11 * prob.b.max()
        assert abs(gn - gn_ref) <= 1e-10 * max(gn_ref, 1e-12)


def test_noalloc_matches_oracle_at_the_size_limit():
    """n = 4096 (the largest accepted width) and m = 1000 rows: the finish
    kernel loops over four columns per thread and every one of the 128 column
    partials of the scratch is used.  Compared with the workspace path and with
    the float64 oracle's column sums P^T a of the row-normalised plan (Eqs. 6-7)
    at the same outer iterate, on two calls in a row."""
    import paper_2603_07156_gb300 as G
    from oracle import ibsn as O
    from paper_2603_07156_gb300 import _native as N
    lib = N.load()
    prob = uniform_points_problem(1000, 4096, seed=94, eta=1e-2)
    gp = G.Problem(a=torch.tensor(prob.a, device="cuda"), b=torch.tensor(prob.b, device="cuda"), eta=prob.eta,
                   C=torch.tensor(prob.C, device="cuda"))
    rng = np.random.default_rng(95)
    k = 2
    gs = [rng.normal(0, 0.3 * prob.eta, prob.n) for _ in range(k)]
    gamma = rng.normal(0, 0.3 * prob.eta, prob.n)
    # oracle: explicit outer recursion log X^{j+1} = log(diag(a) P^j(g_j)) from X^0 = a b^T
    logX = O.initial_log_plan(prob.a, prob.b)
    for g in gs:
        logX = np.log(prob.a)[:, None] + O.log_plan(logX, prob.C, prob.eta, g)
    P = O.plan(logX, prob.C, prob.eta, gamma)
    c_orc = P.T @ prob.a
    gn_orc = float(np.linalg.norm(O.gradient(P, prob.a, prob.b)))
    Gam = torch.tensor(np.sum(gs, axis=0), device="cuda")
    gam = torch.tensor(gamma, device="cuda")
    c_ref, gn_ref = _reference(gp, k, Gam, gam)
    pr = gp.struct()
    for _ in range(2):
        c, gn = _noalloc(lib, pr, k, Gam, gam, prob.n)
        assert np.abs(c - c_ref).max() <= 1e-11 * prob.b.max()
        assert np.abs(c - c_orc).max() <= 1e-11 * prob.b.max()
        assert abs(gn - gn_orc) <= 1e-10 * gn_orc


def test_noalloc_refuses_oversized_problems():
    import paper_2603_07156_gb300 as G
    from paper_2603_07156_gb300 import _native as N
    lib = N.load()
    n = 4097
    a = torch.full((2,), 0.5, dtype=torch.float64, device="cuda")
    b = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    Cm = torch.zeros((2, n), dtype=torch.float64, device="cuda")
    pr = G.Problem(a=a, b=b, eta=1e-2, C=Cm).struct()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    code = lib.ibsn_plan_pass_noalloc(C.byref(pr), 0, None, None, C.c_void_p(out.data_ptr()), None, None)
    assert code == 8  # IBSN_ERR_UNSUPPORTED

"""Batched solve (ibsn_solve_batch) of uneven independent problems on the GPU.

The batched call runs the problems concurrently on several streams; every
solve is deterministic and independent, so its results must equal solving
the problems one by one, bit for bit, and each must certify the LP optimum
(checked against the float64 oracle's network simplex on the small ones).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import lp as LP  # noqa: E402
from workloads import batched_problems  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_07156_gb300 import build as B
    B.build()


def _gpu(prob, cost_dtype=torch.float32):
    import paper_2603_07156_gb300 as G
    return G.Problem(a=torch.tensor(prob.a, device="cuda"), b=torch.tensor(prob.b, device="cuda"), eta=prob.eta,
                     C=torch.tensor(prob.C, dtype=cost_dtype, device="cuda"))


def test_batch_equals_one_by_one():
    import paper_2603_07156_gb300 as G
    probs = batched_problems(count=4, lo=20, hi=64, eta=1e-4)
    gps = [_gpu(p) for p in probs]
    prm = G.params(precision="mixed")
    batch = G.solve_batch(gps, prm, threads=2)
    for p, gp, rb in zip(probs, gps, batch):
        r1 = G.solve(gp, prm)
        assert rb["status"] in (0, 9)
        assert rb["primal"] == r1["primal"] and rb["dual"] == r1["dual"]
        assert rb["outer_iters"] == r1["outer_iters"] and rb["cg_iters"] == r1["cg_iters"]
        assert torch.equal(rb["gamma"], r1["gamma"])
        assert rb["converged"] and rb["rel_gap"] <= 1e-8


def test_batch_certifies_lp_optima():
    import paper_2603_07156_gb300 as G
    probs = batched_problems(count=3, lo=20, hi=40, eta=1e-4, seed0=300)
    gps = [_gpu(p, torch.float64) for p in probs]
    out = G.solve_batch(gps, G.params(precision="fp64"), threads=4)
    for p, r in zip(probs, out):
        opt = LP.network_simplex(p.C, p.a, p.b)[0]
        assert r["converged"]
        assert abs(r["primal"] - opt) <= 1e-8 * abs(opt)
        assert r["dual"] <= opt * (1 + 1e-12) + 1e-15


def test_empty_batch_and_bad_arguments():
    import ctypes as C
    from paper_2603_07156_gb300 import _native as N
    lib = N.load()
    assert lib.ibsn_solve_batch(0, None, None, None, None, None, None, 0) == 0
    assert lib.ibsn_solve_batch(-1, None, None, None, None, None, None, 0) == 1
    prm = N.IbsnParams()
    lib.ibsn_params_default(C.byref(prm))
    assert lib.ibsn_solve_batch(2, None, C.byref(prm), None, None, None, None, 0) == 1

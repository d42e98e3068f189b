"""Failure detection without a GPU fault: bounded device waits.

The persistent PCG kernels (Newton direction of Alg. 2) synchronise their
blocks with grid-wide barriers whose waits are bounded in time.  Here one
block is withheld from such a barrier (a count that nothing completes), so
the wait must run out: the call returns IBSN_ERR_TIMEOUT within about the
requested limit, and afterwards the same barrier, and a full solve, still
work in the same CUDA context.  Nothing traps, faults or hangs.
"""

import ctypes as C
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads import uniform_points_problem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_07156_gb300 import build as B
    B.build()


def test_withheld_barrier_times_out_and_context_stays_usable():
    import paper_2603_07156_gb300 as G
    from paper_2603_07156_gb300 import _native as N
    lib = N.load()
    scratch = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = min(64, nsm)
    assert lib.ibsn_wait_probe(blocks, 0, 0.5, C.c_void_p(scratch.data_ptr()), C.c_void_p(st)) == 0
    t0 = time.perf_counter()
    code = lib.ibsn_wait_probe(blocks, 1, 0.2, C.c_void_p(scratch.data_ptr()), C.c_void_p(st))
    dt = time.perf_counter() - t0
    assert code == 6, code  # IBSN_ERR_TIMEOUT
    assert 0.15 <= dt <= 5.0, dt
    # the context is still usable: the barrier completes, and a solve converges
    assert lib.ibsn_wait_probe(blocks, 0, 0.5, C.c_void_p(scratch.data_ptr()), C.c_void_p(st)) == 0
    prob = uniform_points_problem(40, 50, seed=7, eta=1e-3)
    t = lambda v: torch.tensor(v, dtype=torch.float64, device="cuda")  # noqa: E731
    res = G.solve(G.Problem(a=t(prob.a), b=t(prob.b), eta=prob.eta, C=t(prob.C)), G.params(precision="mixed"))
    assert res["converged"] and res["rel_gap"] <= 1e-8


def test_wait_probe_argument_errors():
    from paper_2603_07156_gb300 import _native as N
    lib = N.load()
    scratch = torch.zeros(2, dtype=torch.int64, device="cuda")
    p = C.c_void_p(scratch.data_ptr())
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert lib.ibsn_wait_probe(1, 0, 0.1, p, None) == 1
    assert lib.ibsn_wait_probe(nsm + 1, 0, 0.1, p, None) == 1
    assert lib.ibsn_wait_probe(4, 0, 0.0, p, None) == 1
    assert lib.ibsn_wait_probe(4, 0, 11.0, p, None) == 1
    assert lib.ibsn_wait_probe(4, 0, 0.1, None, None) == 1
    assert np.all(scratch.cpu().numpy() == 0)

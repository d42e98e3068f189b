"""C ABI checks that need no GPU: the library loads, exports every function
declared in include/ibsn.h, and the ctypes structs match the C layout."""

import ctypes
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_07156_gb300 import build as B
    B.build()
    from paper_2603_07156_gb300 import _native as N
    return N.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2603_07156_gb300 import _native as N
    names = N.header_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name
    # and the binding declares a signature for each of them
    assert set(names) == set(N._SIGS)


def test_struct_layout_matches_c_compiler():
    from paper_2603_07156_gb300 import _native as N
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "ibsn.h"
#define F(T, f) printf(#T " " #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("sizeof ibsn_problem %zu\n", sizeof(ibsn_problem));
  printf("sizeof ibsn_params %zu\n", sizeof(ibsn_params));
  printf("sizeof ibsn_result %zu\n", sizeof(ibsn_result));
  F(ibsn_problem, eta); F(ibsn_problem, cost_kind); F(ibsn_problem, grid_w); F(ibsn_problem, dim); F(ibsn_problem, x); F(ibsn_problem, y);
  F(ibsn_params, gamma0); F(ibsn_params, nnz_cap); F(ibsn_params, max_outer); F(ibsn_params, profile); F(ibsn_params, eot_gtol); F(ibsn_params, eot); F(ibsn_params, recompute);
  F(ibsn_result, primal); F(ibsn_result, outer_iters); F(ibsn_result, status); F(ibsn_result, dense_passes);
  F(ibsn_result, kernel_launches); F(ibsn_result, pass_ms); F(ibsn_result, pass_calls); F(ibsn_result, pass_bytes);
  printf("sizeof ibsn_ws_batch %zu\n", sizeof(ibsn_ws_batch));
  printf("sizeof ibsn_ws_adam %zu\n", sizeof(ibsn_ws_adam));
  F(ibsn_ws_batch, m); F(ibsn_ws_batch, n); F(ibsn_ws_batch, x); F(ibsn_ws_batch, b);
  F(ibsn_ws_adam, lr); F(ibsn_ws_adam, eps);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if not line:
            continue
        parts = line.split()
        got[(parts[0], parts[1])] = int(parts[2])
    assert got[("sizeof", "ibsn_problem")] == ctypes.sizeof(N.IbsnProblem)
    assert got[("sizeof", "ibsn_params")] == ctypes.sizeof(N.IbsnParams)
    assert got[("sizeof", "ibsn_result")] == ctypes.sizeof(N.IbsnResult)
    assert got[("sizeof", "ibsn_ws_batch")] == ctypes.sizeof(N.IbsnWsBatch)
    assert got[("sizeof", "ibsn_ws_adam")] == ctypes.sizeof(N.IbsnWsAdam)
    structs = {"ibsn_problem": N.IbsnProblem, "ibsn_params": N.IbsnParams, "ibsn_result": N.IbsnResult,
               "ibsn_ws_batch": N.IbsnWsBatch, "ibsn_ws_adam": N.IbsnWsAdam}
    for (s, f), off in got.items():
        if s in structs:
            assert getattr(structs[s], f).offset == off, (s, f)


def test_defaults_are_the_papers_constants(lib):
    from paper_2603_07156_gb300 import _native as N
    p = N.IbsnParams()
    lib.ibsn_params_default(ctypes.byref(p))
    assert p.sigma == 1e-4 and p.beta == 0.8          # Alg. 2 inputs
    assert p.sinkhorn_tol == 1e-3                     # Sec. 5 warm-up stop
    assert p.mu0 == 1e-4 and p.mu_min == 1e-11        # Eq. 8
    assert p.sparsify == 1


def test_status_strings(lib):
    for code in range(11):
        assert lib.ibsn_status_string(code)
    assert lib.ibsn_status_string(99) == b"unknown status"


def test_workspace_size_rejects_bad_problems(lib):
    from paper_2603_07156_gb300 import _native as N
    pr = N.IbsnProblem()
    pm = N.IbsnParams()
    lib.ibsn_params_default(ctypes.byref(pm))
    out = ctypes.c_size_t()
    pr.m, pr.n, pr.eta = 4, 4, 1e-3
    assert lib.ibsn_workspace_size(ctypes.byref(pr), ctypes.byref(pm), ctypes.byref(out)) == 1  # null a, b
    pr.a, pr.b, pr.C, pr.ldc = 8, 8, 8, 4
    pr.eta = -1.0
    assert lib.ibsn_workspace_size(ctypes.byref(pr), ctypes.byref(pm), ctypes.byref(out)) == 1
    pr.eta = 1e-3
    pr.n, pr.ldc = 70000, 70000
    assert lib.ibsn_workspace_size(ctypes.byref(pr), ctypes.byref(pm), ctypes.byref(out)) == 8  # unsupported
    pr.n, pr.ldc = 4, 2
    assert lib.ibsn_workspace_size(ctypes.byref(pr), ctypes.byref(pm), ctypes.byref(out)) == 1  # ldc < n


def test_warm_start_host_checks(lib):
    """Parameter count, Adam defaults and argument checks of the warm-start
    calls (paths that return before any device work)."""
    from paper_2603_07156_gb300 import _native as N
    assert lib.ibsn_ws_param_count() == 50433
    hp = N.IbsnWsAdam()
    lib.ibsn_ws_adam_default(ctypes.byref(hp))
    assert (hp.lr, hp.beta1, hp.beta2, hp.eps) == (1e-3, 0.9, 0.999, 1e-8)
    out = ctypes.c_size_t()
    b = N.IbsnWsBatch()
    b.count = 0
    assert lib.ibsn_ws_workspace_size(ctypes.byref(b), ctypes.byref(out)) == 1
    ms = (ctypes.c_int64 * 2)(5, 300)
    ns = (ctypes.c_int64 * 2)(7, 1)
    b.count, b.m, b.n = 2, ms, ns
    assert lib.ibsn_ws_workspace_size(ctypes.byref(b), ctypes.byref(out)) == 0
    small = out.value
    assert small >= 4 * 128 * (305 * 2 + 8 * 4) and small % 256 == 0
    ms[1] = 3000
    assert lib.ibsn_ws_workspace_size(ctypes.byref(b), ctypes.byref(out)) == 0 and out.value > small
    ms[1] = 16385
    assert lib.ibsn_ws_workspace_size(ctypes.byref(b), ctypes.byref(out)) == 8      # above the point limit
    ms[1] = 0
    assert lib.ibsn_ws_workspace_size(ctypes.byref(b), ctypes.byref(out)) == 1      # empty cloud
    ms[1] = 300
    # null device pointers, then a misaligned workspace: rejected before any device work
    assert lib.ibsn_ws_predict(ctypes.byref(b), 256, 256, 256, 1 << 30, None) == 1
    b.x = b.y = b.a = b.b = 256
    assert lib.ibsn_ws_predict(ctypes.byref(b), 256, 256, 300, 1 << 30, None) == 4
    assert lib.ibsn_ws_predict(ctypes.byref(b), 256, 256, 512, 16, None) == 4       # too small
    assert lib.ibsn_ws_adam_step(10, 256, 256, 256, 256, 0, ctypes.byref(hp), None) == 1  # t = 0
    hp.beta1 = 1.0
    assert lib.ibsn_ws_adam_step(10, 256, 256, 256, 256, 1, ctypes.byref(hp), None) == 1

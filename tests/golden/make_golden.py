"""Write tests/golden/oracle_optima.json from the CPU oracle and the exact LP references.

Only oracle/ and workloads/ are used; nothing here touches the CUDA path.
Run:  python tests/golden/make_golden.py
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ibsn as O  # noqa: E402
from oracle import lp  # noqa: E402
from workloads import grid_problem, uniform_points_problem, workload  # noqa: E402


def main():
    out = {"source": "oracle/ibsn.py (Alg. 2, FP64) and oracle/lp.py network simplex; inputs from workloads/",
           "cases": {}}
    cases = {
        "c0_uniform2d_256": workload("c0"),
        "uniform2d_96x131_s21": uniform_points_problem(96, 131, seed=21, eta=1e-4),
        "grid16x16_s2": grid_problem(16, 16, seed=2, eta=1e-3),
    }
    for name, prob in cases.items():
        t = time.time()
        res = O.ibsn(prob.C, prob.a, prob.b, O.IBSNParams(eta=prob.eta, gap_tol=1e-9))
        t_or = time.time() - t
        t = time.time()
        opt, X, u, v = lp.network_simplex(prob.C, prob.a, prob.b)
        t_lp = time.time() - t
        out["cases"][name] = dict(m=prob.m, n=prob.n, eta=prob.eta, oracle_primal=res.primal, oracle_dual=res.dual,
                                  oracle_gap=res.rel_gap, oracle_outer=res.outer_iters, lp_optimum=opt,
                                  oracle_seconds=round(t_or, 2), lp_seconds=round(t_lp, 2))
        print(name, out["cases"][name], flush=True)
    with open(os.path.join(HERE, "oracle_optima.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

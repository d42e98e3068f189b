"""Python front end of the IBSN CUDA library.

Thin marshalling over the C ABI of include/ibsn.h: tensors are passed as
device pointers, the stream as torch's current CUDA stream, and the
workspace as a torch-allocated byte buffer.  Every step runs in the
library's kernels.
"""

from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _native as N

COST_DENSE_F64, COST_DENSE_F32, COST_GRID2D, COST_SQEUCLID_POINTS = 0, 1, 2, 3
PREC_FP64, PREC_MIXED = 0, 1
_PREC = {"fp64": PREC_FP64, "mixed": PREC_MIXED, "ff": 2, PREC_FP64: PREC_FP64, PREC_MIXED: PREC_MIXED, 2: 2}


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _stream_ptr(stream: torch.cuda.Stream | None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def params(**overrides) -> N.IbsnParams:
    """ibsn_params_default() plus keyword overrides (names as in the C struct;
    precision may be 'fp64' or 'mixed')."""
    lib = N.load()
    p = N.IbsnParams()
    lib.ibsn_params_default(C.byref(p))
    for k, v in overrides.items():
        if k == "precision":
            v = _PREC[v]
        if k == "gamma0":
            v = _ptr(v)
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


@dataclass
class Problem:
    """An OT instance on the GPU (Eq. 1).  Keeps the tensors alive."""

    a: torch.Tensor
    b: torch.Tensor
    eta: float
    C: torch.Tensor | None = None
    grid: tuple[int, int] | None = None
    cost_scale: float = 1.0
    x: torch.Tensor | None = None  # point cost: (m, dim) float64 source points
    y: torch.Tensor | None = None  # point cost: (n, dim) float64 target points

    def __post_init__(self):
        for name in ("a", "b"):
            t = getattr(self, name)
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
        if self.x is not None or self.y is not None:
            for name in ("x", "y"):
                t = getattr(self, name)
                if t is None or t.dtype != torch.float64 or not t.is_cuda or t.dim() != 2 or not t.is_contiguous():
                    raise ValueError(f"{name} must be a contiguous 2-D float64 CUDA tensor")
            if self.x.shape[1] != self.y.shape[1]:
                raise ValueError("x and y must have the same number of coordinates")
        if self.C is not None:
            if self.C.dtype not in (torch.float64, torch.float32) or not self.C.is_cuda or self.C.dim() != 2:
                raise ValueError("C must be a 2-D float32/float64 CUDA tensor")
            if self.C.stride(1) != 1:
                raise ValueError("C rows must be contiguous")

    def struct(self) -> N.IbsnProblem:
        s = N.IbsnProblem()
        s.m, s.n = int(self.a.numel()), int(self.b.numel())
        s.a, s.b = _ptr(self.a), _ptr(self.b)
        s.eta = float(self.eta)
        if self.x is not None:
            s.cost_kind = COST_SQEUCLID_POINTS
            s.x, s.y = _ptr(self.x), _ptr(self.y)
            s.dim = int(self.x.shape[1])
            s.cost_scale = float(self.cost_scale)
            s.ldc = s.n
        elif self.grid is not None:
            s.cost_kind = COST_GRID2D
            s.grid_h, s.grid_w = int(self.grid[0]), int(self.grid[1])
            s.cost_scale = float(self.cost_scale)
            s.ldc = s.n
        else:
            s.cost_kind = COST_DENSE_F64 if self.C.dtype == torch.float64 else COST_DENSE_F32
            s.C = _ptr(self.C)
            s.ldc = int(self.C.stride(0))
            s.cost_scale = 1.0
        return s


def workspace_size(problem: Problem, prm: N.IbsnParams) -> int:
    lib = N.load()
    out = C.c_size_t(0)
    pr = problem.struct()
    N.check(lib.ibsn_workspace_size(C.byref(pr), C.byref(prm), C.byref(out)), "ibsn_workspace_size")
    return int(out.value)


def alloc_workspace(problem: Problem, prm: N.IbsnParams) -> torch.Tensor:
    nbytes = workspace_size(problem, prm)
    return torch.empty(nbytes, dtype=torch.uint8, device=problem.a.device)


def solve(problem: Problem, prm: N.IbsnParams | None = None, *, want_plan: bool = False,
          workspace: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None) -> dict:
    """Run ibsn_solve; returns the result fields plus gamma, zeta (and plan)."""
    lib = N.load()
    prm = prm if prm is not None else params()
    ws = workspace if workspace is not None else alloc_workspace(problem, prm)
    m, n = int(problem.a.numel()), int(problem.b.numel())
    dev = problem.a.device
    gamma = torch.empty(n, dtype=torch.float64, device=dev)
    zeta = torch.empty(m, dtype=torch.float64, device=dev)
    plan = torch.empty((m, n), dtype=torch.float64, device=dev) if want_plan else None
    res = N.IbsnResult()
    res.gamma, res.zeta, res.plan = _ptr(gamma), _ptr(zeta), _ptr(plan)
    pr = problem.struct()
    code = lib.ibsn_solve(C.byref(pr), C.byref(prm), C.c_void_p(ws.data_ptr()), C.c_size_t(ws.numel()),
                          C.byref(res), C.c_void_p(_stream_ptr(stream)))
    N.check(code, "ibsn_solve", allow=(0, 9))
    out = {f: getattr(res, f) for f, _ in N.IbsnResult._fields_
           if f not in ("gamma", "zeta", "plan", "pass_ms", "pass_calls", "pass_bytes")}
    prof = {}
    for q in range(16):
        if res.pass_calls[q]:
            hi = "_ff" if prm.precision == PREC_MIXED else "_f64"
            key = N.PASS_KINDS[q % 8] + (hi if q >= 8 else "_f32")
            prof[key] = dict(ms=res.pass_ms[q], calls=res.pass_calls[q], bytes=res.pass_bytes[q])
    out["profile"] = prof
    out.update(gamma=gamma, zeta=zeta, plan=plan, converged=(code == 0))
    return out


def solve_batch(problems: list, prm: N.IbsnParams | None = None, *, threads: int = 8,
                workspaces: list | None = None) -> list[dict]:
    """ibsn_solve_batch: independent problems solved concurrently (results as
    from solve() one by one); returns one result dict per problem."""
    lib = N.load()
    prm = prm if prm is not None else params()
    count = len(problems)
    if count == 0:
        return []
    wss = workspaces if workspaces is not None else [alloc_workspace(p, prm) for p in problems]
    probs = (N.IbsnProblem * count)(*[p.struct() for p in problems])
    results = (N.IbsnResult * count)()
    gammas, zetas = [], []
    for q, p in enumerate(problems):
        m, n = int(p.a.numel()), int(p.b.numel())
        g = torch.empty(n, dtype=torch.float64, device=p.a.device)
        z = torch.empty(m, dtype=torch.float64, device=p.a.device)
        results[q].gamma, results[q].zeta, results[q].plan = _ptr(g), _ptr(z), None
        gammas.append(g)
        zetas.append(z)
    ptrs = (C.c_void_p * count)(*[w.data_ptr() for w in wss])
    sizes = (C.c_size_t * count)(*[w.numel() for w in wss])
    torch.cuda.synchronize()  # inputs written on torch's streams are complete
    code = lib.ibsn_solve_batch(count, probs, C.byref(prm), ptrs, sizes, results, None, int(threads))
    N.check(code, "ibsn_solve_batch", allow=(0, 9))
    out = []
    for q in range(count):
        r = results[q]
        d = {f: getattr(r, f) for f, _ in N.IbsnResult._fields_
             if f not in ("gamma", "zeta", "plan", "pass_ms", "pass_calls", "pass_bytes")}
        d.update(gamma=gammas[q], zeta=zetas[q], converged=(r.status == 0))
        out.append(d)
    return out


class Context:
    """Step-level access to one run of Alg. 2 (the hot-path rows one by one)."""

    def __init__(self, problem: Problem, prm: N.IbsnParams | None = None,
                 stream: torch.cuda.Stream | None = None):
        self.lib = N.load()
        self.problem = problem
        self.prm = prm if prm is not None else params()
        self.ws = alloc_workspace(problem, self.prm)
        self.stream = _stream_ptr(stream)
        self.m, self.n = int(problem.a.numel()), int(problem.b.numel())
        h = C.c_void_p()
        pr = problem.struct()
        N.check(self.lib.ibsn_ctx_create(C.byref(pr), C.byref(self.prm), C.c_void_p(self.ws.data_ptr()),
                                         C.c_size_t(self.ws.numel()), C.c_void_p(self.stream), C.byref(h)),
                "ibsn_ctx_create")
        self.h = h

    def close(self):
        if self.h:
            self.lib.ibsn_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, k):
        return torch.empty(k, dtype=torch.float64, device=self.problem.a.device)

    def set_state(self, k: int, Gamma: torch.Tensor | None, gamma: torch.Tensor | None, precision="fp64"):
        N.check(self.lib.ibsn_ctx_set_state(self.h, int(k), _ptr(Gamma), _ptr(gamma), _PREC[precision]),
                "ibsn_ctx_set_state")

    def plan(self):
        c = self._vec(self.n)
        gn = C.c_double()
        N.check(self.lib.ibsn_ctx_plan(self.h, C.c_void_p(c.data_ptr()), C.byref(gn)), "ibsn_ctx_plan")
        return c, gn.value

    def export_plan(self) -> torch.Tensor:
        P = torch.empty((self.m, self.n), dtype=torch.float64, device=self.problem.a.device)
        N.check(self.lib.ibsn_ctx_export_plan(self.h, C.c_void_p(P.data_ptr())), "ibsn_ctx_export_plan")
        return P

    def gamma(self) -> torch.Tensor:
        g = self._vec(self.n)
        N.check(self.lib.ibsn_ctx_get_gamma(self.h, C.c_void_p(g.data_ptr())), "ibsn_ctx_get_gamma")
        return g

    def sinkhorn(self, tol: float, max_iter: int):
        it = C.c_int32()
        gn = C.c_double()
        N.check(self.lib.ibsn_ctx_sinkhorn(self.h, float(tol), int(max_iter), C.byref(it), C.byref(gn)),
                "ibsn_ctx_sinkhorn")
        return it.value, gn.value

    def sparsify(self, rho: float) -> int:
        nnz = C.c_int64()
        N.check(self.lib.ibsn_ctx_sparsify(self.h, float(rho), C.byref(nnz)), "ibsn_ctx_sparsify")
        return nnz.value

    def export_sparse(self) -> torch.Tensor:
        P = torch.empty((self.m, self.n), dtype=torch.float64, device=self.problem.a.device)
        N.check(self.lib.ibsn_ctx_export_sparse(self.h, C.c_void_p(P.data_ptr())), "ibsn_ctx_export_sparse")
        return P

    def newton_direction(self, shift: float = -1.0, rtol: float = 1e-12, max_cg: int = 1000):
        d = self._vec(self.n)
        it = C.c_int32()
        rs = C.c_double()
        N.check(self.lib.ibsn_ctx_newton_direction(self.h, float(shift), float(rtol), int(max_cg),
                                                   C.c_void_p(d.data_ptr()), C.byref(it), C.byref(rs)),
                "ibsn_ctx_newton_direction")
        return d, it.value, rs.value

    def armijo_trial(self, t: float, accept: bool = False):
        dL, sl = C.c_double(), C.c_double()
        acc = C.c_int32()
        N.check(self.lib.ibsn_ctx_armijo_trial(self.h, float(t), int(accept), C.byref(dL), C.byref(sl),
                                               C.byref(acc)), "ibsn_ctx_armijo_trial")
        return dL.value, sl.value, bool(acc.value)

    def stop_check(self) -> float:
        d = C.c_double()
        N.check(self.lib.ibsn_ctx_stop_check(self.h, C.byref(d)), "ibsn_ctx_stop_check")
        return d.value

    def certify(self, want_plan: bool = False) -> dict:
        p, d, gap, viol = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        plan = torch.empty((self.m, self.n), dtype=torch.float64, device=self.problem.a.device) if want_plan else None
        zeta = self._vec(self.m)
        N.check(self.lib.ibsn_ctx_certify(self.h, C.byref(p), C.byref(d), C.byref(gap), C.byref(viol),
                                          C.c_void_p(_ptr(plan)), C.c_void_p(zeta.data_ptr())),
                "ibsn_ctx_certify")
        return dict(primal=p.value, dual=d.value, rel_gap=gap.value, marg_viol=viol.value, plan=plan, zeta=zeta)

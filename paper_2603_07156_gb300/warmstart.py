"""Learned warm start: Python front end of the ibsn_ws_* calls and of
ibsn_judge_warm_start in include/ibsn.h (argument marshalling only).

The network's forward pass, backward pass and Adam step run in the
library's kernels.  This module concatenates point clouds into the batch
layout of the C ABI, keeps the tensors alive across calls, and drives the
training loop from the host.
"""

from __future__ import annotations

import ctypes as C

import torch

from . import _native as N
from .api import Problem, _ptr, _stream_ptr, alloc_workspace, solve


def param_count() -> int:
    return int(N.load().ibsn_ws_param_count())


class PointBatch:
    """Q point-cloud problems in the concatenated layout of ibsn_ws_batch.

    xs, ys: per-problem (m_q, 2) / (n_q, 2) coordinates; as_, bs: marginals.
    Any array-likes; stored as contiguous float64 CUDA tensors."""

    def __init__(self, xs, ys, as_, bs, device="cuda"):
        def cat(parts, cols):
            ts = [torch.as_tensor(p, dtype=torch.float64).reshape(-1, cols) if cols else
                  torch.as_tensor(p, dtype=torch.float64).reshape(-1) for p in parts]
            return torch.cat(ts).to(device).contiguous()

        if not (len(xs) == len(ys) == len(as_) == len(bs)) or len(xs) == 0:
            raise ValueError("need the same positive number of clouds and marginals")
        self.m = [int(len(a)) for a in as_]
        self.n = [int(len(b)) for b in bs]
        self.x, self.y = cat(xs, 2), cat(ys, 2)
        self.a, self.b = cat(as_, 0), cat(bs, 0)
        if self.x.shape[0] != sum(self.m) or self.y.shape[0] != sum(self.n):
            raise ValueError("coordinates and marginals disagree in length")
        self._m = (C.c_int64 * len(self.m))(*self.m)
        self._n = (C.c_int64 * len(self.n))(*self.n)
        self._ws = None

    @classmethod
    def from_problems(cls, problems, device="cuda") -> "PointBatch":
        """From OTProblem-like objects with x, y, a, b arrays."""
        return cls([p.x for p in problems], [p.y for p in problems], [p.a for p in problems],
                   [p.b for p in problems], device)

    def struct(self) -> N.IbsnWsBatch:
        s = N.IbsnWsBatch()
        s.count = len(self.m)
        s.m, s.n = self._m, self._n
        s.x, s.y, s.a, s.b = _ptr(self.x), _ptr(self.y), _ptr(self.a), _ptr(self.b)
        return s

    def workspace(self) -> torch.Tensor:
        if self._ws is None:
            out = C.c_size_t(0)
            b = self.struct()
            N.check(N.load().ibsn_ws_workspace_size(C.byref(b), C.byref(out)), "ibsn_ws_workspace_size")
            self._ws = torch.empty(int(out.value), dtype=torch.uint8, device=self.x.device)
        return self._ws

    def split(self, v: torch.Tensor) -> list[torch.Tensor]:
        """Per-problem views of a (sum n) vector."""
        return list(torch.split(v, self.n))


def predict(batch: PointBatch, theta: torch.Tensor, stream=None) -> torch.Tensor:
    """gamma_hat (sum n, float64, centred per problem) from float32 parameters."""
    _check_theta(theta)
    out = torch.empty(sum(batch.n), dtype=torch.float64, device=batch.x.device)
    ws = batch.workspace()
    b = batch.struct()
    N.check(N.load().ibsn_ws_predict(C.byref(b), _ptr(theta), _ptr(out), _ptr(ws), ws.numel(), _stream_ptr(stream)),
            "ibsn_ws_predict")
    return out


def loss_grad(batch: PointBatch, theta: torch.Tensor, gamma_star: torch.Tensor, stream=None,
              grad: torch.Tensor | None = None):
    """(loss, grad, gamma_hat) of the batch against targets gamma_star (sum n)."""
    _check_theta(theta)
    if gamma_star.dtype != torch.float64 or gamma_star.numel() != sum(batch.n) or not gamma_star.is_contiguous():
        raise ValueError("gamma_star must be a contiguous float64 tensor of sum(n) values")
    g = grad if grad is not None else torch.empty_like(theta)
    gh = torch.empty(sum(batch.n), dtype=torch.float64, device=batch.x.device)
    loss = C.c_double(0.0)
    ws = batch.workspace()
    b = batch.struct()
    N.check(N.load().ibsn_ws_loss_grad(C.byref(b), _ptr(theta), _ptr(gamma_star), C.byref(loss), _ptr(g), _ptr(gh),
                                       _ptr(ws), ws.numel(), _stream_ptr(stream)), "ibsn_ws_loss_grad")
    return float(loss.value), g, gh


def adam_hparams(**kw) -> N.IbsnWsAdam:
    hp = N.IbsnWsAdam()
    N.load().ibsn_ws_adam_default(C.byref(hp))
    for k, v in kw.items():
        setattr(hp, k, float(v))
    return hp


def adam_step(theta, m1, m2, grad, t: int, hp: N.IbsnWsAdam | None = None, stream=None) -> None:
    """One Adam step (in place on theta, m1, m2)."""
    hp = hp if hp is not None else adam_hparams()
    for name, v in (("theta", theta), ("m1", m1), ("m2", m2), ("grad", grad)):
        if v.dtype != torch.float32 or not v.is_cuda or not v.is_contiguous() or v.numel() != theta.numel():
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor like theta")
    N.check(N.load().ibsn_ws_adam_step(theta.numel(), _ptr(theta), _ptr(m1), _ptr(m2), _ptr(grad), int(t),
                                       C.byref(hp), _stream_ptr(stream)), "ibsn_ws_adam_step")


class Trainer:
    """Adam on the network over minibatches of solved problems."""

    def __init__(self, theta0, hp: N.IbsnWsAdam | None = None, device="cuda"):
        self.theta = torch.as_tensor(theta0, dtype=torch.float32).to(device).contiguous()
        if self.theta.numel() != param_count():
            raise ValueError("wrong number of parameters")
        self.m1 = torch.zeros_like(self.theta)
        self.m2 = torch.zeros_like(self.theta)
        self.grad = torch.empty_like(self.theta)
        self.hp = hp if hp is not None else adam_hparams()
        self.t = 0

    def step(self, batch: PointBatch, gamma_star: torch.Tensor) -> float:
        loss, _, _ = loss_grad(batch, self.theta, gamma_star, grad=self.grad)
        self.t += 1
        adam_step(self.theta, self.m1, self.m2, self.grad, self.t, self.hp)
        return loss


def judge(problem: Problem, prm: N.IbsnParams, gamma_hat: torch.Tensor, workspace=None, stream=None,
          fallback: torch.Tensor | None = None) -> dict:
    """ibsn_judge_warm_start: the semi-dual objective L^0 (Eq. 5) and the
    gradient norm from gamma_hat and from the fallback start (zero, or the
    given potential); use_warm when gamma_hat's L^0 is smaller."""
    ws = workspace if workspace is not None else alloc_workspace(problem, prm)
    lw, lz, gw, gz = (C.c_double(0.0) for _ in range(4))
    use = C.c_int32(0)
    pr = problem.struct()
    N.check(N.load().ibsn_judge_warm_start(C.byref(pr), C.byref(prm), _ptr(gamma_hat), _ptr(fallback), _ptr(ws),
                                           ws.numel(),
                                           C.byref(lw), C.byref(lz), C.byref(gw), C.byref(gz), C.byref(use),
                                           _stream_ptr(stream)), "ibsn_judge_warm_start")
    return dict(use_warm=bool(use.value), objective_warm=lw.value, objective_fallback=lz.value,
                grad_norm_warm=gw.value, grad_norm_fallback=gz.value)


def solve_warm(problem: Problem, prm: N.IbsnParams, gamma_hat: torch.Tensor, workspace=None,
               fallback: torch.Tensor | None = None, **kw) -> dict:
    """Judge gamma_hat against the fallback start (zero, or the given
    potential), then solve from the winner.  The result carries warm_used
    and the judge's objectives and gradient norms."""
    if fallback is None and prm.gamma0:
        raise ValueError("prm.gamma0 is set: pass that start as `fallback` so that the judge compares with it")
    ws = workspace if workspace is not None else alloc_workspace(problem, prm)
    j = judge(problem, prm, gamma_hat, ws, fallback=fallback)
    p2 = N.IbsnParams.from_buffer_copy(prm)
    p2.gamma0 = _ptr(gamma_hat) if j["use_warm"] else _ptr(fallback)
    res = solve(problem, p2, workspace=ws, **kw)
    res.update(warm_used=j["use_warm"], **{k: v for k, v in j.items() if k != "use_warm"})
    return res


def _check_theta(theta: torch.Tensor) -> None:
    if theta.dtype != torch.float32 or not theta.is_cuda or not theta.is_contiguous() or \
            theta.numel() != param_count():
        raise ValueError("theta must be a contiguous float32 CUDA tensor of ibsn_ws_param_count() values")


__all__ = ["PointBatch", "param_count", "predict", "loss_grad", "adam_hparams", "adam_step", "Trainer", "judge",
           "solve_warm"]

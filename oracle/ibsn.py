"""Plain float64 oracle of IBSN -- TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Every function restates one definition of the paper (arXiv 2603.07156) in
the paper's notation.  Nothing is blocked, fused or reordered beyond what the
stated definition or algorithm does; numpy/scipy primitives (matmul, exp,
log, argmax) are the only library steps.

Readings where the paper is silent or garbled (same list as the design notes):
  R1  ||.|| is the Euclidean norm everywhere (Sec. 1 notation).
  R2  Newton system sign: Alg. 2 (Delta = -(H_rho + ||g|| I)^{-1} g).
  R3  The Newton system is solved by Jacobi-preconditioned CG from 0, stopped
      when ||r|| <= rtol ||g||, rtol = min(cg_rtol, max(||g||, mu_k / (4 ||g||))),
      or after max_cg iterations: the superlinear forcing term ||g||, relaxed
      to the accuracy at which the linear model already predicts the next
      gradient below the gate mu_k of Eq. 8; the direction is then centred
      (L^k is invariant to gamma + c 1).
  R4  Armijo starts at t = 1, shrinks by beta, at most max_armijo trials.
  R5  Newton phase stop (Eq. 8): gate ||g|| < mu_k, then
      D_phi(Proj(X), X) <= min(m, n) * mu_k, mu_k = max(1e-4/(k+1)^2, 1e-11).
  R6  Alg. 3 as printed (column sums of X for y); identical to the cited
      rounding when X = diag(a) P because then z = 1.
  R7  D_phi is evaluated in the log domain so that underflowed X_ij give
      finite terms; 0 log 0 = 0.
  R9  Threshold keeps P_ij >= rho; i* is the lowest index attaining max a.
  R11 Outer stop: relative duality gap (p - d) / max(|p|, |d|) <= gap_tol with
      p = <C, Proj(X^{k+1})> and d = a^T zeta + b^T gamma, zeta the c-transform
      of the current gamma (App. C.1).
  R13 Sinkhorn warm-up cap max_sinkhorn iterations; R14 Newton cap max_newton.

Parity pins (tests/test_oracle_*.py): finite differences of L^k (gradient,
Hessian), Thm 3.2-3.4 invariants, Lemma 4.1, Alg. 3 feasibility, D_phi
properties, and end-to-end LP optima from oracle/lp.py.  The iteration
trajectory itself (counts per outer step) has no independent pin:
parity unpinned for trajectories; only the certified optimum is pinned.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------
# Eq. 4-7: semi-dual objective, plan, gradient, Hessian
# ----------------------------------------------------------------------------

def initial_log_plan(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """log X^0 with X^0 = a b^T (Alg. 2 input)."""
    return np.log(a)[:, None] + np.log(b)[None, :]


def _exponent(logX: np.ndarray, C: np.ndarray, eta: float, gamma: np.ndarray) -> np.ndarray:
    """log( X^k_ij exp((gamma_j - C_ij)/eta) ), the summand of Eq. 5 in log form."""
    return logX + (gamma[None, :] - C) / eta


def _logsumexp_rows(E: np.ndarray) -> np.ndarray:
    mx = E.max(axis=1)
    return mx + np.log(np.exp(E - mx[:, None]).sum(axis=1))


def semi_dual_objective(logX, C, a, b, eta, gamma) -> float:
    """L^k(gamma) = -b^T gamma + eta sum_i a_i log sum_j X^k_ij exp((gamma_j - C_ij)/eta)  (Eq. 5)."""
    return float(-b @ gamma + eta * (a @ _logsumexp_rows(_exponent(logX, C, eta, gamma))))


def best_zeta(logX, C, a, eta, gamma) -> np.ndarray:
    """zeta(gamma)_i = eta log a_i - eta log sum_j X^k_ij exp((gamma_j - C_ij)/eta)  (Eq. 4)."""
    return eta * np.log(a) - eta * _logsumexp_rows(_exponent(logX, C, eta, gamma))


def log_plan(logX, C, eta, gamma) -> np.ndarray:
    """log P^k(gamma): row-normalised log of X^k_ij exp((gamma_j - C_ij)/eta)  (Eq. 6)."""
    E = _exponent(logX, C, eta, gamma)
    return E - _logsumexp_rows(E)[:, None]


def plan(logX, C, eta, gamma) -> np.ndarray:
    """P^k(gamma) (Eq. 6)."""
    return np.exp(log_plan(logX, C, eta, gamma))


def gradient(P, a, b) -> np.ndarray:
    """g^k(gamma) = P^T a - b  (Eq. 7)."""
    return P.T @ a - b


def hessian(P, a, eta) -> np.ndarray:
    """H^k(gamma) = (diag(P^T a) - P^T diag(a) P) / eta  (Eq. 7)."""
    return (np.diag(P.T @ a) - P.T @ (a[:, None] * P)) / eta


# ----------------------------------------------------------------------------
# Alg. 1: sparsified Hessian
# ----------------------------------------------------------------------------

def istar(a) -> int:
    """i* = argmax_i a_i, lowest index on ties (reading R9)."""
    return int(np.argmax(a))


def sparsify_plan(P, a, rho) -> np.ndarray:
    """P_rho of Alg. 1: keep P_ij >= rho, renormalise rows to 1; row i* kept as is."""
    keep = P >= rho
    Q = np.where(keep, P, 0.0)
    Q = Q / Q.sum(axis=1, keepdims=True)
    s = istar(a)
    Q[s, :] = P[s, :]
    return Q


def sparsified_hessian(P_rho, a, eta) -> np.ndarray:
    """H_rho = (diag(P_rho^T a) - P_rho^T diag(a) P_rho) / eta  (Alg. 1 output)."""
    return (np.diag(P_rho.T @ a) - P_rho.T @ (a[:, None] * P_rho)) / eta


def sparsification_threshold(eta, m, n, gnorm) -> float:
    """rho = eta ||g|| / (m n)  (Alg. 2, Newton step 1)."""
    return eta * gnorm / (m * n)


# ----------------------------------------------------------------------------
# Newton direction (Alg. 2): (H_rho + ||g|| I) Delta = -g by preconditioned CG
# ----------------------------------------------------------------------------

def pcg(A: np.ndarray, rhs: np.ndarray, diag: np.ndarray, rtol: float, maxit: int):
    """Textbook Jacobi-preconditioned conjugate gradients from x0 = 0.

    Stops when ||r|| <= rtol * ||rhs|| or after maxit iterations.
    Returns (x, iterations, final residual norm).
    """
    x = np.zeros_like(rhs)
    r = rhs.copy()
    bnorm = np.linalg.norm(rhs)
    if bnorm == 0.0:
        return x, 0, 0.0
    z = r / diag
    p = z.copy()
    rz = r @ z
    it = 0
    rnorm = bnorm
    while it < maxit and rnorm > rtol * bnorm:
        q = A @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rnorm = np.linalg.norm(r)
        z = r / diag
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, float(rnorm)


def cg_tolerance(gnorm: float, cg_rtol: float, mu: float | None) -> float:
    """Relative CG tolerance of reading R3."""
    if mu is None or gnorm == 0.0:
        return min(cg_rtol, gnorm)
    return min(cg_rtol, max(gnorm, 0.25 * mu / gnorm))


def newton_direction(H_rho, g, cg_rtol: float, max_cg: int, mu: float | None = None):
    """Delta = -(H_rho + ||g|| I)^{-1} g (Alg. 2), by Jacobi PCG, then centred (R3).

    Returns (Delta, cg_iterations).
    """
    gnorm = float(np.linalg.norm(g))
    A = H_rho + gnorm * np.eye(len(g))
    rtol = cg_tolerance(gnorm, cg_rtol, mu)
    delta, it, _ = pcg(A, -g, np.diag(A).copy(), rtol, max_cg)
    delta = delta - delta.mean()
    return delta, it


# ----------------------------------------------------------------------------
# Armijo backtracking (Alg. 2) on L^k evaluated directly
# ----------------------------------------------------------------------------

def armijo(logX, C, a, b, eta, gamma, delta, g, sigma, beta, max_trials):
    """Largest t in {1, beta, beta^2, ...} with L(gamma + t Delta) <= L(gamma) + sigma t g^T Delta.

    Returns (t, trials, accepted).  If no trial is accepted within max_trials,
    returns the last t tried and accepted=False (reading R4).
    """
    L0 = semi_dual_objective(logX, C, a, b, eta, gamma)
    slope = float(g @ delta)
    t = 1.0
    for trial in range(1, max_trials + 1):
        Lt = semi_dual_objective(logX, C, a, b, eta, gamma + t * delta)
        if Lt <= L0 + sigma * t * slope:
            return t, trial, True
        t *= beta
    return t / beta, max_trials, False


# ----------------------------------------------------------------------------
# Sinkhorn warm-up (Alg. 2 line "Solve ... using Sinkhorn"), semi-dual form
# ----------------------------------------------------------------------------

def sinkhorn_warmup(logX, C, a, b, eta, gamma, tol, max_iter):
    """Alternating minimisation of the two-dual Z^k (Eq. 3).

    The zeta-step is Eq. 4 (zeta = zeta(gamma)); the gamma-step sets
    dZ/dgamma = 0, i.e. gamma_j <- eta log b_j - eta log sum_i X^k_ij exp((zeta_i - C_ij)/eta).
    Stops once ||g^k(gamma)|| < tol (Sec. 5 setup).  Returns (gamma, iterations, ||g||).
    """
    gamma = gamma.copy()
    it = 0
    while True:
        zeta = best_zeta(logX, C, a, eta, gamma)
        P = np.exp(_exponent(logX, C, eta, gamma) + zeta[:, None] / eta)
        g = P.sum(axis=0) - b
        gnorm = float(np.linalg.norm(g))
        if gnorm < tol or it >= max_iter:
            return gamma, it, gnorm
        # gamma-step of Z^k with zeta fixed
        F = logX + (zeta[:, None] - C) / eta
        colmax = F.max(axis=0)
        lse_col = colmax + np.log(np.exp(F - colmax[None, :]).sum(axis=0))
        gamma = eta * np.log(b) - eta * lse_col
        it += 1


# ----------------------------------------------------------------------------
# Alg. 3 rounding, Bregman divergence, c-transform, certificate, Delta_kkt
# ----------------------------------------------------------------------------

def round_to_feasible(X, a, b):
    """Alg. 3 (rounding of Altschuler et al. as printed in App. A).

    Returns (Xhat, z, y, e_r, e_c).
    """
    z = np.minimum(a / X.sum(axis=1), 1.0)
    F = z[:, None] * X
    y = np.minimum(b / X.sum(axis=0), 1.0)
    F = F * y[None, :]
    e_r = a - F.sum(axis=1)
    e_c = b - F.sum(axis=0)
    s = np.abs(e_r).sum()
    Xhat = F + (np.outer(e_r, e_c) / s if s > 0 else 0.0)
    return Xhat, z, y, e_r, e_c


def bregman_divergence_log(Xhat, logX) -> float:
    """D_phi(Xhat, X) = sum Xhat log(Xhat/X) - sum Xhat + sum X (Sec. 3.1), X given by log X (R7)."""
    X = np.exp(logX)
    pos = Xhat > 0
    term = np.zeros_like(Xhat)
    term[pos] = Xhat[pos] * (np.log(Xhat[pos]) - logX[pos])
    return float(term.sum() - Xhat.sum() + X.sum())


def c_transform(C, gamma) -> np.ndarray:
    """zeta_i = min_j (C_ij - gamma_j)  (App. C.1)."""
    return (C - gamma[None, :]).min(axis=1)


def dual_objective(a, b, zeta, gamma) -> float:
    """a^T zeta + b^T gamma (dual of Eq. 1, App. C.1)."""
    return float(a @ zeta + b @ gamma)


def relative_gap(p: float, d: float) -> float:
    """(p - d) / max(|p|, |d|) (reading R11)."""
    den = max(abs(p), abs(d))
    return (p - d) / den if den > 0 else abs(p - d)


def kkt_residual(X, C, a, b, gamma, zeta) -> float:
    """Delta_kkt = max(Delta_p, Delta_d, Delta_c) of App. C.1."""
    U = C - zeta[:, None] - gamma[None, :]
    dp = max(np.linalg.norm(X.sum(axis=1) - a) / (1 + np.linalg.norm(a)),
             np.linalg.norm(X.sum(axis=0) - b) / (1 + np.linalg.norm(b)),
             np.linalg.norm(np.minimum(X, 0.0)) / (1 + np.linalg.norm(X)))
    cf = 1 + np.linalg.norm(C)
    dd = np.linalg.norm(np.minimum(U, 0.0)) / cf
    dc = abs(float((X * U).sum())) / cf
    return float(max(dp, dd, dc))


def certify(logX_next, C, a, b, gamma):
    """Primal of the rounded plan, c-transform dual and relative gap at X^{k+1} = diag(a)P."""
    X = np.exp(logX_next)
    Xhat = round_to_feasible(X, a, b)[0]
    p = float((C * Xhat).sum())
    zeta = c_transform(C, gamma)
    d = dual_objective(a, b, zeta, gamma)
    return p, d, relative_gap(p, d), Xhat, zeta


# ----------------------------------------------------------------------------
# Alg. 2: IBSN
# ----------------------------------------------------------------------------

@dataclass
class IBSNParams:
    eta: float
    sigma: float = 1e-4          # Armijo parameter (Alg. 2 input)
    beta: float = 0.8            # backtracking factor (Alg. 2 input)
    sinkhorn_tol: float = 1e-3   # warm-up stop (Sec. 5 setup)
    mu0: float = 1e-4            # mu_k = max(mu0/(k+1)^2, mu_min)  (Eq. 8)
    mu_min: float = 1e-11
    gap_tol: float = 1e-8        # outer stop on the relative duality gap (R11)
    max_outer: int = 5000
    max_newton: int = 50
    max_cg: int = 1000
    max_sinkhorn: int = 10000
    max_armijo: int = 60
    cg_rtol: float = 0.1
    sparsify: bool = True        # False gives IBN (App. C.3 ablation)
    # CG forcing term (the paper is silent, reading R3): "gate" relaxes
    # min(cg_rtol, ||g||) to the accuracy at which the linear model reaches the
    # gate mu_k; "plain" is min(cg_rtol, ||g||) alone
    cg_forcing: str = "gate"


@dataclass
class IBSNResult:
    gamma: np.ndarray
    logX: np.ndarray
    plan: np.ndarray
    zeta: np.ndarray
    primal: float
    dual: float
    rel_gap: float
    kkt: float
    outer_iters: int
    newton_iters: int
    cg_iters: int
    sinkhorn_iters: int
    converged: bool
    history: list = field(default_factory=list)


def mu_k(k: int, params: IBSNParams) -> float:
    """Inexactness tolerance mu_k = max(mu0/(k+1)^2, mu_min)  (Eq. 8)."""
    return max(params.mu0 / (k + 1) ** 2, params.mu_min)


def ibsn(C, a, b, params: IBSNParams, gamma0=None, record=False) -> IBSNResult:
    """Algorithm 2 (IBSN), literally: explicit log X^k, dense H_rho, direct L^k."""
    C = np.asarray(C, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m, n = C.shape
    eta = params.eta
    logX = initial_log_plan(a, b)
    gamma = np.zeros(n) if gamma0 is None else np.asarray(gamma0, dtype=np.float64).copy()
    tot_newton = tot_cg = tot_sk = 0
    hist = []
    p = d = gap = np.inf
    Xhat = zeta = None
    converged = False
    k = 0
    for k in range(params.max_outer):
        mu = mu_k(k, params)
        gamma, sk_it, _ = sinkhorn_warmup(logX, C, a, b, eta, gamma, params.sinkhorn_tol, params.max_sinkhorn)
        tot_sk += sk_it
        gamma = gamma - gamma.mean()
        inner = []
        for v in range(params.max_newton):
            P = plan(logX, C, eta, gamma)
            g = gradient(P, a, b)
            gnorm = float(np.linalg.norm(g))
            if params.sparsify:
                rho = sparsification_threshold(eta, m, n, gnorm)
                H = sparsified_hessian(sparsify_plan(P, a, rho), a, eta)
            else:
                H = hessian(P, a, eta)
            delta, cg_it = newton_direction(H, g, params.cg_rtol, params.max_cg,
                                            mu if params.cg_forcing == "gate" else None)
            tot_cg += cg_it
            t, _, _ = armijo(logX, C, a, b, eta, gamma, delta, g, params.sigma, params.beta, params.max_armijo)
            if record:
                inner.append(dict(L=semi_dual_objective(logX, C, a, b, eta, gamma), gnorm=gnorm, t=t,
                                  slope=float(g @ delta), mean_gamma=float(gamma.mean()), cg=cg_it))
            gamma = gamma + t * delta
            tot_newton += 1
            lp_next = log_plan(logX, C, eta, gamma)
            P = np.exp(lp_next)
            gnorm = float(np.linalg.norm(gradient(P, a, b)))
            if gnorm < mu:
                logX_next = np.log(a)[:, None] + lp_next
                Xhat = round_to_feasible(np.exp(logX_next), a, b)[0]
                if bregman_divergence_log(Xhat, logX_next) <= min(m, n) * mu:
                    break
        # outer update X^{k+1} = diag(a) P^k(gamma^{k,v+1}); gamma^{k+1,0} = gamma^{k,v+1}
        logX_prev = logX
        logX = np.log(a)[:, None] + log_plan(logX, C, eta, gamma)
        p, d, gap, Xhat, zeta = certify(logX, C, a, b, gamma)
        if record:
            inner.append(dict(L=semi_dual_objective(logX_prev, C, a, b, eta, gamma), gnorm=gnorm))
            hist.append(dict(k=k, sinkhorn=sk_it, newton=v + 1, gnorm=gnorm, primal=p, dual=d, gap=gap,
                             inner=inner))
        if gap <= params.gap_tol:
            converged = True
            break
    X = np.exp(logX)
    return IBSNResult(gamma=gamma, logX=logX, plan=Xhat, zeta=zeta, primal=p, dual=d, rel_gap=gap,
                      kkt=kkt_residual(X, C, a, b, gamma, zeta), outer_iters=k + 1,
                      newton_iters=tot_newton, cg_iters=tot_cg, sinkhorn_iters=tot_sk,
                      converged=converged, history=hist)


# ----------------------------------------------------------------------------
# (E)IBSN (App. C.4): the inner solve alone on one entropic subproblem
# ----------------------------------------------------------------------------

@dataclass
class EIBSNResult:
    gamma: np.ndarray
    plan: np.ndarray
    gnorm: float
    newton_iters: int
    cg_per_direction: list
    sinkhorn_iters: int
    converged: bool


def eibsn(C, a, b, params: IBSNParams, gtol: float = 1e-9, gamma0=None) -> EIBSNResult:
    """(E)IBSN of App. C.4: Alg. 2's inner loop on the single subproblem with
    X^k fixed at 1 1^T (the entropic OT problem with cost C), no outer update.

    Sinkhorn warm-up to ||g|| < sinkhorn_tol, centring, then Newton steps
    (Alg. 1 sparsification, shifted Newton system by PCG, Armijo) until
    ||g|| < gtol or max_newton steps.  The CG tolerance is reading R3 with the
    gate gtol in place of mu_k.
    """
    C = np.asarray(C, dtype=np.float64)
    m, n = C.shape
    eta = params.eta
    logX = np.zeros((m, n))  # X = 1 1^T
    gamma = np.zeros(n) if gamma0 is None else np.asarray(gamma0, dtype=np.float64).copy()
    gamma, sk_it, _ = sinkhorn_warmup(logX, C, a, b, eta, gamma, params.sinkhorn_tol, params.max_sinkhorn)
    gamma = gamma - gamma.mean()
    cgs = []
    converged = False
    v = 0
    for v in range(params.max_newton + 1):
        P = plan(logX, C, eta, gamma)
        g = gradient(P, a, b)
        gnorm = float(np.linalg.norm(g))
        if gnorm < gtol:
            converged = True
            break
        if v == params.max_newton:
            break
        if params.sparsify:
            rho = sparsification_threshold(eta, m, n, gnorm)
            H = sparsified_hessian(sparsify_plan(P, a, rho), a, eta)
        else:
            H = hessian(P, a, eta)
        delta, cg_it = newton_direction(H, g, params.cg_rtol, params.max_cg, gtol)
        cgs.append(cg_it)
        t, _, _ = armijo(logX, C, a, b, eta, gamma, delta, g, params.sigma, params.beta, params.max_armijo)
        gamma = gamma + t * delta
    return EIBSNResult(gamma=gamma, plan=P, gnorm=gnorm, newton_iters=len(cgs), cg_per_direction=cgs,
                       sinkhorn_iters=sk_it, converged=converged)

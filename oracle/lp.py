"""Exact LP references that pin the IBSN oracle -- TEST INFRASTRUCTURE ONLY.

They solve the OT linear program of Eq. 1 (min <C,X>, X1=a, X^T1=b, X>=0)
by methods that share nothing with IBSN:

  permutation_optimum  -- uniform marginals a = b = 1/n: by Birkhoff's theorem
                          an optimal vertex is a permutation matrix / n, so the
                          optimum is the best of all n! assignments (n <= 8).
  network_simplex      -- the transportation simplex (u-v / MODI method) with a
                          north-west-corner start, written from the textbook
                          description; returns the plan and dual potentials.
  monotone_1d_optimum  -- 1-D supports with a convex cost of (x - y): the
                          monotone (north-west corner on sorted supports)
                          coupling is optimal.
  separable_optimum    -- C = u 1^T + 1 v^T: every feasible plan costs a^T u + b^T v.

Parity status: each is checked against the others and against scipy's HiGHS
LP solver in tests/test_oracle_lp.py.
"""

from __future__ import annotations

import itertools
from collections import deque

import numpy as np


def permutation_optimum(C: np.ndarray) -> float:
    """min over permutations s of (1/n) sum_i C[i, s(i)]  (uniform marginals, n <= 8)."""
    n = C.shape[0]
    assert C.shape == (n, n) and n <= 8
    best = np.inf
    rows = np.arange(n)
    for perm in itertools.permutations(range(n)):
        best = min(best, float(C[rows, list(perm)].sum()))
    return best / n


def monotone_1d_optimum(x: np.ndarray, y: np.ndarray, a: np.ndarray, b: np.ndarray, cost) -> float:
    """Optimal value for 1-D supports x (m), y (n) and a convex cost(x_i - y_j):
    transport greedily along the two sorted supports (north-west corner rule)."""
    ix = np.argsort(x, kind="stable")
    iy = np.argsort(y, kind="stable")
    ra = a[ix].astype(np.float64).copy()
    rb = b[iy].astype(np.float64).copy()
    i = j = 0
    total = 0.0
    while i < len(ra) and j < len(rb):
        f = min(ra[i], rb[j])
        total += f * cost(x[ix[i]] - y[iy[j]])
        ra[i] -= f
        rb[j] -= f
        if ra[i] <= rb[j]:
            i += 1
        else:
            j += 1
    return total


def separable_optimum(u: np.ndarray, v: np.ndarray, a: np.ndarray, b: np.ndarray) -> float:
    """Every X in Omega has <u 1^T + 1 v^T, X> = a^T u + b^T v."""
    return float(a @ u + b @ v)


def _northwest_corner(a, b):
    m, n = len(a), len(b)
    ra, rb = a.astype(np.float64).copy(), b.astype(np.float64).copy()
    basis = []
    flow = {}
    i = j = 0
    while i < m and j < n:
        f = min(ra[i], rb[j])
        basis.append((i, j))
        flow[(i, j)] = f
        ra[i] -= f
        rb[j] -= f
        if i == m - 1 and j == n - 1:
            break
        # move right when the row is exhausted last, keeping m + n - 1 basic cells
        if (ra[i] <= rb[j] and i < m - 1) or j == n - 1:
            i += 1
        else:
            j += 1
    return basis, flow


def _potentials(C, basis, m, n):
    """Solve u_i + v_j = C_ij on the basis tree (u_0 = 0)."""
    adj_r = [[] for _ in range(m)]
    adj_c = [[] for _ in range(n)]
    for (i, j) in basis:
        adj_r[i].append(j)
        adj_c[j].append(i)
    u = np.full(m, np.nan)
    v = np.full(n, np.nan)
    u[0] = 0.0
    q = deque([("r", 0)])
    while q:
        kind, k = q.popleft()
        if kind == "r":
            for j in adj_r[k]:
                if np.isnan(v[j]):
                    v[j] = C[k, j] - u[k]
                    q.append(("c", j))
        else:
            for i in adj_c[k]:
                if np.isnan(u[i]):
                    u[i] = C[i, k] - v[k]
                    q.append(("r", i))
    return u, v


def _cycle(basis, m, n, enter):
    """Path in the basis tree from column j back to row i, closed by the entering cell (i, j)."""
    i0, j0 = enter
    adj = {("r", i): [] for i in range(m)}
    adj.update({("c", j): [] for j in range(n)})
    for (i, j) in basis:
        adj[("r", i)].append(("c", j))
        adj[("c", j)].append(("r", i))
    start, goal = ("c", j0), ("r", i0)
    prev = {start: None}
    q = deque([start])
    while q:
        node = q.popleft()
        if node == goal:
            break
        for nb in adj[node]:
            if nb not in prev:
                prev[nb] = node
                q.append(nb)
    path = []
    node = goal
    while node is not None:
        path.append(node)
        node = prev[node]
    # path: row i0 -> ... -> col j0 ; cells alternate along it
    cells = [enter]
    for s in range(len(path) - 1):
        x, y = path[s], path[s + 1]
        cell = (x[1], y[1]) if x[0] == "r" else (y[1], x[1])
        cells.append(cell)
    return cells  # cells[0] gains, cells[1] loses, cells[2] gains, ...


def network_simplex(C: np.ndarray, a: np.ndarray, b: np.ndarray, max_iter: int = 100000, tol: float = 1e-13):
    """Transportation simplex.  Returns (value, X, u, v) with u_i + v_j <= C_ij
    (dual feasible) and equality on the basis."""
    C = np.asarray(C, dtype=np.float64)
    m, n = C.shape
    basis, flow = _northwest_corner(np.asarray(a, np.float64), np.asarray(b, np.float64))
    for it in range(max_iter):
        u, v = _potentials(C, basis, m, n)
        red = C - u[:, None] - v[None, :]
        bset = set(basis)
        # Dantzig's rule, Bland's rule (first negative) after many iterations
        if it < 20 * (m + n) ** 2:
            i, j = np.unravel_index(np.argmin(red), red.shape)
            if red[i, j] >= -tol:
                break
        else:
            neg = np.argwhere(red < -tol)
            neg = [tuple(c) for c in neg if tuple(c) not in bset]
            if not neg:
                break
            i, j = neg[0]
        cells = _cycle(basis, m, n, (int(i), int(j)))
        minus = cells[1::2]
        theta = min(flow[c] for c in minus)
        leave = min((c for c in minus if flow[c] == theta), key=lambda c: (c[0], c[1]))
        flow[(int(i), int(j))] = 0.0
        for s, c in enumerate(cells):
            flow[c] += theta if s % 2 == 0 else -theta
        basis.remove(leave)
        del flow[leave]
        basis.append((int(i), int(j)))
    X = np.zeros((m, n))
    for (i, j), f in flow.items():
        X[i, j] = f
    u, v = _potentials(C, basis, m, n)
    return float((C * X).sum()), X, u, v

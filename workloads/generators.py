"""Synthetic workloads shaped like the paper's experiments (Sec. 5, App. C).

Every generator uses numpy's PCG64 ``default_rng(seed)`` and a fixed draw
order, stated per function, so that a seed fully determines the bytes.

Workload recipes (the five standard configurations):

* ``c0``  m=n=256, points i.i.d. U[0,1]^2, squared Euclidean cost / max,
          a, b ~ U(0.1, 1) normalised, seed 0, eta = 1e-4 (Sec. 5 synthetic eta).
* ``c1``  m=n=4096, two different 8-component Gaussian mixtures in R^10
          (means U[-3,3]^10, unit isotropic covariance, equal weights),
          squared Euclidean / max, U(0.1,1) marginals, seed 1, eta = 1e-4.
* ``c2``  m=n=16384, 128x128 grid histograms: C = squared grid distance / max,
          a, b = Gaussian blur (sigma 4 px) of i.i.d. U(0,1) noise + 1e-6,
          normalised, seed 2, eta = 1e-3 (Sec. 5.2 image eta).  Stands in for
          the DOTmark / MNIST image pairs, which are not used here.
* ``c3``  64 problems, seeds 100..163, m, n ~ U{500..5000} independently,
          2-D uniform points, squared Euclidean / max, eta = 1e-4.
* ``c4``  2-D 4-component Gaussian mixtures with random weights (warm start):
          ``warmstart_gmm_problem``; network initial weights from
          ``warmstart_init_params``.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class OTProblem:
    """One discrete OT instance min <C,X> s.t. X1=a, X^T1=b, X>=0 (Eq. 1)."""

    C: np.ndarray  # (m, n) float64 or float32; the problem is exactly these values
    a: np.ndarray  # (m,) float64, positive, sums to 1
    b: np.ndarray  # (n,) float64, positive, sums to 1
    eta: float
    name: str = ""
    # optional geometry that produced C (for the on-the-fly cost kinds)
    x: np.ndarray | None = None  # (m, d) source points
    y: np.ndarray | None = None  # (n, d) target points
    grid: tuple[int, int] | None = None  # (h, w) for grid problems
    cost_scale: float = 1.0  # C = cost_scale * raw geometric cost
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.C.shape[0])

    @property
    def n(self) -> int:
        return int(self.C.shape[1])


def random_marginal(rng: np.random.Generator, size: int, low: float = 0.1, high: float = 1.0) -> np.ndarray:
    """U(low, high) weights normalised to sum 1 (Sec. 5.1 marginals)."""
    w = rng.uniform(low, high, size=size)
    return w / w.sum()


def sq_euclidean_cost(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Raw squared Euclidean distances ||x_i - y_j||^2 in float64 (exact loop-free form)."""
    diff = x[:, None, :] - y[None, :, :]
    return np.einsum("ijk,ijk->ij", diff, diff)


def grid_sq_cost(h: int, w: int) -> np.ndarray:
    """Integer squared grid distances between the h*w bins of one grid (row-major bins)."""
    idx = np.arange(h * w)
    r = idx // w
    c = idx % w
    dr = r[:, None] - r[None, :]
    dc = c[:, None] - c[None, :]
    return (dr * dr + dc * dc).astype(np.float64)


def square_index_cost(m: int, n: int) -> np.ndarray:
    """The paper's 'Square' synthetic cost C_ij = (i - j)^2 (Sec. 5.1)."""
    i = np.arange(m)[:, None].astype(np.float64)
    j = np.arange(n)[None, :].astype(np.float64)
    return (i - j) ** 2


def paper_synthetic_problem(kind: str, m: int, n: int, seed: int, eta: float = 1e-4,
                            cost_dtype=np.float64) -> OTProblem:
    """The paper's synthetic settings (Sec. 5.1): a, b ~ U(0, 1) normalised and
    C / max with C_ij ~ U(0, 1) ('uniform') or C_ij = (i - j)^2 ('square').

    Draw order: a (m), b (n), then the uniform cost (m*n) for 'uniform'.
    """
    rng = np.random.default_rng(seed)
    a = random_marginal(rng, m, 0.0, 1.0)
    b = random_marginal(rng, n, 0.0, 1.0)
    if kind == "uniform":
        raw = rng.uniform(0.0, 1.0, size=(m, n))
    elif kind == "square":
        raw = square_index_cost(m, n)
    else:
        raise KeyError(kind)
    C, scale = _normalised_by_max(raw)
    return OTProblem(C=C.astype(cost_dtype), a=a, b=b, eta=eta, name=f"{kind}_{m}x{n}_s{seed}", cost_scale=scale)


def _unit_rows(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def sphere_problem(m: int, n: int, seed: int, eta: float = 1e-3, clusters: int = 24,
                   cost_dtype=np.float64) -> OTProblem:
    """Unbalanced spherical transport (the App. C.4 m > n setting, synthetic):
    demand points x_i on the unit sphere S^2 drawn from `clusters` clustered
    populations (cluster centres uniform on S^2, Dirichlet(1) cluster weights,
    angular spread U[0.02, 0.3] rad, Gaussian in the tangent plane), supply
    points y_j uniform on S^2, C_ij = arccos(<x_i, y_j>) / max, a, b ~ U(0, 1)
    normalised.  Stands in for the population-density and landmass data,
    which are not used.

    Draw order: centres (clusters x 3), weights, spreads, labels (m), tangent
    noise (m x 3), supply directions (n x 3), a (m), b (n).
    """
    rng = np.random.default_rng(seed)
    centres = _unit_rows(rng.standard_normal(size=(clusters, 3)))
    wts = rng.dirichlet(np.ones(clusters))
    spread = rng.uniform(0.02, 0.3, size=clusters)
    labels = rng.choice(clusters, size=m, p=wts)
    noise = rng.standard_normal(size=(m, 3)) * spread[labels][:, None]
    c = centres[labels]
    noise -= (noise * c).sum(axis=1, keepdims=True) * c  # tangent component only
    x = _unit_rows(c + noise)
    y = _unit_rows(rng.standard_normal(size=(n, 3)))
    a = random_marginal(rng, m, 0.0, 1.0)
    b = random_marginal(rng, n, 0.0, 1.0)
    raw = np.arccos(np.clip(x @ y.T, -1.0, 1.0))
    C, scale = _normalised_by_max(raw)
    return OTProblem(C=C.astype(cost_dtype), a=a, b=b, eta=eta, name=f"sphere_{m}x{n}_s{seed}", x=x, y=y,
                     cost_scale=scale)


def _normalised_by_max(raw: np.ndarray) -> tuple[np.ndarray, float]:
    mx = float(raw.max())
    scale = 1.0 / mx if mx > 0 else 1.0
    return raw * scale, scale


def uniform_points_problem(m: int, n: int, seed: int, d: int = 2, eta: float = 1e-4,
                           cost_dtype=np.float64) -> OTProblem:
    """Points i.i.d. U[0,1]^d; C = squared Euclidean / max; U(0.1,1) marginals.

    Draw order: x (m*d), y (n*d), a (m), b (n).
    """
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, size=(m, d))
    y = rng.uniform(0.0, 1.0, size=(n, d))
    a = random_marginal(rng, m)
    b = random_marginal(rng, n)
    C, scale = _normalised_by_max(sq_euclidean_cost(x, y))
    return OTProblem(C=C.astype(cost_dtype), a=a, b=b, eta=eta, name=f"uniform{d}d_{m}x{n}_s{seed}",
                     x=x, y=y, cost_scale=scale)


def _gmm_sample(rng: np.random.Generator, count: int, means: np.ndarray, weights: np.ndarray,
                std: np.ndarray) -> np.ndarray:
    labels = rng.choice(len(weights), size=count, p=weights)
    noise = rng.standard_normal(size=(count, means.shape[1]))
    return means[labels] + noise * std[labels][:, None]


def gmm_points_problem(m: int, n: int, seed: int, d: int = 10, k: int = 8, eta: float = 1e-4,
                       cost_dtype=np.float64) -> OTProblem:
    """Two different k-component Gaussian mixtures in R^d (means U[-3,3]^d, unit cov, equal weights).

    Draw order: source means (k*d), target means (k*d), source labels + noise,
    target labels + noise, a (m), b (n).
    """
    rng = np.random.default_rng(seed)
    mu_s = rng.uniform(-3.0, 3.0, size=(k, d))
    mu_t = rng.uniform(-3.0, 3.0, size=(k, d))
    wts = np.full(k, 1.0 / k)
    std = np.ones(k)
    x = _gmm_sample(rng, m, mu_s, wts, std)
    y = _gmm_sample(rng, n, mu_t, wts, std)
    a = random_marginal(rng, m)
    b = random_marginal(rng, n)
    C, scale = _normalised_by_max(sq_euclidean_cost(x, y))
    return OTProblem(C=C.astype(cost_dtype), a=a, b=b, eta=eta, name=f"gmm{d}d_{m}x{n}_s{seed}",
                     x=x, y=y, cost_scale=scale)


def _gaussian_blur(img: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian blur, radius 4*sigma, reflected boundary, normalised taps."""
    radius = int(np.ceil(4.0 * sigma))
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    taps = np.exp(-0.5 * (t / sigma) ** 2)
    taps /= taps.sum()
    out = img
    for axis in (0, 1):
        padded = np.pad(out, [(radius, radius) if ax == axis else (0, 0) for ax in range(2)],
                        mode="symmetric")
        acc = np.zeros_like(out)
        for s, wgt in enumerate(taps):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(s, s + out.shape[axis])
            acc += wgt * padded[tuple(sl)]
        out = acc
    return out


def grid_marginals(h: int, w: int, seed: int, sigma: float = 4.0):
    """The marginals and cost scale of grid_problem without the (h w)^2 cost
    matrix: (a, b, scale).  Draw order: source noise (h*w), target noise (h*w).
    Marginals are blur(noise) + 1e-6, normalised; scale = 1 / ((h-1)^2 + (w-1)^2)."""
    rng = np.random.default_rng(seed)
    src = _gaussian_blur(rng.uniform(0.0, 1.0, size=(h, w)), sigma) + 1e-6
    dst = _gaussian_blur(rng.uniform(0.0, 1.0, size=(h, w)), sigma) + 1e-6
    a = (src / src.sum()).ravel()
    b = (dst / dst.sum()).ravel()
    mx = float((h - 1) ** 2 + (w - 1) ** 2)
    scale = 1.0 / mx if mx > 0 else 1.0
    return a, b, scale


def grid_problem(h: int, w: int, seed: int, sigma: float = 4.0, eta: float = 1e-3,
                 cost_dtype=np.float64) -> OTProblem:
    """Smoothed random fields on an h x w grid; C = squared grid distance / max
    (marginals and scale from grid_marginals)."""
    a, b, scale = grid_marginals(h, w, seed, sigma)
    C = grid_sq_cost(h, w) * scale
    return OTProblem(C=C.astype(cost_dtype), a=a, b=b, eta=eta, name=f"grid{h}x{w}_s{seed}",
                     grid=(h, w), cost_scale=scale)


def batched_problems(count: int = 64, seed0: int = 100, lo: int = 500, hi: int = 5000,
                     eta: float = 1e-4, cost_dtype=np.float64, scale_sizes: float = 1.0) -> list[OTProblem]:
    """Independent rectangular problems, seeds seed0..seed0+count-1.

    Per seed, draw order: m, n ~ U{lo..hi} (integers), then the uniform-points
    recipe with that seed's generator continuing.  ``scale_sizes`` < 1 shrinks
    m, n for quick tests while keeping the same draws.
    """
    out = []
    for s in range(seed0, seed0 + count):
        rng = np.random.default_rng(s)
        m = int(rng.integers(lo, hi + 1))
        n = int(rng.integers(lo, hi + 1))
        m = max(1, int(round(m * scale_sizes)))
        n = max(1, int(round(n * scale_sizes)))
        x = rng.uniform(0.0, 1.0, size=(m, 2))
        y = rng.uniform(0.0, 1.0, size=(n, 2))
        a = random_marginal(rng, m)
        b = random_marginal(rng, n)
        C, scale = _normalised_by_max(sq_euclidean_cost(x, y))
        out.append(OTProblem(C=C.astype(cost_dtype), a=a, b=b, eta=eta, name=f"batch_s{s}_{m}x{n}",
                             x=x, y=y, cost_scale=scale))
    return out


def batched_points(count: int = 64, seed0: int = 100, lo: int = 500, hi: int = 5000, eta: float = 1e-4):
    """The draws of batched_problems without the cost matrices: per problem
    (m, n, x, y, a, b, eta); the squared Euclidean cost divided by its max is
    formed by the caller (on the device for the full-size batch)."""
    out = []
    for s in range(seed0, seed0 + count):
        rng = np.random.default_rng(s)
        m = int(rng.integers(lo, hi + 1))
        n = int(rng.integers(lo, hi + 1))
        x = rng.uniform(0.0, 1.0, size=(m, 2))
        y = rng.uniform(0.0, 1.0, size=(n, 2))
        a = random_marginal(rng, m)
        b = random_marginal(rng, n)
        out.append((m, n, x, y, a, b, eta))
    return out


def warmstart_gmm_problem(n: int, seed: int, k: int = 4, eta: float = 1e-4,
                          cost_dtype=np.float64) -> OTProblem:
    """2-D k-component Gaussian mixtures with Dirichlet(1) weights, means U[0,1]^2,
    isotropic std U[0.03, 0.15]; source and target independent; m = n.

    Draw order: source (weights, means, stds, labels + noise), target (same),
    a (n), b (n).
    """
    rng = np.random.default_rng(seed)

    def cloud():
        wts = rng.dirichlet(np.ones(k))
        means = rng.uniform(0.0, 1.0, size=(k, 2))
        std = rng.uniform(0.03, 0.15, size=k)
        return _gmm_sample(rng, n, means, wts, std)

    x = cloud()
    y = cloud()
    a = random_marginal(rng, n)
    b = random_marginal(rng, n)
    C, scale = _normalised_by_max(sq_euclidean_cost(x, y))
    return OTProblem(C=C.astype(cost_dtype), a=a, b=b, eta=eta, name=f"ws_gmm_{n}_s{seed}",
                     x=x, y=y, cost_scale=scale)


# Shapes of the warm-start network's parameters, in the order of its flat
# float32 vector (W_s, b_s, W_t, b_t, W_h, b_h, w_o, b_o; row-major).
WARMSTART_SHAPES = [(128, 3), (128,), (128, 3), (128,), (128, 384), (128,), (128,), (1,)]


def warmstart_init_params(seed: int) -> np.ndarray:
    """Initial float32 parameters of the warm-start network: weights drawn
    U(-sqrt(6/fan_in), +sqrt(6/fan_in)) (fan_in = the row length; 128 for
    w_o), biases 0.  Draw order: the weight tensors in layout order."""
    rng = np.random.default_rng(seed)
    parts = []
    for k, shape in enumerate(WARMSTART_SHAPES):
        if k in (1, 3, 5, 7):
            parts.append(np.zeros(shape))
        else:
            fan_in = shape[-1]
            lim = np.sqrt(6.0 / fan_in)
            parts.append(rng.uniform(-lim, lim, size=shape))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def workload(name: str, cost_dtype=np.float64) -> OTProblem:
    """The named standard workloads (see module docstring)."""
    if name == "c0":
        return uniform_points_problem(256, 256, seed=0, d=2, eta=1e-4, cost_dtype=cost_dtype)
    if name == "c1":
        return gmm_points_problem(4096, 4096, seed=1, d=10, k=8, eta=1e-4, cost_dtype=cost_dtype)
    if name == "c2":
        return grid_problem(128, 128, seed=2, sigma=4.0, eta=1e-3, cost_dtype=cost_dtype)
    raise KeyError(name)

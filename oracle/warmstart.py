"""Float64 oracle of the learned warm start -- TEST INFRASTRUCTURE ONLY.

The paper starts every solve from gamma^{0,0} = 0 (Alg. 2).  The learned warm
start replaces that start by a prediction gamma_hat of the optimal dual
potential (cost units, centred) made by a small network from the two point
clouds and their marginals; the plain start stays as the fallback, and the
start with the smaller semi-dual objective L^0 (Eq. 5 at k = 0) is kept.

Network (three layers of width 128; weights are bfloat16 values):
  source point i:  f_i = [x_i1, x_i2, m a_i],  e_i = relu(W_s f_i + b_s)
  target point j:  g_j = [y_j1, y_j2, n b_j],  h_j = relu(W_t g_j + b_t)
  pools:           p_s = mean_i e_i,  p_t = mean_j h_j
  head:            z_j = W_h [h_j; p_s; p_t] + b_h,  u_j = relu(z_j)
                   o_j = w_o . u_j + b_o,  gamma_hat_j = o_j - mean_l o_l
Loss of a batch of Q problems:
  (1/Q) sum_q (1/n_q) sum_j (gamma_hat_qj - (gamma*_qj - mean gamma*_q))^2.
Flat parameter layout (float32 master copy, in this order, row-major):
  W_s 128x3, b_s 128, W_t 128x3, b_t 128, W_h 128x384, b_h 128, w_o 128, b_o 1.

Everything here is float64 arithmetic on the bfloat16-rounded weights.  The
relu derivative at 0 is taken as 0.  Adam follows Kingma & Ba (2015),
Algorithm 1, with bias-corrected moments.

Pins (tests/test_oracle_warmstart.py): bfloat16 rounding against a
nearest-neighbour search on the bfloat16 grid; the analytic gradient against
central finite differences of the loss; invariance of gamma_hat to a
permutation of the source points and equivariance under a permutation of the
target points; centring; the closed forms of Adam's first step and of its
steps under a constant gradient.
"""

from __future__ import annotations

import numpy as np

H = 128
SHAPES = [("W_s", (H, 3)), ("b_s", (H,)), ("W_t", (H, 3)), ("b_t", (H,)),
          ("W_h", (H, 3 * H)), ("b_h", (H,)), ("w_o", (H,)), ("b_o", (1,))]
PARAM_COUNT = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(theta: np.ndarray) -> dict[str, np.ndarray]:
    """Views of the flat parameter vector, in the layout above."""
    out, off = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = theta[off:off + size].reshape(shape)
        off += size
    assert off == theta.size
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (8-bit significand), ties to even,
    returned as float64.  Finite inputs only."""
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def features(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """[coordinate 1, coordinate 2, count * weight] per point (count = len(w))."""
    return np.column_stack([x[:, 0], x[:, 1], len(w) * w]).astype(np.float64)


def relu(v):
    return np.maximum(v, 0.0)


def forward(P: dict, x, a, y, b) -> dict:
    """Forward pass for one problem; P holds float64 weights (already rounded)."""
    f, g = features(x, a), features(y, b)
    pre_s = f @ P["W_s"].T + P["b_s"]
    pre_t = g @ P["W_t"].T + P["b_t"]
    e, h = relu(pre_s), relu(pre_t)
    p_s, p_t = e.mean(axis=0), h.mean(axis=0)
    n = len(b)
    inp = np.hstack([h, np.tile(p_s, (n, 1)), np.tile(p_t, (n, 1))])
    z = inp @ P["W_h"].T + P["b_h"]
    u = relu(z)
    o = u @ P["w_o"] + P["b_o"][0]
    return dict(f=f, g=g, pre_s=pre_s, pre_t=pre_t, e=e, h=h, p_s=p_s, p_t=p_t, inp=inp, z=z, u=u, o=o,
                gamma_hat=o - o.mean())


def predict(theta: np.ndarray, x, a, y, b) -> np.ndarray:
    """gamma_hat for one problem from the float32 master parameters."""
    return forward(unflatten(bf16_round(theta)), x, a, y, b)["gamma_hat"]


def loss(theta: np.ndarray, batch: list, gamma_star: list, *, rounded: bool = True) -> float:
    """Batch loss (mean over problems of the per-point mean squared error of
    the centred prediction against the centred target).  rounded=False uses
    the weights as given instead of their bfloat16 rounding."""
    P = unflatten(bf16_round(theta) if rounded else np.asarray(theta, dtype=np.float64))
    tot = 0.0
    for (x, a, y, b), gs in zip(batch, gamma_star):
        gh = forward(P, x, a, y, b)["gamma_hat"]
        d = gh - (gs - gs.mean())
        tot += float(d @ d) / len(b)
    return tot / len(batch)


def loss_and_grad(theta: np.ndarray, batch: list, gamma_star: list, *, rounded: bool = True):
    """Loss and its gradient with respect to the (rounded) weights, by the
    chain rule written out layer by layer.  With rounded=False the weights
    are used as given (for finite-difference checks in float64)."""
    w = bf16_round(theta) if rounded else np.asarray(theta, dtype=np.float64)
    P = unflatten(w)
    G = {k: np.zeros_like(v) for k, v in P.items()}
    Q = len(batch)
    tot = 0.0
    for (x, a, y, b), gs in zip(batch, gamma_star):
        m, n = len(a), len(b)
        F = forward(P, x, a, y, b)
        d = F["gamma_hat"] - (gs - gs.mean())
        tot += float(d @ d) / n
        # d loss / d gamma_hat, then through the centring gamma_hat = o - mean(o)
        dg = 2.0 * d / (n * Q)
        do = dg - dg.mean()
        G["w_o"] += F["u"].T @ do
        G["b_o"][0] += do.sum()
        dz = np.outer(do, P["w_o"]) * (F["z"] > 0)
        G["W_h"] += dz.T @ F["inp"]
        G["b_h"] += dz.sum(axis=0)
        dinp = dz @ P["W_h"]
        dh = dinp[:, :H] + dinp[:, 2 * H:].sum(axis=0) / n
        dps = dinp[:, H:2 * H].sum(axis=0)
        dpre_t = dh * (F["pre_t"] > 0)
        G["W_t"] += dpre_t.T @ F["g"]
        G["b_t"] += dpre_t.sum(axis=0)
        dpre_s = np.tile(dps / m, (m, 1)) * (F["pre_s"] > 0)
        G["W_s"] += dpre_s.T @ F["f"]
        G["b_s"] += dpre_s.sum(axis=0)
    grad = np.concatenate([G[name].ravel() for name, _ in SHAPES])
    return tot / Q, grad


def adam_step(theta, m1, m2, grad, t: int, lr: float, beta1: float, beta2: float, eps: float):
    """One Adam update at step t >= 1 (Kingma & Ba 2015, Algorithm 1); returns
    new (theta, m1, m2) in float64."""
    m1 = beta1 * m1 + (1.0 - beta1) * grad
    m2 = beta2 * m2 + (1.0 - beta2) * grad * grad
    mh = m1 / (1.0 - beta1 ** t)
    vh = m2 / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m1, m2

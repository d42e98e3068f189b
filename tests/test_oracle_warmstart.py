"""Pins of the warm-start network oracle (oracle/warmstart.py), on the CPU.

Each check ties the oracle to something other than itself: a brute-force
search on the bfloat16 grid, finite differences of the loss, symmetries of
mean pooling, and closed forms of Adam's update.
"""

import os
import re

import numpy as np
import pytest

from oracle import warmstart as O
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tiny_batch(seed=0, sizes=((5, 4), (3, 6))):
    rng = np.random.default_rng(seed)
    batch, gstar = [], []
    for m, n in sizes:
        x = rng.uniform(0, 1, (m, 2))
        y = rng.uniform(0, 1, (n, 2))
        a = rng.uniform(0.1, 1, m)
        b = rng.uniform(0.1, 1, n)
        batch.append((x, a / a.sum(), y, b / b.sum()))
        gstar.append(rng.normal(0, 0.1, n))
    return batch, gstar


def test_param_count_matches_layout_and_header():
    assert O.PARAM_COUNT == 50433
    assert sum(int(np.prod(s)) for s in W.WARMSTART_SHAPES) == O.PARAM_COUNT
    assert [s for _, s in O.SHAPES] == [tuple(s) for s in W.WARMSTART_SHAPES]
    text = open(os.path.join(ROOT, "include", "ibsn.h")).read()
    m = re.search(r"#define IBSN_WS_PARAM_COUNT (\d+)", text)
    assert m and int(m.group(1)) == O.PARAM_COUNT


def test_bf16_round_is_nearest_with_ties_to_even():
    rng = np.random.default_rng(1)
    bits = rng.integers(0, 2 ** 32, 20000, dtype=np.uint64).astype(np.uint32)
    bits = bits[((bits >> 23) & 0xFF) < 0xFE]                 # finite, below the largest binade
    ties = (bits & 0xFFFF0000) | 0x8000                       # exact midpoints
    bits = np.concatenate([bits, ties.astype(np.uint32), np.array([0, 0x80000000], np.uint32)])
    x = bits.view(np.float32)
    got = O.bf16_round(x)
    for xi, gi in zip(x.astype(np.float64), got):
        mag = abs(xi)
        # the two bfloat16 neighbours of |x|: truncate, and truncate + one unit
        lo = float(np.array([np.float32(mag).view(np.uint32) & 0xFFFF0000], np.uint32).view(np.float32)[0])
        lo_bits = np.float32(lo).view(np.uint32)
        hi = float(np.array([lo_bits + 0x10000], np.uint32).view(np.float32)[0])
        dl, dh = mag - lo, hi - mag
        if dl < dh or (dl == dh and ((lo_bits >> 16) & 1) == 0):
            want = lo
        else:
            want = hi
        assert abs(gi) == want and (gi == 0 or np.sign(gi) == np.sign(xi)), (xi, gi, want)


def test_gradient_matches_central_differences():
    batch, gstar = _tiny_batch()
    rng = np.random.default_rng(2)
    theta = W.warmstart_init_params(3).astype(np.float64)
    theta[O.PARAM_COUNT - 1] = 0.3                             # b_o
    _, g = O.loss_and_grad(theta, batch, gstar, rounded=False)
    idx = np.concatenate([rng.choice(O.PARAM_COUNT, 300, replace=False),
                          np.arange(0, 8), np.arange(384, 392),  # W_s, b_s rows
                          np.arange(O.PARAM_COUNT - 257, O.PARAM_COUNT)])  # b_h tail, w_o, b_o
    h = 1e-6
    scale = np.abs(g).max()
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (O.loss(tp, batch, gstar, rounded=False) - O.loss(tm, batch, gstar, rounded=False)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * scale + 1e-6 * abs(g[i]), (i, fd, g[i])


def test_output_bias_has_no_gradient_and_prediction_is_centred():
    batch, gstar = _tiny_batch(4)
    theta = W.warmstart_init_params(5)
    _, g = O.loss_and_grad(theta, batch, gstar)
    assert abs(g[-1]) < 1e-15
    for x, a, y, b in batch:
        gh = O.predict(theta, x, a, y, b)
        assert abs(gh.sum()) < 1e-12 * max(1.0, np.abs(gh).max() * len(gh))


def test_pooling_symmetries():
    (x, a, y, b), = _tiny_batch(6, sizes=((9, 7),))[0]
    theta = W.warmstart_init_params(7)
    base = O.predict(theta, x, a, y, b)
    ps = np.random.default_rng(8).permutation(len(a))
    assert np.allclose(O.predict(theta, x[ps], a[ps], y, b), base, rtol=0, atol=1e-12)
    pt = np.random.default_rng(9).permutation(len(b))
    assert np.allclose(O.predict(theta, x, a, y[pt], b[pt]), base[pt], rtol=0, atol=1e-12)


def test_adam_first_step_and_constant_gradient_closed_forms():
    rng = np.random.default_rng(10)
    g = rng.normal(0, 1, 50)
    th0 = rng.normal(0, 1, 50)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    th, m1, m2 = O.adam_step(th0, np.zeros(50), np.zeros(50), g, 1, lr, b1, b2, eps)
    assert np.allclose(th, th0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    # a constant gradient gives bias-corrected moments g and g^2 at every step
    for t in range(2, 7):
        prev = th
        th, m1, m2 = O.adam_step(th, m1, m2, g, t, lr, b1, b2, eps)
        assert np.allclose(prev - th, lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-16)


def test_a_few_adam_steps_reduce_the_loss():
    batch, gstar = _tiny_batch(11, sizes=((6, 5), (4, 8), (7, 7)))
    theta = W.warmstart_init_params(12).astype(np.float64)
    m1 = np.zeros_like(theta)
    m2 = np.zeros_like(theta)
    l0, _ = O.loss_and_grad(theta, batch, gstar, rounded=False)
    for t in range(1, 41):
        _, g = O.loss_and_grad(theta, batch, gstar, rounded=False)
        theta, m1, m2 = O.adam_step(theta, m1, m2, g, t, 1e-3, 0.9, 0.999, 1e-8)
    l1, _ = O.loss_and_grad(theta, batch, gstar, rounded=False)
    assert l1 < 0.5 * l0, (l0, l1)


@pytest.mark.parametrize("seed", [0, 1])
def test_init_params_draw(seed):
    t = W.warmstart_init_params(seed)
    P = O.unflatten(t.astype(np.float64))
    for name in ("b_s", "b_t", "b_h", "b_o"):
        assert not P[name].any()
    assert np.abs(P["W_s"]).max() <= np.sqrt(2.0) and np.abs(P["W_h"]).max() <= np.sqrt(6 / 384)

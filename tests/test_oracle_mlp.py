"""Pins of the oracle's radiance-cache MLP (CPU only)."""
import math

import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S


@pytest.fixture()
def exact(oracle_mod):
    oracle_mod.mlp_set_rounding(False)
    yield oracle_mod
    oracle_mod.mlp_set_rounding(True)


def test_encoding_closed_forms(oracle_mod):
    """Features at hand-derived points: sin/cos(2^k pi x) at x = 0, 1/2, 1; constants."""
    lo, hi = (-1.0, 0.0, -1.0), (1.0, 2.0, 1.0)
    oracle_mod.mlp_set_rounding(False)
    try:
        # position at the box centre (x = 1/2 on every axis), direction +x, normal -z, alpha 0.25
        raw = np.array([[0.0, 1.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, -1.0, 0.25]])
        e = oracle_mod.nrc_encode(raw, lo, hi)[0]
        # k = 0: sin(pi/2) = 1, cos = 0; k = 1: sin(pi) = 0, cos = -1; k >= 2: sin = 0, cos = 1
        want_pos = [1, 0, 0, -1, 0, 1, 0, 1, 0, 1, 0, 1]
        for a in range(3):
            assert np.allclose(e[12 * a:12 * a + 12], want_pos, atol=1e-12)
        # direction +x -> x = 1 on axis 0 (sin(pi)=0, cos=-1; sin(2pi)=0, cos=1); axes 1, 2 -> x = 1/2
        assert np.allclose(e[36:40], [0, -1, 0, 1], atol=1e-12)
        assert np.allclose(e[40:44], [1, 0, 0, -1], atol=1e-12)
        # normal -z -> axis 2 x = 0: sin 0 = 0, cos 0 = 1
        assert np.allclose(e[56:60], [0, 1, 0, 1], atol=1e-12)
        assert e[60] == 0.25 and np.all(e[61:] == 1.0)
    finally:
        oracle_mod.mlp_set_rounding(True)


def test_bf16_rounding_points(oracle_mod):
    """With rounding on, encoded features are exactly representable in BF16."""
    raw, _ = S.random_cache_records(64, 1)
    e = oracle_mod.nrc_encode(raw, (-1, 0, -1), (1, 2, 1))
    bits = e.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)


def test_backward_matches_finite_differences(exact):
    """Plain FP64 network: analytic weight gradient of the relative-L2 loss vs central FD
    on 24 weights spread over all six layers (denominator held fixed, as in the loss)."""
    raw, tgt = S.random_cache_records(32, 2)
    enc = exact.nrc_encode(raw, (-1, 0, -1), (1, 2, 1))
    W = S.mlp_init_weights(3).astype(np.float64)
    loss, g, y = exact.mlp_loss_grad(W, enc, tgt)
    den = y * y + 0.01  # the loss treats the denominator as a constant

    def loss_fixed_den(w):
        yy = exact.mlp_forward(w, enc)
        return np.mean(np.sum((yy - tgt) ** 2 / den, axis=1))
    assert abs(loss_fixed_den(W) - loss) < 1e-12 * max(1, loss)
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.integers(l * 4096, (l + 1) * 4096, 4) for l in range(5)] +
                         [rng.integers(5 * 4096, 5 * 4096 + 192, 4)])
    for i in idx:
        h = 1e-6
        wp, wm = W.copy(), W.copy()
        wp[i] += h
        wm[i] -= h
        fd = (loss_fixed_den(wp) - loss_fixed_den(wm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * np.abs(g).max() + 1e-9 * abs(g[i])


def test_adam_first_step_closed_form(oracle_mod):
    """Bias-corrected first step: w1 = w0 - lr * g / (|g| + eps)."""
    W = np.linspace(-1, 1, 50)
    g = np.linspace(-0.3, 0.5, 50)
    m, v = np.zeros(50), np.zeros(50)
    W1 = W.copy()
    oracle_mod.mlp_adam(W1, g, m, v, 1, lr=0.01, b1=0.9, b2=0.99, eps=1e-8)
    assert np.allclose(W1, W - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_training_reduces_loss(oracle_mod):
    raw, tgt = S.random_cache_records(256, 5)
    enc = oracle_mod.nrc_encode(raw, (-1, 0, -1), (1, 2, 1))
    W = S.mlp_init_weights(6).astype(np.float64)
    m, v = np.zeros_like(W), np.zeros_like(W)
    l0 = None
    for t in range(1, 61):
        loss, g, _ = oracle_mod.mlp_loss_grad(W, enc, tgt)
        l0 = loss if l0 is None else l0
        oracle_mod.mlp_adam(W, g, m, v, t, lr=5e-3)
    assert loss < 0.2 * l0

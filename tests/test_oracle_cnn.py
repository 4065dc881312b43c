"""Pins of the fp64 CNN oracle: finite differences of the loss for every
parameter tensor, the convolution against scipy's correlation, the thumbnail
against its definition on a hand-made frame, the softmax-CE gradient."""
import numpy as np
import pytest
from scipy.signal import correlate

from oracle import cnn


def test_conv3x3_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 7, 9))
    w = rng.normal(size=(3, 3, 3, 4))
    b = rng.normal(size=4)
    y = cnn.conv3x3(x, w, b)
    for co in range(4):
        ref = b[co] + sum(correlate(x[ci], w[:, :, ci, co], mode="same") for ci in range(3))
        assert np.allclose(y[co], ref, atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    P = cnn.init_params(C=3, K=4, seed=2)
    for k in P:
        P[k] = P[k] + 0.1 * rng.normal(size=P[k].shape)   # non-zero biases too
    x = rng.normal(size=(2, 6, 5))
    label = 2
    G = cnn.backward(P, x, label)
    eps = 1e-6
    for name, arr in P.items():
        flat = arr.reshape(-1)
        for idx in rng.choice(flat.size, min(flat.size, 6), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = cnn.loss(P, x, label)
            flat[idx] = old - eps
            lm = cnn.loss(P, x, label)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            g = G[name].reshape(-1)[idx]
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g)


def test_softmax_ce_gradient_closed_form():
    P = cnn.init_params(C=2, K=3, seed=3)
    x = np.zeros((2, 4, 4))
    G = cnn.backward(P, x, 1)
    logits, _ = cnn.forward(P, x)
    p = np.exp(logits - logits.max())
    p /= p.sum()
    p[1] -= 1
    assert np.allclose(G["bl"], p)


def test_thumbnail_definition():
    p = 2
    fr = np.full((4, 6), 100, dtype=np.uint16)
    fr[0, 0] = 100 + 1000
    th = cnn.thumbnail(fr, p)
    assert th.shape == (2, 256, 256)
    # bs = ceil(6 / 256) = 1: every pixel is its own block
    assert th[0, 0, 0] == pytest.approx(np.log1p(1000) / 8)
    assert th[0, 0, 1] == 0 and th[0, 4:, :].sum() == 0
    vm = cnn.view_major(fr, p)
    assert vm[0, 0] == fr[0, 0] and th[1, 0, 0] == pytest.approx(np.log1p(1000) / 8)
    big = np.full((600, 300), 150, dtype=np.uint16)
    tb = cnn.thumbnail(big, 15)  # bs = 3 -> 200 x 100 blocks of value log1p(50)/8
    assert np.allclose(tb[0, :200, :100], np.log1p(50) / 8) and tb[0, 200:].sum() == 0


def test_bf16_rounding_bit_patterns():
    """BF16 = the top 16 bits of binary32, rounded to nearest, ties to even
    (hand-worked bit patterns)."""
    cases = [
        (1.0, 1.0),                          # 0x3F800000 exact
        (1.0 + 2.0 ** -8, 1.0),              # 0x3F808000: tie, kept bit 0 -> down
        (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),  # 0x3F818000: tie, kept bit 1 -> up
        (1.0 + 2.0 ** -8 + 2.0 ** -20, 1.0 + 2.0 ** -7),  # above the tie -> up
        (-2.5, -2.5),                        # exact
        (0.1, 0.10009765625),                # 0x3DCCCCCD -> 0x3DCD0000
        (0.0, 0.0),
    ]
    for v, exp in cases:
        assert cnn.bf16(v) == exp, (v, cnn.bf16(v), exp)


def test_rounding_hook_identity_is_the_fp64_network():
    rng = np.random.default_rng(3)
    P = cnn.init_params(C=3, K=4, seed=4)
    x = rng.normal(size=(2, 6, 5))
    G0 = cnn.backward(P, x, 1)
    G1 = cnn.backward(P, x, 1, act_round=lambda a: a)
    for k in G0:
        assert np.array_equal(G0[k], G1[k])
    Gq = cnn.backward(P, x, 1, act_round=cnn.bf16)
    # BF16 storage changes the gradients by a few BF16 units at most
    for k in G0:
        assert np.allclose(Gq[k], G0[k], rtol=5e-2, atol=5e-2 * np.abs(G0[k]).max())

"""Pins of the reranker MLP reference (CPU only).

The learned reranker is not in the paper; it orders LSH candidates by a predicted Jaccard.
Network: d_in -> 64 -> 64 -> 1 with ReLU, ReLU, sigmoid and mean squared error.  Pins:
central finite differences of the exact fp64 network (bf16 emulation off), and the bf16
network staying within bf16 rounding distance of the exact one.
"""
import numpy as np
import pytest


def params(rng, d_in=40, d_h=64):
    return dict(
        w1=rng.normal(0, 1 / np.sqrt(d_in), (d_h, d_in)), b1=rng.normal(0, 0.1, d_h),
        w2=rng.normal(0, 1 / np.sqrt(d_h), (d_h, d_h)), b2=rng.normal(0, 0.1, d_h),
        w3=rng.normal(0, 1 / np.sqrt(d_h), d_h), b3=rng.normal(0, 0.1, 1))


def test_finite_differences_exact_network(orc):
    rng = np.random.default_rng(0)
    d_in, d_h = 9, 8
    p = params(rng, d_in, d_h)
    x = rng.normal(0, 1, (13, d_in)).astype(np.float32)
    y = rng.uniform(0, 1, 13).astype(np.float32)
    _, loss, g = orc.mlp_forward_backward(x, y, **p, bf16=False)
    names = ["w1", "b1", "w2", "b2", "w3", "b3"]
    eps = 1e-6
    for name, grad in zip(names, g):
        flat = p[name].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + eps
            _, lp, _ = orc.mlp_forward_backward(x, y, **p, grads=False, bf16=False)
            flat[idx] = old - eps
            _, lm, _ = orc.mlp_forward_backward(x, y, **p, grads=False, bf16=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert grad.reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (name, idx)


def test_bf16_network_is_close_to_exact(orc):
    rng = np.random.default_rng(1)
    p = params(rng)
    x = rng.normal(0, 1, (256, 40)).astype(np.float32)
    y = rng.uniform(0, 1, 256).astype(np.float32)
    pe, le, ge = orc.mlp_forward_backward(x, y, **p, bf16=False)
    pb, lb, gb = orc.mlp_forward_backward(x, y, **p, bf16=True)
    assert np.max(np.abs(pe - pb)) < 2e-2
    # gradients sum signed terms over rows, so bf16 operand rounding (2^-9 relative) is
    # amplified by cancellation; the direction and the size must still agree closely
    for a, b in zip(ge, gb):
        a, b = a.reshape(-1), b.reshape(-1)
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        assert cos > 0.99
        assert abs(np.linalg.norm(b) / np.linalg.norm(a) - 1) < 0.1


def test_bf16_rounding_is_nearest_even(orc):
    assert orc.bf16_round(1.0) == 1.0
    assert orc.bf16_round(1.0 + 2 ** -8) == 1.0            # tie -> even (mantissa 0)
    assert orc.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie -> even (round up)
    assert orc.bf16_round(1.0 + 2 ** -7) == 1.0 + 2 ** -7   # representable
    assert orc.bf16_round(-3.0) == -3.0

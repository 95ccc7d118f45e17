"""Pins of the CPU MLP oracle (learned alpha): finite differences, an affine
regime with a closed form, bfloat16 rounding and Adam's first step."""
import numpy as np
import pytest

from oracle.mlp_oracle import adam_update, bf16_round, mlp_forward, mlp_loss_and_grads


def _params(rng, d=7, w=5, scale=0.5):
    return {"W1": rng.normal(0, scale, (w, d)), "b1": rng.normal(0, scale, w),
            "W2": rng.normal(0, scale, (w, w)), "b2": rng.normal(0, scale, w),
            "w3": rng.normal(0, scale, w), "b3": np.array(rng.normal())}


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    p = _params(rng)
    x = rng.normal(size=(9, 7))
    t = rng.normal(size=9)
    _, g = mlp_loss_and_grads(p, x, t)
    eps = 1e-6
    for k, v in p.items():
        v = np.atleast_1d(v)
        flat = v.reshape(-1)
        for i in range(flat.size):
            q = {kk: np.array(vv, dtype=np.float64, copy=True) for kk, vv in p.items()}
            qa = np.atleast_1d(q[k]).reshape(-1)
            qa[i] += eps
            q[k] = qa.reshape(np.shape(p[k]))
            lp, _ = mlp_loss_and_grads(q, x, t)
            qa[i] -= 2 * eps
            q[k] = qa.reshape(np.shape(p[k]))
            lm, _ = mlp_loss_and_grads(q, x, t)
            fd = (lp - lm) / (2 * eps)
            an = np.atleast_1d(g[k]).reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, i, fd, an)


def test_affine_regime_closed_form():
    """Positive weights and inputs keep every ReLU active: the network is the
    affine map w3.(W2 (W1 x + b1) + b2) + b3."""
    rng = np.random.default_rng(1)
    p = {k: np.abs(v) for k, v in _params(rng).items()}
    x = np.abs(rng.normal(size=(4, 7)))
    y, _ = mlp_forward(p, x)
    want = (p["W2"] @ (p["W1"] @ x.T + p["b1"][:, None]) + p["b2"][:, None]).T @ p["w3"] + p["b3"]
    np.testing.assert_allclose(y, want, rtol=1e-13)
    t = np.zeros(4)
    _, g = mlp_loss_and_grads(p, x, t)
    np.testing.assert_allclose(g["b3"], np.mean(y - t), rtol=1e-13)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -(1.0 + 2.0 ** -7 + 2.0 ** -8), 0.0, 3.0e38],
                    dtype=np.float32)
    got = bf16_round(vals)
    want = [1.0, 1.0, 1.0 + 2.0 ** -7, -(1.0 + 2.0 ** -6), 0.0, bf16_round(np.float32(3.0e38))[()]]
    np.testing.assert_array_equal(got[:5], want[:5])       # ties to even, sign kept
    assert got[5] > 2.9e38


def test_adam_first_step_is_signed_lr():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = adam_update(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01, eps=0.0)
    np.testing.assert_allclose(p, -0.01 * np.sign(g), rtol=1e-12)

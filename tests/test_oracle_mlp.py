"""Pins for the MLP oracle: its gradient against central finite differences
(in the smooth surrogate without BF16 rounding, where the loss is
differentiable), and the BF16 rounding against a bit-level definition."""
import numpy as np

from oracle import mlp_oracle as M


def test_bf16_rounding_definition():
    # exactly representable values are unchanged; halfway cases tie to even
    vals = np.array([1.0, -2.5, 3.0, 0.0], dtype=np.float32)
    assert np.array_equal(M.bf16_round(vals), vals.astype(np.float64))
    one = np.float32(1.0)
    ulp = 2.0 ** -7                        # BF16 spacing at 1.0
    half = np.float32(1.0 + ulp / 2)       # tie -> 1.0 (even mantissa)
    assert M.bf16_round(np.array([half]))[0] == 1.0
    up = np.float32(1.0 + 1.5 * ulp)       # tie between 1+ulp and 1+2ulp -> 1+2ulp
    assert M.bf16_round(np.array([up]))[0] == 1.0 + 2 * ulp
    assert M.bf16_round(np.array([np.float32(1.0 + 0.6 * ulp)]))[0] == 1.0 + ulp
    del one


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = rng.normal(scale=0.3, size=M.N_PARAMS)
    x = rng.normal(size=(17, M.N_IN))
    t = rng.normal(size=17)
    loss, g = M.loss_grad(p, x, t, rounding=False)
    idx = rng.choice(M.N_PARAMS, 60, replace=False).tolist() + [M.OFF_B3, M.OFF_W3, M.OFF_B1]
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        # float32 cast in forward() would destroy the step: evaluate in fp64
        lp = _loss64(pp, x, t)
        lm = _loss64(pm, x, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(g[i]), (i, fd, g[i])
    assert abs(loss - _loss64(p, x, t)) < 1e-9 * max(1, abs(loss))


def _loss64(p, x, t):
    W1, b1, W2, b2, w3, b3 = M.unpack(p)
    a1 = x @ W1.T + b1
    h1 = np.maximum(a1, 0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0)
    y = h2 @ w3 + b3
    return float(np.mean((y - t) ** 2))

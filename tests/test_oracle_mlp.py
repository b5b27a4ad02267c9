"""Pins for the MLP oracle: the forward pass on hand-built routing networks
whose outputs follow by hand from the parameter layout the public header
documents (W1[64][12], b1[64], W2[64][64], b2[64], w3[64], b3, row-major,
output index first); its gradient against central finite differences of its
own forward pass (in the smooth surrogate without BF16 rounding, where the
loss is differentiable); and the BF16 rounding against a bit-level
definition."""
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
        # the surrogate keeps the parameters in fp64 (a float32 cast would
        # destroy the step)
        lp = _loss64(pp, x, t)
        lm = _loss64(pm, x, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(g[i]), (i, fd, g[i])
    assert abs(loss - _loss64(p, x, t)) < 1e-9 * max(1, abs(loss))


def _loss64(p, x, t):
    y, _ = M.forward(np.asarray(p, np.float64), x, rounding=False)
    return float(np.mean((y - t) ** 2))


# offsets of the documented layout, typed from the header's description
IN, HID = 12, 64
W1_AT = lambda i, j: i * IN + j                        # noqa: E731  W1[i][j], i hidden, j input
B1_AT = lambda i: HID * IN + i                         # noqa: E731
W2_AT = lambda k, i: HID * IN + HID + k * HID + i      # noqa: E731  W2[k][i]
B2_AT = lambda k: HID * IN + HID + HID * HID + k       # noqa: E731
W3_AT = lambda k: HID * IN + 2 * HID + HID * HID + k   # noqa: E731
B3_AT = HID * IN + 3 * HID + HID * HID


def _net(entries):
    p = np.zeros(B3_AT + 1, np.float32)
    for at, v in entries:
        p[at] = v
    return p


def test_layout_constants():
    assert M.N_PARAMS == B3_AT + 1 == 5057
    assert (M.OFF_B1, M.OFF_W2, M.OFF_B2, M.OFF_W3, M.OFF_B3) == (B1_AT(0), W2_AT(0, 0), B2_AT(0), W3_AT(0), B3_AT)


def test_forward_routing_networks():
    rng = np.random.default_rng(5)
    x = rng.integers(-8, 9, size=(9, IN)).astype(np.float64)   # BF16-exact inputs
    # only the output bias: a constant
    y, _ = M.forward(_net([(B3_AT, 0.75)]), x)
    assert np.array_equal(y, np.full(9, 0.75))
    # input j -> hidden i -> hidden k -> output: y = 2 max(x_j, 0) - 1; hidden
    # and input indices chosen so that a transposed W1 or W2 routes elsewhere
    for j, i, k in ((5, 40, 7), (0, 63, 62), (11, 13, 0)):
        p = _net([(W1_AT(i, j), 1.0), (W2_AT(k, i), 1.0), (W3_AT(k), 2.0), (B3_AT, -1.0)])
        y, _ = M.forward(p, x)
        assert np.array_equal(y, 2 * np.maximum(x[:, j], 0) - 1), (j, i, k)
    # biases: h1_i = relu(3) = 3, a2_k = 0.5 * 3 - 1 = 0.5, y = -4 * 0.5
    p = _net([(B1_AT(20), 3.0), (W2_AT(33, 20), 0.5), (B2_AT(33), -1.0), (W3_AT(33), -4.0)])
    assert np.array_equal(M.forward(p, x)[0], np.full(9, -2.0))
    # a negative pre-activation is cut by the first ReLU
    p = _net([(B1_AT(20), -3.0), (W2_AT(33, 20), 0.5), (B2_AT(33), 1.0), (W3_AT(33), 1.0)])
    assert np.array_equal(M.forward(p, x)[0], np.full(9, 1.0))
    # ... and by the second
    p = _net([(B1_AT(20), 3.0), (W2_AT(33, 20), -1.0), (W3_AT(33), 1.0), (B3_AT, 0.25)])
    assert np.array_equal(M.forward(p, x)[0], np.full(9, 0.25))


def test_forward_rounds_inputs_and_activations_to_bf16():
    # an input off the BF16 grid is rounded before the first layer
    p = _net([(W1_AT(2, 3), 1.0), (W2_AT(4, 2), 1.0), (W3_AT(4), 1.0)])
    x = np.zeros((1, IN))
    x[0, 3] = 1.0 + 2.0 ** -9
    assert M.forward(p, x)[0][0] == 1.0
    # a hidden activation off the grid is rounded: (1 + 2^-7)^2 = 1 + 2^-6 + 2^-14 -> 1 + 2^-6
    a = 1.0 + 2.0 ** -7
    p = _net([(W1_AT(2, 3), a), (W2_AT(4, 2), 1.0), (W3_AT(4), 1.0)])
    x[0, 3] = a
    assert M.forward(p, x)[0][0] == 1.0 + 2.0 ** -6
    # parameters are rounded too: 1 + 2^-9 is used as 1
    p = _net([(W1_AT(2, 3), 1.0 + 2.0 ** -9), (W2_AT(4, 2), 1.0), (W3_AT(4), 1.0)])
    x[0, 3] = 3.0
    assert M.forward(p, x)[0][0] == 3.0
    # without rounding the same network is exact in fp64
    p64 = np.zeros(B3_AT + 1)
    p64[[W1_AT(2, 3), W2_AT(4, 2), W3_AT(4)]] = (1.0 + 2.0 ** -9, 1.0, 1.0)
    assert M.forward(p64, x, rounding=False)[0][0] == 3.0 * (1.0 + 2.0 ** -9)

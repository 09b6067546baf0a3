"""Pins of the FP64 warm-start perceptron (oracle/mlp.py) against values
fixed outside it: finite differences, a network worked by hand, the
bfloat16 format's rounding rule and torch's conversion, Adam's closed form."""

import numpy as np
import pytest

from oracle import mlp


def _rand_net(n_in, H, n_out, N, seed):
    r = np.random.default_rng(seed)
    lay = mlp.layout(n_in, H, n_out)
    w = r.normal(0.0, 0.5, size=lay["count"])
    X = r.normal(size=(N, n_in))
    T = r.normal(size=(N, n_out))
    return w, X, T


def test_layout_offsets():
    lay = mlp.layout(16, 256, 3)
    assert lay["W1"] == (0, 4096)
    assert lay["b1"] == (4096, 4352)
    assert lay["W2"] == (4352, 4352 + 65536)
    assert lay["b3"][1] == lay["count"] == 4096 + 256 + 65536 + 256 + 768 + 3


def test_hand_worked_network():
    # two inputs, two hidden units, one output; every value below is worked by hand
    W1 = [[1.0, -1.0], [0.5, 2.0]]
    b1 = [0.0, -1.0]
    W2 = [[1.0, 1.0], [-1.0, 1.0]]
    b2 = [0.5, 0.0]
    W3 = [[2.0, -4.0]]
    b3 = [0.25]
    flat = mlp.pack([W1, b1, W2, b2, W3, b3])
    X = np.array([[1.0, 2.0]])
    # z1 = (-1, 3.5) -> h1 = (0, 3.5); z2 = (4, 3.5) = h2; y = 8 - 14 + 0.25
    assert mlp.forward(flat, X, 2, 2, 1)[0, 0] == -5.75
    T = np.array([[-6.75]])
    L, g = mlp.loss_and_grad(flat, X, T, 2, 2, 1)
    assert L == 1.0
    # dy = 2; dW3 = dy h2; dh2 = dy W3 = (4, -8); dW2 = dh2^T h1;
    # dh1 = dh2 W2 = (12, -4) masked by h1 > 0 -> (0, -4); dW1 = dh1^T x
    want = mlp.pack([[[0.0, 0.0], [-4.0, -8.0]], [0.0, -4.0],
                     [[0.0, 14.0], [0.0, -28.0]], [4.0, -8.0],
                     [[8.0, 7.0]], [2.0]])
    np.testing.assert_array_equal(g, want)


@pytest.mark.parametrize("shape", [(3, 5, 2, 7), (16, 12, 3, 40)])
def test_gradient_central_differences(shape):
    n_in, H, n_out, N = shape
    w, X, T = _rand_net(n_in, H, n_out, N, seed=sum(shape))
    _, g = mlp.loss_and_grad(w, X, T, n_in, H, n_out)
    h = 1e-5
    fd = np.empty_like(w)
    for i in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd[i] = (mlp.loss(wp, X, T, n_in, H, n_out) - mlp.loss(wm, X, T, n_in, H, n_out)) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-6 * max(1.0, np.max(np.abs(g)))


def test_gradient_zero_at_exact_fit():
    w, X, _ = _rand_net(4, 6, 2, 9, seed=3)
    T = mlp.forward(w, X, 4, 6, 2)
    L, g = mlp.loss_and_grad(w, X, T, 4, 6, 2)
    assert L == 0.0 and not np.any(g)


def test_bf16_rounding_ties_and_halves():
    one = np.float32(1.0)
    ulp = 2.0 ** -7                          # bfloat16 spacing at 1
    x = np.array([1.0, 1.0 + ulp / 2, 1.0 + 1.5 * ulp, 1.0 + ulp / 2 + 2.0 ** -20,
                  -(1.0 + 1.5 * ulp), 3.0, 2.0 ** -130], dtype=np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2 * ulp, 1.0 + ulp, -(1.0 + 2 * ulp), 3.0, 2.0 ** -130],
                    dtype=np.float32)
    np.testing.assert_array_equal(mlp.bf16_round(x), want)
    assert mlp.bf16_round(one) == one


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(5)
    x = (r.normal(size=20000) * 10.0 ** r.integers(-8, 8, 20000)).astype(np.float32)
    # add exact halfway cases
    b = x.view(np.uint32) & np.uint32(0xFFFF0000)
    x = np.concatenate([x, (b | np.uint32(0x8000)).view(np.float32)])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), want)


def test_adam_constant_gradient_closed_form():
    # under a constant gradient both bias-corrected moments are exact:
    # m^ = g and v^ = g^2, so every step moves w by lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    w0 = np.array([1.0, 2.0, 3.0, 4.0])
    opt = mlp.Adam(4, lr=0.01)
    w = w0.copy()
    for _ in range(5):
        w = opt.step(w, g)
    np.testing.assert_allclose(w, w0 - 5 * 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_init_params_bounds_and_biases():
    n_in, H, n_out = 16, 256, 3
    w = mlp.init_params(n_in, H, n_out, seed=7)
    assert w.dtype == np.float32
    W1, b1, W2, b2, W3, b3 = mlp.unpack(w.astype(np.float64), n_in, H, n_out)
    for Wm, bound in ((W1, np.sqrt(6 / n_in)), (W2, np.sqrt(6 / H)), (W3, 0.1 * np.sqrt(6 / H))):
        assert np.all(np.abs(Wm) <= bound * (1 + 1e-7))
        # uniform on [-bound, bound): variance bound^2 / 3
        assert abs(Wm.var() / (bound ** 2 / 3) - 1.0) < 0.1
    assert not np.any(b1) and not np.any(b2) and not np.any(b3)

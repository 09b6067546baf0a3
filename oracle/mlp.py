"""FP64 reference of the warm-start perceptron.

Test infrastructure (see ``oracle/__init__``).  The paper has no learned
component; this is the definition the CUDA network is checked against.

Network: ``n_in -> H -> H -> n_out`` with ReLU after both hidden layers and
no activation after the output, on standardised inputs
``X' = (X - mu) * inv_sigma`` (float32 arithmetic, as stored; identity by
default): ``H1 = relu(X' W1^T + b1)``,
``H2 = relu(H1 W2^T + b2)``, ``Y = H2 W3^T + b3``.  Loss: the mean of the
squared differences over all ``N * n_out`` outputs.  Parameters are one flat
array ``[W1 (H x n_in, row-major), b1, W2 (H x H), b2, W3 (n_out x H), b3]``.
Optimiser: Adam (Kingma and Ba, "Adam: a method for stochastic
optimization", ICLR 2015) with bias-corrected moments.

The CUDA network multiplies with weights rounded to bfloat16 (round to
nearest, ties to even, on the float32 master value); ``bf16_round`` writes
that rounding out from the bfloat16 format (the top 16 bits of a binary32),
and ``forward`` / ``loss_and_grad`` take ``weight_round="bf16"`` to use it.
Everything else is float64.

Pins (tests/test_oracle_mlp.py): central finite differences of the loss
against the analytic gradient; a hand-computed two-unit network; bf16
rounding against fixed ties and against torch's float32 -> bfloat16
conversion; Adam's closed form under a constant gradient; the seeded
initialisation against splitmix64 outputs computed from its definition.
"""

import numpy as np

from . import rng


def layout(n_in, H, n_out):
    """Offsets of [W1, b1, W2, b2, W3, b3] in the flat parameter array."""
    o = {}
    at = 0
    for name, size in (("W1", H * n_in), ("b1", H), ("W2", H * H), ("b2", H),
                       ("W3", n_out * H), ("b3", n_out)):
        o[name] = (at, at + size)
        at += size
    o["count"] = at
    return o


def unpack(flat, n_in, H, n_out):
    lay = layout(n_in, H, n_out)
    g = lambda k: flat[lay[k][0]:lay[k][1]]  # noqa: E731
    return (g("W1").reshape(H, n_in), g("b1"), g("W2").reshape(H, H), g("b2"),
            g("W3").reshape(n_out, H), g("b3"))


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def init_params(n_in, H, n_out, seed):
    """He-uniform weights with bound sqrt(6 / fan_in) drawn as
    u_e * bound from the splitmix64 doubles u_e in [-1, 1) (element e of
    the flat array, generator seeded with ``seed``); the output layer's
    weights are further scaled by 0.1 (0.1 * u_e first, then the bound);
    biases are zero.  Rounded once to float32 (the master copy's type)."""
    lay = layout(n_in, H, n_out)
    u = rng.uniform_pm1(seed, lay["count"])
    w = np.zeros(lay["count"])
    a, b = lay["W1"]
    w[a:b] = u[a:b] * np.sqrt(6.0 / n_in)
    a, b = lay["W2"]
    w[a:b] = u[a:b] * np.sqrt(6.0 / H)
    a, b = lay["W3"]
    w[a:b] = (0.1 * u[a:b]) * np.sqrt(6.0 / H)
    return w.astype(np.float32)


def bf16_round(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float32.

    bfloat16 keeps the sign, the 8 exponent bits and the top 7 fraction bits
    of a binary32 value; rounding adds half a unit of the 16 dropped bits,
    minus one when the kept part is even (so exact halves go to even), and
    truncates.  Finite inputs only (the network never holds NaN or Inf)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = (b + np.uint64(0x7FFF) + lsb) >> np.uint64(16) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32)


def _weights(flat, n_in, H, n_out, weight_round):
    flat = np.asarray(flat)
    W1, b1, W2, b2, W3, b3 = unpack(flat.astype(np.float64), n_in, H, n_out)
    if weight_round == "bf16":
        r = lambda w: bf16_round(w.astype(np.float32)).astype(np.float64)  # noqa: E731
        W1, W2, W3 = r(W1), r(W2), r(W3)
    elif weight_round is not None:
        raise ValueError(weight_round)
    return W1, b1, W2, b2, W3, b3


def standardize(X, mu=None, inv_sigma=None):
    """(X - mu) * inv_sigma, each step rounded to float32 like the stored
    float32 features; no-op without mu."""
    if mu is None:
        return np.asarray(X, dtype=np.float64)
    X = np.asarray(X, dtype=np.float32)
    d = (X - np.asarray(mu, dtype=np.float32)).astype(np.float32)
    return (d * np.asarray(inv_sigma, dtype=np.float32)).astype(np.float32).astype(np.float64)


def fit_normalizer(X):
    """Column means and 1 / population standard deviations (1 where the
    deviation is <= 1e-12 * max(1, |mean|)), as float32."""
    X = np.asarray(X, dtype=np.float64)
    m = X.mean(axis=0)
    sd = X.std(axis=0)
    inv = np.where(sd > 1e-12 * np.maximum(1.0, np.abs(m)), 1.0 / np.where(sd > 0, sd, 1.0), 1.0)
    return m.astype(np.float32), inv.astype(np.float32)


def forward(flat, X, n_in, H, n_out, weight_round=None, keep=False, norm=None):
    """Y = network(X), X [N, n_in] -> [N, n_out] in float64; ``norm`` is
    (mu, inv_sigma) or None."""
    W1, b1, W2, b2, W3, b3 = _weights(flat, n_in, H, n_out, weight_round)
    X = standardize(X, *(norm or (None, None)))
    H1 = np.maximum(X @ W1.T + b1, 0.0)
    H2 = np.maximum(H1 @ W2.T + b2, 0.0)
    Y = H2 @ W3.T + b3
    if keep:
        return Y, (X, H1, H2, W1, W2, W3)
    return Y


def loss(flat, X, T, n_in, H, n_out, weight_round=None, norm=None):
    Y = forward(flat, X, n_in, H, n_out, weight_round, norm=norm)
    return float(np.mean((Y - np.asarray(T, dtype=np.float64)) ** 2))


def loss_and_grad(flat, X, T, n_in, H, n_out, weight_round=None, norm=None):
    """(loss, gradient as a flat float64 array), by the chain rule.  With
    weight_round the gradient is taken with respect to the rounded weights
    (the straight-through rule the CUDA network follows)."""
    Y, (X, H1, H2, W1, W2, W3) = forward(flat, X, n_in, H, n_out, weight_round, keep=True,
                                         norm=norm)
    T = np.asarray(T, dtype=np.float64)
    N = X.shape[0]
    L = float(np.mean((Y - T) ** 2))
    dY = 2.0 * (Y - T) / (N * n_out)
    gW3 = dY.T @ H2
    gb3 = dY.sum(axis=0)
    dH2 = (dY @ W3) * (H2 > 0)
    gW2 = dH2.T @ H1
    gb2 = dH2.sum(axis=0)
    dH1 = (dH2 @ W2) * (H1 > 0)
    gW1 = dH1.T @ X
    gb1 = dH1.sum(axis=0)
    return L, pack([gW1, gb1, gW2, gb2, gW3, gb3])


class Adam:
    """m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
    w -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""

    def __init__(self, count, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(count)
        self.v = np.zeros(count)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, w, g):
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * g
        self.v = self.b2 * self.v + (1.0 - self.b2) * g * g
        mh = self.m / (1.0 - self.b1 ** self.t)
        vh = self.v / (1.0 - self.b2 ** self.t)
        return w - self.lr * mh / (np.sqrt(vh) + self.eps)

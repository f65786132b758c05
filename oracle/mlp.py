"""FP64 oracle of the warm-rain surrogate network -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU-baseline leg use it;
it shares no code with the CUDA path.

Network: 12 inputs -> 256 -> 256 -> 256 -> 4 outputs, tanh on the hidden
layers, linear output.  Inputs are the standardised features of a point,
outputs the standardised logarithms of the four warm-rain rates
(autoconversion, accretion, cloud and rain self-collection).  The loss is the
squared error summed over the outputs a point defines (mask), divided by the
number of defined outputs.

The GPU form keeps weights and every GEMM operand in BF16 with FP32
accumulation.  With `bf16_round=True` this oracle rounds at exactly those
points (weights, the input of every layer, the back-propagated pre-activation
gradients) and is FP64 everywhere else, so the two differ only by
accumulation order and FP32 tanh.

Flat parameter order (FP32 on the GPU): W1[12][256], b1[256], W2[256][256],
b2[256], W3[256][256], b3[256], W4[256][4], b4[4]; W[k][n] multiplies input k
into unit n.
"""
from __future__ import annotations

import numpy as np

SIZES = (12, 256, 256, 256, 4)


def param_count() -> int:
    return sum(SIZES[i] * SIZES[i + 1] + SIZES[i + 1] for i in range(4))


def unflatten(theta: np.ndarray):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (param_count(),)
    out, o = [], 0
    for i in range(4):
        k, n = SIZES[i], SIZES[i + 1]
        W = theta[o:o + k * n].reshape(k, n)
        o += k * n
        b = theta[o:o + n]
        o += n
        out.append((W, b))
    return out


def flatten(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers])


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _q(bf16_round):
    return bf16 if bf16_round else (lambda a: np.asarray(a, dtype=np.float64))


def forward(theta: np.ndarray, X: np.ndarray, bf16_round: bool = False):
    """Returns (Y, hs, zs): outputs [n][4], layer inputs h_0..h_3 and
    pre-activations z_0..z_3 (z_i = h_i W_i + b_i, h_{i+1} = tanh z_i)."""
    q = _q(bf16_round)
    layers = unflatten(theta)
    h = q(X)
    hs, zs = [h], []
    for i, (W, b) in enumerate(layers):
        z = h @ q(W) + b
        zs.append(z)
        if i < 3:
            h = q(np.tanh(z))
            hs.append(h)
    return zs[3], hs, zs


def loss_grad(theta: np.ndarray, X: np.ndarray, T: np.ndarray, M: np.ndarray, bf16_round: bool = False):
    """Masked squared-error loss and its gradient with respect to theta
    (the chain rule, layer by layer)."""
    q = _q(bf16_round)
    layers = unflatten(theta)
    Y, hs, zs = forward(theta, X, bf16_round)
    cnt = max(float(M.sum()), 1.0)
    diff = (Y - T) * M
    loss = float((diff * diff).sum() / cnt)
    dz = 2.0 * diff / cnt
    grads = [None] * 4
    for i in range(3, -1, -1):
        W, _ = layers[i]
        gW = hs[i].T @ q(dz)
        gb = dz.sum(axis=0)
        grads[i] = (gW, gb)
        if i > 0:
            dh = q(dz) @ q(W).T
            dz = dh * (1.0 - np.tanh(zs[i - 1]) ** 2)
    return loss, flatten(grads)


def init_params(seed: int) -> np.ndarray:
    """Xavier-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    layers = []
    for i in range(4):
        k, n = SIZES[i], SIZES[i + 1]
        lim = np.sqrt(6.0 / (k + n))
        layers.append((rng.uniform(-lim, lim, size=(k, n)), np.zeros(n)))
    return flatten(layers)

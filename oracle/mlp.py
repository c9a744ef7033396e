"""Plain FP64 reference of the rank-proposal network (forward, backward,
Adam step).

TEST INFRASTRUCTURE ONLY: imported by the tests and nothing else.  The
product library trains and evaluates the network with its own CUDA kernels.

The network is not part of the paper: RS-S determines every skeleton rank by
column-pivoted QR (Sec. 2.2, Definition 2.1).  The proposal only presizes
storage; the QR still decides each rank.  What is defined here:

  features x (16 values per box, the last ones zero), then
      h1 = tanh(W1 x  + b1)      W1: 64 x 16
      h2 = tanh(W2 h1 + b2)      W2: 64 x 64
      h3 = tanh(W3 h2 + b3)      W3: 64 x 64
      o  = w4 . h3 + b4          w4: 64, b4: scalar
  prediction of the rank fraction k / b; loss = mean over samples of
  (o - y)^2.

Parameters are one flat FP32 vector in the order W1 (row-major, row = output
unit), b1, W2, b2, W3, b3, w4, b4: 9473 values.  The network computes with
the parameters rounded to bfloat16 (round to nearest, ties to even, on the
FP32 bit pattern); this module rounds the same way and then works in FP64.
"""
from __future__ import annotations

import numpy as np

NFEAT = 16
HID = 64
SHAPES = [("W1", (HID, NFEAT)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, HID)), ("b3", (HID,)), ("w4", (HID,)), ("b4", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    """Split the flat parameter vector into named arrays (views)."""
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    assert o == theta.size == NPARAM
    return out


def pack(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def bf16_round(a) -> np.ndarray:
    """Round FP32 values to bfloat16 (nearest, ties to even), returned as FP64.
    bfloat16 keeps the top 16 bits of the FP32 pattern; the discarded low half
    is rounded into the kept half."""
    u = np.asarray(a, dtype=np.float32).reshape(-1).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


def forward(theta: np.ndarray, X: np.ndarray):
    """Output o (n,) and the activations the backward pass needs."""
    p = unpack(np.asarray(theta, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    h3 = np.tanh(h2 @ p["W3"].T + p["b3"])
    o = h3 @ p["w4"] + p["b4"][0]
    return o, (X, h1, h2, h3)


def loss(theta: np.ndarray, X: np.ndarray, y: np.ndarray) -> float:
    o, _ = forward(theta, X)
    return float(np.mean((o - np.asarray(y, dtype=np.float64)) ** 2))


def backward(theta: np.ndarray, X: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Gradient of the mean squared loss with respect to the flat parameters,
    by the chain rule layer by layer (tanh' = 1 - tanh^2)."""
    p = unpack(np.asarray(theta, dtype=np.float64))
    o, (X, h1, h2, h3) = forward(theta, X)
    n = X.shape[0]
    do = 2.0 * (o - np.asarray(y, dtype=np.float64)) / n
    g = {}
    g["w4"] = h3.T @ do
    g["b4"] = np.array([do.sum()])
    dz3 = np.outer(do, p["w4"]) * (1.0 - h3 * h3)
    g["W3"] = dz3.T @ h2
    g["b3"] = dz3.sum(axis=0)
    dz2 = (dz3 @ p["W3"]) * (1.0 - h2 * h2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (1.0 - h1 * h1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return pack(g)


def adam_step(theta, m, v, g, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma and Ba, 2015) at step t >= 1, with the bias
    corrections 1 - beta^t.  Returns the new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(uniform01: np.ndarray) -> np.ndarray:
    """Glorot-uniform weights from given uniform numbers in [0, 1) (one per
    parameter, in the flat order); biases zero.  A layer with fan-in a and
    fan-out c draws from U(-s, s), s = sqrt(6 / (a + c))."""
    u = np.asarray(uniform01, dtype=np.float64)
    assert u.size == NPARAM
    theta = np.zeros(NPARAM)
    o = 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        if name.startswith("W") or name == "w4":
            fan_out, fan_in = (shp[0], shp[1]) if len(shp) == 2 else (1, shp[0])
            s = np.sqrt(6.0 / (fan_in + fan_out))
            theta[o:o + n] = (2.0 * u[o:o + n] - 1.0) * s
        o += n
    return theta

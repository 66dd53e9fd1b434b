"""FP64 forward / backward of the selectivity-surrogate MLP -- TEST INFRASTRUCTURE.

The surrogate is not in the paper (it is this project's learned estimator,
evaluated against exact selectivity computation).  Network: x (64) -> W1 x + b1 ->
ReLU -> W2 h1 + b2 -> ReLU -> w3 . h2 + b3 = y (the predicted log10
selectivity); loss = mean over the batch of (y - t)^2.

The flat parameter vector is laid out as W1 (rows of 64), b1, W2 (rows of
128), b2, w3, b3 -- the same order the CUDA library uses.  The oracle takes
the weights and inputs exactly as the device sees them (already rounded to
bfloat16 by the caller) and computes in float64.

Pins (tests/test_mlp_oracle_pins.py): central finite differences of the
loss, a closed form for one hidden unit per layer, and the reduction to a
linear model when every pre-activation is positive.
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np


def sizes(d_in: int = 64, h1: int = 128, h2: int = 128) -> Dict[str, Tuple[int, ...]]:
    return {"W1": (h1, d_in), "b1": (h1,), "W2": (h2, h1), "b2": (h2,), "w3": (h2,), "b3": (1,)}


def unflatten(p: np.ndarray, d_in: int = 64, h1: int = 128, h2: int = 128) -> Dict[str, np.ndarray]:
    out, o = {}, 0
    for k, shp in sizes(d_in, h1, h2).items():
        n = int(np.prod(shp))
        out[k] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    assert o == len(p)
    return out


def flatten(params: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(params[k], dtype=np.float64).ravel() for k in ("W1", "b1", "W2", "b2", "w3", "b3")])


def forward(p: np.ndarray, x: np.ndarray, d_in: int = 64, h1: int = 128, h2: int = 128):
    """Returns (y, cache) for x of shape (B, d_in)."""
    P = unflatten(p, d_in, h1, h2)
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ P["W1"].T + P["b1"]
    z1 = np.maximum(a1, 0.0)
    a2 = z1 @ P["W2"].T + P["b2"]
    z2 = np.maximum(a2, 0.0)
    y = z2 @ P["w3"] + P["b3"][0]
    return y, (x, a1, z1, a2, z2, P)


def loss(p: np.ndarray, x: np.ndarray, t: np.ndarray, **kw) -> float:
    y, _ = forward(p, x, **kw)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def grad(p: np.ndarray, x: np.ndarray, t: np.ndarray, d_in: int = 64, h1: int = 128, h2: int = 128):
    """(loss, gradient of the loss with respect to the flat parameters)."""
    y, (x, a1, z1, a2, z2, P) = forward(p, x, d_in, h1, h2)
    t = np.asarray(t, dtype=np.float64)
    B = x.shape[0]
    dy = 2.0 * (y - t) / B                      # d loss / d y
    g = {"w3": z2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, P["w3"])
    da2 = dz2 * (a2 > 0)
    g["W2"] = da2.T @ z1
    g["b2"] = da2.sum(axis=0)
    dz1 = da2 @ P["W2"]
    da1 = dz1 * (a1 > 0)
    g["W1"] = da1.T @ x
    g["b1"] = da1.sum(axis=0)
    return float(np.mean((y - t) ** 2)), flatten(g)


def round_bf16(a: np.ndarray) -> np.ndarray:
    """Float32 values rounded to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)

"""FP64 oracle of the learned operator generator.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The learned-operator
extension replaces the table lookup of Sec. III by a small network that maps
the normalised wavenumber x = k / k_max to the L+1 symmetric complex taps of
Eq. 1 (interleaved Re, Im), trained on operators of the least-squares design.

Network: 1 -> H -> H -> H -> 2(L+1) reals, GELU (erf form) after each hidden
layer, no activation on the output:
    a1 = W1 x + b1,  h1 = gelu(a1)
    a2 = W2 h1 + b2, h2 = gelu(a2)
    a3 = W3 h2 + b3, h3 = gelu(a3)
    y  = W4 h3 + b4
Loss: mean over samples and outputs of (y - t)^2.  Weights are stored as
W[out][in].  Optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


def shapes(hidden: int = 64, n_out: int = 26) -> dict:
    return {"W1": (hidden, 1), "b1": (hidden,), "W2": (hidden, hidden), "b2": (hidden,),
            "W3": (hidden, hidden), "b3": (hidden,), "W4": (n_out, hidden), "b4": (n_out,)}


def flatten(p: dict) -> np.ndarray:
    """Parameters packed in PARAM_ORDER, each row-major."""
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in PARAM_ORDER])


def unflatten(v: np.ndarray, hidden: int = 64, n_out: int = 26) -> dict:
    out, o = {}, 0
    for k in PARAM_ORDER:
        shp = shapes(hidden, n_out)[k]
        n = int(np.prod(shp))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def gelu(a):
    return 0.5 * a * (1.0 + erf(a / math.sqrt(2.0)))


def gelu_grad(a):
    return 0.5 * (1.0 + erf(a / math.sqrt(2.0))) + a * np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)


def forward(p: dict, x: np.ndarray):
    """y [n][n_out] and the cache of pre-activations / activations."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 1)
    a1 = x @ p["W1"].T + p["b1"]
    h1 = gelu(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(a2)
    a3 = h2 @ p["W3"].T + p["b3"]
    h3 = gelu(a3)
    y = h3 @ p["W4"].T + p["b4"]
    return y, {"x": x, "a1": a1, "h1": h1, "a2": a2, "h2": h2, "a3": a3, "h3": h3}


def loss(y: np.ndarray, t: np.ndarray) -> float:
    d = y - t
    return float(np.mean(d * d))


def backward(p: dict, cache: dict, y: np.ndarray, t: np.ndarray) -> dict:
    """Gradients of the mean squared error with respect to every parameter."""
    n = y.shape[0]
    dy = 2.0 * (y - t) / (n * y.shape[1])
    g = {"W4": dy.T @ cache["h3"], "b4": dy.sum(axis=0)}
    da3 = (dy @ p["W4"]) * gelu_grad(cache["a3"])
    g["W3"], g["b3"] = da3.T @ cache["h2"], da3.sum(axis=0)
    da2 = (da3 @ p["W3"]) * gelu_grad(cache["a2"])
    g["W2"], g["b2"] = da2.T @ cache["h1"], da2.sum(axis=0)
    da1 = (da2 @ p["W2"]) * gelu_grad(cache["a1"])
    g["W1"], g["b1"] = da1.T @ cache["x"], da1.sum(axis=0)
    return g


def adam_step(v: np.ndarray, grad: np.ndarray, m: np.ndarray, s: np.ndarray, step: int, lr: float,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update of the flat parameter vector (step counts from 1)."""
    m = b1 * m + (1 - b1) * grad
    s = b2 * s + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    sh = s / (1 - b2 ** step)
    return v - lr * mh / (np.sqrt(sh) + eps), m, s


def taps_from_output(y: np.ndarray) -> np.ndarray:
    """[n][2(L+1)] interleaved (Re, Im) -> [n][L+1] complex taps."""
    return y[:, 0::2] + 1j * y[:, 1::2]


def taps_at(v: np.ndarray, k, k_max: float, L: int, hidden: int = 64) -> np.ndarray:
    """Operators generated by the network with flat parameters v at the
    wavenumbers k: input x = k / k_max clipped to [0, 1] (the domain the
    network is trained on); [n][L+1] complex128."""
    x = np.clip(np.asarray(k, dtype=np.float64) / k_max, 0.0, 1.0)
    y, _ = forward(unflatten(v, hidden, 2 * (L + 1)), x)
    return taps_from_output(y)


def taps_fn(v: np.ndarray, k_max: float, L: int, hidden: int = 64):
    """``taps_at`` as the operator generator of ``oracle.migrate_pointwise``
    (pairs of frequency w and slowness s, k = w s)."""
    def fn(wp, sp):
        k = np.asarray(wp, dtype=np.float64) * np.asarray(sp, dtype=np.float32).astype(np.float64)
        ku, inv = np.unique(k, return_inverse=True)
        return taps_at(v, ku, k_max, L, hidden)[inv.ravel()]
    return fn

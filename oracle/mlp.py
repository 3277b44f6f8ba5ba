"""FP64 CPU oracle for the learned warm start: a per-node MLP that predicts the scaled dual
ybar^i of a scenario-tree node from the node's data, trained with Adam on a mean squared error.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the benchmark's
CPU-baseline leg, never by the library.  It shares no code with the CUDA path.

The paper warm-starts its solvers from a few iterations of an accelerated dual gradient method
(Section III-F); the learned predictor is the batched workload's alternative to that.  What it
computes:

* features of node i of one draw (x0, c): [x0 (nx), t/N (1), c^i, c^anc(i), c^anc(anc(i))],
  where missing ancestors, and the root's c, are zeros; nx + 1 + 3 nx inputs;
* a three-layer perceptron in -> H -> H -> nx + nu with the tanh form of the Gaussian error
  linear unit [Hendrycks and Gimpel 2016],
      gelu(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))),
  on both hidden layers and a linear output;
* the loss: the mean over the valid outputs (nx + nu at nonleaf nodes, nx at leaves) of the
  squared difference to the target ybar^i;
* gradients by the chain rule, written out layer by layer;
* Adam [Kingma and Ba 2015] with bias correction.

With ``bf16=True`` every tensor that the GPU path keeps in BF16 between its products (inputs,
weights, hidden activations, output gradients) is rounded to BF16 (round to nearest even)
at the same place, and all arithmetic stays FP64; this models the storage precision of the
tensor-core path without modelling its accumulation order.
"""
from __future__ import annotations

import math

import numpy as np

GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def bf16_round(a) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as FP64.  The value is first
    rounded to FP32 (BF16 is the upper half of an FP32 word)."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def gelu(z):
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    """d gelu / dz, by the product and chain rules."""
    z = np.asarray(z, dtype=np.float64)
    th = np.tanh(GELU_C * (z + GELU_A * z ** 3))
    return 0.5 * (1.0 + th) + 0.5 * z * (1.0 - th * th) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)


def node_features(parent: np.ndarray, stage: np.ndarray, horizon: int, x0: np.ndarray, c: np.ndarray,
                  nodes=None) -> np.ndarray:
    """Feature rows for the given nodes of one draw (all nodes if None).  c is [num_nodes][nx]
    with c[0] = 0."""
    nx = x0.shape[0]
    nodes = np.arange(len(parent)) if nodes is None else np.asarray(nodes)
    out = np.zeros((len(nodes), 4 * nx + 1))
    for r, i in enumerate(nodes):
        out[r, :nx] = x0
        out[r, nx] = stage[i] / horizon
        j = int(i)
        for a in range(3):
            if j < 0:
                break
            if j > 0:
                out[r, nx + 1 + a * nx: nx + 1 + (a + 1) * nx] = c[j]
            j = int(parent[j])
    return out


def init_params(rng: np.random.Generator, d_in: int, hidden: int, d_out: int) -> dict:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases."""
    def lin(fi, fo):
        s = 1.0 / math.sqrt(fi)
        return rng.uniform(-s, s, size=(fo, fi)), rng.uniform(-s, s, size=fo)
    W1, b1 = lin(d_in, hidden)
    W2, b2 = lin(hidden, hidden)
    W3, b3 = lin(hidden, d_out)
    return {"W1": W1, "b1": b1, "W2": W2, "b2": b2, "W3": W3, "b3": b3}


def _r(a, bf16):
    return bf16_round(a) if bf16 else np.asarray(a, dtype=np.float64)


def forward(params: dict, X: np.ndarray, bf16: bool = False) -> dict:
    """Layer by layer; returns every intermediate for the backward pass."""
    W1, W2, W3 = (_r(params[k], bf16) for k in ("W1", "W2", "W3"))
    X = _r(X, bf16)
    Z1 = X @ W1.T + params["b1"]
    A1 = _r(gelu(Z1), bf16)
    Z2 = A1 @ W2.T + params["b2"]
    A2 = _r(gelu(Z2), bf16)
    Y = A2 @ W3.T + params["b3"]
    return {"X": X, "W1": W1, "W2": W2, "W3": W3, "Z1": Z1, "A1": A1, "Z2": Z2, "A2": A2, "Y": Y}


def loss_and_grads(params: dict, X: np.ndarray, T: np.ndarray, nvalid: np.ndarray, bf16: bool = False):
    """Mean squared error over the valid outputs (the first nvalid[b] of row b) and its gradient
    with respect to every parameter."""
    f = forward(params, X, bf16)
    d_out = T.shape[1]
    mask = (np.arange(d_out)[None, :] < np.asarray(nvalid)[:, None]).astype(np.float64)
    count = mask.sum()
    diff = (f["Y"] - T) * mask
    loss = float((diff ** 2).sum() / count)
    dY = _r(2.0 * diff / count, bf16)
    g = {"W3": dY.T @ f["A2"], "b3": dY.sum(axis=0)}
    dA2 = dY @ f["W3"]
    dZ2 = _r(dA2 * gelu_grad(f["Z2"]), bf16)
    g["W2"] = dZ2.T @ f["A1"]
    g["b2"] = dZ2.sum(axis=0)
    dA1 = dZ2 @ f["W2"]
    dZ1 = _r(dA1 * gelu_grad(f["Z1"]), bf16)
    g["W1"] = dZ1.T @ f["X"]
    g["b1"] = dZ1.sum(axis=0)
    return loss, g, f


def adam_init(params: dict) -> dict:
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in params.items()},
            "v": {k: np.zeros_like(v) for k, v in params.items()}}


def adam_step(params: dict, grads: dict, state: dict, lr: float = 1e-3, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8) -> None:
    """In place: first and second moment estimates, bias-corrected, then the step."""
    state["t"] += 1
    t = state["t"]
    for k in params:
        m = state["m"][k] = beta1 * state["m"][k] + (1.0 - beta1) * grads[k]
        v = state["v"][k] = beta2 * state["v"][k] + (1.0 - beta2) * grads[k] ** 2
        mh = m / (1.0 - beta1 ** t)
        vh = v / (1.0 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)

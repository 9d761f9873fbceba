"""Scorer network of the learned operator proposal (test infrastructure,
oracle).  The paper selects the operator with the largest exact pool gradient
(Sec. IV.B, Eq. 12); the learned proposal only ranks the pool so that fewer
operators need an exact gradient.  Its network is defined here in float64:

    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  s = w3 . h2 + b3,

x in R^32, 256 hidden units, with every weight and bias rounded to bfloat16
(round to nearest, ties to even) before use.  Gradients are with respect to
those rounded values (they are passed straight to the fp32 master copies).

The loss of one ranking list is the softmax cross-entropy against a target
distribution p:  loss = -sum_k p_k log softmax(s)_k, with d loss / d s =
softmax(s) - p.  Adam (Kingma and Ba, 2015, Algorithm 1) with beta1 = 0.9,
beta2 = 0.999, eps = 1e-8 and bias correction updates the master copies.

Parameter order (74,497 values): W1[256][32], b1[256], W2[256][256], b2[256],
w3[256], b3.
"""
from __future__ import annotations

import numpy as np

F, H = 32, 256
SHAPES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", ())]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as
    float64.  bfloat16 keeps the top 16 bits of the float32 pattern."""
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def unpack(P):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(P[o:o + n]).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def forward(P, X, rounded=True):
    """Scores of the rows of X (rows x 32) and the activations the backward
    pass needs.  rounded=False uses the weights as given (for finite
    differences)."""
    w = unpack(bf16_round(P) if rounded else np.asarray(P, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(z2, 0.0)
    s = h2 @ w["w3"] + w["b3"]
    return s, dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2, w=w)


def backward(cache, ds):
    """Gradient of sum_r ds[r] s_r with respect to every parameter (chain rule,
    relu'(z) = [z > 0])."""
    w, X, h1, h2 = cache["w"], cache["X"], cache["h1"], cache["h2"]
    ds = np.asarray(ds, dtype=np.float64)
    g = {"w3": h2.T @ ds, "b3": ds.sum()}
    d2 = np.outer(ds, w["w3"]) * (cache["z2"] > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ w["W2"]) * (cache["z1"] > 0)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return pack(g)


def listwise_loss(s, p):
    """Softmax cross-entropy of one list and its gradient."""
    s = np.asarray(s, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    if s.size == 0:
        return 0.0, s.copy()
    m = s.max()
    lse = m + np.log(np.exp(s - m).sum())
    return float(-(p * (s - lse)).sum()), np.exp(s - lse) - p


class Adam:
    """Algorithm 1 of Kingma and Ba with the bias-corrected step."""

    def __init__(self, n, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.t = 0

    def step(self, P, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return P - self.lr * mh / (np.sqrt(vh) + self.eps)

"""The learned excitation proposal, written out plainly in FP64 numpy --
TEST INFRASTRUCTURE ONLY (tests/ may import it; the GPU path never does).

The paper has no learned part: its UEG and molecular excitation generators are
uniform or heat-bath (Sec. 2.1, Sec. 4).  The learned proposal replaces the
uniform choice of the particle orbital A of a UEG double excitation
(i, j) -> (a, b), b fixed by momentum conservation, by a table of integer
weights per row r = (I, J, same spin) that a small MLP produces:

  features x(r) = [one-hot(I) (M), one-hot(J) (M), same spin (1)]   (2M + 1)
  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3        (width H)
  p(A | r) = exp(z_A) / sum_{A' drawable} exp(z_A')  over drawable A
  q_r(A) = max(1, floor(p(A | r) 2^24)) on drawable A, 0 elsewhere.

Training (on the spawning attempts the run itself draws): sample n drew A_n in
row r_n with probability p_n under the current table and has matrix element
H_n; with c_n = (|H_n| / p_n) / sum_m (|H_m| / p_m),
  L = - sum_n c_n log p(A_n | r_n)
is a self-normalised estimate of the cross-entropy to the distribution
proportional to |H| (the heat-bath choice, which minimises the variance of the
spawned weight tau |H| / p_gen).

`bf16=True` mirrors the points where the tensor-core kernels round to BF16:
the weights, the hidden activations h1 and h2, and the backward signals
dz (logits), dz2, dz1 that enter the GEMMs; everything else is FP64 here.
"""
from __future__ import annotations

import numpy as np


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    return out.reshape(a.shape)


def features(rows, M: int) -> np.ndarray:
    """x(r) for row indices r = (I M + J) 2 + same."""
    rows = np.asarray(rows, dtype=np.int64)
    same = rows & 1
    IJ = rows >> 1
    I, J = IJ // M, IJ % M
    X = np.zeros((len(rows), 2 * M + 1))
    X[np.arange(len(rows)), I] = 1.0
    X[np.arange(len(rows)), M + J] = 1.0
    X[:, 2 * M] = same
    return X


def init_params(M: int, width: int, seed: int):
    """Seeded initial weights: uniform(+-sqrt(6 / fan_in)) (He), zero biases."""
    rng = np.random.Generator(np.random.Philox(seed))
    d = 2 * M + 1
    lim = lambda fan: np.sqrt(6.0 / fan)
    return {"W1": rng.uniform(-lim(d), lim(d), (width, d)), "b1": np.zeros(width),
            "W2": rng.uniform(-lim(width), lim(width), (width, width)), "b2": np.zeros(width),
            "W3": rng.uniform(-lim(width), lim(width), (M, width)), "b3": np.zeros(M)}


def forward(params, X, mask, bf=False):
    """Logits z and the masked softmax p (rows of `mask` give the drawable A)."""
    r = bf16 if bf else (lambda v: v)
    z1 = X @ r(params["W1"]).T + params["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ r(params["W2"]).T + params["b2"]
    h2 = r(np.maximum(z2, 0.0))
    z = h2 @ r(params["W3"]).T + params["b3"]
    zm = np.where(mask, z, -np.inf)
    zmax = np.max(zm, axis=1, keepdims=True)
    zmax = np.where(np.isfinite(zmax), zmax, 0.0)          # rows with nothing drawable
    e = np.where(mask, np.exp(np.where(mask, z - zmax, 0.0)), 0.0)
    tot = e.sum(axis=1, keepdims=True)
    p = e / np.where(tot > 0.0, tot, 1.0)
    return {"z1": z1, "h1": h1, "z2": z2, "h2": h2, "z": z, "p": p}


def loss_and_grads(params, X, mask, target, weight, bf=False):
    """L = -sum_n c_n log p(target_n) with c = weight / sum(weight), and its
    gradients with respect to every parameter (same keys as params)."""
    r = bf16 if bf else (lambda v: v)
    f = forward(params, X, mask, bf)
    n = X.shape[0]
    c = np.asarray(weight, dtype=np.float64)
    c = c / c.sum()
    p = f["p"]
    loss = -float(np.sum(c * np.log(p[np.arange(n), target])))
    onehot = np.zeros_like(p)
    onehot[np.arange(n), target] = 1.0
    dz = r(c[:, None] * (p - onehot) * mask)
    g = {"W3": dz.T @ f["h2"], "b3": dz.sum(axis=0)}
    dh2 = dz @ r(params["W3"])
    dz2 = r(dh2 * (f["z2"] > 0.0))
    g["W2"] = dz2.T @ f["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ r(params["W2"])
    dz1 = r(dh1 * (f["z1"] > 0.0))
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def table_from_probabilities(p, mask) -> np.ndarray:
    """Integer weights q = max(1, floor(p 2^24)) on drawable entries, 0 elsewhere."""
    q = np.floor(np.asarray(p) * float(1 << 24))
    q = np.maximum(q, 1.0)
    return np.where(mask, q, 0.0).astype(np.uint32)

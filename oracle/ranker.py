"""Oracle of the learned representative ranker, float64 (TEST INFRASTRUCTURE ONLY).

The paper has no learned component; this network is the part of the build that orders and
prunes representative comparisons.  It is written here from its definition:

  X0 = E[code] (20 x 32);  Z1 = relu(conv9(X0, W1) + b1);  Z2 = relu(conv9(Z1, W2) + b2);
  Z3 = conv9(Z2, W3) + b3;  v = mean over rows of Z3 (0 for an empty sequence);
  logit(a, b) = alpha * cos(v_a, v_b) + beta,
      cos(a, b) = <a, b> / sqrt((|a|^2 + 1e-6)(|b|^2 + 1e-6));  loss = mean BCE(sigmoid(logit), y)

conv9(X, W)[r] = sum_{k=0..8} X[r + k - 4] @ W[k] with zero rows outside the sequence
("same" padding, every sequence on its own).  The forward is plain numpy; the gradient uses
torch autograd in float64 on the same formula, and tests pin it by central finite differences
computed with the numpy forward.
"""
from __future__ import annotations

import numpy as np

EMB, CH, TAPS = 32, 128, 9
SHAPES = [("E", (20, EMB)), ("W1", (TAPS, EMB, CH)), ("b1", (CH,)), ("W2", (TAPS, CH, CH)),
          ("b2", (CH,)), ("W3", (TAPS, CH, CH)), ("b3", (CH,)), ("alpha", ()), ("beta", ())]


def num_params():
    return int(sum(int(np.prod(s)) for _, s in SHAPES))


def unpack(flat):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = flat[o:o + n].reshape(shp)
        o += n
    return out


def conv9(X, W):
    L = X.shape[0]
    Xp = np.zeros((L + 8, X.shape[1]), dtype=np.float64)
    Xp[4:4 + L] = X
    Y = np.zeros((L, W.shape[2]), dtype=np.float64)
    for k in range(TAPS):
        Y += Xp[k:k + L] @ W[k]
    return Y


def embed_one(codes, p):
    codes = np.asarray(codes, dtype=np.int64)
    if len(codes) == 0:
        return np.zeros(CH, dtype=np.float64)
    X0 = p["E"][codes]
    Z1 = np.maximum(conv9(X0, p["W1"]) + p["b1"], 0.0)
    Z2 = np.maximum(conv9(Z1, p["W2"]) + p["b2"], 0.0)
    Z3 = conv9(Z2, p["W3"]) + p["b3"]
    return Z3.mean(axis=0)


def embed(seqs, offsets, params, ids=None):
    p = unpack(np.asarray(params, dtype=np.float64))
    ids = range(len(offsets) - 1) if ids is None else ids
    return np.stack([embed_one(seqs[offsets[i]:offsets[i + 1]], p) for i in ids])


def logits(seqs, offsets, params, pairs):
    p = unpack(np.asarray(params, dtype=np.float64))
    pairs = np.asarray(pairs).reshape(-1, 2)
    ids = np.unique(pairs)
    V = dict(zip(ids.tolist(), embed(seqs, offsets, params, ids)))
    return np.array([float(p["alpha"]) * cosine(V[a], V[b]) + float(p["beta"]) for a, b in pairs])


COS_EPS = 1e-6


def cosine(a, b):
    return float(a @ b / np.sqrt((a @ a + COS_EPS) * (b @ b + COS_EPS)))


def loss(seqs, offsets, params, pairs, labels):
    z = logits(seqs, offsets, params, pairs)
    y = np.asarray(labels, dtype=np.float64)
    return float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def loss_grad(seqs, offsets, params, pairs, labels):
    """(loss, gradient) in float64 via torch autograd on the same definition."""
    import torch
    flat = torch.tensor(np.asarray(params, dtype=np.float64), requires_grad=True)
    o, P = 0, {}
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        P[name] = flat[o:o + n].reshape(shp)
        o += n
    pairs = np.asarray(pairs).reshape(-1, 2)
    ids = np.unique(pairs)
    V = {}
    for i in ids.tolist():
        codes = torch.tensor(np.asarray(seqs[offsets[i]:offsets[i + 1]], dtype=np.int64))
        L = len(codes)
        if L == 0:
            V[i] = torch.zeros(CH, dtype=torch.float64)
            continue
        h = P["E"][codes]
        for W, b, relu in ((P["W1"], P["b1"], True), (P["W2"], P["b2"], True),
                           (P["W3"], P["b3"], False)):
            hp = torch.nn.functional.pad(h, (0, 0, 4, 4))
            y = sum(hp[k:k + L] @ W[k] for k in range(TAPS)) + b
            h = torch.relu(y) if relu else y
        V[i] = h.mean(dim=0)
    z = torch.stack([P["alpha"] * (V[a] @ V[b]) /
                     torch.sqrt((V[a] @ V[a] + COS_EPS) * (V[b] @ V[b] + COS_EPS)) + P["beta"]
                     for a, b in pairs.tolist()])
    y = torch.tensor(np.asarray(labels, dtype=np.float64))
    lo = torch.nn.functional.binary_cross_entropy_with_logits(z, y)
    lo.backward()
    return float(lo.item()), flat.grad.numpy().copy()


def init_params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in SHAPES:
        if name == "E":
            parts.append(rng.normal(0, 1.0, shp))
        elif name.startswith("W"):
            fan = shp[0] * shp[1]
            parts.append(rng.normal(0, np.sqrt(2.0 / fan) * scale, shp))
        elif name == "alpha":
            parts.append(np.array([10.0]))
        elif name == "beta":
            parts.append(np.array([-2.0]))
        else:
            parts.append(rng.normal(0, 0.05, shp))
    return np.concatenate([np.ravel(x) for x in parts])

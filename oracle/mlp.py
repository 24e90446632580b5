"""CPU reference of the warm-start network (an extension of the method; the paper has no
learned component).  TEST INFRASTRUCTURE ONLY, like the rest of oracle/.

Y = relu(relu(X W1' + b1) W2' + b2) W3' + b3, loss L = sum (Y - T)^2 / (2 rows n_out),
in float64.  With bf16=True the operands of every product are rounded to bfloat16 at
the same points as the GPU network (X, W1..W3, the hidden activations and the
backpropagated signals that feed products); with bf16=False it is the plain network,
which the tests pin with finite differences.
"""
from __future__ import annotations

import numpy as np


def bf16(a):
    """Round to the nearest bfloat16 (ties to even) and return float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def forward(params, X, use_bf16=True):
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, dtype=np.float64) for p in params]
    rd = bf16 if use_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    Xb = rd(X)
    H1 = np.maximum(Xb @ rd(W1).T + b1, 0.0)
    H1b = rd(H1)
    H2 = np.maximum(H1b @ rd(W2).T + b2, 0.0)
    H2b = rd(H2)
    Y = H2b @ rd(W3).T + b3
    return dict(Xb=Xb, H1=H1, H1b=H1b, H2=H2, H2b=H2b, Y=Y)


def loss_and_grads(params, X, T, use_bf16=True):
    """Loss and gradients (gW1, gb1, gW2, gb2, gW3, gb3) of L at params on (X, T)."""
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, dtype=np.float64) for p in params]
    rd = bf16 if use_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    f = forward(params, X, use_bf16)
    R, O = np.asarray(T).shape
    E = f["Y"] - np.asarray(T, dtype=np.float64)
    loss = float(np.sum(E * E) / (2.0 * R * O))
    dY = E / (R * O)
    dYb = rd(dY)
    gW3 = dYb.T @ f["H2b"]
    gb3 = dY.sum(axis=0)
    dZ2 = (dYb @ rd(W3)) * (f["H2"] > 0)
    dZ2b = rd(dZ2)
    gW2 = dZ2b.T @ f["H1b"]
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2b @ rd(W2)) * (f["H1"] > 0)
    dZ1b = rd(dZ1)
    gW1 = dZ1b.T @ f["Xb"]
    gb1 = dZ1.sum(axis=0)
    return loss, [gW1, gb1, gW2, gb2, gW3, gb3]


def init_params(n_in, hidden, n_out, seed=0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases, float32."""
    rng = np.random.default_rng(seed)
    out = []
    for fi, fo in ((n_in, hidden), (hidden, hidden), (hidden, n_out)):
        a = 1.0 / np.sqrt(fi)
        out.append(rng.uniform(-a, a, (fo, fi)).astype(np.float32))
        out.append(rng.uniform(-a, a, fo).astype(np.float32))
    return out

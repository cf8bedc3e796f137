"""FP64 reference of the level-of-detail network (numpy).

TEST INFRASTRUCTURE: see the package docstring.

Model: y = w3 . relu(relu(x W1 + b1) W2 + b2) + b3, x in R^8, hidden 64;
loss = mean over rows of w (y - t)^2, w = `under` where y < t, else 1.  Parameters in one vector:
W1 [8][64] | b1 [64] | W2 [64][64] | b2 [64] | w3 [64] | b3 (4801 values).
The gradient is plain reverse-mode differentiation written out layer by
layer (the chain rule, nothing fused).
"""
import numpy as np

NPARAMS = 8 * 64 + 64 + 64 * 64 + 64 + 64 + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + 512].reshape(8, 64); o += 512
    b1 = p[o:o + 64]; o += 64
    W2 = p[o:o + 4096].reshape(64, 64); o += 4096
    b2 = p[o:o + 64]; o += 64
    w3 = p[o:o + 64]; o += 64
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def forward(p, x):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    return h2 @ w3 + b3


def loss_and_grad(p, x, t, under=1.0):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    n = x.shape[0]
    a1 = x @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    e = y - t
    w = np.where(e < 0, under, 1.0)
    loss = float(np.mean(w * e * e))
    dy = 2.0 * w * e / n                   # d loss / d y
    gb3 = dy.sum()
    gw3 = h2.T @ dy
    dh2 = np.outer(dy, w3) * (a2 > 0)      # through the second ReLU
    gb2 = dh2.sum(axis=0)
    gW2 = h1.T @ dh2
    dh1 = (dh2 @ W2.T) * (a1 > 0)          # through the first ReLU
    gb1 = dh1.sum(axis=0)
    gW1 = x.T @ dh1
    return loss, pack(gW1, gb1, gW2, gb2, gw3, gb3)


def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (ties to even), as floats."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)

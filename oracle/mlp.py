"""FP64 reference of the learned-initialisation MLP -- TEST INFRASTRUCTURE ONLY.

Plain numpy forward and backward of the 32 -> 128 -> 128 -> r ReLU network with
mean-squared-error loss, in the parameter layout of the library
(W1 [32x128] | W2 [128x128] | W3 [128xr] | b1 | b2 | b3), and the row sketch
(nearest-rank quantiles of the given entries, centred on the median).  The
network's weights are used as given (the tests round them to BF16 first when
they compare with the library, whose forward pass reads BF16 weights).
Pinned by finite differences in tests/test_oracle_mlp.py.
"""
import numpy as np

SK, HID = 32, 128


def split(params, r):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + SK * HID].reshape(SK, HID); o += SK * HID
    W2 = p[o:o + HID * HID].reshape(HID, HID); o += HID * HID
    W3 = p[o:o + HID * r].reshape(HID, r); o += HID * r
    b1 = p[o:o + HID]; o += HID
    b2 = p[o:o + HID]; o += HID
    b3 = p[o:o + r]; o += r
    assert o == p.size
    return W1, W2, W3, b1, b2, b3


def forward(params, X, r):
    W1, W2, W3, b1, b2, b3 = split(params, r)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    return h2 @ W3 + b3, (X, h1, h2)


def loss_and_grad(params, X, T, r):
    """MSE = mean over batch and outputs of (Y - T)^2, and its gradient."""
    W1, W2, W3, b1, b2, b3 = split(params, r)
    Y, (X, h1, h2) = forward(params, X, r)
    T = np.asarray(T, dtype=np.float64)
    B = X.shape[0]
    d = Y - T
    loss = float(np.sum(d * d) / (B * r))
    dY = 2.0 * d / (B * r)
    gW3 = h2.T @ dY; gb3 = dY.sum(axis=0)
    dH2 = (dY @ W3.T) * (h2 > 0)
    gW2 = h1.T @ dH2; gb2 = dH2.sum(axis=0)
    dH1 = (dH2 @ W2.T) * (h1 > 0)
    gW1 = X.T @ dH1; gb1 = dH1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gW2.ravel(), gW3.ravel(), gb1, gb2, gb3])
    return loss, grad


def row_sketch(R, M):
    """(sketch m x 32, median m): nearest-rank quantiles of each row's given entries."""
    R = np.asarray(R, dtype=np.float64)
    m = R.shape[0]
    sk = np.zeros((m, SK)); med = np.zeros(m)
    for s in range(m):
        v = np.sort(R[s][np.asarray(M[s], dtype=bool)])
        c = v.size
        if c == 0:
            continue
        md = v[c // 2]
        idx = np.minimum(((np.arange(SK) + 0.5) * c / SK).astype(np.int64), c - 1)
        sk[s] = v[idx] - md
        med[s] = md
    return sk, med

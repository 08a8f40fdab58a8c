"""FP64 reference of the learned-initialisation MLP -- TEST INFRASTRUCTURE ONLY.

Plain numpy forward and backward of the 32 -> 128 -> 128 -> r ReLU network with
mean-squared-error loss, in the parameter layout of the library
(W1 [32x128] | W2 [128x128] | W3 [128xr] | b1 | b2 | b3), and the row sketch
(nearest-rank quantiles of the given entries, centred on the median).  The
network's weights are used as given (the tests round them to BF16 first when
they compare with the library, whose forward pass reads BF16 weights); with
bf16_operands=True every operand of a matrix product is rounded to BF16 as in
the library's tensor-core kernels.
Also the gauge-fixed training targets and the hand-over of predicted values
by rank (plain loops, FP32 arithmetic as stated per function).
Pinned by finite differences, gauge invariance and brute force in
tests/test_oracle_mlp.py.
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


def bf16(x):
    """x rounded to FP32, then to bfloat16 (round to nearest, ties to even),
    returned as float64: the rounding of an FP32 value that becomes a BF16
    operand of a matrix product."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, X, r, bf16_operands=False):
    """bf16_operands: round every operand of the three products to BF16 (the
    weights are expected to be BF16 already), as the library's kernels do;
    products, sums, biases and ReLU stay in FP64."""
    q = bf16 if bf16_operands else (lambda a: a)
    W1, W2, W3, b1, b2, b3 = split(params, r)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(q(X) @ W1 + b1, 0.0)
    h2 = np.maximum(q(h1) @ W2 + b2, 0.0)
    return q(h2) @ W3 + b3, (X, h1, h2)


def loss_and_grad(params, X, T, r, bf16_operands=False):
    """MSE = mean over batch and outputs of (Y - T)^2, and its gradient.
    bf16_operands: every operand of the products of the forward and backward
    passes rounded to BF16, as in the library's kernels."""
    q = bf16 if bf16_operands else (lambda a: a)
    W1, W2, W3, b1, b2, b3 = split(params, r)
    Y, (X, h1, h2) = forward(params, X, r, bf16_operands)
    T = np.asarray(T, dtype=np.float64)
    B = X.shape[0]
    d = Y - T
    loss = float(np.sum(d * d) / (B * r))
    dY = 2.0 * d / (B * r)
    gW3 = q(h2).T @ q(dY); gb3 = dY.sum(axis=0)
    dH2 = (q(dY) @ W3.T) * (h2 > 0)
    gW2 = q(h1).T @ q(dH2); gb2 = dH2.sum(axis=0)
    dH1 = (q(dH2) @ W2.T) * (h1 > 0)
    gW1 = q(X).T @ q(dH1); gb1 = dH1.sum(axis=0)
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


def targets(U, V, med, sorted_rows=False):
    """Training targets of the learned start from a factorization (U m x r,
    V r x n, med m), in FP32 arithmetic like the library.  U (x) V is
    unchanged by U_.l + c, V_l. - c and by any order of the components; the
    gauge is fixed by c_l = max_t V_lt and by ordering the components by
    decreasing sum over rows of x_sl = fl32(U_sl + c_l), the sum in FP64 with
    rows in index order (equal sums: the smaller l first).  canonical:
    T[s, p] = fl32(x[s, l_p] - med_s); sorted_rows: row s's x values in
    decreasing order, minus med_s."""
    U = np.asarray(U, dtype=np.float32)
    V = np.asarray(V, dtype=np.float32)
    med = np.asarray(med, dtype=np.float32)
    m, r = U.shape
    c = V.max(axis=1)
    x = (U + c[None, :]).astype(np.float32)
    key = np.zeros(r)
    for l in range(r):
        acc = 0.0
        for s in range(m):
            acc += float(x[s, l])
        key[l] = acc
    order = sorted(range(r), key=lambda l: (-key[l], l))
    if sorted_rows:
        y = -np.sort(-x, axis=1)
    else:
        y = x[:, order]
    return (y - med[:, None]).astype(np.float32)


def assign_by_rank(Y, U_ref):
    """out[s, l] = the value of Y[s] whose rank in its row (decreasing) equals
    the rank of U_ref[s, l] in its row (decreasing; equal values: the smaller
    index first)."""
    Y = np.asarray(Y, dtype=np.float32)
    U_ref = np.asarray(U_ref, dtype=np.float32)
    out = np.empty_like(Y)
    for s in range(Y.shape[0]):
        vals = sorted(Y[s].tolist(), reverse=True)
        order = sorted(range(Y.shape[1]), key=lambda l: (-float(U_ref[s, l]), l))
        for p, l in enumerate(order):
            out[s, l] = vals[p]
    return out

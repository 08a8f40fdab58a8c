"""Learned initialisation of U for FastSTMF (an addition to the paper, which
initialises with Random Acol; Random Acol stays the fallback).

Pipeline (every numeric step runs in the library's CUDA kernels):
  1. training data: the method itself factorizes many seeded gene-expression
     style matrices (one batched launch); each factor row U_i. becomes a
     target after the gauge is fixed (below), with the 32-quantile sketch of
     row i of R (centred on its median) as input;
  2. the MLP 32 -> 128 -> 128 -> r (BF16 weights, FP32 accumulation) is
     trained with Adam by the library's forward/backward kernels;
  3. at initialisation, U_i. = MLP(sketch_i) + median_i, then V is the
     residuation (-U)^T (x)* R as for Random Acol (Algorithm 3, "initialize U
     and compute V").

Gauge: U (x) V is unchanged by U_.l + c, V_l. - c (any c per component) and by
permuting components.  Targets are made canonical (stmf_mlp_targets): each
component is shifted so that max_t V_lt = 0, and components are ordered by
decreasing sum over rows of U_.l.  Row shifts of R move U_i. with them, hence
the median centring.

Two kinds of target.  "canonical": the gauge-fixed row itself, components in
the global order above.  "sorted": the gauge-fixed row's values sorted in
decreasing order, a target that does not depend on how the components are
numbered; at initialisation the predicted values are handed to the
components in the order of a reference start's row (Random Acol's), so the
start keeps Acol's structure (which component leads in which row) and takes
its magnitudes from the network.
"""
from __future__ import annotations

import numpy as np

from . import api, synth

SK, HID = 32, 128


def init_params(rank, seed=0):
    """He-normal weights, zero biases, in the library's parameter layout."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / SK), size=(SK, HID))
    W2 = rng.normal(0, np.sqrt(2.0 / HID), size=(HID, HID))
    W3 = rng.normal(0, np.sqrt(1.0 / HID), size=(HID, rank))
    return np.concatenate([W1.ravel(), W2.ravel(), W3.ravel(), np.zeros(HID), np.zeros(HID),
                           np.zeros(rank)]).astype(np.float32)


def gene_like(m, n, seed):
    """A gene-expression style matrix (the recipe of the 1000 x 5000 workload at
    another size): planted rank 10, 0.5*log2(1+LogNormal(3,2)) factors,
    N(0, 0.05) noise, 80% given."""
    R, M, _, _ = synth.lognormal_planted(m, n, 10, 0.05, 0.8, seed)
    return R, M


def training_set(count, m, n, rank, sweeps, seed, target="canonical", chunk=64):
    """(X, T) CUDA tensors: sketches and targets ("canonical" or "sorted") from
    `count` factorizations computed by the method (batched launches of up to
    `chunk` problems)."""
    import torch
    rng = np.random.default_rng(seed)
    probs, masks = [], []
    for q in range(count):
        R, M = gene_like(m, n, int(rng.integers(0, 2**31 - 1)))
        probs.append(dict(R=torch.from_numpy(R).cuda(), mask_words=api.pack_mask(M), rank=rank, sweeps=sweeps,
                          seed=int(rng.integers(0, 2**31 - 1))))
    outs = []
    for a in range(0, count, chunk):
        outs += api.factorize_batched(probs[a:a + chunk])[0]
    X, T = [], []
    for pr, (U, V, _) in zip(probs, outs):
        sk, md = api.row_sketch(pr["R"], pr["mask_words"])
        X.append(sk)
        T.append(api.mlp_targets(U, V, md, sorted_rows=(target == "sorted")))
    return torch.cat(X), torch.cat(T)


def train(X, T, rank, epochs=30, batch=256, lr=1e-3, seed=0):
    """Trains a new MLP on (X, T); returns (mlp, per-epoch mean losses)."""
    import torch
    net = api.MLP(rank, init_params(rank, seed))
    g = torch.Generator(device="cpu").manual_seed(seed)
    N = X.shape[0]
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(N, generator=g).cuda()
        tot, nb = 0.0, 0
        for a in range(0, N - batch + 1, batch):
            idx = perm[a:a + batch]
            tot += net.train_step(X[idx].contiguous(), T[idx].contiguous(), lr)
            nb += 1
        hist.append(tot / max(nb, 1))
    return net, hist


def predict_U(net, R, mask_words, U_ref=None):
    """U (m x r, caller frame) = MLP(sketch) + row median.  With U_ref (a net
    trained on "sorted" targets, and a reference start in the same frame),
    row s's predicted values, in decreasing order, go to its components in
    decreasing order of U_ref[s]."""
    Y = net.predict(R, mask_words)
    return Y if U_ref is None else api.assign_by_rank(Y, U_ref.contiguous())

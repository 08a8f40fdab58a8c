"""Seeded synthetic inputs for FastSTMF workloads.

This module only draws data.  It holds none of the factorization method's
arithmetic; the one max-plus sum it forms is the data model the paper uses to
plant a tropical low-rank structure (Section "Synthetic data":
R_lambda = lambda (A (x) B) + (1 - lambda)(A . B)).  Both the CUDA path's tests
and benchmarks and the oracle's tests draw their inputs here.

All draws use NumPy's PCG64 (``numpy.random.default_rng(seed)``) in a fixed
order, so a (recipe, seed) pair always yields the same matrices.  Masks are
boolean (True = given / observed); every row and every column is forced to
keep at least one given entry (the method needs one, see the validation rules
of the library).
"""
from __future__ import annotations

import numpy as np


def _planted_maxplus(Us: np.ndarray, Vs: np.ndarray, chunk: int = 256) -> np.ndarray:
    """max_l (Us[:, l] + Vs[l, :]) in float64, computed in row chunks."""
    m = Us.shape[0]
    out = np.empty((m, Vs.shape[1]), np.float64)
    for a in range(0, m, chunk):
        out[a:a + chunk] = np.max(Us[a:a + chunk, :, None] + Vs[None, :, :], axis=1)
    return out


def _fix_mask(mask: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    m, n = mask.shape
    for s in np.flatnonzero(~mask.any(axis=1)):
        mask[s, rng.integers(n)] = True
    for t in np.flatnonzero(~mask.any(axis=0)):
        mask[rng.integers(m), t] = True
    return mask


def mask_iid(m: int, n: int, observed: float, rng: np.random.Generator) -> np.ndarray:
    """Each entry given independently with probability ``observed`` (the paper
    masks entries uniformly at random, Section "Evaluation")."""
    return _fix_mask(rng.random((m, n)) < observed, rng)


def uniform_planted(m: int, n: int, rank: int, noise_sd: float, observed: float, seed: int):
    """R = U* (x) V* + N(0, noise_sd), U*, V* ~ U[0,1) (paper's tropical synthetic
    data with lambda = 1, plus Gaussian noise; noise_sd is a standard deviation).

    Returns (R float32 m x n, mask bool m x n, U* float32, V* float32)."""
    rng = np.random.default_rng(seed)
    Us = rng.random((m, rank))
    Vs = rng.random((rank, n))
    R = _planted_maxplus(Us, Vs)
    if noise_sd > 0:
        R = R + rng.normal(0.0, noise_sd, size=(m, n))
    mask = mask_iid(m, n, observed, rng)
    return R.astype(np.float32), mask, Us.astype(np.float32), Vs.astype(np.float32)


def lognormal_planted(m: int, n: int, rank: int, noise_sd: float, observed: float, seed: int,
                      mu: float = 3.0, sigma: float = 2.0):
    """Gene-expression-like planted structure: U*_il, V*_lj = 0.5*log2(1+x),
    x ~ LogNormal(mu, sigma); R = U* (x) V* + N(0, noise_sd).  Each entry of R
    is a max of sums of two such halves, so its marginal resembles the
    log2(1 + expression) values of the paper's TCGA matrices (which are not
    available; this recipe stands in for them)."""
    rng = np.random.default_rng(seed)
    Us = 0.5 * np.log2(1.0 + rng.lognormal(mu, sigma, size=(m, rank)))
    Vs = 0.5 * np.log2(1.0 + rng.lognormal(mu, sigma, size=(rank, n)))
    R = _planted_maxplus(Us, Vs)
    if noise_sd > 0:
        R = R + rng.normal(0.0, noise_sd, size=(m, n))
    mask = mask_iid(m, n, observed, rng)
    return R.astype(np.float32), mask, Us.astype(np.float32), Vs.astype(np.float32)


def r_lambda(m: int, n: int, rank: int, lam: float, observed: float, seed: int):
    """The paper's R_lambda = lambda (A (x) B) + (1 - lambda) (A . B), A, B ~ U[0,1)
    (Section "Synthetic data"); lam = 1 is purely tropical, 0 purely linear."""
    rng = np.random.default_rng(seed)
    A = rng.random((m, rank))
    B = rng.random((rank, n))
    R = lam * _planted_maxplus(A, B) + (1.0 - lam) * (A @ B)
    mask = mask_iid(m, n, observed, rng)
    return R.astype(np.float32), mask


def dyadic_planted(m: int, n: int, rank: int, observed: float, seed: int, levels: int = 64):
    """Planted structure on a dyadic grid: U*, V* are multiples of 1/8 in
    [0, levels/8).  Every sum, difference and mean of a few such values is
    exact in fp32, so results are independent of rounding."""
    rng = np.random.default_rng(seed)
    Us = rng.integers(0, levels, size=(m, rank)) / 8.0
    Vs = rng.integers(0, levels, size=(rank, n)) / 8.0
    R = _planted_maxplus(Us, Vs)
    mask = mask_iid(m, n, observed, rng)
    return R.astype(np.float32), mask, Us.astype(np.float32), Vs.astype(np.float32)


def dyadic_noise(m: int, n: int, observed: float, seed: int, levels: int = 256):
    """Unstructured dyadic data: R_ij = integer/8 in [0, levels/8)."""
    rng = np.random.default_rng(seed)
    R = rng.integers(0, levels, size=(m, n)) / 8.0
    mask = mask_iid(m, n, observed, rng)
    return R.astype(np.float32), mask


# ---------------------------------------------------------------------------
# Named workloads (sizes of the paper-shaped benchmark and test cases)

def workload_small(seed: int = 0):
    """200 x 100, U*(200x3) (x) V*(3x100), U[0,1) factors, N(0, 0.01) noise,
    20% of entries masked; rank 3, 10 sweeps (runs as 100 x 200 after the
    wide orientation)."""
    R, M, _, _ = uniform_planted(200, 100, 3, 0.01, 0.8, seed)
    return dict(R=R, mask=M, rank=3, sweeps=10)


def workload_gene(seed: int = 0, m: int = 1000, n: int = 5000):
    """Gene-expression scale: 1000 x 5000, planted rank 10 with
    0.5*log2(1+LogNormal(3,2)) factors, N(0, 0.05) noise, 80% given; rank 10,
    50 sweeps."""
    R, M, _, _ = lognormal_planted(m, n, 10, 0.05, 0.8, seed)
    return dict(R=R, mask=M, rank=10, sweeps=50)


def workload_large(seed: int = 0, m: int = 4000, n: int = 20000):
    """Precision study size: 4000 x 20000 generated like the small case
    (U[0,1) factors, N(0, 0.01) noise), rank 20, 50% given."""
    R, M, _, _ = uniform_planted(m, n, 20, 0.01, 0.5, seed)
    return dict(R=R, mask=M, rank=20, sweeps=50)


def workload_batch(seed: int = 0, count: int = 64):
    """Many independent problems of uneven size: rows ~ U{100..2000},
    cols ~ U{200..8000}, rank ~ U{3..20}, density ~ U[0.2, 0.9], each
    generated like the small case; 10 sweeps each."""
    rng = np.random.default_rng(seed)
    probs = []
    for q in range(count):
        m = int(rng.integers(100, 2001)); n = int(rng.integers(200, 8001))
        r = int(rng.integers(3, 21)); d = float(rng.uniform(0.2, 0.9))
        sub_seed = int(rng.integers(0, 2**31 - 1))
        R, M, _, _ = uniform_planted(m, n, r, 0.01, d, sub_seed)
        probs.append(dict(R=R, mask=M, rank=r, sweeps=10))
    return probs

"""Pins of the oracle's RMSE-A / RMSE-P (Section "Evaluation metrics"; the
held-out protocol of Section "Evaluation") against a hand-computed example
and properties that the definition fixes."""
import os

import numpy as np

from paper_2205_06619_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    blocks, key = {}, None
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line[0].isalpha():
            key = line
            blocks[key] = []
        else:
            blocks[key].append([float(x) for x in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}


def test_rmse_golden(orc):
    g = _golden("rmse_2x3.txt")
    a, p, na, np_ = orc.rmse(g["R"], g["M"].astype(bool), g["U"], g["V"])
    assert (na, np_) == (4, 2)
    assert a == g["rmse_a"][0, 0] and p == g["rmse_p"][0, 0]


def test_rmse_zero_on_an_exact_factorization(orc):
    """Noiseless tropical low-rank data with its planted factors: every
    residual, given or held out, is exactly 0 (dyadic values)."""
    R, M, Us, Vs = synth.dyadic_planted(12, 17, 3, 0.7, seed=3)
    a, p, na, np_ = orc.rmse(R, M, Us.astype(float), Vs.astype(float))
    assert a == 0.0 and p == 0.0 and na == int(M.sum()) and np_ == M.size - int(M.sum())


def test_rmse_against_the_bnorm_and_constant_residuals(orc):
    """sqrt(mean d^2) >= mean |d| (the b-norm over the count), with equality
    exactly when every |d| is the same: R = P + c on the given entries and
    P - c on the held-out ones gives RMSE-A = RMSE-P = c."""
    w = synth.workload_small(seed=2)
    R, M = w["R"][:30, :40].astype(np.float64), w["mask"][:30, :40]
    rng = np.random.default_rng(2)
    U = rng.integers(0, 32, size=(30, 3)) / 8.0
    V = rng.integers(0, 32, size=(3, 40)) / 8.0
    a, p, na, _ = orc.rmse(R, M, U, V)
    assert a >= orc.error(R, M, U, V) / na
    P = np.max(U[:, :, None] + V[None, :, :], axis=1)
    Rc = np.where(M, P + 0.375, P - 0.375)
    a, p, _, _ = orc.rmse(Rc, M, U, V)
    assert a == 0.375 and p == 0.375


def test_rmse_swaps_with_the_mask_and_skips_unknown_truth(orc):
    """The complement mask swaps the training and test sets; a held-out entry
    without a true value (NaN) is left out of RMSE-P; a shift R + c, U + c
    (dyadic c) leaves both unchanged."""
    R, M = synth.dyadic_noise(14, 19, 0.8, seed=5, levels=64)
    rng = np.random.default_rng(5)
    U = rng.integers(0, 64, size=(14, 2)) / 8.0
    V = rng.integers(0, 64, size=(2, 19)) / 8.0
    a, p, na, np_ = orc.rmse(R, M, U, V)
    b, q, nb, nq = orc.rmse(R, ~M, U, V)
    assert (a, p, na, np_) == (q, b, nq, nb)
    Rn = R.copy()
    hid = np.argwhere(~M)
    Rn[tuple(hid[0])] = np.nan
    _, p2, _, np2 = orc.rmse(Rn, M, U, V)
    P = np.max(U[:, :, None] + V[None, :, :], axis=1)
    keep = ~M & ~np.isnan(Rn)
    assert np2 == np_ - 1 and p2 == np.sqrt(np.mean((Rn - P)[keep] ** 2))
    a3, p3, _, _ = orc.rmse(R + 2.5, M, U + 2.5, V)
    assert (a3, p3) == (a, p)
